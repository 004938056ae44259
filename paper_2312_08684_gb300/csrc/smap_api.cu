// smap_api.cu -- the C ABI of libsmap (declared in include/smap.h): handle,
// device buffers, launches, the CUDA graph of the batched run, backtracking,
// the variant autotuner and the debug entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "smap.h"
#include "smap_internal.h"
#include "smap_kernels.cuh"
#include "smap_pf.cuh"

using namespace smap;

namespace smap {

std::atomic<uint64_t> g_launches{0};

namespace {
std::mutex g_smem_attr_mu;
}

cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_smem_attr_mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// Backtracking (Section IV-B): one warp per sequence. i_T = argmax phi_T
// (lowest index on ties), i_t = psi_{t+1}(i_{t+1}); path rows gathered from
// the particle history; J = phi_T(i_T).
// ---------------------------------------------------------------------------
__global__ void backtrack_kernel(int B, int Nmax, int maxT, int d, const int* __restrict__ tcur,
                                 const int* __restrict__ Nseq, const double* __restrict__ phi,
                                 const uint16_t* __restrict__ psi, const float* __restrict__ hist,
                                 const double* __restrict__ x0, const int* __restrict__ status,
                                 int* __restrict__ idxbuf, float* __restrict__ path,
                                 double* __restrict__ J) {
    const int warps = blockDim.x >> 5;
    const int b = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const int T = tcur[b], N = Nseq[b];
    double bv = -INFINITY;
    int bi = 0x7fffffff;
    if (T > 0) {
        for (int i = lane; i < N; i += 32) {
            const double v = phi[(size_t)b * Nmax + i];
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    int* idx = idxbuf + (size_t)b * maxT;
    const bool ok = status[b] == 0 && T <= maxT && N >= 1 && N <= Nmax;
    if (lane == 0 && T > 0 && ok) {
        int it = (bi == 0x7fffffff) ? 0 : bi;
        for (int t = T; t >= 1; --t) {
            idx[t - 1] = it;
            if (t > 1) it = min((int)psi[((size_t)b * maxT + (t - 1)) * Nmax + it], N - 1);
        }
    }
    __syncwarp();
    for (int e = lane; e < (maxT + 1) * d; e += 32) {
        const int t = e / d, c = e - t * d;
        float v;
        if (t == 0) v = (float)x0[(size_t)b * d + c];
        else if (t <= T && ok) v = hist[(((size_t)b * maxT + (t - 1)) * Nmax + idx[t - 1]) * d + c];
        else v = __int_as_float(0x7fc00000);
        path[((size_t)b * (maxT + 1) + t) * d + c] = v;
    }
    if (lane == 0) J[b] = (T > 0 && ok) ? bv : (T == 0 ? 0.0 : __longlong_as_double(0x7ff8000000000000LL));
}

__global__ void philox_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                              uint32_t k1, int n, uint32_t* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t w[4];
    philox4x32_10(c0 + (uint32_t)k, c1, c2, c3, k0, k1, w);
    for (int e = 0; e < 4; ++e) out[(size_t)k * 4 + e] = w[e];
}

#ifdef SMAP_DEBUG
// Debug build: one checked row load from a shared array of `rows` rows filled
// with 1; out = {code, index} of the failed check (or 0), then the loaded value.
__global__ void bounds_probe_kernel(int rows, int index, int* out) {
    extern __shared__ __align__(16) float probe_sm[];
    SMAP_DBG_BEGIN(rows, out);
    for (int e = threadIdx.x; e < 4 * rows; e += blockDim.x) probe_sm[e] = 1.0f;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r[4];
        load_row<4, 4>(probe_sm, index, r);
        out[2] = __float_as_int(r[0]);
    }
}
#endif

// Double-float exp (fn 0), log (1), sqrt (2) of FP64 inputs split into (hi, lo).
__global__ void df_kernel(int fn, const double* in, int n, double* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double v = in[k];
    const float hi = (float)v;
    const df::F a = df::make(hi, (float)(v - (double)hi));
    const df::F r = fn == 0 ? df::exp(a) : fn == 1 ? df::log(a) : df::sqrt(a);
    out[k] = df::to_double(r);
}

template <int D>
__global__ void normals_kernel(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i0, int n, float* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float z[D];
    draw_normals<D>(seed, seq, t, i0 + (uint32_t)k, z);
    for (int c = 0; c < D; ++c) out[(size_t)k * D + c] = z[c];
}

const ModelKernels* kernels_for(int kind) {
    static ModelKernels tab[8];
    static bool init = false;
    if (!init) {
        tab[1] = kernels_ngm1d();
        tab[2] = kernels_range_cv();
        tab[3] = kernels_clutter_cv();
        tab[4] = kernels_planar_arm7();
        tab[5] = kernels_linear_gauss();
        tab[6] = kernels_range_zv();
        tab[7] = kernels_se2_rb();
        init = true;
    }
    if (kind < 1 || kind > 7) return nullptr;
    return &tab[kind];
}

// Fills the device-side model constants; returns false on a bad vector.
bool make_model(int kind, const double* p, int np, ModelParams& mp, std::string& err) {
    memset(&mp, 0, sizeof(mp));
    if (!p || np < 1 || np > kMaxParams) { err = "params: null or bad length"; return false; }
    mp.kind = kind;
    mp.np = np;
    for (int k = 0; k < np; ++k) { mp.p[k] = p[k]; mp.pf[k] = (float)p[k]; }
    const double two_pi = 6.283185307179586;
    switch (kind) {
    case SMAP_MODEL_NGM1D:
        if (np != 8) { err = "NGM1D expects 8 parameters"; return false; }
        mp.d = 1; mp.dy = 1; mp.q[0] = p[5];
        if (!(p[6] > 0)) { err = "NGM1D: r must be > 0"; return false; }
        mp.aux[0] = -0.5 * std::log(two_pi * p[6]); mp.auxf[0] = (float)(1.0 / p[6]);
        break;
    case SMAP_MODEL_RANGE_CV2D: {
        const int nb = np >= 7 ? (int)p[6] : 0;
        if (nb < 1 || nb > 8 || np != 7 + 2 * nb) { err = "RANGE_CV2D: expects 7 + 2 nb parameters, nb 1..8"; return false; }
        if (!(p[5] > 0)) { err = "RANGE_CV2D: r must be > 0"; return false; }
        mp.d = 4; mp.dy = nb;
        for (int c = 0; c < 4; ++c) mp.q[c] = p[1 + c];
        mp.aux[0] = -0.5 * std::log(two_pi * p[5]); mp.auxf[0] = (float)(1.0 / p[5]);
        break;
    }
    case SMAP_MODEL_CLUTTER_CV2D: {
        if (np != 9) { err = "CLUTTER_CV2D expects 9 parameters"; return false; }
        const int M = (int)p[6];
        if (M < 1 || M > 32) { err = "CLUTTER_CV2D: M must be 1..32"; return false; }
        if (!(p[5] > 0) || !(p[7] > 0 && p[7] < 1) || !(p[8] > 0)) { err = "CLUTTER_CV2D: need r > 0, 0 < beta < 1, area > 0"; return false; }
        mp.d = 4; mp.dy = 2 * M;
        for (int c = 0; c < 4; ++c) mp.q[c] = p[1 + c];
        mp.aux[0] = std::log((1.0 - p[7]) / M) - std::log(two_pi * p[5]);
        mp.aux[1] = std::log(p[7] / p[8]);
        mp.auxf[0] = (float)(1.0 / p[5]);
        mp.auxf[1] = (float)(mp.aux[0] * 1.4426950408889634);
        mp.auxf[2] = (float)(mp.aux[1] * 1.4426950408889634);
        break;
    }
    case SMAP_MODEL_PLANAR_ARM: {
        const int nl = np >= 3 ? (int)p[1] : 0;
        if (nl != 7 || np != 3 + 3 * nl) { err = "PLANAR_ARM: the library is compiled for nl = 7 (24 parameters)"; return false; }
        if (!(p[2] > 0)) { err = "PLANAR_ARM: r must be > 0"; return false; }
        mp.d = 2 * nl; mp.dy = 2;
        for (int c = 0; c < 2 * nl; ++c) mp.q[c] = p[3 + c];
        mp.aux[0] = -std::log(two_pi * p[2]); mp.auxf[0] = (float)(1.0 / p[2]);
        break;
    }
    case SMAP_MODEL_RANGE_ZV2D: {
        const int nb = np >= 4 ? (int)p[3] : 0;
        if (nb < 1 || nb > 8 || np != 4 + 2 * nb) { err = "RANGE_ZV2D: expects 4 + 2 nb parameters, nb 1..8"; return false; }
        if (!(p[2] > 0)) { err = "RANGE_ZV2D: r must be > 0"; return false; }
        mp.d = 2; mp.dy = nb;
        mp.q[0] = p[0]; mp.q[1] = p[1];
        mp.aux[0] = -0.5 * std::log(two_pi * p[2]); mp.auxf[0] = (float)(1.0 / p[2]);
        break;
    }
    case SMAP_MODEL_SE2_RB: {
        const int nl = np >= 9 ? (int)p[8] : 0;
        if (nl < 1 || nl > 8 || np != 9 + 2 * nl) { err = "SE2_RB: expects 9 + 2 nl parameters, nl 1..8"; return false; }
        if (!(p[4] > 0) || !(p[5] > 0)) { err = "SE2_RB: rr and rb must be > 0"; return false; }
        if (!std::isfinite(p[0]) || !std::isfinite(p[6]) || !std::isfinite(p[7])) { err = "SE2_RB: dt, v, w must be finite"; return false; }
        mp.d = 3; mp.dy = 2;
        for (int c = 0; c < 3; ++c) mp.q[c] = p[1 + c];
        const double log2e = 1.4426950408889634;
        mp.aux[0] = -std::log((double)nl) - 0.5 * std::log(two_pi * p[4]) - 0.5 * std::log(two_pi * p[5]);
        mp.auxf[0] = (float)(p[6] * p[0]); mp.auxf[1] = (float)(p[7] * p[0]);
        mp.auxf[2] = (float)(-0.5 * log2e / p[4]); mp.auxf[3] = (float)(-0.5 * log2e / p[5]);
        mp.auxf[4] = (float)(1.0 / p[4]); mp.auxf[5] = (float)(1.0 / p[5]);
        break;
    }
    case SMAP_MODEL_LINEAR_GAUSS:
        if (np != 6) { err = "LINEAR_GAUSS expects 6 parameters"; return false; }
        if (!(p[5] > 0)) { err = "LINEAR_GAUSS: r must be > 0"; return false; }
        mp.d = 4; mp.dy = 2;
        for (int c = 0; c < 4; ++c) mp.q[c] = p[1 + c];
        mp.aux[0] = -std::log(two_pi * p[5]); mp.auxf[0] = (float)(1.0 / p[5]);
        break;
    default:
        err = "unknown model";
        return false;
    }
    // model constants the double-float paths read: -1/(2 r) of the Gaussian
    // observation noise (range, zero-velocity range, clutter, linear models)
    if (kind == SMAP_MODEL_RANGE_CV2D || kind == SMAP_MODEL_CLUTTER_CV2D || kind == SMAP_MODEL_LINEAR_GAUSS)
        mp.aux[4] = -0.5 / p[5];
    else if (kind == SMAP_MODEL_RANGE_ZV2D)
        mp.aux[4] = -0.5 / p[2];
    mp.logtrans_c = 0.0;
    for (int c = 0; c < mp.d; ++c) {
        if (!(mp.q[c] > 0) || !std::isfinite(mp.q[c])) { err = "process noise variances must be finite and > 0"; return false; }
        mp.qinv[c] = 1.0 / mp.q[c];
        mp.sqrt_q[c] = std::sqrt(mp.q[c]);
        mp.sqrt_qinv[c] = std::sqrt(mp.qinv[c]);
        mp.qinv_f[c] = (float)mp.qinv[c];
        mp.sqrt_qinv_f[c] = (float)mp.sqrt_qinv[c];
        mp.logtrans_c += -0.5 * std::log(two_pi * mp.q[c]);
    }
    auto lo = [](double v) { return (float)(v - (double)(float)v); };
    for (int k = 0; k < np; ++k) mp.pl[k] = lo(p[k]);
    for (int c = 0; c < mp.d; ++c) mp.qinv_lo[c] = lo(mp.qinv[c]);
    mp.ltc[0] = (float)mp.logtrans_c;
    mp.ltc[1] = lo(mp.logtrans_c);
    for (int k = 0; k < 8; ++k) {
        mp.auxh[k] = (float)mp.aux[k];
        mp.auxl[k] = lo(mp.aux[k]);
    }
    return true;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Block size of variant v for Nmax particles, or 0 if the variant cannot hold them.
int variant_threads(int v, int Nmax) {
    const VariantInfo& vi = kVariants[v];
    int nt = round_up((Nmax + vi.ppt - 1) / vi.ppt * vi.tpp, 32);
    nt = std::max(nt, 32);
    return nt <= vi.maxt ? nt : 0;
}

// Built-in choice of variant for state dimension d, Nmax particles and B
// sequences on an SM count of sms. Fewer sequences than SMs: one block per
// sequence, so the step's latency decides, and splitting each particle's
// sums over 8 (or 4) lanes shortens the serial chains.
int pick_variant(int d, int Nmax, int B, int sms) {
    if (d < 8 && B < sms) {
        if (variant_threads(4, Nmax)) return 4;
        if (variant_threads(5, Nmax)) return 5;
    }
    if (d >= 8) return variant_threads(1, Nmax) ? 1 : 2;
    if (Nmax >= 128 && variant_threads(3, Nmax)) return 3;
    if (variant_threads(0, Nmax)) return 0;
    return variant_threads(1, Nmax) ? 1 : 2;
}

// Block size of recursion variant v for Nmax particles, or 0 if it cannot hold them.
int rec_variant_threads(int v, int Nmax) {
    const RecVariantInfo& vi = kRecVariants[v];
    const int nt = std::max(round_up((Nmax + vi.ppt - 1) / vi.ppt, 32), 32);
    return nt <= vi.maxt ? nt : 0;
}

// Built-in choice of recursion variant: the first that holds Nmax. Two
// particles per thread (each predecessor row loaded once for both) with the
// registers of a 512-thread block measured fastest on the data-association,
// range-only and arm workloads (N = 512, 256, 1024).
int pick_rec_variant(int, int Nmax) {
    for (int v = 0; v < kNumRecVariants; ++v)
        if (rec_variant_threads(v, Nmax)) return v;
    return -1;
}

}  // namespace smap

struct smap_handle {
    smap_config cfg{};
    std::vector<double> params, x0h;
    ModelParams mp{};
    const ModelKernels* K = nullptr;
    int d = 0, dy = 0, B = 0, Nmax = 0, maxT = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    size_t max_smem = 0;
    std::string err;
    bool failed = false;
    int variant = -1;          // -1: heuristic
    // device buffers
    float* hist = nullptr;
    uint16_t* psi = nullptr;
    double* phi = nullptr;
    int* tcur = nullptr;
    int* Nseq = nullptr;
    int* Tend = nullptr;
    int* order = nullptr;
    double* x0 = nullptr;
    double* f64 = nullptr;
    float* bwguess = nullptr;
    int* status = nullptr;     // [B + kStatusExtra]: per-sequence status, then median stats
    int* queue = nullptr;
    float* y = nullptr;        // [B][maxT][dy]
    float* ystep = nullptr;    // [B][dy]
    uint8_t* active = nullptr; // [B]
    int* idxbuf = nullptr;     // [B][maxT]
    unsigned long long* rstats = nullptr;   // [3] recursion counters since the last read
    float* path = nullptr;     // [B][maxT+1][d]
    double* J = nullptr;       // [B]
    // host mirrors
    std::vector<int> tcur_h, Nseq_h, Tend_h;
    // CUDA graph of the batched run
    cudaGraphExec_t graph = nullptr;
    int graph_variant = -2, graph_grid = 0, graph_threads = 0, graph_items = -1;
    int last_threads = 0, last_grid = 0;
    bool configured[kNumVariants * 2 + kNumRecVariants] = {};   // shared-memory carveout set
    bool capturing = false;                    // inside smap_run_batch's stream capture
    // pinned staging of smap_step's inputs; step_done marks when they were consumed
    float* ystep_h = nullptr;
    uint8_t* active_h = nullptr;
    cudaEvent_t step_done = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // batch start, kernel end, batch end
    // learned proposal (attached with smap_set_proposal) and its step buffers
    smap_proposal* prop = nullptr;
    int L_learned = 5;
    float* lfeat = nullptr;    // [B][Nmax][32]
    float* lu = nullptr;       // [B][Nmax][d]
    float* lxinit = nullptr;   // [B][Nmax][d]
    cudaStream_t side = nullptr;   // second chain of the learned launches
    float* dbg_init = nullptr;     // debug: every step's learned initial particles [B][maxT][Nmax][d]
    // PF-MAP-Seq state (allocated by the first smap_pf_run_batch)
    double* pf_x64 = nullptr;  // [B][Nmax][d]
    double* pf_lw = nullptr;   // [B][Nmax]
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace {

smap_status fail(smap_handle* h, smap_status s, const std::string& msg) {
    if (h) {
        h->err = msg;
        if (s == SMAP_E_CUDA) h->failed = true;
    }
    return s;
}

smap_status cuda_fail(smap_handle* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, SMAP_E_CUDA, m);
}

#define SMAP_CUDA(h, call)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

int heuristic_variant(const smap_handle* h) { return pick_variant(h->d, h->Nmax, h->B, h->num_sms); }

smap_status configure_kernel(smap_handle* h, const void* fn, size_t smem) {
    if (smem > h->max_smem)
        return fail(h, SMAP_E_UNSUPPORTED, "shared memory need exceeds the device limit for this N and d");
    // inside a stream capture the caller raised the limit just before it began
    // (smap_run_batch), and no call of this library ever lowers it
    if (h->capturing) return SMAP_OK;
    SMAP_CUDA(h, ensure_dynamic_smem(fn, smem));
    for (int k = 0; k < kNumVariants || k < kNumRecVariants; ++k) {
        bool* flag = k < kNumVariants && fn == h->K->seq[k]      ? &h->configured[k]
                     : k < kNumVariants && fn == h->K->dbg[k]    ? &h->configured[kNumVariants + k]
                     : k < kNumRecVariants && fn == h->K->rec[k] ? &h->configured[2 * kNumVariants + k]
                                                                 : nullptr;
        if (!flag) continue;
        if (!*flag) {
            // the whole unified L1 as shared memory: as many resident sequences as registers allow
            SMAP_CUDA(h, cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared));
            *flag = true;
        }
        break;
    }
    return SMAP_OK;
}

// Options of a one-step launch (mode 1) beyond the handle's configuration.
struct StepOpts {
    const float* xinit = nullptr;   // initial particles of the step [B][Nmax][d]
    int y_full = 0;                 // y is [B][maxT][dy]
    int skip_done = 0;              // skip sequences with tcur >= Tend
    int L = -1;                     // SVGD iterations (-1: the handle's L)
    const uint8_t* active = nullptr;  // per-sequence step mask [B] (smap_step)
    int seq_base = 0;               // items are sequences seq_base .. seq_base + items - 1
    int queue_slot = 0;             // work-queue counter (one per concurrent launch)
    double* f64 = nullptr;          // FP64 scratch of this launch (default: the handle's)
    cudaStream_t stream = nullptr;  // launch stream (default: the handle's)
};

// Launches the sequence kernel of variant v over `items` work items.
smap_status launch_seq(smap_handle* h, int v, int items, int mode, const float* y, int viterbi_only,
                       const int* order, int* grid_out = nullptr, int* threads_out = nullptr,
                       const StepOpts& opts = StepOpts()) {
    const int nt = variant_threads(v, h->Nmax);
    if (!nt) return fail(h, SMAP_E_UNSUPPORTED, "kernel variant cannot hold N particles");
    const void* fn = h->K->seq[v];
    const size_t smem = smem_layout(h->Nmax, h->K->DP).total;
    smap_status st = configure_kernel(h, fn, smem);
    if (st) return st;
    int occ = 0;
    SMAP_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem));
    if (occ < 1) return fail(h, SMAP_E_UNSUPPORTED, "kernel variant does not fit on an SM");
    const int grid = std::max(1, std::min(items, occ * h->num_sms));
    SeqArgs a;
    memset(&a, 0, sizeof(a));
    a.mp = h->mp;
    a.B = items;
    a.Nmax = h->Nmax;
    a.maxT = h->maxT;
    a.L = h->cfg.L;
    a.bw_rule = h->cfg.bw_rule;
    a.prior = h->cfg.prior;
    a.kernel = h->cfg.kernel;
    a.mode = mode;
    a.eps = (float)h->cfg.step;
    a.bw_value = (float)h->cfg.bw_value;
    a.seed = h->cfg.seed;
    a.y = y;
    a.x0 = h->x0;
    a.hist = h->hist;
    a.psi = h->psi;
    a.phi = h->phi;
    a.tcur = h->tcur;
    a.Nseq = h->Nseq;
    a.Tend = h->Tend;
    a.active = (mode == 1) ? opts.active : nullptr;
    a.order = order;
    a.f64 = opts.f64 ? opts.f64 : h->f64;
    a.bwguess = h->bwguess;
    a.status = h->status;
    a.stats = h->status + h->B;
    a.queue = h->queue + opts.queue_slot;
    a.viterbi_only = viterbi_only;
    a.xinit = opts.xinit;
    a.y_full = opts.y_full;
    a.skip_done = opts.skip_done;
    a.seq_base = opts.seq_base;
    a.Btot = h->B;
    a.rstats = h->rstats;
    if (opts.L >= 0) a.L = opts.L;
    void* args[] = {&a};
    cudaStream_t ls = opts.stream ? opts.stream : h->stream;
    SMAP_CUDA(h, cudaMemsetAsync(a.queue, 0, sizeof(int), ls));
    SMAP_CUDA(h, cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, ls));
    SMAP_CUDA(h, cudaGetLastError());
    g_launches.fetch_add(1);
    h->last_threads = nt;
    h->last_grid = grid;
    if (grid_out) *grid_out = grid;
    if (threads_out) *threads_out = nt;
    return SMAP_OK;
}

// The recursion alone on the particle sets in h->hist (every sequence from
// t = 1; the state reset beforehand): rec_kernel over the work queue.
smap_status launch_rec(smap_handle* h) {
    const int v = pick_rec_variant(h->d, h->Nmax);
    const int nt = v >= 0 ? rec_variant_threads(v, h->Nmax) : 0;
    if (!nt) return fail(h, SMAP_E_UNSUPPORTED, "no recursion kernel variant holds N particles");
    const void* fn = h->K->rec[v];
    const size_t smem = rec_smem_layout(h->Nmax, h->K->DP).total;
    smap_status st = configure_kernel(h, fn, smem);
    if (st) return st;
    int occ = 0;
    SMAP_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem));
    if (occ < 1) return fail(h, SMAP_E_UNSUPPORTED, "recursion kernel does not fit on an SM");
    // the FP64 scratch holds one [Nmax][d] slice per sequence: grid <= B
    const int grid = std::max(1, std::min(h->B, occ * h->num_sms));
    SeqArgs a;
    memset(&a, 0, sizeof(a));
    a.mp = h->mp;
    a.B = h->B;
    a.Nmax = h->Nmax;
    a.maxT = h->maxT;
    a.seed = h->cfg.seed;
    a.y = h->y;
    a.x0 = h->x0;
    a.hist = h->hist;
    a.psi = h->psi;
    a.phi = h->phi;
    a.tcur = h->tcur;
    a.Nseq = h->Nseq;
    a.Tend = h->Tend;
    a.order = h->order;
    a.f64 = h->f64;
    a.bwguess = h->bwguess;
    a.status = h->status;
    a.stats = h->status + h->B;
    a.queue = h->queue;
    a.viterbi_only = 1;
    a.y_full = 1;
    a.Btot = h->B;
    a.rstats = h->rstats;
    void* args[] = {&a};
    SMAP_CUDA(h, cudaMemsetAsync(a.queue, 0, sizeof(int), h->stream));
    SMAP_CUDA(h, cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, h->stream));
    SMAP_CUDA(h, cudaGetLastError());
    g_launches.fetch_add(1);
    h->last_threads = nt;
    h->last_grid = grid;
    return SMAP_OK;
}

smap_status launch_backtrack(smap_handle* h) {
    const int warps = 4;
    const int grid = (h->B + warps - 1) / warps;
    backtrack_kernel<<<grid, 32 * warps, 0, h->stream>>>(h->B, h->Nmax, h->maxT, h->d, h->tcur, h->Nseq,
                                                         h->phi, h->psi, h->hist, h->x0, h->status,
                                                         h->idxbuf, h->path, h->J);
    SMAP_CUDA(h, cudaGetLastError());
    g_launches.fetch_add(1);
    return SMAP_OK;
}

smap_status check_usable(smap_handle* h) {
    if (!h) return SMAP_E_INVAL;
    if (h->failed) return SMAP_E_STATE;
    return SMAP_OK;
}

cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// Reads the per-sequence status words; returns the first failure or OK.
smap_status collect_status(smap_handle* h) {
    std::vector<int> st(h->B + kStatusExtra);
    SMAP_CUDA(h, cudaMemcpyAsync(st.data(), h->status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost, h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st[h->B + 4] != 0)
        return fail(h, SMAP_E_TIMEOUT, "learned proposal: a bounded wait of the tensor-core network kernel ran out");
    if (st[h->B + kDbgWord] != 0)
        return fail(h, SMAP_E_INVAL, "debug build: bounds check " + std::to_string(st[h->B + kDbgWord]) +
                                         " failed at index " + std::to_string(st[h->B + kDbgWord + 1]));
    for (int b = 0; b < h->B; ++b) {
        if (st[b] == SMAP_E_NONFINITE)
            return fail(h, SMAP_E_NONFINITE, "sequence " + std::to_string(b) + ": particles or scores became non-finite");
        if (st[b] != 0)
            return fail(h, SMAP_E_INVAL, "sequence " + std::to_string(b) + ": rejected by the kernel (length or particle count)");
    }
    return SMAP_OK;
}

smap_status upload_counts(smap_handle* h, const int* T_per_seq, const int* N_per_seq) {
    for (int b = 0; b < h->B; ++b) {
        const int T = T_per_seq ? T_per_seq[b] : h->maxT;
        const int N = N_per_seq ? N_per_seq[b] : h->Nmax;
        if (T < 1 || T > h->maxT) return fail(h, SMAP_E_INVAL, "T_per_seq out of 1..max_T");
        if (N < 1 || N > h->Nmax) return fail(h, SMAP_E_INVAL, "N_per_seq out of 1..N");
        h->Tend_h[b] = T;
        h->Nseq_h[b] = N;
    }
    // longest work first: T N^2 decreasing
    std::vector<int> ord(h->B);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        return (double)h->Tend_h[a] * h->Nseq_h[a] * h->Nseq_h[a] > (double)h->Tend_h[b] * h->Nseq_h[b] * h->Nseq_h[b];
    });
    SMAP_CUDA(h, cudaMemcpyAsync(h->Tend, h->Tend_h.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream));
    SMAP_CUDA(h, cudaMemcpyAsync(h->Nseq, h->Nseq_h.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream));
    SMAP_CUDA(h, cudaMemcpyAsync(h->order, ord.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));   // host vectors above are temporaries
    return SMAP_OK;
}

smap_status reset_device_state(smap_handle* h) {
    SMAP_CUDA(h, cudaMemsetAsync(h->tcur, 0, sizeof(int) * h->B, h->stream));
    SMAP_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int) * (h->B + kStatusExtra), h->stream));
    SMAP_CUDA(h, cudaMemsetAsync(h->bwguess, 0, sizeof(float) * h->B, h->stream));
    return SMAP_OK;
}

smap_status copy_outputs(smap_handle* h, float* path, double* J, int on_device) {
    if (path)
        SMAP_CUDA(h, cudaMemcpyAsync(path, h->path, sizeof(float) * (size_t)h->B * (h->maxT + 1) * h->d,
                                     kind_out(on_device), h->stream));
    if (J) SMAP_CUDA(h, cudaMemcpyAsync(J, h->J, sizeof(double) * h->B, kind_out(on_device), h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

// The device work of one batched run: state reset, the persistent kernel
// over all sequences, backtracking. Recorded once into a CUDA graph.
smap_status batch_device_work(smap_handle* h, int v) {
    SMAP_CUDA(h, cudaEventRecordWithFlags(h->ev[0], h->stream, cudaEventRecordExternal));
    smap_status st = reset_device_state(h);
    if (st) return st;
    if (h->prop) {
        // learned initialisation: per step, rows (u, features) -> MLP -> one
        // step of L_learned SVGD iterations for every unfinished sequence. The
        // batch is split into two independent chains on two streams, so one
        // half's network and step tail overlap the other half's step kernel.
        const int nch = h->B >= 2 ? 2 : 1;
        SMAP_CUDA(h, cudaEventRecord(h->fork_ev, h->stream));
        SMAP_CUDA(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
        for (int c = 0; c < nch; ++c) {
            const int b0 = (int)((long)h->B * c / nch), b1 = (int)((long)h->B * (c + 1) / nch);
            cudaStream_t cs = c == 0 ? h->stream : h->side;
            const size_t r0 = (size_t)b0 * h->Nmax;
            ProposalRowsArgs ra;
            memset(&ra, 0, sizeof(ra));
            ra.mp = h->mp;
            ra.B = b1 - b0; ra.b_base = b0; ra.Nmax = h->Nmax; ra.maxT = h->maxT; ra.capture = 0;
            ra.seed = h->cfg.seed;
            ra.x0 = h->x0; ra.hist = h->hist; ra.y = h->y;
            ra.tcur = h->tcur; ra.Tend = h->Tend; ra.Nseq = h->Nseq;
            ra.feat = h->lfeat + r0 * 32; ra.u = h->lu + r0 * h->d;
            ra.err = h->status + h->B + 4;
            StepOpts so;
            so.xinit = h->lxinit;
            so.y_full = 1;
            so.skip_done = 1;
            so.L = h->L_learned;
            so.seq_base = b0;
            so.queue_slot = c;
            so.f64 = h->f64 + r0 * h->d;
            so.stream = cs;
            for (int t = 1; t <= h->maxT; ++t) {
                st = proposal_launch_init(h->prop, ra, h->lxinit + r0 * h->d, cs);
                if (st) return fail(h, st, smap_proposal_last_error(h->prop));
                if (h->dbg_init) {
                    const size_t row = sizeof(float) * (size_t)h->Nmax * h->d;
                    SMAP_CUDA(h, cudaMemcpy2DAsync(h->dbg_init + ((size_t)b0 * h->maxT + (t - 1)) * h->Nmax * h->d,
                                                   row * h->maxT, h->lxinit + r0 * h->d, row, row, b1 - b0,
                                                   cudaMemcpyDeviceToDevice, cs));
                }
                st = launch_seq(h, v, b1 - b0, 1, h->y, 0, nullptr, nullptr, nullptr, so);
                if (st) return st;
            }
        }
        SMAP_CUDA(h, cudaEventRecord(h->join_ev, h->side));
        SMAP_CUDA(h, cudaStreamWaitEvent(h->stream, h->join_ev, 0));
    } else {
        st = launch_seq(h, v, h->B, 0, h->y, 0, h->order);
        if (st) return st;
    }
    SMAP_CUDA(h, cudaEventRecordWithFlags(h->ev[1], h->stream, cudaEventRecordExternal));
    st = launch_backtrack(h);
    if (st) return st;
    SMAP_CUDA(h, cudaEventRecordWithFlags(h->ev[2], h->stream, cudaEventRecordExternal));
    return SMAP_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint of the online state: a header that identifies the handle's
// configuration, then x0 [B][d] FP64, tcur / Nseq / Tend / status [B] int32,
// the median guesses [B] FP32, the scores phi [B][N] FP64, and for every
// sequence b its first tcur[b] particle sets [tcur_b][N][d] FP32 and
// backpointer rows [tcur_b][N] uint16.
// ---------------------------------------------------------------------------
constexpr uint64_t kStateMagic = 0x31765453'50414D53ull;   // "SMAPSTv1"

struct StateHeader {
    uint64_t magic, bytes, params_hash, seed;
    int32_t model, d, dy, B, Nmax, maxT, L, bw_rule, prior, kernel, n_params, reserved;
    double step, bw_value;
};

uint64_t params_hash(const std::vector<double>& p) {
    uint64_t x = 1469598103934665603ull;   // FNV-1a over the bytes of the vector
    const unsigned char* c = reinterpret_cast<const unsigned char*>(p.data());
    for (size_t k = 0; k < p.size() * sizeof(double); ++k) x = (x ^ c[k]) * 1099511628211ull;
    return x;
}

StateHeader state_header(const smap_handle* h) {
    StateHeader H;
    memset(&H, 0, sizeof(H));
    H.magic = kStateMagic;
    H.params_hash = params_hash(h->params);
    H.seed = h->cfg.seed;
    H.model = h->cfg.model; H.d = h->d; H.dy = h->dy; H.B = h->B; H.Nmax = h->Nmax; H.maxT = h->maxT;
    H.L = h->cfg.L; H.bw_rule = h->cfg.bw_rule; H.prior = h->cfg.prior; H.kernel = h->cfg.kernel;
    H.n_params = (int32_t)h->params.size();
    H.step = h->cfg.step; H.bw_value = h->cfg.bw_value;
    return H;
}

size_t state_bytes(const smap_handle* h, const std::vector<int>& tcur) {
    size_t n = sizeof(StateHeader) + sizeof(double) * (size_t)h->B * h->d + sizeof(int32_t) * 4 * (size_t)h->B +
               sizeof(float) * (size_t)h->B + sizeof(double) * (size_t)h->B * h->Nmax;
    for (int b = 0; b < h->B; ++b)
        n += (size_t)tcur[b] * h->Nmax * (sizeof(float) * h->d + sizeof(uint16_t));
    return n;
}

}  // namespace

extern "C" {

smap_status smap_state_size(const smap_handle* h, size_t* bytes) {
    if (!h || !bytes) return SMAP_E_INVAL;
    *bytes = state_bytes(h, h->tcur_h);
    return SMAP_OK;
}

smap_status smap_save(smap_handle* h, void* buf, size_t bytes) {
    NvtxRange nvtx_("smap_save");
    smap_status st = check_usable(h);
    if (st) return st;
    const size_t need = state_bytes(h, h->tcur_h);
    if (!buf || bytes < need) return fail(h, SMAP_E_INVAL, "smap_save: buffer smaller than smap_state_size");
    unsigned char* o = static_cast<unsigned char*>(buf);
    StateHeader H = state_header(h);
    H.bytes = need;
    memcpy(o, &H, sizeof(H));
    o += sizeof(H);
    const size_t B = h->B, N = h->Nmax, d = h->d, T = h->maxT;
    auto d2h = [&](const void* src, size_t n) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(o, src, n, cudaMemcpyDeviceToHost, h->stream);
        o += n;
        return e;
    };
    SMAP_CUDA(h, d2h(h->x0, sizeof(double) * B * d));
    SMAP_CUDA(h, d2h(h->tcur, sizeof(int) * B));
    SMAP_CUDA(h, d2h(h->Nseq, sizeof(int) * B));
    SMAP_CUDA(h, d2h(h->Tend, sizeof(int) * B));
    SMAP_CUDA(h, d2h(h->status, sizeof(int) * B));
    SMAP_CUDA(h, d2h(h->bwguess, sizeof(float) * B));
    SMAP_CUDA(h, d2h(h->phi, sizeof(double) * B * N));
    for (size_t b = 0; b < B; ++b)
        if (h->tcur_h[b] > 0) SMAP_CUDA(h, d2h(h->hist + b * T * N * d, sizeof(float) * h->tcur_h[b] * N * d));
    for (size_t b = 0; b < B; ++b)
        if (h->tcur_h[b] > 0) SMAP_CUDA(h, d2h(h->psi + b * T * N, sizeof(uint16_t) * h->tcur_h[b] * N));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_load(smap_handle* h, const void* buf, size_t bytes) {
    NvtxRange nvtx_("smap_load");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!buf || bytes < sizeof(StateHeader)) return fail(h, SMAP_E_INVAL, "smap_load: no state");
    StateHeader H;
    memcpy(&H, buf, sizeof(H));
    StateHeader mine = state_header(h);
    mine.bytes = H.bytes;
    if (memcmp(&H, &mine, sizeof(H)) != 0)
        return fail(h, SMAP_E_INVAL, "smap_load: the state was saved by a handle of another configuration");
    const size_t B = h->B, N = h->Nmax, d = h->d, T = h->maxT;
    const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(H);
    const size_t fixed = sizeof(H) + sizeof(double) * B * d + sizeof(int32_t) * 4 * B + sizeof(float) * B +
                         sizeof(double) * B * N;
    if (bytes < fixed || H.bytes > bytes) return fail(h, SMAP_E_INVAL, "smap_load: truncated state");
    std::vector<int> tc(B), ns(B), te(B);
    memcpy(tc.data(), in + sizeof(double) * B * d, sizeof(int) * B);
    memcpy(ns.data(), in + sizeof(double) * B * d + sizeof(int) * B, sizeof(int) * B);
    memcpy(te.data(), in + sizeof(double) * B * d + 2 * sizeof(int) * B, sizeof(int) * B);
    for (size_t b = 0; b < B; ++b)
        if (tc[b] < 0 || tc[b] > (int)T || ns[b] < 1 || ns[b] > (int)N || te[b] < 1 || te[b] > (int)T)
            return fail(h, SMAP_E_INVAL, "smap_load: step counts or particle counts out of range");
    if (H.bytes != state_bytes(h, tc)) return fail(h, SMAP_E_INVAL, "smap_load: size does not match its contents");
    std::vector<double> x0(B * d);
    memcpy(x0.data(), in, sizeof(double) * B * d);
    for (double v : x0)
        if (!std::isfinite(v)) return fail(h, SMAP_E_NONFINITE, "smap_load: x0 not finite");
    auto h2d = [&](void* dst, size_t n) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(dst, in, n, cudaMemcpyHostToDevice, h->stream);
        in += n;
        return e;
    };
    SMAP_CUDA(h, h2d(h->x0, sizeof(double) * B * d));
    SMAP_CUDA(h, h2d(h->tcur, sizeof(int) * B));
    SMAP_CUDA(h, h2d(h->Nseq, sizeof(int) * B));
    SMAP_CUDA(h, h2d(h->Tend, sizeof(int) * B));
    SMAP_CUDA(h, h2d(h->status, sizeof(int) * B));
    SMAP_CUDA(h, h2d(h->bwguess, sizeof(float) * B));
    SMAP_CUDA(h, h2d(h->phi, sizeof(double) * B * N));
    for (size_t b = 0; b < B; ++b)
        if (tc[b] > 0) SMAP_CUDA(h, h2d(h->hist + b * T * N * d, sizeof(float) * tc[b] * N * d));
    for (size_t b = 0; b < B; ++b)
        if (tc[b] > 0) SMAP_CUDA(h, h2d(h->psi + b * T * N, sizeof(uint16_t) * tc[b] * N));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    h->x0h = x0;
    h->cfg.x0 = h->x0h.data();
    h->tcur_h = tc;
    h->Nseq_h = ns;
    h->Tend_h = te;
    return SMAP_OK;
}

const char* smap_status_string(smap_status s) {
    switch (s) {
    case SMAP_OK: return "ok";
    case SMAP_E_INVAL: return "invalid argument";
    case SMAP_E_NOMEM: return "out of memory";
    case SMAP_E_CUDA: return "CUDA error";
    case SMAP_E_STATE: return "handle in a failed state or call out of order";
    case SMAP_E_TIMEOUT: return "bounded wait ran out";
    case SMAP_E_NONFINITE: return "non-finite particles or observations";
    case SMAP_E_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* smap_last_error(const smap_handle* h) { return h ? h->err.c_str() : "null handle"; }

uint64_t smap_kernel_launches(void) { return g_launches.load(); }

smap_status smap_set_proposal(smap_handle* h, smap_proposal* p, int L_learned) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (p && (proposal_kind(p) != h->mp.kind || proposal_d(p) != h->d))
        return fail(h, SMAP_E_INVAL, "proposal was made for another model");
    if (L_learned < 0) return fail(h, SMAP_E_INVAL, "L_learned < 0");
    if (p && !h->lfeat) {
        const size_t rows = (size_t)h->B * h->Nmax;
        if (cudaMalloc(&h->lfeat, sizeof(float) * rows * 32) != cudaSuccess ||
            cudaMalloc(&h->lu, sizeof(float) * rows * h->d) != cudaSuccess ||
            cudaMalloc(&h->lxinit, sizeof(float) * rows * h->d) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SMAP_E_NOMEM, "learned-step buffers");
        }
        SMAP_CUDA(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        SMAP_CUDA(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        SMAP_CUDA(h, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    }
    h->prop = p;
    h->L_learned = L_learned;
    if (h->graph) {   // the device work changes: record a new graph
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SMAP_OK;
}

smap_status smap_debug_record_learned_init(smap_handle* h, float* xinit_all) {
    smap_status st = check_usable(h);
    if (st) return st;
    h->dbg_init = xinit_all;
    if (h->graph) {   // the device work changes: record a new graph
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SMAP_OK;
}

smap_status smap_proposal_capture(smap_proposal* p, smap_handle* h, float* feat, float* targ, long max_rows,
                                  long* rows) {
    NvtxRange nvtx_("smap_proposal_capture");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!p || !feat || !targ) return fail(h, SMAP_E_INVAL, "null argument");
    if (proposal_kind(p) != h->mp.kind) return fail(h, SMAP_E_INVAL, "proposal was made for another model");
    std::vector<long long> base((size_t)h->B * h->maxT, 0);
    long long total = 0;
    for (int b = 0; b < h->B; ++b)
        for (int t = 1; t <= h->tcur_h[b]; ++t) {
            base[(size_t)b * h->maxT + (t - 1)] = total;
            total += h->Nseq_h[b];
        }
    if (rows) *rows = (long)total;
    if (total > max_rows) return fail(h, SMAP_E_INVAL, "capture needs " + std::to_string(total) + " rows");
    long long* dbase = nullptr;
    SMAP_CUDA(h, cudaMalloc(&dbase, sizeof(long long) * base.size()));
    cudaError_t e = cudaMemcpyAsync(dbase, base.data(), sizeof(long long) * base.size(), cudaMemcpyHostToDevice,
                                    h->stream);
    ProposalRowsArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.mp = h->mp;
    ra.B = h->B; ra.Nmax = h->Nmax; ra.maxT = h->maxT; ra.capture = 1;
    ra.seed = h->cfg.seed;
    ra.x0 = h->x0; ra.hist = h->hist; ra.y = h->y;
    ra.tcur = h->tcur; ra.Tend = h->tcur; ra.Nseq = h->Nseq;
    ra.row_base = dbase;
    ra.feat = feat; ra.targ = targ;
    if (e == cudaSuccess) st = proposal_launch_capture(p, ra, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dbase);
    if (e != cudaSuccess) return cuda_fail(h, e, "smap_proposal_capture");
    return st;
}

smap_status smap_debug_median_stats(smap_handle* h, int* counts) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!counts) return fail(h, SMAP_E_INVAL, "null output");
    SMAP_CUDA(h, cudaMemcpyAsync(counts, h->status + h->B, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_debug_recursion_stats(smap_handle* h, unsigned long long* counts) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!counts) return fail(h, SMAP_E_INVAL, "null output");
    SMAP_CUDA(h, cudaMemcpyAsync(counts, h->rstats, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost,
                                 h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    counts[2] += counts[0] - counts[1];   // one exact score per particle proven unique, plus the near-ties' candidates
    SMAP_CUDA(h, cudaMemsetAsync(h->rstats, 0, sizeof(unsigned long long) * 4, h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_last_kernel_ms(smap_handle* h, float* seq_ms, float* batch_ms) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!h->graph) return fail(h, SMAP_E_STATE, "no batched run yet");
    SMAP_CUDA(h, cudaEventSynchronize(h->ev[2]));
    if (seq_ms) SMAP_CUDA(h, cudaEventElapsedTime(seq_ms, h->ev[0], h->ev[1]));
    if (batch_ms) SMAP_CUDA(h, cudaEventElapsedTime(batch_ms, h->ev[0], h->ev[2]));
    return SMAP_OK;
}

int smap_num_variants(void) { return kNumVariants; }

smap_status smap_variant_info(int v, int* ppt, int* maxt, int* tpp) {
    if (v < 0 || v >= kNumVariants) return SMAP_E_INVAL;
    if (ppt) *ppt = kVariants[v].ppt;
    if (maxt) *maxt = kVariants[v].maxt;
    if (tpp) *tpp = kVariants[v].tpp;
    return SMAP_OK;
}

void smap_destroy(smap_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->step_done) cudaEventDestroy(h->step_done);
    for (void* q : {(void*)h->lfeat, (void*)h->lu, (void*)h->lxinit, (void*)h->pf_x64, (void*)h->pf_lw})
        if (q) cudaFree(q);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    for (cudaEvent_t ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    if (h->ystep_h) cudaFreeHost(h->ystep_h);
    if (h->active_h) cudaFreeHost(h->active_h);
    void* bufs[] = {h->hist, h->psi, h->phi, h->tcur, h->Nseq, h->Tend, h->order, h->x0, h->f64,
                    h->bwguess, h->status, h->queue, h->y, h->ystep, h->active, h->idxbuf, h->path, h->J,
                    h->rstats};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

smap_status smap_create(const smap_config* cfg, smap_handle** out) {
    NvtxRange nvtx_("smap_create");
    if (!out) return SMAP_E_INVAL;
    *out = nullptr;
    if (!cfg) return SMAP_E_INVAL;
    smap_handle* h = new smap_handle();
    h->cfg = *cfg;
    auto bail = [&](smap_status s, const std::string& msg) {
        std::fprintf(stderr, "smap_create: %s\n", msg.c_str());
        smap_destroy(h);
        return s;
    };
    h->K = kernels_for(cfg->model);
    if (!h->K) return bail(SMAP_E_INVAL, "unknown model");
    std::string err;
    if (!make_model(cfg->model, cfg->params, cfg->n_params, h->mp, err)) return bail(SMAP_E_INVAL, err);
    h->params.assign(cfg->params, cfg->params + cfg->n_params);
    h->cfg.params = h->params.data();
    h->d = h->mp.d;
    h->dy = h->mp.dy;
    if (h->d != h->K->D) return bail(SMAP_E_INVAL, "state dimension does not match the compiled model");
    if (cfg->N < 1 || cfg->N > kMaxN) return bail(SMAP_E_INVAL, "N out of 1..4096");
    if (cfg->L < 0) return bail(SMAP_E_INVAL, "L < 0");
    if (cfg->batch < 1) return bail(SMAP_E_INVAL, "batch < 1");
    if (cfg->max_T < 1) return bail(SMAP_E_INVAL, "max_T < 1");
    if (!(std::isfinite(cfg->step))) return bail(SMAP_E_INVAL, "step not finite");
    if (cfg->bw_rule < 0 || cfg->bw_rule > 2) return bail(SMAP_E_INVAL, "bw_rule");
    if (!(cfg->bw_value > 0) || !std::isfinite(cfg->bw_value)) return bail(SMAP_E_INVAL, "bw_value must be > 0");
    if (cfg->prior < 0 || cfg->prior > 2) return bail(SMAP_E_INVAL, "prior");
    if (cfg->kernel < 0 || cfg->kernel > 2) return bail(SMAP_E_INVAL, "kernel");
    if (!cfg->x0) return bail(SMAP_E_INVAL, "x0 is null");
    h->B = cfg->batch;
    h->Nmax = cfg->N;
    h->maxT = cfg->max_T;
    h->x0h.assign(cfg->x0, cfg->x0 + (size_t)h->B * h->d);
    for (double v : h->x0h)
        if (!std::isfinite(v)) return bail(SMAP_E_NONFINITE, "x0 not finite");
    h->cfg.x0 = h->x0h.data();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, h->device);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    h->num_sms = prop.multiProcessorCount;
    h->max_smem = prop.sharedMemPerBlockOptin;
    if (smem_layout(h->Nmax, h->K->DP).total > h->max_smem)
        return bail(SMAP_E_UNSUPPORTED, "N too large for shared memory at this state dimension");
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        e = cudaStreamCreate(&h->stream);
        if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
        h->own_stream = true;
    }
    const size_t B = h->B, N = h->Nmax, T = h->maxT, d = h->d, dy = h->dy;
    struct A { void** p; size_t bytes; } allocs[] = {
        {(void**)&h->hist, sizeof(float) * B * T * N * d},
        {(void**)&h->psi, sizeof(uint16_t) * B * T * N},
        {(void**)&h->phi, sizeof(double) * B * N},
        {(void**)&h->tcur, sizeof(int) * B},
        {(void**)&h->Nseq, sizeof(int) * B},
        {(void**)&h->Tend, sizeof(int) * B},
        {(void**)&h->order, sizeof(int) * B},
        {(void**)&h->x0, sizeof(double) * B * d},
        {(void**)&h->f64, sizeof(double) * B * N * d},
        {(void**)&h->bwguess, sizeof(float) * B},
        {(void**)&h->status, sizeof(int) * (B + kStatusExtra)},
        {(void**)&h->queue, sizeof(int) * 4},
        {(void**)&h->y, sizeof(float) * B * T * dy},
        {(void**)&h->ystep, sizeof(float) * B * dy},
        {(void**)&h->active, B},
        {(void**)&h->idxbuf, sizeof(int) * B * T},
        {(void**)&h->path, sizeof(float) * B * (T + 1) * d},
        {(void**)&h->J, sizeof(double) * B},
        {(void**)&h->rstats, sizeof(unsigned long long) * 4},
    };
    // fault injection for tests: SMAP_FAIL_ALLOC=k makes the k-th device
    // allocation of this call fail as if the device were out of memory
    const char* inj = std::getenv("SMAP_FAIL_ALLOC");
    const int fail_at = inj ? std::atoi(inj) : 0;
    int n_alloc = 0;
    for (auto& al : allocs) {
        if (++n_alloc == fail_at)
            return bail(SMAP_E_NOMEM, "cudaMalloc: injected failure (SMAP_FAIL_ALLOC)");
        e = cudaMalloc(al.p, al.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(SMAP_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    e = cudaMemset(h->rstats, 0, sizeof(unsigned long long) * 4);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    if (cudaMallocHost(&h->ystep_h, sizeof(float) * B * dy) != cudaSuccess ||
        cudaMallocHost(&h->active_h, B) != cudaSuccess) {
        cudaGetLastError();
        return bail(SMAP_E_NOMEM, "cudaMallocHost failed");
    }
    e = cudaEventCreateWithFlags(&h->step_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    for (cudaEvent_t& ev : h->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    }
    h->tcur_h.assign(B, 0);
    h->Nseq_h.assign(B, (int)N);
    h->Tend_h.assign(B, (int)T);
    e = cudaMemcpy(h->x0, h->x0h.data(), sizeof(double) * B * d, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    if (upload_counts(h, nullptr, nullptr) != SMAP_OK) return bail(SMAP_E_CUDA, h->err);
    if (reset_device_state(h) != SMAP_OK) return bail(SMAP_E_CUDA, h->err);
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(SMAP_E_CUDA, cudaGetErrorString(e));
    h->variant = -1;
    *out = h;
    return SMAP_OK;
}

smap_status smap_dims(const smap_handle* h, int* d, int* dy) {
    if (!h) return SMAP_E_INVAL;
    if (d) *d = h->d;
    if (dy) *dy = h->dy;
    return SMAP_OK;
}

smap_status smap_reset(smap_handle* h, const double* x0) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (x0) {
        for (size_t k = 0; k < (size_t)h->B * h->d; ++k)
            if (!std::isfinite(x0[k])) return fail(h, SMAP_E_NONFINITE, "x0 not finite");
        h->x0h.assign(x0, x0 + (size_t)h->B * h->d);
        SMAP_CUDA(h, cudaMemcpyAsync(h->x0, h->x0h.data(), sizeof(double) * h->x0h.size(),
                                     cudaMemcpyHostToDevice, h->stream));
    }
    std::fill(h->tcur_h.begin(), h->tcur_h.end(), 0);
    st = reset_device_state(h);
    if (st) return st;
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_set_particle_counts(smap_handle* h, const int* N_per_seq) {
    smap_status st = check_usable(h);
    if (st) return st;
    for (int b = 0; b < h->B; ++b)
        if (h->tcur_h[b] != 0) return fail(h, SMAP_E_STATE, "particle counts can only change at t = 0");
    return upload_counts(h, h->Tend_h.data(), N_per_seq);
}

smap_status smap_set_variant(smap_handle* h, int v) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (v >= kNumVariants) return fail(h, SMAP_E_INVAL, "variant out of range");
    if (v >= 0 && !variant_threads(v, h->Nmax)) return fail(h, SMAP_E_UNSUPPORTED, "variant cannot hold N particles");
    h->variant = v < 0 ? -1 : v;
    return SMAP_OK;
}

smap_status smap_get_variant(const smap_handle* h, int* v, int* threads, int* grid) {
    if (!h) return SMAP_E_INVAL;
    const int vv = h->variant >= 0 ? h->variant : heuristic_variant(h);
    if (v) *v = vv;
    if (threads) *threads = variant_threads(vv, h->Nmax);
    if (grid) *grid = h->last_grid;
    return SMAP_OK;
}

smap_status smap_step(smap_handle* h, const float* y, const uint8_t* active, int on_device) {
    NvtxRange nvtx_("smap_step");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!y) return fail(h, SMAP_E_INVAL, "y is null");
    for (int b = 0; b < h->B; ++b)
        if ((!active || active[b]) && h->tcur_h[b] >= h->maxT)
            return fail(h, SMAP_E_INVAL, "a sequence is already at max_T");
    if (!on_device) {
        for (size_t k = 0; k < (size_t)h->B * h->dy; ++k)
            if (std::isinf(y[k])) return fail(h, SMAP_E_NONFINITE, "observation is infinite");
    }
    // the pinned staging buffers may still feed the previous step's copies
    SMAP_CUDA(h, cudaEventSynchronize(h->step_done));
    if (on_device) {
        SMAP_CUDA(h, cudaMemcpyAsync(h->ystep, y, sizeof(float) * h->B * h->dy, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        memcpy(h->ystep_h, y, sizeof(float) * h->B * h->dy);
        SMAP_CUDA(h, cudaMemcpyAsync(h->ystep, h->ystep_h, sizeof(float) * h->B * h->dy, cudaMemcpyHostToDevice, h->stream));
    }
    for (int b = 0; b < h->B; ++b) h->active_h[b] = (!active || active[b]) ? 1 : 0;
    SMAP_CUDA(h, cudaMemcpyAsync(h->active, h->active_h, h->B, cudaMemcpyHostToDevice, h->stream));
    SMAP_CUDA(h, cudaEventRecord(h->step_done, h->stream));
    const int v = h->variant >= 0 ? h->variant : heuristic_variant(h);
    StepOpts so;
    so.active = h->active;
    st = launch_seq(h, v, h->B, 1, h->ystep, 0, nullptr, nullptr, nullptr, so);
    if (st) return st;
    for (int b = 0; b < h->B; ++b)
        if (h->active_h[b]) h->tcur_h[b] += 1;
    return SMAP_OK;
}

smap_status smap_map_sequence(smap_handle* h, float* path, double* J, int on_device) {
    NvtxRange nvtx_("smap_map_sequence");
    smap_status st = check_usable(h);
    if (st) return st;
    st = launch_backtrack(h);
    if (st) return st;
    st = copy_outputs(h, path, J, on_device);
    if (st) return st;
    return collect_status(h);
}

smap_status smap_run_batch(smap_handle* h, const float* y_all, const int* T_per_seq, const int* N_per_seq,
                           float* path, double* J, int on_device) {
    NvtxRange nvtx_("smap_run_batch");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!y_all) return fail(h, SMAP_E_INVAL, "y_all is null");
    st = upload_counts(h, T_per_seq, N_per_seq);
    if (st) return st;
    SMAP_CUDA(h, cudaMemcpyAsync(h->y, y_all, sizeof(float) * (size_t)h->B * h->maxT * h->dy,
                                 kind_in(on_device), h->stream));
    const int v = h->variant >= 0 ? h->variant : heuristic_variant(h);
    if (!variant_threads(v, h->Nmax)) return fail(h, SMAP_E_UNSUPPORTED, "kernel variant cannot hold N particles");
    st = configure_kernel(h, h->K->seq[v], smem_layout(h->Nmax, h->K->DP).total);
    if (st) return st;
    if (!h->graph || h->graph_variant != v) {
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        SMAP_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = g_launches.load();
        h->capturing = true;
        smap_status cst = batch_device_work(h, v);
        h->capturing = false;
        cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        g_launches.store(before);   // capture records launches; they run at replay
        if (cst) {
            if (g) cudaGraphDestroy(g);
            return cst;
        }
        if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaGraphInstantiate");
        h->graph_variant = v;
    }
    SMAP_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
    g_launches.fetch_add(2);
    for (int b = 0; b < h->B; ++b) h->tcur_h[b] = h->Tend_h[b];
    st = copy_outputs(h, path, J, on_device);
    if (st) return st;
    return collect_status(h);
}

smap_status smap_get_history(smap_handle* h, float* hist, int on_device) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!hist) return fail(h, SMAP_E_INVAL, "null output");
    SMAP_CUDA(h, cudaMemcpyAsync(hist, h->hist, sizeof(float) * (size_t)h->B * h->maxT * h->Nmax * h->d,
                                 kind_out(on_device), h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_get_backpointers(smap_handle* h, uint16_t* psi, int on_device) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!psi) return fail(h, SMAP_E_INVAL, "null output");
    SMAP_CUDA(h, cudaMemcpyAsync(psi, h->psi, sizeof(uint16_t) * (size_t)h->B * h->maxT * h->Nmax,
                                 kind_out(on_device), h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_get_scores(smap_handle* h, double* phi, int on_device) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!phi) return fail(h, SMAP_E_INVAL, "null output");
    SMAP_CUDA(h, cudaMemcpyAsync(phi, h->phi, sizeof(double) * (size_t)h->B * h->Nmax, kind_out(on_device), h->stream));
    SMAP_CUDA(h, cudaStreamSynchronize(h->stream));
    return SMAP_OK;
}

smap_status smap_get_steps(smap_handle* h, int* t) {
    if (!h || !t) return SMAP_E_INVAL;
    std::copy(h->tcur_h.begin(), h->tcur_h.end(), t);
    return SMAP_OK;
}

smap_status smap_viterbi(smap_handle* h, const float* hist, const float* y_all, const int* T_per_seq,
                         const int* N_per_seq, float* path, double* J, uint16_t* psi, int on_device) {
    NvtxRange nvtx_("smap_viterbi");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!hist || !y_all) return fail(h, SMAP_E_INVAL, "null input");
    st = upload_counts(h, T_per_seq, N_per_seq);
    if (st) return st;
    SMAP_CUDA(h, cudaMemcpyAsync(h->hist, hist, sizeof(float) * (size_t)h->B * h->maxT * h->Nmax * h->d,
                                 kind_in(on_device), h->stream));
    SMAP_CUDA(h, cudaMemcpyAsync(h->y, y_all, sizeof(float) * (size_t)h->B * h->maxT * h->dy,
                                 kind_in(on_device), h->stream));
    st = reset_device_state(h);
    if (st) return st;
    st = launch_rec(h);
    if (st) return st;
    st = launch_backtrack(h);
    if (st) return st;
    for (int b = 0; b < h->B; ++b) h->tcur_h[b] = h->Tend_h[b];
    if (psi)
        SMAP_CUDA(h, cudaMemcpyAsync(psi, h->psi, sizeof(uint16_t) * (size_t)h->B * h->maxT * h->Nmax,
                                     kind_out(on_device), h->stream));
    st = copy_outputs(h, path, J, on_device);
    if (st) return st;
    return collect_status(h);
}

smap_status smap_pf_run_batch(smap_handle* h, const float* y_all, const int* T_per_seq, const int* N_per_seq,
                              float* path, double* J, int on_device) {
    NvtxRange nvtx_("smap_pf_run_batch");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!y_all) return fail(h, SMAP_E_INVAL, "y_all is null");
    st = upload_counts(h, T_per_seq, N_per_seq);
    if (st) return st;
    if (!h->pf_x64) {
        if (cudaMalloc(&h->pf_x64, sizeof(double) * (size_t)h->B * h->Nmax * h->d) != cudaSuccess ||
            cudaMalloc(&h->pf_lw, sizeof(double) * (size_t)h->B * h->Nmax) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SMAP_E_NOMEM, "PF-MAP-Seq: cudaMalloc failed");
        }
    }
    SMAP_CUDA(h, cudaMemcpyAsync(h->y, y_all, sizeof(float) * (size_t)h->B * h->maxT * h->dy,
                                 kind_in(on_device), h->stream));
    st = reset_device_state(h);
    if (st) return st;
    const int v = h->Nmax <= 1024 ? 0 : 1;
    const void* fn = h->K->pf[v];
    const int nt = round_up(v == 0 ? h->Nmax : (h->Nmax + 3) / 4, 32);
    const size_t smem = smem_layout(h->Nmax, h->K->DP).total;
    st = configure_kernel(h, fn, smem);
    if (st) return st;
    int occ = 0;
    SMAP_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem));
    if (occ < 1) return fail(h, SMAP_E_UNSUPPORTED, "PF-MAP-Seq kernel does not fit on an SM");
    PfArgs a;
    memset(&a, 0, sizeof(a));
    a.mp = h->mp;
    a.B = h->B;
    a.Nmax = h->Nmax;
    a.maxT = h->maxT;
    a.seed = h->cfg.seed;
    a.y = h->y;
    a.x0 = h->x0;
    a.hist = h->hist;
    a.psi = h->psi;
    a.phi = h->phi;
    a.tcur = h->tcur;
    a.Nseq = h->Nseq;
    a.Tend = h->Tend;
    a.order = h->order;
    a.f64 = h->f64;
    a.x64 = h->pf_x64;
    a.lw = h->pf_lw;
    a.status = h->status;
    a.queue = h->queue;
    const int grid = std::max(1, std::min(h->B, occ * h->num_sms));
    void* args[] = {&a};
    SMAP_CUDA(h, cudaMemsetAsync(a.queue, 0, sizeof(int), h->stream));
    SMAP_CUDA(h, cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, h->stream));
    SMAP_CUDA(h, cudaGetLastError());
    g_launches.fetch_add(1);
    h->last_threads = nt;
    h->last_grid = grid;
    st = launch_backtrack(h);
    if (st) return st;
    for (int b = 0; b < h->B; ++b) h->tcur_h[b] = h->Tend_h[b];
    st = copy_outputs(h, path, J, on_device);
    if (st) return st;
    return collect_status(h);
}

smap_status smap_autotune(smap_handle* h, const float* y_all, int sample, int steps, int on_device,
                          int* chosen, float* ms_per_variant, int n_ms) {
    NvtxRange nvtx_("smap_autotune");
    smap_status st = check_usable(h);
    if (st) return st;
    if (!y_all || sample < 1 || steps < 1) return fail(h, SMAP_E_INVAL, "autotune: bad arguments");
    const int items = std::min(sample, h->B);
    const int T = std::min(steps, h->maxT);
    std::vector<int> Tl(h->B, T);
    st = upload_counts(h, Tl.data(), h->Nseq_h.data());
    if (st) return st;
    SMAP_CUDA(h, cudaMemcpyAsync(h->y, y_all, sizeof(float) * (size_t)h->B * h->maxT * h->dy,
                                 kind_in(on_device), h->stream));
    cudaEvent_t e0, e1;
    SMAP_CUDA(h, cudaEventCreate(&e0));
    SMAP_CUDA(h, cudaEventCreate(&e1));
    int best = -1;
    float best_ms = INFINITY;
    for (int v = 0; v < kNumVariants; ++v) {
        float ms = INFINITY;
        const size_t smem = smem_layout(h->Nmax, h->K->DP).total;
        int occ = 0;
        if (variant_threads(v, h->Nmax) && smem <= h->max_smem &&
            configure_kernel(h, h->K->seq[v], smem) == SMAP_OK &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, h->K->seq[v], variant_threads(v, h->Nmax), smem) == cudaSuccess &&
            occ > 0) {
            for (int rep = 0; rep < 2; ++rep) {   // first run warms up
                if ((st = reset_device_state(h))) break;
                SMAP_CUDA(h, cudaEventRecord(e0, h->stream));
                if ((st = launch_seq(h, v, items, 0, h->y, 0, h->order))) break;
                SMAP_CUDA(h, cudaEventRecord(e1, h->stream));
                SMAP_CUDA(h, cudaEventSynchronize(e1));
                SMAP_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
            }
            if (st) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        }
        cudaGetLastError();
        if (ms_per_variant && v < n_ms) ms_per_variant[v] = ms;
        if (ms < best_ms) { best_ms = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) return fail(h, SMAP_E_UNSUPPORTED, "no kernel variant fits");
    h->variant = best;
    if (chosen) *chosen = best;
    std::vector<int> Tfull(h->B, h->maxT);
    st = upload_counts(h, Tfull.data(), h->Nseq_h.data());
    if (st) return st;
    return smap_reset(h, nullptr);
}

smap_status smap_debug_svgd(smap_handle* h, int t, const float* x_prev, int n_prev, const float* x_init,
                            const float* y, int n_iters, float* x_out, float* h_out, const double* phi_prev) {
    smap_status st = check_usable(h);
    if (st) return st;
    if (!x_prev || !x_init || !y || !x_out || t < 1 || n_iters < 0) return fail(h, SMAP_E_INVAL, "debug_svgd: bad arguments");
    if (n_prev != 1 && n_prev != h->Nmax) return fail(h, SMAP_E_INVAL, "debug_svgd: n_prev must be 1 or N");
    const size_t B = h->B, N = h->Nmax, d = h->d;
    float *dxp = nullptr, *dxi = nullptr, *dy = nullptr, *dxo = nullptr, *dho = nullptr;
    double *df = nullptr, *dph = nullptr;
    auto cleanup = [&]() { cudaFree(dxp); cudaFree(dxi); cudaFree(dy); cudaFree(dxo); cudaFree(dho); cudaFree(df); cudaFree(dph); };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&dxp, sizeof(float) * B * n_prev * d)) || (e = cudaMalloc(&dxi, sizeof(float) * B * N * d)) ||
        (e = cudaMalloc(&dy, sizeof(float) * B * h->dy)) || (e = cudaMalloc(&dxo, sizeof(float) * B * N * d)) ||
        (e = cudaMalloc(&dho, sizeof(float) * B * std::max(n_iters, 1))) || (e = cudaMalloc(&df, sizeof(double) * B * n_prev * d)) ||
        (phi_prev && (e = cudaMalloc(&dph, sizeof(double) * B * n_prev)))) {
        cleanup();
        return cuda_fail(h, e, "debug_svgd cudaMalloc");
    }
    cudaMemcpy(dxp, x_prev, sizeof(float) * B * n_prev * d, cudaMemcpyHostToDevice);
    cudaMemcpy(dxi, x_init, sizeof(float) * B * N * d, cudaMemcpyHostToDevice);
    cudaMemcpy(dy, y, sizeof(float) * B * h->dy, cudaMemcpyHostToDevice);
    if (phi_prev) cudaMemcpy(dph, phi_prev, sizeof(double) * B * n_prev, cudaMemcpyHostToDevice);
    DebugSvgdArgs a;
    memset(&a, 0, sizeof(a));
    a.mp = h->mp;
    a.B = (int)B; a.N = (int)N; a.Np = n_prev; a.t = t; a.iters = n_iters;
    a.bw_rule = h->cfg.bw_rule; a.prior = h->cfg.prior; a.kernel = h->cfg.kernel;
    a.eps = (float)h->cfg.step; a.bw_value = (float)h->cfg.bw_value;
    a.xprev = dxp; a.x0 = h->x0; a.xinit = dxi; a.y = dy; a.xout = dxo; a.hout = dho; a.f64 = df;
    a.phiprev = dph;
    a.stats = h->status + h->B;   // the median counters (and the debug word) count this call alone
    e = cudaMemsetAsync(a.stats, 0, sizeof(int) * kStatusExtra, h->stream);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(h, e, "debug_svgd"); }
    const int v = h->variant >= 0 ? h->variant : heuristic_variant(h);
    const int nt = variant_threads(v, h->Nmax);
    const size_t smem = smem_layout(h->Nmax, h->K->DP).total;
    if ((st = configure_kernel(h, h->K->dbg[v], smem))) { cleanup(); return st; }
    void* args[] = {&a};
    e = cudaLaunchKernel(h->K->dbg[v], dim3((unsigned)B), dim3(nt), args, smem, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    g_launches.fetch_add(1);
    if (e == cudaSuccess) e = cudaMemcpy(x_out, dxo, sizeof(float) * B * N * d, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_out && n_iters > 0) e = cudaMemcpy(h_out, dho, sizeof(float) * B * n_iters, cudaMemcpyDeviceToHost);
    int dbg[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(dbg, h->status + h->B + kDbgWord, sizeof(dbg), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(h, e, "debug_svgd");
    if (dbg[0] != 0)
        return fail(h, SMAP_E_INVAL, "debug build: bounds check " + std::to_string(dbg[0]) + " failed at index " +
                                         std::to_string(dbg[1]));
    return SMAP_OK;
}

smap_status smap_debug_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t key0, uint32_t key1,
                              int n, uint32_t* out) {
    if (n < 1 || !out) return SMAP_E_INVAL;
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 4 * n) != cudaSuccess) return SMAP_E_NOMEM;
    philox_kernel<<<(n + 255) / 256, 256>>>(c0, c1, c2, c3, key0, key1, n, d);
    g_launches.fetch_add(1);
    cudaError_t e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? SMAP_OK : SMAP_E_CUDA;
}

smap_status smap_debug_bounds_probe(int rows, int index, float* value, int* code, int* at) {
#ifdef SMAP_DEBUG
    if (rows < 1 || rows > 1024 || !value || !code || !at) return SMAP_E_INVAL;
    int* dv = nullptr;
    if (cudaMalloc(&dv, sizeof(int) * 4) != cudaSuccess) return SMAP_E_NOMEM;
    cudaError_t e = cudaMemset(dv, 0, sizeof(int) * 4);
    if (e == cudaSuccess) {
        bounds_probe_kernel<<<1, 32, sizeof(float) * 4 * rows>>>(rows, index, dv);
        g_launches.fetch_add(1);
        e = cudaGetLastError();
    }
    int hv[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(hv, dv, sizeof(hv), cudaMemcpyDeviceToHost);
    cudaFree(dv);
    if (e != cudaSuccess) return SMAP_E_CUDA;
    *code = hv[0];
    *at = hv[1];
    memcpy(value, &hv[2], sizeof(float));
    return SMAP_OK;
#else
    (void)rows; (void)index; (void)value; (void)code; (void)at;
    return SMAP_E_UNSUPPORTED;
#endif
}

smap_status smap_debug_df(int fn, const double* in, int n, double* out) {
    if (fn < 0 || fn > 2 || n < 1 || !in || !out) return SMAP_E_INVAL;
    double* dv = nullptr;
    if (cudaMalloc(&dv, sizeof(double) * 2 * n) != cudaSuccess) return SMAP_E_NOMEM;
    cudaError_t e = cudaMemcpy(dv, in, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        df_kernel<<<(n + 255) / 256, 256>>>(fn, dv, n, dv + n);
        g_launches.fetch_add(1);
        e = cudaMemcpy(out, dv + n, sizeof(double) * n, cudaMemcpyDeviceToHost);
    }
    cudaFree(dv);
    return e == cudaSuccess ? SMAP_OK : SMAP_E_CUDA;
}

smap_status smap_debug_normals(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i0, int n, int d, float* out) {
    if (n < 1 || !out) return SMAP_E_INVAL;
    if (d != 1 && d != 4 && d != 14) return SMAP_E_UNSUPPORTED;
    float* dv = nullptr;
    if (cudaMalloc(&dv, sizeof(float) * d * n) != cudaSuccess) return SMAP_E_NOMEM;
    const int g = (n + 255) / 256;
    if (d == 1) normals_kernel<1><<<g, 256>>>(seed, seq, t, i0, n, dv);
    else if (d == 4) normals_kernel<4><<<g, 256>>>(seed, seq, t, i0, n, dv);
    else normals_kernel<14><<<g, 256>>>(seed, seq, t, i0, n, dv);
    g_launches.fetch_add(1);
    cudaError_t e = cudaMemcpy(out, dv, sizeof(float) * d * n, cudaMemcpyDeviceToHost);
    cudaFree(dv);
    return e == cudaSuccess ? SMAP_OK : SMAP_E_CUDA;
}

}  // extern "C"
