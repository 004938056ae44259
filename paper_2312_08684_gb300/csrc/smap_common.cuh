// smap_common.cuh -- device-side types and helpers shared by the step kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smap {

constexpr int kMaxD = 16;        // largest compiled state dimension
constexpr int kMaxParams = 128;  // model parameter vector length
constexpr int kMaxDy = 64;       // largest observation dimension
constexpr int kCandCap = 2048;   // median bracket candidates kept in shared memory
constexpr int kMaxN = 4096;      // particles per sequence (backpointers are uint16)
constexpr int kStatusExtra = 7;  // after the B per-sequence status words: 4 median counters, 1 error word,
                                 // 2 words of the debug build's first failed bounds check (code, index)
constexpr int kDbgWord = 5;      // offset of those 2 words after the B status words

// Model constants, passed by value in the kernel parameters (constant bank).
struct ModelParams {
    int kind, d, dy, np;
    double p[kMaxParams];     // raw parameters
    float pf[kMaxParams];     // the same in FP32
    double q[kMaxD];          // diag(Q)
    double qinv[kMaxD];
    double sqrt_q[kMaxD];
    double sqrt_qinv[kMaxD];
    float qinv_f[kMaxD];
    float sqrt_qinv_f[kMaxD];
    double logtrans_c;        // -1/2 sum_d log(2 pi q_d)
    double aux[8];            // model-specific constants (see smap_models.cuh)
    float auxf[8];
    // double-float (hi, lo) forms of the FP64 constants: p = pf + pl,
    // qinv = qinv_f + qinv_lo, logtrans_c = ltc[0] + ltc[1], aux = auxh + auxl
    float pl[kMaxParams];
    float qinv_lo[kMaxD];
    float ltc[2];
    float auxh[8], auxl[8];
};

// Per-launch arguments of the sequence kernel.
struct SeqArgs {
    ModelParams mp;
    int B, Nmax, maxT, L, bw_rule, prior;
    int mode;                 // 0: run each sequence from tcur to Tend; 1: one step
    float eps, bw_value;
    uint64_t seed;
    const float* y;           // mode 0: [B][maxT][dy]; mode 1: [B][dy]
    const double* x0;         // [B][d]
    float* hist;              // [B][maxT][Nmax][d]
    uint16_t* psi;            // [B][maxT][Nmax]
    double* phi;              // [B][Nmax]
    int* tcur;                // [B]
    const int* Nseq;          // [B]
    const int* Tend;          // [B]
    const uint8_t* active;    // [B] or null (mode 1)
    const int* order;         // [B] processing order or null
    double* f64;              // [gridDim][Nmax][d] FP64 transition means (scratch)
    float* bwguess;           // [B] last median of squared distances (scratch)
    int* status;              // [B] per-sequence status (0 or an smap_status)
    int* queue;               // [1] work-queue head
    int* stats;               // [3] median-path counters (shared by all launches of a handle)
    int viterbi_only;         // 1: particle sets are given in hist (no SVGD)
    const float* xinit;       // mode 1: [B][Nmax][d] initial particles of the step, or null
    int y_full;               // mode 1: y is [B][maxT][dy] (indexed by the step)
    int skip_done;            // mode 1: skip sequences with tcur >= Tend
    int seq_base;             // without `order`, item k is sequence seq_base + k
    int Btot;                 // sequences of the handle's arrays (debug build's bounds checks)
    unsigned long long* rstats;  // [3] recursion counters: particle-steps, near-ties, FP64 candidate scores (or null)
    int kernel;               // Stein kernel: 0 RBF, 1 IMQ, 2 Matern 3/2
};

// Arguments of the debug SVGD kernel.
struct DebugSvgdArgs {
    ModelParams mp;
    int B, N, Np, t, iters, bw_rule, prior;
    float eps, bw_value;
    const float* xprev;       // [B][Np][d]
    const double* x0;         // [B][d] (t == 1, Np == 1)
    const float* xinit;       // [B][N][d]
    const float* y;           // [B][dy]
    float* xout;              // [B][N][d]
    float* hout;              // [B][iters]
    double* f64;              // [B][Np][d] scratch
    const double* phiprev;    // [B][Np] previous scores (MAP-conditioned prior), or null = zeros
    int kernel;               // Stein kernel: 0 RBF, 1 IMQ, 2 Matern 3/2
    int* stats;               // median-path counters [4] (see median_sqdist), or null
};

#ifdef SMAP_DEBUG
// Debug build (SMAP_DEBUG): the row index of every shared-memory particle
// array access and the sequence / step / particle indices of the global
// arrays are checked before the access; a failed check records (code, index)
// in the launch's debug word (the first failure wins) and the access is
// skipped: loads return zeros, stores are dropped. Nothing traps.
__shared__ int g_dbg_rows;    // rows of the shared [rows][DP] arrays of this block
__shared__ int* g_dbg_word;   // [2] (code, index), or null
__device__ __forceinline__ bool dbg_check(bool ok, int code, long long index) {
    if (!ok && g_dbg_word && atomicCAS(g_dbg_word, 0, code) == 0) g_dbg_word[1] = (int)index;
    return ok;
}
// Called by every thread at the start of a kernel that uses the shared rows.
__device__ __forceinline__ void dbg_begin(int rows, int* word) {
    if (threadIdx.x == 0) {
        g_dbg_rows = rows;
        g_dbg_word = word;
    }
    __syncthreads();
}
#define SMAP_DBG(ok, code, index) ::smap::dbg_check((ok), (code), (long long)(index))
#define SMAP_DBG_BEGIN(rows, word) ::smap::dbg_begin((rows), (word))
#else
#define SMAP_DBG(ok, code, index) true
#define SMAP_DBG_BEGIN(rows, word) ((void)0)
#endif
// Codes of the debug build's bounds checks.
enum DbgCode { kDbgRow = 1, kDbgSeq = 2, kDbgStep = 3, kDbgPart = 4, kDbgPrev = 5 };

// ex2.approx: 2^x on the special-function unit (max rel. error ~2^-22).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplies; round keys advance by the Weyl constants.
__host__ __device__ inline void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
#else
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Standard normals of particle i at step t of sequence seq: dimension block b
// (four dimensions) uses counter (i, t, seq, b) under key (seed lo, seed hi);
// each pair of words gives two normals by Box-Muller, u = (w + 1/2) 2^-32.
template <int D>
__device__ inline void draw_normals(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i, float* z) {
#pragma unroll
    for (int b = 0; 4 * b < D; ++b) {
        uint32_t w[4];
        philox4x32_10(i, t, seq, (uint32_t)b, (uint32_t)seed, (uint32_t)(seed >> 32), w);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float u1 = ((float)w[2 * h] + 0.5f) * 2.3283064365386963e-10f;
            float u2 = ((float)w[2 * h + 1] + 0.5f) * 2.3283064365386963e-10f;
            u1 = fmaxf(u1, 1.1754944e-38f);
            float rad = sqrtf(-2.0f * logf(u1));
            float s, c;
            sincospif(2.0f * u2, &s, &c);
            const int k0 = 4 * b + 2 * h;
            if (k0 < D) z[k0] = rad * c;
            if (k0 + 1 < D) z[k0 + 1] = rad * s;
        }
    }
}

// ---- block reductions (every thread of the block must call) --------------
__device__ inline int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ inline float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// red: >= 33 ints of shared scratch.
__device__ inline int block_sum_int(int v, int* red) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_int(v);
    __syncthreads();
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = (int)lane_id() < nw ? red[lane_id()] : 0;
        s = warp_sum_int(s);
        if (lane_id() == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// red: >= 33 doubles of shared scratch.
__device__ inline double block_max_d(double v, double* red) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max_d(v);
    __syncthreads();
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double s = (int)lane_id() < nw ? red[lane_id()] : -INFINITY;
        s = warp_max_d(s);
        if (lane_id() == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// red: >= 33 floats of shared scratch.
__device__ inline float block_max_f(float v, float* red) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float s = (int)lane_id() < nw ? red[lane_id()] : -INFINITY;
#pragma unroll
        for (int o = 16; o; o >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane_id() == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// red: >= 33 floats of shared scratch.
__device__ inline float block_sum_f(float v, float* red) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_f(v);
    __syncthreads();
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float s = (int)lane_id() < nw ? red[lane_id()] : 0.0f;
        s = warp_sum_f(s);
        if (lane_id() == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

}  // namespace smap
