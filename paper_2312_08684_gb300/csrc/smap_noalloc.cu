// smap_noalloc.cu -- smap_viterbi_noalloc: the particle dynamic programme
// (forward recursion + backtracking over given particle sets) without any
// device allocation.
//
// Some callers cannot call cudaMalloc: a plug-in whose host application owns
// the whole device-memory budget and hands it only input and output buffers,
// or a control loop that must never enter the allocator once it runs (an
// allocation can block or fail). smap_viterbi needs a handle, and a handle
// allocates its buffers. This entry point keeps its working state (scores,
// backpointers, transition means, work queue, status words, the backtracking
// index chain) in one file-scope device array of fixed size instead, which
// every GPU that loads the library holds until the process exits.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "smap.h"
#include "smap_internal.h"
#include "smap_kernels.cuh"

using namespace smap;

namespace {

// Working state of smap_viterbi_noalloc on each device: 16 MiB.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// and context: a device reset creates a new context, in which the module (and
// the array) may be loaded at another address, so the lookup is redone when
// the current context's identity changes.
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 256;
struct ScratchAddr {
    unsigned long long ctx = 0;   // cuCtxGetId of the context the address belongs to (0: none yet)
    void* addr = nullptr;
};
ScratchAddr g_noalloc_addr[kMaxDevices];

// Identity of the calling thread's current context, unique over the process's
// lifetime (cuCtxGetId); 0 when no context is current or the driver entry
// points are unavailable. The library links only the runtime, so the two
// driver calls are reached through the runtime's entry-point lookup.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // called with g_noalloc_mu held
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 4000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            get_cur = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carved {
    uint16_t* psi;
    double* phi;
    double* f64;
    int *tcur, *Nseq, *Tend, *status, *queue, *idx;
    float* bwguess;
    size_t total;
};

// Sub-buffers of the scratch array (base may be null to size them).
Carved carve(unsigned char* base, int B, int N, int T, int d, int grid) {
    Carved c{};
    size_t off = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base ? base + off : nullptr; off += a256(bytes); return p; };
    c.psi = (uint16_t*)take(sizeof(uint16_t) * (size_t)B * T * N);
    c.phi = (double*)take(sizeof(double) * (size_t)B * N);
    c.f64 = (double*)take(sizeof(double) * (size_t)grid * N * d);
    c.tcur = (int*)take(sizeof(int) * (size_t)B);
    c.Nseq = (int*)take(sizeof(int) * (size_t)B);
    c.Tend = (int*)take(sizeof(int) * (size_t)B);
    c.status = (int*)take(sizeof(int) * ((size_t)B + kStatusExtra));
    c.queue = (int*)take(sizeof(int) * 4);
    c.bwguess = (float*)take(sizeof(float) * (size_t)B);
    c.idx = (int*)take(sizeof(int) * (size_t)B * T);
    c.total = off;
    return c;
}

// Clears what the previous call left in the shared array.
__global__ void noalloc_init_kernel(int B, int N, int T, int* tcur, int* Nseq, int* Tend, int* status,
                                    int* queue, float* bwguess) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B + kStatusExtra; b += gridDim.x * blockDim.x) {
        status[b] = 0;
        if (b < B) {
            tcur[b] = 0;
            Nseq[b] = N;
            Tend[b] = T;
            bwguess[b] = 0.0f;
        }
        if (b == 0) queue[0] = 0;
    }
}

smap_status reject(const char* msg) {
    std::fprintf(stderr, "smap_viterbi_noalloc: %s\n", msg);
    return SMAP_E_INVAL;
}

}  // namespace

extern "C" smap_status smap_viterbi_noalloc(int model, const double* params, int n_params, int B, int N,
                                            int T, const double* x0, const float* hist, const float* y,
                                            float* path, double* J, void* stream) {
    if (!params || !x0 || !hist || !y || !path || !J) return reject("null pointer argument");
    if (B < 1 || T < 1 || N < 1 || N > kMaxN) return reject("need B >= 1, T >= 1, 1 <= N <= 4096");
    const ModelKernels* K = kernels_for(model);
    if (!K) return reject("unknown model");
    ModelParams mp;
    std::string err;
    if (!make_model(model, params, n_params, mp, err)) return reject(err.c_str());
    const int d = mp.d;
    if (d != K->D) return reject("state dimension does not match the compiled model");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SMAP_E_CUDA;
    void* base = nullptr;
    {
        // set-up, once per device (and again after a device reset), with that
        // device current
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        ScratchAddr& sa = g_noalloc_addr[dev];
        const unsigned long long ctx = current_context_id();
        if (!sa.addr || ctx == 0 || ctx != sa.ctx) {
            void* addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                sa = ScratchAddr();
                std::fprintf(stderr, "smap_viterbi_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
                return SMAP_E_CUDA;
            }
            sa.addr = addr;
            sa.ctx = current_context_id();   // the lookup made the primary context current if none was
        }
        base = sa.addr;
    }

    const int v = pick_variant(d, N, B, 0);   // the recursion alone: no lane split (sms = 0)
    const int nt = variant_threads(v, N);
    const void* fn = K->seq[v];
    const size_t smem = smem_layout(N, K->DP).total;
    int smem_optin = 0, sms = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SMAP_E_CUDA;
    if (!nt || smem > (size_t)smem_optin) return reject("N too large for shared memory at this state dimension");
    // raise, never lower: live handles launch the same kernel with larger sizes
    if (ensure_dynamic_smem(fn, smem) != cudaSuccess) return SMAP_E_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem) != cudaSuccess || occ < 1)
        return SMAP_E_CUDA;
    const int grid = std::max(1, std::min(B, occ * sms));

    const Carved c = carve((unsigned char*)base, B, N, T, d, grid);
    if (c.total > kNoallocScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof(msg), "B=%d, N=%d, T=%d need %zu bytes of working state; the maximum is %zu",
                      B, N, T, c.total, kNoallocScratchBytes);
        return reject(msg);
    }

    cudaStream_t st = (cudaStream_t)stream;
    auto launch_failed = [](cudaError_t e) {
        std::fprintf(stderr, "smap_viterbi_noalloc: %s\n", cudaGetErrorString(e));
        return SMAP_E_CUDA;
    };
    noalloc_init_kernel<<<(B + kStatusExtra + 255) / 256, 256, 0, st>>>(B, N, T, c.tcur, c.Nseq, c.Tend, c.status,
                                                             c.queue, c.bwguess);
    g_launches.fetch_add(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launch_failed(e);
    SeqArgs a;
    memset(&a, 0, sizeof(a));
    a.mp = mp;
    a.B = B;
    a.Nmax = N;
    a.maxT = T;
    a.mode = 0;
    a.viterbi_only = 1;
    a.y = y;
    a.x0 = x0;
    a.hist = const_cast<float*>(hist);   // read only when viterbi_only = 1
    a.psi = c.psi;
    a.phi = c.phi;
    a.tcur = c.tcur;
    a.Nseq = c.Nseq;
    a.Tend = c.Tend;
    a.f64 = c.f64;
    a.bwguess = c.bwguess;
    a.status = c.status;
    a.stats = c.status + B;
    a.Btot = B;
    a.queue = c.queue;
    void* args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, st);
    if (e != cudaSuccess) return launch_failed(e);
    g_launches.fetch_add(1);
    // backtracking reads what the recursion wrote: enqueued only after that
    // launch was accepted
    backtrack_kernel<<<(B + 3) / 4, 128, 0, st>>>(B, N, T, d, c.tcur, c.Nseq, c.phi, c.psi, hist, x0,
                                                  c.status, c.idx, path, J);
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_failed(e);
    g_launches.fetch_add(1);
    return SMAP_OK;
}
