// smap_internal.h -- kernel tables shared by the instantiation units and the ABI.
#pragma once

#include <atomic>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "smap.h"
#include "smap_common.cuh"

namespace smap {

// Compiled variants of the step kernels: particles per thread, the block-size
// bound given to the compiler, the minimum resident blocks it targets, and
// threads per particle (the lanes that split one particle's sums over the
// other particles: shorter serial chains when a sequence's block would
// otherwise hold only a warp or two).
struct VariantInfo {
    int ppt, maxt, minb, tpp;
};
constexpr int kNumVariants = 6;
constexpr VariantInfo kVariants[kNumVariants] = {{1, 1024, 1, 1}, {2, 512, 1, 1}, {4, 256, 1, 1},
                                                 {2, 256, 4, 1}, {1, 1024, 1, 8}, {1, 1024, 1, 4}};

// Compiled variants of the recursion-only kernel (particles per thread, block
// size bound, minimum resident blocks).
struct RecVariantInfo {
    int ppt, maxt, minb;
};
constexpr int kNumRecVariants = 3;
constexpr RecVariantInfo kRecVariants[kNumRecVariants] = {{2, 512, 1}, {2, 1024, 1}, {4, 1024, 1}};

struct ModelKernels {
    int kind, D, DP;
    const void* seq[kNumVariants];   // seq_kernel<M, ...>
    const void* rec[kNumRecVariants];   // rec_kernel<M, ...>
    const void* dbg[kNumVariants];   // debug_svgd_kernel<M, ...>
    const void* pf[2];               // pf_seq_kernel<M, 1, 1024> (N <= 1024), <M, 4, 1024> (N <= 4096)
};

ModelKernels kernels_ngm1d();
ModelKernels kernels_range_cv();
ModelKernels kernels_clutter_cv();
ModelKernels kernels_planar_arm7();
ModelKernels kernels_linear_gauss();
ModelKernels kernels_range_zv();
ModelKernels kernels_se2_rb();

// Rows of the learned proposal: propagated particles u = f_t(x_{t-1}^i) + noise
// (drawn exactly like the step kernels' initialisation) and their features.
//   capture = 0: one row per (b, i) at t = tcur[b] + 1 (learned initialisation);
//   capture = 1: one row per (b, t <= Tend[b], i), row_base[b][t-1] + i, with
//                the displacement target x_t^i - u (training data).
struct ProposalRowsArgs {
    ModelParams mp;
    int B, Nmax, maxT, capture;
    int b_base;                   // learned initialisation: rows are sequences b_base .. b_base + B - 1
    uint64_t seed;
    const double* x0;             // [B][d]
    const float* hist;            // [B][maxT][Nmax][d]
    const float* y;               // [B][maxT][dy]
    const int* tcur;              // [B]
    const int* Tend;              // [B]
    const int* Nseq;              // [B]
    const long long* row_base;    // [B][maxT] (capture)
    float* feat;                  // [rows][32]
    float* u;                     // [rows][d] or null
    float* targ;                  // [rows][16] or null (capture)
    int* err;                     // learned initialisation: set to 1 if the network kernel gave up a wait
};

// Defined in smap_mlp.cu.
smap_status proposal_launch_init(smap_proposal* p, const ProposalRowsArgs& ra, float* xinit, cudaStream_t st);
smap_status proposal_launch_capture(smap_proposal* p, const ProposalRowsArgs& ra, cudaStream_t st);
int proposal_kind(const smap_proposal* p);
int proposal_d(const smap_proposal* p);

// A named NVTX range over the lifetime of the object (a no-op unless a
// profiler is attached): the entry points mark their host-side phases.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Shared by the ABI translation units (defined in smap_api.cu).
extern std::atomic<uint64_t> g_launches;
// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes`, and never lowers it: handles of different N and the
// handle-free entry points launch the same kernel functions with different
// sizes, and the limit is one per function and device. Reads the current limit
// from the device each time (so it holds across a device reset) under one
// process-wide mutex (so two threads cannot interleave a read and a lower
// write). Not a stream operation.
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);
const ModelKernels* kernels_for(int kind);
bool make_model(int kind, const double* p, int np, ModelParams& mp, std::string& err);
int variant_threads(int v, int Nmax);
int pick_variant(int d, int Nmax, int B, int sms);
int rec_variant_threads(int v, int Nmax);
int pick_rec_variant(int d, int Nmax);
__global__ void backtrack_kernel(int B, int Nmax, int maxT, int d, const int* __restrict__ tcur,
                                 const int* __restrict__ Nseq, const double* __restrict__ phi,
                                 const uint16_t* __restrict__ psi, const float* __restrict__ hist,
                                 const double* __restrict__ x0, const int* __restrict__ status,
                                 int* __restrict__ idxbuf, float* __restrict__ path,
                                 double* __restrict__ J);

}  // namespace smap
