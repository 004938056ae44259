// smap_internal.h -- kernel tables shared by the instantiation units and the ABI.
#pragma once

#include "smap_common.cuh"

namespace smap {

// Compiled variants of the step kernels: particles per thread, the block-size
// bound given to the compiler, and the minimum resident blocks it targets.
struct VariantInfo {
    int ppt, maxt, minb;
};
constexpr int kNumVariants = 4;
constexpr VariantInfo kVariants[kNumVariants] = {{1, 1024, 1}, {2, 512, 1}, {4, 256, 1}, {2, 256, 4}};

struct ModelKernels {
    int kind, D, DP;
    const void* seq[kNumVariants];   // seq_kernel<M, ...>
    const void* dbg[kNumVariants];   // debug_svgd_kernel<M, ...>
};

ModelKernels kernels_ngm1d();
ModelKernels kernels_range_cv();
ModelKernels kernels_clutter_cv();
ModelKernels kernels_planar_arm7();
ModelKernels kernels_linear_gauss();

}  // namespace smap
