// Step-kernel instantiations for ModelPlanarArm<7>.
#include "smap_internal.h"
#include "smap_kernels.cuh"
#include "smap_pf.cuh"

namespace smap {

ModelKernels kernels_planar_arm7() {
    using M = ModelPlanarArm<7>;
    ModelKernels k;
    k.kind = M::KIND;
    k.D = M::D;
    k.DP = M::DP;
    k.seq[0] = (const void*)seq_kernel<M, 1, 1024, 1>;
    k.seq[1] = (const void*)seq_kernel<M, 2, 512, 1>;
    k.seq[2] = (const void*)seq_kernel<M, 4, 256, 1>;
    k.seq[3] = (const void*)seq_kernel<M, 2, 256, 4>;
    k.seq[4] = (const void*)seq_kernel<M, 1, 1024, 1, 8>;
    k.seq[5] = (const void*)seq_kernel<M, 1, 1024, 1, 4>;
    k.dbg[0] = (const void*)debug_svgd_kernel<M, 1, 1024, 1>;
    k.dbg[1] = (const void*)debug_svgd_kernel<M, 2, 512, 1>;
    k.dbg[2] = (const void*)debug_svgd_kernel<M, 4, 256, 1>;
    k.dbg[3] = (const void*)debug_svgd_kernel<M, 2, 256, 4>;
    k.dbg[4] = (const void*)debug_svgd_kernel<M, 1, 1024, 1, 8>;
    k.dbg[5] = (const void*)debug_svgd_kernel<M, 1, 1024, 1, 4>;
    k.rec[0] = (const void*)rec_kernel<M, 2, 512, 1>;
    k.rec[1] = (const void*)rec_kernel<M, 2, 1024, 1>;
    k.rec[2] = (const void*)rec_kernel<M, 4, 1024, 1>;
    k.pf[0] = (const void*)pf_seq_kernel<M, 1, 1024>;
    k.pf[1] = (const void*)pf_seq_kernel<M, 4, 1024>;
    return k;
}

}  // namespace smap
