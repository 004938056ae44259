// smap_mlp.cuh -- the learned proposal's network on the tensor cores.
//
// A 3-layer perceptron in -> H -> H -> out (H = 256), GELU after the two
// hidden layers, BF16 weights and activations as MMA operands, FP32
// accumulation (mma.sync m16n8k16). Inputs are standardised features of a
// propagated particle and the observation; the output is the standardised
// displacement from that particle to where plain SVGD takes it.
#pragma once

#include <cuda_bf16.h>

#include "smap_common.cuh"
#include "smap_models.cuh"

namespace smap {

constexpr int kMlpH = 256;      // hidden width
constexpr int kMlpInP = 32;     // padded input width
constexpr int kMlpOutP = 16;    // padded output width
constexpr int kMlpRows = 32;    // rows per tile of the fused forward
constexpr int kMlpPad = 8;      // bf16 padding per smem row (16 bytes)

// Packed FP32 master parameters (padded layout):
// W1 [H][InP], b1 [H], W2 [H][H], b2 [H], W3 [OutP][H], b3 [OutP].
constexpr long kMlpW1 = 0;
constexpr long kMlpB1 = kMlpW1 + (long)kMlpH * kMlpInP;
constexpr long kMlpW2 = kMlpB1 + kMlpH;
constexpr long kMlpB2 = kMlpW2 + (long)kMlpH * kMlpH;
constexpr long kMlpW3 = kMlpB2 + kMlpH;
constexpr long kMlpB3 = kMlpW3 + (long)kMlpOutP * kMlpH;
constexpr long kMlpNP = kMlpB3 + kMlpOutP;

// Inference forward on the 5th-generation tensor cores (smap_mlp_tc.cu):
// xout[r][c] = u[r][c] (or 0) + sd_out[c] clamp(MLP(standardised feat[r]), +-8)[c] + mu_out[c].
struct MlpTcArgs {
    const __nv_bfloat16 *W1, *W2, *W3;   // compact BF16 [H][InP], [H][H], [OutP][H]
    const float *b1, *b2, *b3;
    const float* norm;                   // mu_in[InP], sd_in[InP], mu_out[OutP], sd_out[OutP]
    long rows;
    int d;                               // real output width
    const float* feat;                   // [rows][InP]
    const float* u;                      // [rows][d] or null
    float* xout;                         // [rows][d]
    int* err;                            // set to 1 when a wait gave up (may be null)
    uint64_t wait_ns;                    // limit of every bounded wait (global-timer nanoseconds)
    int stall;                           // test only: the MMA lane first waits on a barrier nothing completes
};
constexpr uint64_t kTcWaitNs = 2000000000ull;   // default wait limit: 2 s
size_t mlp_forward_tc_smem();
cudaError_t mlp_forward_tc_launch(const MlpTcArgs& a, int num_sms, cudaStream_t st);

__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU, tanh form: x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
__device__ __forceinline__ float gelu_f(float x) {
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    return 0.5f * x * (1.0f + tanh_approx(u));
}

__device__ __forceinline__ float gelu_grad_f(float x) {
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    const float th = tanh_approx(u);
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * 0.7978845608028654f *
                                    fmaf(3.0f * 0.044715f, x * x, 1.0f);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// D = A B + D, A 16x16 bf16 (row), B 16x8 bf16 (col), D 16x8 fp32.
__device__ __forceinline__ void mma_16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Proposal features of a propagated particle u and the observation z; each
// ends with the likelihood score grad_u log p(z | u) (the direction SVGD's
// drive starts from).
//   planar arm : [u (14), z (2), z - h(u) (2), score of the angles (7)]   25
//   clutter    : [velocity (2), z_m - position for the 10 points sorted
//                 by distance to the position (20), score of the position (2)] 24
//   others     : [u (d), z (dy) with unheard entries 0, heard flags, score (d)]
// Returns the number of features written (<= kMlpInP).
// ---------------------------------------------------------------------------
template <class M>
__device__ int proposal_features(const ModelParams& mp, const float* u, const float* z, float* f) {
    constexpr int D = M::D;
    float g[D];
    M::grad_loglik(mp, z, u, g);
    if constexpr (M::KIND == 4) {
        constexpr int NL = D / 2;
        const float* len = mp.pf + 3 + 2 * NL;
        float th = 0.0f, ex = 0.0f, ey = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            th += u[l];
            float s, c;
            __sincosf(th, &s, &c);
            ex = fmaf(len[l], c, ex);
            ey = fmaf(len[l], s, ey);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) f[c] = u[c];
        f[D] = z[0];
        f[D + 1] = z[1];
        f[D + 2] = z[0] - ex;
        f[D + 3] = z[1] - ey;
#pragma unroll
        for (int l = 0; l < NL; ++l) f[D + 4 + l] = g[l];
        return D + 4 + NL;
    } else if constexpr (M::KIND == 3) {
        const int Mz = (int)mp.p[6];
        f[0] = u[2];
        f[1] = u[3];
        float dist[32];
        int ord[32];
        for (int m = 0; m < Mz; ++m) {
            const float ex = z[2 * m] - u[0], ey = z[2 * m + 1] - u[1];
            dist[m] = ex * ex + ey * ey;
            ord[m] = m;
        }
        for (int a = 1; a < Mz; ++a) {   // insertion sort, nearest first
            const int o = ord[a];
            const float v = dist[o];
            int k = a - 1;
            while (k >= 0 && dist[ord[k]] > v) { ord[k + 1] = ord[k]; --k; }
            ord[k + 1] = o;
        }
        const int nm = Mz < (kMlpInP - 4) / 2 ? Mz : (kMlpInP - 4) / 2;
        for (int m = 0; m < nm; ++m) {
            f[2 + 2 * m] = z[2 * ord[m]] - u[0];
            f[3 + 2 * m] = z[2 * ord[m] + 1] - u[1];
        }
        f[2 + 2 * nm] = g[0];
        f[3 + 2 * nm] = g[1];
        return 4 + 2 * nm;
    } else {
        int n = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) f[n++] = u[c];
        const int dy = mp.dy < (kMlpInP - 2 * D) / 2 ? mp.dy : (kMlpInP - 2 * D) / 2;
        for (int c = 0; c < dy; ++c) {
            const float v = z[c];
            f[n++] = (v == v) ? v : 0.0f;
        }
        for (int c = 0; c < dy; ++c) f[n++] = (z[c] == z[c]) ? 1.0f : 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) f[n++] = g[c];
        return n;
    }
}

}  // namespace smap
