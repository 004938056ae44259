// smap_mlp.cu -- kernels and C ABI of the learned proposal (smap_proposal_*).
//
// Forward: one fused kernel, weights resident in shared memory as BF16 (the
// 256-wide arrays XOR-swizzled instead of padded), 64-row tiles through three
// mma.sync layers with GELU, FP32 accumulation.
// Backward: a tiled BF16 GEMM (split-K for the weight gradients), GELU
// derivative fused into its epilogue, column sums for the bias gradients.
// Update: Adam on FP32 master weights, BF16 copies refreshed each step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "smap.h"
#include "smap_internal.h"
#include "smap_kernels.cuh"
#include "smap_mlp.cuh"

using namespace smap;
typedef __nv_bfloat16 bf16;

namespace smap {

// ---------------------------------------------------------------------------
// Fused forward.
// ---------------------------------------------------------------------------
struct MlpFwdArgs {
    const bf16 *W1, *W2, *W3;     // compact [H][InP], [H][H], [OutP][H]
    const float *b1, *b2, *b3;
    const float* norm;            // mu_in[InP], sd_in[InP], mu_out[OutP], sd_out[OutP]
    long rows;
    int d;                        // real output width
    const float* feat;            // [*][InP]
    const int* idx;               // optional row gather (training)
    bf16* xn;                     // optional [rows][InP] standardised input (training)
    float* z1;                    // optional [rows][H] pre-activations (training)
    bf16* h1;
    float* z2;
    bf16* h2;
    float* o;                     // optional [rows][OutP] standardised output (training)
    const float* u;               // optional [rows][d] base particles
    float* xout;                  // optional [rows][d]: u + displacement (physical units)
};

constexpr int kLdIn = kMlpInP + kMlpPad;   // padded row of the 32-wide arrays (W1, X)
constexpr int kFwdRows = 64;                 // rows per tile of the fused forward

// Element index in a 256-wide bf16 array whose 16-byte chunks are XOR-swizzled
// by the row (chunk q of row r lives at q ^ (r & 7)): ldmatrix on 8 rows at the
// same logical chunk touches 8 different bank groups.
__device__ __forceinline__ int swz256(int r, int c) { return r * kMlpH + ((((c >> 3) ^ (r & 7))) << 3) + (c & 7); }

__host__ __device__ inline size_t mlp_fwd_smem() {
    return sizeof(bf16) * ((size_t)kMlpH * kLdIn +          // W1
                           (size_t)kMlpH * kMlpH +          // W2 (swizzled)
                           (size_t)kMlpOutP * kMlpH +       // W3 (swizzled)
                           (size_t)kFwdRows * kMlpH +       // H1 (swizzled)
                           (size_t)kFwdRows * kMlpH) +      // H2 (swizzled), X aliased at its start
           sizeof(float) * (2 * kMlpH + kMlpOutP + 2 * kMlpInP + 2 * kMlpOutP);
}

// One hidden layer for the 64-row tile: warp w computes columns [32w, 32w+32)
// of all 64 rows (4 x 4 MMA tiles). A is the padded 32-wide input (layer 1) or
// a swizzled 256-wide activation (layer 2); W likewise.
template <int K>
__device__ __forceinline__ void mlp_hidden(const bf16* sA, const bf16* sW, const float* bias, bf16* sOut,
                                           float* zg, bf16* hg, long row0, long rows) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = warp * 32;
    float acc[4][4][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    const int q = lane >> 3, r8 = lane & 7;
#pragma unroll 2
    for (int kk = 0; kk < K; kk += 16) {
        uint32_t a[4][4];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int r = mt * 16 + (q & 1) * 8 + r8, c = kk + (q >> 1) * 8;
            const bf16* pa = (K == kMlpH) ? sA + swz256(r, c) : sA + r * kLdIn + c;
            ldsm_x4(smem_addr(pa), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {
            const int r = n0 + np * 16 + (q >> 1) * 8 + r8, c = kk + (q & 1) * 8;
            const bf16* pw = (K == kMlpH) ? sW + swz256(r, c) : sW + r * kLdIn + c;
            uint32_t b0, b1, b2, b3;
            ldsm_x4(smem_addr(pw), b0, b1, b2, b3);
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                mma_16816(acc[mt][2 * np], a[mt], b0, b1);
                mma_16816(acc[mt][2 * np + 1], a[mt], b2, b3);
            }
        }
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = mt * 16 + g + hh * 8;
                const int c = n0 + nt * 8 + 2 * tq;
                const float za = acc[mt][nt][2 * hh] + bias[c];
                const float zb = acc[mt][nt][2 * hh + 1] + bias[c + 1];
                __nv_bfloat162 pr;
                pr.x = __float2bfloat16(gelu_f(za));
                pr.y = __float2bfloat16(gelu_f(zb));
                *reinterpret_cast<__nv_bfloat162*>(sOut + swz256(r, c)) = pr;
                const long gr = row0 + r;
                if (gr < rows) {
                    if (zg) *reinterpret_cast<float2*>(zg + gr * kMlpH + c) = make_float2(za, zb);
                    if (hg) *reinterpret_cast<__nv_bfloat162*>(hg + gr * kMlpH + c) = pr;
                }
            }
}

__global__ void __launch_bounds__(256, 1) mlp_forward_kernel(const __grid_constant__ MlpFwdArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16* sW1 = reinterpret_cast<bf16*>(smraw);
    bf16* sW2 = sW1 + kMlpH * kLdIn;
    bf16* sW3 = sW2 + kMlpH * kMlpH;
    bf16* sH1 = sW3 + kMlpOutP * kMlpH;
    bf16* sH2 = sH1 + kFwdRows * kMlpH;
    bf16* sX = sH2;   // the input tile is dead once layer 1 has run
    float* sb1 = reinterpret_cast<float*>(sH2 + kFwdRows * kMlpH);
    float* sb2 = sb1 + kMlpH;
    float* sb3 = sb2 + kMlpH;
    float* snorm = sb3 + kMlpOutP;   // mu_in, sd_in, mu_out, sd_out
    const int tid = threadIdx.x;
    for (int e = tid; e < kMlpH * kMlpInP; e += blockDim.x) sW1[(e / kMlpInP) * kLdIn + e % kMlpInP] = a.W1[e];
    for (int e = tid; e < kMlpH * kMlpH / 8; e += blockDim.x) {
        const int r = (e * 8) / kMlpH, c = (e * 8) % kMlpH;
        *reinterpret_cast<uint4*>(sW2 + swz256(r, c)) = reinterpret_cast<const uint4*>(a.W2)[e];
    }
    for (int e = tid; e < kMlpOutP * kMlpH / 8; e += blockDim.x) {
        const int r = (e * 8) / kMlpH, c = (e * 8) % kMlpH;
        *reinterpret_cast<uint4*>(sW3 + swz256(r, c)) = reinterpret_cast<const uint4*>(a.W3)[e];
    }
    for (int e = tid; e < kMlpH; e += blockDim.x) { sb1[e] = a.b1[e]; sb2[e] = a.b2[e]; }
    for (int e = tid; e < kMlpOutP; e += blockDim.x) sb3[e] = a.b3[e];
    for (int e = tid; e < 2 * kMlpInP + 2 * kMlpOutP; e += blockDim.x) snorm[e] = a.norm[e];
    __syncthreads();
    const float* mu_in = snorm;
    const float* sd_in = snorm + kMlpInP;
    const float* mu_out = snorm + 2 * kMlpInP;
    const float* sd_out = mu_out + kMlpOutP;
    const int warp = tid >> 5, lane = tid & 31;
    for (long tile = blockIdx.x; tile * kFwdRows < a.rows; tile += gridDim.x) {
        const long row0 = tile * kFwdRows;
        for (int e = tid; e < kFwdRows * kMlpInP; e += blockDim.x) {
            const int r = e / kMlpInP, c = e % kMlpInP;
            const long gr = row0 + r;
            float v = 0.0f;
            if (gr < a.rows) {
                const long src = a.idx ? (long)a.idx[gr] : gr;
                v = (a.feat[src * kMlpInP + c] - mu_in[c]) / sd_in[c];
            }
            const bf16 bv = __float2bfloat16(v);
            sX[r * kLdIn + c] = bv;
            if (a.xn && gr < a.rows) a.xn[gr * kMlpInP + c] = bv;
        }
        __syncthreads();
        mlp_hidden<kMlpInP>(sX, sW1, sb1, sH1, a.z1, a.h1, row0, a.rows);
        __syncthreads();
        mlp_hidden<kMlpH>(sH1, sW2, sb2, sH2, a.z2, a.h2, row0, a.rows);
        __syncthreads();
        {   // output layer: m-tile warp/2, n-tile warp%2
            const int mt = warp >> 1, nt = warp & 1;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const int q = lane >> 3, r8 = lane & 7;
#pragma unroll 4
            for (int kk = 0; kk < kMlpH; kk += 16) {
                uint32_t av[4], b0, b1;
                ldsm_x4(smem_addr(sH2 + swz256(mt * 16 + (q & 1) * 8 + r8, kk + (q >> 1) * 8)), av[0], av[1],
                        av[2], av[3]);
                ldsm_x2(smem_addr(sW3 + swz256(nt * 8 + r8, kk + (q & 1) * 8)), b0, b1);
                mma_16816(acc, av, b0, b1);
            }
            const int g = lane >> 2, tq = lane & 3;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const long gr = row0 + mt * 16 + g + hh * 8;
                if (gr >= a.rows) continue;
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int c = nt * 8 + 2 * tq + cc;
                    const float ov = acc[2 * hh + cc] + sb3[c];
                    if (a.o) a.o[gr * kMlpOutP + c] = ov;
                    if (a.xout && c < a.d) {
                        // a displacement beyond 8 standard deviations of the
                        // training targets is not trusted: clamp it there
                        const float disp = fmaf(fminf(fmaxf(ov, -8.0f), 8.0f), sd_out[c], mu_out[c]);
                        a.xout[gr * a.d + c] = a.u ? a.u[gr * a.d + c] + disp : disp;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Tiled BF16 GEMM for the backward pass:
//   C[m][n] (+)= sum_k A(m,k) B(k,n),  A(m,k) = TA ? A[k lda + m] : A[m lda + k],
//   B(k,n) = B[k ldb + n]; optional epilogue factor gelu'(Z[m][n]).
// 64x64x32 tiles, 4 warps (32x32 each). gridDim.z > 1 splits K and adds into C
// with atomics (C must be zero beforehand).
// ---------------------------------------------------------------------------
template <bool TA, typename TAe, typename TBe>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const TAe* __restrict__ A, int lda,
                                                        const TBe* __restrict__ B, int ldb, float* C, int ldc,
                                                        const float* __restrict__ Z, int ldz) {
    constexpr int BM = 64, BN = 64, BK = 32, LD = BK + 8;
    __shared__ __align__(16) bf16 sA[BM * LD];
    __shared__ __align__(16) bf16 sB[BN * LD];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int kchunk = (K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    const int q = lane >> 3, r8 = lane & 7;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            int m, k;
            if (TA) { k = e / BM; m = e % BM; } else { m = e / BK; k = e % BK; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.0f;
            if (gm < M && gk < kend) v = (float)(TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk]);
            sA[m * LD + k] = __float2bfloat16(v);
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int k = e / BN, n = e % BN;
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.0f;
            if (gn < N && gk < kend) v = (float)B[(long)gk * ldb + gn];
            sB[n * LD + k] = __float2bfloat16(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm_x4(smem_addr(sA + (wm + mt * 16 + (q & 1) * 8 + r8) * LD + kk + (q >> 1) * 8), a[mt][0],
                        a[mt][1], a[mt][2], a[mt][3]);
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t b0, b1, b2, b3;
                ldsm_x4(smem_addr(sB + (wn + np * 16 + (q >> 1) * 8 + r8) * LD + kk + (q & 1) * 8), b0, b1, b2, b3);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_16816(acc[mt][2 * np], a[mt], b0, b1);
                    mma_16816(acc[mt][2 * np + 1], a[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + mt * 16 + g + (e >> 1) * 8;
                const int n = n0 + wn + nt * 8 + 2 * tq + (e & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mt][nt][e];
                if (Z) v *= gelu_grad_f(Z[(long)m * ldz + n]);
                if (gridDim.z > 1) atomicAdd(&C[(long)m * ldc + n], v);
                else C[(long)m * ldc + n] = v;
            }
}

__device__ inline float bf_to_f(bf16 v) { return __bfloat162float(v); }

// dO = 2 (o - t) / (rows d) on the real outputs, 0 on the padding; loss sum.
__global__ void mlp_loss_kernel(long rows, int d, const float* o, const float* targ, const int* idx,
                                const float* norm, float* dO, double* loss) {
    const float* mu_out = norm + 2 * kMlpInP;
    const float* sd_out = mu_out + kMlpOutP;
    const double scale = 1.0 / ((double)rows * d);
    double part = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rows * kMlpOutP; e += (long)gridDim.x * blockDim.x) {
        const long r = e / kMlpOutP;
        const int c = (int)(e % kMlpOutP);
        float g = 0.0f;
        if (c < d) {
            const long src = idx ? (long)idx[r] : r;
            const float tn = (targ[src * kMlpOutP + c] - mu_out[c]) / sd_out[c];
            const float err = o[e] - tn;
            g = (float)(2.0 * err * scale);
            part += (double)err * err * scale;
        }
        dO[e] = g;
    }
    for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// out[c] += sum_r X[r][c] (block: 32 columns x 8 row lanes).
__global__ void colsum_kernel(long rows, int cols, const float* X, int ldx, float* out) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (c < cols)
        for (long r = blockIdx.y * 8 + threadIdx.y; r < rows; r += (long)gridDim.y * 8) s += X[r * ldx + c];
    __shared__ float red[8][33];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        for (int k = 1; k < 8; ++k) s += red[k][threadIdx.x];
        atomicAdd(&out[c], s);
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master vector, then the BF16 copies.
__global__ void adam_kernel(long n, float* theta, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float c1, float c2, float eps, bf16* W1b, bf16* W2b, bf16* W3b) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float th = theta[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        theta[k] = th;
        if (k < kMlpB1) W1b[k - kMlpW1] = __float2bfloat16(th);
        else if (k >= kMlpW2 && k < kMlpB2) W2b[k - kMlpW2] = __float2bfloat16(th);
        else if (k >= kMlpW3 && k < kMlpB3) W3b[k - kMlpW3] = __float2bfloat16(th);
    }
}

__global__ void refresh_bf16_kernel(const float* theta, bf16* W1b, bf16* W2b, bf16* W3b) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < kMlpNP; k += (long)gridDim.x * blockDim.x) {
        const float th = theta[k];
        if (k < kMlpB1) W1b[k - kMlpW1] = __float2bfloat16(th);
        else if (k >= kMlpW2 && k < kMlpB2) W2b[k - kMlpW2] = __float2bfloat16(th);
        else if (k >= kMlpW3 && k < kMlpB3) W3b[k - kMlpW3] = __float2bfloat16(th);
    }
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the real entries, 0 for the padding.
__global__ void mlp_init_kernel(float* theta, int in, int out, uint64_t seed) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < kMlpNP; k += (long)gridDim.x * blockDim.x) {
        float bound = 0.0f;
        if (k < kMlpB1) bound = ((k - kMlpW1) % kMlpInP) < in ? rsqrtf((float)in) : 0.0f;
        else if (k < kMlpW2) bound = rsqrtf((float)in);
        else if (k < kMlpW3) bound = rsqrtf((float)kMlpH);
        else if (k < kMlpB3) bound = ((k - kMlpW3) / kMlpH) < out ? rsqrtf((float)kMlpH) : 0.0f;
        else bound = (k - kMlpB3) < out ? rsqrtf((float)kMlpH) : 0.0f;
        uint32_t w[4];
        philox4x32_10((uint32_t)k, (uint32_t)(k >> 32), 0x51u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
        const float u01 = ((float)(w[0] >> 8) + 0.5f) * (1.0f / 16777216.0f);
        theta[k] = bound * (2.0f * u01 - 1.0f);
    }
}

// Random minibatch rows of a step.
__global__ void gather_idx_kernel(long n_rows, int R, uint64_t seed, uint32_t step, int* idx) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        uint32_t w[4];
        philox4x32_10((uint32_t)r, step, 0xD1u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
        const uint64_t x = ((uint64_t)w[0] << 32) | w[1];
        idx[r] = (int)(x % (uint64_t)n_rows);
    }
}

// Column means and standard deviations of X [rows][ld] (first `cols` columns):
// sums in FP64.
__global__ void moments_kernel(long rows, int cols, const float* X, int ld, double* acc) {
    const int c = threadIdx.x;
    if (c >= cols) return;
    double s = 0.0, s2 = 0.0;
    for (long r = blockIdx.x; r < rows; r += gridDim.x) {
        const double v = X[r * ld + c];
        s += v;
        s2 += v * v;
    }
    atomicAdd(&acc[c], s);
    atomicAdd(&acc[cols + c], s2);
}

// ---------------------------------------------------------------------------
// Features + base particles for the learned initialisation (and the training
// capture): u = f_t(x_{t-1}^i) + Q^{1/2} xi_i exactly as the step kernels draw
// it, features of (u, z_t).
// ---------------------------------------------------------------------------
template <class M>
__global__ void proposal_rows_kernel(const __grid_constant__ ProposalRowsArgs a) {
    constexpr int D = M::D;
    // capture: one row per (b, t, i); learned initialisation: one per (b, i)
    const long total = (long)a.B * a.Nmax * (a.capture ? a.maxT : 1);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int b, t, i;
        long row;
        if (a.capture) {
            b = (int)(e / ((long)a.maxT * a.Nmax));
            const long rem = e % ((long)a.maxT * a.Nmax);
            t = (int)(rem / a.Nmax) + 1;
            i = (int)(rem % a.Nmax);
            if (t > a.Tend[b] || i >= a.Nseq[b]) continue;
            row = a.row_base[(size_t)b * a.maxT + (t - 1)] + i;
        } else {
            b = a.b_base + (int)(e / a.Nmax);
            i = (int)(e % a.Nmax);
            if (a.tcur[b] >= a.Tend[b] || i >= a.Nseq[b]) continue;
            t = a.tcur[b] + 1;
            row = e;
        }
        double xp[D], f[D];
        if (t == 1) {
#pragma unroll
            for (int c = 0; c < D; ++c) xp[c] = a.x0[(size_t)b * D + c];
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) xp[c] = (double)a.hist[(((size_t)b * a.maxT + (t - 2)) * a.Nmax + i) * D + c];
        }
        M::transition64(a.mp, M::step_const(a.mp, t), xp, f);
        float z[D], u[D];
        draw_normals<D>(a.seed, (uint32_t)b, (uint32_t)t, (uint32_t)i, z);
#pragma unroll
        for (int c = 0; c < D; ++c) u[c] = (float)(f[c] + a.mp.sqrt_q[c] * (double)z[c]);
        float ft[kMlpInP];
        const int nf = proposal_features<M>(a.mp, u, a.y + ((size_t)b * a.maxT + (t - 1)) * a.mp.dy, ft);
        float* fo = a.feat + row * kMlpInP;
        for (int c = 0; c < kMlpInP; ++c) fo[c] = c < nf ? ft[c] : 0.0f;
        if (a.u) {
#pragma unroll
            for (int c = 0; c < D; ++c) a.u[row * D + c] = u[c];
        }
        if (a.targ) {
            const float* xf = a.hist + (((size_t)b * a.maxT + (t - 1)) * a.Nmax + i) * D;
            for (int c = 0; c < kMlpOutP; ++c) a.targ[row * kMlpOutP + c] = c < D ? xf[c] - u[c] : 0.0f;
        }
    }
}

const void* proposal_rows_fn(int kind) {
    switch (kind) {
    case 1: return (const void*)proposal_rows_kernel<ModelNGM1D>;
    case 2: return (const void*)proposal_rows_kernel<ModelRangeCV>;
    case 3: return (const void*)proposal_rows_kernel<ModelClutterCV>;
    case 4: return (const void*)proposal_rows_kernel<ModelPlanarArm<7>>;
    case 5: return (const void*)proposal_rows_kernel<ModelLinearGauss>;
    case 6: return (const void*)proposal_rows_kernel<ModelRangeZV>;
    case 7: return (const void*)proposal_rows_kernel<ModelSE2RB>;
    }
    return nullptr;
}

int proposal_in_dim(int kind, int d, int dy) {
    switch (kind) {
    case 4: return d + 4 + d / 2;
    case 3: return 4 + 2 * std::min(dy / 2, (kMlpInP - 4) / 2);
    default: return 2 * d + 2 * std::min(dy, (kMlpInP - 2 * d) / 2);
    }
}

}  // namespace smap

// ---------------------------------------------------------------------------
// The proposal object.
// ---------------------------------------------------------------------------
struct smap_proposal {
    int kind = 0, d = 0, dy = 0, in = 0;
    ModelParams mp{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t seed = 0;
    int adam_t = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *norm = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr;
    double* lossd = nullptr;
    int* tcerr = nullptr;         // error word of the tensor-core forward
    // training scratch (capacity R_cap rows)
    long R_cap = 0;
    int* idx = nullptr;
    bf16 *xn = nullptr, *h1 = nullptr, *h2 = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *o = nullptr, *dO = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    std::string err;
};

namespace {

smap_status pfail(smap_proposal* p, smap_status s, const std::string& m) {
    if (p) p->err = m;
    std::fprintf(stderr, "smap_proposal: %s\n", m.c_str());
    return s;
}

#define PCUDA(p, call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return pfail((p), SMAP_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void free_scratch(smap_proposal* p) {
    void* bufs[] = {p->idx, p->xn, p->h1, p->h2, p->z1, p->z2, p->o, p->dO, p->dz2, p->dz1};
    for (void* b : bufs)
        if (b) cudaFree(b);
    p->idx = nullptr; p->xn = p->h1 = p->h2 = nullptr;
    p->z1 = p->z2 = p->o = p->dO = p->dz2 = p->dz1 = nullptr;
    p->R_cap = 0;
}

smap_status ensure_scratch(smap_proposal* p, long R) {
    if (R <= p->R_cap) return SMAP_OK;
    free_scratch(p);
    struct A { void** q; size_t bytes; } al[] = {
        {(void**)&p->idx, sizeof(int) * R}, {(void**)&p->xn, sizeof(bf16) * R * kMlpInP},
        {(void**)&p->h1, sizeof(bf16) * R * kMlpH}, {(void**)&p->h2, sizeof(bf16) * R * kMlpH},
        {(void**)&p->z1, sizeof(float) * R * kMlpH}, {(void**)&p->z2, sizeof(float) * R * kMlpH},
        {(void**)&p->o, sizeof(float) * R * kMlpOutP}, {(void**)&p->dO, sizeof(float) * R * kMlpOutP},
        {(void**)&p->dz2, sizeof(float) * R * kMlpH}, {(void**)&p->dz1, sizeof(float) * R * kMlpH},
    };
    for (auto& a : al)
        if (cudaMalloc(a.q, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_scratch(p);
            return pfail(p, SMAP_E_NOMEM, "training scratch allocation failed");
        }
    p->R_cap = R;
    return SMAP_OK;
}

int grid_for(long n, int block) { return (int)std::min<long>((n + block - 1) / block, 152L * 16); }

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

// Inference (no training outputs, no gather) runs on the tcgen05 kernel;
// training passes keep the mma.sync kernel, which also writes the layer
// activations that the backward pass reads.
smap_status launch_forward(smap_proposal* p, const float* feat, const int* idx, long rows, bool train,
                           const float* u, float* xout, cudaStream_t st, int* err = nullptr,
                           uint64_t wait_ns = kTcWaitNs, int stall = 0) {
    if (!train && !idx && xout) {
        MlpTcArgs t;
        t.W1 = p->W1b; t.W2 = p->W2b; t.W3 = p->W3b;
        t.b1 = p->theta + kMlpB1; t.b2 = p->theta + kMlpB2; t.b3 = p->theta + kMlpB3;
        t.norm = p->norm;
        t.rows = rows;
        t.d = p->d;
        t.feat = feat;
        t.u = u;
        t.xout = xout;
        t.err = err ? err : p->tcerr;
        t.wait_ns = wait_ns;
        t.stall = stall;
        PCUDA(p, mlp_forward_tc_launch(t, num_sms(), st));
        g_launches.fetch_add(1);
        return SMAP_OK;
    }
    PCUDA(p, ensure_dynamic_smem((const void*)mlp_forward_kernel, mlp_fwd_smem()));
    MlpFwdArgs a;
    memset(&a, 0, sizeof(a));
    a.W1 = p->W1b; a.W2 = p->W2b; a.W3 = p->W3b;
    a.b1 = p->theta + kMlpB1; a.b2 = p->theta + kMlpB2; a.b3 = p->theta + kMlpB3;
    a.norm = p->norm;
    a.rows = rows;
    a.d = p->d;
    a.feat = feat;
    a.idx = idx;
    if (train) {
        a.xn = p->xn; a.z1 = p->z1; a.h1 = p->h1; a.z2 = p->z2; a.h2 = p->h2; a.o = p->o;
    }
    a.u = u;
    a.xout = xout;
    const long tiles = (rows + kFwdRows - 1) / kFwdRows;
    const int grid = (int)std::max<long>(1, std::min<long>(tiles, num_sms()));
    mlp_forward_kernel<<<grid, 256, mlp_fwd_smem(), st>>>(a);
    PCUDA(p, cudaGetLastError());
    g_launches.fetch_add(1);
    return SMAP_OK;
}

template <bool TA, typename TAe, typename TBe>
smap_status gemm(smap_proposal* p, int M, int N, int K, const TAe* A, int lda, const TBe* B, int ldb, float* C,
                 int ldc, const float* Z, int ldz, int splitk, cudaStream_t st) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, splitk);
    gemm_bf16_kernel<TA, TAe, TBe><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, Z, ldz);
    PCUDA(p, cudaGetLastError());
    g_launches.fetch_add(1);
    return SMAP_OK;
}

// Forward + backward over R rows (gathered by idx when given): gradient into p->grad, loss into p->lossd.
smap_status loss_and_grad(smap_proposal* p, const float* feat, const float* targ, const int* idx, long R) {
    cudaStream_t st = p->stream;
    smap_status s = launch_forward(p, feat, idx, R, true, nullptr, nullptr, st);
    if (s) return s;
    PCUDA(p, cudaMemsetAsync(p->lossd, 0, sizeof(double), st));
    PCUDA(p, cudaMemsetAsync(p->grad, 0, sizeof(float) * kMlpNP, st));
    mlp_loss_kernel<<<grid_for(R * kMlpOutP, 256), 256, 0, st>>>(R, p->d, p->o, targ, idx, p->norm, p->dO, p->lossd);
    g_launches.fetch_add(1);
    // dz2 = (dO W3) * gelu'(z2); dz1 = (dz2 W2) * gelu'(z1)
    if ((s = gemm<false, float, bf16>(p, (int)R, kMlpH, kMlpOutP, p->dO, kMlpOutP, p->W3b, kMlpH, p->dz2, kMlpH, p->z2,
                                      kMlpH, 1, st)))
        return s;
    if ((s = gemm<false, float, bf16>(p, (int)R, kMlpH, kMlpH, p->dz2, kMlpH, p->W2b, kMlpH, p->dz1, kMlpH, p->z1,
                                      kMlpH, 1, st)))
        return s;
    // weight gradients: dW3 = dO^T h2, dW2 = dz2^T h1, dW1 = dz1^T xn (split over the rows)
    const int split = (int)std::max<long>(1, std::min<long>(32, R / 512));
    if ((s = gemm<true, float, bf16>(p, kMlpOutP, kMlpH, (int)R, p->dO, kMlpOutP, p->h2, kMlpH, p->grad + kMlpW3, kMlpH,
                                     nullptr, 0, split, st)))
        return s;
    if ((s = gemm<true, float, bf16>(p, kMlpH, kMlpH, (int)R, p->dz2, kMlpH, p->h1, kMlpH, p->grad + kMlpW2, kMlpH,
                                     nullptr, 0, split, st)))
        return s;
    if ((s = gemm<true, float, bf16>(p, kMlpH, kMlpInP, (int)R, p->dz1, kMlpH, p->xn, kMlpInP, p->grad + kMlpW1, kMlpInP,
                                     nullptr, 0, split, st)))
        return s;
    dim3 cb(32, 8);
    const int gy = (int)std::min<long>(64, (R + 7) / 8);
    colsum_kernel<<<dim3((kMlpOutP + 31) / 32, gy), cb, 0, st>>>(R, kMlpOutP, p->dO, kMlpOutP, p->grad + kMlpB3);
    colsum_kernel<<<dim3((kMlpH + 31) / 32, gy), cb, 0, st>>>(R, kMlpH, p->dz2, kMlpH, p->grad + kMlpB2);
    colsum_kernel<<<dim3((kMlpH + 31) / 32, gy), cb, 0, st>>>(R, kMlpH, p->dz1, kMlpH, p->grad + kMlpB1);
    g_launches.fetch_add(3);
    PCUDA(p, cudaGetLastError());
    return SMAP_OK;
}

}  // namespace

namespace smap {

smap_status proposal_launch_init(smap_proposal* p, const ProposalRowsArgs& ra, float* xinit, cudaStream_t st) {
    const void* fn = proposal_rows_fn(p->kind);
    if (!fn) return pfail(p, SMAP_E_INVAL, "model has no proposal features");
    const long total = (long)ra.B * ra.Nmax;
    void* args[] = {const_cast<ProposalRowsArgs*>(&ra)};
    PCUDA(p, cudaLaunchKernel(fn, dim3(grid_for(total, 256)), dim3(256), args, 0, st));
    g_launches.fetch_add(1);
    return launch_forward(p, ra.feat, nullptr, total, false, ra.u, xinit, st, ra.err);
}

smap_status proposal_launch_capture(smap_proposal* p, const ProposalRowsArgs& ra, cudaStream_t st) {
    const void* fn = proposal_rows_fn(p->kind);
    if (!fn) return pfail(p, SMAP_E_INVAL, "model has no proposal features");
    const long total = (long)ra.B * ra.Nmax * ra.maxT;
    void* args[] = {const_cast<ProposalRowsArgs*>(&ra)};
    PCUDA(p, cudaLaunchKernel(fn, dim3(grid_for(total, 256)), dim3(256), args, 0, st));
    g_launches.fetch_add(1);
    return SMAP_OK;
}

int proposal_kind(const smap_proposal* p) { return p->kind; }
int proposal_d(const smap_proposal* p) { return p->d; }

}  // namespace smap

extern "C" {

smap_status smap_proposal_create(int model, const double* params, int n_params, uint64_t seed, void* stream,
                                 smap_proposal** out) {
    if (!out) return SMAP_E_INVAL;
    *out = nullptr;
    smap_proposal* p = new smap_proposal();
    std::string err;
    if (!make_model(model, params, n_params, p->mp, err)) {
        delete p;
        std::fprintf(stderr, "smap_proposal_create: %s\n", err.c_str());
        return SMAP_E_INVAL;
    }
    p->kind = model;
    p->d = p->mp.d;
    p->dy = p->mp.dy;
    p->in = proposal_in_dim(model, p->d, p->dy);
    p->seed = seed;
    if (p->d > kMlpOutP || p->in > kMlpInP) {
        delete p;
        return SMAP_E_UNSUPPORTED;
    }
    auto bail = [&](smap_status s) { smap_proposal_destroy(p); return s; };
    if (stream) p->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreate(&p->stream) != cudaSuccess) return bail(SMAP_E_CUDA);
        p->own_stream = true;
    }
    struct A { void** q; size_t bytes; } al[] = {
        {(void**)&p->theta, sizeof(float) * kMlpNP}, {(void**)&p->m, sizeof(float) * kMlpNP},
        {(void**)&p->v, sizeof(float) * kMlpNP}, {(void**)&p->grad, sizeof(float) * kMlpNP},
        {(void**)&p->norm, sizeof(float) * (2 * kMlpInP + 2 * kMlpOutP)},
        {(void**)&p->W1b, sizeof(bf16) * kMlpH * kMlpInP}, {(void**)&p->W2b, sizeof(bf16) * kMlpH * kMlpH},
        {(void**)&p->W3b, sizeof(bf16) * kMlpOutP * kMlpH}, {(void**)&p->lossd, sizeof(double) * 4}, {(void**)&p->tcerr, sizeof(int)},
    };
    for (auto& a : al)
        if (cudaMalloc(a.q, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(SMAP_E_NOMEM);
        }
    cudaMemsetAsync(p->m, 0, sizeof(float) * kMlpNP, p->stream);
    cudaMemsetAsync(p->tcerr, 0, sizeof(int), p->stream);
    cudaMemsetAsync(p->v, 0, sizeof(float) * kMlpNP, p->stream);
    std::vector<float> norm(2 * kMlpInP + 2 * kMlpOutP, 0.0f);
    for (int c = 0; c < kMlpInP; ++c) norm[kMlpInP + c] = 1.0f;
    for (int c = 0; c < kMlpOutP; ++c) norm[2 * kMlpInP + kMlpOutP + c] = 1.0f;
    cudaMemcpy(p->norm, norm.data(), sizeof(float) * norm.size(), cudaMemcpyHostToDevice);
    mlp_init_kernel<<<64, 256, 0, p->stream>>>(p->theta, p->in, p->d, seed);
    refresh_bf16_kernel<<<64, 256, 0, p->stream>>>(p->theta, p->W1b, p->W2b, p->W3b);
    g_launches.fetch_add(2);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return bail(SMAP_E_CUDA);
    *out = p;
    return SMAP_OK;
}

void smap_proposal_destroy(smap_proposal* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    free_scratch(p);
    void* bufs[] = {p->theta, p->m, p->v, p->grad, p->norm, p->W1b, p->W2b, p->W3b, p->lossd, p->tcerr};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

smap_status smap_proposal_dims(const smap_proposal* p, int* in, int* out, int* hidden, long* n_params) {
    if (!p) return SMAP_E_INVAL;
    if (in) *in = p->in;
    if (out) *out = p->d;
    if (hidden) *hidden = kMlpH;
    if (n_params) *n_params = kMlpNP;
    return SMAP_OK;
}

smap_status smap_proposal_get_weights(smap_proposal* p, float* theta, float* norm) {
    if (!p) return SMAP_E_INVAL;
    if (theta) PCUDA(p, cudaMemcpyAsync(theta, p->theta, sizeof(float) * kMlpNP, cudaMemcpyDeviceToHost, p->stream));
    if (norm)
        PCUDA(p, cudaMemcpyAsync(norm, p->norm, sizeof(float) * (2 * kMlpInP + 2 * kMlpOutP), cudaMemcpyDeviceToHost,
                                 p->stream));
    PCUDA(p, cudaStreamSynchronize(p->stream));
    return SMAP_OK;
}

smap_status smap_proposal_set_weights(smap_proposal* p, const float* theta, const float* norm) {
    if (!p) return SMAP_E_INVAL;
    if (norm) {
        for (int c = 0; c < kMlpInP; ++c)
            if (!(norm[kMlpInP + c] > 0.0f)) return pfail(p, SMAP_E_INVAL, "input scales must be > 0");
        for (int c = 0; c < kMlpOutP; ++c)
            if (!(norm[2 * kMlpInP + kMlpOutP + c] > 0.0f)) return pfail(p, SMAP_E_INVAL, "output scales must be > 0");
        PCUDA(p, cudaMemcpyAsync(p->norm, norm, sizeof(float) * (2 * kMlpInP + 2 * kMlpOutP), cudaMemcpyHostToDevice,
                                 p->stream));
    }
    if (theta) {
        PCUDA(p, cudaMemcpyAsync(p->theta, theta, sizeof(float) * kMlpNP, cudaMemcpyHostToDevice, p->stream));
        refresh_bf16_kernel<<<64, 256, 0, p->stream>>>(p->theta, p->W1b, p->W2b, p->W3b);
        g_launches.fetch_add(1);
    }
    PCUDA(p, cudaStreamSynchronize(p->stream));
    return SMAP_OK;
}

smap_status smap_proposal_fit_normalization(smap_proposal* p, const float* feat, const float* targ, long rows) {
    if (!p || !feat || !targ || rows < 2) return SMAP_E_INVAL;
    double* acc = nullptr;
    PCUDA(p, cudaMalloc(&acc, sizeof(double) * 2 * (kMlpInP + kMlpOutP)));
    cudaMemsetAsync(acc, 0, sizeof(double) * 2 * (kMlpInP + kMlpOutP), p->stream);
    const int g = (int)std::min<long>(rows, 4096);
    moments_kernel<<<g, 32, 0, p->stream>>>(rows, kMlpInP, feat, kMlpInP, acc);
    moments_kernel<<<g, 32, 0, p->stream>>>(rows, kMlpOutP, targ, kMlpOutP, acc + 2 * kMlpInP);
    g_launches.fetch_add(2);
    std::vector<double> h(2 * (kMlpInP + kMlpOutP));
    cudaError_t e = cudaMemcpyAsync(h.data(), acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(acc);
    if (e != cudaSuccess) return pfail(p, SMAP_E_CUDA, cudaGetErrorString(e));
    std::vector<float> norm(2 * kMlpInP + 2 * kMlpOutP);
    for (int c = 0; c < kMlpInP; ++c) {
        const double mu = h[c] / rows, var = h[kMlpInP + c] / rows - mu * mu;
        norm[c] = (float)mu;
        norm[kMlpInP + c] = (float)(var > 1e-12 ? std::sqrt(var) : 1.0);
    }
    // Output scales: each target column's spread, floored at 1% of the widest
    // one, so that coordinates that barely move (noise-level displacements)
    // do not weigh as much in the loss as the ones that carry the update.
    double widest = 0.0;
    for (int c = 0; c < p->d; ++c) {
        const double mu = h[2 * kMlpInP + c] / rows, var = h[2 * kMlpInP + kMlpOutP + c] / rows - mu * mu;
        widest = std::max(widest, var > 0.0 ? std::sqrt(var) : 0.0);
    }
    for (int c = 0; c < kMlpOutP; ++c) {
        const double mu = h[2 * kMlpInP + c] / rows, var = h[2 * kMlpInP + kMlpOutP + c] / rows - mu * mu;
        const double sd = std::max(var > 0.0 ? std::sqrt(var) : 0.0, 1e-2 * widest);
        norm[2 * kMlpInP + c] = (float)mu;
        norm[2 * kMlpInP + kMlpOutP + c] = (float)(c < p->d && sd > 1e-10 ? sd : 1.0);
    }
    return smap_proposal_set_weights(p, nullptr, norm.data());
}

static smap_status forward_checked(smap_proposal* p, const float* feat, long rows, float* disp, uint64_t wait_ns,
                                   int stall) {
    NvtxRange nvtx_("smap_proposal_forward");
    if (!p || !feat || !disp || rows < 1) return SMAP_E_INVAL;
    smap_status s = launch_forward(p, feat, nullptr, rows, false, nullptr, disp, p->stream, nullptr, wait_ns, stall);
    if (s) return s;
    int err = 0;
    PCUDA(p, cudaMemcpyAsync(&err, p->tcerr, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PCUDA(p, cudaStreamSynchronize(p->stream));
    if (err) {
        PCUDA(p, cudaMemsetAsync(p->tcerr, 0, sizeof(int), p->stream));
        PCUDA(p, cudaStreamSynchronize(p->stream));
        return pfail(p, SMAP_E_TIMEOUT, "tensor-core forward: a bounded wait ran out (results not written)");
    }
    return SMAP_OK;
}

smap_status smap_proposal_forward(smap_proposal* p, const float* feat, long rows, float* disp) {
    return forward_checked(p, feat, rows, disp, kTcWaitNs, 0);
}

smap_status smap_debug_proposal_forward(smap_proposal* p, const float* feat, long rows, float* disp,
                                        uint64_t wait_ns, int stall) {
    return forward_checked(p, feat, rows, disp, wait_ns, stall);
}

smap_status smap_proposal_loss_grad(smap_proposal* p, const float* feat, const float* targ, long rows, float* grad,
                                    double* loss) {
    if (!p || !feat || !targ || rows < 1) return SMAP_E_INVAL;
    smap_status s = ensure_scratch(p, rows);
    if (s) return s;
    if ((s = loss_and_grad(p, feat, targ, nullptr, rows))) return s;
    if (grad) PCUDA(p, cudaMemcpyAsync(grad, p->grad, sizeof(float) * kMlpNP, cudaMemcpyDeviceToHost, p->stream));
    if (loss) PCUDA(p, cudaMemcpyAsync(loss, p->lossd, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PCUDA(p, cudaStreamSynchronize(p->stream));
    return SMAP_OK;
}

smap_status smap_proposal_train(smap_proposal* p, const float* feat, const float* targ, long n_rows, int steps,
                                int batch, double lr, double lr_final, float* loss_curve) {
    NvtxRange nvtx_("smap_proposal_train");
    if (!p || !feat || !targ || n_rows < 1 || steps < 0 || batch < 1) return SMAP_E_INVAL;
    smap_status s = ensure_scratch(p, batch);
    if (s) return s;
    std::vector<double> losses;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int k = 0; k < steps; ++k) {
        gather_idx_kernel<<<grid_for(batch, 256), 256, 0, p->stream>>>(n_rows, batch, p->seed, (uint32_t)(p->adam_t + 1),
                                                                       p->idx);
        g_launches.fetch_add(1);
        if ((s = loss_and_grad(p, feat, targ, p->idx, batch))) return s;
        ++p->adam_t;
        // cosine decay from lr to lr_final over the call
        const double frac = steps > 1 ? (double)k / (steps - 1) : 0.0;
        const double lrk = lr_final + 0.5 * (lr - lr_final) * (1.0 + std::cos(3.141592653589793 * frac));
        const float c1 = (float)(1.0 - std::pow((double)b1, p->adam_t));
        const float c2 = (float)(1.0 - std::pow((double)b2, p->adam_t));
        adam_kernel<<<grid_for(kMlpNP, 256), 256, 0, p->stream>>>(kMlpNP, p->theta, p->grad, p->m, p->v, (float)lrk, b1,
                                                                 b2, c1, c2, 1e-8f, p->W1b, p->W2b, p->W3b);
        g_launches.fetch_add(1);
        PCUDA(p, cudaGetLastError());
        if (loss_curve) {
            double l = 0.0;
            PCUDA(p, cudaMemcpyAsync(&l, p->lossd, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
            PCUDA(p, cudaStreamSynchronize(p->stream));
            loss_curve[k] = (float)l;
        }
    }
    PCUDA(p, cudaStreamSynchronize(p->stream));
    return SMAP_OK;
}

const char* smap_proposal_last_error(const smap_proposal* p) { return p ? p->err.c_str() : "null proposal"; }

}  // extern "C"
