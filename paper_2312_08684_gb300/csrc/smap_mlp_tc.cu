// smap_mlp_tc.cu -- inference forward of the learned proposal on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// One persistent CTA per SM, 288 threads:
//   warps 0-7  epilogue: standardise the feature tile into shared memory,
//              read accumulators from TMEM (tcgen05.ld), add the bias, GELU,
//              write BF16 activations back as the next layer's A operand,
//              and finally the output displacement;
//   warp 8     issues the MMAs (one elected lane) and commits them to an
//              mbarrier.
// Per 128-row tile:
//   L1  X[128x32]  . W1^T -> D1 = TMEM columns   0..255   (2 MMAs, K = 16 each)
//   L2  H1[128x256] . W2^T -> D2 = TMEM columns 256..511  (16 MMAs)
//   L3  H2[128x256] . W3^T -> D3 = TMEM columns   0..15   (16 MMAs, N = 16)
// The hidden activations are written in four 64-column panels; each panel has
// its own mbarrier so the MMA warp starts the next layer on a panel as soon
// as its 128 rows are in shared memory, overlapping the GELU epilogue with
// the tensor cores. Every wait is bounded (about 2 s); a wait that gives up
// sets *err and the CTA leaves its loop, frees its tensor memory and returns.
//
// Shared memory (offsets from a 1024-byte aligned base):
//   W2  4 panels x [256 rows][128 B], SW128        131072 B
//   H   4 panels x [128 rows][128 B], SW128         65536 B  (X tile [128][64 B], SW64, aliased at its start)
//   W1  [256 rows][64 B], SW64                      16384 B
//   W3  4 panels x [16 rows][128 B], SW128           8192 B
//   b1, b2, b3, normalisation, mbarriers, TMEM address
#include <cuda_bf16.h>

#include "smap_mlp.cuh"
#include "smap_tc.cuh"

namespace smap {

namespace {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 288;
constexpr uint32_t kOffW2 = 0;
constexpr uint32_t kOffH = 131072;
constexpr uint32_t kOffW1 = 196608;
constexpr uint32_t kOffW3 = 212992;
constexpr uint32_t kOffB1 = 221184;
constexpr uint32_t kOffB2 = kOffB1 + 4 * kMlpH;
constexpr uint32_t kOffB3 = kOffB2 + 4 * kMlpH;
constexpr uint32_t kOffNorm = kOffB3 + 4 * kMlpOutP;
constexpr uint32_t kOffBar = kOffNorm + 4 * (2 * kMlpInP + 2 * kMlpOutP);
constexpr uint32_t kOffTmem = kOffBar + 64;
constexpr uint32_t kTcSmemUsed = kOffTmem + 16;
constexpr uint32_t kTcSmem = kTcSmemUsed + 1024;   // slack for aligning the base
constexpr uint32_t kPanelH = kTcRows * 128;         // bytes of one activation panel
constexpr uint32_t kPanelW2 = kMlpH * 128;
constexpr uint32_t kPanelW3 = kMlpOutP * 128;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kIdescN256 = tc::idesc_bf16_f32(128, 256);
constexpr uint32_t kIdescN16 = tc::idesc_bf16_f32(128, 16);

static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");
static_assert(kTcSmem <= 232448, "shared memory above the per-CTA limit");
static_assert(kOffH % 1024 == 0 && kOffW1 % 1024 == 0 && kOffW3 % 1024 == 0, "operand regions need 1024-byte alignment");

// Bias + GELU on 32 accumulator columns of this thread's row, BF16 into the
// row's 64-byte slice of an SW128 panel; arrival on the panel's mbarrier once
// the warp's two slices of that panel are written.
__device__ __forceinline__ void hidden_epilogue(uint32_t tl, const float* bias, int ch, int row, unsigned char* H,
                                                uint64_t* bar_panel) {
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const int c0 = 128 * ch + 32 * j;
        uint32_t r[32];
        tc::tmem_ld32(tl + (uint32_t)c0, r);
        tc::wait_ld();
        uint32_t pk[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float z0 = __uint_as_float(r[2 * e]) + bias[c0 + 2 * e];
            const float z1 = __uint_as_float(r[2 * e + 1]) + bias[c0 + 2 * e + 1];
            __nv_bfloat162 h = __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
            pk[e] = *reinterpret_cast<uint32_t*>(&h);
        }
        const int p = c0 >> 6, cb = (c0 & 63) >> 3;
        unsigned char* rowp = H + p * kPanelH + row * 128;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4*>(rowp + (((cb + k) ^ (row & 7)) << 4)) =
                make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
        if (j & 1) {
            tc::fence_async_smem();
            tc::fence_before_sync();
            tc::mbar_arrive(bar_panel + p);
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_forward_tc_kernel(const __grid_constant__ MlpTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t raw_s = tc::saddr(smraw);
    unsigned char* sm = smraw + ((1024u - (raw_s & 1023u)) & 1023u);
    const uint32_t sb = tc::saddr(sm);
    float* sb1 = reinterpret_cast<float*>(sm + kOffB1);
    float* sb2 = reinterpret_cast<float*>(sm + kOffB2);
    float* sb3 = reinterpret_cast<float*>(sm + kOffB3);
    float* snorm = reinterpret_cast<float*>(sm + kOffNorm);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* bar_x = bar_mma + 1;
    uint64_t* bar_panel = bar_mma + 2;   // [4]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffTmem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- weights into the swizzled operand layouts -----------------------
    const uint4* gW2 = reinterpret_cast<const uint4*>(a.W2);
    for (int e = tid; e < kMlpH * (kMlpH / 8); e += kTcThreads) {
        const int n = e >> 5, kc = e & 31;
        *reinterpret_cast<uint4*>(sm + kOffW2 + (kc >> 3) * kPanelW2 + n * 128 + (((kc & 7) ^ (n & 7)) << 4)) = gW2[e];
    }
    const uint4* gW3 = reinterpret_cast<const uint4*>(a.W3);
    for (int e = tid; e < kMlpOutP * (kMlpH / 8); e += kTcThreads) {
        const int n = e >> 5, kc = e & 31;
        *reinterpret_cast<uint4*>(sm + kOffW3 + (kc >> 3) * kPanelW3 + n * 128 + (((kc & 7) ^ (n & 7)) << 4)) = gW3[e];
    }
    const uint4* gW1 = reinterpret_cast<const uint4*>(a.W1);
    for (int e = tid; e < kMlpH * (kMlpInP / 8); e += kTcThreads) {
        const int n = e >> 2, c = e & 3;
        *reinterpret_cast<uint4*>(sm + kOffW1 + n * 64 + ((c ^ ((n >> 1) & 3)) << 4)) = gW1[e];
    }
    for (int e = tid; e < kMlpH; e += kTcThreads) { sb1[e] = a.b1[e]; sb2[e] = a.b2[e]; }
    for (int e = tid; e < kMlpOutP; e += kTcThreads) sb3[e] = a.b3[e];
    for (int e = tid; e < 2 * kMlpInP + 2 * kMlpOutP; e += kTcThreads) snorm[e] = a.norm[e];
    if (tid == 0) {
        tc::mbar_init(bar_mma, 1);
        tc::mbar_init(bar_x, 256);
        for (int p = 0; p < 4; ++p) tc::mbar_init(bar_panel + p, 128);
        tc::mbar_init_fence();
    }
    if (warp == 8) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    const long ntiles = (a.rows + kTcRows - 1) / kTcRows;
    bool ok = true;
    uint32_t it = 0;
    if (warp < 8) {
        // ---------------- epilogue warps ----------------
        const int q = warp & 3, ch = warp >> 2;
        const int erow = 32 * q + lane;                               // row of the tile = TMEM lane
        const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16);
        const int xr = tid >> 1, xh = tid & 1;                        // feature loader: row, half
        const float* mu_in = snorm;
        const float* sd_in = snorm + kMlpInP;
        const float* mu_out = snorm + 2 * kMlpInP;
        const float* sd_out = mu_out + kMlpOutP;
        float4 pf[4];
        auto load_feat = [&](long tile) {
            const long gr = tile * kTcRows + xr;
            if (gr < a.rows) {
                const float4* src = reinterpret_cast<const float4*>(a.feat + gr * kMlpInP + 16 * xh);
#pragma unroll
                for (int k = 0; k < 4; ++k) pf[k] = __ldg(src + k);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) pf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        long tile = blockIdx.x;
        if (tile < ntiles) load_feat(tile);
        for (; tile < ntiles; tile += gridDim.x, ++it) {
            // X tile: standardised, BF16, SW64 rows (zero rows past the end)
            {
                const long gr = tile * kTcRows + xr;
                const float* v = reinterpret_cast<const float*>(pf);
                uint32_t pk[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int c = 16 * xh + 2 * e;
                    float x0 = 0.0f, x1 = 0.0f;
                    if (gr < a.rows) {
                        x0 = (v[2 * e] - mu_in[c]) / sd_in[c];
                        x1 = (v[2 * e + 1] - mu_in[c + 1]) / sd_in[c + 1];
                    }
                    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                    pk[e] = *reinterpret_cast<uint32_t*>(&h);
                }
                unsigned char* rowp = sm + kOffH + xr * 64;
                const int sw = (xr >> 1) & 3;
                *reinterpret_cast<uint4*>(rowp + (((2 * xh) ^ sw) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(rowp + (((2 * xh + 1) ^ sw) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            tc::fence_async_smem();
            tc::mbar_arrive(bar_x);
            if (tile + gridDim.x < ntiles) load_feat(tile + gridDim.x);   // in flight during this tile
            const long orow = tile * kTcRows + erow;
            float uu[kMlpOutP];
#pragma unroll
            for (int c = 0; c < kMlpOutP; ++c) uu[c] = 0.0f;
            if (warp < 4 && a.u && orow < a.rows) {
#pragma unroll
                for (int c = 0; c < kMlpOutP; ++c)
                    if (c < a.d) uu[c] = __ldg(a.u + orow * a.d + c);
            }
            // layer 1 -> GELU -> H1
            if (!tc::warp_wait(bar_mma, (3 * it) & 1, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            hidden_epilogue(tl, sb1, ch, erow, sm + kOffH, bar_panel);
            // layer 2 -> GELU -> H2
            if (!tc::warp_wait(bar_mma, (3 * it + 1) & 1, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            hidden_epilogue(tl + 256, sb2, ch, erow, sm + kOffH, bar_panel);
            // layer 3 -> output
            if (!tc::warp_wait(bar_mma, (3 * it + 2) & 1, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            if (warp < 4) {
                uint32_t r[16];
                tc::tmem_ld16(tl, r);
                tc::wait_ld();
                if (orow < a.rows) {
#pragma unroll
                    for (int c = 0; c < kMlpOutP; ++c) {
                        if (c < a.d) {
                            // a displacement beyond 8 standard deviations of the
                            // training targets is not trusted: clamp it there
                            const float ov = __uint_as_float(r[c]) + sb3[c];
                            const float disp = fmaf(fminf(fmaxf(ov, -8.0f), 8.0f), sd_out[c], mu_out[c]);
                            a.xout[orow * a.d + c] = uu[c] + disp;
                        }
                    }
                }
            }
            tc::fence_before_sync();
        }
    } else {
        // ---------------- MMA warp ----------------
        const uint32_t dX = sb + kOffH, dW1 = sb + kOffW1, dH = sb + kOffH, dW2 = sb + kOffW2, dW3 = sb + kOffW3;
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            if (!tc::warp_wait(bar_x, it & 1, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            if (lane == 0) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    tc::mma_bf16(tbase, tc::smem_desc(dX + 32 * ks, 512, tc::kSwizzle64),
                                 tc::smem_desc(dW1 + 32 * ks, 512, tc::kSwizzle64), kIdescN256, ks);
                tc::mma_commit(bar_mma);
            }
            __syncwarp();
            // layer 2, panel by panel as the epilogue writes them (0 and 2 come first)
#pragma unroll 1
            for (int j = 0; j < 4 && ok; ++j) {
                const int p = ((j & 1) << 1) | (j >> 1);
                if (!tc::warp_wait(bar_panel + p, 0, kWaitNs)) { ok = false; break; }
                tc::fence_after_sync();
                if (lane == 0) {
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc::mma_bf16(tbase + 256, tc::smem_desc(dH + p * kPanelH + 32 * ks, 1024, tc::kSwizzle128),
                                     tc::smem_desc(dW2 + p * kPanelW2 + 32 * ks, 1024, tc::kSwizzle128), kIdescN256,
                                     (j | ks) != 0);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) tc::mma_commit(bar_mma);
            __syncwarp();
#pragma unroll 1
            for (int j = 0; j < 4 && ok; ++j) {
                const int p = ((j & 1) << 1) | (j >> 1);
                if (!tc::warp_wait(bar_panel + p, 1, kWaitNs)) { ok = false; break; }
                tc::fence_after_sync();
                if (lane == 0) {
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc::mma_bf16(tbase, tc::smem_desc(dH + p * kPanelH + 32 * ks, 1024, tc::kSwizzle128),
                                     tc::smem_desc(dW3 + p * kPanelW3 + 32 * ks, 1024, tc::kSwizzle128), kIdescN16,
                                     (j | ks) != 0);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) tc::mma_commit(bar_mma);
            __syncwarp();
        }
    }
    if (!ok && lane == 0 && a.err) atomicExch(a.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 8) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

}  // namespace

size_t mlp_forward_tc_smem() { return kTcSmem; }

cudaError_t mlp_forward_tc_launch(const MlpTcArgs& a, int num_sms, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long tiles = (a.rows + kTcRows - 1) / kTcRows;
    const int grid = (int)(tiles < num_sms ? (tiles > 0 ? tiles : 1) : num_sms);
    mlp_forward_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace smap
