// smap_mlp_tc.cu -- inference forward of the learned proposal on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// One persistent CTA per SM, 544 threads:
//   warps 0-15 epilogue: standardise the feature tile into shared memory,
//              read accumulators from TMEM (tcgen05.ld), add the bias, GELU,
//              write BF16 activations back as the next layer's A operand,
//              and finally the output displacement. Warp w reads TMEM lanes
//              32 (w % 4) .. +31 (the tile's rows) and owns hidden columns
//              64 (w / 4) .. +63, i.e. one 64-column activation panel;
//   warp 16    issues the MMAs (one elected lane) and commits them to
//              mbarriers.
// Per 128-row tile:
//   L1  X[128x32]  . W1^T -> D1 = TMEM columns   0..255   (2 x 2 MMAs, N = 128, K = 16)
//   L2  H1[128x256] . W2^T -> D2 = TMEM columns 256..511  (2 x 16 MMAs, N = 128)
//   L3  H2[128x256] . W3^T -> D3 = TMEM columns 256..271  (16 MMAs, N = 16)
// Layers 1 and 2 are issued as two 128-column output halves with separate
// commits. The hidden activations are signalled in four K quarters (columns
// 16 j .. 16 j + 15 of every panel), so the MMA warp runs the next layer's K
// steps while the GELU epilogue writes the following quarters. The next
// tile's X goes into shared memory as soon as layer 3 completed, so its layer
// 1 overlaps this tile's output epilogue. Every wait is bounded (a.wait_ns,
// 2 s by default); a wait that gives up sets *err and the CTA leaves its loop,
// waits (bounded) for the MMAs it already issued to complete, frees its
// tensor memory and returns.
//
// Shared memory (offsets from a 1024-byte aligned base):
//   W2  4 panels x [256 rows][128 B], SW128        131072 B
//   H   4 panels x [128 rows][128 B], SW128         65536 B  (X tile [128][64 B], SW64, aliased at panel 2)
//   W1  [256 rows][64 B], SW64                      16384 B
//   W3  4 panels x [16 rows][128 B], SW128           8192 B
//   b1, b2, b3, normalisation, mbarriers, TMEM address
#include <cuda_bf16.h>

#include "smap_internal.h"
#include "smap_mlp.cuh"
#include "smap_tc.cuh"

namespace smap {

namespace {

constexpr int kTcRows = 128;
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kTcThreads = kEpiThreads + 32;
constexpr uint32_t kOffW2 = 0;
constexpr uint32_t kOffH = 131072;
constexpr uint32_t kOffW1 = 196608;
constexpr uint32_t kOffW3 = 212992;
constexpr uint32_t kOffB1 = 221184;
constexpr uint32_t kOffB2 = kOffB1 + 4 * kMlpH;
constexpr uint32_t kOffB3 = kOffB2 + 4 * kMlpH;
constexpr uint32_t kOffNorm = kOffB3 + 4 * kMlpOutP;
constexpr uint32_t kOffInvSd = kOffNorm + 4 * (2 * kMlpInP + 2 * kMlpOutP);   // 1 / sd_in
constexpr uint32_t kOffBar = kOffInvSd + 4 * kMlpInP;
constexpr int kNumBars = 12;
constexpr uint32_t kOffTmem = kOffBar + 8 * kNumBars;
constexpr uint32_t kTcSmemUsed = kOffTmem + 16;
constexpr uint32_t kTcSmem = kTcSmemUsed + 1024;   // slack for aligning the base
constexpr uint32_t kPanelH = kTcRows * 128;         // bytes of one activation panel
// The X tile shares the activation region's third panel: that panel is first
// rewritten by the warps of columns 128..191 after the second layer-1 half
// (the last reader of X) completed, and X is rewritten only after layer 3 of
// the previous tile.
constexpr uint32_t kOffX = kOffH + 2 * kPanelH;
constexpr uint32_t kPanelW2 = kMlpH * 128;
constexpr uint32_t kPanelW3 = kMlpOutP * 128;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdescN128 = tc::idesc_bf16_f32(128, 128);
constexpr uint32_t kIdescN16 = tc::idesc_bf16_f32(128, 16);

static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");
static_assert(kTcSmem <= 232448, "shared memory above the per-CTA limit");
static_assert(kOffH % 1024 == 0 && kOffW1 % 1024 == 0 && kOffW3 % 1024 == 0 && kOffX % 1024 == 0,
              "operand regions need 1024-byte alignment");

// Eight BF16 values times 1/2 (exact: products of BF16 by 1/2 are BF16 unless
// they fall below the normal range, where round-to-nearest applies).
__device__ __forceinline__ uint4 half_bf16x8(uint4 v) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(0.5f, 0.5f);
    uint32_t* w = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 x = *reinterpret_cast<__nv_bfloat162*>(&w[k]);
        x = __hmul2(x, hh);
        w[k] = *reinterpret_cast<uint32_t*>(&x);
    }
    return v;
}

// Packed pairs of FP32 (Blackwell f32x2 arithmetic: one instruction for two
// lanes' worth of IEEE single-precision operations, same rounding).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// 2 GELU(z) for a pair, tanh form: z + z tanh(z (c0 + c1 z^2)), c0 =
// sqrt(2/pi), c1 = 0.044715 sqrt(2/pi), z = accumulator + bias: five packed
// FP32 operations and two MUFU per pair. The factor 2 is taken back exactly by
// the halved copies of W2 and W3 in shared memory (scaling by a power of two
// commutes with BF16 rounding). Returns the pair rounded to BF16.
__device__ __forceinline__ uint32_t gelu2_pair(uint32_t acc_lo, uint32_t acc_hi, float2 b) {
    const uint64_t kC0 = f2_pack(0.7978845608028654f, 0.7978845608028654f);
    const uint64_t kC1 = f2_pack(0.035677408136300125f, 0.035677408136300125f);
    const uint64_t z = f2_add((uint64_t)acc_lo | ((uint64_t)acc_hi << 32), f2_pack(b.x, b.y));
    const uint64_t u = f2_mul(z, f2_fma(kC1, f2_mul(z, z), kC0));
    const uint64_t th = f2_pack(tanh_approx(f2_lo(u)), tanh_approx(f2_hi(u)));
    const uint64_t h = f2_fma(z, th, z);
    __nv_bfloat162 r = __floats2bfloat162_rn(f2_lo(h), f2_hi(h));
    return *reinterpret_cast<uint32_t*>(&r);
}

// Bias + GELU on 16 accumulator columns c0 .. c0+15 of this thread's row,
// BF16 into two 16-byte chunks of the row in its SW128 panel.
__device__ __forceinline__ void gelu_store16(const uint32_t (&r)[16], const float* bias, int c0, int row,
                                             unsigned char* H) {
    uint32_t pk[8];
    const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float4 bb = b4[e];
        pk[2 * e] = gelu2_pair(r[4 * e], r[4 * e + 1], make_float2(bb.x, bb.y));
        pk[2 * e + 1] = gelu2_pair(r[4 * e + 2], r[4 * e + 3], make_float2(bb.z, bb.w));
    }
    const int p = c0 >> 6, cb = (c0 & 63) >> 3;
    unsigned char* rowp = H + p * kPanelH + row * 128;
    *reinterpret_cast<uint4*>(rowp + ((cb ^ (row & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(rowp + (((cb + 1) ^ (row & 7)) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Makes this warp's activation stores visible to the tensor cores and adds
// its arrival (one per warp) on an mbarrier.
__device__ __forceinline__ void publish(uint64_t* bar) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(bar);
}

// The warp's 64 accumulator columns = panel cq, in four chunks of 16 (K
// quarters) with the TMEM load of the next chunk in flight while one is
// processed; after chunk j the warp arrives on quarter j's mbarrier.
__device__ __forceinline__ void hidden_epilogue(uint32_t tl, const float* bias, int cq, int row, unsigned char* H,
                                                uint64_t* bar_hq) {
    uint32_t ra[16], rb[16];
    const int c = 64 * cq;
    tc::tmem_ld16(tl + (uint32_t)c, ra);
    tc::wait_ld();
    tc::tmem_ld16(tl + (uint32_t)(c + 16), rb);
    gelu_store16(ra, bias, c, row, H);
    publish(bar_hq);
    tc::wait_ld();
    tc::tmem_ld16(tl + (uint32_t)(c + 32), ra);
    gelu_store16(rb, bias, c + 16, row, H);
    publish(bar_hq + 1);
    tc::wait_ld();
    tc::tmem_ld16(tl + (uint32_t)(c + 48), rb);
    gelu_store16(ra, bias, c + 32, row, H);
    publish(bar_hq + 2);
    tc::wait_ld();
    gelu_store16(rb, bias, c + 48, row, H);
    publish(bar_hq + 3);
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
    float* sinv = reinterpret_cast<float*>(sm + kOffInvSd);
    // mbarriers, each completing once per tile: layer-1 halves [2], layer-2
    // halves [2], layer 3, X tile written; activation quarters [4] (columns
    // 16 j .. 16 j + 15 of every panel written; twice per tile)
    uint64_t* bar_l1 = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* bar_l2 = bar_l1 + 2;
    uint64_t* bar_l3 = bar_l1 + 4;
    uint64_t* bar_x = bar_l1 + 5;
    uint64_t* bar_hq = bar_l1 + 6;   // [quarter]
    // completion of every MMA issued (waited on only when giving up), and a
    // barrier no thread ever completes (the stall test's wait)
    uint64_t* bar_drain = bar_l1 + 10;
    uint64_t* bar_never = bar_l1 + 11;
    const uint64_t kWaitNs = a.wait_ns;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffTmem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- weights into the swizzled operand layouts -----------------------
    // W2 and W3 multiply 2 GELU(z): stored halved (exact in BF16)
    const uint4* gW2 = reinterpret_cast<const uint4*>(a.W2);
    for (int e = tid; e < kMlpH * (kMlpH / 8); e += kTcThreads) {
        const int n = e >> 5, kc = e & 31;
        *reinterpret_cast<uint4*>(sm + kOffW2 + (kc >> 3) * kPanelW2 + n * 128 + (((kc & 7) ^ (n & 7)) << 4)) =
            half_bf16x8(gW2[e]);
    }
    const uint4* gW3 = reinterpret_cast<const uint4*>(a.W3);
    for (int e = tid; e < kMlpOutP * (kMlpH / 8); e += kTcThreads) {
        const int n = e >> 5, kc = e & 31;
        *reinterpret_cast<uint4*>(sm + kOffW3 + (kc >> 3) * kPanelW3 + n * 128 + (((kc & 7) ^ (n & 7)) << 4)) =
            half_bf16x8(gW3[e]);
    }
    const uint4* gW1 = reinterpret_cast<const uint4*>(a.W1);
    for (int e = tid; e < kMlpH * (kMlpInP / 8); e += kTcThreads) {
        const int n = e >> 2, c = e & 3;
        *reinterpret_cast<uint4*>(sm + kOffW1 + n * 64 + ((c ^ ((n >> 1) & 3)) << 4)) = gW1[e];
    }
    for (int e = tid; e < kMlpH; e += kTcThreads) { sb1[e] = a.b1[e]; sb2[e] = a.b2[e]; }
    for (int e = tid; e < kMlpOutP; e += kTcThreads) sb3[e] = a.b3[e];
    for (int e = tid; e < 2 * kMlpInP + 2 * kMlpOutP; e += kTcThreads) snorm[e] = a.norm[e];
    for (int e = tid; e < kMlpInP; e += kTcThreads) sinv[e] = 1.0f / a.norm[kMlpInP + e];
    if (tid == 0) {
        for (int k = 0; k < 5; ++k) tc::mbar_init(bar_l1 + k, 1);
        // one arrival per epilogue warp (after __syncwarp over its lanes' writes)
        tc::mbar_init(bar_x, kEpiWarps);
        for (int k = 0; k < 4; ++k) tc::mbar_init(bar_hq + k, kEpiWarps);
        tc::mbar_init(bar_drain, 1);
        tc::mbar_init(bar_never, 1);
        tc::mbar_init_fence();
    }
    if (warp == kEpiWarps) {
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
    if (warp < kEpiWarps) {
        // ---------------- epilogue warps ----------------
        const int q = warp & 3, cq = warp >> 2, hf = cq >> 1;
        const int erow = 32 * q + lane;                               // row of the tile = TMEM lane
        const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16);
        const int xr = tid >> 2, xq = tid & 3;                        // feature loader: row, quarter
        const float* mu_in = snorm;
        const float* mu_out = snorm + 2 * kMlpInP;
        const float* sd_out = mu_out + kMlpOutP;
        float4 pf[2];
        auto load_feat = [&](long tile) {
            const long gr = tile * kTcRows + xr;
            if (gr < a.rows) {
                const float4* src = reinterpret_cast<const float4*>(a.feat + gr * kMlpInP + 8 * xq);
                pf[0] = __ldg(src);
                pf[1] = __ldg(src + 1);
            } else {
                pf[0] = pf[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        // X tile: standardised, BF16, SW64 rows (zero rows past the end)
        auto write_x = [&](long tile) {
            const long gr = tile * kTcRows + xr;
            const float* v = reinterpret_cast<const float*>(pf);
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * xq + 2 * e;
                float x0 = 0.0f, x1 = 0.0f;
                if (gr < a.rows) {
                    x0 = (v[2 * e] - mu_in[c]) * sinv[c];
                    x1 = (v[2 * e + 1] - mu_in[c + 1]) * sinv[c + 1];
                }
                __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                pk[e] = *reinterpret_cast<uint32_t*>(&h);
            }
            *reinterpret_cast<uint4*>(sm + kOffX + xr * 64 + ((xq ^ ((xr >> 1) & 3)) << 4)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar_x);
        };
        long tile = blockIdx.x;
        const long G = gridDim.x;
        if (tile < ntiles) {
            load_feat(tile);
            write_x(tile);
            if (tile + G < ntiles) load_feat(tile + G);
        }
        for (; tile < ntiles; tile += G, ++it) {
            const long orow = tile * kTcRows + erow;
            float uu[kMlpOutP];
#pragma unroll
            for (int c = 0; c < kMlpOutP; ++c) uu[c] = 0.0f;
            if (cq == 0 && a.u && orow < a.rows) {
#pragma unroll
                for (int c = 0; c < kMlpOutP; ++c)
                    if (c < a.d) uu[c] = __ldg(a.u + orow * a.d + c);
            }
            const uint32_t par = it & 1;
            // layer 1 -> GELU -> H1
            if (!tc::warp_wait(bar_l1 + hf, par, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            hidden_epilogue(tl, sb1, cq, erow, sm + kOffH, bar_hq);
            // layer 2 -> GELU -> H2
            if (!tc::warp_wait(bar_l2 + hf, par, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            hidden_epilogue(tl + 256, sb2, cq, erow, sm + kOffH, bar_hq);
            // layer 3 done: the activations are free, so the next X tile goes
            // in now and its layer 1 (TMEM columns 0..255) runs while warps
            // 0-3 finish this tile's output (read from columns 256..271)
            if (!tc::warp_wait(bar_l3, par, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            uint32_t r[16];
            if (cq == 0) {   // the output accumulators, read before the next layer 1 is issued
                tc::tmem_ld16(tl + 256, r);
                tc::wait_ld();
            }
            if (tile + G < ntiles) {
                write_x(tile + G);
                if (tile + 2 * G < ntiles) load_feat(tile + 2 * G);   // in flight during the next tile
            }
            if (cq == 0) {
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
        // ---------------- MMA warp: lane 0 alone waits and issues ----------
        // Descriptors are built once; every MMA adds a compile-time byte offset
        // to the start-address field (all loops below are fully unrolled):
        // building them inside the issue loop costs far more than the MMA.
        bool issued = false;
        if (lane == 0 && a.stall && !tc::mbar_wait(bar_never, 0, kWaitNs)) ok = false;
        if (lane == 0 && ok) {
            const uint64_t gX = tc::smem_desc(sb + kOffX, 512, tc::kSwizzle64);
            const uint64_t gW1 = tc::smem_desc(sb + kOffW1, 512, tc::kSwizzle64);
            const uint64_t gH = tc::smem_desc(sb + kOffH, 1024, tc::kSwizzle128);
            const uint64_t gW2 = tc::smem_desc(sb + kOffW2, 1024, tc::kSwizzle128);
            const uint64_t gW3 = tc::smem_desc(sb + kOffW3, 1024, tc::kSwizzle128);
            for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                if (!tc::mbar_wait(bar_x, it & 1, kWaitNs)) { ok = false; break; }
                tc::fence_after_sync();
                issued = true;
                // two 128-column halves, each committed on its own so that
                // the epilogue warps of the first half start early
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
                        tc::mma_bf16(tbase + 128 * h, tc::desc_add(gX, 32 * ks),
                                     tc::desc_add(gW1, h * 128 * 64 + 32 * ks), kIdescN128, ks);
                    tc::mma_commit(bar_l1 + h);
                }
                // layer 2 by K quarters (columns 16 j .. 16 j + 15 of every
                // panel) as the epilogue writes them. In the last quarter the
                // first output half is committed before the second half's
                // panels 2 and 3: once that commit fired, the MMAs still in
                // flight read only panels 2 and 3, which the warps of the
                // first output half (columns 0..127 = panels 0, 1) do not
                // overwrite with the next activations.
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!tc::mbar_wait(bar_hq + j, 0, kWaitNs)) { ok = false; break; }
                    tc::fence_after_sync();
#pragma unroll
                    for (int step = 0; step < 3; ++step) {
                        // step 0: second output half, panels 0-1; step 1: first
                        // output half, panels 0-3; step 2: second half, panels 2-3
                        const int h = step == 1 ? 0 : 1;
                        const int p0 = step == 2 ? 2 : 0, p1 = step == 0 ? 2 : 4;
#pragma unroll
                        for (int p = p0; p < p1; ++p)
                            tc::mma_bf16(tbase + 256 + 128 * h, tc::desc_add(gH, p * kPanelH + 32 * j),
                                         tc::desc_add(gW2, p * kPanelW2 + h * 128 * 128 + 32 * j), kIdescN128,
                                         (j | p) != 0);
                        if (j == 3 && step >= 1) tc::mma_commit(bar_l2 + h);
                    }
                }
                if (!ok) break;
                // layer 3 into TMEM columns 256..271 (layer 2's, all read by now)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!tc::mbar_wait(bar_hq + j, 1, kWaitNs)) { ok = false; break; }
                    tc::fence_after_sync();
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        tc::mma_bf16(tbase + 256, tc::desc_add(gH, p * kPanelH + 32 * j),
                                     tc::desc_add(gW3, p * kPanelW3 + 32 * j), kIdescN16, (j | p) != 0);
                    if (j == 3) tc::mma_commit(bar_l3);
                }
                if (!ok) break;
            }
            if (!ok && issued) {
                // gave up with MMAs possibly in flight: they must complete
                // before the tensor memory they write is freed
                tc::mma_commit(bar_drain);
                tc::mbar_wait(bar_drain, 0, kWaitNs);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        __syncwarp();
    }
    if (!ok && lane == 0 && a.err) atomicExch(a.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kEpiWarps) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

}  // namespace

size_t mlp_forward_tc_smem() { return kTcSmem; }

cudaError_t mlp_forward_tc_launch(const MlpTcArgs& a, int num_sms, cudaStream_t st) {
    const cudaError_t e = ensure_dynamic_smem((const void*)mlp_forward_tc_kernel, kTcSmem);
    if (e != cudaSuccess) return e;
    const long tiles = (a.rows + kTcRows - 1) / kTcRows;
    const int grid = (int)(tiles < num_sms ? (tiles > 0 ? tiles : 1) : num_sms);
    mlp_forward_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace smap
