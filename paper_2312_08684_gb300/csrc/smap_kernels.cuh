// smap_kernels.cuh -- the fused per-step kernel of Stein-MAP-Seq.
//
// One CTA owns one sequence at a time and runs its time steps with the
// particle sets resident in shared memory:
//   a1  f_j = f_t(x_{t-1}^j) for the previous set (FP32 for the SVGD prior,
//       FP64 for the recursion), centred and scaled by Q^-1/2;
//   a2  x_t^{i,(0)} = f_t(x_{t-1}^i) + Q^{1/2} xi_i (Philox noise);
//   a3  h = s * med / log N from an exact median of the squared distances;
//   a4  g_k = grad log p(z_t | x_k) + grad log prior(x_k) (mixture over j);
//   a5  x_i += eps/N sum_k kappa_ik [g_k + (2/h)(x_i - x_k)]   (Eq. svgd_iterate);
//   a6  a3..a5 L times (Algorithm 1);
//   a7  psi_t(i), phi_t(i) of Eq. forward_recursion with FP64 scores;
// then stores x_t and psi_t to HBM. Sequences are taken from a device work
// queue (persistent CTAs), so uneven lengths and particle counts balance.
#pragma once

#include "smap_common.cuh"
#include "smap_models.cuh"

namespace smap {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
    size_t phis, xs, gs, fs, cand, zs, red, misc, total;
};

// Dynamic shared memory of the step kernels for Nmax particles of stride DP.
__host__ __device__ inline SmemLayout smem_layout(int Nmax, int DP) {
    SmemLayout L;
    size_t off = 0;
    L.phis = off; off = align16(off + sizeof(double) * Nmax);
    L.xs = off;   off = align16(off + sizeof(float) * Nmax * DP);
    L.gs = off;   off = align16(off + sizeof(float) * Nmax * (DP < 2 ? 2 : DP));
    L.fs = off;   off = align16(off + sizeof(float) * Nmax * DP);
    L.cand = off; off = align16(off + sizeof(uint32_t) * kCandCap);
    L.zs = off;   off = align16(off + sizeof(float) * kMaxDy);
    L.red = off;  off = align16(off + sizeof(double) * 40);
    L.misc = off; off = align16(off + sizeof(float) * 64);
    L.total = off;
    return L;
}

struct Sm {
    double* phis;   // phi_{t-1}(j), j < Np
    float* xs;      // particles [N][DP]
    float* gs;      // scores [N][DP]; later (A+, A-) pairs of the recursion screen
    float* fs;      // (f_t(x_{t-1}^j) - c) * Q^-1/2, [Np][DP]
    uint32_t* cand; // median candidates / radix histogram
    float* zs;      // observation z_t
    double* redd;   // reduction scratch (aliases redi / redf)
    int* redi;
    float* redf;
    float* misc;    // [0..15] centre c, [16..31] mean of fs (MEANGRAD)
    int* ncand;
};

__device__ inline Sm bind_smem(unsigned char* base, int Nmax, int DP) {
    const SmemLayout L = smem_layout(Nmax, DP);
    Sm s;
    s.phis = reinterpret_cast<double*>(base + L.phis);
    s.xs = reinterpret_cast<float*>(base + L.xs);
    s.gs = reinterpret_cast<float*>(base + L.gs);
    s.fs = reinterpret_cast<float*>(base + L.fs);
    s.cand = reinterpret_cast<uint32_t*>(base + L.cand);
    s.zs = reinterpret_cast<float*>(base + L.zs);
    s.redd = reinterpret_cast<double*>(base + L.red);
    s.redi = reinterpret_cast<int*>(base + L.red);
    s.redf = reinterpret_cast<float*>(base + L.red);
    s.misc = reinterpret_cast<float*>(base + L.misc);
    s.ncand = reinterpret_cast<int*>(base + L.misc) + 48;
    return s;
}

template <int D>
__device__ __forceinline__ float sqdist(const float* a, const float* b) {
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float e = a[c] - b[c];
        s = fmaf(e, e, s);
    }
    return s;
}

template <int D, int DP>
__device__ __forceinline__ void load_row(const float* xs, int i, float* r) {
#pragma unroll
    for (int c = 0; c < D; ++c) r[c] = xs[i * DP + c];
}

// ---------------------------------------------------------------------------
// a3: exact median of the N(N-1)/2 squared distances.
// ---------------------------------------------------------------------------

// Visits every unordered pair (i < k) once. Unit u pairs row u with row N-1-u,
// so every unit has N-1 pairs; a unit is split over S threads when the block
// has more threads than units.
template <int D, int DP, class F>
__device__ __forceinline__ void for_each_pair(const float* xs, int N, F& f) {
    if (N < 2) return;
    const int units = (N + 1) >> 1;
    const int NT = blockDim.x;
    const int S = NT >= units ? NT / units : 1;
    for (int w = threadIdx.x; w < units * S; w += NT) {
        const int u = w / S, s = w - u * S;
        const int r = u, r2 = N - 1 - u;
        const int len1 = N - 1 - r, len2 = (r2 > r) ? r : 0;
        const int total = len1 + len2;
        const int C = (total + S - 1) / S;
        const int m0 = s * C, m1 = min(total, m0 + C);
        const int e1 = min(m1, len1);
        if (m0 < e1) {
            float xr[D];
            load_row<D, DP>(xs, r, xr);
            for (int m = m0; m < e1; ++m) f(sqdist<D>(xr, xs + (r + 1 + m) * DP));
        }
        const int b2 = max(m0, len1);
        if (b2 < m1) {
            float xr[D];
            load_row<D, DP>(xs, r2, xr);
            for (int m = b2; m < m1; ++m) f(sqdist<D>(xr, xs + (r2 + 1 + (m - len1)) * DP));
        }
    }
}

struct BracketCount {
    uint32_t lo, hi;
    int nlo;
    uint32_t* cand;
    int* ncand;
    __device__ __forceinline__ void operator()(float v) {
        const uint32_t key = __float_as_uint(v);
        nlo += key < lo;
        const bool in = (key >= lo) & (key <= hi);
        const unsigned act = __activemask();
        const unsigned bal = __ballot_sync(act, in);
        if (bal) {
            const int leader = __ffs(act) - 1;
            int base = 0;
            if ((int)lane_id() == leader) base = atomicAdd(ncand, __popc(bal));
            base = __shfl_sync(act, base, leader);
            if (in) {
                const int idx = base + __popc(bal & ((1u << lane_id()) - 1u));
                if (idx < kCandCap) cand[idx] = key;
            }
        }
    }
};

struct RadixHist {
    uint32_t prefix, mask;
    int shift;
    int* hist;
    __device__ __forceinline__ void operator()(float v) {
        const uint32_t key = __float_as_uint(v);
        const bool ok = (key & mask) == prefix;
        const uint32_t bin = ok ? ((key >> shift) & 255u) : 256u;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, bin);
        if (ok && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
};

// Key of rank `rank` (0-based) among all pair distances: four 8-bit passes.
template <int D, int DP>
__device__ uint32_t radix_select(const Sm& s, int N, int rank) {
    int* hist = reinterpret_cast<int*>(s.cand);
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        RadixHist f{prefix, mask, shift, hist};
        for_each_pair<D, DP>(s.xs, N, f);
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0, bsel = 255;
            for (int bin = 0; bin < 256; ++bin) {
                if (cum + hist[bin] > rank) { bsel = bin; break; }
                cum += hist[bin];
            }
            s.redi[36] = bsel;
            s.redi[37] = rank - cum;
        }
        __syncthreads();
        const int bsel = s.redi[36];
        rank = s.redi[37];
        prefix |= (uint32_t)bsel << shift;
        mask |= 255u << shift;
        __syncthreads();
    }
    return prefix;
}

// Ascending bitonic sort of cand[0, n2) (n2 a power of two).
__device__ inline void bitonic_sort(uint32_t* c, int n2) {
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
                const int lo = (i / stride) * 2 * stride + (i % stride);
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint32_t a = c[lo], b = c[hi];
                if ((a > b) == up) { c[lo] = b; c[hi] = a; }
            }
            __syncthreads();
        }
    }
}

// Median of the squared pairwise distances. A bracket around the previous
// median is counted in one pass and its members sorted; if the bracket misses
// the middle ranks or overflows, an exact radix select decides. guess / w
// (bracket half-width, relative) carry over between calls. stats (may be
// null): [0] bracket hits, [1] radix fallbacks.
template <int D, int DP>
__device__ float median_sqdist(const Sm& s, int N, float& guess, float& w, bool& have_guess,
                               int* stats) {
    const int P = N * (N - 1) / 2;
    const int r1 = (P & 1) ? (P - 1) / 2 : P / 2 - 1;
    const int r2 = (P & 1) ? r1 : P / 2;
    uint32_t v1 = 0, v2 = 0;
    bool done = false;
    if (have_guess && guess > 0.0f && isfinite(guess)) {
        if (threadIdx.x == 0) *s.ncand = 0;
        __syncthreads();
        BracketCount f{__float_as_uint(guess * (1.0f - w)), __float_as_uint(guess * (1.0f + w)), 0,
                       s.cand, s.ncand};
        for_each_pair<D, DP>(s.xs, N, f);
        const int nlo = block_sum_int(f.nlo, s.redi);   // ends with a barrier
        const int nc = *s.ncand;
        if (nlo <= r1 && r2 < nlo + nc && nc <= kCandCap) {
            int n2 = 1;
            while (n2 < nc) n2 <<= 1;
            for (int i = nc + threadIdx.x; i < n2; i += blockDim.x) s.cand[i] = 0xFFFFFFFFu;
            __syncthreads();
            bitonic_sort(s.cand, n2);
            v1 = s.cand[r1 - nlo];
            v2 = s.cand[r2 - nlo];
            done = true;
            if (nc * 8 < kCandCap) w = fmaxf(w * 0.7f, 1e-4f);
            else if (nc * 2 > kCandCap) w *= 0.5f;
        } else if (nc > kCandCap) {
            w *= 0.3f;
        } else {
            w = fminf(w * 3.0f, 1.0f);
        }
        __syncthreads();
    }
    if (!done) {
        v1 = radix_select<D, DP>(s, N, r1);
        v2 = (r2 == r1) ? v1 : radix_select<D, DP>(s, N, r2);
    }
    if (stats && threadIdx.x == 0) atomicAdd(&stats[done ? 0 : 1], 1);
    const float med = 0.5f * (__uint_as_float(v1) + __uint_as_float(v2));
    guess = med;
    have_guess = true;
    return med;
}

// ---------------------------------------------------------------------------
// a1/a2: transition means of the previous set and the initial particles.
// On return (after a barrier): fs, misc (centre, fs mean), zs, f64 are set
// and xs holds the initial particles of step t. first = the previous set is
// {x_0^true} (taken in FP64 from x0).
// ---------------------------------------------------------------------------
template <class M, int PPT>
__device__ void prepare_step(const ModelParams& mp, const Sm& s, int t, int N, int Np, bool first,
                             const double* x0, const float* yt, double* f64, int prior,
                             uint64_t seed, uint32_t seq, const float* xinit) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int c = tid; c < mp.dy; c += NT) s.zs[c] = yt[c];
    const double sc = M::step_const(mp, t);
    double xp0[D], f0[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xp0[c] = first ? x0[c] : (double)s.xs[c];
    M::transition64(mp, sc, xp0, f0);
    float cf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) cf[c] = (float)f0[c];
    if (tid < D) s.misc[tid] = cf[tid];
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        double fd[D];
        if (i < Np) {
            if (first) {
#pragma unroll
                for (int c = 0; c < D; ++c) fd[c] = f0[c];
            } else {
                double xd[D];
#pragma unroll
                for (int c = 0; c < D; ++c) xd[c] = (double)s.xs[i * DP + c];
                M::transition64(mp, sc, xd, fd);
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                f64[(size_t)i * D + c] = fd[c];
                s.fs[i * DP + c] = (float)((fd[c] - (double)cf[c]) * mp.sqrt_qinv[c]);
            }
#pragma unroll
            for (int c = D; c < DP; ++c) s.fs[i * DP + c] = 0.0f;
        }
        if (i < N) {
            float xi[D];
            if (xinit) {
#pragma unroll
                for (int c = 0; c < D; ++c) xi[c] = xinit[(size_t)i * D + c];
            } else {
                const double* fa = (Np == 1) ? f0 : fd;
                float z[D];
                draw_normals<D>(seed, seq, (uint32_t)t, (uint32_t)i, z);
#pragma unroll
                for (int c = 0; c < D; ++c) xi[c] = (float)(fa[c] + mp.sqrt_q[c] * (double)z[c]);
            }
#pragma unroll
            for (int c = 0; c < D; ++c) s.xs[i * DP + c] = xi[c];
#pragma unroll
            for (int c = D; c < DP; ++c) s.xs[i * DP + c] = 0.0f;
        }
    }
    if (prior == 1) {   // MEANGRAD needs mean_j fs_j
        __syncthreads();
        for (int c = 0; c < D; ++c) {
            float v = 0.0f;
            for (int j = tid; j < Np; j += NT) v += s.fs[j * DP + c];
            v = block_sum_f(v, s.redf);
            if (tid == 0) s.misc[16 + c] = v / (float)Np;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// a4: scores g_i = grad log p(z_t | x_i) + grad log prior(x_i) -> gs.
// ---------------------------------------------------------------------------
template <class M, int PPT>
__device__ __forceinline__ void compute_scores(const ModelParams& mp, const Sm& s, int N, int Np,
                                               int prior) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    const float kL2E = 1.4426950408889634f;
    float xt[PPT][D], A[PPT][D], S[PPT], Mx[PPT];
    float sq[D], cf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { sq[c] = mp.sqrt_qinv_f[c]; cf[c] = s.misc[c]; }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xt[p][c] = (s.xs[i * DP + c] - cf[c]) * sq[c];
            A[p][c] = 0.0f;
        }
        S[p] = 0.0f;
        Mx[p] = -INFINITY;
    }
    if (prior == 0) {
        // mixture: responsibilities w_ij = softmax_j(-1/2 |x_i - f_j|^2_{Q^-1}),
        // accumulated with a running maximum (log2 units)
        for (int j = 0; j < Np; ++j) {
            float fj[D];
            load_row<D, DP>(s.fs, j, fj);
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                float diff[D], m = 0.0f;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    diff[c] = xt[p][c] - fj[c];
                    m = fmaf(diff[c], diff[c], m);
                }
                const float lg = m * (-0.5f * kL2E);
                if (lg > Mx[p]) {
                    const float r = fast_exp2(Mx[p] - lg);
                    S[p] *= r;
#pragma unroll
                    for (int c = 0; c < D; ++c) A[p][c] *= r;
                    Mx[p] = lg;
                }
                const float e = fast_exp2(lg - Mx[p]);
                S[p] += e;
#pragma unroll
                for (int c = 0; c < D; ++c) A[p][c] = fmaf(e, diff[c], A[p][c]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) continue;
        float x[D], g[D];
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = s.xs[i * DP + c];
        M::grad_loglik(mp, s.zs, x, g);
        if (prior == 0) {
            const float inv = 1.0f / S[p];
#pragma unroll
            for (int c = 0; c < D; ++c) g[c] -= sq[c] * A[p][c] * inv;
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) g[c] -= sq[c] * (xt[p][c] - s.misc[16 + c]);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) s.gs[i * DP + c] = g[c];
#pragma unroll
        for (int c = D; c < DP; ++c) s.gs[i * DP + c] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// a5: one SVGD update of the block's particles (Eq. svgd_iterate).
// ---------------------------------------------------------------------------
template <class M, int PPT>
__device__ __forceinline__ void rbf_update(const Sm& s, int N, float h, float eps) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    const float c2 = -1.4426950408889634f / h;
    const float twoh = 2.0f / h;
    float xi[PPT][D], Sg[PPT][D], Sd[PPT][D];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xi[p][c] = s.xs[i * DP + c];
            Sg[p][c] = 0.0f;
            Sd[p][c] = 0.0f;
        }
    }
    for (int k = 0; k < N; ++k) {
        float xk[D], gk[D];
        load_row<D, DP>(s.xs, k, xk);
        load_row<D, DP>(s.gs, k, gk);
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            float diff[D], m = 0.0f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                diff[c] = xi[p][c] - xk[c];
                m = fmaf(diff[c], diff[c], m);
            }
            const float kap = fast_exp2(m * c2);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                Sg[p][c] = fmaf(kap, gk[c], Sg[p][c]);
                Sd[p][c] = fmaf(kap, diff[c], Sd[p][c]);
            }
        }
    }
    const float sc = eps / (float)N;
    __syncthreads();   // every thread is done reading xs / gs
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < D; ++c) s.xs[i * DP + c] = fmaf(sc, fmaf(twoh, Sd[p][c], Sg[p][c]), xi[p][c]);
    }
    __syncthreads();
}

// a3..a6: L iterations. hout (may be null) receives h per iteration.
template <class M, int PPT>
__device__ void svgd_iterations(const ModelParams& mp, const Sm& s, int N, int Np, int L, float eps,
                                int bw_rule, float bw_value, int prior, float& guess, float& w,
                                bool& have_guess, float* hout, int* stats) {
    float h = 1.0f;
    for (int l = 0; l < L; ++l) {
        if (bw_rule == 2) {
            h = bw_value;
        } else if (bw_rule == 0 || l == 0) {
            if (N < 2) {
                h = 1.0f;
            } else {
                if (l == 0) w = fmaxf(w, 0.25f);
                const float med = median_sqdist<M::D, M::DP>(s, N, guess, w, have_guess, stats);
                h = (med > 0.0f) ? bw_value * med / logf((float)N) : 1.0f;
            }
        }
        if (hout && threadIdx.x == 0) hout[l] = h;
        compute_scores<M, PPT>(mp, s, N, Np, prior);
        __syncthreads();
        rbf_update<M, PPT>(s, N, h, eps);
    }
}

// ---------------------------------------------------------------------------
// a7: forward recursion. The argmax over j of phi_{t-1}(j) + log p(x_i | x^j)
// is screened in FP32 with a rigorous rounding bound (centred, Q^-1/2-scaled
// coordinates), and every j that can still be the FP64 maximum is evaluated
// in FP64; phi_t is accumulated in FP64. Lowest j wins ties.
// On return: best[p], phinew[p] for the block's particles.
// ---------------------------------------------------------------------------
template <class M, int PPT>
__device__ void viterbi_step(const ModelParams& mp, const Sm& s, int N, int Np, const double* f64,
                             int* best, double* phinew) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    // K u with u = 2^-24, K = 64: covers the FP32 errors of the screen.
    const float Ku = 3.814697265625e-06f;
    double pmax = -INFINITY;
    for (int j = tid; j < Np; j += NT) pmax = fmax(pmax, s.phis[j]);
    pmax = block_max_d(pmax, s.redd);
    float2* ab = reinterpret_cast<float2*>(s.gs);
    for (int j = tid; j < Np; j += NT) {
        const double dphi = s.phis[j] - pmax;
        const float ph = (float)dphi;
        float F = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) F = fmaf(s.fs[j * DP + c], s.fs[j * DP + c], F);
        const float B = Ku * (F + fabsf(ph)) +
                        (float)(4.4408920985006262e-16 * (fabs(s.phis[j]) + fabs(pmax)));
        ab[j] = make_float2(ph + B, ph - B);
    }
    __syncthreads();
    float xc[PPT][D], C[PPT], Lmax[PPT];
    float sq[D], cf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { sq[c] = mp.sqrt_qinv_f[c]; cf[c] = s.misc[c]; }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
        float X = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xc[p][c] = (s.xs[i * DP + c] - cf[c]) * sq[c];
            X = fmaf(xc[p][c], xc[p][c], X);
        }
        C[p] = Ku * X;
        Lmax[p] = -INFINITY;
    }
    // pass 1: the best guaranteed lower bound
    for (int j = 0; j < Np; ++j) {
        float fj[D];
        load_row<D, DP>(s.fs, j, fj);
        const float am = ab[j].y;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            float m = 0.0f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float e = xc[p][c] - fj[c];
                m = fmaf(e, e, m);
            }
            Lmax[p] = fmaxf(Lmax[p], fmaf(-(0.5f + Ku), m, am - C[p]));
        }
    }
    // pass 2: FP64 evaluation of every candidate whose upper bound reaches Lmax
    double bs[PPT], blt[PPT], xd[PPT][D];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
        bs[p] = -INFINITY;
        blt[p] = 0.0;
        best[p] = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) xd[p][c] = (double)s.xs[i * DP + c];
    }
    for (int j = 0; j < Np; ++j) {
        float fj[D];
        load_row<D, DP>(s.fs, j, fj);
        const float ap = ab[j].x;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            float m = 0.0f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float e = xc[p][c] - fj[c];
                m = fmaf(e, e, m);
            }
            const float U = fmaf(-(0.5f - Ku), m, ap + C[p]);
            if (U >= Lmax[p]) {
                double m64 = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const double e = xd[p][c] - f64[(size_t)j * D + c];
                    m64 += e * e * mp.qinv[c];
                }
                const double lt = mp.logtrans_c - 0.5 * m64;
                const double sv = s.phis[j] + lt;
                if (sv > bs[p]) { bs[p] = sv; blt[p] = lt; best[p] = j; }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (bs[p] == -INFINITY) {
            // no candidate passed the screen (non-finite inputs): plain FP64 scan
            for (int j = 0; j < Np; ++j) {
                double m64 = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const double e = xd[p][c] - f64[(size_t)j * D + c];
                    m64 += e * e * mp.qinv[c];
                }
                const double lt = mp.logtrans_c - 0.5 * m64;
                const double sv = s.phis[j] + lt;
                if (sv > bs[p]) { bs[p] = sv; blt[p] = lt; best[p] = j; }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) { phinew[p] = 0.0; continue; }
        phinew[p] = M::loglik64(mp, s.zs, xd[p]) + blt[p] + s.phis[best[p]];
    }
}

// ---------------------------------------------------------------------------
// The persistent sequence kernel.
// ---------------------------------------------------------------------------
template <class M, int PPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) seq_kernel(const __grid_constant__ SeqArgs a) {
    constexpr int D = M::D, DP = M::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sm s = bind_smem(smem_raw, a.Nmax, DP);
    const ModelParams& mp = a.mp;
    const int tid = threadIdx.x, NT = blockDim.x;
    __shared__ int s_item;
    double* f64 = a.f64 + (size_t)blockIdx.x * a.Nmax * D;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.B) break;
        const int b = a.order ? a.order[item] : item;
        if (a.mode == 1 && a.active && !a.active[b]) continue;
        if (a.status[b] != 0) continue;
        const int N = a.Nseq[b];
        const int t0 = a.tcur[b];
        const int t1 = (a.mode == 1) ? t0 + 1 : a.Tend[b];
        if (t1 > a.maxT || N < 1 || N > a.Nmax) {
            if (tid == 0) a.status[b] = 1;
            continue;
        }
        int Np = 1;
        if (t0 == 0) {
            if (tid == 0) s.phis[0] = 0.0;
        } else {
            Np = N;
            const float* src = a.hist + (((size_t)b * a.maxT + (t0 - 1)) * a.Nmax) * D;
            for (int e = tid; e < N * D; e += NT) s.xs[(e / D) * DP + (e % D)] = src[e];
            for (int j = tid; j < N; j += NT) s.phis[j] = a.phi[(size_t)b * a.Nmax + j];
        }
        float guess = a.bwguess[b], w = 0.25f;
        bool have_guess = (t0 > 0) && guess > 0.0f;
        int tdone = t0;
        __syncthreads();
        for (int t = t0 + 1; t <= t1; ++t) {
            const float* yt = (a.mode == 1) ? a.y + (size_t)b * mp.dy
                                            : a.y + ((size_t)b * a.maxT + (t - 1)) * mp.dy;
            const float* xin = a.viterbi_only
                                   ? a.hist + (((size_t)b * a.maxT + (t - 1)) * a.Nmax) * D
                                   : nullptr;
            prepare_step<M, PPT>(mp, s, t, N, Np, t == 1, a.x0 + (size_t)b * D, yt, f64, a.prior,
                                 a.seed, (uint32_t)b, xin);
            if (!a.viterbi_only)
                svgd_iterations<M, PPT>(mp, s, N, Np, a.L, a.eps, a.bw_rule, a.bw_value, a.prior,
                                        guess, w, have_guess, nullptr, a.status + a.B);
            int best[PPT];
            double phinew[PPT];
            viterbi_step<M, PPT>(mp, s, N, Np, f64, best, phinew);
            __syncthreads();   // all reads of phis / xs done
            bool bad = false;
            float* dst = a.hist + (((size_t)b * a.maxT + (t - 1)) * a.Nmax) * D;
            uint16_t* pdst = a.psi + ((size_t)b * a.maxT + (t - 1)) * a.Nmax;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const int i = tid + p * NT;
                if (i >= N) continue;
                s.phis[i] = phinew[p];
                bad |= !isfinite(phinew[p]);
                if (!a.viterbi_only) {
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        const float v = s.xs[i * DP + c];
                        bad |= !isfinite(v);
                        dst[(size_t)i * D + c] = v;
                    }
                }
                pdst[i] = (uint16_t)best[p];
            }
            bad = __syncthreads_or(bad);
            if (bad) {
                if (tid == 0) a.status[b] = 6;   // SMAP_E_NONFINITE
                break;
            }
            tdone = t;
            Np = N;
        }
        __syncthreads();
        for (int j = tid; j < N; j += NT) a.phi[(size_t)b * a.Nmax + j] = s.phis[j];
        if (tid == 0) {
            a.tcur[b] = tdone;
            a.bwguess[b] = guess;
        }
    }
}

// Debug: n iterations of SVGD from given particles (one CTA per sequence).
template <class M, int PPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) debug_svgd_kernel(const __grid_constant__ DebugSvgdArgs a) {
    constexpr int D = M::D, DP = M::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Nmax = a.N > a.Np ? a.N : a.Np;
    const Sm s = bind_smem(smem_raw, Nmax, DP);
    const int b = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    const bool first = (a.t == 1 && a.Np == 1);
    // the previous set goes through xs (prepare_step reads it there)
    const float* xp = a.xprev + (size_t)b * a.Np * D;
    for (int e = tid; e < a.Np * D; e += NT) s.xs[(e / D) * DP + (e % D)] = xp[e];
    __syncthreads();
    prepare_step<M, PPT>(a.mp, s, a.t, a.N, a.Np, first, a.x0 + (size_t)b * D, a.y + (size_t)b * a.mp.dy,
                         a.f64 + (size_t)b * a.Np * D, a.prior, 0, 0,
                         a.xinit + (size_t)b * a.N * D);
    float guess = 0.0f, w = 0.25f;
    bool have_guess = false;
    svgd_iterations<M, PPT>(a.mp, s, a.N, a.Np, a.iters, a.eps, a.bw_rule, a.bw_value, a.prior, guess,
                            w, have_guess, a.hout ? a.hout + (size_t)b * a.iters : nullptr, nullptr);
    for (int e = tid; e < a.N * D; e += NT)
        a.xout[(size_t)b * a.N * D + e] = s.xs[(e / D) * DP + (e % D)];
}

}  // namespace smap
