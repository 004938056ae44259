// smap_kernels.cuh -- the fused per-step kernel of Stein-MAP-Seq.
//
// One CTA owns one sequence at a time and runs its time steps with the
// particle sets resident in shared memory:
//   a1  f_j = f_t(x_{t-1}^j) for the previous set (FP64, kept for the
//       recursion; FP32 copies centred and scaled by Q^-1/2 for the prior);
//   a2  x_t^{i,(0)} = f_t(x_{t-1}^i) + Q^{1/2} xi_i (Philox noise);
//   a3  h = s * med / log N from an exact median of the squared distances;
//   a4  g_k = grad log p(z_t | x_k) + grad log prior(x_k) (mixture over j);
//   a5  x_i += eps/N sum_k kappa_ik [g_k + (2/h)(x_i - x_k)]   (Eq. svgd_iterate);
//   a6  a3..a5 L times (Algorithm 1);
//   a7  psi_t(i), phi_t(i) of Eq. forward_recursion with FP64 scores;
// then stores x_t and psi_t to HBM. Sequences are taken from a device work
// queue (persistent CTAs), so uneven lengths and particle counts balance.
//
// During the SVGD iterations the particles are held centred (on c = f_t of
// the first previous particle) and scaled by sqrt(log2(e)/h), so that
// kappa_ik = 2^-|x^_i - x^_k|^2 costs one ex2 and no multiply; the prior works
// in coordinates scaled by Q^-1/2 sqrt(log2(e)/2), where the mixture logit of
// j is -|x~ - f~_j|^2 in log2 units.
#pragma once

#include "smap_common.cuh"
#include "smap_models.cuh"

namespace smap {

constexpr float kL2E = 1.4426950408889634f;    // log2(e)
constexpr float kKm = 0.84932180028801907f;    // sqrt(log2(e) / 2)
constexpr float kLam = 1.3862943611198906f;    // 1 / kKm^2 = 2 ln 2

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
    size_t phis, xs, gs, fs, nrm, phf, cand, zs, red, misc, total;
};

// The recursion screen takes predecessors in pairs (2q, 2q+1) and in chunks of
// kRecPairs pairs. Its per-pair arrays are padded after every chunk (16 bytes
// in the g rows, 8 bytes in the aU pairs), so that lanes rescanning different
// chunks read different shared-memory banks.
constexpr int kRecPairs = 16;
__host__ __device__ inline int rec_pairs(int Np) { return (Np + 1) >> 1; }
__host__ __device__ inline int rec_chunks(int Np) { return (rec_pairs(Np) + kRecPairs - 1) / kRecPairs; }
// Offsets in 8-byte units: g row of pair q (DP words), aU word of pair q.
__host__ __device__ inline int rec_grow(int q, int DP) { return q * DP + 2 * (q / kRecPairs); }
__host__ __device__ inline int rec_arow(int q) { return q + q / kRecPairs; }

// Dynamic shared memory of the step kernels for Nmax particles of stride DP.
__host__ __device__ inline SmemLayout smem_layout(int Nmax, int DP) {
    SmemLayout L;
    size_t off = 0;
    const size_t P = rec_pairs(Nmax), C = rec_chunks(Nmax);
    L.phis = off; off = align16(off + sizeof(double) * Nmax);
    L.xs = off;   off = align16(off + sizeof(float) * Nmax * DP);
    // gs: SVGD's w rows, or the recursion's aU pairs and 2e array
    const size_t gsf = (size_t)Nmax * (DP < 2 ? 2 : DP);
    const size_t recf = 2 * (P + C) + 2 * P + 4;
    L.gs = off;   off = align16(off + sizeof(float) * (gsf > recf ? gsf : recf));
    // fs: the previous set's rows, or the recursion's g rows in pairs
    const size_t fsf = (size_t)(Nmax + 1) * DP, gpf = 2 * (P * DP + 2 * C);
    L.fs = off;   off = align16(off + sizeof(float) * (fsf > gpf ? fsf : gpf));
    L.nrm = off;  off = align16(off + sizeof(float) * Nmax);
    L.phf = off;  off = align16(off + sizeof(float) * Nmax);
    L.cand = off; off = align16(off + sizeof(uint32_t) * kCandCap);
    L.zs = off;   off = align16(off + sizeof(float) * kMaxDy);
    L.red = off;  off = align16(off + sizeof(double) * 40);
    L.misc = off; off = align16(off + sizeof(float) * 64);
    L.total = off;
    return L;
}

struct Sm {
    double* phis;   // phi_{t-1}(j), j < Np
    float* xs;      // particles [N][DP] (absolute, or centred+scaled inside SVGD)
    float* gs;      // w_k = A g_k - Bc x^_k [N][DP]; later (A+, A-) of the recursion screen
    float* fs;      // (f_t(x_{t-1}^j) - c) Q^-1/2 kKm, [Np][DP]
    float* nrm;     // |x^_k|^2 of the scaled particles
    float* phf;     // (phi_{t-1}(j) - max) log2(e) in FP32 (MAP-conditioned prior)
    uint32_t* cand; // median candidates / histograms
    float* zs;      // observation z_t
    double* redd;   // reduction scratch (aliases redi / redf)
    int* redi;
    float* redf;
    float* misc;    // [0..15] centre c, [16..31] mean of fs (MEANGRAD)
    int* ncand;
};

// Dynamic shared memory of the recursion-only kernel: the arrays prepare_step
// and viterbi_step use (none of the median's or the prior's).
__host__ __device__ inline SmemLayout rec_smem_layout(int Nmax, int DP) {
    SmemLayout L;
    size_t off = 0;
    const size_t P = rec_pairs(Nmax), C = rec_chunks(Nmax);
    L.phis = off; off = align16(off + sizeof(double) * Nmax);
    L.xs = off;   off = align16(off + sizeof(float) * Nmax * DP);
    L.gs = off;   off = align16(off + sizeof(float) * (2 * (P + C) + 2 * P + 4));
    const size_t fsf = (size_t)(Nmax + 1) * DP, gpf = 2 * (P * DP + 2 * C);
    L.fs = off;   off = align16(off + sizeof(float) * (fsf > gpf ? fsf : gpf));
    L.zs = off;   off = align16(off + sizeof(float) * kMaxDy);
    L.red = off;  off = align16(off + sizeof(double) * 40);
    L.misc = off; off = align16(off + sizeof(float) * 64);
    L.nrm = L.phf = L.cand = off;   // not used by the recursion
    L.total = off;
    return L;
}

__device__ inline Sm bind_smem_at(unsigned char* base, const SmemLayout& L) {
    Sm s;
    s.phis = reinterpret_cast<double*>(base + L.phis);
    s.xs = reinterpret_cast<float*>(base + L.xs);
    s.gs = reinterpret_cast<float*>(base + L.gs);
    s.fs = reinterpret_cast<float*>(base + L.fs);
    s.nrm = reinterpret_cast<float*>(base + L.nrm);
    s.phf = reinterpret_cast<float*>(base + L.phf);
    s.cand = reinterpret_cast<uint32_t*>(base + L.cand);
    s.zs = reinterpret_cast<float*>(base + L.zs);
    s.redd = reinterpret_cast<double*>(base + L.red);
    s.redi = reinterpret_cast<int*>(base + L.red);
    s.redf = reinterpret_cast<float*>(base + L.red);
    s.misc = reinterpret_cast<float*>(base + L.misc);
    s.ncand = reinterpret_cast<int*>(base + L.misc) + 48;
    return s;
}
__device__ inline Sm bind_smem(unsigned char* base, int Nmax, int DP) {
    return bind_smem_at(base, smem_layout(Nmax, DP));
}

// Row i of a [*][DP] shared array: 128-bit loads when DP is a multiple of 4.
template <int D, int DP>
__device__ __forceinline__ void load_row(const float* base, int i, float* r) {
#ifdef SMAP_DEBUG
    if (!SMAP_DBG((unsigned)i < (unsigned)g_dbg_rows, kDbgRow, i)) {
#pragma unroll
        for (int c = 0; c < D; ++c) r[c] = 0.0f;
        return;
    }
#endif
    if constexpr (DP % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(base + i * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 v = p[q];
            if (4 * q + 0 < D) r[4 * q + 0] = v.x;
            if (4 * q + 1 < D) r[4 * q + 1] = v.y;
            if (4 * q + 2 < D) r[4 * q + 2] = v.z;
            if (4 * q + 3 < D) r[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) r[c] = base[i * DP + c];
    }
}

template <int D, int DP>
__device__ __forceinline__ void store_row(float* base, int i, const float* r) {
    if (!SMAP_DBG((unsigned)i < (unsigned)g_dbg_rows, kDbgRow, i)) return;
#pragma unroll
    for (int c = 0; c < DP; ++c) base[i * DP + c] = c < D ? r[c] : 0.0f;
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

// Sum over the TPP consecutive lanes that share a particle (TPP divides 32;
// every lane of the warp must call).
template <int TPP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// a3: exact median of the N(N-1)/2 squared distances.
// ---------------------------------------------------------------------------

// Visits every unordered pair (i < k) once, as f(d_ik) with the squared
// distance d_ik = |x_i|^2 + |x_k|^2 - 2 x_i . x_k from the norms in nrm,
// clamped at 0 (so the keys order as unsigned integers). Unit u pairs row u
// with row N-1-u, so every unit has N-1 pairs; a unit is split over S threads
// when the block has more threads than units.
template <int D, int DP, class F>
__device__ __forceinline__ void for_each_pair(const float* xs, const float* nrm, int N, F& f) {
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
            const float nr = nrm[r];
#pragma unroll
            for (int c = 0; c < D; ++c) xr[c] *= -2.0f;
#pragma unroll 4
            for (int m = m0; m < e1; ++m) {
                float xk[D];
                load_row<D, DP>(xs, r + 1 + m, xk);
                float v = nr + nrm[r + 1 + m];
#pragma unroll
                for (int c = 0; c < D; ++c) v = fmaf(xr[c], xk[c], v);
                f(fmaxf(v, 0.0f));
            }
        }
        const int b2 = max(m0, len1);
        if (b2 < m1) {
            float xr[D];
            load_row<D, DP>(xs, r2, xr);
            const float nr = nrm[r2];
#pragma unroll
            for (int c = 0; c < D; ++c) xr[c] *= -2.0f;
#pragma unroll 4
            for (int m = b2; m < m1; ++m) {
                const int k = r2 + 1 + (m - len1);
                float xk[D];
                load_row<D, DP>(xs, k, xk);
                float v = nr + nrm[k];
#pragma unroll
                for (int c = 0; c < D; ++c) v = fmaf(xr[c], xk[c], v);
                f(fmaxf(v, 0.0f));
            }
        }
    }
}

// Counts keys below lo and collects the keys in [lo, hi]. A bracket holds a
// few hundred of the N(N-1)/2 keys, so the collection is a rarely taken branch
// with a plain shared atomic (cheaper per pair than a warp vote).
struct BracketCount {
    float lo, hi;
    int nlo;
    uint32_t* cand;
    int* ncand;
    __device__ __forceinline__ void operator()(float v) {
        nlo += v < lo;
        if (v >= lo && v <= hi) {
            const int idx = atomicAdd(ncand, 1);
            if (idx < kCandCap) cand[idx] = __float_as_uint(v);
        }
    }
};

// 256-bin histogram of keys: bin = (key - key_lo) >> shift, clamped, so bin 0
// and bin 255 also collect everything below and above the covered range.
struct KeyHist {
    uint32_t key_lo;
    int shift;
    int* hist;
    __device__ __forceinline__ void operator()(float v) {
        const uint32_t key = __float_as_uint(v);
        const uint32_t off = key >= key_lo ? (key - key_lo) >> shift : 0u;
        const int bin = (int)min(off, 255u);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, bin);
        if ((int)lane_id() == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
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
        for_each_pair<D, DP>(s.xs, s.nrm, N, f);
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

// One bracket pass over all pairs: on success (the middle ranks fall inside
// [lo, hi] and at most kCandCap keys do) v1, v2 are the keys of ranks r1, r2.
template <int D, int DP>
__device__ bool bracket_pass(const Sm& s, int N, float lo, float hi, int r1, int r2, uint32_t& v1,
                             uint32_t& v2, int& nc_out) {
    if (threadIdx.x == 0) *s.ncand = 0;
    __syncthreads();
    BracketCount f{lo, hi, 0, s.cand, s.ncand};
    for_each_pair<D, DP>(s.xs, s.nrm, N, f);
    const int nlo = block_sum_int(f.nlo, s.redi);   // ends with a barrier
    const int nc = *s.ncand;
    nc_out = nc;
    const bool inside = nlo <= r1 && r2 < nlo + nc;
    bool ok = inside && nc <= kCandCap;
    if (ok && nc <= 256) {
        // rank of each candidate by counting (ties by position): one barrier
        const int k1 = r1 - nlo, k2 = r2 - nlo;
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const uint32_t key = s.cand[c];
            int rank = 0;
            for (int o = 0; o < nc; ++o) {
                const uint32_t v = s.cand[o];
                rank += (v < key) | ((v == key) & (o < c));
            }
            if (rank == k1) s.redi[40] = (int)key;
            if (rank == k2) s.redi[41] = (int)key;
        }
        __syncthreads();
        v1 = (uint32_t)s.redi[40];
        v2 = (uint32_t)s.redi[41];
    } else if (ok) {
        int n2 = 1;
        while (n2 < nc) n2 <<= 1;
        for (int i = nc + threadIdx.x; i < n2; i += blockDim.x) s.cand[i] = 0xFFFFFFFFu;
        __syncthreads();
        bitonic_sort(s.cand, n2);
        v1 = s.cand[r1 - nlo];
        v2 = s.cand[r2 - nlo];
    }
    __syncthreads();
    if (threadIdx.x == 0) s.redi[39] = inside ? 1 : 0;
    __syncthreads();
    return ok;
}

// Median state carried across iterations and steps (uniform over the block).
struct MedState {
    float med;     // last median (absolute units)
    float trend;   // ratio of the last two medians
    float w;       // bracket half-width, relative
    int have;      // med is valid
    int fresh;     // the set changed beyond one SVGD update (new step)
};

// One histogram pass (KeyHist) that locates ranks r1 <= r2: on success
// [lo, hi] is the key range of their bins, n_in the number of keys in it.
template <int D, int DP>
__device__ bool locate_pass(const Sm& s, int N, uint32_t key_lo, int shift, int r1, int r2, uint32_t& lo,
                            uint32_t& hi, int& n_in) {
    int* hist = reinterpret_cast<int*>(s.cand);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    KeyHist f{key_lo, shift, hist};
    for_each_pair<D, DP>(s.xs, s.nrm, N, f);
    __syncthreads();
    if (threadIdx.x == 0) {
        int cum = 0, b1 = -1, b2 = -1, c1 = 0, cnt = 0;
        for (int bin = 0; bin < 256; ++bin) {
            const int c = hist[bin];
            if (b1 < 0 && cum + c > r1) { b1 = bin; c1 = cum; }
            if (b1 >= 0) cnt += c;
            if (cum + c > r2) { b2 = bin; break; }
            cum += c;
        }
        s.redi[36] = b1;
        s.redi[37] = b2;
        s.redi[38] = cnt;
        (void)c1;
    }
    __syncthreads();
    const int b1 = s.redi[36], b2 = s.redi[37];
    n_in = s.redi[38];
    __syncthreads();
    // the end bins also hold keys outside the covered range: not usable
    if (b1 <= 0 || b2 >= 255 || b2 < b1) return false;
    lo = key_lo + ((uint32_t)b1 << shift);
    hi = key_lo + ((uint32_t)(b2 + 1) << shift) - 1u;
    return true;
}

// Bracket [lo, hi] (keys) known to contain the middle ranks but too many
// keys: a histogram of 256 bins over it, then the bracket of the located bins.
template <int D, int DP>
__device__ bool refine_pass(const Sm& s, int N, uint32_t lo, uint32_t hi, int r1, int r2, uint32_t& v1,
                            uint32_t& v2, int& nc, float& width) {
    int shift = 0;
    while (shift < 31 && ((hi - lo) >> shift) >= 254u) ++shift;
    uint32_t l2, h2;
    int n2;
    // key_lo one bin below lo keeps bin 0 for the keys under the range
    const uint32_t klo = lo >= (1u << shift) ? lo - (1u << shift) : 0u;
    if (!locate_pass<D, DP>(s, N, klo, shift, r1, r2, l2, h2, n2)) return false;
    width = __uint_as_float(h2) - __uint_as_float(l2);
    return bracket_pass<D, DP>(s, N, __uint_as_float(l2), __uint_as_float(h2), r1, r2, v1, v2, nc);
}

// Median of the squared pairwise distances of the particles in xs, whose
// coordinates are scaled by sqrt(s2) (so scaled distances = s2 * true ones).
// Returns the median in true units. Path: a tight bracket around the
// extrapolated previous median (usual case); at a new step, a 256-bin
// histogram over +-4 octaves of a guess locates the middle ranks (and a second
// histogram over the located bins when they hold more than kCandCap keys); an
// exact radix select is the last resort. stats (may be null): [0] bracket
// hits, [1] histogram locates, [2] radix fallbacks, [3] of [1], those that
// needed the refining second histogram.
template <int D, int DP>
__device__ float median_sqdist(const Sm& s, int N, float s2, float q_extra, MedState& st, int* stats) {
    const int P = N * (N - 1) / 2;
    const int r1 = (P & 1) ? (P - 1) / 2 : P / 2 - 1;
    const int r2 = (P & 1) ? r1 : P / 2;
    const int target = 128;   // candidates a bracket aims at
    // norms of the (scaled) particles for the pair distances; nrm is free here
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        float xi[D];
        load_row<D, DP>(s.xs, i, xi);
        float n = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) n = fmaf(xi[c], xi[c], n);
        s.nrm[i] = n;
    }
    __syncthreads();
    uint32_t v1 = 0, v2 = 0;
    int nc = 0, path = 2;
    bool refined = false;     // the located keys needed the second, refining histogram
    float width = 0.0f;       // key-value width of the bracket that succeeded
    bool done = false;
    if (st.have && !st.fresh) {
        const float g = st.med * st.trend * s2;
        const float lo = g * (1.0f - st.w), hi = g * (1.0f + st.w);
        done = bracket_pass<D, DP>(s, N, lo, hi, r1, r2, v1, v2, nc);
        width = hi - lo;
        if (done) {
            path = 0;
        } else if (nc > kCandCap && s.redi[39]) {
            // the middle ranks are inside but the bracket is too wide
            done = refine_pass<D, DP>(s, N, __float_as_uint(lo), __float_as_uint(hi), r1, r2, v1, v2, nc, width);
            if (done) { path = 1; refined = true; }
        }
    }
    if (!done) {
        float g;
        if (st.have) {
            g = (st.med + q_extra) * s2;
        } else {
            // crude guess: mean of a few pair distances
            float a = 0.0f;
            if (threadIdx.x < 32) {
                const int i = (threadIdx.x * 7) % N, k = (threadIdx.x * 13 + N / 2 + 1) % N;
                float xi[D], xk[D];
                load_row<D, DP>(s.xs, i, xi);
                load_row<D, DP>(s.xs, k, xk);
                a = sqdist<D>(xi, xk);
            }
            a = warp_sum_f(a);
            if (threadIdx.x == 0) s.redf[38] = a / 32.0f;
            __syncthreads();
            g = s.redf[38];
            __syncthreads();
        }
        if (g > 0.0f && isfinite(g)) {
            // 1/32 octave per bin, +-4 octaves around g
            const uint32_t gk = __float_as_uint(g);
            const uint32_t klo = gk > (128u << 18) ? gk - (128u << 18) : 0u;
            uint32_t lo, hi;
            int n_in;
            if (locate_pass<D, DP>(s, N, klo, 18, r1, r2, lo, hi, n_in)) {
                if (n_in <= kCandCap) {
                    done = bracket_pass<D, DP>(s, N, __uint_as_float(lo), __uint_as_float(hi), r1, r2, v1, v2, nc);
                    width = __uint_as_float(hi) - __uint_as_float(lo);
                } else {
                    done = refine_pass<D, DP>(s, N, lo, hi, r1, r2, v1, v2, nc, width);
                    refined = done;
                }
                if (done) path = 1;
            }
        }
    }
    if (!done) {
        v1 = radix_select<D, DP>(s, N, r1);
        v2 = (r2 == r1) ? v1 : radix_select<D, DP>(s, N, r2);
    }
    if (stats && threadIdx.x == 0) {
        atomicAdd(&stats[path], 1);
        if (refined) atomicAdd(&stats[3], 1);
    }
    const float med_s = 0.5f * (__uint_as_float(v1) + __uint_as_float(v2));
    const float med = med_s / s2;
    if (st.have && !st.fresh && st.med > 0.0f) st.trend = fminf(fmaxf(med / st.med, 0.8f), 1.25f);
    else st.trend = 1.0f;
    // next bracket: the width that held nc keys, scaled to hold about `target`
    if (done && nc > 0 && med_s > 0.0f)
        st.w = fminf(fmaxf(0.5f * width / med_s * fminf(fmaxf((float)target / (float)nc, 0.25f), 4.0f),
                           1e-6f), 0.05f);
    else
        st.w = 0.004f;
    st.med = med;
    st.have = 1;
    st.fresh = 0;
    return med;
}

// ---------------------------------------------------------------------------
// a1/a2: transition means of the previous set and the initial particles.
// On return (after a barrier): fs, misc (centre, fs mean), zs, f64 are set
// and xs holds the initial particles of step t (absolute FP32). first = the
// previous set is {x_0^true} (taken in FP64 from x0).
// ---------------------------------------------------------------------------
template <class M, int PPT>
__device__ void prepare_step(const ModelParams& mp, const Sm& s, int t, int N, int Np, bool first,
                             const double* x0, const float* yt, double* f64, int prior,
                             uint64_t seed, uint32_t seq, const float* xinit, bool df_means = false) {
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
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) s.misc[c] = cf[c];
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        double fd[D];
        if constexpr (M::kTransDF) {
            // the recursion alone on given sets: the recursion's double-float
            // terms read the previous set itself, so only the centred FP32
            // means of its screen are needed (no FP64 means)
            if (df_means && i < Np) {
                float xp[D], fc[D], fr[D];
                load_row<D, DP>(s.xs, i, xp);
                M::centred_mean(mp, xp, cf, fc);
#pragma unroll
                for (int c = 0; c < D; ++c) fr[c] = __fmul_rn(fc[c], mp.sqrt_qinv_f[c] * kKm);
                store_row<D, DP>(s.fs, i, fr);
                if (i < N) {
                    float xi[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) xi[c] = xinit[(size_t)i * D + c];
                    store_row<D, DP>(s.xs, i, xi);
                }
                continue;
            }
        }
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
            float fr[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                f64[(size_t)i * D + c] = fd[c];
                fr[c] = (float)((fd[c] - (double)cf[c]) * (mp.sqrt_qinv[c] * (double)kKm));
            }
            store_row<D, DP>(s.fs, i, fr);
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
            store_row<D, DP>(s.xs, i, xi);
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
// MAP-conditioned prior: per particle the predecessor j maximising
// phi_{t-1}(j) + log p(x_i | x_{t-1}^j), i.e. phf_j - |x~_i - f~_j|^2 in log2
// units (FP32, lowest j on ties), from the particles in xs at scale 1/inv_sc.
// The index goes to nrm (as an int) for rescale_and_score; a separate pass so
// that the other priors' score code keeps its registers (for wide states a
// called function: inlined, its live ranges still cost the kernel spills).
// ---------------------------------------------------------------------------
template <class M, int PPT, int TPP = 1>
__device__ __forceinline__ void mapcond_select(const ModelParams& mp, const Sm& s, int N, int Np, float inv_sc) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x / TPP, NT = blockDim.x / TPP, r = threadIdx.x % TPP;
    float xt[PPT][D], bv[PPT];
    int bj[PPT];
    float qk[D];
#pragma unroll
    for (int c = 0; c < D; ++c) qk[c] = mp.sqrt_qinv_f[c] * kKm * inv_sc;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        float xh[D];
        load_row<D, DP>(s.xs, min(tid + p * NT, N - 1), xh);
#pragma unroll
        for (int c = 0; c < D; ++c) xt[p][c] = xh[c] * qk[c];
        bv[p] = -INFINITY;
        bj[p] = 0;
    }
    for (int j = r; j < Np; j += TPP) {
        float fj[D];
        load_row<D, DP>(s.fs, j, fj);
        const float pj = s.phf[j];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const float v = pj - sqdist<D>(xt[p], fj);
            const bool nb = v > bv[p];
            bv[p] = nb ? v : bv[p];
            bj[p] = nb ? j : bj[p];
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if constexpr (TPP > 1) {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv[p], o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj[p], o);
                if (ov > bv[p] || (ov == bv[p] && oj < bj[p])) { bv[p] = ov; bj[p] = oj; }
            }
        }
        const int i = tid + p * NT;
        if (i < N && r == 0) reinterpret_cast<int*>(s.nrm)[i] = bj[p];
    }
}
template <class M, int PPT, int TPP>
__device__ __noinline__ void mapcond_select_call(const ModelParams& mp, const Sm& s, int N, int Np, float inv_sc) {
    mapcond_select<M, PPT, TPP>(mp, s, N, Np, inv_sc);
}

// ---------------------------------------------------------------------------
// a4: scores g_i = grad log p(z_t | x_i) + grad log prior(x_i) for the block's
// particles held as x^ = (x - c) * sc in xs; each particle is first rescaled
// by `rescale` (the new kernel scale over the old) and written back. What is
// stored is what the update needs: w_i = Aw g_i - Bw x^_i in gs and |x^_i|^2
// in nrm (see rbf_update). With TPP > 1 threads per particle, the lanes of a
// group split the loop over the previous set and combine by shuffles.
// ---------------------------------------------------------------------------
template <class M, int PPT, int TPP = 1>
__device__ __forceinline__ void rescale_and_score(const ModelParams& mp, const Sm& s, int N, int Np,
                                                  int prior, float rescale, float inv_sc, float Aw,
                                                  float Bw) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x / TPP, NT = blockDim.x / TPP, r = threadIdx.x % TPP;
    float xt[PPT][D], A[PPT][D], S[PPT], Mref[PPT];
    float cf[D], qk[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        cf[c] = s.misc[c];
        qk[c] = mp.sqrt_qinv_f[c] * kKm * inv_sc;   // x^ -> mixture coordinates
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        const int ii = min(i, N - 1);
        float xh[D];
        load_row<D, DP>(s.xs, ii, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xh[c] *= rescale;
            xt[p][c] = xh[c] * qk[c];
            A[p][c] = 0.0f;
        }
        if constexpr (TPP > 1) __syncwarp();   // the group has read the row before it is rewritten
        if (i < N && r == 0) store_row<D, DP>(s.xs, i, xh);
        S[p] = 0.0f;
        // reference logit: the particle's own parent in the previous set
        float fr[D];
        load_row<D, DP>(s.fs, Np == 1 ? 0 : min(ii, Np - 1), fr);
        Mref[p] = sqdist<D>(xt[p], fr);
    }
    if (prior == 2) {
        // MAP-conditioned: the predecessor chosen by mapcond_select (its index
        // is parked in nrm, which is rewritten below); its transition alone
        // gives the prior score
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int i = tid + p * NT;
            int jb = i < N ? reinterpret_cast<const int*>(s.nrm)[i] : 0;
            jb = min(max(jb, 0), Np - 1);
            float fj[D];
            load_row<D, DP>(s.fs, jb, fj);
            S[p] = 1.0f;
#pragma unroll
            for (int c = 0; c < D; ++c) A[p][c] = xt[p][c] - fj[c];
        }
    }
    if (prior == 0) {
        // mixture responsibilities w_ij = 2^(Mref - |x~_i - f~_j|^2) / sum:
        // the parent's term is 1, so the sum is >= 1; a sum above 2^100 (a
        // far better component than the parent) is redone with the true max
        for (int j = r; j < Np; j += TPP) {
            float fj[D];
            load_row<D, DP>(s.fs, j, fj);
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                float diff[D], m = Mref[p];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    diff[c] = xt[p][c] - fj[c];
                    m = fmaf(-diff[c], diff[c], m);
                }
                const float e = fast_exp2(m);
                S[p] += e;
#pragma unroll
                for (int c = 0; c < D; ++c) A[p][c] = fmaf(e, diff[c], A[p][c]);
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if constexpr (TPP > 1) {
                S[p] = group_sum<TPP>(S[p]);
#pragma unroll
                for (int c = 0; c < D; ++c) A[p][c] = group_sum<TPP>(A[p][c]);
            }
            const bool redo = !(S[p] <= 1.2676506e30f);   // 2^100, or NaN
            if constexpr (TPP == 1) {
                if (redo) {
                    float mn = INFINITY;
                    for (int j = 0; j < Np; ++j) {
                        float fj[D];
                        load_row<D, DP>(s.fs, j, fj);
                        mn = fminf(mn, sqdist<D>(xt[p], fj));
                    }
                    S[p] = 0.0f;
#pragma unroll
                    for (int c = 0; c < D; ++c) A[p][c] = 0.0f;
                    for (int j = 0; j < Np; ++j) {
                        float fj[D], diff[D], m = -mn;
                        load_row<D, DP>(s.fs, j, fj);
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            diff[c] = xt[p][c] - fj[c];
                            m = fmaf(diff[c], diff[c], m);
                        }
                        const float e = fast_exp2(-m);
                        S[p] += e;
#pragma unroll
                        for (int c = 0; c < D; ++c) A[p][c] = fmaf(e, diff[c], A[p][c]);
                    }
                }
            } else if (__any_sync(0xffffffffu, redo)) {
                // the redo path shuffles, so the whole warp enters it
                float mn = INFINITY;
                for (int j = r; j < Np; j += TPP) {
                    float fj[D];
                    load_row<D, DP>(s.fs, j, fj);
                    mn = fminf(mn, sqdist<D>(xt[p], fj));
                }
#pragma unroll
                for (int o = TPP / 2; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                float S2 = 0.0f, A2[D];
#pragma unroll
                for (int c = 0; c < D; ++c) A2[c] = 0.0f;
                for (int j = r; j < Np; j += TPP) {
                    float fj[D], diff[D], m = -mn;
                    load_row<D, DP>(s.fs, j, fj);
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        diff[c] = xt[p][c] - fj[c];
                        m = fmaf(diff[c], diff[c], m);
                    }
                    const float e = fast_exp2(-m);
                    S2 += e;
#pragma unroll
                    for (int c = 0; c < D; ++c) A2[c] = fmaf(e, diff[c], A2[c]);
                }
                S2 = group_sum<TPP>(S2);
#pragma unroll
                for (int c = 0; c < D; ++c) A2[c] = group_sum<TPP>(A2[c]);
                if (redo) {
                    S[p] = S2;
#pragma unroll
                    for (int c = 0; c < D; ++c) A[p][c] = A2[c];
                }
            }
        }
    }
    if constexpr (TPP > 1) __syncwarp();   // the group has read nrm before lane 0 rewrites it
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N || r != 0) continue;
        float x[D], g[D];
        float xh[D];
        load_row<D, DP>(s.xs, i, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = fmaf(xh[c], inv_sc, cf[c]);
        M::grad_loglik(mp, s.zs, x, g);
        // Q^-1 (f - x) = -(Q^-1/2 / kKm) (x~ - f~)
        if (prior != 1) {
            const float inv = 1.0f / S[p];
#pragma unroll
            for (int c = 0; c < D; ++c) g[c] -= mp.sqrt_qinv_f[c] * (1.0f / kKm) * A[p][c] * inv;
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c)
                g[c] -= mp.sqrt_qinv_f[c] * (1.0f / kKm) * (xt[p][c] - s.misc[16 + c]);
        }
        float n2 = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            n2 = fmaf(xh[c], xh[c], n2);
            g[c] = fmaf(Aw, g[c], -Bw * xh[c]);
        }
        store_row<D, DP>(s.gs, i, g);
        s.nrm[i] = n2;
    }
}

// ---------------------------------------------------------------------------
// a5: one SVGD update (Eq. svgd_iterate) in the scaled coordinates, where
// kappa_ik = 2^-|x^_i - x^_k|^2 and the update
//   x^_i += A sum_k kappa_ik g_k + Bc sum_k kappa_ik (x^_i - x^_k)
// (A = sc eps / N, Bc = 2 eps / (N h)) is regrouped as
//   x^_i += sum_k kappa_ik w_k + Bc x^_i sum_k kappa_ik,   w_k = A g_k - Bc x^_k,
// so a pair costs one dot product, one ex2 and d + 1 accumulations; the
// distance is |x^_i|^2 + |x^_k|^2 - 2 x^_i . x^_k, well conditioned because the
// coordinates are in units of the kernel width.
// ---------------------------------------------------------------------------
template <class M, int PPT, int TPP = 1>
__device__ __forceinline__ void rbf_update(const Sm& s, int N, float Bc) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x / TPP, NT = blockDim.x / TPP, r = threadIdx.x % TPP;
    float xi[PPT][D], ni[PPT], Sw[PPT][D], S0[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
        load_row<D, DP>(s.xs, i, xi[p]);
        ni[p] = -s.nrm[i];
        S0[p] = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xi[p][c] *= 2.0f;   // the dot product then lands as 2 x^_i . x^_k
            Sw[p][c] = 0.0f;
        }
    }
#pragma unroll 2
    for (int k = r; k < N; k += TPP) {
        float xk[D], wk[D];
        load_row<D, DP>(s.xs, k, xk);
        load_row<D, DP>(s.gs, k, wk);
        const float nk = s.nrm[k];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            float m = ni[p] - nk;   // accumulates -|x^_i - x^_k|^2
#pragma unroll
            for (int c = 0; c < D; ++c) m = fmaf(xi[p][c], xk[c], m);
            const float kap = fast_exp2(m);
            S0[p] += kap;
#pragma unroll
            for (int c = 0; c < D; ++c) Sw[p][c] = fmaf(kap, wk[c], Sw[p][c]);
        }
    }
    if constexpr (TPP > 1) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            S0[p] = group_sum<TPP>(S0[p]);
#pragma unroll
            for (int c = 0; c < D; ++c) Sw[p][c] = group_sum<TPP>(Sw[p][c]);
        }
    }
    __syncthreads();   // every thread is done reading xs / gs / nrm
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N || r != 0) continue;
        const float cx = 0.5f * fmaf(Bc, S0[p], 1.0f);
        float xn[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xn[c] = fmaf(cx, xi[p][c], Sw[p][c]);
        store_row<D, DP>(s.xs, i, xn);
    }
    __syncthreads();
}

// a5 for the other Stein kernels of the kernel ablation (Table Ex6), as
// functions of u = r^2 / h = |x^_i - x^_k|^2 ln 2:
//   KER 1, IMQ         kappa = (1 + u)^-1/2,            repulsion weight kappa^3
//   KER 2, Matern 3/2  kappa = (1 + s) e^-s, s = sqrt(3u), repulsion weight e^-s
// The drive (gs = A g_k) and the repulsion Bk (x^_i sum rho - sum rho x^_k)
// accumulate separately, their weights differing.
template <class M, int PPT, int KER, int TPP = 1>
__device__ __forceinline__ void kernel_update(const Sm& s, int N, float Bk) {
    constexpr int D = M::D, DP = M::DP;
    constexpr float kLn2 = 0.6931471805599453f;
    const int tid = threadIdx.x / TPP, NT = blockDim.x / TPP, r = threadIdx.x % TPP;
    float xi[PPT][D], ni[PPT], Sg[PPT][D], Sx[PPT][D], Sr[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
        load_row<D, DP>(s.xs, i, xi[p]);
        ni[p] = -s.nrm[i];
        Sr[p] = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xi[p][c] *= 2.0f;
            Sg[p][c] = 0.0f;
            Sx[p][c] = 0.0f;
        }
    }
#pragma unroll 2
    for (int k = r; k < N; k += TPP) {
        float xk[D], gk[D];
        load_row<D, DP>(s.xs, k, xk);
        load_row<D, DP>(s.gs, k, gk);
        const float nk = s.nrm[k];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            float m = ni[p] - nk;   // -|x^_i - x^_k|^2
#pragma unroll
            for (int c = 0; c < D; ++c) m = fmaf(xi[p][c], xk[c], m);
            const float u = fmaxf(-m, 0.0f) * kLn2;
            float kap, rho;
            if constexpr (KER == 1) {
                kap = rsqrtf(1.0f + u);
                rho = kap * kap * kap;
            } else {
                const float sq = sqrtf(3.0f * u);
                rho = fast_exp2(-sq * kL2E);
                kap = fmaf(sq, rho, rho);
            }
            Sr[p] += rho;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                Sg[p][c] = fmaf(kap, gk[c], Sg[p][c]);
                Sx[p][c] = fmaf(rho, xk[c], Sx[p][c]);
            }
        }
    }
    if constexpr (TPP > 1) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            Sr[p] = group_sum<TPP>(Sr[p]);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                Sg[p][c] = group_sum<TPP>(Sg[p][c]);
                Sx[p][c] = group_sum<TPP>(Sx[p][c]);
            }
        }
    }
    __syncthreads();   // every thread is done reading xs / gs / nrm
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N || r != 0) continue;
        float xn[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float x = 0.5f * xi[p][c];
            xn[c] = x + Sg[p][c] + Bk * fmaf(x, Sr[p], -Sx[p][c]);
        }
        store_row<D, DP>(s.xs, i, xn);
    }
    __syncthreads();
}

// a3..a6: L iterations on the absolute particles in xs (left absolute on
// return). hout (may be null) receives h per iteration.
template <class M, int PPT, int TPP = 1>
__device__ void svgd_iterations(const ModelParams& mp, const Sm& s, int N, int Np, int L, float eps,
                                int bw_rule, float bw_value, int prior, MedState& st, float q_extra,
                                float* hout, int* stats, int kernel) {
    constexpr int D = M::D, DP = M::DP;
    if (L <= 0) return;
    const int tid = threadIdx.x, NT = blockDim.x;
    float cf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) cf[c] = s.misc[c];
    if (prior == 2) {
        // the previous scores relative to their maximum, in log2 units
        double pmax = -INFINITY;
        for (int j = tid; j < Np; j += NT) pmax = fmax(pmax, s.phis[j]);
        pmax = block_max_d(pmax, s.redd);
        for (int j = tid; j < Np; j += NT) s.phf[j] = (float)((s.phis[j] - pmax) * 1.4426950408889634);
    }
    // centre (scale 1)
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) continue;
        float xr[D];
        load_row<D, DP>(s.xs, i, xr);
#pragma unroll
        for (int c = 0; c < D; ++c) xr[c] -= cf[c];
        store_row<D, DP>(s.xs, i, xr);
    }
    __syncthreads();
    float sc = 1.0f;   // current scale of xs
    float h = 1.0f;
    for (int l = 0; l < L; ++l) {
        if (bw_rule == 2) {
            h = bw_value;
        } else if (bw_rule == 0 || l == 0) {
            if (N < 2) {
                h = 1.0f;
            } else {
                const float med = median_sqdist<D, DP>(s, N, sc * sc, q_extra, st, stats);
                h = (med > 0.0f) ? bw_value * med / logf((float)N) : 1.0f;
            }
        }
        if (hout && tid == 0) hout[l] = h;
        const float sc_new = sqrtf(kL2E / h);
        const float A = sc_new * eps / (float)N;
        const float Bc = 2.0f * eps / ((float)N * h);
        // RBF: the update is regrouped around w_k = A g_k - Bc x^_k; the
        // other kernels keep A g_k and add their repulsion separately
        if (prior == 2) {
            if constexpr (D >= 8) mapcond_select_call<M, PPT, TPP>(mp, s, N, Np, 1.0f / sc);
            else mapcond_select<M, PPT, TPP>(mp, s, N, Np, 1.0f / sc);
            __syncthreads();
        }
        rescale_and_score<M, PPT, TPP>(mp, s, N, Np, prior, sc_new / sc, 1.0f / sc_new, A, kernel == 0 ? Bc : 0.0f);
        sc = sc_new;
        __syncthreads();
        if (kernel == 1) kernel_update<M, PPT, 1, TPP>(s, N, eps / ((float)N * h));
        else if (kernel == 2) kernel_update<M, PPT, 2, TPP>(s, N, 3.0f * eps / ((float)N * h));
        else rbf_update<M, PPT, TPP>(s, N, Bc);
    }
    // back to absolute coordinates
    const float inv = 1.0f / sc;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) continue;
        float xr[D];
        load_row<D, DP>(s.xs, i, xr);
#pragma unroll
        for (int c = 0; c < D; ++c) xr[c] = fmaf(xr[c], inv, cf[c]);
        store_row<D, DP>(s.xs, i, xr);
    }
    __syncthreads();
}

// |x - f|^2_{Q^-1} in FP64 for an FP32 particle x and an FP64 mean f.
template <int D>
__device__ __forceinline__ double trans_m64(const ModelParams& mp, const float* x, const double* f) {
    double m64 = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double e = (double)x[c] - f[c];
        m64 += e * e * mp.qinv[c];
    }
    return m64;
}

// Two FP32 lanes in one 64-bit register: the packed FMA (fma.rn.f32x2) rounds
// each lane exactly as fmaf does, in one issue slot.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// max(a, b, c) in one instruction (a NaN operand is ignored, as by fmaxf).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ---------------------------------------------------------------------------
// a7: forward recursion. The argmax over j of phi_{t-1}(j) + log p(x_i | x^j)
// is screened in FP32 with a rigorous rounding bound, and every j that can
// still be the FP64 maximum is evaluated in FP64; phi_t is accumulated in
// FP64. Lowest j wins ties.
//
// Screen (dot-product form). With X_i = (x_i - c) Q^-1/2 and Y_j = (f_j - c)
// Q^-1/2 the score is, up to a term of i alone,
//   S_ij = A_j + X_i . Y_j,   A_j = phi_{t-1}(j) - max_k phi_{t-1}(k) - |Y_j|^2 / 2,
// so one pair costs d FMAs of x~ = kKm X against g = kLam f~ = Y / kKm (x~ . g
// = X . Y, as kKm^2 kLam = 1) plus the running top two. Rounding (u = 2^-24,
// first order): the FP32 scale qk = sqrt(Q^-1) kKm carries 2.5u, x~ and f~
// each two roundings (f~ is rounded from FP64, or from the double-float
// centred mean of the recursion-only path), g one more, and kKm^2 kLam differs
// from 1 by 1.5u, so x~ . g is within 11.5u |X_i| |Y_j| of X . Y; A_j in FP32
// from the FP32 phi~ and f~ is within (d + 12.5) u H_j of the exact value,
// H_j = |phi~_j| + kLam |f~_j|^2 / 2; the start value aU_j = A_j + e_j adds
// u (H_j + e_j); the FMA chain adds d u (|aU_j| + |x~_i| |g_j|). With
// e_j = (2d + 14) u H_j (1.01) plus a margin for the rounding of the exact
// evaluation (2^-46 of the magnitudes involved), and
// E_i = (d + 12) u |x~_i| max_j |g_j| (1.01) (plus the same margin), the
// computed chain v_ij satisfies
//   v_ij - 2 e_j - E_i <= S_ij <= v_ij + E_i.
// So with v1 = max_j v_ij at j1 (first j attaining it) and v2 the largest v_ij
// of every other j, v1 - v2 > 2 e_j1 + 2 E_i proves j1 the unique maximum of
// S (and of its FP64 evaluation). Otherwise (a near-tie) every j with
// v_ij >= v1 - 2 e_j1 - 2 E_i is evaluated in FP64, lowest j first.
// FP64 scores: phi_t(i) = log p(z_t | x_i) + log p(x_i | x_{t-1}^j) +
// phi_{t-1}(j), accumulated in FP64. The two log-density terms are evaluated
// in double-float arithmetic (about 48 bits, on the FP32 pipe) where the model
// provides it and the previous set xprev (FP32, global [Np][D]) is given;
// otherwise in FP64 from the FP64 transition means f64.
// On return: best[p], phinew[p] for the block's particles. fs is overwritten
// (g_j replaces f~_j).
// ---------------------------------------------------------------------------
template <class M, int PPT, bool kPaired>
__device__ void viterbi_step(const ModelParams& mp, const Sm& s, int N, int Np, const double* f64,
                             const float* xprev, int* best, double* phinew,
                             unsigned long long* rcnt = nullptr) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    constexpr float u = 5.9604644775390625e-08f;   // 2^-24
    constexpr float Ke = (2 * D + 14) * u * 1.01f;  // e_j per unit of H_j
    constexpr float Ki = (D + 12) * u * 1.01f;      // E_i per unit of |x~_i| max |g|
    constexpr float K64 = 1.4210854715202004e-14f;  // 2^-46: margin of the exact scores
    double pmax = -INFINITY;
    for (int j = tid; j < Np; j += NT) pmax = fmax(pmax, s.phis[j]);
    pmax = block_max_d(pmax, s.redd);
    // FP32 magnitudes for the margin of the exact scores: |phi_j| <= |phi~_j| + |max|
    const float mag0 = 2.0f * fabsf((float)pmax) + fabsf(mp.ltc[0]);
    // Per predecessor: aU_j (start of the chain), 2 e_j and g_j = kLam f~_j
    // (which replaces f~_j in fs once every row has been read). Two layouts:
    //   kPaired = false: (aU_j, 2 e_j) pairs in gs, g_j rows [j][DP] in fs;
    //   kPaired = true:  predecessor pairs (2q, 2q+1) interleaved per
    //     coordinate, g as [q][c][2] in fs and aU as [q][2] in gs, each with a
    //     pad after every chunk of kRecPairs pairs; 2 e_j after the aU pairs.
    const int nq = rec_pairs(Np);
    float* const aUa = s.gs;
    float* const wa = kPaired ? s.gs + 2 * (nq + rec_chunks(Np)) : s.gs + 1;
    auto aidx = [&](int j) { return kPaired ? 2 * rec_arow(j >> 1) + (j & 1) : 2 * j; };
    auto widx = [&](int j) { return kPaired ? j : 2 * j; };
    auto gidx = [&](int j, int c) { return kPaired ? 2 * (rec_grow(j >> 1, DP) + c) + (j & 1) : j * DP + c; };
    float gmax2 = 0.0f;
    float gown[PPT][D];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int j = tid + k * NT;
        if (j >= Np) continue;
        const double dphi = s.phis[j] - pmax;
        const float ph = (float)dphi;
        float fr[D];
        load_row<D, DP>(s.fs, j, fr);
        float F = 0.0f, G = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            F = fmaf(fr[c], fr[c], F);
            gown[k][c] = fr[c] * kLam;
            G = fmaf(gown[k][c], gown[k][c], G);
        }
        gmax2 = fmaxf(gmax2, G);
        const float half = 0.5f * kLam * F;
        const float H = fabsf(ph) + half;
        const float e = Ke * H + K64 * (fabsf(ph) + mag0 + kLam * F);
        aUa[aidx(j)] = (ph - half) + e;
        wa[widx(j)] = 2.0f * e;
        if constexpr (!kPaired) store_row<D, DP>(s.fs, j, gown[k]);   // the thread's own row
    }
    const float gmax = sqrtf(block_max_f(gmax2, s.redf)) * 1.0000005f;   // its barriers: every fs row read
    if constexpr (kPaired) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int j = tid + k * NT;
            if (j >= Np) continue;
#pragma unroll
            for (int c = 0; c < D; ++c) s.fs[gidx(j, c)] = gown[k][c];
        }
        if (tid == 0 && (Np & 1)) {   // the pad predecessor: never above any other
            aUa[aidx(Np)] = -INFINITY;
#pragma unroll
            for (int c = 0; c < D; ++c) s.fs[gidx(Np, c)] = 0.0f;
        }
        __syncthreads();
    }
    float xc[PPT][D], Ei[PPT];
    float cf[D], qk[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        cf[c] = s.misc[c];
        qk[c] = mp.sqrt_qinv_f[c] * kKm;
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = min(tid + p * NT, N - 1);
        float xr[D];
        load_row<D, DP>(s.xs, i, xr);
        float X = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xc[p][c] = (xr[c] - cf[c]) * qk[c];
            X = fmaf(xc[p][c], xc[p][c], X);
        }
        Ei[p] = Ki * sqrtf(X) * 1.0000005f * gmax + K64 * kLam * X;
    }
    // The FP32 pass: per particle the largest chain value v1, the first j1
    // reaching it, and the largest value v2 of every other j.
    float v1[PPT], v2[PPT];
    int j1[PPT];
    if constexpr (!kPaired) {
        // One chain per predecessor, the running top two (three min/max per
        // pair), and the chunk of 32 predecessors in which v1 was first
        // reached; that chunk is then scanned again for the first j whose
        // chain value (computed the same way, so bit-identical) equals v1.
        constexpr int kChunk = 32;
        const float2* ab = reinterpret_cast<const float2*>(aUa);
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            v1[p] = -INFINITY;
            v2[p] = -INFINITY;
            j1[p] = 0;
        }
        for (int j0 = 0; j0 < Np; j0 += kChunk) {
            float vb[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) vb[p] = v1[p];
            const int je = min(j0 + kChunk, Np);
            for (int j = j0; j < je; ++j) {
                float gj[D];
                load_row<D, DP>(s.fs, j, gj);
                const float aU = ab[j].x;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    float v = aU;
#pragma unroll
                    for (int c = 0; c < D; ++c) v = fmaf(xc[p][c], gj[c], v);
                    const float lo = fminf(v1[p], v);
                    v1[p] = fmaxf(v1[p], v);
                    v2[p] = fmaxf(v2[p], lo);
                }
            }
#pragma unroll
            for (int p = 0; p < PPT; ++p) j1[p] = v1[p] > vb[p] ? j0 : j1[p];
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int j0 = j1[p], je = min(j0 + kChunk, Np);
            for (int j = j0; j < je; ++j) {
                float gj[D];
                load_row<D, DP>(s.fs, j, gj);
                float v = ab[j].x;
#pragma unroll
                for (int c = 0; c < D; ++c) v = fmaf(xc[p][c], gj[c], v);
                if (v == v1[p]) {
                    j1[p] = j;
                    break;
                }
            }
        }
    } else {
        // Predecessor pairs: one packed FMA advances the chains of j and j + 1
        // together, and a three-input max keeps the largest chain value of the
        // chunk (kRecPairs pairs). Over the chunks each particle keeps the
        // largest value (v1), the first chunk reaching it, and the largest
        // value c2 of every other chunk. The chunk of v1 is then scanned again
        // (the same packed chains, so bit-identical values) for the first j
        // whose value equals v1 and the largest value of its other members.
        float c2[PPT];
        unsigned long long xd[PPT][D];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            v1[p] = -INFINITY;
            c2[p] = -INFINITY;
            j1[p] = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) xd[p][c] = pk2(xc[p][c], xc[p][c]);
        }
        const unsigned long long* g2 = reinterpret_cast<const unsigned long long*>(s.fs);
        const unsigned long long* a2 = reinterpret_cast<const unsigned long long*>(aUa);
        // the g row of pair q of a chunk (DP words, 16-byte aligned when DP is even)
        auto load_g = [&](const unsigned long long* gq, unsigned long long* gp) {
            if constexpr (DP % 2 == 0) {
#pragma unroll
                for (int c = 0; c < D; c += 2) {
                    const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(gq + c);
                    gp[c] = w.x;
                    if (c + 1 < D) gp[c + 1] = w.y;
                }
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) gp[c] = gq[c];
            }
        };
        for (int q0 = 0; q0 < nq; q0 += kRecPairs) {
            const unsigned long long* gq = g2 + rec_grow(q0, DP);
            const unsigned long long* aq = a2 + rec_arow(q0);
            float cm[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) cm[p] = -INFINITY;
            auto pair_step = [&](int t) {
                unsigned long long gp[D];
                load_g(gq + t * DP, gp);
                const unsigned long long aU = aq[t];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    unsigned long long v = aU;
#pragma unroll
                    for (int c = 0; c < D; ++c) v = ffma2(xd[p][c], gp[c], v);
                    float va, vz;
                    upk2(v, va, vz);
                    cm[p] = fmax3(cm[p], va, vz);
                }
            };
            const int n = min(kRecPairs, nq - q0);
            if (n == kRecPairs) {
#pragma unroll 4
                for (int t = 0; t < kRecPairs; ++t) pair_step(t);
            } else {
                for (int t = 0; t < n; ++t) pair_step(t);
            }
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float lo = fminf(v1[p], cm[p]);
                j1[p] = cm[p] > v1[p] ? q0 : j1[p];
                v1[p] = fmaxf(v1[p], cm[p]);
                c2[p] = fmaxf(c2[p], lo);
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int q0 = j1[p], n = min(kRecPairs, nq - q0);
            const unsigned long long* gq = g2 + rec_grow(q0, DP);
            const unsigned long long* aq = a2 + rec_arow(q0);
            float s2 = -INFINITY;
            int jj = -1;
            for (int t = 0; t < n; ++t) {
                unsigned long long gp[D];
                load_g(gq + t * DP, gp);
                unsigned long long v = aq[t];
#pragma unroll
                for (int c = 0; c < D; ++c) v = ffma2(xd[p][c], gp[c], v);
                float va, vz;
                upk2(v, va, vz);
                if (jj < 0 && va == v1[p]) jj = 2 * (q0 + t);
                else s2 = fmaxf(s2, va);
                if (jj < 0 && vz == v1[p]) jj = 2 * (q0 + t) + 1;
                else s2 = fmaxf(s2, vz);
            }
            j1[p] = jj < 0 ? 2 * q0 : jj;
            v2[p] = fmaxf(c2[p], s2);
        }
    }
    // candidate threshold: v_ij >= v1 - 2 e_j1 - 2 E_i can still be the maximum
    float thr[PPT];
    bool uniq[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const float m = (wa[widx(j1[p])] + 2.0f * Ei[p]) * 1.0000005f;
        uniq[p] = (v1[p] - v2[p]) > m;
        thr[p] = v1[p] - m;
    }
    // log p(x_i | x_{t-1}^j) of the particle at row r of xs
    auto logtrans = [&](int r, int j) -> double {
        if constexpr (M::kTransDF) {
            if (xprev && SMAP_DBG(j >= 0 && j < Np, kDbgPrev, j)) {
                const df::F q = M::trans_sq_df(mp, s.xs + r, xprev + (size_t)j * D);
                return df::to_double(df::add(df::make(mp.ltc[0], mp.ltc[1]), df::scale2(q, -0.5f)));
            }
        }
        return mp.logtrans_c - 0.5 * trans_m64<D>(mp, s.xs + r, f64 + (size_t)j * D);
    };
    double bs[PPT], blt[PPT];
    int row[PPT];
    bool multi = false;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        row[p] = min(tid + p * NT, N - 1) * DP;
        bs[p] = -INFINITY;
        blt[p] = 0.0;
        best[p] = 0;
        if (uniq[p]) {
            const int j = j1[p];
            blt[p] = logtrans(row[p], j);
            bs[p] = s.phis[j] + blt[p];
            best[p] = j;
        } else {
            multi = true;
            if (rcnt && tid + p * NT < N) atomicAdd(&rcnt[1], 1ull);
        }
    }
    if (__any_sync(0xffffffffu, multi)) {
        // near-ties (rare): the warp takes each such particle in turn, its 32
        // lanes splitting the predecessors; every candidate is scored exactly
        // and the warp keeps the largest score (lowest j on ties)
        const int lane = tid & 31;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            unsigned m = __ballot_sync(0xffffffffu, !uniq[p] && tid + p * NT < N);
            while (m) {
                const int L = __ffs(m) - 1;
                m &= m - 1;
                float xb[D];
#pragma unroll
                for (int c = 0; c < D; ++c) xb[c] = __shfl_sync(0xffffffffu, xc[p][c], L);
                const float tb = __shfl_sync(0xffffffffu, thr[p], L);
                const int rb = __shfl_sync(0xffffffffu, row[p], L);
                double bsv = -INFINITY, blv = 0.0;
                int bj = 0x7fffffff;
                for (int j = lane; j < Np; j += 32) {
                    float v = aUa[aidx(j)];
#pragma unroll
                    for (int c = 0; c < D; ++c) v = fmaf(xb[c], s.fs[gidx(j, c)], v);
                    if (v >= tb) {
                        const double lt = logtrans(rb, j);
                        if (rcnt) atomicAdd(&rcnt[2], 1ull);
                        const double sv = s.phis[j] + lt;
                        if (sv > bsv) { bsv = sv; blv = lt; bj = j; }
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const double osv = __shfl_xor_sync(0xffffffffu, bsv, o);
                    const double olv = __shfl_xor_sync(0xffffffffu, blv, o);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (osv > bsv || (osv == bsv && oj < bj)) { bsv = osv; blv = olv; bj = oj; }
                }
                if (lane == L && bsv > -INFINITY) {
                    bs[p] = bsv;
                    blt[p] = blv;
                    best[p] = bj;
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (bs[p] == -INFINITY) {
            // no candidate passed the screen (non-finite inputs): plain FP64 scan
            for (int j = 0; j < Np; ++j) {
                const double lt = logtrans(row[p], j);
                const double sv = s.phis[j] + lt;
                if (sv > bs[p]) { bs[p] = sv; blt[p] = lt; best[p] = j; }
            }
            if (bs[p] == -INFINITY) {
                // no finite candidate at all: predecessor 0, scored with its
                // own (non-finite) transition term, so the score is not finite
                best[p] = 0;
                blt[p] = logtrans(row[p], 0);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) { phinew[p] = 0.0; continue; }
        double ll;
        if constexpr (M::kLikDF) {
            ll = df::to_double(M::loglik_df(mp, s.zs, s.xs + row[p]));
        } else {
            double xd[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xd[c] = (double)s.xs[row[p] + c];
            ll = M::loglik64(mp, s.zs, xd);
        }
        phinew[p] = ll + blt[p] + s.phis[best[p]];
    }
    if (rcnt && tid == 0) rcnt[0] += (unsigned long long)N;
}

// Extra squared-distance spread the initial noise adds: 2 sum_d q_d.
__device__ inline float init_spread(const ModelParams& mp) {
    float v = 0.0f;
    for (int c = 0; c < mp.d; ++c) v += (float)mp.q[c];
    return 2.0f * v;
}

// ---------------------------------------------------------------------------
// The persistent sequence kernel.
// ---------------------------------------------------------------------------
template <class M, int PPT, int MAXT, int MINB, int TPP = 1>
__global__ void __launch_bounds__(MAXT, MINB) seq_kernel(const __grid_constant__ SeqArgs a) {
    constexpr int D = M::D, DP = M::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sm s = bind_smem(smem_raw, a.Nmax, DP);
    SMAP_DBG_BEGIN(a.Nmax, a.stats ? a.stats + kDbgWord : nullptr);
    const ModelParams& mp = a.mp;
    const int tid = threadIdx.x, NT = blockDim.x;
    __shared__ int s_item;
    double* f64 = a.f64 + (size_t)blockIdx.x * a.Nmax * D;
    const float q_extra = init_spread(mp);
    // recursion counters of the block (shared, so that nothing stays live in
    // registers across the persistent loop): particle-steps, near-ties,
    // exact scores beyond one per particle
    __shared__ unsigned long long s_rcnt[3];
    if (tid < 3) s_rcnt[tid] = 0ull;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.B) break;
        const int b = a.order ? a.order[item] : a.seq_base + item;
        if (!SMAP_DBG(b >= 0 && b < a.Btot, kDbgSeq, b)) continue;
        if (a.mode == 1 && a.active && !a.active[b]) continue;
        if (a.status[b] != 0) continue;
        const int N = a.Nseq[b];
        const int t0 = a.tcur[b];
        if (a.mode == 1 && a.skip_done && t0 >= a.Tend[b]) continue;
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
        MedState st;
        st.med = a.bwguess[b];
        st.have = (t0 > 0) && st.med > 0.0f;
        st.trend = 1.0f;
        st.w = 0.004f;
        st.fresh = 1;
        int tdone = t0;
        __syncthreads();
        for (int t = t0 + 1; t <= t1; ++t) {
            const float* yt = (a.mode == 1 && !a.y_full) ? a.y + (size_t)b * mp.dy
                                                         : a.y + ((size_t)b * a.maxT + (t - 1)) * mp.dy;
            const float* xin = a.viterbi_only
                                   ? a.hist + (((size_t)b * a.maxT + (t - 1)) * a.Nmax) * D
                                   : (a.xinit ? a.xinit + (size_t)b * a.Nmax * D : nullptr);
            prepare_step<M, PPT>(mp, s, t, N, Np, t == 1, a.x0 + (size_t)b * D, yt, f64, a.prior,
                                 a.seed, (uint32_t)b, xin, a.viterbi_only && t >= 2);
            if (!a.viterbi_only) {
                st.fresh = 1;
                svgd_iterations<M, PPT, TPP>(mp, s, N, Np, a.L, a.eps, a.bw_rule, a.bw_value, a.prior, st,
                                             q_extra, nullptr, a.stats, a.kernel);
            }
            int best[PPT];
            double phinew[PPT];
            if (!SMAP_DBG(t >= 1 && t <= a.maxT, kDbgStep, t)) break;
            const float* xprev = (t >= 2) ? a.hist + (((size_t)b * a.maxT + (t - 2)) * a.Nmax) * D : nullptr;
            viterbi_step<M, PPT, false>(mp, s, N, Np, f64, xprev, best, phinew, s_rcnt);
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
            a.bwguess[b] = st.have ? st.med : 0.0f;
        }
    }
    __syncthreads();
    if (a.rstats && tid < 3 && s_rcnt[tid]) atomicAdd(&a.rstats[tid], s_rcnt[tid]);
}

// ---------------------------------------------------------------------------
// The forward recursion and its stores alone, on given particle sets (hist
// holds x_t of every step): persistent CTAs over the same work queue as the
// step kernel, the previous set resident in shared memory, the screen of
// viterbi_step in its paired form. On return phi, psi, tcur of every
// sequence are those of the whole sequence (status 6 where a score is not
// finite), exactly as the step kernel's recursion-only mode leaves them.
// ---------------------------------------------------------------------------
template <class M, int PPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) rec_kernel(const __grid_constant__ SeqArgs a) {
    constexpr int D = M::D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sm s = bind_smem_at(smem_raw, rec_smem_layout(a.Nmax, M::DP));
    SMAP_DBG_BEGIN(a.Nmax, a.stats ? a.stats + kDbgWord : nullptr);
    const ModelParams& mp = a.mp;
    const int tid = threadIdx.x, NT = blockDim.x;
    __shared__ int s_item;
    double* f64 = a.f64 + (size_t)blockIdx.x * a.Nmax * D;
    __shared__ unsigned long long s_rcnt[3];
    if (tid < 3) s_rcnt[tid] = 0ull;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.B) break;
        const int b = a.order ? a.order[item] : a.seq_base + item;
        if (!SMAP_DBG(b >= 0 && b < a.Btot, kDbgSeq, b)) continue;
        if (a.status[b] != 0) continue;
        const int N = a.Nseq[b], T = a.Tend[b];
        if (T > a.maxT || N < 1 || N > a.Nmax) {
            if (tid == 0) a.status[b] = 1;
            continue;
        }
        if (tid == 0) s.phis[0] = 0.0;
        int Np = 1, tdone = 0;
        __syncthreads();
        for (int t = 1; t <= T; ++t) {
            if (!SMAP_DBG(t <= a.maxT, kDbgStep, t)) break;
            const size_t row = (size_t)b * a.maxT + (t - 1);
            const float* xt = a.hist + row * a.Nmax * D;
            prepare_step<M, PPT>(mp, s, t, N, Np, t == 1, a.x0 + (size_t)b * D, a.y + row * mp.dy, f64, 0,
                                 a.seed, (uint32_t)b, xt, t >= 2);
            int best[PPT];
            double phinew[PPT];
            const float* xprev = (t >= 2) ? xt - (size_t)a.Nmax * D : nullptr;
            viterbi_step<M, PPT, true>(mp, s, N, Np, f64, xprev, best, phinew, s_rcnt);
            __syncthreads();   // all reads of phis / xs done
            bool bad = false;
            uint16_t* pdst = a.psi + row * a.Nmax;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const int i = tid + p * NT;
                if (i >= N) continue;
                s.phis[i] = phinew[p];
                bad |= !isfinite(phinew[p]);
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
            a.bwguess[b] = 0.0f;
        }
    }
    __syncthreads();
    if (a.rstats && tid < 3 && s_rcnt[tid]) atomicAdd(&a.rstats[tid], s_rcnt[tid]);
}

// Debug: n iterations of SVGD from given particles (one CTA per sequence).
template <class M, int PPT, int MAXT, int MINB, int TPP = 1>
__global__ void __launch_bounds__(MAXT, MINB) debug_svgd_kernel(const __grid_constant__ DebugSvgdArgs a) {
    constexpr int D = M::D, DP = M::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Nmax = a.N > a.Np ? a.N : a.Np;
    const Sm s = bind_smem(smem_raw, Nmax, DP);
    SMAP_DBG_BEGIN(Nmax, a.stats ? a.stats + kDbgWord : nullptr);
    const int b = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    const bool first = (a.t == 1 && a.Np == 1);
    // the previous set goes through xs (prepare_step reads it there)
    const float* xp = a.xprev + (size_t)b * a.Np * D;
    for (int e = tid; e < a.Np * D; e += NT) s.xs[(e / D) * DP + (e % D)] = xp[e];
    for (int j = tid; j < a.Np; j += NT) s.phis[j] = a.phiprev ? a.phiprev[(size_t)b * a.Np + j] : 0.0;
    __syncthreads();
    prepare_step<M, PPT>(a.mp, s, a.t, a.N, a.Np, first, a.x0 + (size_t)b * D, a.y + (size_t)b * a.mp.dy,
                         a.f64 + (size_t)b * a.Np * D, a.prior, 0, 0,
                         a.xinit + (size_t)b * a.N * D);
    MedState st;
    st.med = 0.0f;
    st.have = 0;
    st.trend = 1.0f;
    st.w = 0.004f;
    st.fresh = 1;
    svgd_iterations<M, PPT, TPP>(a.mp, s, a.N, a.Np, a.iters, a.eps, a.bw_rule, a.bw_value, a.prior, st,
                            init_spread(a.mp), a.hout ? a.hout + (size_t)b * a.iters : nullptr, a.stats, a.kernel);
    for (int e = tid; e < a.N * D; e += NT)
        a.xout[(size_t)b * a.N * D + e] = s.xs[(e / D) * DP + (e % D)];
}

}  // namespace smap
