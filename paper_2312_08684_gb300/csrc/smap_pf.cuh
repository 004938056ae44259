// smap_pf.cuh -- PF-MAP-Seq, the particle-filter comparison method of the
// paper's Section V (Godsill, Doucet and West 2001): a bootstrap particle
// filter with stratified resampling at every step supplies the particle sets,
// and the same forward recursion (Eq. forward_recursion) and backtracking as
// Stein-MAP-Seq pick the MAP sequence over them.
//
// One CTA per sequence, persistent over a work queue, like seq_kernel. Per
// step t (readings, the same as the oracle's):
//   x_1^i = f_1(x_0) + sqrt(q) (.) xi_i;
//   t >= 2: normalised cumulative weights C_j of step t-1, u_i = (i + U_i)/N,
//   ancestor a_i = first j with C_j > u_i, x_t^i = f_t(x_{t-1}^{a_i}) +
//   sqrt(q) (.) xi_i;  log w_t^i = log p(z_t | x_t^i).
// The filter runs in FP64 (particles, weights, cumulative sums, Box-Muller
// normals from the same Philox words as the oracle), so the integer decisions
// of the resampling are taken in the oracle's precision; only the summation
// order of the cumulative weights differs (a parallel scan). The recursion
// sees FP32 copies of the particles, as it does for the Stein sets.
#pragma once

#include "smap_kernels.cuh"

namespace smap {

struct PfArgs {
    ModelParams mp;
    int B, Nmax, maxT;
    uint64_t seed;
    const float* y;           // [B][maxT][dy]
    const double* x0;         // [B][d]
    float* hist;              // [B][maxT][Nmax][d]  FP32 copies of the particle sets
    uint16_t* psi;            // [B][maxT][Nmax]
    double* phi;              // [B][Nmax]
    int* tcur;                // [B]
    const int* Nseq;          // [B]
    const int* Tend;          // [B]
    const int* order;         // [B] processing order
    double* f64;              // [gridDim][Nmax][d] FP64 transition means of the previous set
    double* x64;              // [gridDim][Nmax][d] FP64 particle set of the current step
    double* lw;               // [gridDim][Nmax] log-weights of the current step
    int* status;              // [B]
    int* queue;               // [1]
};

// d standard normals in FP64 from the Philox words of counter (i, t, seq, block).
template <int D>
__device__ inline void draw_normals64(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i, double* z) {
#pragma unroll
    for (int b = 0; 4 * b < D; ++b) {
        uint32_t w[4];
        philox4x32_10(i, t, seq, (uint32_t)b, (uint32_t)seed, (uint32_t)(seed >> 32), w);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double u1 = ((double)w[2 * h] + 0.5) * (1.0 / 4294967296.0);
            const double u2 = ((double)w[2 * h + 1] + 0.5) * (1.0 / 4294967296.0);
            const double rad = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);   // the angle 2 pi u2 without a pi-sized range reduction
            const int k0 = 4 * b + 2 * h;
            if (k0 < D) z[k0] = rad * cs;
            if (k0 + 1 < D) z[k0 + 1] = rad * sn;
        }
    }
}

// U_i of the stratified resampling: counter (i, t, seq, 256), first word.
__device__ inline double draw_uniform64(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i) {
    uint32_t w[4];
    philox4x32_10(i, t, seq, 256u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    return ((double)w[0] + 0.5) * (1.0 / 4294967296.0);
}

// Exclusive prefix sum of one double per thread over the block; red: >= 34
// doubles. Every thread of the block must call.
__device__ inline double block_exclusive_scan_d(double v, double* red, double* total) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    __syncthreads();
    if (lane == 31) red[w] = incl;
    __syncthreads();
    if (w == 0) {
        double si = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double n = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += n;
        }
        double se = __shfl_up_sync(0xffffffffu, si, 1);
        if (lane == 0) se = 0.0;
        if (lane < nw) red[lane] = se;      // exclusive prefix of the warp totals
        if (lane == 31) red[33] = si;
    }
    __syncthreads();
    const double r = red[w] + excl;
    *total = red[33];
    __syncthreads();
    return r;
}

// The particle set of step t (bootstrap proposal after stratified resampling)
// into x64 / xs, the previous set's transition means into f64 / fs, and the
// new log-weights into lw.
template <class M, int PPT>
__device__ void pf_prepare_step(const ModelParams& mp, const Sm& s, int t, int N, int Np, const double* x0,
                                const float* yt, double* f64, double* x64, double* lw, uint64_t seed,
                                uint32_t seq) {
    constexpr int D = M::D, DP = M::DP;
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int c = tid; c < mp.dy; c += NT) s.zs[c] = yt[c];
    const double sc = M::step_const(mp, t);
    double f0[D];
    {
        double xp0[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xp0[c] = t == 1 ? x0[c] : x64[c];
        M::transition64(mp, sc, xp0, f0);
    }
    float cf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) cf[c] = (float)f0[c];
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) s.misc[c] = cf[c];
    }
    // transition means of the previous set, FP64 and centred / scaled FP32
    for (int j = tid; j < Np; j += NT) {
        double fd[D];
        if (t == 1) {
#pragma unroll
            for (int c = 0; c < D; ++c) fd[c] = f0[c];
        } else {
            double xd[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xd[c] = x64[(size_t)j * D + c];
            M::transition64(mp, sc, xd, fd);
        }
        float fr[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            f64[(size_t)j * D + c] = fd[c];
            fr[c] = (float)((fd[c] - (double)cf[c]) * (mp.sqrt_qinv[c] * (double)kKm));
        }
        store_row<D, DP>(s.fs, j, fr);
    }
    double* cum = reinterpret_cast<double*>(s.gs);   // N doubles fit in gs
    double W = 1.0;
    if (t > 1) {
        // cumulative weights exp(lw - max) in FP64: contiguous chunks per thread,
        // then a block scan of the chunk sums
        double mx = -INFINITY;
        for (int j = tid; j < Np; j += NT) mx = fmax(mx, lw[j]);
        mx = block_max_d(mx, s.redd);
        const int chunk = (Np + NT - 1) / NT;
        const int j0 = min(tid * chunk, Np), j1 = min(j0 + chunk, Np);
        double part = 0.0;
        for (int j = j0; j < j1; ++j) {
            const double w = exp(lw[j] - mx);
            cum[j] = w;
            part += w;
        }
        double tot;
        double run = block_exclusive_scan_d(part, s.redd, &tot);
        for (int j = j0; j < j1; ++j) {
            run += cum[j];
            cum[j] = run;
        }
        W = tot;
    }
    __syncthreads();   // f64 and cum complete; every read of x64 as the previous set is done
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = tid + p * NT;
        if (i >= N) continue;
        int a = 0;
        if (t > 1) {
            const double u = ((double)i + draw_uniform64(seed, seq, (uint32_t)t, (uint32_t)i)) / (double)N;
            // first j with cum[j] / W > u (the oracle's normalised comparison)
            int lo = 0, hi = Np - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cum[mid] / W > u) hi = mid; else lo = mid + 1;
            }
            a = lo;
        }
        double z[D];
        draw_normals64<D>(seed, seq, (uint32_t)t, (uint32_t)i, z);
        double xn[D];
        float xr[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xn[c] = f64[(size_t)a * D + c] + mp.sqrt_q[c] * z[c];
            xr[c] = (float)xn[c];
        }
        store_row<D, DP>(s.xs, i, xr);
        lw[i] = M::loglik64(mp, s.zs, xn);
        // x64 is written after the barrier below: other threads may still read
        // f64 rows, not x64, so the order only matters across steps
#pragma unroll
        for (int c = 0; c < D; ++c) x64[(size_t)i * D + c] = xn[c];
    }
    __syncthreads();
}

template <class M, int PPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) pf_seq_kernel(const __grid_constant__ PfArgs a) {
    constexpr int D = M::D, DP = M::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sm s = bind_smem(smem_raw, a.Nmax, DP);
    SMAP_DBG_BEGIN(a.Nmax, a.status + a.B + kDbgWord);
    const ModelParams& mp = a.mp;
    const int tid = threadIdx.x, NT = blockDim.x;
    __shared__ int s_item;
    double* f64 = a.f64 + (size_t)blockIdx.x * a.Nmax * D;
    double* x64 = a.x64 + (size_t)blockIdx.x * a.Nmax * D;
    double* lw = a.lw + (size_t)blockIdx.x * a.Nmax;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.B) break;
        const int b = a.order ? a.order[item] : item;
        if (a.status[b] != 0) continue;
        const int N = a.Nseq[b];
        const int T = a.Tend[b];
        if (T > a.maxT || N < 1 || N > a.Nmax || N > PPT * NT) {
            if (tid == 0) a.status[b] = 1;
            continue;
        }
        if (tid == 0) s.phis[0] = 0.0;
        int Np = 1, tdone = 0;
        __syncthreads();
        for (int t = 1; t <= T; ++t) {
            pf_prepare_step<M, PPT>(mp, s, t, N, Np, a.x0 + (size_t)b * D,
                                    a.y + ((size_t)b * a.maxT + (t - 1)) * mp.dy, f64, x64, lw, a.seed,
                                    (uint32_t)b);
            int best[PPT];
            double phinew[PPT];
            viterbi_step<M, PPT, true>(mp, s, N, Np, f64, nullptr, best, phinew);   // FP64 states: FP64 terms
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
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float v = s.xs[i * DP + c];
                    bad |= !isfinite(v);
                    dst[(size_t)i * D + c] = v;
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
        if (tid == 0) a.tcur[b] = tdone;
    }
}

}  // namespace smap
