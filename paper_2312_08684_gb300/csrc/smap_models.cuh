// smap_models.cuh -- the scenario models as device functions.
//
// Each model provides, with D the state dimension and DP the shared-memory row
// stride of a particle:
//   step_const(mp, t)               FP64 constant of the transition at step t
//   transition(mp, sc, x, f)        f = f_t(x) in FP32          (Eq. SSM-x mean)
//   transition64(mp, sc, x, f)      the same in FP64
//   grad_loglik(mp, z, x, g)        grad_x log p(z | x) in FP32 (Eq. SSM-z)
//   loglik64(mp, z, x)              log p(z | x) in FP64, full normaliser
// and, where kTransDF / kLikDF say so, the same terms in double-float
// arithmetic (about 48 bits, on the FP32 pipe) from the FP32 particles:
//   trans_sq_df(mp, x, xp)          |x - f_t(xp)|^2_{Q^-1}, the residual formed
//                                   from x and the previous particle xp
//   centred_mean(mp, xp, c, out)    f_t(xp) - c rounded once to FP32
//   loglik_df(mp, z, x)             log p(z | x)
// Parameter layouts are documented in include/smap.h; aux[] holds constants
// the host precomputes in FP64 (listed per model; aux[4] = -1/(2 r) for the
// Gaussian-noise models that have a double-float likelihood).
#pragma once

#include "smap_common.cuh"
#include "smap_df.cuh"

namespace smap {

__device__ __forceinline__ df::F dfp(const ModelParams& mp, int k) { return df::make(mp.pf[k], mp.pl[k]); }
__device__ __forceinline__ df::F dfaux(const ModelParams& mp, int k) { return df::make(mp.auxh[k], mp.auxl[k]); }
__device__ __forceinline__ df::F dfqinv(const ModelParams& mp, int c) { return df::make(mp.qinv_f[c], mp.qinv_lo[c]); }
// (x - xp) exactly, as a double-float
__device__ __forceinline__ df::F df_diff(float x, float xp) { return df::two_sum(x, -xp); }
// log-density sum over heard range measurements: sum_l [aux0 - (z_l - |p - b_l|)^2 / (2 r)],
// beacon l at parameters (k0 + 2 l, k0 + 2 l + 1)
__device__ __forceinline__ df::F range_loglik_df(const ModelParams& mp, const float* z, const float* x, int nb,
                                                 int k0) {
    df::F s = df::make(0.0f, 0.0f);
    int heard = 0;
    for (int l = 0; l < nb; ++l) {
        const float zl = z[l];
        if (zl != zl) continue;
        const df::F dx = df::sub(df::make(x[0], 0.0f), dfp(mp, k0 + 2 * l));
        const df::F dy = df::sub(df::make(x[1], 0.0f), dfp(mp, k0 + 2 * l + 1));
        const df::F rho = df::sqrt(df::add(df::sqr(dx), df::sqr(dy)));
        s = df::add(s, df::sqr(df::sub(df::make(zl, 0.0f), rho)));
        ++heard;
    }
    return df::add(df::mul(s, dfaux(mp, 4)), df::mul_f(dfaux(mp, 0), (float)heard));
}

// 1-D nonstationary growth model. p = [a, b, c, omega, t_off, q, r, hcoef].
// aux[0] = -1/2 log(2 pi r), auxf[0] = 1/r.
struct ModelNGM1D {
    static constexpr int KIND = 1, D = 1, DP = 1, DY = 1;
    static constexpr bool kTransDF = false, kLikDF = false;
    __device__ static double step_const(const ModelParams& mp, int t) {
        return mp.p[2] * cos(mp.p[3] * ((double)t + mp.p[4]));
    }
    __device__ static void transition(const ModelParams& mp, double sc, const float* x, float* f) {
        const float v = x[0];
        f[0] = mp.pf[0] * v + mp.pf[1] * v / (1.0f + v * v) + (float)sc;
    }
    __device__ static void transition64(const ModelParams& mp, double sc, const double* x, double* f) {
        const double v = x[0];
        f[0] = mp.p[0] * v + mp.p[1] * v / (1.0 + v * v) + sc;
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        const float res = z[0] - mp.pf[7] * x[0] * x[0];
        g[0] = res * mp.auxf[0] * 2.0f * mp.pf[7] * x[0];
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const double res = (double)z[0] - mp.p[7] * x[0] * x[0];
        return -0.5 * res * res / mp.p[6] + mp.aux[0];
    }
};

// Constant-velocity transition shared by the three planar-target models.
struct CVTransition {
    __device__ static double step_const(const ModelParams&, int) { return 0.0; }
    __device__ static void transition(const ModelParams& mp, double, const float* x, float* f) {
        const float dt = mp.pf[0];
        f[0] = fmaf(dt, x[2], x[0]);
        f[1] = fmaf(dt, x[3], x[1]);
        f[2] = x[2];
        f[3] = x[3];
    }
    __device__ static void transition64(const ModelParams& mp, double, const double* x, double* f) {
        const double dt = mp.p[0];
        f[0] = x[0] + dt * x[2];
        f[1] = x[1] + dt * x[3];
        f[2] = x[2];
        f[3] = x[3];
    }
    // f_t(xp) - c, rounded once from its double-float value
    __device__ static void centred_mean(const ModelParams& mp, const float* xp, const float* cf, float* out) {
        const df::F dt = dfp(mp, 0);
#pragma unroll
        for (int c = 0; c < 2; ++c) out[c] = df::add(df_diff(xp[c], cf[c]), df::mul_f(dt, xp[c + 2])).hi;
#pragma unroll
        for (int c = 2; c < 4; ++c) out[c] = __fsub_rn(xp[c], cf[c]);
    }
    // position residual (x - xp) - dt vp, velocity residual v - vp
    __device__ static df::F trans_sq_df(const ModelParams& mp, const float* x, const float* xp) {
        const df::F dt = dfp(mp, 0);
        df::F s = df::make(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const df::F e = df::sub(df_diff(x[c], xp[c]), df::mul_f(dt, xp[c + 2]));
            s = df::add(s, df::mul(df::sqr(e), dfqinv(mp, c)));
        }
#pragma unroll
        for (int c = 2; c < 4; ++c) s = df::add(s, df::mul(df::sqr(df_diff(x[c], xp[c])), dfqinv(mp, c)));
        return s;
    }
};

// Section V-C's target without a motion prior: x = (px, py), zero-velocity
// random walk x_t = x_{t-1} + v; ranges to nb anchors. Parameters
// [q0, q1, r, nb, a0x, a0y, ...]; NaN = anchor not heard.
// aux[0] = -1/2 log(2 pi r), auxf[0] = 1/r.
struct ModelRangeZV {
    static constexpr int KIND = 6, D = 2, DP = 2, DY = 8;
    static constexpr bool kTransDF = true, kLikDF = true;
    __device__ static void centred_mean(const ModelParams&, const float* xp, const float* cf, float* out) {
        out[0] = __fsub_rn(xp[0], cf[0]);
        out[1] = __fsub_rn(xp[1], cf[1]);
    }
    __device__ static df::F trans_sq_df(const ModelParams& mp, const float* x, const float* xp) {
        return df::add(df::mul(df::sqr(df_diff(x[0], xp[0])), dfqinv(mp, 0)),
                       df::mul(df::sqr(df_diff(x[1], xp[1])), dfqinv(mp, 1)));
    }
    __device__ static df::F loglik_df(const ModelParams& mp, const float* z, const float* x) {
        return range_loglik_df(mp, z, x, (int)mp.p[3], 4);
    }
    __device__ static double step_const(const ModelParams&, int) { return 0.0; }
    __device__ static void transition(const ModelParams&, double, const float* x, float* f) {
        f[0] = x[0];
        f[1] = x[1];
    }
    __device__ static void transition64(const ModelParams&, double, const double* x, double* f) {
        f[0] = x[0];
        f[1] = x[1];
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        const int nb = (int)mp.p[3];
        float g0 = 0.0f, g1 = 0.0f;
        for (int l = 0; l < nb; ++l) {
            const float zl = z[l];
            if (zl != zl) continue;
            const float dx = x[0] - mp.pf[4 + 2 * l], dy = x[1] - mp.pf[5 + 2 * l];
            const float rho = fmaxf(sqrtf(dx * dx + dy * dy), 1e-9f);
            const float c = (zl - rho) * mp.auxf[0] / rho;
            g0 = fmaf(c, dx, g0);
            g1 = fmaf(c, dy, g1);
        }
        g[0] = g0; g[1] = g1;
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const int nb = (int)mp.p[3];
        double s = 0.0;
        for (int l = 0; l < nb; ++l) {
            const float zl = z[l];
            if (zl != zl) continue;
            const double dx = x[0] - mp.p[4 + 2 * l], dy = x[1] - mp.p[5 + 2 * l];
            const double res = (double)zl - sqrt(dx * dx + dy * dy);
            s += -0.5 * res * res / mp.p[2] + mp.aux[0];
        }
        return s;
    }
};

// Section V-B's pose on SE(2) under unknown association: x = (px, py, th),
// constant controls (v, w): th' = th + w dt, p' = p + v dt (cos th', sin th').
// One measurement z = (zr, zb) per step from one of nl landmarks, association
// marginalised with weights 1/nl:
//   p(z | x) = (1/nl) sum_l N(zr; rho_l, rr) N(wrap(zb - b_l); 0, rb),
//   rho_l = |p - L_l|, b_l = atan2(py - L_ly, px - L_lx), wrap into [-pi, pi].
// p = [dt, q0, q1, q2, rr, rb, v, w, nl, L0x, L0y, ...]; NaN zr = no measurement.
// aux[0] = -log nl - 1/2 log(2 pi rr) - 1/2 log(2 pi rb);
// auxf[0] = v dt, auxf[1] = w dt, auxf[2] = -log2(e) / (2 rr), auxf[3] = -log2(e) / (2 rb),
// auxf[4] = 1/rr, auxf[5] = 1/rb.
struct ModelSE2RB {
    static constexpr int KIND = 7, D = 3, DP = 4, DY = 2;
    static constexpr bool kTransDF = false, kLikDF = false;
    __device__ static double step_const(const ModelParams&, int) { return 0.0; }
    __device__ static void transition(const ModelParams& mp, double, const float* x, float* f) {
        const float th = x[2] + mp.auxf[1];
        float sn, cs;
        sincosf(th, &sn, &cs);
        f[0] = fmaf(mp.auxf[0], cs, x[0]);
        f[1] = fmaf(mp.auxf[0], sn, x[1]);
        f[2] = th;
    }
    __device__ static void transition64(const ModelParams& mp, double, const double* x, double* f) {
        const double dt = mp.p[0], th = x[2] + mp.p[7] * dt;
        f[0] = x[0] + mp.p[6] * dt * cos(th);
        f[1] = x[1] + mp.p[6] * dt * sin(th);
        f[2] = th;
    }
    __device__ static float wrapf(float a) {
        return fmaf(-6.2831853071795865f, rintf(a * 0.15915494309189535f), a);
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        g[0] = 0.0f; g[1] = 0.0f; g[2] = 0.0f;
        if (z[0] != z[0]) return;
        const int nl = (int)mp.p[8];
        // log2 of each association term (shared constants dropped), then
        // responsibilities by a max-shifted sum
        float lt[8], cr[8], cb[8], ddx[8], ddy[8];
        float mx = -INFINITY;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            if (l >= nl) break;
            const float dx = x[0] - mp.pf[9 + 2 * l], dy = x[1] - mp.pf[10 + 2 * l];
            const float rho2 = fmaxf(fmaf(dx, dx, dy * dy), 1e-18f);
            const float rho = sqrtf(rho2);
            const float er = z[0] - rho;
            const float eb = wrapf(z[1] - atan2f(dy, dx));
            lt[l] = fmaf(mp.auxf[2], er * er, mp.auxf[3] * eb * eb);
            cr[l] = er * mp.auxf[4] / rho;
            cb[l] = eb * mp.auxf[5] / rho2;
            ddx[l] = dx; ddy[l] = dy;
            mx = fmaxf(mx, lt[l]);
        }
        float s = 0.0f, g0 = 0.0f, g1 = 0.0f;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            if (l >= nl) break;
            const float w = fast_exp2(lt[l] - mx);
            s += w;
            g0 = fmaf(w, fmaf(cr[l], ddx[l], -cb[l] * ddy[l]), g0);
            g1 = fmaf(w, fmaf(cr[l], ddy[l], cb[l] * ddx[l]), g1);
        }
        const float k = 1.0f / s;
        g[0] = g0 * k; g[1] = g1 * k;
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        if (z[0] != z[0]) return 0.0;
        const int nl = (int)mp.p[8];
        const double zr = z[0], zb = z[1];
        double lt[8], mx = -INFINITY;
        for (int l = 0; l < nl; ++l) {
            const double dx = x[0] - mp.p[9 + 2 * l], dy = x[1] - mp.p[10 + 2 * l];
            const double er = zr - sqrt(dx * dx + dy * dy);
            double eb = zb - atan2(dy, dx);
            eb -= 6.283185307179586 * rint(eb / 6.283185307179586);
            lt[l] = -0.5 * (er * er / mp.p[4] + eb * eb / mp.p[5]);
            mx = fmax(mx, lt[l]);
        }
        double s = 0.0;
        for (int l = 0; l < nl; ++l) s += exp(lt[l] - mx);
        return mp.aux[0] + mx + log(s);
    }
};

// Range-only localisation. p = [dt, q0..q3, r, nb, b0x, b0y, ...].
// aux[0] = -1/2 log(2 pi r), auxf[0] = 1/r. NaN observation = beacon not heard.
struct ModelRangeCV : CVTransition {
    static constexpr int KIND = 2, D = 4, DP = 4, DY = 8;
    static constexpr bool kTransDF = true, kLikDF = true;
    __device__ static df::F loglik_df(const ModelParams& mp, const float* z, const float* x) {
        return range_loglik_df(mp, z, x, (int)mp.p[6], 7);
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        const int nb = (int)mp.p[6];
        float g0 = 0.0f, g1 = 0.0f;
        for (int l = 0; l < nb; ++l) {
            const float zl = z[l];
            if (zl != zl) continue;
            const float dx = x[0] - mp.pf[7 + 2 * l], dy = x[1] - mp.pf[8 + 2 * l];
            float rho = sqrtf(dx * dx + dy * dy);
            rho = fmaxf(rho, 1e-9f);
            const float c = (zl - rho) * mp.auxf[0] / rho;
            g0 = fmaf(c, dx, g0);
            g1 = fmaf(c, dy, g1);
        }
        g[0] = g0; g[1] = g1; g[2] = 0.0f; g[3] = 0.0f;
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const int nb = (int)mp.p[6];
        double s = 0.0;
        for (int l = 0; l < nb; ++l) {
            const float zl = z[l];
            if (zl != zl) continue;
            const double dx = x[0] - mp.p[7 + 2 * l], dy = x[1] - mp.p[8 + 2 * l];
            const double res = (double)zl - sqrt(dx * dx + dy * dy);
            s += -0.5 * res * res / mp.p[5] + mp.aux[0];
        }
        return s;
    }
};

// Unknown association with clutter. p = [dt, q0..q3, r, M, beta, area].
// aux[0] = log((1-beta)/M) - log(2 pi r), aux[1] = log(beta/area);
// auxf[0] = 1/r, auxf[1] = aux[0] * log2(e), auxf[2] = aux[1] * log2(e).
struct ModelClutterCV : CVTransition {
    static constexpr int KIND = 3, D = 4, DP = 4, DY = 64;
    static constexpr bool kTransDF = true, kLikDF = true;
    // The same mixture in double-float: the FP32 pass finds the largest term
    // (its value shifts the sum: the result does not depend on the shift) and
    // the terms within 45 nats of it; the shifted sum s >= 1 and its log are
    // double-float (the largest term contributes exp(0) = 1 exactly).
    __device__ static df::F loglik_df(const ModelParams& mp, const float* z, const float* x) {
        if (!(isfinite(x[0]) && isfinite(x[1]))) return df::make(__int_as_float(0x7fc00000), 0.0f);
        const int M = (int)mp.p[6];
        const float c2 = -0.5f * mp.auxf[0];
        const float a0f = mp.auxh[0], a1f = mp.auxh[1];
        float mxf = a1f;
        int mi = -1;   // -1: the outlier term is the largest
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - x[0], ey = z[2 * m + 1] - x[1];
            const float a = fmaf(c2, fmaf(ex, ex, ey * ey), a0f);
            if (a > mxf) { mxf = a; mi = m; }
        }
        const float keep = mxf - 45.0f;
        const df::F c = dfaux(mp, 4);
        auto term = [&](int m) {
            const df::F ex = df_diff(z[2 * m], x[0]), ey = df_diff(z[2 * m + 1], x[1]);
            return df::add(dfaux(mp, 0), df::mul(df::add(df::sqr(ex), df::sqr(ey)), c));
        };
        const df::F mx = mi < 0 ? dfaux(mp, 1) : term(mi);
        df::F s = df::make(1.0f, 0.0f);
        if (mi >= 0 && a1f >= keep) s = df::add(s, df::exp(df::sub(dfaux(mp, 1), mx)));
        for (int m = 0; m < M; ++m) {
            if (m == mi) continue;
            const float ex = z[2 * m] - x[0], ey = z[2 * m + 1] - x[1];
            if (!(fmaf(c2, fmaf(ex, ex, ey * ey), a0f) >= keep)) continue;
            s = df::add(s, df::exp(df::sub(term(m), mx)));
        }
        return df::add(mx, df::log(s));
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        const int M = (int)mp.p[6];
        const float rinv = mp.auxf[0];
        const float c2 = -0.5f * 1.4426950408889634f * rinv;   // log2 units
        // log2 of each mixture term, then responsibilities by a max-shifted sum
        float mx = mp.auxf[2];
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - x[0], ey = z[2 * m + 1] - x[1];
            mx = fmaxf(mx, fmaf(c2, ex * ex + ey * ey, mp.auxf[1]));
        }
        float s = fast_exp2(mp.auxf[2] - mx), a0 = 0.0f, a1 = 0.0f;
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - x[0], ey = z[2 * m + 1] - x[1];
            const float w = fast_exp2(fmaf(c2, ex * ex + ey * ey, mp.auxf[1]) - mx);
            s += w;
            a0 = fmaf(w, ex, a0);
            a1 = fmaf(w, ey, a1);
        }
        const float k = rinv / s;
        g[0] = a0 * k; g[1] = a1 * k; g[2] = 0.0f; g[3] = 0.0f;
    }
    // log of the mixture by a max-shifted sum. A term more than 40 nats below
    // the largest adds less than e^-40 < 2^-57 to a sum that is at least 1,
    // below the FP64 rounding of the result: such terms are found with an
    // FP32 pass (its error is far inside the 5-nat margin) and skipped, so
    // that the FP64 work is the few terms near the maximum (usually the
    // true point's and the outlier term).
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const int M = (int)mp.p[6];
        const double rinv = 1.0 / mp.p[5];
        const float xf0 = (float)x[0], xf1 = (float)x[1];
        const float c2 = -0.5f * mp.auxf[0];
        const float a0f = (float)mp.aux[0], a1f = (float)mp.aux[1];
        float mxf = a1f;
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - xf0, ey = z[2 * m + 1] - xf1;
            mxf = fmaxf(mxf, fmaf(c2, fmaf(ex, ex, ey * ey), a0f));
        }
        const float keep = mxf - 45.0f;
        double mx = mp.aux[1];
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - xf0, ey = z[2 * m + 1] - xf1;
            if (fmaf(c2, fmaf(ex, ex, ey * ey), a0f) < keep) continue;
            const double ed = (double)z[2 * m] - x[0], fd = (double)z[2 * m + 1] - x[1];
            mx = fmax(mx, mp.aux[0] - 0.5 * (ed * ed + fd * fd) * rinv);
        }
        double s = (a1f < keep) ? 0.0 : exp(mp.aux[1] - mx);
        for (int m = 0; m < M; ++m) {
            const float ex = z[2 * m] - xf0, ey = z[2 * m + 1] - xf1;
            if (fmaf(c2, fmaf(ex, ex, ey * ey), a0f) < keep) continue;
            const double ed = (double)z[2 * m] - x[0], fd = (double)z[2 * m + 1] - x[1];
            s += exp(mp.aux[0] - 0.5 * (ed * ed + fd * fd) * rinv - mx);
        }
        return mx + log(s);
    }
};

// Planar chain of NL links. p = [dt, nl, r, q_0..q_{2nl-1}, len_0..len_{nl-1}].
// aux[0] = -log(2 pi r), auxf[0] = 1/r.
template <int NL>
struct ModelPlanarArm {
    static constexpr int KIND = 4, D = 2 * NL, DP = (2 * NL + 3) & ~3, DY = 2;
    static constexpr bool kTransDF = true, kLikDF = false;
    __device__ static void centred_mean(const ModelParams& mp, const float* xp, const float* cf, float* out) {
        const df::F dt = dfp(mp, 0);
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            out[k] = df::add(df_diff(xp[k], cf[k]), df::mul_f(dt, xp[NL + k])).hi;
            out[NL + k] = __fsub_rn(xp[NL + k], cf[NL + k]);
        }
    }
    // angle residual (th - thp) - dt wp, rate residual w - wp
    __device__ static df::F trans_sq_df(const ModelParams& mp, const float* x, const float* xp) {
        const df::F dt = dfp(mp, 0);
        df::F s = df::make(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const df::F e = df::sub(df_diff(x[k], xp[k]), df::mul_f(dt, xp[NL + k]));
            s = df::add(s, df::mul(df::sqr(e), dfqinv(mp, k)));
            s = df::add(s, df::mul(df::sqr(df_diff(x[NL + k], xp[NL + k])), dfqinv(mp, NL + k)));
        }
        return s;
    }
    __device__ static double step_const(const ModelParams&, int) { return 0.0; }
    __device__ static void transition(const ModelParams& mp, double, const float* x, float* f) {
        const float dt = mp.pf[0];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            f[k] = fmaf(dt, x[NL + k], x[k]);
            f[NL + k] = x[NL + k];
        }
    }
    __device__ static void transition64(const ModelParams& mp, double, const double* x, double* f) {
        const double dt = mp.p[0];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            f[k] = x[k] + dt * x[NL + k];
            f[NL + k] = x[NL + k];
        }
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        const float* len = mp.pf + 3 + 2 * NL;
        float lc[NL], ls[NL];
        float th = 0.0f, ex = 0.0f, ey = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            th += x[l];
            float s, c;
            __sincosf(th, &s, &c);
            lc[l] = len[l] * c;
            ls[l] = len[l] * s;
            ex += lc[l];
            ey += ls[l];
        }
        const float rx = (z[0] - ex) * mp.auxf[0], ry = (z[1] - ey) * mp.auxf[0];
        // d e / d angle_m = sum_{l >= m} len_l (-sin th_l, cos th_l): suffix sums
        float sx = 0.0f, sy = 0.0f;
#pragma unroll
        for (int m = NL - 1; m >= 0; --m) {
            sx -= ls[m];
            sy += lc[m];
            g[m] = fmaf(sx, rx, sy * ry);
            g[NL + m] = 0.0f;
        }
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const double* len = mp.p + 3 + 2 * NL;
        double th = 0.0, ex = 0.0, ey = 0.0;
        for (int l = 0; l < NL; ++l) {
            th += x[l];
            double s, c;
            sincos(th, &s, &c);
            ex += len[l] * c;
            ey += len[l] * s;
        }
        const double rx = (double)z[0] - ex, ry = (double)z[1] - ey;
        return -0.5 * (rx * rx + ry * ry) / mp.p[2] + mp.aux[0];
    }
};

// Linear-Gaussian test model. p = [dt, q0..q3, r].
// aux[0] = -log(2 pi r), auxf[0] = 1/r.
struct ModelLinearGauss : CVTransition {
    static constexpr int KIND = 5, D = 4, DP = 4, DY = 2;
    static constexpr bool kTransDF = true, kLikDF = true;
    __device__ static df::F loglik_df(const ModelParams& mp, const float* z, const float* x) {
        const df::F q = df::add(df::sqr(df_diff(z[0], x[0])), df::sqr(df_diff(z[1], x[1])));
        return df::add(dfaux(mp, 0), df::mul(q, dfaux(mp, 4)));
    }
    __device__ static void grad_loglik(const ModelParams& mp, const float* z, const float* x, float* g) {
        g[0] = (z[0] - x[0]) * mp.auxf[0];
        g[1] = (z[1] - x[1]) * mp.auxf[0];
        g[2] = 0.0f; g[3] = 0.0f;
    }
    __device__ static double loglik64(const ModelParams& mp, const float* z, const double* x) {
        const double ex = (double)z[0] - x[0], ey = (double)z[1] - x[1];
        return -0.5 * (ex * ex + ey * ey) / mp.p[5] + mp.aux[0];
    }
};

}  // namespace smap
