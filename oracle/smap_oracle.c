/*
 * smap_oracle.c -- plain, slow FP64 CPU oracle for the Stein-MAP-Seq hot path
 * (Seo & Kia, "A Computationally Efficient Maximum A Posteriori Sequence
 * Estimation via Stein Variational Inference", arXiv 2312.08684).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this file's library. The product (the CUDA library
 * under paper_2312_08684_gb300/csrc) shares no code, header, table or constant
 * generator with it; the scenario models and the counter-based RNG are
 * written a second time here from their definitions.
 *
 * What it computes, in the paper's order (Algorithm 2):
 *   1. t = 1: SVGD with the direction of Eq. (SVGD_initial_newupdate), the
 *      prior being the transition density around f_1(x_0^true).
 *   2. phi_1(i) = log p(z_1, x_1^i | x_0^true).
 *   3. t >= 2: SVGD with the direction of Eq. (SVGD_newupdate) given the
 *      previous particle set, then the forward recursion Eq. (forward_recursion).
 *   4. Backtracking (Section IV-B, "Backtracking the MAP Sequence").
 * SVGD itself is Algorithm 1 with the empirical direction Eq. (svgd_iterate).
 *
 * Readings of points the paper leaves open:
 *   - Kernel: RBF kappa(x,x') = exp(-||x-x'||^2 / h); the paper names the RBF
 *     kernel and the median heuristic (Section V, Table Ex6 caption) without a
 *     formula; h = s * med / log(N) with med the median of the squared pairwise
 *     distances over i<k (mean of the two middle values when their number is
 *     even), s a scale (1 = plain heuristic). N = 1 or med = 0: h = 1.
 *   - Prior term of Eq. (SVGD_newupdate): three readings. MIXTURE (default): the
 *     score of log (1/N) sum_j p(x | x_{t-1}^j), i.e. responsibilities w_kj;
 *     MEANGRAD (literal average of the N gradients): Q^-1 (mean_j f_j - x).
 *     MAPCOND (the prior conditioned on the previous MAP estimates that
 *     Section V-C describes): the score of max_j [phi_{t-1}(j) +
 *     log p(x | x_{t-1}^j)], i.e. Q^-1 (f_{j*} - x) for the maximising j*.
 *     The three coincide when the previous set has one particle (t = 1).
 *   - Initial particles at step t (unspecified): x_t^{i,(0)} = f_t(x_{t-1}^i)
 *     + sqrt(q) (.) xi_i, xi ~ N(0, I) from Philox-4x32-10 (Salmon et al.
 *     2011) keyed by the seed, counter (i, t, seq, block), Box-Muller in FP64.
 *     At t = 1 every particle starts from f_1(x_0^true).
 *   - Scores carry full Gaussian normalisers; log p(x_0) is a constant and is
 *     left out of J. Ties: lowest index.
 *
 * Every pair sum is a plain double loop; the median is a sort.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OM_MAXD 16
#define OM_MAXDY 64
#define OM_MAXP 128

enum { OM_NGM1D = 1, OM_RANGE_CV2D = 2, OM_CLUTTER_CV2D = 3, OM_PLANAR_ARM = 4,
       OM_LINEAR_GAUSS = 5, OM_RANGE_ZV2D = 6, OM_SE2_RB = 7 };
enum { OM_BW_MEDIAN_ITER = 0, OM_BW_MEDIAN_STEP = 1, OM_BW_FIXED = 2 };
enum { OM_PRIOR_MIXTURE = 0, OM_PRIOR_MEANGRAD = 1, OM_PRIOR_MAPCOND = 2 };

static const double OM_PI = 3.14159265358979323846;

typedef struct {
    int kind, d, dy;
    double q[OM_MAXD];      /* diagonal of the process-noise covariance Q */
    double p[OM_MAXP];      /* the raw parameter vector */
    int np;
} om_model;

/* ------------------------------------------------------------------------ */
/* Scenario models: transition mean f_t, likelihood log p(z|x) and its       */
/* gradient. Parameter layouts:                                              */
/*  NGM1D        [a, b, c, omega, t_off, q, r, hcoef]                        */
/*               f_t(x) = a x + b x/(1+x^2) + c cos(omega (t + t_off))       */
/*               z = hcoef x^2 + N(0, r)                                     */
/*  RANGE_CV2D   [dt, q0..q3, r, nb, b0x, b0y, ...]  state (px,py,vx,vy)      */
/*               constant velocity; z_l = ||p - b_l|| + N(0, r); NaN = none  */
/*  CLUTTER_CV2D [dt, q0..q3, r, M, beta, area]; z = M points (x,y);         */
/*               p(z|x) = (1-beta)(1/M) sum_m N(z_m; p, r I) + beta/area     */
/*  PLANAR_ARM   [dt, nl, r, q_0..q_{2nl-1}, len_0..len_{nl-1}]               */
/*               state (angles, rates); z = sum_l len_l (cos th_l, sin th_l) */
/*               th_l = sum_{m<=l} angle_m, noise N(0, r I_2)                 */
/*  LINEAR_GAUSS [dt, q0..q3, r]; constant velocity, z = p + N(0, r I_2)      */
/*  RANGE_ZV2D   [q0, q1, r, nb, b0x, b0y, ...]  state (px, py); zero-velocity */
/*               random walk x_t = x_{t-1} + v (Section V-C's target model);  */
/*               z_l = ||p - b_l|| + N(0, r); NaN = anchor not heard          */
/*  SE2_RB       [dt, q0, q1, q2, rr, rb, v, omega, nl, L0x, L0y, ...]        */
/*               pose (px, py, th) on SE(2) under constant controls (v, w)   */
/*               (Section V-B's motion model): th' = th + w dt,              */
/*               p' = p + v dt (cos th', sin th'); one range-bearing pair    */
/*               z = (zr, zb) from ONE of nl landmarks, association unknown: */
/*               p(z|x) = (1/nl) sum_l N(zr; rho_l, rr) N(wrap(zb - b_l); 0, rb) */
/*               rho_l = ||p - L_l||, b_l = atan2(py - Lly, px - Llx);       */
/*               wrap(a) = a - 2 pi n, n the nearest integer to a / (2 pi).  */
/*               NaN zr = no measurement at that step.                       */
/* ------------------------------------------------------------------------ */

int om_setup(om_model* m, int kind, const double* p, int np)
{
    memset(m, 0, sizeof(*m));
    if (np > OM_MAXP || np < 1) return -1;
    m->kind = kind;
    m->np = np;
    memcpy(m->p, p, sizeof(double) * np);
    switch (kind) {
    case OM_NGM1D:
        if (np != 8) return -1;
        m->d = 1; m->dy = 1; m->q[0] = p[5];
        break;
    case OM_RANGE_CV2D: {
        if (np < 7) return -1;
        int nb = (int)p[6];
        if (nb < 1 || nb > 8 || np != 7 + 2 * nb) return -1;
        m->d = 4; m->dy = nb;
        for (int k = 0; k < 4; ++k) m->q[k] = p[1 + k];
        break;
    }
    case OM_CLUTTER_CV2D: {
        if (np != 9) return -1;
        int M = (int)p[6];
        if (M < 1 || M > 32) return -1;
        m->d = 4; m->dy = 2 * M;
        for (int k = 0; k < 4; ++k) m->q[k] = p[1 + k];
        break;
    }
    case OM_PLANAR_ARM: {
        if (np < 3) return -1;
        int nl = (int)p[1];
        if (nl < 1 || nl > 8 || np != 3 + 3 * nl) return -1;
        m->d = 2 * nl; m->dy = 2;
        for (int k = 0; k < 2 * nl; ++k) m->q[k] = p[3 + k];
        break;
    }
    case OM_LINEAR_GAUSS:
        if (np != 6) return -1;
        m->d = 4; m->dy = 2;
        for (int k = 0; k < 4; ++k) m->q[k] = p[1 + k];
        break;
    case OM_RANGE_ZV2D: {
        if (np < 4) return -1;
        int nb = (int)p[3];
        if (nb < 1 || nb > 8 || np != 4 + 2 * nb) return -1;
        m->d = 2; m->dy = nb;
        m->q[0] = p[0]; m->q[1] = p[1];
        break;
    }
    case OM_SE2_RB: {
        if (np < 9) return -1;
        int nl = (int)p[8];
        if (nl < 1 || nl > 8 || np != 9 + 2 * nl) return -1;
        if (!(p[4] > 0.0) || !(p[5] > 0.0)) return -1;
        m->d = 3; m->dy = 2;
        for (int k = 0; k < 3; ++k) m->q[k] = p[1 + k];
        break;
    }
    default:
        return -1;
    }
    for (int k = 0; k < m->d; ++k) if (!(m->q[k] > 0.0)) return -1;
    return 0;
}

/* x_t = f_t(x_{t-1}) + v_{t-1}: the transition mean (Eq. SSM-x). */
void om_transition(const om_model* m, int t, const double* x, double* f)
{
    const double* p = m->p;
    switch (m->kind) {
    case OM_NGM1D:
        f[0] = p[0] * x[0] + p[1] * x[0] / (1.0 + x[0] * x[0])
             + p[2] * cos(p[3] * ((double)t + p[4]));
        break;
    case OM_RANGE_CV2D:
    case OM_CLUTTER_CV2D:
    case OM_LINEAR_GAUSS: {
        double dt = p[0];
        f[0] = x[0] + dt * x[2];
        f[1] = x[1] + dt * x[3];
        f[2] = x[2];
        f[3] = x[3];
        break;
    }
    case OM_RANGE_ZV2D:
        f[0] = x[0];
        f[1] = x[1];
        break;
    case OM_SE2_RB: {
        double dt = p[0], th = x[2] + p[7] * dt;
        f[0] = x[0] + p[6] * dt * cos(th);
        f[1] = x[1] + p[6] * dt * sin(th);
        f[2] = th;
        break;
    }
    case OM_PLANAR_ARM: {
        int nl = (int)p[1];
        double dt = p[0];
        for (int k = 0; k < nl; ++k) {
            f[k] = x[k] + dt * x[nl + k];
            f[nl + k] = x[nl + k];
        }
        break;
    }
    }
}

/* Forward kinematics of the planar chain and its Jacobian (2 x nl). */
static void om_arm_fk(const om_model* m, const double* x, double* e, double* J)
{
    int nl = (int)m->p[1];
    const double* len = m->p + 3 + 2 * nl;
    double th = 0.0, ex = 0.0, ey = 0.0;
    double lc[8], ls[8];
    for (int l = 0; l < nl; ++l) {
        th += x[l];
        lc[l] = len[l] * cos(th);
        ls[l] = len[l] * sin(th);
        ex += lc[l];
        ey += ls[l];
    }
    e[0] = ex; e[1] = ey;
    if (J) {
        /* d e / d angle_m = sum_{l >= m} len_l (-sin th_l, cos th_l) */
        for (int mm = 0; mm < nl; ++mm) {
            double jx = 0.0, jy = 0.0;
            for (int l = mm; l < nl; ++l) { jx -= ls[l]; jy += lc[l]; }
            J[mm] = jx;
            J[nl + mm] = jy;
        }
    }
}

/* log N(v; 0, s) for a scalar variance s. */
static double om_lognorm1(double v, double s)
{
    return -0.5 * v * v / s - 0.5 * log(2.0 * OM_PI * s);
}

/* log p(z_t | x_t) (Eq. SSM-z). */
/* Range measurements to nb anchors b (x, y pairs), variance r: the log
 * likelihood and its gradient in the position (x[0], x[1]); NaN = not heard. */
static double om_range_loglik(const double* x, const double* z, int nb, double r, const double* b)
{
    double s = 0.0;
    for (int l = 0; l < nb; ++l) {
        if (isnan(z[l])) continue;
        double dx = x[0] - b[2 * l], dy = x[1] - b[2 * l + 1];
        s += om_lognorm1(z[l] - sqrt(dx * dx + dy * dy), r);
    }
    return s;
}
static void om_range_grad(const double* x, const double* z, int nb, double r, const double* b, double* g)
{
    for (int l = 0; l < nb; ++l) {
        if (isnan(z[l])) continue;
        double dx = x[0] - b[2 * l], dy = x[1] - b[2 * l + 1];
        double rho = sqrt(dx * dx + dy * dy);
        if (rho < 1e-9) rho = 1e-9;
        double c = (z[l] - rho) / r / rho;
        g[0] += c * dx;
        g[1] += c * dy;
    }
}

/* Bearing residual brought to [-pi, pi]. */
static double om_wrap(double a)
{
    return a - 2.0 * OM_PI * nearbyint(a / (2.0 * OM_PI));
}

/* log of the nl association terms of SE2_RB (each with its 1/nl weight). */
static void om_se2_terms(const double* p, const double* z, const double* x, double* terms)
{
    int nl = (int)p[8];
    for (int l = 0; l < nl; ++l) {
        double dx = x[0] - p[9 + 2 * l], dy = x[1] - p[10 + 2 * l];
        double rho = sqrt(dx * dx + dy * dy);
        double eb = om_wrap(z[1] - atan2(dy, dx));
        terms[l] = -log((double)nl) + om_lognorm1(z[0] - rho, p[4]) + om_lognorm1(eb, p[5]);
    }
}

double om_loglik(const om_model* m, int t, const double* z, const double* x)
{
    const double* p = m->p;
    (void)t;
    switch (m->kind) {
    case OM_NGM1D:
        return om_lognorm1(z[0] - p[7] * x[0] * x[0], p[6]);
    case OM_RANGE_CV2D:
        return om_range_loglik(x, z, (int)p[6], p[5], p + 7);
    case OM_RANGE_ZV2D:
        return om_range_loglik(x, z, (int)p[3], p[2], p + 4);
    case OM_SE2_RB: {
        if (isnan(z[0])) return 0.0;
        int nl = (int)p[8];
        double terms[8], mx = -INFINITY, s = 0.0;
        om_se2_terms(p, z, x, terms);
        for (int l = 0; l < nl; ++l) if (terms[l] > mx) mx = terms[l];
        for (int l = 0; l < nl; ++l) s += exp(terms[l] - mx);
        return mx + log(s);
    }
    case OM_CLUTTER_CV2D: {
        double r = p[5], beta = p[7], area = p[8];
        int M = (int)p[6];
        /* log( (1-beta)/M * sum_m N(z_m; p, rI) + beta/area ) by log-sum-exp */
        double terms[33];
        double mx = -INFINITY;
        for (int k = 0; k < M; ++k) {
            double ex = z[2 * k] - x[0], ey = z[2 * k + 1] - x[1];
            terms[k] = log((1.0 - beta) / M) + om_lognorm1(ex, r) + om_lognorm1(ey, r);
            if (terms[k] > mx) mx = terms[k];
        }
        terms[M] = log(beta / area);
        if (terms[M] > mx) mx = terms[M];
        double s = 0.0;
        for (int k = 0; k <= M; ++k) s += exp(terms[k] - mx);
        return mx + log(s);
    }
    case OM_PLANAR_ARM: {
        double e[2];
        om_arm_fk(m, x, e, NULL);
        return om_lognorm1(z[0] - e[0], p[2]) + om_lognorm1(z[1] - e[1], p[2]);
    }
    case OM_LINEAR_GAUSS:
        return om_lognorm1(z[0] - x[0], p[5]) + om_lognorm1(z[1] - x[1], p[5]);
    }
    return NAN;
}

/* grad_x log p(z_t | x_t). */
void om_grad_loglik(const om_model* m, int t, const double* z, const double* x, double* g)
{
    const double* p = m->p;
    (void)t;
    for (int k = 0; k < m->d; ++k) g[k] = 0.0;
    switch (m->kind) {
    case OM_NGM1D: {
        double res = z[0] - p[7] * x[0] * x[0];
        g[0] = res / p[6] * 2.0 * p[7] * x[0];
        break;
    }
    case OM_RANGE_CV2D:
        om_range_grad(x, z, (int)p[6], p[5], p + 7, g);
        break;
    case OM_RANGE_ZV2D:
        om_range_grad(x, z, (int)p[3], p[2], p + 4, g);
        break;
    case OM_SE2_RB: {
        /* sum over landmarks of responsibility x gradient of that term;
         * d b_l / d(px, py) = (-dy, dx) / rho^2 */
        if (isnan(z[0])) break;
        int nl = (int)p[8];
        double terms[8];
        double ll = om_loglik(m, t, z, x);
        om_se2_terms(p, z, x, terms);
        for (int l = 0; l < nl; ++l) {
            double w = exp(terms[l] - ll);
            double dx = x[0] - p[9 + 2 * l], dy = x[1] - p[10 + 2 * l];
            double rho2 = dx * dx + dy * dy;
            if (rho2 < 1e-18) rho2 = 1e-18;
            double rho = sqrt(rho2);
            double cr = (z[0] - rho) / p[4] / rho;
            double cb = om_wrap(z[1] - atan2(dy, dx)) / p[5] / rho2;
            g[0] += w * (cr * dx - cb * dy);
            g[1] += w * (cr * dy + cb * dx);
        }
        break;
    }
    case OM_CLUTTER_CV2D: {
        double r = p[5], beta = p[7], area = p[8];
        int M = (int)p[6];
        double ll = om_loglik(m, t, z, x);
        for (int k = 0; k < M; ++k) {
            double ex = z[2 * k] - x[0], ey = z[2 * k + 1] - x[1];
            double lt = log((1.0 - beta) / M) + om_lognorm1(ex, r) + om_lognorm1(ey, r);
            double w = exp(lt - ll);              /* responsibility of measurement k */
            g[0] += w * ex / r;
            g[1] += w * ey / r;
        }
        (void)area;
        break;
    }
    case OM_PLANAR_ARM: {
        int nl = (int)p[1];
        double e[2], J[16];
        om_arm_fk(m, x, e, J);
        double rx = (z[0] - e[0]) / p[2], ry = (z[1] - e[1]) / p[2];
        for (int mm = 0; mm < nl; ++mm) g[mm] = J[mm] * rx + J[nl + mm] * ry;
        break;
    }
    case OM_LINEAR_GAUSS:
        g[0] = (z[0] - x[0]) / p[5];
        g[1] = (z[1] - x[1]) / p[5];
        break;
    }
}

/* log p(x_t | x_{t-1}) = log N(x_t; f, Q), Q = diag(q). */
double om_logtrans(const om_model* m, const double* x, const double* f)
{
    double s = 0.0;
    for (int k = 0; k < m->d; ++k) s += om_lognorm1(x[k] - f[k], m->q[k]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Counter-based RNG: Philox-4x32-10 as defined by Salmon, Moraes, Dror and  */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC 2011): ten rounds */
/* of two 32x32->64 multiplies with the round keys bumped by the Weyl        */
/* constants after each round.                                               */
/* ------------------------------------------------------------------------ */
void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* d standard normals for (seed, seq, t, i): block b of four dimensions uses
 * counter (i, t, seq, b); words (w0, w1) and (w2, w3) each give two normals
 * by Box-Muller with u = (w + 1/2) / 2^32. */
void om_normals(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i, int d, double* z)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int b = 0; 4 * b < d; ++b) {
        uint32_t ctr[4] = { i, t, seq, (uint32_t)b }, w[4];
        om_philox4x32_10(ctr, key, w);
        for (int h = 0; h < 2; ++h) {
            double u1 = ((double)w[2 * h] + 0.5) * (1.0 / 4294967296.0);
            double u2 = ((double)w[2 * h + 1] + 0.5) * (1.0 / 4294967296.0);
            double rad = sqrt(-2.0 * log(u1));
            double ang = 2.0 * OM_PI * u2;
            int k0 = 4 * b + 2 * h;
            if (k0 < d) z[k0] = rad * cos(ang);
            if (k0 + 1 < d) z[k0 + 1] = rad * sin(ang);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Bandwidth: median of the squared pairwise distances (i < k), by sorting.  */
/* ------------------------------------------------------------------------ */
static int om_cmp(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

double om_median_sqdist(const double* x, int N, int d)
{
    if (N < 2) return 0.0;
    long P = (long)N * (N - 1) / 2, n = 0;
    double* v = (double*)malloc(sizeof(double) * P);
    for (int i = 0; i < N; ++i)
        for (int k = i + 1; k < N; ++k) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) {
                double e = x[(long)i * d + c] - x[(long)k * d + c];
                s += e * e;
            }
            v[n++] = s;
        }
    qsort(v, P, sizeof(double), om_cmp);
    double med = (P % 2) ? v[P / 2] : 0.5 * (v[P / 2 - 1] + v[P / 2]);
    free(v);
    return med;
}

double om_bandwidth(const double* x, int N, int d, double scale)
{
    if (N < 2) return 1.0;
    double med = om_median_sqdist(x, N, d);
    if (!(med > 0.0)) return 1.0;
    return scale * med / log((double)N);
}

/* Stein kernels k(a, b) = k(r^2), r^2 = |a - b|^2, with bandwidth h:
 *   RBF        exp(-r^2 / h)                         (Section V's kernel);
 *   IMQ        (1 + r^2 / h)^(-1/2)                  (Gorham & Mackey 2017);
 *   Matern 3/2 (1 + s) exp(-s), s = sqrt(3 r^2 / h)  (length scale sqrt(h)),
 * the alternatives of the kernel ablation (Table Ex6). *kap = k(a, b) and
 * *rho the factor with grad_b k(b, a) = rho (a - b), i.e. -2 dk/d(r^2):
 * 2k/h, k^3/h and 3 exp(-s)/h respectively. */
enum { OM_KERNEL_RBF = 0, OM_KERNEL_IMQ = 1, OM_KERNEL_MATERN32 = 2 };
static void om_kernel(int kernel, const double* a, const double* b, int d, double h, double* kap,
                      double* rho)
{
    double r2 = 0.0;
    for (int c = 0; c < d; ++c) { double e = a[c] - b[c]; r2 += e * e; }
    if (kernel == OM_KERNEL_IMQ) {
        double k = 1.0 / sqrt(1.0 + r2 / h);
        *kap = k;
        *rho = k * k * k / h;
    } else if (kernel == OM_KERNEL_MATERN32) {
        double sr = sqrt(3.0 * r2 / h), e = exp(-sr);
        *kap = (1.0 + sr) * e;
        *rho = 3.0 * e / h;
    } else {
        double k = exp(-r2 / h);
        *kap = k;
        *rho = 2.0 * k / h;
    }
}

/* ------------------------------------------------------------------------ */
/* Score of the per-step SVGD target p(z_t, x_t | previous set).             */
/* ------------------------------------------------------------------------ */

/* grad_x of the prior term. fprev[j] = f_t(x_{t-1}^j), j < Np. */
void om_grad_prior(const om_model* m, int prior, const double* fprev, const double* phiprev, int Np,
                   const double* x, double* g)
{
    int d = m->d;
    for (int c = 0; c < d; ++c) g[c] = 0.0;
    if (prior == OM_PRIOR_MAPCOND) {
        /* MAP-conditioned (the prior conditioned on the previous MAP estimates,
         * Section V-C): the score of max_j [phi_{t-1}(j) + log N(x; f_j, Q)],
         * i.e. Q^-1 (f_{j*} - x) with j* that maximiser (lowest j on ties);
         * phiprev NULL counts as all zeros. */
        int best = 0;
        double bv = -INFINITY;
        for (int j = 0; j < Np; ++j) {
            double v = (phiprev ? phiprev[j] : 0.0) + om_logtrans(m, x, fprev + (long)j * d);
            if (v > bv) { bv = v; best = j; }
        }
        for (int c = 0; c < d; ++c) g[c] = (fprev[(long)best * d + c] - x[c]) / m->q[c];
        return;
    }
    if (prior == OM_PRIOR_MEANGRAD) {
        /* (1/Np) sum_j grad log N(x; f_j, Q) = Q^-1 (mean_j f_j - x) */
        for (int j = 0; j < Np; ++j)
            for (int c = 0; c < d; ++c) g[c] += (fprev[(long)j * d + c] - x[c]) / m->q[c];
        for (int c = 0; c < d; ++c) g[c] /= Np;
        return;
    }
    /* MIXTURE: grad log (1/Np) sum_j N(x; f_j, Q)
     *        = sum_j w_j Q^-1 (f_j - x),  w_j proportional to N(x; f_j, Q). */
    double* lw = (double*)malloc(sizeof(double) * Np);
    double mx = -INFINITY;
    for (int j = 0; j < Np; ++j) {
        lw[j] = om_logtrans(m, x, fprev + (long)j * d);
        if (lw[j] > mx) mx = lw[j];
    }
    double s = 0.0;
    for (int j = 0; j < Np; ++j) { lw[j] = exp(lw[j] - mx); s += lw[j]; }
    for (int j = 0; j < Np; ++j) {
        double w = lw[j] / s;
        for (int c = 0; c < d; ++c) g[c] += w * (fprev[(long)j * d + c] - x[c]) / m->q[c];
    }
    free(lw);
}

/* grad_x log p(z_t, x | previous set) at one particle. */
static void om_score(const om_model* m, int prior, int t, const double* z,
                     const double* fprev, const double* phiprev, int Np, const double* x, double* g)
{
    double gl[OM_MAXD], gp[OM_MAXD];
    om_grad_loglik(m, t, z, x, gl);
    om_grad_prior(m, prior, fprev, phiprev, Np, x, gp);
    for (int c = 0; c < m->d; ++c) g[c] = gl[c] + gp[c];
}

/* One SVGD iteration (Algorithm 1, Eq. svgd_iterate with the score of
 * Eq. SVGD_initial_newupdate / SVGD_newupdate): all particles move together. */
void om_svgd_iteration(const om_model* m, int prior, int t, const double* z,
                       const double* fprev, const double* phiprev, int Np, double* x, int N,
                       double h, double eps, int kernel)
{
    int d = m->d;
    double* g = (double*)malloc(sizeof(double) * N * d);
    double* phi = (double*)calloc((size_t)N * d, sizeof(double));
    for (int k = 0; k < N; ++k) om_score(m, prior, t, z, fprev, phiprev, Np, x + (long)k * d, g + (long)k * d);
    for (int i = 0; i < N; ++i) {
        const double* xi = x + (long)i * d;
        for (int k = 0; k < N; ++k) {
            const double* xk = x + (long)k * d;
            double kap, rho;
            om_kernel(kernel, xi, xk, d, h, &kap, &rho);
            for (int c = 0; c < d; ++c) {
                double drive = kap * g[(long)k * d + c];
                double repulse = rho * (xi[c] - xk[c]);  /* grad_{x_k} kappa(x_k, x_i) */
                phi[(long)i * d + c] += drive + repulse;
            }
        }
        for (int c = 0; c < d; ++c) phi[(long)i * d + c] /= N;
    }
    for (long n = 0; n < (long)N * d; ++n) x[n] += eps * phi[n];
    free(g);
    free(phi);
}

/* L SVGD iterations at step t from the given initial particles.
 * h_out[l] receives the bandwidth used at iteration l (may be NULL). */
void om_svgd_iters(const om_model* m, int prior, int bw_rule, double bw_value,
                   int t, const double* z, const double* fprev, const double* phiprev, int Np,
                   double* x, int N, int L, double eps, double* h_out, int kernel)
{
    double h = 1.0;
    for (int l = 0; l < L; ++l) {
        if (bw_rule == OM_BW_FIXED) h = bw_value;
        else if (bw_rule == OM_BW_MEDIAN_ITER || l == 0) h = om_bandwidth(x, N, m->d, bw_value);
        if (h_out) h_out[l] = h;
        om_svgd_iteration(m, prior, t, z, fprev, phiprev, Np, x, N, h, eps, kernel);
    }
}

/* ------------------------------------------------------------------------ */
/* Particle dynamic programming (Section IV-B, Eq. forward_recursion).       */
/* ------------------------------------------------------------------------ */

/* One forward step. Np == 1 is the initialisation phi_1(i) =
 * log p(z_1, x_1^i | x_0^true) (phi_prev = {0}); otherwise
 *   psi_t(i) = argmax_j { log p(x_t^i | x_{t-1}^j) + phi_{t-1}(j) }  (lowest j)
 *   phi_t(i) = log p(z_t, x_t^i | x_{t-1}^{psi}) + phi_{t-1}(psi).            */
void om_forward(const om_model* m, int t, const double* z, const double* fprev,
                int Np, const double* phi_prev, const double* x, int N,
                int* psi, double* phi)
{
    int d = m->d;
    for (int i = 0; i < N; ++i) {
        const double* xi = x + (long)i * d;
        int best = 0;
        double bestv = -INFINITY;
        for (int j = 0; j < Np; ++j) {
            double v = om_logtrans(m, xi, fprev + (long)j * d) + phi_prev[j];
            if (v > bestv) { bestv = v; best = j; }
        }
        psi[i] = best;
        phi[i] = om_loglik(m, t, z, xi) + om_logtrans(m, xi, fprev + (long)best * d)
               + phi_prev[best];
    }
}

/* Backtracking: i_T = argmax phi_T (lowest i); i_t = psi_{t+1}(i_{t+1}).
 * hist is [T][N][d] (steps 1..T), psi [T][N]; path [T+1][d] with path[0]=x0.
 * Returns J = phi_T(i_T). */
double om_backtrack(int d, int N, int T, const double* x0, const double* hist,
                    const int* psi, const double* phiT, double* path, int* idx)
{
    int it = 0;
    for (int i = 1; i < N; ++i) if (phiT[i] > phiT[it]) it = i;
    double J = phiT[it];
    for (int t = T; t >= 1; --t) {
        if (idx) idx[t - 1] = it;
        for (int c = 0; c < d; ++c) path[(long)t * d + c] = hist[((long)(t - 1) * N + it) * d + c];
        if (t > 1) it = psi[(long)(t - 1) * N + it];
    }
    for (int c = 0; c < d; ++c) path[c] = x0[c];
    return J;
}

/* J(s) = sum_{t>=1} log p(z_t, s_t | s_{t-1}) for a given path s_{0:T}
 * (Theorem 1, with the constant log p(s_0) left out). */
double om_path_score(const om_model* m, int T, const double* path, const double* z)
{
    int d = m->d;
    double J = 0.0, f[OM_MAXD];
    for (int t = 1; t <= T; ++t) {
        om_transition(m, t, path + (long)(t - 1) * d, f);
        J += om_loglik(m, t, z + (long)(t - 1) * m->dy, path + (long)t * d)
           + om_logtrans(m, path + (long)t * d, f);
    }
    return J;
}

/* ------------------------------------------------------------------------ */
/* Whole sequence (Algorithm 2).                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind; const double* params; int np;
    int N, L; double eps; int bw_rule; double bw_value; int prior;
    uint64_t seed;
    int kernel;   /* OM_KERNEL_* */
} om_run_cfg;

/* Runs one sequence of length T. z is [T][dy]. Outputs (any may be NULL
 * except path/J): hist [T][N][d] (final particles of each step), psi [T][N],
 * path [T+1][d], J. Returns 0 or -1 on bad input. */
int om_run_sequence(const om_run_cfg* cfg, uint32_t seq, const double* x0, int T,
                    const double* z, double* hist, int* psi, double* path, double* J)
{
    om_model m;
    if (om_setup(&m, cfg->kind, cfg->params, cfg->np)) return -1;
    int d = m.d, N = cfg->N;
    if (N < 1 || T < 1) return -1;
    double* xprev = (double*)malloc(sizeof(double) * N * d);
    double* fprev = (double*)malloc(sizeof(double) * N * d);
    double* x = (double*)malloc(sizeof(double) * N * d);
    double* phi_prev = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    int* psi_t = (int*)malloc(sizeof(int) * N);
    double* H = hist ? hist : (double*)malloc(sizeof(double) * (size_t)T * N * d);
    int* PSI = psi ? psi : (int*)malloc(sizeof(int) * (size_t)T * N);
    int Np = 1;
    memcpy(xprev, x0, sizeof(double) * d);
    phi_prev[0] = 0.0;
    for (int t = 1; t <= T; ++t) {
        const double* zt = z + (long)(t - 1) * m.dy;
        for (int j = 0; j < Np; ++j) om_transition(&m, t, xprev + (long)j * d, fprev + (long)j * d);
        for (int i = 0; i < N; ++i) {
            double xi[OM_MAXD];
            om_normals(cfg->seed, seq, (uint32_t)t, (uint32_t)i, d, xi);
            const double* fi = fprev + (long)(Np == 1 ? 0 : i) * d;
            for (int c = 0; c < d; ++c) x[(long)i * d + c] = fi[c] + sqrt(m.q[c]) * xi[c];
        }
        om_svgd_iters(&m, cfg->prior, cfg->bw_rule, cfg->bw_value, t, zt, fprev, phi_prev, Np,
                      x, N, cfg->L, cfg->eps, NULL, cfg->kernel);
        om_forward(&m, t, zt, fprev, Np, phi_prev, x, N, psi_t, phi);
        memcpy(H + (size_t)(t - 1) * N * d, x, sizeof(double) * N * d);
        memcpy(PSI + (size_t)(t - 1) * N, psi_t, sizeof(int) * N);
        memcpy(xprev, x, sizeof(double) * N * d);
        memcpy(phi_prev, phi, sizeof(double) * N);
        Np = N;
    }
    double Jv = om_backtrack(d, N, T, x0, H, PSI, phi_prev, path, NULL);
    if (J) *J = Jv;
    if (!hist) free(H);
    if (!psi) free(PSI);
    free(xprev); free(fprev); free(x); free(phi_prev); free(phi); free(psi_t);
    return 0;
}

/* DP only (forward recursion + backtracking) over given particle sets
 * hist [T][N][d]: the second stage of Algorithm 2 on fixed supports. */
int om_viterbi_sets(int kind, const double* params, int np, int N, int T,
                    const double* x0, const double* hist, const double* z,
                    int* psi, double* phiT, double* path, double* J)
{
    om_model m;
    if (om_setup(&m, kind, params, np)) return -1;
    int d = m.d;
    double* fprev = (double*)malloc(sizeof(double) * N * d);
    double* phi_prev = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    int Np = 1;
    phi_prev[0] = 0.0;
    om_transition(&m, 1, x0, fprev);
    for (int t = 1; t <= T; ++t) {
        if (t > 1)
            for (int j = 0; j < N; ++j)
                om_transition(&m, t, hist + ((size_t)(t - 2) * N + j) * d, fprev + (long)j * d);
        om_forward(&m, t, z + (long)(t - 1) * m.dy, fprev, Np, phi_prev,
                   hist + (size_t)(t - 1) * N * d, N, psi + (size_t)(t - 1) * N, phi);
        memcpy(phi_prev, phi, sizeof(double) * N);
        Np = N;
    }
    if (phiT) memcpy(phiT, phi_prev, sizeof(double) * N);
    double Jv = om_backtrack(d, N, T, x0, hist, psi, phi_prev, path, NULL);
    if (J) *J = Jv;
    free(fprev); free(phi_prev); free(phi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* PF-MAP-Seq, the comparison method of Section V (Godsill, Doucet and West, */
/* "Maximum a posteriori sequence estimation using Monte Carlo particle      */
/* filters", 2001): a bootstrap particle filter supplies the supports, the   */
/* same forward recursion and backtracking then pick the MAP sequence.       */
/* Readings (the paper names the method and its stratified resampling at     */
/* every step, nothing more):                                                */
/*   x_1^i = f_1(x_0) + sqrt(q) (.) xi, log w_1^i = log p(z_1 | x_1^i);       */
/*   t >= 2: stratified resampling of the step t-1 weights, u_i = (i + U_i)/N,*/
/*   ancestor a_i = the first j whose normalised cumulative weight exceeds   */
/*   u_i; x_t^i = f_t(x_{t-1}^{a_i}) + sqrt(q) (.) xi; log w_t^i =            */
/*   log p(z_t | x_t^i). xi: om_normals with counter (i, t, seq, block);      */
/*   U_i = (w0 + 1/2) / 2^32 from the Philox word w0 of counter               */
/*   (i, t, seq, 256). The supports of the recursion are the sets x_t.       */
/* ------------------------------------------------------------------------ */
double om_uniform(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { i, t, seq, 256u }, w[4];
    om_philox4x32_10(ctr, key, w);
    return ((double)w[0] + 0.5) * (1.0 / 4294967296.0);
}

/* hist [T][N][d] (out), anc [T][N] ancestors (out, anc[0][i] = 0; may be NULL). */
int om_pf_sets(int kind, const double* params, int np, int N, int T, uint64_t seed, uint32_t seq,
               const double* x0, const double* z, double* hist, int* anc)
{
    om_model m;
    if (om_setup(&m, kind, params, np) || N < 1 || T < 1) return -1;
    int d = m.d;
    double* lw = (double*)malloc(sizeof(double) * N);
    double* c = (double*)malloc(sizeof(double) * N);
    double f[OM_MAXD], xi[OM_MAXD];
    for (int t = 1; t <= T; ++t) {
        double* cur = hist + (size_t)(t - 1) * N * d;
        const double* prev = t > 1 ? hist + (size_t)(t - 2) * N * d : NULL;
        if (t > 1) {
            /* normalised cumulative weights of step t-1 */
            double mx = -INFINITY, W = 0.0;
            for (int j = 0; j < N; ++j) if (lw[j] > mx) mx = lw[j];
            for (int j = 0; j < N; ++j) { W += exp(lw[j] - mx); c[j] = W; }
            for (int j = 0; j < N; ++j) c[j] /= W;
            for (int i = 0; i < N; ++i) {
                double u = ((double)i + om_uniform(seed, seq, (uint32_t)t, (uint32_t)i)) / (double)N;
                int a = 0;
                while (a < N - 1 && !(c[a] > u)) ++a;
                if (anc) anc[(size_t)(t - 1) * N + i] = a;
                om_transition(&m, t, prev + (size_t)a * d, f);
                om_normals(seed, seq, (uint32_t)t, (uint32_t)i, d, xi);
                for (int k = 0; k < d; ++k) cur[(size_t)i * d + k] = f[k] + sqrt(m.q[k]) * xi[k];
            }
        } else {
            om_transition(&m, 1, x0, f);
            for (int i = 0; i < N; ++i) {
                if (anc) anc[i] = 0;
                om_normals(seed, seq, 1u, (uint32_t)i, d, xi);
                for (int k = 0; k < d; ++k) cur[(size_t)i * d + k] = f[k] + sqrt(m.q[k]) * xi[k];
            }
        }
        for (int i = 0; i < N; ++i) lw[i] = om_loglik(&m, t, z + (size_t)(t - 1) * m.dy, cur + (size_t)i * d);
    }
    free(lw); free(c);
    return 0;
}

/* For fixed particle sets: the relative margin of every backpointer,
 * (best - second best) / max(1, |best|) over j of phi_{t-1}(j) +
 * log p(x_t^i | x_{t-1}^j), margin[T][N] (t = 1 has a single candidate:
 * +inf). Used to decide where backpointers are unique to 1e-6. */
int om_viterbi_margins(int kind, const double* params, int np, int N, int T, const double* x0,
                       const double* hist, const double* z, double* margin)
{
    om_model m;
    if (om_setup(&m, kind, params, np)) return -1;
    int d = m.d;
    double* fprev = (double*)malloc(sizeof(double) * N * d);
    double* phi_prev = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    int* psi = (int*)malloc(sizeof(int) * N);
    int Np = 1;
    phi_prev[0] = 0.0;
    om_transition(&m, 1, x0, fprev);
    for (int t = 1; t <= T; ++t) {
        const double* xt = hist + (size_t)(t - 1) * N * d;
        if (t > 1)
            for (int j = 0; j < N; ++j)
                om_transition(&m, t, hist + ((size_t)(t - 2) * N + j) * d, fprev + (long)j * d);
        for (int i = 0; i < N; ++i) {
            double b1 = -INFINITY, b2 = -INFINITY;
            for (int j = 0; j < Np; ++j) {
                double v = om_logtrans(&m, xt + (long)i * d, fprev + (long)j * d) + phi_prev[j];
                if (v > b1) { b2 = b1; b1 = v; } else if (v > b2) { b2 = v; }
            }
            double den = fabs(b1) > 1.0 ? fabs(b1) : 1.0;
            margin[(size_t)(t - 1) * N + i] = (Np == 1) ? INFINITY : (b1 - b2) / den;
        }
        om_forward(&m, t, z + (long)(t - 1) * m.dy, fprev, Np, phi_prev, xt, N, psi, phi);
        memcpy(phi_prev, phi, sizeof(double) * N);
        Np = N;
    }
    free(fprev); free(phi_prev); free(phi); free(psi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Many sequences on host threads (the CPU baseline runs this).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    const om_run_cfg* cfg;
    const double* x0; const double* z; const int* T; const int* seq_ids;
    int maxT, d, dy, nseq, nthreads, tid;
    double* path; double* J; int rc;
} om_job;

static void* om_worker(void* arg)
{
    om_job* jb = (om_job*)arg;
    for (int s = jb->tid; s < jb->nseq; s += jb->nthreads) {
        int rc = om_run_sequence(jb->cfg, (uint32_t)jb->seq_ids[s], jb->x0 + (long)s * jb->d,
                                 jb->T[s], jb->z + (size_t)s * jb->maxT * jb->dy, NULL, NULL,
                                 jb->path + (size_t)s * (jb->maxT + 1) * jb->d, jb->J + s);
        if (rc) jb->rc = rc;
    }
    return NULL;
}

int om_run_batch(int kind, const double* params, int np, int N, int L, double eps,
                 int bw_rule, double bw_value, int prior, uint64_t seed,
                 int nseq, const int* seq_ids, const double* x0, int maxT, const int* T,
                 const double* z, double* path, double* J, int nthreads, int kernel)
{
    om_model m;
    if (om_setup(&m, kind, params, np)) return -1;
    om_run_cfg cfg = { kind, params, np, N, L, eps, bw_rule, bw_value, prior, seed, kernel };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    om_job jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        om_job jb = { &cfg, x0, z, T, seq_ids, maxT, m.d, m.dy, nseq, nthreads, k, path, J, 0 };
        jobs[k] = jb;
        pthread_create(&th[k], NULL, om_worker, &jobs[k]);
    }
    int rc = 0;
    for (int k = 0; k < nthreads; ++k) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Learned proposal: a 3-layer perceptron in -> H -> H -> out, GELU after    */
/* the two hidden layers, trained by mean squared error with Adam. This part */
/* is not in the paper (the build adds it); the oracle is the plain FP64     */
/* definition used to check the GPU's forward and backward passes.           */
/* Packed parameters: W1 [H][in], b1 [H], W2 [H][H], b2 [H], W3 [out][H],    */
/* b3 [out]. GELU in its tanh form (Hendrycks & Gimpel 2016):                */
/*   gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).                */
/* ------------------------------------------------------------------------ */
static double om_gelu(double x)
{
    const double k0 = 0.7978845608028654, k1 = 0.044715;
    return 0.5 * x * (1.0 + tanh(k0 * (x + k1 * x * x * x)));
}

static double om_gelu_grad(double x)
{
    const double k0 = 0.7978845608028654, k1 = 0.044715;
    double u = k0 * (x + k1 * x * x * x), th = tanh(u);
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * k0 * (1.0 + 3.0 * k1 * x * x);
}

long om_mlp_nparams(int in, int H, int out)
{
    return (long)H * in + H + (long)H * H + H + (long)out * H + out;
}

/* y = MLP(x) for `rows` rows of X [rows][in]; Y [rows][out]. */
void om_mlp_forward(int in, int H, int out, const double* W, long rows, const double* X, double* Y)
{
    const double *W1 = W, *b1 = W1 + (long)H * in, *W2 = b1 + H, *b2 = W2 + (long)H * H;
    const double *W3 = b2 + H, *b3 = W3 + (long)out * H;
    double* h1 = (double*)malloc(sizeof(double) * H);
    double* h2 = (double*)malloc(sizeof(double) * H);
    for (long r = 0; r < rows; ++r) {
        const double* x = X + r * in;
        for (int j = 0; j < H; ++j) {
            double z = b1[j];
            for (int k = 0; k < in; ++k) z += W1[(long)j * in + k] * x[k];
            h1[j] = om_gelu(z);
        }
        for (int j = 0; j < H; ++j) {
            double z = b2[j];
            for (int k = 0; k < H; ++k) z += W2[(long)j * H + k] * h1[k];
            h2[j] = om_gelu(z);
        }
        for (int o = 0; o < out; ++o) {
            double z = b3[o];
            for (int k = 0; k < H; ++k) z += W3[(long)o * H + k] * h2[k];
            Y[r * out + o] = z;
        }
    }
    free(h1); free(h2);
}

/* loss = mean over rows and outputs of (y - t)^2 and its gradient G (packed
 * like W) by the chain rule, row by row. Returns the loss. */
double om_mlp_loss_grad(int in, int H, int out, const double* W, long rows, const double* X,
                        const double* Tg, double* G)
{
    const double *W1 = W, *b1 = W1 + (long)H * in, *W2 = b1 + H, *b2 = W2 + (long)H * H;
    const double *W3 = b2 + H, *b3 = W3 + (long)out * H;
    double *G1 = G, *g1 = G1 + (long)H * in, *G2 = g1 + H, *g2 = G2 + (long)H * H;
    double *G3 = g2 + H, *g3 = G3 + (long)out * H;
    long np = om_mlp_nparams(in, H, out);
    for (long k = 0; k < np; ++k) G[k] = 0.0;
    double* z1 = (double*)malloc(sizeof(double) * H);
    double* h1 = (double*)malloc(sizeof(double) * H);
    double* z2 = (double*)malloc(sizeof(double) * H);
    double* h2 = (double*)malloc(sizeof(double) * H);
    double* dy = (double*)malloc(sizeof(double) * out);
    double* d2 = (double*)malloc(sizeof(double) * H);
    double* d1 = (double*)malloc(sizeof(double) * H);
    double loss = 0.0, scale = 1.0 / ((double)rows * out);
    for (long r = 0; r < rows; ++r) {
        const double* x = X + r * in;
        for (int j = 0; j < H; ++j) {
            double z = b1[j];
            for (int k = 0; k < in; ++k) z += W1[(long)j * in + k] * x[k];
            z1[j] = z; h1[j] = om_gelu(z);
        }
        for (int j = 0; j < H; ++j) {
            double z = b2[j];
            for (int k = 0; k < H; ++k) z += W2[(long)j * H + k] * h1[k];
            z2[j] = z; h2[j] = om_gelu(z);
        }
        for (int o = 0; o < out; ++o) {
            double z = b3[o];
            for (int k = 0; k < H; ++k) z += W3[(long)o * H + k] * h2[k];
            double e = z - Tg[r * out + o];
            loss += e * e * scale;
            dy[o] = 2.0 * e * scale;
        }
        /* layer 3 */
        for (int o = 0; o < out; ++o) {
            g3[o] += dy[o];
            for (int k = 0; k < H; ++k) G3[(long)o * H + k] += dy[o] * h2[k];
        }
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int o = 0; o < out; ++o) s += dy[o] * W3[(long)o * H + k];
            d2[k] = s * om_gelu_grad(z2[k]);
        }
        /* layer 2 */
        for (int j = 0; j < H; ++j) {
            g2[j] += d2[j];
            for (int k = 0; k < H; ++k) G2[(long)j * H + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int j = 0; j < H; ++j) s += d2[j] * W2[(long)j * H + k];
            d1[k] = s * om_gelu_grad(z1[k]);
        }
        /* layer 1 */
        for (int j = 0; j < H; ++j) {
            g1[j] += d1[j];
            for (int k = 0; k < in; ++k) G1[(long)j * in + k] += d1[j] * x[k];
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(dy); free(d2); free(d1);
    return loss;
}

/* One Adam step (Kingma & Ba 2015) with bias correction, step count t >= 1. */
void om_adam(long n, double* theta, const double* g, double* m, double* v, int t, double lr,
             double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (long k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* Proposal features of a propagated particle u and observation z (at most 32),
 * each list ending with the likelihood score g = grad_u log p(z | u):
 *   PLANAR_ARM   [u, z, z - h(u), g of the angles]
 *   CLUTTER_CV2D [velocity, z_m - position for the points nearest first, g of the position]
 *   others       [u, z with NaN -> 0, 1 where z is a number, g]
 * Returns the count. */
int om_proposal_features(int kind, const double* params, int np, const double* u, const double* z,
                         double* f)
{
    om_model m;
    if (om_setup(&m, kind, params, np)) return -1;
    int d = m.d, n = 0;
    double g[OM_MAXD];
    om_grad_loglik(&m, 1, z, u, g);
    if (kind == OM_PLANAR_ARM) {
        double e[2];
        om_arm_fk(&m, u, e, NULL);
        for (int c = 0; c < d; ++c) f[n++] = u[c];
        f[n++] = z[0]; f[n++] = z[1];
        f[n++] = z[0] - e[0]; f[n++] = z[1] - e[1];
        for (int c = 0; c < d / 2; ++c) f[n++] = g[c];
    } else if (kind == OM_CLUTTER_CV2D) {
        int M = (int)m.p[6], nm = M < 14 ? M : 14;
        double dist[32];
        int used[32] = {0};
        f[n++] = u[2]; f[n++] = u[3];
        for (int k = 0; k < M; ++k) {
            double ex = z[2 * k] - u[0], ey = z[2 * k + 1] - u[1];
            dist[k] = ex * ex + ey * ey;
        }
        for (int r = 0; r < nm; ++r) {          /* nearest remaining point */
            int best = -1;
            for (int k = 0; k < M; ++k)
                if (!used[k] && (best < 0 || dist[k] < dist[best])) best = k;
            used[best] = 1;
            f[n++] = z[2 * best] - u[0];
            f[n++] = z[2 * best + 1] - u[1];
        }
        f[n++] = g[0]; f[n++] = g[1];
    } else {
        int dy = m.dy < (32 - 2 * d) / 2 ? m.dy : (32 - 2 * d) / 2;
        for (int c = 0; c < d; ++c) f[n++] = u[c];
        for (int c = 0; c < dy; ++c) f[n++] = isnan(z[c]) ? 0.0 : z[c];
        for (int c = 0; c < dy; ++c) f[n++] = isnan(z[c]) ? 0.0 : 1.0;
        for (int c = 0; c < d; ++c) f[n++] = g[c];
    }
    return n;
}
