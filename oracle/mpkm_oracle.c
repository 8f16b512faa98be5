/*
 * mpkm_oracle.c -- CPU FP64 oracle for mixed-precision Lloyd's k-means.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only tests/, the smoke
 * check and the bench's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA library (the library never includes
 * or links it), and nothing in it is tuned.
 *
 * Source: E. Carson, X. Chen, X. Liu, "Computing k-means in Mixed Precision"
 * (arXiv 2407.12208).  Each function names the passage it follows.
 *
 * Layout: X is n x d row-major fp32 (points as rows, as in Eq. (dist-blas3)),
 * C is k x d row-major fp32.  All arithmetic is binary64 unless a function
 * says it emulates a lower format.  Build with -ffp-contract=off so that no
 * compiler fuses a*b+c: results are then identical on x86-64 and aarch64.
 *
 * Pins (see tests/test_oracle_*.py): brute force in exact rational arithmetic
 * on tiny inputs, Theorem 4.1's bound, Lemma 2.1's identity, monotone SSE,
 * the argmin / lowest-index property, Table 1.1 formats against torch's
 * conversions, the closed-form all-flag thresholds of Alg. 2, the worked
 * cancellation example of Section 4.3, and the rigorous error bounds of
 * Theorem 4.2 / Eq. (quantis-rel-bound-expand).  No function is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EUNSUPPORTED 7

/* ------------------------------------------------------------------------ */
/* Table 1.1: floating-point formats.  fmt 0 = binary16, 1 = bfloat16,
 * 2 = FP8 E4M3 ("fn" variant: no infinities, largest finite 448; not in the
 * paper's table, t = 4 significand bits), 3 = binary32.  Rounding is to nearest, ties to
 * even; fp16/bf16 overflow to infinity, E4M3 saturates to +-448 (the
 * behaviour of the hardware's satfinite conversion).                       */
/* ------------------------------------------------------------------------ */
static void fmt_params(int fmt, int* t, int* emin, double* xmax, int* sat) {
    switch (fmt) {
    case 0: *t = 11; *emin = -14;  *xmax = 65504.0; *sat = 0; break;
    case 1: *t = 8;  *emin = -126; *xmax = ldexp(255.0, 120); *sat = 0; break;
    case 3: *t = 24; *emin = -126; *xmax = ldexp(16777215.0, 104); *sat = 0; break;  /* binary32 */
    default: *t = 4; *emin = -6;   *xmax = 448.0; *sat = 1; break;
    }
}

/* unit roundoff u = 2^-t of Table 1.1 */
double orc_unit_roundoff(int fmt) {
    if (fmt == 3) return ldexp(1.0, -24);   /* binary32 */
    if (fmt == 4) return ldexp(1.0, -53);   /* binary64 */
    int t, emin, sat; double xmax;
    fmt_params(fmt, &t, &emin, &xmax, &sat);
    return ldexp(1.0, -t);
}

/* Round an exact binary64 value v to the format: the significand keeps t bits
 * at the value's own exponent, or at emin for subnormals (fixed quantum). */
double orc_round_to_format(double v, int fmt) {
    int t, emin, sat; double xmax;
    if (v == 0.0 || isnan(v)) return v;
    fmt_params(fmt, &t, &emin, &xmax, &sat);
    if (isinf(v)) return sat ? copysign(xmax, v) : v;
    double a = fabs(v);
    int e;
    frexp(a, &e);                 /* a = f * 2^e, f in [0.5, 1) */
    int E = e - 1;                /* exponent of the leading bit */
    if (E < emin) E = emin;       /* subnormal range: quantum 2^(emin-t+1) */
    double quantum = ldexp(1.0, E - (t - 1));
    double r = nearbyint(a / quantum) * quantum;   /* ties to even */
    if (r > xmax) r = sat ? xmax : INFINITY;
    return copysign(r, v);
}

void orc_quantize(const float* x, int64_t len, int fmt, float* out) {
    for (int64_t i = 0; i < len; i++) out[i] = (float)orc_round_to_format((double)x[i], fmt);
}

/* gamma_m = m u / (1 - m u), Eq. (fpmode-vecprod); returns +inf if m u >= 1 */
double orc_gamma(int m, double u) {
    double mu = (double)m * u;
    if (mu >= 1.0) return INFINITY;
    return mu / (1.0 - mu);
}

/* ------------------------------------------------------------------------ */
/* Eq. (dist-direct): d(x,y)^2 = (x-y)^T (x-y), evaluated in binary64.      */
/* ------------------------------------------------------------------------ */
double orc_dist_direct_pair(const float* x, const float* y, int d) {
    double s = 0.0;
    for (int l = 0; l < d; l++) {
        double t = (double)x[l] - (double)y[l];
        s += t * t;
    }
    return s;
}

/* Eq. (dist-direct) for one given centre per point: out[i] = d(x_i, c_{labels[i]})^2,
 * the distance the assignment reports for the centre it chose.            */
void orc_dist_labelled(const float* X, int64_t n, const float* C, int k, int d, const int32_t* labels,
                       double* out) {
    for (int64_t i = 0; i < n; i++) {
        int j = labels[i];
        out[i] = (j >= 0 && j < k) ? orc_dist_direct_pair(X + i * d, C + (int64_t)j * d, d) : NAN;
    }
}

void orc_dist_direct(const float* X, int64_t n, const float* C, int k, int d, double* D) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int j = 0; j < k; j++)
            D[i * k + j] = orc_dist_direct_pair(X + i * d, C + (int64_t)j * d, d);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1, assignment lines: label_i = argmin_j d(p_i, c_j)^2.  Ties go to
 * the lowest centre index.  d1 = best distance, d2 = second-best distance
 * (over the other centres; +inf when k = 1).                               */
/* ------------------------------------------------------------------------ */
void orc_assign(const float* X, int64_t n, const float* C, int k, int d,
                int32_t* labels, double* d1, double* d2) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double best = INFINITY, second = INFINITY;
        int32_t arg = 0;
        for (int j = 0; j < k; j++) {
            double v = orc_dist_direct_pair(X + i * d, C + (int64_t)j * d, d);
            if (v < best) { second = best; best = v; arg = j; }
            else if (v < second) { second = v; }
        }
        labels[i] = arg;
        if (d1) d1[i] = best;
        if (d2) d2[i] = second;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (center) with Lemma 4.4's recursive summation: for each cluster the
 * members are summed in ascending point index in binary64, divided by m_j,
 * and the mean is stored in the working precision (fp32), Alg. 3.
 *
 * Empty clusters (the paper only says they are "automatically
 * reinitialised", Section 6.2): empty_policy 0 keeps the old centre;
 * empty_policy 1 takes, for the empty clusters in ascending j, the point
 * with the largest min_dist (ties: lowest index), each point at most once.
 * shift = max_j ||c_new_j - c_old_j|| (Euclidean, not squared), Alg. 1.    */
/* ------------------------------------------------------------------------ */
int orc_update(const float* X, int64_t n, int d, const int32_t* labels, int k,
               const float* C_old, int empty_policy, const double* min_dist,
               float* C_new, int64_t* counts, double* shift) {
    double* sum = (double*)calloc((size_t)k * d, sizeof(double));
    if (!sum) return ORC_EINVAL;
    for (int j = 0; j < k; j++) counts[j] = 0;
    for (int64_t i = 0; i < n; i++) {
        int j = labels[i];
        if (j < 0 || j >= k) { free(sum); return ORC_EINVAL; }
        counts[j]++;
        for (int l = 0; l < d; l++) sum[(int64_t)j * d + l] += (double)X[i * d + l];
    }
    unsigned char* taken = NULL;
    for (int j = 0; j < k; j++) {
        if (counts[j] > 0) {
            for (int l = 0; l < d; l++)
                C_new[(int64_t)j * d + l] = (float)(sum[(int64_t)j * d + l] / (double)counts[j]);
        } else if (empty_policy == 1 && min_dist != NULL) {
            if (!taken) taken = (unsigned char*)calloc((size_t)n, 1);
            int64_t arg = -1; double best = -1.0;
            for (int64_t i = 0; i < n; i++)
                if (!taken[i] && min_dist[i] > best) { best = min_dist[i]; arg = i; }
            if (arg >= 0) {
                taken[arg] = 1;
                for (int l = 0; l < d; l++) C_new[(int64_t)j * d + l] = X[arg * d + l];
            } else {
                for (int l = 0; l < d; l++) C_new[(int64_t)j * d + l] = C_old[(int64_t)j * d + l];
            }
        } else {
            for (int l = 0; l < d; l++) C_new[(int64_t)j * d + l] = C_old[(int64_t)j * d + l];
        }
    }
    double mx = 0.0;
    for (int j = 0; j < k; j++) {
        double s = 0.0;
        for (int l = 0; l < d; l++) {
            double t = (double)C_new[(int64_t)j * d + l] - (double)C_old[(int64_t)j * d + l];
            s += t * t;
        }
        if (sqrt(s) > mx) mx = sqrt(s);
    }
    *shift = mx;
    free(taken);
    free(sum);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (Lloyd) with binary64 direct distances.  tau <= 0 runs exactly
 * max_iter iterations.  sse_per_iter[t] = SSE (Eq. (sse)) of the assignment
 * made in iteration t+1 (against the centres c^(t)); sse_per_iter[iters] is
 * the SSE of the final reassignment (last line of Alg. 1).                 */
/* ------------------------------------------------------------------------ */
int orc_lloyd(const float* X, int64_t n, int d, int k, const float* C_init,
              int max_iter, double tau, int empty_policy,
              float* C_out, int32_t* labels, double* sse_per_iter, int* iters_done) {
    if (n < 1 || d < 1 || k < 1 || k > n || max_iter < 0) return ORC_EINVAL;
    float* Cc = (float*)malloc(sizeof(float) * (size_t)k * d);
    float* Cn = (float*)malloc(sizeof(float) * (size_t)k * d);
    double* md = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    if (!Cc || !Cn || !md || !cnt) { free(Cc); free(Cn); free(md); free(cnt); return ORC_EINVAL; }
    memcpy(Cc, C_init, sizeof(float) * (size_t)k * d);
    int t = 0;
    for (t = 0; t < max_iter; t++) {
        orc_assign(X, n, Cc, k, d, labels, md, NULL);
        double sse = 0.0;
        for (int64_t i = 0; i < n; i++) sse += md[i];
        if (sse_per_iter) sse_per_iter[t] = sse;
        double shift = 0.0;
        orc_update(X, n, d, labels, k, Cc, empty_policy, md, Cn, cnt, &shift);
        memcpy(Cc, Cn, sizeof(float) * (size_t)k * d);
        if (tau > 0.0 && shift < tau) { t++; break; }
    }
    orc_assign(X, n, Cc, k, d, labels, md, NULL);
    double sse = 0.0;
    for (int64_t i = 0; i < n; i++) sse += md[i];
    if (sse_per_iter) sse_per_iter[t] = sse;
    memcpy(C_out, Cc, sizeof(float) * (size_t)k * d);
    *iters_done = t;
    free(Cc); free(Cn); free(md); free(cnt);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2, verbatim, in emulated low precision ("paper" test).  Every
 * operation on the quantised data is rounded to the low format: the dot
 * products by recursive summation, then d = max(fl(d_xx - 2 d_xy + d_yy), 0)
 * and E = fl(rho * c_A * gamma^l_{r+2} * (d_xx + d_yy)).  c_A is 1 for Alg. 2
 * as printed and 2 for E^l of Eq. (quantis-reliability-test).  If d <= E the
 * pair falls back to the direct formula on the ORIGINAL data in binary64
 * (Section 4.3).  Returns 1 if the pair was flagged, 0 if not, -1 if
 * gamma^l_{r+2} is undefined ((r+2) u_l >= 1).  d_out receives the value
 * Alg. 2 returns; dhat_out and E_out the low-precision quantities.         */
/* ------------------------------------------------------------------------ */
int orc_mp_dist_paper(const float* x, const float* y, int r, double rho, double c_A, int fmt,
                      double* d_out, double* dhat_out, double* E_out);

static double lo_dot(const float* a, const float* b, int r, int fmt) {
    double s = 0.0;
    for (int l = 0; l < r; l++) {
        double qa = orc_round_to_format((double)a[l], fmt);
        double qb = orc_round_to_format((double)b[l], fmt);
        double prod = orc_round_to_format(qa * qb, fmt);
        s = orc_round_to_format(s + prod, fmt);
    }
    return s;
}

/* Eq. (dist-direct) with every operation rounded to the format (Section
 * 4.2's fallback in precision u_h, here u_h = u of fmt): the inputs rounded
 * to it, then per coordinate t = fl(x~ - y~), s = fl(s + fl(t t)), in order.
 * fmt 4 (binary64) is orc_dist_direct_pair.                                 */
double orc_dist_direct_fmt(const float* x, const float* y, int r, int fmt) {
    if (fmt == 4) return orc_dist_direct_pair(x, y, r);
    double s = 0.0;
    for (int l = 0; l < r; l++) {
        double t = orc_round_to_format(orc_round_to_format((double)x[l], fmt) - orc_round_to_format((double)y[l], fmt), fmt);
        s = orc_round_to_format(s + orc_round_to_format(t * t, fmt), fmt);
    }
    return s;
}

/* Alg. 2 with the fallback of Eq. (fallback-rule) in the precision fb_fmt
 * (4 = binary64 as in Alg. 2, 3 = binary32, or fmt itself: the same-precision
 * fallback).  Otherwise as orc_mp_dist_paper.                               */
int orc_mp_dist_fb(const float* x, const float* y, int r, double rho, double c_A, int fmt, int fb_fmt,
                   double* d_out, double* dhat_out, double* E_out) {
    double d = 0.0;
    int f = orc_mp_dist_paper(x, y, r, rho, c_A, fmt, &d, dhat_out, E_out);
    if (f == 1) d = orc_dist_direct_fmt(x, y, r, fb_fmt);
    if (d_out) *d_out = d;
    return f;
}

int orc_mp_dist_paper(const float* x, const float* y, int r, double rho, double c_A, int fmt,
                      double* d_out, double* dhat_out, double* E_out) {
    double ul = orc_unit_roundoff(fmt);
    double g = orc_gamma(r + 2, ul);
    if (!isfinite(g)) return -1;
    double dxx = lo_dot(x, x, r, fmt);
    double dyy = lo_dot(y, y, r, fmt);
    double dxy = lo_dot(x, y, r, fmt);
    double t1 = orc_round_to_format(dxx - 2.0 * dxy, fmt);
    double dh = orc_round_to_format(t1 + dyy, fmt);
    if (dh < 0.0) dh = 0.0;
    double s = orc_round_to_format(dxx + dyy, fmt);
    double coef = orc_round_to_format(rho * c_A * g, fmt);
    double E = orc_round_to_format(coef * s, fmt);
    if (dhat_out) *dhat_out = dh;
    if (E_out) *E_out = E;
    if (dh <= E) {
        if (d_out) *d_out = orc_dist_direct_pair(x, y, r);
        return 1;
    }
    if (d_out) *d_out = dh;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reliability test instantiated for tensor-core arithmetic ("tc" test).
 *
 * The hardware multiplies the quantised operands exactly and accumulates in
 * fp32; the norms p = ||x||^2, q = ||c||^2 are formed in binary64 from the
 * fp32 originals and stored in fp32; the distance is d^ = p + (q - 2 g^).
 * Following Theorem 4.2 and Eq. (quantis-convert-error), with r_x = x~ - x,
 * r_c = c~ - c (exact residuals of the quantisation), the identity
 *   x~^T c~ - x^T c = r_x^T c + x~^T r_c
 * and Cauchy-Schwarz give the computable bound
 *   |d^ - d(x,c)^2| <= B = 2||r_x|| ||c|| + 2||x~|| ||r_c||
 *                          + k_acc ||x~|| ||c~|| + k_n (p + q),
 *   k_acc = 2 gamma_d(u_acc) + 4 u32,  k_n = 2 u32 + 2 u32,
 * with u_acc the accumulation unit (2^-21 assumed for 16-bit inputs,
 * 2^-13 for E4M3; the GPU tests measure the real accumulation error against
 * it).  The "tc" test flags a pair iff d^ <= rho * B; an unflagged pair then
 * has relative error <= 1/(rho-1), as in Eq. (expanded-rel-bound).
 * Row/column quantities are passed in so that this function is a plain
 * evaluation of the formula.                                               */
/* ------------------------------------------------------------------------ */
double orc_tc_bound(double nrx, double nc, double nxq, double nrc, double ncq,
                    double p, double q, int d, int fmt) {
    double u32 = ldexp(1.0, -24);
    double uacc = (fmt == 2) ? ldexp(1.0, -13) : ldexp(1.0, -21);
    double kacc = 2.0 * orc_gamma(d, uacc) + 4.0 * u32;
    double kn = 4.0 * u32;
    return 2.0 * nrx * nc + 2.0 * nxq * nrc + kacc * nxq * ncq + kn * (p + q);
}

/* Per-row (or per-centre) quantities for the tc bound: the fp32-rounded
 * squared norm of the original, and the norms of the original, of the
 * quantised vector and of the quantisation residual.  scale is the per-row
 * power-of-two scale for E4M3 (x~ = s * fl_l(x / s)); 1 for fp16/bf16.     */
void orc_row_quant_stats(const float* X, int64_t n, int d, int fmt, int per_row_scale,
                         float* Xq, double* sq_norm, double* nrm, double* nq, double* nres,
                         double* scale_out) {
    for (int64_t i = 0; i < n; i++) {
        const float* x = X + i * d;
        double s = 1.0;
        if (per_row_scale) {
            double amax = 0.0;
            for (int l = 0; l < d; l++) if (fabs((double)x[l]) > amax) amax = fabs((double)x[l]);
            /* s = 2^ceil(log2(amax / 448)): the row maximum lands in the top
             * binade; s is kept a normal binary32 number (s >= 2^-126), the
             * scale being applied in binary32; an all-zero row keeps s = 1 */
            if (amax > 0.0) {
                int e;
                frexp(amax / 448.0, &e);
                s = ldexp(1.0, e);
                if (amax / 448.0 == ldexp(1.0, e - 1)) s = ldexp(1.0, e - 1);
                if (s < ldexp(1.0, -126)) s = ldexp(1.0, -126);
            }
        }
        double a = 0.0, b = 0.0, c = 0.0;
        for (int l = 0; l < d; l++) {
            double xv = (double)x[l];
            double qv = s * orc_round_to_format(xv / s, fmt);
            if (Xq) Xq[i * d + l] = (float)qv;
            a += xv * xv;
            b += qv * qv;
            c += (qv - xv) * (qv - xv);
        }
        if (sq_norm) sq_norm[i] = (double)(float)a;
        if (nrm) nrm[i] = sqrt(a);
        if (nq) nq[i] = sqrt(b);
        if (nres) nres[i] = sqrt(c);
        if (scale_out) scale_out[i] = s;
    }
}

/* Expanded distance on the quantised data with the cross term taken exactly
 * (Eq. (dist-expanded) with p, q from the originals): the value the
 * hardware approximates, and from which the GPU flag decisions differ by at
 * most the accumulation and rounding terms of the tc bound.                */
double orc_expanded_quantised(const float* xq, const float* cq, int d, double p, double q) {
    /* x~_l c~_l is exact in binary64 for 16-bit and 8-bit formats; the sum
     * of d such products is exact unless exponents span > 30 binades.      */
    double g = 0.0;
    for (int l = 0; l < d; l++) g += (double)xq[l] * (double)cq[l];
    return p + q - 2.0 * g;
}

/* ------------------------------------------------------------------------ */
/* Seeding by D^2 sampling (k-means++; Section 2 names it as an alternative
 * to uniform initial centres, and leaves it outside the method).  The
 * random draws are inputs: u[0..k-1] in [0, 1).
 *   i_0 = min(floor(u_0 n), n - 1);
 *   D^2_i = d(x_i, x_{i_0})^2 (Eq. (dist-direct), binary64);
 *   for t = 1..k-1: T = sum_i D^2_i (ascending i); when T > 0, i_t is the
 *   smallest i whose prefix sum P_i = sum_{l <= i} D^2_l exceeds u_t T (the
 *   largest i with D^2_i > 0 when rounding leaves none); when T = 0 (every
 *   point on a chosen centre), i_t = min(floor(u_t n), n - 1); then
 *   D^2_i = min(D^2_i, d(x_i, x_{i_t})^2).
 * follow (nullable): after computing its own choice idx[t], continue from
 * follow[t] instead (a check of another implementation's sequence, step by
 * step).  margin (nullable): per step, min over i of |P_i - u_t T| / T, the
 * distance of the draw from the nearest boundary between two choices
 * (+inf at t = 0 and when T = 0).                                          */
/* ------------------------------------------------------------------------ */
int orc_kmeanspp(const float* X, int64_t n, int d, int k, const double* u, const int64_t* follow,
                 int64_t* idx, double* margin) {
    if (n < 1 || d < 1 || k < 1 || k > n) return ORC_EINVAL;
    double* D2 = (double*)malloc(sizeof(double) * (size_t)n);
    if (!D2) return ORC_EINVAL;
    int64_t cur = (int64_t)floor(u[0] * (double)n);
    if (cur > n - 1) cur = n - 1;
    idx[0] = cur;
    if (margin) margin[0] = INFINITY;
    if (follow) cur = follow[0];
    for (int64_t i = 0; i < n; i++) D2[i] = orc_dist_direct_pair(X + i * d, X + cur * d, d);
    for (int t = 1; t < k; t++) {
        double T = 0.0;
        for (int64_t i = 0; i < n; i++) T += D2[i];
        int64_t pick = -1;
        double mg = INFINITY;
        if (T > 0.0) {
            const double target = u[t] * T;
            double P = 0.0;
            int64_t last_pos = -1;
            for (int64_t i = 0; i < n; i++) {
                P += D2[i];
                if (D2[i] > 0.0) last_pos = i;
                const double gap = fabs(P - target) / T;
                if (gap < mg) mg = gap;
                if (pick < 0 && P > target) pick = i;
            }
            if (pick < 0) pick = last_pos;
        } else {
            pick = (int64_t)floor(u[t] * (double)n);
            if (pick > n - 1) pick = n - 1;
        }
        idx[t] = pick;
        if (margin) margin[t] = mg;
        cur = follow ? follow[t] : pick;
        for (int64_t i = 0; i < n; i++) {
            const double v = orc_dist_direct_pair(X + i * d, X + cur * d, d);
            if (v < D2[i]) D2[i] = v;
        }
    }
    free(D2);
    return ORC_OK;
}
