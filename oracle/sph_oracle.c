/*
 * Plain CPU oracle for the SPH neighbour-sum hot path of Bonsai-SPH
 * (arXiv 1909.07439).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product library
 * (the CUDA path) never links, includes or calls anything in this directory,
 * and this file shares no code, header or constant table with it.
 *
 * Every function is the plain definition written out: brute force over all
 * particle pairs (O(N^2)), double precision.  Two parts are not double
 * precision because their contract is an exact single-precision replay:
 *   - the Morton key quantisation (Sect. 3.1), and
 *   - the neighbour-set membership test (Sect. 3.2),
 * both written as separate FP32 operations in a fixed order.  The library is
 * compiled with -ffp-contract=off so those operations are never fused.
 *
 * Targets are processed independently (OpenMP over targets); each target's
 * sum runs over j = 0..n-1 in ascending order.
 *
 * Periodic boundaries (the Sod and blast tube tests of Sect. 4.1-4.2 are
 * periodic in y and z): `box` gives the period L of each axis, 0 for an open
 * axis (box = NULL: all open).  A pair's separation along a periodic axis is
 * the nearest image: d = x_i - x_j, then d - L if d > L/2, d + L if d < -L/2
 * (positions lie in one period, so |d| < L and one correction suffices; the
 * support radius must stay below L/2 so that a pair meets one image only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Smoothing kernels, 3D (Sect. 2.3 and Eq. 14): W(r, h) = C f(q) / h^3 with */
/* q = r/h, zero for q >= R (the support radius in units of h), C such that  */
/* 4 pi int_0^R C f(q) q^2 dq = 1.  The paper names the kernels and leaves   */
/* their formulas to the literature; these are the standard forms:          */
/*   0  M4 cubic spline, R = 2, C = 1/pi:                                    */
/*        f = 1 - 3/2 q^2 + 3/4 q^3 (q < 1), 1/4 (2 - q)^3 (1 <= q < 2)       */
/*   1  M6 quintic spline, R = 3, C = 1/(120 pi):                            */
/*        f = (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 (q < 1),                       */
/*            (3-q)^5 - 6 (2-q)^5 (1 <= q < 2), (3-q)^5 (2 <= q < 3)          */
/*   2  Wendland C6, R = 2, C = 1365/(512 pi):                               */
/*        f = (1 - q/2)^8 (4 q^3 + 25/4 q^2 + 4 q + 1) (q < 2)                */
/* ------------------------------------------------------------------------- */
static const double PI_D = 3.14159265358979323846264338327950288;

static double kern_support(int kernel) { return kernel == 1 ? 3.0 : 2.0; }

static double kern_norm(int kernel)
{
    if (kernel == 1) return 1.0 / (120.0 * PI_D);
    if (kernel == 2) return 1365.0 / (512.0 * PI_D);
    return 1.0 / PI_D;
}

static double shape_f(int kernel, double q)
{
    if (kernel == 1) {
        double a = 3.0 - q, b = 2.0 - q, c = 1.0 - q;
        if (q < 1.0) return a * a * a * a * a - 6.0 * b * b * b * b * b + 15.0 * c * c * c * c * c;
        if (q < 2.0) return a * a * a * a * a - 6.0 * b * b * b * b * b;
        if (q < 3.0) return a * a * a * a * a;
        return 0.0;
    }
    if (kernel == 2) {
        if (q >= 2.0) return 0.0;
        double s = 1.0 - 0.5 * q, s2 = s * s, s4 = s2 * s2, s8 = s4 * s4;
        return s8 * (4.0 * q * q * q + 6.25 * q * q + 4.0 * q + 1.0);
    }
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}

static double shape_df(int kernel, double q) /* df/dq */
{
    if (kernel == 1) {
        double a = 3.0 - q, b = 2.0 - q, c = 1.0 - q;
        if (q < 1.0) return -5.0 * a * a * a * a + 30.0 * b * b * b * b - 75.0 * c * c * c * c;
        if (q < 2.0) return -5.0 * a * a * a * a + 30.0 * b * b * b * b;
        if (q < 3.0) return -5.0 * a * a * a * a;
        return 0.0;
    }
    if (kernel == 2) {
        /* product rule on s^8 P(q), s = 1 - q/2, P = 4 q^3 + 25/4 q^2 + 4 q + 1 */
        if (q >= 2.0) return 0.0;
        double s = 1.0 - 0.5 * q, s2 = s * s, s4 = s2 * s2, s7 = s4 * s2 * s, s8 = s7 * s;
        double P = 4.0 * q * q * q + 6.25 * q * q + 4.0 * q + 1.0;
        double dP = 12.0 * q * q + 12.5 * q + 4.0;
        return 8.0 * s7 * (-0.5) * P + s8 * dP;
    }
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
    return 0.0;
}

/* nearest-image separation along one axis (L = 0: open axis) */
static double wrap_d(double d, double L)
{
    if (L > 0.0) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

/* the same in FP32: with L/2 <= |d| < L the correction is exact (Sterbenz) */
static float wrap_f(float d, float L)
{
    if (L > 0.0f) {
        if (d > 0.5f * L) d = d - L;
        else if (d < -0.5f * L) d = d + L;
    }
    return d;
}

/* separation x_i - x_j (3 components) with nearest images */
static void sep3(const double *x, int64_t i, int64_t j, const double *box, double *d)
{
    for (int a = 0; a < 3; ++a) {
        d[a] = x[3 * i + a] - x[3 * j + a];
        if (box) d[a] = wrap_d(d[a], box[a]);
    }
}

/* W(r, h) */
static double kern_w(int k, double r, double h) { return kern_norm(k) * shape_f(k, r / h) / (h * h * h); }
/* F(r, h) = C f'(q) / h^4 = dW/dr (Eq. 14); grad_i W_ij(h) = rhat_ij F(r_ij, h) */
static double kern_F(int k, double r, double h)
{
    return kern_norm(k) * shape_df(k, r / h) / (h * h * h * h);
}
/* dW/dh at fixed r: -C (3 f(q) + q f'(q)) / h^4 */
static double kern_dwdh(int k, double r, double h)
{
    double q = r / h;
    return -kern_norm(k) * (3.0 * shape_f(k, q) + q * shape_df(k, q)) / (h * h * h * h);
}

ORC_API void orc_kernel_eval(const double *r, const double *h, int64_t n,
                             double *w, double *F, double *dwdh, int kernel)
{
    for (int64_t i = 0; i < n; ++i) {
        if (w) w[i] = kern_w(kernel, r[i], h[i]);
        if (F) F[i] = kern_F(kernel, r[i], h[i]);
        if (dwdh) dwdh[i] = kern_dwdh(kernel, r[i], h[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Space-filling-curve keys (Sect. 3.1): 21 bits per axis, 63-bit Morton key. */
/* Canonical FP32 quantisation:                                              */
/*   lo_a = min_i x_a,i ; size = max_a (hi_a - lo_a)                         */
/*   s = 2097152 / size (0 if size == 0)                                     */
/*   c_a = min(floor((x_a - lo_a) * s), 2^21 - 1)                            */
/*   key bit 3k+2 = bit k of c_x, 3k+1 = c_y, 3k = c_z                       */
/* ------------------------------------------------------------------------- */
ORC_API void orc_bbox(const float *pos4, int64_t n, float *out4)
{
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    if (n > 0)
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = pos4[a];
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float x = pos4[4 * i + a];
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    float size = 0.f;
    for (int a = 0; a < 3; ++a) {
        float e = hi[a] - lo[a];
        if (e > size) size = e;
    }
    out4[0] = lo[0]; out4[1] = lo[1]; out4[2] = lo[2]; out4[3] = size;
}

ORC_API void orc_morton_keys(const float *pos4, int64_t n, uint64_t *keys)
{
    float box[4];
    orc_bbox(pos4, n, box);
    float s = 0.f;
    if (box[3] > 0.f) s = 2097152.0f / box[3];
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[3];
        for (int a = 0; a < 3; ++a) {
            float d = pos4[4 * i + a] - box[a];
            float t = d * s;
            float f = floorf(t);
            uint32_t v = (uint32_t)f;
            if (v > 2097151u) v = 2097151u;
            c[a] = v;
        }
        uint64_t key = 0;
        for (int k = 0; k < 21; ++k) {
            key |= (uint64_t)((c[0] >> k) & 1u) << (3 * k + 2);
            key |= (uint64_t)((c[1] >> k) & 1u) << (3 * k + 1);
            key |= (uint64_t)((c[2] >> k) & 1u) << (3 * k);
        }
        keys[i] = key;
    }
}

typedef struct { uint64_t key; int64_t idx; } key_idx;

static int cmp_key_idx(const void *a, const void *b)
{
    const key_idx *x = (const key_idx *)a, *y = (const key_idx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* order[k] = original index of the k-th particle in ascending (key, index). */
ORC_API int orc_sort_order(const uint64_t *keys, int64_t n, int64_t *order)
{
    key_idx *t = (key_idx *)malloc(sizeof(key_idx) * (size_t)(n > 0 ? n : 1));
    if (!t) return -1;
    for (int64_t i = 0; i < n; ++i) { t[i].key = keys[i]; t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(key_idx), cmp_key_idx);
    for (int64_t i = 0; i < n; ++i) order[i] = t[i].idx;
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Octree / group chop (Sect. 3.1).  The sorted key array is cut level by    */
/* level: a node at level L is a maximal run of particles that share the top */
/* 3L key bits; a node with more than `thresh` particles (and L < 21) is     */
/* split into the maximal runs sharing the top 3(L+1) bits.  Nodes are       */
/* numbered level by level, and inside a level by first particle.            */
/* Returns the node count, or -1 if it exceeds cap.                          */
/* ------------------------------------------------------------------------- */
ORC_API int64_t orc_chop(const uint64_t *skeys, int64_t n, int32_t thresh,
                         int32_t *level, int64_t *first, int64_t *count,
                         int64_t *child_first, int32_t *nchild, int64_t cap)
{
    if (n <= 0) return 0;
    if (cap < 1) return -1;
    int64_t nn = 1;
    level[0] = 0; first[0] = 0; count[0] = n; child_first[0] = -1; nchild[0] = 0;
    int64_t cur_begin = 0, cur_end = 1;
    for (int L = 0; L < 21 && cur_begin < cur_end; ++L) {
        int shift = 63 - 3 * (L + 1);
        for (int64_t i = cur_begin; i < cur_end; ++i) {
            child_first[i] = -1;
            nchild[i] = 0;
            if (count[i] <= thresh) continue;
            child_first[i] = nn;
            int64_t p = first[i], end = first[i] + count[i];
            while (p < end) {
                int64_t q = p + 1;
                while (q < end && (skeys[q] >> shift) == (skeys[p] >> shift)) ++q;
                if (nn >= cap) return -1;
                level[nn] = L + 1; first[nn] = p; count[nn] = q - p;
                child_first[nn] = -1; nchild[nn] = 0;
                ++nn;
                ++nchild[i];
                p = q;
            }
        }
        cur_begin = cur_end;
        cur_end = nn;
    }
    return nn;
}

/* ------------------------------------------------------------------------- */
/* Neighbour sets (Sect. 3.2), canonical FP32 membership test:               */
/*   dx = x_i - x_j (per axis, then the nearest image on a periodic axis),    */
/*   r2 = (dx*dx + dy*dy) + dz*dz                                            */
/*   density set  D_i = { j : r2 < (R h_i)*(R h_i) }        (includes i)     */
/*   force set    F_i = { j != i : r2 < (R m)*(R m) }, m = max(h_i, h_j)     */
/* with R the kernel's support radius in units of h (2, or 3 for M6) and     */
/* R h one FP32 multiplication.                                              */
/* The force set uses the larger smoothing length of the pair so that a pair */
/* interacts if either particle lies inside the other's range.               */
/* ------------------------------------------------------------------------- */
static float canon_r2(const float *pi, const float *pj, const float *box)
{
    float dx = pi[0] - pj[0];
    float dy = pi[1] - pj[1];
    float dz = pi[2] - pj[2];
    if (box) {
        dx = wrap_f(dx, box[0]);
        dy = wrap_f(dy, box[1]);
        dz = wrap_f(dz, box[2]);
    }
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    s = s + zz;
    return s;
}

static int canon_in_set(int mode, int kernel, int64_t i, int64_t j, const float *pos4, const float *h,
                        const float *box)
{
    const float kr = kernel == 1 ? 3.0f : 2.0f; /* support radius in units of h */
    float r2 = canon_r2(pos4 + 4 * i, pos4 + 4 * j, box);
    if (mode == 0) {
        float R = kr * h[i];
        float R2 = R * R;
        return r2 < R2;
    }
    if (i == j) return 0;
    float m = h[i] > h[j] ? h[i] : h[j];
    float R = kr * m;
    float R2 = R * R;
    return r2 < R2;
}

/* Row counts for the given targets (cnt[t]). */
ORC_API void orc_neighbour_counts(const float *pos4, const float *h, int64_t n, int mode,
                                  const int64_t *targets, int64_t nt, int64_t *cnt, int kernel,
                                  const float *box)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t], c = 0;
        for (int64_t j = 0; j < n; ++j) c += canon_in_set(mode, kernel, i, j, pos4, h, box);
        cnt[t] = c;
    }
}

/* Rows written at off[t] (caller computed from the counts), ascending j. */
ORC_API void orc_neighbour_lists(const float *pos4, const float *h, int64_t n, int mode,
                                 const int64_t *targets, int64_t nt, const int64_t *off,
                                 int64_t *idx, int kernel, const float *box)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t], c = off[t];
        for (int64_t j = 0; j < n; ++j)
            if (canon_in_set(mode, kernel, i, j, pos4, h, box)) idx[c++] = j;
    }
}

/* ------------------------------------------------------------------------- */
/* Density and smoothing length (Eqs. 1-4).                                  */
/*   rho_sum(h) = sum_j m_j W(r_ij, h)            (j = i included, Eq. 1)     */
/*   rho_h(h)   = m_i (hfact / h)^3               (Eq. 2 solved for rho)      */
/* The smoothing length is the root of g(h) = rho_sum(h) - rho_h(h).         */
/*   g'(h) = sum_j m_j dW/dh + 3 rho_h / h                                   */
/*   Omega = 1 - (dh/drho) sum_j m_j dW/dh with dh/drho = -h / (3 rho)  (Eq. 4)*/
/*   drho/dt = (1/Omega) sum_j m_j (v_i - v_j) . rhat_ij F(r_ij, h)   (Eq. 3)  */
/* Newton steps on g, safeguarded by a bracket [lo, hi] on the root: a step  */
/* that leaves the bracket or [h/2, 2h], or a non-positive g', is replaced   */
/* by bisection (bracket known) or by doubling / halving h.                  */
/* fixed_iters > 0 runs exactly that many updates and skips the tolerance.   */
/* Returns the number of targets that did not converge.                      */
/* ------------------------------------------------------------------------- */
static void density_sums(int k, int64_t i, double h, const double *x, const double *m, int64_t n,
                         const double *box, double *rho_sum, double *dwdh_sum)
{
    double s0 = 0.0, s1 = 0.0;
    const double R = kern_support(k);
    for (int64_t j = 0; j < n; ++j) {
        double d[3];
        sep3(x, i, j, box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r >= R * h) continue;
        s0 += m[j] * kern_w(k, r, h);
        s1 += m[j] * kern_dwdh(k, r, h);
    }
    *rho_sum = s0;
    *dwdh_sum = s1;
}

ORC_API int64_t orc_density(const double *x, const double *v, const double *m, int64_t n,
                            const int64_t *targets, int64_t nt, const double *h0,
                            double hfact, double tol, int32_t max_iter, int32_t fixed_iters,
                            double *h_out, double *rho, double *omega, double *drhodt,
                            int32_t *nngb, int32_t *iters, int kernel, const double *box)
{
    const double R = kern_support(kernel);
    int64_t failures = 0;
    double hf3 = hfact * hfact * hfact;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : failures)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double h = h0[i], lo = 0.0, hi = INFINITY;
        int it = 0, converged = 0;
        int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        while (it < limit) {
            double rs, ds;
            density_sums(kernel, i, h, x, m, n, box, &rs, &ds);
            double rho_h = m[i] * hf3 / (h * h * h);
            double g = rs - rho_h;
            double gp = ds + 3.0 * rho_h / h;
            if (g == 0.0) { ++it; converged = 1; break; } /* exact root */
            if (g < 0.0) lo = h; else hi = h;
            double hn = h - g / gp;
            int ok = gp > 0.0 && hn >= lo && hn <= hi && hn >= 0.5 * h && hn <= 2.0 * h;
            if (!ok) {
                if (lo > 0.0 && hi < INFINITY) hn = 0.5 * (lo + hi);
                else if (g < 0.0) hn = 2.0 * h;
                else hn = 0.5 * h;
            }
            ++it;
            double rel = fabs(hn - h) / h;
            h = hn;
            if (fixed_iters <= 0 && rel < tol) { converged = 1; break; }
        }
        if (fixed_iters > 0) converged = 1;
        if (!converged) failures += 1;
        /* final quantities at the accepted h */
        double rs, ds;
        density_sums(kernel, i, h, x, m, n, box, &rs, &ds);
        double rho_h = m[i] * hf3 / (h * h * h);
        double om = 1.0 + h / (3.0 * rho_h) * ds;
        double div = 0.0;
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            double d[3];
            sep3(x, i, j, box, d);
            double dx = d[0], dy = d[1], dz = d[2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r >= R * h) continue;
            ++cnt;
            if (r <= 0.0) continue;
            double vr = ((v[3 * i] - v[3 * j]) * dx + (v[3 * i + 1] - v[3 * j + 1]) * dy +
                         (v[3 * i + 2] - v[3 * j + 2]) * dz) / r;
            div += m[j] * vr * kern_F(kernel, r, h);
        }
        h_out[t] = h;
        rho[t] = rho_h;
        omega[t] = om;
        drhodt[t] = div / om;
        nngb[t] = cnt;
        iters[t] = it;
    }
    return failures;
}

/* ------------------------------------------------------------------------- */
/* Hydro force (Eqs. 9-15), no gravity.  Adiabatic equation of state         */
/* P = (gamma-1) rho u, c = sqrt(gamma P / rho) (the paper uses P and c_s    */
/* without stating the EOS).                                                  */
/*   a_i = - sum_j m_j [ (P_i + q^i)/(rho_i^2 Om_i) F(r,h_i)                 */
/*                     + (P_j + q^j)/(rho_j^2 Om_j) F(r,h_j) ] rhat_ij   (9)  */
/*   q^i = -1/2 rho_i (alpha c_i + beta |vr|) vr  if vr < 0 else 0   (11,12)  */
/*   q^j = -1/2 rho_j (alpha c_j + beta |vr|) vr  if vr < 0 else 0            */
/*   du_i/dt = P_i/(rho_i^2 Om_i) sum_j m_j vr F(r,h_i)                 (10)  */
/*           - 1/(Om_i rho_i) sum_{vr<0} m_j 1/2 (alpha c_i + beta|vr|) vr^2 F(r,h_i) */
/*           + sum_j m_j alpha_u vsig_u (u_i - u_j)                           */
/*               * 1/2 [F(r,h_i)/(Om_i rho_i) + F(r,h_j)/(Om_j rho_j)]  (13)  */
/*   vsig_u = sqrt(|P_i - P_j| / (1/2 (rho_i + rho_j)))                 (15)  */
/*   vsigmax_i = max(alpha c_i, max_{j in F_i} alpha c_i + beta |vr|)   (8)   */
/* vr = (v_i - v_j) . rhat_ij.  F(r, h) vanishes for r >= R h, so the sums   */
/* run over every j != i.  The set for vsigmax is r < R max(h_i,h_j) * vsig_scale */
/* (vsig_scale = 1 is the definition; other values give the bracketing sets  */
/* the parity tests use).                                                     */
/* ------------------------------------------------------------------------- */
ORC_API void orc_force(const double *x, const double *v, const double *m, const double *u,
                       const double *h, const double *rho, const double *omega, int64_t n,
                       const int64_t *targets, int64_t nt, double gamma, double alpha,
                       double beta, double alpha_u, double vsig_scale, double *acc,
                       double *dudt, double *vsigmax, int32_t *nforce, int kernel,
                       const double *box)
{
    const double R = kern_support(kernel);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double Pi = (gamma - 1.0) * rho[i] * u[i];
        double ci = sqrt(gamma * Pi / rho[i]);
        double ax = 0.0, ay = 0.0, az = 0.0;
        double du_p = 0.0, du_av = 0.0, du_cond = 0.0;
        double vs = alpha * ci;
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            sep3(x, i, j, box, d);
            double dx = d[0], dy = d[1], dz = d[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double hm = h[i] > h[j] ? h[i] : h[j];
            double rad = R * hm * vsig_scale;
            double r = sqrt(r2);
            double vr = 0.0;
            if (r > 0.0)
                vr = ((v[3 * i] - v[3 * j]) * dx + (v[3 * i + 1] - v[3 * j + 1]) * dy +
                      (v[3 * i + 2] - v[3 * j + 2]) * dz) / r;
            if (r < rad) {
                double s = alpha * ci + beta * fabs(vr);
                if (s > vs) vs = s;
            }
            if (r >= R * hm) continue;
            ++cnt;
            if (r <= 0.0) continue;
            double Fi = kern_F(kernel, r, h[i]);
            double Fj = kern_F(kernel, r, h[j]);
            double Pj = (gamma - 1.0) * rho[j] * u[j];
            double cj = sqrt(gamma * Pj / rho[j]);
            double qi = 0.0, qj = 0.0;
            if (vr < 0.0) {
                qi = -0.5 * rho[i] * (alpha * ci + beta * fabs(vr)) * vr;
                qj = -0.5 * rho[j] * (alpha * cj + beta * fabs(vr)) * vr;
            }
            double coef = m[j] * ((Pi + qi) / (rho[i] * rho[i] * omega[i]) * Fi +
                                  (Pj + qj) / (rho[j] * rho[j] * omega[j]) * Fj);
            ax -= coef * dx / r;
            ay -= coef * dy / r;
            az -= coef * dz / r;
            du_p += m[j] * vr * Fi;
            if (vr < 0.0) du_av += m[j] * 0.5 * (alpha * ci + beta * fabs(vr)) * vr * vr * Fi;
            double vsu = sqrt(fabs(Pi - Pj) / (0.5 * (rho[i] + rho[j])));
            du_cond += m[j] * alpha_u * vsu * (u[i] - u[j]) * 0.5 *
                       (Fi / (omega[i] * rho[i]) + Fj / (omega[j] * rho[j]));
        }
        acc[3 * t] = ax;
        acc[3 * t + 1] = ay;
        acc[3 * t + 2] = az;
        dudt[t] = Pi / (rho[i] * rho[i] * omega[i]) * du_p - du_av / (omega[i] * rho[i]) + du_cond;
        vsigmax[t] = vs;
        nforce[t] = cnt;
    }
}

/* ------------------------------------------------------------------------- */
/* Conserved quantities (Sect. 4.5): E_kin, E_th, momentum, angular momentum */
/* out8 = { sum m v^2/2, sum m u, px, py, pz, Lx, Ly, Lz }                    */
/* ------------------------------------------------------------------------- */
ORC_API void orc_conserved(const double *x, const double *v, const double *m, const double *u,
                           int64_t n, double *out8)
{
    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        const double *r = x + 3 * i, *w = v + 3 * i;
        e[0] += 0.5 * m[i] * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        e[1] += m[i] * u[i];
        e[2] += m[i] * w[0];
        e[3] += m[i] * w[1];
        e[4] += m[i] * w[2];
        e[5] += m[i] * (r[1] * w[2] - r[2] * w[1]);
        e[6] += m[i] * (r[2] * w[0] - r[0] * w[2]);
        e[7] += m[i] * (r[0] * w[1] - r[1] * w[0]);
    }
    memcpy(out8, e, sizeof(e));
}

/* ------------------------------------------------------------------------- */
/* Self-gravity (the a_grav term of Eq. 9), the plain definition: a direct   */
/* sum over every other particle with Plummer softening eps,                 */
/*   a_i   = -G sum_{j != i} m_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^(3/2) */
/*   phi_i = -G sum_{j != i} m_j / (|x_i - x_j|^2 + eps^2)^(1/2)            */
/* (the tree code of the paper approximates this sum with the Barnes-Hut    */
/* walk; the potential energy is 1/2 sum_i m_i phi_i).                       */
/* out4[4 t .. 4 t + 3] = (a_x, a_y, a_z, phi) of target t.                  */
/* ------------------------------------------------------------------------- */
ORC_API void orc_gravity(const double *x, const double *m, int64_t n, const int64_t *targets,
                         int64_t nt, double G, double eps, double *out4)
{
    const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double ax = 0.0, ay = 0.0, az = 0.0, phi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1],
                   dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz + e2;
            double rinv = 1.0 / sqrt(r2);
            double mr3 = m[j] * rinv * rinv * rinv;
            ax -= mr3 * dx;
            ay -= mr3 * dy;
            az -= mr3 * dz;
            phi -= m[j] * rinv;
        }
        out4[4 * t] = G * ax;
        out4[4 * t + 1] = G * ay;
        out4[4 * t + 2] = G * az;
        out4[4 * t + 3] = G * phi;
    }
}
