/*
 * oracle.c -- plain, slow, FP64 CPU oracle for one 2D vortex-blob FMM
 * velocity evaluation (Cruz, Knepley & Barba, "PetFMM -- a dynamically
 * load-balancing parallel fast multipole library").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   O1  direct sum      u(x_i) = sum_{j != i} gamma_j K_sigma(x_i - x_j)
 *                       (Sec. 3, Eq. 8 and Eq. 9; targets = sources, Eq. 1)
 *   O2  substituted sum the same loop, but pairs whose leaves are more than
 *                       one leaf apart use the singular kernel of Eq. 7
 *                       (kernel substitution, end of Sec. 3)
 *   O3  textbook FMM    binning into a uniform quadtree (Sec. 2.1, z-order
 *                       numbering Sec. 5.1), P2M, M2M, M2L over the
 *                       interaction list, L2L, L2P and the near-field P2P
 *                       (Sec. 2.2, Fig. 2; costs in Sec. 5.2).  The paper
 *                       leaves the series out (Sec. 2.2) and points to
 *                       Greengard-Rokhlin; the Cauchy-kernel Laurent/Taylor
 *                       series used here are written out from that
 *                       mathematics, unscaled, with p terms k = 0..p-1.
 *
 * Readings where the paper is silent or garbled:
 *   - p terms per expansion (k = 0..p-1): Sec. 2 "truncated after p terms"
 *     and Table 1 (16p bytes per box), not the p+1 of Eq. 3.
 *   - Far field: w(z) = sum_j gamma_j / (z - z_j) with z = x + i y; the
 *     velocity is u = Im(w) / 2pi, v = Re(w) / 2pi (the singular Biot-Savart
 *     kernel of Eq. 7 written in complex form).
 *   - Near domain = the leaf and its (up to 8) same-level neighbours; the
 *     interaction list (at most 27, Table 1) = the children of the parent's
 *     neighbours that are not neighbours of the box.  Levels 0 and 1 have an
 *     empty interaction list.
 *   - Self and coincident pairs contribute 0 (the limit of Eq. 8 at x = 0).
 *   - Binning of a point: t = x - x0; s = t * (2^L / W); ix = floor(s),
 *     clamped to [0, 2^L - 1]; the domain is the closed square
 *     [x0, x0 + W] x [y0, y0 + W]; a point outside it is an error.
 *     Morton key: bit b of ix goes to bit 2b, bit b of iy to bit 2b + 1.
 *     Ties in the sort are broken by input index (stable sort).
 *
 * Compiled with -O2 -ffp-contract=off so that no multiply-add is fused.
 * OpenMP (if enabled) splits only independent outputs (targets, boxes); each
 * output is computed by one thread in a fixed order, so results do not
 * depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EDOMAIN (-3)

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846264338327950288;

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Kernels: Eq. 8 (regularised) and Eq. 7 (singular), as velocity    */
/* contributions of a unit-strength source at offset (dx, dy) =        */
/* target minus source.                                                */
/* ------------------------------------------------------------------ */

/* K_sigma(x) = (-x2, x1) (1 - exp(-|x|^2 / 2 sigma^2)) / (2 pi |x|^2).
 * 1 - exp(-q) is evaluated as -expm1(-q) to keep full precision at small q. */
static void k_sigma(double dx, double dy, double sigma, double *ku, double *kv) {
    double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) { *ku = 0.0; *kv = 0.0; return; }
    double f = -expm1(-r2 / (2.0 * sigma * sigma)) / (2.0 * ORC_PI * r2);
    *ku = -dy * f;
    *kv = dx * f;
}

/* Singular Biot-Savart kernel of a point vortex, (-x2, x1) / (2 pi |x|^2). */
static void k_singular(double dx, double dy, double *ku, double *kv) {
    double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) { *ku = 0.0; *kv = 0.0; return; }
    double f = 1.0 / (2.0 * ORC_PI * r2);
    *ku = -dy * f;
    *kv = dx * f;
}

/* Exposed so that tests can pin the kernel itself. */
void orc_kernel_sigma(double dx, double dy, double sigma, double *ku, double *kv) {
    k_sigma(dx, dy, sigma, ku, kv);
}

/* ------------------------------------------------------------------ */
/* O1: direct sum (Eq. 9 with Eq. 8), targets = sources, j != i.       */
/* targets == NULL means every particle is a target.                   */
/* ------------------------------------------------------------------ */
void orc_direct(int64_t n, const double *x, const double *y, const double *g,
                double sigma, int64_t nt, const int64_t *targets,
                double *u, double *v, int nthreads) {
    set_threads(nthreads);
    if (targets == NULL) nt = n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double ku, kv;
            k_sigma(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            su += g[j] * ku;
            sv += g[j] * kv;
        }
        u[t] = su;
        v[t] = sv;
    }
}

/* ------------------------------------------------------------------ */
/* Binning and z-order (Sec. 2.1, Sec. 5.1).                           */
/* ------------------------------------------------------------------ */
static uint32_t interleave(uint32_t ix, uint32_t iy, int L) {
    uint32_t key = 0;
    for (int b = 0; b < L; ++b) {
        key |= ((ix >> b) & 1u) << (2 * b);
        key |= ((iy >> b) & 1u) << (2 * b + 1);
    }
    return key;
}

static void deinterleave(uint32_t key, int L, uint32_t *ix, uint32_t *iy) {
    uint32_t a = 0, b2 = 0;
    for (int b = 0; b < L; ++b) {
        a |= ((key >> (2 * b)) & 1u) << b;
        b2 |= ((key >> (2 * b + 1)) & 1u) << b;
    }
    *ix = a;
    *iy = b2;
}

uint32_t orc_morton(uint32_t ix, uint32_t iy, int L) { return interleave(ix, iy, L); }

static uint32_t bin1(double xv, double x0, double scale, uint32_t nb) {
    double t = xv - x0;
    double s = t * scale;
    double f = floor(s);
    if (f < 0.0) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (uint32_t)f;
}

/* Leaf coordinates and Morton key of every particle.  Returns ORC_EDOMAIN if
 * a particle lies outside the closed domain square (or is NaN). */
int orc_bin(int64_t n, const double *x, const double *y, double x0, double y0,
            double W, int L, uint32_t *ix, uint32_t *iy, uint32_t *key) {
    if (L < 0 || L > 15 || !(W > 0.0)) return ORC_EINVAL;
    double scale = ldexp(1.0, L) / W;
    double x1 = x0 + W, y1 = y0 + W;
    uint32_t nb = 1u << L;
    for (int64_t i = 0; i < n; ++i) {
        if (!(x[i] >= x0 && x[i] <= x1 && y[i] >= y0 && y[i] <= y1)) return ORC_EDOMAIN;
        uint32_t bx = bin1(x[i], x0, scale, nb);
        uint32_t by = bin1(y[i], y0, scale, nb);
        if (ix) ix[i] = bx;
        if (iy) iy[i] = by;
        key[i] = interleave(bx, by, L);
    }
    return ORC_OK;
}

/* Stable counting sort of the keys: perm[r] = input index of rank r;
 * start[b] = first rank with key >= b, for b = 0..4^L (start[4^L] = n). */
int orc_sort(int64_t n, const uint32_t *key, int L, uint32_t *perm, uint32_t *start) {
    uint64_t nbox = 1ull << (2 * L);
    uint64_t *cursor = (uint64_t *)calloc(nbox + 1, sizeof(uint64_t));
    if (!cursor) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) cursor[key[i] + 1] += 1;
    for (uint64_t b = 0; b < nbox; ++b) cursor[b + 1] += cursor[b];
    for (uint64_t b = 0; b <= nbox; ++b) start[b] = (uint32_t)cursor[b];
    for (int64_t i = 0; i < n; ++i) perm[cursor[key[i]]++] = (uint32_t)i;
    free(cursor);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Interaction list (Sec. 2.2; at most 27 members, Table 1): the       */
/* in-domain children of the parent's neighbours that are not          */
/* neighbours of the box itself.  Output: (sx, sy) pairs in ascending  */
/* Morton order of the source.  Returns the count.                     */
/* ------------------------------------------------------------------ */
int orc_interaction_list(int l, int ix, int iy, int32_t *out) {
    if (l < 2) return 0;
    int nside = 1 << l, nparent = 1 << (l - 1);
    int px = ix >> 1, py = iy >> 1;
    int cnt = 0;
    uint32_t keys[36];
    int32_t xs[36], ys[36];
    for (int qy = py - 1; qy <= py + 1; ++qy) {
        for (int qx = px - 1; qx <= px + 1; ++qx) {
            if (qx < 0 || qy < 0 || qx >= nparent || qy >= nparent) continue;
            for (int c = 0; c < 4; ++c) {
                int sx = 2 * qx + (c & 1), sy = 2 * qy + (c >> 1);
                if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
                if (abs(sx - ix) <= 1 && abs(sy - iy) <= 1) continue;
                keys[cnt] = interleave((uint32_t)sx, (uint32_t)sy, l);
                xs[cnt] = sx;
                ys[cnt] = sy;
                ++cnt;
            }
        }
    }
    /* insertion sort by Morton key */
    for (int a = 1; a < cnt; ++a) {
        uint32_t k = keys[a];
        int32_t bx = xs[a], by = ys[a];
        int b = a - 1;
        while (b >= 0 && keys[b] > k) {
            keys[b + 1] = keys[b]; xs[b + 1] = xs[b]; ys[b + 1] = ys[b];
            --b;
        }
        keys[b + 1] = k; xs[b + 1] = bx; ys[b + 1] = by;
    }
    for (int a = 0; a < cnt; ++a) { out[2 * a] = xs[a]; out[2 * a + 1] = ys[a]; }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Expansion operators, unscaled, p terms (k = 0..p-1).                */
/*   ME about zc:  w(z) = sum_k a_k / (z - zc)^(k+1)                   */
/*   LE about zl:  w(z) = sum_m b_m (z - zl)^m                         */
/* ------------------------------------------------------------------ */
static double binom(int n, int k) {
    /* exact for the sizes used here (n <= 2 * 40); product form in FP64 */
    if (k < 0 || k > n) return 0.0;
    if (k > n - k) k = n - k;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return floor(r + 0.5);
}

/* P2M: a_k = sum_j gamma_j (z_j - zc)^k. */
static void p2m(int64_t n, const double *x, const double *y, const double *g,
                const uint32_t *idx, cplx zc, int p, cplx *a) {
    for (int k = 0; k < p; ++k) a[k] = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t j = idx ? idx[t] : t;
        cplx d = (x[j] + I * y[j]) - zc;
        cplx pw = g[j];
        for (int k = 0; k < p; ++k) {
            a[k] += pw;
            pw *= d;
        }
    }
}

/* M2M: ME about zc -> ME about zp: a'_l = sum_{k<=l} C(l,k) a_k (zc - zp)^(l-k). */
static void m2m(int p, const cplx *a, cplx zc, cplx zp, cplx *out) {
    cplx d = zc - zp;
    cplx dpow[81];
    dpow[0] = 1.0;
    for (int i = 1; i < p; ++i) dpow[i] = dpow[i - 1] * d;
    for (int l = 0; l < p; ++l) {
        cplx s = 0.0;
        for (int k = 0; k <= l; ++k) s += binom(l, k) * a[k] * dpow[l - k];
        out[l] = s;
    }
}

/* M2L: ME about zs -> LE about zt, d = zs - zt:
 * b_m = sum_k (-1)^(k+1) C(k+m, k) a_k d^-(k+m+1). */
static void m2l(int p, const cplx *a, cplx zs, cplx zt, cplx *b) {
    cplx d = zs - zt;
    cplx inv = 1.0 / d;
    cplx ipow[81];
    ipow[0] = 1.0;
    for (int i = 1; i <= 2 * p; ++i) ipow[i] = ipow[i - 1] * inv;
    for (int m = 0; m < p; ++m) {
        cplx s = 0.0;
        for (int k = 0; k < p; ++k) {
            double sign = (k % 2 == 0) ? -1.0 : 1.0;
            s += sign * binom(k + m, k) * a[k] * ipow[k + m + 1];
        }
        b[m] = s;
    }
}

/* L2L: LE about zp -> LE about zc: b'_n = sum_{m>=n} C(m,n) b_m (zc - zp)^(m-n). */
static void l2l(int p, const cplx *b, cplx zp, cplx zc, cplx *out) {
    cplx d = zc - zp;
    cplx dpow[81];
    dpow[0] = 1.0;
    for (int i = 1; i < p; ++i) dpow[i] = dpow[i - 1] * d;
    for (int nn = 0; nn < p; ++nn) {
        cplx s = 0.0;
        for (int m = nn; m < p; ++m) s += binom(m, nn) * b[m] * dpow[m - nn];
        out[nn] = s;
    }
}

/* L2P: w(z) = sum_m b_m (z - zl)^m. */
static cplx l2p(int p, const cplx *b, cplx zl, cplx z) {
    cplx d = z - zl, pw = 1.0, w = 0.0;
    for (int m = 0; m < p; ++m) {
        w += b[m] * pw;
        pw *= d;
    }
    return w;
}

/* Direct evaluation of a multipole expansion (for pins). */
static cplx me_eval(int p, const cplx *a, cplx zc, cplx z) {
    cplx inv = 1.0 / (z - zc), pw = inv, w = 0.0;
    for (int k = 0; k < p; ++k) {
        w += a[k] * pw;
        pw *= inv;
    }
    return w;
}

/* Exposed single operators (interleaved re/im arrays of p complex values). */
void orc_p2m(int64_t n, const double *x, const double *y, const double *g,
             double zc_re, double zc_im, int p, double *a_out) {
    p2m(n, x, y, g, NULL, zc_re + I * zc_im, p, (cplx *)a_out);
}
void orc_m2m(int p, const double *a, double zc_re, double zc_im, double zp_re,
             double zp_im, double *out) {
    m2m(p, (const cplx *)a, zc_re + I * zc_im, zp_re + I * zp_im, (cplx *)out);
}
void orc_m2l(int p, const double *a, double zs_re, double zs_im, double zt_re,
             double zt_im, double *b) {
    m2l(p, (const cplx *)a, zs_re + I * zs_im, zt_re + I * zt_im, (cplx *)b);
}
void orc_l2l(int p, const double *b, double zp_re, double zp_im, double zc_re,
             double zc_im, double *out) {
    l2l(p, (const cplx *)b, zp_re + I * zp_im, zc_re + I * zc_im, (cplx *)out);
}
void orc_l2p(int p, const double *b, double zl_re, double zl_im, double z_re,
             double z_im, double *w_out) {
    cplx w = l2p(p, (const cplx *)b, zl_re + I * zl_im, z_re + I * z_im);
    w_out[0] = creal(w);
    w_out[1] = cimag(w);
}
void orc_me_eval(int p, const double *a, double zc_re, double zc_im, double z_re,
                 double z_im, double *w_out) {
    cplx w = me_eval(p, (const cplx *)a, zc_re + I * zc_im, z_re + I * z_im);
    w_out[0] = creal(w);
    w_out[1] = cimag(w);
}

/* ------------------------------------------------------------------ */
/* Tree helpers                                                        */
/* ------------------------------------------------------------------ */
static int64_t level_offset(int l) { return (((int64_t)1 << (2 * l)) - 1) / 3; }

static cplx box_centre(int l, uint32_t bx, uint32_t by, double x0, double y0, double W) {
    double r = W / (double)(1u << l);
    return (x0 + ((double)bx + 0.5) * r) + I * (y0 + ((double)by + 0.5) * r);
}

/* ------------------------------------------------------------------ */
/* O2: substituted direct sum.  Pairs in the near domain (leaf          */
/* Chebyshev distance <= 1) use K_sigma, all others the singular kernel.*/
/* ------------------------------------------------------------------ */
int orc_substituted(int64_t n, const double *x, const double *y, const double *g,
                    double x0, double y0, double W, int L, double sigma, int64_t nt,
                    const int64_t *targets, double *u, double *v, int nthreads) {
    uint32_t *ix = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *iy = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!ix || !iy || !key) { free(ix); free(iy); free(key); return ORC_ENOMEM; }
    int rc = orc_bin(n, x, y, x0, y0, W, L, ix, iy, key);
    if (rc != ORC_OK) { free(ix); free(iy); free(key); return rc; }
    set_threads(nthreads);
    if (targets == NULL) nt = n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double ku, kv;
            int64_t ddx = (int64_t)ix[i] - (int64_t)ix[j];
            int64_t ddy = (int64_t)iy[i] - (int64_t)iy[j];
            if (llabs(ddx) <= 1 && llabs(ddy) <= 1)
                k_sigma(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            else
                k_singular(x[i] - x[j], y[i] - y[j], &ku, &kv);
            su += g[j] * ku;
            sv += g[j] * kv;
        }
        u[t] = su;
        v[t] = sv;
    }
    free(ix); free(iy); free(key);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* O3: textbook FMM.                                                   */
/*                                                                     */
/* targets == NULL: every particle is evaluated and, if me_out/le_out  */
/* are given, the full ME/LE arrays are exported: Lambda(L) boxes x p  */
/* complex values (re, im interleaved), box index = (4^l - 1)/3 + m,   */
/* m = Morton index of the box at level l.                             */
/* targets != NULL: the upward pass is complete, the downward pass     */
/* runs only for the ancestors of the leaves holding a target, and     */
/* only the targets are evaluated (u[t], v[t] for targets[t]).         */
/* ------------------------------------------------------------------ */
int orc_fmm(int64_t n, const double *x, const double *y, const double *g,
            double x0, double y0, double W, int L, int p, double sigma,
            int64_t nt, const int64_t *targets, double *u, double *v,
            double *me_out, double *le_out, int nthreads) {
    if (L < 0 || L > 13 || p < 1 || p > 40 || !(sigma > 0.0) || !(W > 0.0) || n < 0)
        return ORC_EINVAL;
    set_threads(nthreads);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const int64_t nleaf = (int64_t)1 << (2 * L);
    const int64_t nbox = level_offset(L + 1);
    uint32_t *ix = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *iy = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nleaf + 1));
    cplx *me = (cplx *)calloc((size_t)nbox * (size_t)p, sizeof(cplx));
    cplx *le = (cplx *)calloc((size_t)nbox * (size_t)p, sizeof(cplx));
    unsigned char *need = (unsigned char *)calloc((size_t)nbox, 1);
    int rc = ORC_OK;
    if (!ix || !iy || !key || !perm || !start || !me || !le || !need) { rc = ORC_ENOMEM; goto done; }

    /* 1. Binning and z-order sort (Sec. 2.1). */
    rc = orc_bin(n, x, y, x0, y0, W, L, ix, iy, key);
    if (rc != ORC_OK) goto done;
    rc = orc_sort(n, key, L, perm, start);
    if (rc != ORC_OK) goto done;

    /* Boxes whose local expansion is needed: ancestors of target leaves. */
    if (targets == NULL) {
        memset(need, 1, (size_t)nbox);
    } else {
        for (int64_t t = 0; t < nt; ++t) {
            uint32_t m = key[targets[t]];
            for (int l = L; l >= 0; --l) need[level_offset(l) + (m >> (2 * (L - l)))] = 1;
        }
    }

    /* 2. Upward sweep: P2M at the leaves (Sec. 2.2, cost O(N_i p)). */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t m = 0; m < nleaf; ++m) {
        uint32_t bx, by;
        deinterleave((uint32_t)m, L, &bx, &by);
        cplx zc = box_centre(L, bx, by, x0, y0, W);
        p2m((int64_t)(start[m + 1] - start[m]), x, y, g, perm + start[m], zc, p,
            me + (level_offset(L) + m) * p);
    }
    /*    M2M from level l+1 to l, l = L-1 .. 0 (cost O(n_c p^2) per box). */
    for (int l = L - 1; l >= 0; --l) {
        int64_t nl = (int64_t)1 << (2 * l);
#pragma omp parallel for schedule(static)
        for (int64_t m = 0; m < nl; ++m) {
            uint32_t bx, by;
            deinterleave((uint32_t)m, l, &bx, &by);
            cplx zp = box_centre(l, bx, by, x0, y0, W);
            cplx *dst = me + (level_offset(l) + m) * p;
            cplx tmp[40];
            for (int c = 0; c < 4; ++c) {
                int64_t child = 4 * m + c;
                uint32_t cx, cy;
                deinterleave((uint32_t)child, l + 1, &cx, &cy);
                cplx zc = box_centre(l + 1, cx, cy, x0, y0, W);
                m2m(p, me + (level_offset(l + 1) + child) * p, zc, zp, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
        }
    }

    /* 3. Downward sweep, levels 2..L: M2L over the interaction list
     *    (O(p^2 n_IL) per box), then L2L from the parent (O(p^2)). */
    for (int l = 2; l <= L; ++l) {
        int64_t nl = (int64_t)1 << (2 * l);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t m = 0; m < nl; ++m) {
            if (!need[level_offset(l) + m]) continue;
            uint32_t bx, by;
            deinterleave((uint32_t)m, l, &bx, &by);
            cplx zt = box_centre(l, bx, by, x0, y0, W);
            cplx *dst = le + (level_offset(l) + m) * p;
            int32_t il[2 * 27];
            int cnt = orc_interaction_list(l, (int)bx, (int)by, il);
            cplx tmp[40];
            for (int s = 0; s < cnt; ++s) {
                uint32_t sx = (uint32_t)il[2 * s], sy = (uint32_t)il[2 * s + 1];
                uint32_t sm = interleave(sx, sy, l);
                cplx zs = box_centre(l, sx, sy, x0, y0, W);
                m2l(p, me + (level_offset(l) + sm) * p, zs, zt, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
            if (l >= 3) {
                uint32_t pm = (uint32_t)m >> 2, pbx, pby;
                deinterleave(pm, l - 1, &pbx, &pby);
                cplx zp = box_centre(l - 1, pbx, pby, x0, y0, W);
                l2l(p, le + (level_offset(l - 1) + pm) * p, zp, zt, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
        }
    }

    /* 4. Evaluation: L2P of the leaf's LE plus P2P over the near domain
     *    (the leaf and its neighbours), self excluded. */
    {
        int64_t ntt = targets ? nt : n;
        uint32_t nside = 1u << L;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t t = 0; t < ntt; ++t) {
            int64_t i = targets ? targets[t] : t;
            uint32_t m = key[i];
            cplx zl = box_centre(L, ix[i], iy[i], x0, y0, W);
            cplx w = l2p(p, le + (level_offset(L) + m) * p, zl, x[i] + I * y[i]);
            double su = cimag(w) / (2.0 * ORC_PI);
            double sv = creal(w) / (2.0 * ORC_PI);
            double nu = 0.0, nv = 0.0;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t sx = (int64_t)ix[i] + dx, sy = (int64_t)iy[i] + dy;
                    if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
                    uint32_t sm = interleave((uint32_t)sx, (uint32_t)sy, L);
                    for (uint32_t r = start[sm]; r < start[sm + 1]; ++r) {
                        uint32_t j = perm[r];
                        if ((int64_t)j == i) continue;
                        double ku, kv;
                        k_sigma(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
                        nu += g[j] * ku;
                        nv += g[j] * kv;
                    }
                }
            }
            u[t] = su + nu;
            v[t] = sv + nv;
        }
    }

    if (me_out) memcpy(me_out, me, sizeof(cplx) * (size_t)nbox * (size_t)p);
    if (le_out) memcpy(le_out, le, sizeof(cplx) * (size_t)nbox * (size_t)p);

done:
    free(ix); free(iy); free(key); free(perm); free(start);
    free(me); free(le); free(need);
    return rc;
}

/* ================================================================== */
/* Second kernel: the 2D logarithmic (Laplace) potential.              */
/*                                                                     */
/* The paper's Evaluator is templated over a Kernel object that        */
/* supplies the expansions and translation operators (Sec. 6.1), and   */
/* names other kernels as the first extensions (Sec. 8).  This is the  */
/* classic one for the same tree, interaction lists and sweeps:        */
/*                                                                     */
/*   phi(x_i) = sum_{j != i} q_j log |x_i - x_j|                        */
/*            = Re sum_{j != i} q_j log(z_i - z_j),   z = x + i y.      */
/*                                                                     */
/* Readings:                                                           */
/*   - p terms per expansion, the logarithm counted as one of them:    */
/*       ME about zc: Phi(z) = a_0 log(z - zc) + sum_{k=1}^{p-1} a_k / (z - zc)^k */
/*       LE about zl: Phi(z) = sum_{m=0}^{p-1} b_m (z - zl)^m           */
/*     The series are those of the complex logarithm, written out from */
/*     log(z - zj) = log(z - zc) + log(1 - (zj - zc)/(z - zc)).         */
/*   - The potential is Re Phi; the imaginary part (a branch-dependent */
/*     harmonic conjugate) is never used.                               */
/*   - Self pairs and coincident pairs contribute 0 (log 0 excluded),  */
/*     like the coincident pairs of the vortex kernel.                 */
/*   - No regularisation: the near field is the same sum evaluated     */
/*     directly.                                                        */
/* ================================================================== */

/* L1: direct sum. */
void orc_laplace_direct(int64_t n, const double *x, const double *y, const double *q,
                        int64_t nt, const int64_t *targets, double *phi, int nthreads) {
    set_threads(nthreads);
    if (targets == NULL) nt = n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j];
            double r2 = dx * dx + dy * dy;
            if (r2 == 0.0) continue;
            s += q[j] * 0.5 * log(r2);
        }
        phi[t] = s;
    }
}

/* P2M: a_0 = sum_j q_j, a_k = -sum_j q_j (z_j - zc)^k / k (k >= 1). */
static void lap_p2m(int64_t n, const double *x, const double *y, const double *q,
                    const uint32_t *idx, cplx zc, int p, cplx *a) {
    for (int k = 0; k < p; ++k) a[k] = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t j = idx ? idx[t] : t;
        cplx d = (x[j] + I * y[j]) - zc;
        a[0] += q[j];
        cplx pw = q[j];
        for (int k = 1; k < p; ++k) {
            pw *= d;
            a[k] -= pw / (double)k;
        }
    }
}

/* M2M: ME about zc -> ME about zp, d = zc - zp:
 *   out_0 = a_0,
 *   out_l = -a_0 d^l / l + sum_{k=1}^{l} C(l-1, k-1) a_k d^(l-k)   (l >= 1). */
static void lap_m2m(int p, const cplx *a, cplx zc, cplx zp, cplx *out) {
    cplx d = zc - zp;
    cplx dpow[81];
    dpow[0] = 1.0;
    for (int i = 1; i < p; ++i) dpow[i] = dpow[i - 1] * d;
    out[0] = a[0];
    for (int l = 1; l < p; ++l) {
        cplx s = -a[0] * dpow[l] / (double)l;
        for (int k = 1; k <= l; ++k) s += binom(l - 1, k - 1) * a[k] * dpow[l - k];
        out[l] = s;
    }
}

/* M2L: ME about zs -> LE about zt, d = zs - zt:
 *   b_0 = a_0 log(-d) + sum_{k>=1} (-1)^k a_k d^-k,
 *   b_m = -a_0 / (m d^m) + sum_{k>=1} (-1)^k C(m+k-1, k-1) a_k d^-(k+m)   (m >= 1). */
static void lap_m2l(int p, const cplx *a, cplx zs, cplx zt, cplx *b) {
    cplx d = zs - zt;
    cplx inv = 1.0 / d;
    cplx ipow[81];
    ipow[0] = 1.0;
    for (int i = 1; i <= 2 * p; ++i) ipow[i] = ipow[i - 1] * inv;
    cplx s0 = a[0] * clog(-d);
    for (int k = 1; k < p; ++k) s0 += ((k % 2) ? -1.0 : 1.0) * a[k] * ipow[k];
    b[0] = s0;
    for (int m = 1; m < p; ++m) {
        cplx s = -a[0] * ipow[m] / (double)m;
        for (int k = 1; k < p; ++k)
            s += ((k % 2) ? -1.0 : 1.0) * binom(m + k - 1, k - 1) * a[k] * ipow[k + m];
        b[m] = s;
    }
}

/* Direct evaluation of a Laplace multipole expansion (for pins). */
static cplx lap_me_eval(int p, const cplx *a, cplx zc, cplx z) {
    cplx inv = 1.0 / (z - zc), pw = inv, w = a[0] * clog(z - zc);
    for (int k = 1; k < p; ++k) {
        w += a[k] * pw;
        pw *= inv;
    }
    return w;
}

/* Exposed single operators (interleaved re/im arrays of p complex values;
 * the local-expansion shift and evaluation are the orc_l2l / orc_l2p above). */
void orc_lap_p2m(int64_t n, const double *x, const double *y, const double *q,
                 double zc_re, double zc_im, int p, double *a_out) {
    lap_p2m(n, x, y, q, NULL, zc_re + I * zc_im, p, (cplx *)a_out);
}
void orc_lap_m2m(int p, const double *a, double zc_re, double zc_im, double zp_re,
                 double zp_im, double *out) {
    lap_m2m(p, (const cplx *)a, zc_re + I * zc_im, zp_re + I * zp_im, (cplx *)out);
}
void orc_lap_m2l(int p, const double *a, double zs_re, double zs_im, double zt_re,
                 double zt_im, double *b_out) {
    lap_m2l(p, (const cplx *)a, zs_re + I * zs_im, zt_re + I * zt_im, (cplx *)b_out);
}
void orc_lap_me_eval(int p, const double *a, double zc_re, double zc_im, double z_re,
                     double z_im, double *w_out) {
    cplx w = lap_me_eval(p, (const cplx *)a, zc_re + I * zc_im, z_re + I * z_im);
    w_out[0] = creal(w);
    w_out[1] = cimag(w);
}

/* L3: FMM of the potential, same binning, sort, interaction lists and sweeps
 * as O3 (Sec. 2.2), with the operators above; targets / exports as in
 * orc_fmm. */
int orc_laplace_fmm(int64_t n, const double *x, const double *y, const double *q,
                    double x0, double y0, double W, int L, int p, int64_t nt,
                    const int64_t *targets, double *phi, double *me_out, double *le_out,
                    int nthreads) {
    if (L < 0 || L > 13 || p < 1 || p > 40 || !(W > 0.0) || n < 0) return ORC_EINVAL;
    set_threads(nthreads);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const int64_t nleaf = (int64_t)1 << (2 * L);
    const int64_t nbox = level_offset(L + 1);
    uint32_t *ix = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *iy = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nleaf + 1));
    cplx *me = (cplx *)calloc((size_t)nbox * (size_t)p, sizeof(cplx));
    cplx *le = (cplx *)calloc((size_t)nbox * (size_t)p, sizeof(cplx));
    unsigned char *need = (unsigned char *)calloc((size_t)nbox, 1);
    int rc = ORC_OK;
    if (!ix || !iy || !key || !perm || !start || !me || !le || !need) { rc = ORC_ENOMEM; goto done; }

    rc = orc_bin(n, x, y, x0, y0, W, L, ix, iy, key);
    if (rc != ORC_OK) goto done;
    rc = orc_sort(n, key, L, perm, start);
    if (rc != ORC_OK) goto done;

    if (targets == NULL) {
        memset(need, 1, (size_t)nbox);
    } else {
        for (int64_t t = 0; t < nt; ++t) {
            uint32_t m = key[targets[t]];
            for (int l = L; l >= 0; --l) need[level_offset(l) + (m >> (2 * (L - l)))] = 1;
        }
    }

    /* upward sweep: P2M at the leaves, M2M to the root */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t m = 0; m < nleaf; ++m) {
        uint32_t bx, by;
        deinterleave((uint32_t)m, L, &bx, &by);
        cplx zc = box_centre(L, bx, by, x0, y0, W);
        lap_p2m((int64_t)(start[m + 1] - start[m]), x, y, q, perm + start[m], zc, p,
                me + (level_offset(L) + m) * p);
    }
    for (int l = L - 1; l >= 0; --l) {
        int64_t nl = (int64_t)1 << (2 * l);
#pragma omp parallel for schedule(static)
        for (int64_t m = 0; m < nl; ++m) {
            uint32_t bx, by;
            deinterleave((uint32_t)m, l, &bx, &by);
            cplx zp = box_centre(l, bx, by, x0, y0, W);
            cplx *dst = me + (level_offset(l) + m) * p;
            cplx tmp[40];
            for (int c = 0; c < 4; ++c) {
                int64_t child = 4 * m + c;
                uint32_t cx, cy;
                deinterleave((uint32_t)child, l + 1, &cx, &cy);
                cplx zc = box_centre(l + 1, cx, cy, x0, y0, W);
                lap_m2m(p, me + (level_offset(l + 1) + child) * p, zc, zp, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
        }
    }

    /* downward sweep, levels 2..L: M2L over the interaction list, L2L */
    for (int l = 2; l <= L; ++l) {
        int64_t nl = (int64_t)1 << (2 * l);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t m = 0; m < nl; ++m) {
            if (!need[level_offset(l) + m]) continue;
            uint32_t bx, by;
            deinterleave((uint32_t)m, l, &bx, &by);
            cplx zt = box_centre(l, bx, by, x0, y0, W);
            cplx *dst = le + (level_offset(l) + m) * p;
            int32_t il[2 * 27];
            int cnt = orc_interaction_list(l, (int)bx, (int)by, il);
            cplx tmp[40];
            for (int s = 0; s < cnt; ++s) {
                uint32_t sx = (uint32_t)il[2 * s], sy = (uint32_t)il[2 * s + 1];
                uint32_t sm = interleave(sx, sy, l);
                cplx zs = box_centre(l, sx, sy, x0, y0, W);
                lap_m2l(p, me + (level_offset(l) + sm) * p, zs, zt, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
            if (l >= 3) {
                uint32_t pm = (uint32_t)m >> 2, pbx, pby;
                deinterleave(pm, l - 1, &pbx, &pby);
                cplx zp = box_centre(l - 1, pbx, pby, x0, y0, W);
                l2l(p, le + (level_offset(l - 1) + pm) * p, zp, zt, tmp);
                for (int k = 0; k < p; ++k) dst[k] += tmp[k];
            }
        }
    }

    /* evaluation: Re of the leaf's LE plus the near-field direct sum */
    {
        int64_t ntt = targets ? nt : n;
        uint32_t nside = 1u << L;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t t = 0; t < ntt; ++t) {
            int64_t i = targets ? targets[t] : t;
            uint32_t m = key[i];
            cplx zl = box_centre(L, ix[i], iy[i], x0, y0, W);
            double s = creal(l2p(p, le + (level_offset(L) + m) * p, zl, x[i] + I * y[i]));
            double nf = 0.0;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t sx = (int64_t)ix[i] + dx, sy = (int64_t)iy[i] + dy;
                    if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
                    uint32_t sm = interleave((uint32_t)sx, (uint32_t)sy, L);
                    for (uint32_t r = start[sm]; r < start[sm + 1]; ++r) {
                        uint32_t j = perm[r];
                        if ((int64_t)j == i) continue;
                        double ddx = x[i] - x[j], ddy = y[i] - y[j];
                        double r2 = ddx * ddx + ddy * ddy;
                        if (r2 == 0.0) continue;
                        nf += q[j] * 0.5 * log(r2);
                    }
                }
            }
            phi[t] = s + nf;
        }
    }

    if (me_out) memcpy(me_out, me, sizeof(cplx) * (size_t)nbox * (size_t)p);
    if (le_out) memcpy(le_out, le, sizeof(cplx) * (size_t)nbox * (size_t)p);

done:
    free(ix); free(iy); free(key); free(perm); free(start);
    free(me); free(le); free(need);
    return rc;
}
