/*
 * oracle3d.c -- plain, slow, FP64 CPU oracle for the three-dimensional
 * extension of the PetFMM evaluation: the Laplace potential and field of
 * point charges on a uniform octree.  The paper names 3D as its first
 * extension (Sec. 8): the tree, the work and communication model and the
 * partition carry over to three dimensions unchanged; what is new is the
 * kernel, with the 3D series and their translation operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes:
 *   D3  direct sum  phi_i = sum_{j != i} q_j / |x_i - x_j|,
 *                   E_i = -grad phi_i = sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3
 *                   (the N-body sum of Eq. 1 with the 3D Laplace kernel)
 *   F3  FMM         binning into a uniform octree (Sec. 2.1 in three
 *                   dimensions, z-order numbering of Sec. 5.1 with three
 *                   interleaved coordinates), P2M, M2M, M2L over the
 *                   interaction list, L2L, L2P and the near-field P2P (the
 *                   steps of Sec. 2.2 and Fig. 2), with p terms: degrees
 *                   n = 0..p-1 of the solid-harmonic series below.
 *
 * Series.  The paper gives no 3D series (it leaves the series out in 2D too,
 * Sec. 2.2); these are the textbook solid harmonics of the 1/r kernel,
 * normalised so that every translation is a plain convolution.  For
 * v = (x, y, z), r = |v|, and P_n^m the associated Legendre function without
 * the Condon-Shortley phase, for m >= 0
 *   R_n^m(v) = r^n P_n^m(z/r) e^{i m phi} / (n + m)!         (regular)
 *   I_n^m(v) = (n - m)! P_n^m(z/r) e^{i m phi} / r^{n + 1}   (irregular)
 * and R_n^{-m} = (-1)^m conj(R_n^m), I_n^{-m} = (-1)^m conj(I_n^m).  The
 * recurrences of P_n^m give them without angles:
 *   R_0^0 = 1, R_m^m = R_{m-1}^{m-1} (x + i y) / (2m),
 *   R_n^m = ((2n - 1) z R_{n-1}^m - r^2 R_{n-2}^m) / (n^2 - m^2);
 *   I_0^0 = 1 / r, I_m^m = (2m - 1) (x + i y) I_{m-1}^{m-1} / r^2,
 *   I_n^m = ((2n - 1) z I_{n-1}^m - ((n - 1)^2 - m^2) I_{n-2}^m) / r^2.
 * They satisfy (each checked by the tests against 1/|x - y| itself)
 *   1/|x - y|    = sum_{n,m} conj(R_n^m(y)) I_n^m(x)                  (|y| < |x|)
 *   R_n^m(a + b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b)
 *   I_n^m(a + b) = sum_{k,l} (-1)^k conj(R_k^l(b)) I_{n+k}^{m+l}(a)  (|b| < |a|)
 *   d/dz R_n^m = R_{n-1}^m,  (d/dx - i d/dy) R_n^m = R_{n-1}^{m-1},
 *   (d/dx + i d/dy) R_n^m = -R_{n-1}^{m+1}.
 * Expansions (every m from -n to n is stored):
 *   ME about c:  phi(x) = sum_{n,m} M_n^m I_n^m(x - c),
 *                M_n^m  = sum_j q_j conj(R_n^m(y_j - c))                 (P2M)
 *   LE about c:  phi(x) = sum_{n,m} L_n^m conj(R_n^m(x - c))             (L2P)
 *   M2M c -> c': M'_n^m = sum_{k,l} conj(R_k^l(c - c')) M_{n-k}^{m-l}
 *   M2L, D = c_t - c_s: L_k^l = (-1)^k sum_{n,m} M_n^m I_{n+k}^{m+l}(D)
 *   L2L c -> c': L'_j^s = sum_{k,l} L_{j+k}^{s+l} conj(R_k^l(c' - c))
 * M2M and L2L are exact for the truncated series; M2L truncates.
 *
 * Readings (as in two dimensions, oracle.c): p terms; near domain = the leaf
 * and its up to 26 neighbours; interaction list = the children of the
 * parent's neighbours that are not neighbours of the box (at most 189), for
 * levels >= 2; self and coincident pairs contribute 0; a point is binned per
 * coordinate as in 2D, the domain is the closed cube [x0, x0 + W]^3; Morton
 * key: bit b of ix to bit 3b, of iy to 3b + 1, of iz to 3b + 2; the sort is
 * stable.
 *
 * Compiled with -O2 -ffp-contract=off.  OpenMP splits only independent
 * outputs (boxes, targets), each computed in a fixed order by one thread.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O3_OK 0
#define O3_EINVAL (-1)
#define O3_ENOMEM (-2)
#define O3_EDOMAIN (-3)

typedef double complex cplx3;

/* coefficient (n, m) of a series of P degrees: index n (2P - 1) + m + P - 1 */
#define O3_IDX(P, n, m) ((n) * (2 * (P) - 1) + (m) + (P) - 1)

/* R_n^m(v) and (if Iv != NULL) I_n^m(v) for n < P, every m: the recurrences
 * above for m >= 0, then the (-1)^m conj rule for m < 0.  Iv needs v != 0. */
static void harmonics(double x, double y, double z, int P, cplx3 *Rv, cplx3 *Iv) {
    const double r2 = x * x + y * y + z * z;
    const cplx3 w = CMPLX(x, y);
    for (int m = 0; m < P; ++m) {
        Rv[O3_IDX(P, m, m)] = m == 0 ? 1.0 : Rv[O3_IDX(P, m - 1, m - 1)] * w / (2.0 * m);
        if (Iv)
            Iv[O3_IDX(P, m, m)] = m == 0 ? 1.0 / sqrt(r2)
                                         : Iv[O3_IDX(P, m - 1, m - 1)] * (2.0 * m - 1.0) * w / r2;
        for (int n = m + 1; n < P; ++n) {
            const cplx3 r1 = Rv[O3_IDX(P, n - 1, m)];
            const cplx3 rr = n - 2 >= m ? Rv[O3_IDX(P, n - 2, m)] : 0.0;
            Rv[O3_IDX(P, n, m)] = ((2.0 * n - 1.0) * z * r1 - r2 * rr) / (double)(n * n - m * m);
            if (Iv) {
                const cplx3 i1 = Iv[O3_IDX(P, n - 1, m)];
                const cplx3 ii = n - 2 >= m ? Iv[O3_IDX(P, n - 2, m)] : 0.0;
                Iv[O3_IDX(P, n, m)] =
                    ((2.0 * n - 1.0) * z * i1 - (double)((n - 1) * (n - 1) - m * m) * ii) / r2;
            }
        }
        if (m > 0) {
            const double sg = (m & 1) ? -1.0 : 1.0;
            for (int n = m; n < P; ++n) {
                Rv[O3_IDX(P, n, -m)] = sg * conj(Rv[O3_IDX(P, n, m)]);
                if (Iv) Iv[O3_IDX(P, n, -m)] = sg * conj(Iv[O3_IDX(P, n, m)]);
            }
        }
    }
}

/* exported for the tests: R and I of v for n < P, as (re, im) pairs in the
 * layout O3_IDX(P, n, m) (entries with |m| > n are left as they are) */
int o3_harmonics(double x, double y, double z, int P, double *R, double *Iout) {
    if (P < 1 || P > 64 || !R) return O3_EINVAL;
    if (Iout && x == 0.0 && y == 0.0 && z == 0.0) return O3_EINVAL;
    cplx3 *Rv = (cplx3 *)R, *Iv = (cplx3 *)Iout;
    harmonics(x, y, z, P, Rv, Iv);
    return O3_OK;
}

/* ------------------------------------------------------------------ */
/* Direct sum (D3)                                                     */
/* ------------------------------------------------------------------ */
int o3_direct(int64_t n, const double *x, const double *y, const double *z, const double *q,
              int64_t nt, const int64_t *targets, double *phi, double *ex, double *ey,
              double *ez) {
    if (n < 0 || nt < 0) return O3_EINVAL;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = targets ? targets[t] : t;
        double sp = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue; /* self and coincident pairs */
            const double r = sqrt(r2);
            const double inv = 1.0 / r;
            const double inv3 = inv / r2;
            sp += q[j] * inv;
            sx += q[j] * dx * inv3;
            sy += q[j] * dy * inv3;
            sz += q[j] * dz * inv3;
        }
        phi[t] = sp;
        ex[t] = sx;
        ey[t] = sy;
        ez[t] = sz;
    }
    return O3_OK;
}

/* ------------------------------------------------------------------ */
/* Octree: binning, z-order keys, stable sort, interaction list        */
/* ------------------------------------------------------------------ */
static uint32_t interleave3(uint32_t ix, uint32_t iy, uint32_t iz, int L) {
    uint32_t key = 0;
    for (int b = 0; b < L; ++b) {
        key |= ((ix >> b) & 1u) << (3 * b);
        key |= ((iy >> b) & 1u) << (3 * b + 1);
        key |= ((iz >> b) & 1u) << (3 * b + 2);
    }
    return key;
}

uint32_t o3_morton(uint32_t ix, uint32_t iy, uint32_t iz, int L) {
    return interleave3(ix, iy, iz, L);
}

static void deinterleave3(uint32_t key, int L, uint32_t *ix, uint32_t *iy, uint32_t *iz) {
    uint32_t a = 0, b = 0, c = 0;
    for (int k = 0; k < L; ++k) {
        a |= ((key >> (3 * k)) & 1u) << k;
        b |= ((key >> (3 * k + 1)) & 1u) << k;
        c |= ((key >> (3 * k + 2)) & 1u) << k;
    }
    *ix = a;
    *iy = b;
    *iz = c;
}

static uint32_t bin1d(double v, double v0, double scale, uint32_t nb) {
    const double t = v - v0;
    const double s = t * scale;
    const double f = floor(s);
    if (f < 0.0) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (uint32_t)f;
}

/* Leaf key of every particle (L <= 10: keys of 3L <= 30 bits).  ORC-style
 * O3_EDOMAIN if a particle lies outside the closed cube (or is NaN). */
int o3_bin(int64_t n, const double *x, const double *y, const double *z, double x0, double y0,
           double z0, double W, int L, uint32_t *key) {
    if (L < 0 || L > 10 || !(W > 0.0)) return O3_EINVAL;
    const double scale = ldexp(1.0, L) / W;
    const uint32_t nb = 1u << L;
    for (int64_t i = 0; i < n; ++i) {
        if (!(x[i] >= x0 && x[i] <= x0 + W && y[i] >= y0 && y[i] <= y0 + W && z[i] >= z0 &&
              z[i] <= z0 + W))
            return O3_EDOMAIN;
        key[i] = interleave3(bin1d(x[i], x0, scale, nb), bin1d(y[i], y0, scale, nb),
                             bin1d(z[i], z0, scale, nb), L);
    }
    return O3_OK;
}

/* Stable counting sort: perm[r] = input index of rank r; start[b] = first
 * rank with key >= b, b = 0..8^L (start[8^L] = n). */
int o3_sort(int64_t n, const uint32_t *key, int L, uint32_t *perm, uint32_t *start) {
    if (L < 0 || L > 8) return O3_EINVAL;
    const uint64_t nbox = 1ull << (3 * L);
    uint64_t *cur = (uint64_t *)calloc(nbox + 1, sizeof(uint64_t));
    if (!cur) return O3_ENOMEM;
    for (int64_t i = 0; i < n; ++i) cur[key[i] + 1] += 1;
    for (uint64_t b = 0; b < nbox; ++b) cur[b + 1] += cur[b];
    for (uint64_t b = 0; b <= nbox; ++b) start[b] = (uint32_t)cur[b];
    for (int64_t i = 0; i < n; ++i) perm[cur[key[i]]++] = (uint32_t)i;
    free(cur);
    return O3_OK;
}

/* The in-domain children of the parent's neighbours that are not neighbours
 * of box (l, ix, iy, iz): (sx, sy, sz) triples in ascending Morton order of
 * the source; returns the count (at most 189; 0 for l < 2). */
int o3_interaction_list(int l, int ix, int iy, int iz, int32_t *out) {
    if (l < 2) return 0;
    const int nside = 1 << l, npar = 1 << (l - 1);
    const int px = ix >> 1, py = iy >> 1, pz = iz >> 1;
    int cnt = 0;
    uint32_t keys[216];
    int32_t c3[216][3];
    for (int qz = pz - 1; qz <= pz + 1; ++qz)
        for (int qy = py - 1; qy <= py + 1; ++qy)
            for (int qx = px - 1; qx <= px + 1; ++qx) {
                if (qx < 0 || qy < 0 || qz < 0 || qx >= npar || qy >= npar || qz >= npar) continue;
                for (int c = 0; c < 8; ++c) {
                    const int sx = 2 * qx + (c & 1), sy = 2 * qy + ((c >> 1) & 1),
                              sz = 2 * qz + (c >> 2);
                    if (sx >= nside || sy >= nside || sz >= nside) continue;
                    if (abs(sx - ix) <= 1 && abs(sy - iy) <= 1 && abs(sz - iz) <= 1) continue;
                    keys[cnt] = interleave3((uint32_t)sx, (uint32_t)sy, (uint32_t)sz, l);
                    c3[cnt][0] = sx;
                    c3[cnt][1] = sy;
                    c3[cnt][2] = sz;
                    ++cnt;
                }
            }
    for (int a = 1; a < cnt; ++a) { /* insertion sort by key */
        const uint32_t k = keys[a];
        int32_t t[3] = {c3[a][0], c3[a][1], c3[a][2]};
        int b = a - 1;
        while (b >= 0 && keys[b] > k) {
            keys[b + 1] = keys[b];
            memcpy(c3[b + 1], c3[b], sizeof(c3[b]));
            --b;
        }
        keys[b + 1] = k;
        memcpy(c3[b + 1], t, sizeof(t));
    }
    for (int a = 0; a < cnt; ++a) memcpy(out + 3 * a, c3[a], sizeof(c3[a]));
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Operators (the formulas of the header), p terms, all m stored        */
/* ------------------------------------------------------------------ */
static int ncoef(int p) { return p * (2 * p - 1); }

/* P2M: M += sum_j q_j conj(R(y_j - c)) */
static void p2m3(int64_t n, const double *x, const double *y, const double *z, const double *q,
                 const double *c, int p, cplx3 *M) {
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    for (int64_t j = 0; j < n; ++j) {
        harmonics(x[j] - c[0], y[j] - c[1], z[j] - c[2], p, R, NULL);
        for (int nn = 0; nn < p; ++nn)
            for (int m = -nn; m <= nn; ++m) M[O3_IDX(p, nn, m)] += q[j] * conj(R[O3_IDX(p, nn, m)]);
    }
    free(R);
}

/* M2M: M'_n^m += sum_{k,l} conj(R_k^l(c - c')) M_{n-k}^{m-l} */
static void m2m3(int p, const cplx3 *M, const double *c, const double *cp, cplx3 *out) {
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    harmonics(c[0] - cp[0], c[1] - cp[1], c[2] - cp[2], p, R, NULL);
    for (int nn = 0; nn < p; ++nn)
        for (int m = -nn; m <= nn; ++m) {
            cplx3 s = 0.0;
            for (int k = 0; k <= nn; ++k)
                for (int l = -k; l <= k; ++l) {
                    const int mm = m - l;
                    if (mm < -(nn - k) || mm > nn - k) continue;
                    s += conj(R[O3_IDX(p, k, l)]) * M[O3_IDX(p, nn - k, mm)];
                }
            out[O3_IDX(p, nn, m)] += s;
        }
    free(R);
}

/* M2L: L_k^l += (-1)^k sum_{n,m} M_n^m I_{n+k}^{m+l}(c_t - c_s) */
static void m2l3(int p, const cplx3 *M, const double *cs, const double *ct, cplx3 *Lout) {
    const int P2 = 2 * p - 1;
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(P2));
    cplx3 *Iv = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(P2));
    harmonics(ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2], P2, R, Iv);
    for (int k = 0; k < p; ++k)
        for (int l = -k; l <= k; ++l) {
            cplx3 s = 0.0;
            for (int nn = 0; nn < p; ++nn)
                for (int m = -nn; m <= nn; ++m)
                    s += M[O3_IDX(p, nn, m)] * Iv[O3_IDX(P2, nn + k, m + l)];
            Lout[O3_IDX(p, k, l)] += ((k & 1) ? -1.0 : 1.0) * s;
        }
    free(R);
    free(Iv);
}

/* L2L: L'_j^s += sum_{k,l} L_{j+k}^{s+l} conj(R_k^l(c' - c)) */
static void l2l3(int p, const cplx3 *Lp, const double *c, const double *cc, cplx3 *out) {
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    harmonics(cc[0] - c[0], cc[1] - c[1], cc[2] - c[2], p, R, NULL);
    for (int j = 0; j < p; ++j)
        for (int s = -j; s <= j; ++s) {
            cplx3 acc = 0.0;
            for (int k = 0; j + k < p; ++k)
                for (int l = -k; l <= k; ++l) {
                    const int ss = s + l;
                    if (ss < -(j + k) || ss > j + k) continue;
                    acc += Lp[O3_IDX(p, j + k, ss)] * conj(R[O3_IDX(p, k, l)]);
                }
            out[O3_IDX(p, j, s)] += acc;
        }
    free(R);
}

/* L2P: phi = sum L_n^m conj(R_n^m(e)), E = -grad phi with
 * d/dz R_n^m = R_{n-1}^m, d/dx R_n^m = (R_{n-1}^{m-1} - R_{n-1}^{m+1}) / 2,
 * d/dy R_n^m = i (R_{n-1}^{m-1} + R_{n-1}^{m+1}) / 2 (from the identities of
 * the header); R with |m| > n counts as zero. */
static void l2p3(int p, const cplx3 *Lc, const double *c, double x, double y, double z,
                 double *phi, double *ex, double *ey, double *ez) {
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    harmonics(x - c[0], y - c[1], z - c[2], p, R, NULL);
    cplx3 f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int nn = 0; nn < p; ++nn)
        for (int m = -nn; m <= nn; ++m) {
            const cplx3 a = Lc[O3_IDX(p, nn, m)];
            f += a * conj(R[O3_IDX(p, nn, m)]);
            if (nn == 0) continue;
            const cplx3 rm = (m - 1 >= -(nn - 1)) ? R[O3_IDX(p, nn - 1, m - 1)] : 0.0;
            const cplx3 rp = (m + 1 <= nn - 1) ? R[O3_IDX(p, nn - 1, m + 1)] : 0.0;
            const cplx3 r0 = (m >= -(nn - 1) && m <= nn - 1) ? R[O3_IDX(p, nn - 1, m)] : 0.0;
            gx += a * conj(0.5 * (rm - rp));
            gy += a * conj(0.5 * I * (rm + rp));
            gz += a * conj(r0);
        }
    *phi += creal(f);
    *ex -= creal(gx);
    *ey -= creal(gy);
    *ez -= creal(gz);
    free(R);
}

/* multipole expansion evaluated at x (for the tests): sum M_n^m I_n^m(x - c) */
static double me_eval3(int p, const cplx3 *M, const double *c, double x, double y, double z) {
    cplx3 *R = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    cplx3 *Iv = (cplx3 *)malloc(sizeof(cplx3) * (size_t)ncoef(p));
    harmonics(x - c[0], y - c[1], z - c[2], p, R, Iv);
    cplx3 f = 0.0;
    for (int nn = 0; nn < p; ++nn)
        for (int m = -nn; m <= nn; ++m) f += M[O3_IDX(p, nn, m)] * Iv[O3_IDX(p, nn, m)];
    free(R);
    free(Iv);
    return creal(f);
}

/* exported operator wrappers (complex arrays as (re, im) pairs) */
void o3_p2m(int64_t n, const double *x, const double *y, const double *z, const double *q,
            const double *c, int p, double *M) {
    p2m3(n, x, y, z, q, c, p, (cplx3 *)M);
}
void o3_m2m(int p, const double *M, const double *c, const double *cp, double *out) {
    m2m3(p, (const cplx3 *)M, c, cp, (cplx3 *)out);
}
void o3_m2l(int p, const double *M, const double *cs, const double *ct, double *out) {
    m2l3(p, (const cplx3 *)M, cs, ct, (cplx3 *)out);
}
void o3_l2l(int p, const double *Lp, const double *c, const double *cc, double *out) {
    l2l3(p, (const cplx3 *)Lp, c, cc, (cplx3 *)out);
}
void o3_l2p(int p, const double *Lc, const double *c, double x, double y, double z, double *out4) {
    out4[0] = out4[1] = out4[2] = out4[3] = 0.0;
    l2p3(p, (const cplx3 *)Lc, c, x, y, z, out4, out4 + 1, out4 + 2, out4 + 3);
}
double o3_me_eval(int p, const double *M, const double *c, double x, double y, double z) {
    return me_eval3(p, (const cplx3 *)M, c, x, y, z);
}

/* ------------------------------------------------------------------ */
/* The FMM (F3)                                                        */
/* ------------------------------------------------------------------ */
static int64_t lvl_off3(int l) { return (((int64_t)1 << (3 * l)) - 1) / 7; }

static void centre3(int l, uint32_t key, double x0, double y0, double z0, double W, double *c) {
    uint32_t ix, iy, iz;
    deinterleave3(key, l, &ix, &iy, &iz);
    const double r = W / (double)(1u << l);
    c[0] = x0 + (ix + 0.5) * r;
    c[1] = y0 + (iy + 0.5) * r;
    c[2] = z0 + (iz + 0.5) * r;
}

int o3_fmm(int64_t n, const double *x, const double *y, const double *z, const double *q,
           double x0, double y0, double z0, double W, int L, int p, double *phi, double *ex,
           double *ey, double *ez) {
    if (n < 0 || L < 1 || L > 6 || p < 1 || p > 30 || !(W > 0.0)) return O3_EINVAL;
    const int nc = ncoef(p);
    const int64_t nbox = lvl_off3(L + 1);
    const uint64_t nleaf = 1ull << (3 * L);
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nleaf + 1));
    cplx3 *ME = (cplx3 *)calloc((size_t)(nbox * nc), sizeof(cplx3));
    cplx3 *LE = (cplx3 *)calloc((size_t)(nbox * nc), sizeof(cplx3));
    /* particle count of every box, all levels (empty boxes are skipped) */
    int64_t *cnt = (int64_t *)calloc((size_t)nbox, sizeof(int64_t));
    int rc = O3_OK;
    if (!key || !perm || !start || !ME || !LE || !cnt) {
        rc = O3_ENOMEM;
        goto done;
    }
    rc = o3_bin(n, x, y, z, x0, y0, z0, W, L, key);
    if (rc) goto done;
    rc = o3_sort(n, key, L, perm, start);
    if (rc) goto done;
    for (uint64_t b = 0; b < nleaf; ++b) {
        const int64_t c = (int64_t)start[b + 1] - (int64_t)start[b];
        for (int l = L; l >= 0; --l) cnt[lvl_off3(l) + (int64_t)(b >> (3 * (L - l)))] += c;
    }
    /* sorted copies of the particles */
    double *xs = (double *)malloc(sizeof(double) * 4 * (size_t)(n ? n : 1));
    if (!xs) {
        rc = O3_ENOMEM;
        goto done;
    }
    double *ys = xs + n, *zs = xs + 2 * n, *qs = xs + 3 * n;
    for (int64_t r = 0; r < n; ++r) {
        xs[r] = x[perm[r]];
        ys[r] = y[perm[r]];
        zs[r] = z[perm[r]];
        qs[r] = q[perm[r]];
    }
    /* P2M at the leaves */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < (int64_t)nleaf; ++b) {
        if (start[b + 1] == start[b]) continue;
        double c[3];
        centre3(L, (uint32_t)b, x0, y0, z0, W, c);
        p2m3((int64_t)(start[b + 1] - start[b]), xs + start[b], ys + start[b], zs + start[b],
             qs + start[b], c, p, ME + (lvl_off3(L) + b) * nc);
    }
    /* M2M, levels L-1 .. 2 */
    for (int l = L - 1; l >= 2; --l) {
        const int64_t nb = (int64_t)1 << (3 * l);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t b = 0; b < nb; ++b) {
            if (!cnt[lvl_off3(l) + b]) continue;
            double cp[3];
            centre3(l, (uint32_t)b, x0, y0, z0, W, cp);
            for (int ch = 0; ch < 8; ++ch) {
                const int64_t cb = 8 * b + ch;
                if (!cnt[lvl_off3(l + 1) + cb]) continue;
                double cc[3];
                centre3(l + 1, (uint32_t)cb, x0, y0, z0, W, cc);
                m2m3(p, ME + (lvl_off3(l + 1) + cb) * nc, cc, cp, ME + (lvl_off3(l) + b) * nc);
            }
        }
    }
    /* M2L over the interaction list, levels 2 .. L (sources in Morton order) */
    for (int l = 2; l <= L; ++l) {
        const int64_t nb = (int64_t)1 << (3 * l);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t b = 0; b < nb; ++b) {
            if (!cnt[lvl_off3(l) + b]) continue;
            uint32_t ix, iy, iz;
            deinterleave3((uint32_t)b, l, &ix, &iy, &iz);
            int32_t il[3 * 189];
            const int k = o3_interaction_list(l, (int)ix, (int)iy, (int)iz, il);
            double ct[3];
            centre3(l, (uint32_t)b, x0, y0, z0, W, ct);
            for (int a = 0; a < k; ++a) {
                const uint32_t sk = interleave3((uint32_t)il[3 * a], (uint32_t)il[3 * a + 1],
                                                (uint32_t)il[3 * a + 2], l);
                if (!cnt[lvl_off3(l) + sk]) continue;
                double cs[3];
                centre3(l, sk, x0, y0, z0, W, cs);
                m2l3(p, ME + (lvl_off3(l) + sk) * nc, cs, ct, LE + (lvl_off3(l) + b) * nc);
            }
        }
    }
    /* L2L, levels 2 .. L-1 to their children */
    for (int l = 2; l < L; ++l) {
        const int64_t nb = (int64_t)1 << (3 * (l + 1));
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t cb = 0; cb < nb; ++cb) {
            if (!cnt[lvl_off3(l + 1) + cb]) continue;
            double cp[3], cc[3];
            centre3(l, (uint32_t)(cb >> 3), x0, y0, z0, W, cp);
            centre3(l + 1, (uint32_t)cb, x0, y0, z0, W, cc);
            l2l3(p, LE + (lvl_off3(l) + (cb >> 3)) * nc, cp, cc, LE + (lvl_off3(l + 1) + cb) * nc);
        }
    }
    /* L2P and the near field over the leaf and its neighbours */
    const int nside = 1 << L;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n; ++r) {
        const uint32_t b = key[perm[r]];
        double c[3];
        centre3(L, b, x0, y0, z0, W, c);
        double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        if (L >= 2) l2p3(p, LE + (lvl_off3(L) + b) * nc, c, xs[r], ys[r], zs[r], &f, &gx, &gy, &gz);
        uint32_t ix, iy, iz;
        deinterleave3(b, L, &ix, &iy, &iz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = (int)ix + dx, sy = (int)iy + dy, sz = (int)iz + dz;
                    if (sx < 0 || sy < 0 || sz < 0 || sx >= nside || sy >= nside || sz >= nside)
                        continue;
                    const uint32_t sb = interleave3((uint32_t)sx, (uint32_t)sy, (uint32_t)sz, L);
                    for (uint32_t j = start[sb]; j < start[sb + 1]; ++j) {
                        const double ddx = xs[r] - xs[j], ddy = ys[r] - ys[j], ddz = zs[r] - zs[j];
                        const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        if (r2 == 0.0) continue;
                        const double inv = 1.0 / sqrt(r2);
                        const double inv3 = inv / r2;
                        f += qs[j] * inv;
                        gx += qs[j] * ddx * inv3;
                        gy += qs[j] * ddy * inv3;
                        gz += qs[j] * ddz * inv3;
                    }
                }
        const uint32_t i = perm[r];
        phi[i] = f;
        ex[i] = gx;
        ey[i] = gy;
        ez[i] = gz;
    }
    free(xs);
done:
    free(key);
    free(perm);
    free(start);
    free(ME);
    free(LE);
    free(cnt);
    return rc;
}
