// fmm3d.cu -- the three-dimensional extension and its C ABI (petfmm3d_* in
// include/petfmm.h).  The paper names 3D as its first extension (Sec. 8):
// tree, work model and partition carry over, and the new part is a kernel
// with the 3D series and translation operators.  This file evaluates the
// Laplace potential and field of point charges,
//     phi_i = sum_{j != i} q_j / |x_i - x_j|,    E_i = -grad phi_i,
// by the FMM on a uniform octree: binning with three-coordinate z-order keys
// (Sec. 2.1, Sec. 5.1), the radix sort and gather of the 2D path, then P2M,
// M2M, M2L over the interaction list (at most 189 boxes), L2L, and a final
// per-leaf pass that sums the near field over the leaf and its up to 26
// neighbours and adds L2P (the steps of Sec. 2.2).
//
// Series (the paper gives none for 3D): solid harmonics of the 1/r kernel,
//   R_n^m(v) = r^n P_n^m(z/r) e^{i m phi} / (n + m)!,
//   I_n^m(v) = (n - m)! P_n^m(z/r) e^{i m phi} / r^(n+1),
// P_n^m without the Condon-Shortley phase and X_n^-m = (-1)^m conj(X_n^m),
// from the Legendre recurrences in Cartesian form (rec_r / rec_i below).
// They obey 1/|x - y| = sum conj(R_n^m(y)) I_n^m(x), R(a + b) = sum
// R_k^l(a) R_{n-k}^{m-l}(b) and I_n^m(a + b) = sum (-1)^k conj(R_k^l(b))
// I_{n+k}^{m+l}(a), so that with M_n^m = sum q conj(R_n^m(y - c)) and
// phi = sum L_n^m conj(R_n^m(x - c)) the translations are plain sums:
//   M2M  M'_n^m = sum conj(R_k^l(c - c')) M_{n-k}^{m-l}
//   M2L  L_k^l  = (-1)^k sum M_n^m I_{n+k}^{m+l}(c_t - c_s)
//   L2L  L'_j^s = sum L_{j+k}^{s+l} conj(R_k^l(c' - c)).
// Expansions are rescaled by the box width w (M~ = M / w^n, L~ = L w^(n+1)):
// every operator is then level independent -- M2L one table of
// I_j^s(delta) per integer offset delta between same-level boxes, M2M and
// L2L one table of R_k^l(e) per child octant e = (+-1/4, +-1/4, +-1/4), with
// the level change a power of two -- and FP32 stays in range for p <= 16.
// Only m >= 0 is stored (p (p + 1) / 2 complex per box, index n (n + 1) / 2
// + m); m < 0 follows from the symmetry of a real potential.
//
// HBM layout: uint32 key / value ping-pong pairs of the radix sort (3L-bit
// keys), 8^L + 1 leaf starts, the sorted particles (FP64 path: SoA x, y, z, q
// in double; mixed path: float4 (xi, eta, zeta, q), the position relative to
// the leaf centre in leaf widths), ME and LE of every level (8^l boxes in
// Morton order, level l at box offset (8^l - 1) / 7), the operator tables.
// Every sum runs in a fixed order: results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/petfmm.h"
#include "kernels.cuh"
#include "tcgen05.cuh"

using namespace petfmm;

namespace {

constexpr int P3_MAX = PETFMM3D_MAX_P;           // terms
constexpr int L3_MAX = PETFMM3D_MAX_L;           // levels (3L <= 30 key bits)
constexpr int NC3_MAX = P3_MAX * (P3_MAX + 1) / 2;  // stored coefficients
constexpr int OUT3 = (NC3_MAX + 31) / 32;          // per lane, one warp per box
constexpr int NSLOT3 = 343;                        // offsets in [-3, 3]^3
constexpr int W3 = 8;                              // warps per block

template <typename T> struct C3;
template <> struct C3<float> { using V = float2; };
template <> struct C3<double> { using V = double2; };

template <typename V, typename T>
__host__ __device__ __forceinline__ V mk(T a, T b) { V v; v.x = a; v.y = b; return v; }

// a sorted particle of the FP64 path: x, y, z, q (32 bytes, one load)
struct __align__(32) Dbl4 {
    double x, y, z, w;
};

__host__ __device__ __forceinline__ int nc3(int p) { return p * (p + 1) / 2; }
// I_j^s, j < 2p - 1, s >= 0
__host__ __device__ __forceinline__ int nci3(int p) { return (2 * p - 1) * (2 * p) / 2; }
__host__ __device__ __forceinline__ int64_t lvl_off3(int l) {
    return ((int64_t(1) << (3 * l)) - 1) / 7;
}

// 3D z-order: bit b of ix, iy, iz to bits 3b, 3b + 1, 3b + 2 (10 bits each)
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030c30c3u;
    v = (v ^ (v >> 4)) & 0x0300f00fu;
    v = (v ^ (v >> 8)) & 0x030000ffu;
    v = (v ^ (v >> 16)) & 0x000003ffu;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
    return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// particles in box b of level l (from the leaf starts)
__device__ __forceinline__ uint32_t box_count3(const uint32_t *start, int L, int l, uint32_t b) {
    const int sh = 3 * (L - l);
    return start[(uint64_t(b) + 1) << sh] - start[uint64_t(b) << sh];
}

// coefficient (n, m) of a stored series; m < 0 by X_n^-m = (-1)^m conj(X_n^m)
template <typename V>
__device__ __forceinline__ V coef3(const V *a, int n, int m) {
    if (m >= 0) return a[n * (n + 1) / 2 + m];
    const V v = a[n * (n + 1) / 2 - m];
    return (m & 1) ? mk<V>(-v.x, v.y) : mk<V>(v.x, -v.y);
}

template <typename V> __device__ __forceinline__ void cmac(V &acc, V a, V b) {  // acc += a b
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
}
template <typename V> __device__ __forceinline__ void cmac_conj(V &acc, V a, V b) {  // acc += conj(a) b
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
}

// ---------------------------------------------------------------------------
// Binning (Sec. 2.1 in 3D): t = x - x0; s = t 2^L / W; floor, clamped; FP64
// with round-to-nearest intrinsics (no contraction), through an FP32
// shortcut with the same result.  recu (mixed path): the record (xi, eta,
// zeta, q) in input order, each coordinate rounded to FP32 and held below
// 0.5 - 2^-24.  The cap moves a point by at most one FP32
// rounding and keeps two particles of adjacent leaves apart by at least
// 2^-24 leaf widths along the axis they differ in, so |d| = 0 in the near
// field can only come from the target's own leaf.
// ---------------------------------------------------------------------------
constexpr float REC_MAX = 0.5f - 0x1p-24f;

struct Dom3 {
    double x0, y0, z0, width, scale;  // scale = 2^L / width
    // float-float copies (x0 = x0h + x0l, ..., scale = sh + sl) for the FP32
    // binning shortcut and the records
    float x0h, x0l, y0h, y0l, z0h, z0l, sh, sl;
};

__device__ __forceinline__ uint32_t bin3(double v, double v0, double scale, uint32_t nb) {
    const double f = floor(__dmul_rn(__dsub_rn(v, v0), scale));
    if (!(f >= 0.0)) return 0u;
    if (f > double(nb - 1)) return nb - 1;
    return uint32_t(f);
}

// FP32 shortcut of bin3 (FP64 arithmetic is slow here), bit-identical: with
// xf, x0f, scalef the FP32 roundings of v, v0, scale, s32 = fl(fl(xf - x0f)
// scalef) is within 4 u scale (|v| + |v0|) (u = 2^-24, plus O(u^2)) of the
// FP64 s, and m = 2^-21 scale (|v| + |v0|) covers that and the roundings of
// s32 -/+ m.  Both ends of [s32 - m, s32 + m] in one bin inside
// (0, nb (1 - 2^-20)) put s in that bin, unclamped, and v inside the domain
// (s > 0: v > v0; s < nb (1 - 2^-20): v <= fl(v0 + W) while |v0 + W| <=
// 2^32 W, and a domain farther out makes m > nb, failing the test);
// otherwise (a bin edge, the boundary, NaN, Inf) false: the FP64 path.
__device__ __forceinline__ bool bin3_fast(float xf, float x0f, float scalef, uint32_t nb,
                                          uint32_t *bin) {
    const float sv = __fmul_rn(__fsub_rn(xf, x0f), scalef);
    const float m = __fmul_rn(__fmul_rn(__fadd_rn(fabsf(xf), fabsf(x0f)), scalef), 0x1p-21f);
    const float lo = __fsub_rn(sv, m), hi = __fadd_rn(sv, m);
    if (!(lo > 0.0f && hi < float(nb) * (1.0f - 0x1p-20f))) return false;
    const float f = floorf(lo);
    if (f != floorf(hi)) return false;
    *bin = uint32_t(f);
    return true;
}

// The record coordinate (v - v0) scale - (i + 1/2) in float-float
// arithmetic (two-sum for the difference, FMA for the product's error
// terms): before its final rounding within about 2^-44 of the exact value,
// relative to (v - v0) scale.
__device__ __forceinline__ void ff_split(float v, float *h, float *l) { *h = v; *l = 0.f; }
__device__ __forceinline__ void ff_split(double v, float *h, float *l) {
    *h = float(v);
    *l = float(v - double(*h));
}
template <typename TIn>
__device__ __forceinline__ float rec3_coord(TIn v, float v0h, float v0l, float sh, float sl,
                                            uint32_t i) {
    float vh, vl;
    ff_split(v, &vh, &vl);
    const float th = __fsub_rn(vh, v0h);
    const float bv = __fsub_rn(th, vh);
    float tl = __fadd_rn(__fsub_rn(vh, __fsub_rn(th, bv)), __fsub_rn(-v0h, bv));
    tl = __fadd_rn(tl, __fsub_rn(vl, v0l));
    const float ph = __fmul_rn(th, sh);
    float pe = __fmaf_rn(th, sh, -ph);
    pe = __fmaf_rn(th, sl, __fmaf_rn(tl, sh, pe));
    return __fadd_rn(__fsub_rn(ph, __fadd_rn(float(i), 0.5f)), pe);
}

template <typename TIn>
__global__ void __launch_bounds__(256) k3_bin(int64_t n, const TIn *__restrict__ x,
                                              const TIn *__restrict__ y, const TIn *__restrict__ z,
                                              const TIn *__restrict__ q, Dom3 d, int L,
                                              uint32_t *__restrict__ keys,
                                              float4 *__restrict__ recu, int *status) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const TIn xv = x[j], yv = y[j], zv = z[j];
    const uint32_t nb = 1u << L;
    uint32_t ix, iy, iz;
    if (!(bin3_fast(float(xv), d.x0h, d.sh, nb, &ix) && bin3_fast(float(yv), d.y0h, d.sh, nb, &iy) &&
          bin3_fast(float(zv), d.z0h, d.sh, nb, &iz))) {
        const double X = double(xv), Y = double(yv), Z = double(zv);
        const double x1 = __dadd_rn(d.x0, d.width), y1 = __dadd_rn(d.y0, d.width),
                     z1 = __dadd_rn(d.z0, d.width);
        if (!(X >= d.x0 && X <= x1 && Y >= d.y0 && Y <= y1 && Z >= d.z0 && Z <= z1))
            set_status(status, ST_EDOMAIN);
        ix = bin3(X, d.x0, d.scale, nb);
        iy = bin3(Y, d.y0, d.scale, nb);
        iz = bin3(Z, d.z0, d.scale, nb);
    }
    keys[j] = morton3(ix, iy, iz);
    if (recu) {
        float4 r;
        r.x = fminf(rec3_coord(xv, d.x0h, d.x0l, d.sh, d.sl, ix), REC_MAX);
        r.y = fminf(rec3_coord(yv, d.y0h, d.y0l, d.sh, d.sl, iy), REC_MAX);
        r.z = fminf(rec3_coord(zv, d.z0h, d.z0l, d.sh, d.sl, iz), REC_MAX);
        r.w = float(q[j]);
        recu[j] = r;
    }
}

// start[b] = first sorted rank with key >= b, b = 0..8^L
__global__ void __launch_bounds__(256) k3_leaf_start(const uint32_t *__restrict__ skeys, int64_t n,
                                                     int64_t nleaf, uint32_t *__restrict__ start) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b > nleaf) return;
    int64_t lo = 0, hi = n;
    if (b == nleaf) {
        lo = n;
    } else {
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (int64_t(skeys[mid]) < b) lo = mid + 1; else hi = mid;
        }
    }
    start[b] = uint32_t(lo);
}

template <typename TIn>
__global__ void __launch_bounds__(256) k3_gather_f64(int64_t n, const uint32_t *__restrict__ perm,
                                                     const TIn *__restrict__ x,
                                                     const TIn *__restrict__ y,
                                                     const TIn *__restrict__ z,
                                                     const TIn *__restrict__ q,
                                                     Dbl4 *__restrict__ out) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t i = perm[r];
    if (!PF_IN(i, n)) return;
    out[r] = Dbl4{double(x[i]), double(y[i]), double(z[i]), double(q[i])};
}

// A particle of the leaf as (position relative to the leaf centre in leaf
// widths, charge).
template <typename T> struct Part3 { T x, y, z, q; };
__device__ __forceinline__ Part3<float> leaf_part(const float4 *rec, int64_t j, double, double,
                                                  double, double) {
    const float4 r = rec[j];
    return {r.x, r.y, r.z, r.w};
}
__device__ __forceinline__ Part3<double> leaf_part(const Dbl4 *xs, int64_t j, double cx,
                                                   double cy, double cz, double inv_w) {
    const Dbl4 r = xs[j];
    return {(r.x - cx) * inv_w, (r.y - cy) * inv_w, (r.z - cz) * inv_w, r.w};
}

// ---------------------------------------------------------------------------
// P2M (leaves): M~_n^m = sum_j q_j conj(R_n^m(xi_j)).  A warp per leaf split
// into 32 / p lane groups; lane m of a group owns column m: R_m^m = (xi + i
// eta)^m / (2^m m!), then the recurrence in n (its reciprocals computed once
// per lane), for every G-th particle of the leaf; the groups' sums are added
// in group order.
// ---------------------------------------------------------------------------
template <typename T, typename P>
__global__ void __launch_bounds__(W3 * 32) k3_p2m(int L, int p, Dom3 d, const uint32_t *__restrict__ start,
                                                  const P *__restrict__ part,
                                                  typename C3<T>::V *__restrict__ me) {
    using V = typename C3<T>::V;
    const int lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * W3 + (threadIdx.x >> 5);
    if (b >= (int64_t(1) << (3 * L))) return;
    const uint32_t s0 = start[b], s1 = start[b + 1];
    if (s0 == s1) return;
    // G = 32 / p lane groups, group g summing particles g, g + G, ...; lane
    // m of a group owns column m
    const int G = 32 / p, g = lane / p, m = lane - g * p;
    const double w = d.width / double(1u << L);
    const double cx = d.x0 + (double(compact3(uint32_t(b))) + 0.5) * w;
    const double cy = d.y0 + (double(compact3(uint32_t(b) >> 1)) + 0.5) * w;
    const double cz = d.z0 + (double(compact3(uint32_t(b) >> 2)) + 0.5) * w;
    V acc[P3_MAX];
    // the lane's constants, out of the particle loop: 1 / (2^m m!) and
    // 1 / (n^2 - m^2) of the recurrence
    T cm = T(1), inv[P3_MAX];
    for (int t = 1; t <= m; ++t) cm /= T(2 * t);
#pragma unroll
    for (int n = 0; n < P3_MAX; ++n) {
        acc[n] = mk<V>(T(0), T(0));
        inv[n] = n > m && n < p ? T(1) / T(n * n - m * m) : T(0);
    }
    // the leaf's records staged 64 at a time in shared memory by coalesced
    // loads, so that no particle's load waits in the groups' loops
    __shared__ P stage[W3][64];
    const int wid = threadIdx.x >> 5;
    for (uint32_t c0 = s0; c0 < s1; c0 += 64u) {
        const uint32_t cn = min(64u, s1 - c0);
        __syncwarp();
        for (uint32_t i = uint32_t(lane); i < cn; i += 32u) stage[wid][i] = part[c0 + i];
        __syncwarp();
        if (g >= G) continue;
        for (uint32_t j = uint32_t(g); j < cn; j += uint32_t(G)) {
            const Part3<T> a = leaf_part(stage[wid], j, cx, cy, cz, 1.0 / w);
            const T r2 = a.x * a.x + a.y * a.y + a.z * a.z;
            V zm = mk<V>(T(1), T(0));  // (xi + i eta)^m
            for (int t = 1; t <= m; ++t) zm = mk<V>(zm.x * a.x - zm.y * a.y, zm.x * a.y + zm.y * a.x);
            const T qc = a.q * cm;
            V r1 = mk<V>(zm.x * qc, zm.y * qc), r2v = mk<V>(T(0), T(0));  // q R_m^m
#pragma unroll
            for (int n = 0; n < P3_MAX; ++n) {
                if (n < m || n >= p) continue;
                V rn = r1;
                if (n > m) {
                    const T c1 = T(2 * n - 1) * a.z;
                    rn = mk<V>((c1 * r1.x - r2 * r2v.x) * inv[n], (c1 * r1.y - r2 * r2v.y) * inv[n]);
                    r2v = r1;
                    r1 = rn;
                }
                acc[n].x += rn.x;  // q conj(R) summed: conj taken at the end
                acc[n].y += rn.y;
            }
        }
    }
    // the groups' partial sums added into group 0 in group order (every lane
    // takes part in the shuffles)
#pragma unroll
    for (int n = 0; n < P3_MAX; ++n) {
        for (int gg = 1; gg < G; ++gg) {
            const int src = m + gg * p;
            const T ox = __shfl_sync(0xffffffffu, acc[n].x, src);
            const T oy = __shfl_sync(0xffffffffu, acc[n].y, src);
            if (g == 0) {
                acc[n].x += ox;
                acc[n].y += oy;
            }
        }
    }
    if (g == 0) {
        V *dst = me + (lvl_off3(L) + b) * nc3(p);
#pragma unroll
        for (int n = 0; n < P3_MAX; ++n)
            if (n >= m && n < p) dst[n * (n + 1) / 2 + m] = mk<V>(acc[n].x, -acc[n].y);
    }
}

// P2M of the mixed path for p <= 8: a warp per leaf with a lane per charge
// (charges j, j + 32, ... of the leaf), each lane computing all p (p + 1) / 2
// terms q R_n^m column by column with compile-time constants and summing
// them over its charges; then a reduce-scatter across the warp (three
// halving exchanges, offsets 16, 8, 4, then a butterfly over offsets 2 and
// 1) leaves each group of four lanes the full sums of a ninth of the 2 NC
// values, which one lane of the group writes.
template <int P>
__global__ void __launch_bounds__(W3 * 32) k3_p2m_lanes(int L, const uint32_t *__restrict__ start,
                                                        const float4 *__restrict__ rec,
                                                        float2 *__restrict__ me) {
    constexpr int NC = P * (P + 1) / 2, NV = 2 * NC;  // values: Re of all, then Im of all
    constexpr int NV8 = (NV + 7) / 8, NVP = 8 * NV8;  // padded to eight equal parts
    const int lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * W3 + (threadIdx.x >> 5);
    if (b >= (int64_t(1) << (3 * L))) return;
    const uint32_t s0 = start[b], s1 = start[b + 1];
    if (s0 == s1) return;
    float v[NVP];
#pragma unroll
    for (int k = 0; k < NVP; ++k) v[k] = 0.f;
    for (uint32_t j = s0 + uint32_t(lane); j < s1; j += 32u) {
        const float4 a = rec[j];
        const float r2 = a.x * a.x + a.y * a.y + a.z * a.z;
        float pr = a.w, pi = 0.f;  // q R_m^m
#pragma unroll
        for (int m = 0; m < P; ++m) {
            if (m > 0) {
                const float sc = 1.f / float(2 * m);
                const float tr = (pr * a.x - pi * a.y) * sc, ti = (pr * a.y + pi * a.x) * sc;
                pr = tr;
                pi = ti;
            }
            float r1r = pr, r1i = pi, r0r = 0.f, r0i = 0.f;
            v[m * (m + 1) / 2 + m] += r1r;
            v[NC + m * (m + 1) / 2 + m] += r1i;
#pragma unroll
            for (int n = m + 1; n < P; ++n) {
                const float c1 = float(2 * n - 1) * a.z;
                const float inv = 1.f / float(n * n - m * m);
                const float rr = (c1 * r1r - r2 * r0r) * inv, ri = (c1 * r1i - r2 * r0i) * inv;
                r0r = r1r;
                r0i = r1i;
                r1r = rr;
                r1i = ri;
                v[n * (n + 1) / 2 + m] += rr;
                v[NC + n * (n + 1) / 2 + m] += ri;
            }
        }
    }
    // halving exchanges: at offset o the lane keeps the lower half of its
    // values if (lane & o) == 0, else the upper half, adding the partner's
    // copy of the half it keeps
#pragma unroll
    for (int k = 0; k < NVP / 2; ++k) {
        const bool up = lane & 16;
        const float send = up ? v[k] : v[k + NVP / 2];
        const float keep = up ? v[k + NVP / 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < NVP / 4; ++k) {
        const bool up = lane & 8;
        const float send = up ? v[k] : v[k + NVP / 4];
        const float keep = up ? v[k + NVP / 4] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < NV8; ++k) {
        const bool up = lane & 4;
        const float send = up ? v[k] : v[k + NV8];
        const float keep = up ? v[k + NV8] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int k = 0; k < NV8; ++k) {
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 2);
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1);
    }
    // this group's values: index 4 NVP/8 bit4 + 2 NVP/8 bit3 + NVP/8 bit2 + k
    if ((lane & 3) == 0) {
        const int base = NV8 * (4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1));
        float *dst = reinterpret_cast<float *>(me + (lvl_off3(L) + b) * NC);
#pragma unroll
        for (int k = 0; k < NV8; ++k) {
            const int vi = base + k;
            if (vi < NC)
                dst[2 * vi] = v[k];
            else if (vi < NV)
                dst[2 * (vi - NC) + 1] = -v[k];  // conj
        }
    }
}

template <int P>
cudaError_t p2m_lanes_p(int L, const uint32_t *start, const float4 *rec, float2 *me, cudaStream_t st) {
    k3_p2m_lanes<P><<<unsigned(((int64_t(1) << (3 * L)) + W3 - 1) / W3), W3 * 32, 0, st>>>(L, start,
                                                                                          rec, me);
    return cudaGetLastError();
}

cudaError_t launch_p2m_lanes(int p, int L, const uint32_t *start, const float4 *rec, float2 *me,
                             cudaStream_t st) {
    switch (p) {
#define PL_CASE(P) case P: return p2m_lanes_p<P>(L, start, rec, me, st);
        PL_CASE(1) PL_CASE(2) PL_CASE(3) PL_CASE(4) PL_CASE(5) PL_CASE(6) PL_CASE(7) PL_CASE(8)
#undef PL_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// M2M (parent level l from level l + 1): M~'_n^m = sum_children sum_{k,l}
// conj(R_k^l(e_c)) 2^-(n-k) M~_{n-k}^{m-l}.  A warp per parent box, lanes over
// output coefficients, children in octant order.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(W3 * 32) k3_m2m(int l, int L, int p, const uint32_t *__restrict__ start,
                                                  const typename C3<T>::V *__restrict__ rtab,
                                                  typename C3<T>::V *__restrict__ me) {
    using V = typename C3<T>::V;
    const int lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * W3 + (threadIdx.x >> 5);
    if (b >= (int64_t(1) << (3 * l))) return;
    if (box_count3(start, L, l, uint32_t(b)) == 0) return;
    const int nc = nc3(p);
    V acc[OUT3];
    int on[OUT3], om[OUT3];
#pragma unroll
    for (int u = 0; u < OUT3; ++u) {
        acc[u] = mk<V>(T(0), T(0));
        const int j = lane + 32 * u;
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= j) ++n;
        on[u] = n;
        om[u] = j - n * (n + 1) / 2;
    }
    for (int c = 0; c < 8; ++c) {
        const uint32_t cb = uint32_t(b) * 8u + uint32_t(c);
        if (box_count3(start, L, l + 1, cb) == 0) continue;
        const V *mc = me + (lvl_off3(l + 1) + cb) * nc;
        const V *rt = rtab + c * nc;
#pragma unroll
        for (int u = 0; u < OUT3; ++u) {
            if (lane + 32 * u >= nc) continue;
            const int n = on[u], m = om[u];
            V s = mk<V>(T(0), T(0));
            for (int k = 0; k <= n; ++k) {
                V sk = mk<V>(T(0), T(0));
                for (int ll = -k; ll <= k; ++ll) {
                    const int mm = m - ll;
                    if (mm < -(n - k) || mm > n - k) continue;
                    cmac_conj(sk, coef3(rt, k, ll), coef3(mc, n - k, mm));
                }
                const T sc = T(ldexp(1.0, -(n - k)));
                s.x += sk.x * sc;
                s.y += sk.y * sc;
            }
            acc[u].x += s.x;
            acc[u].y += s.y;
        }
    }
    V *dst = me + (lvl_off3(l) + b) * nc;
#pragma unroll
    for (int u = 0; u < OUT3; ++u)
        if (lane + 32 * u < nc) dst[lane + 32 * u] = acc[u];
}

// ---------------------------------------------------------------------------
// M2L (level l >= 2): L~_k^l = (-1)^k sum_{n,m} M~_n^m I_{n+k}^{m+l}(delta),
// delta = target - source in box widths, over the interaction list: the
// children of the parent's neighbours that are not neighbours of the box,
// in a fixed order.  A warp per target box; the source's expansion is staged
// in shared memory for the warp, lanes over output coefficients.  The result
// is written (the L2L that follows adds the parent's part).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(W3 * 32) k3_m2l(int l, int L, int p, const uint32_t *__restrict__ start,
                                                  const typename C3<T>::V *__restrict__ itab,
                                                  const typename C3<T>::V *__restrict__ me,
                                                  typename C3<T>::V *__restrict__ le) {
    using V = typename C3<T>::V;
    __shared__ V sme[W3][NC3_MAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b = int64_t(blockIdx.x) * W3 + wid;
    if (b >= (int64_t(1) << (3 * l))) return;
    if (box_count3(start, L, l, uint32_t(b)) == 0) return;
    const int nc = nc3(p), nci = nci3(p);
    const int ix = int(compact3(uint32_t(b))), iy = int(compact3(uint32_t(b) >> 1)),
              iz = int(compact3(uint32_t(b) >> 2));
    const int pside = 1 << (l - 1);
    V acc[OUT3];
    int on[OUT3], om[OUT3];
#pragma unroll
    for (int u = 0; u < OUT3; ++u) {
        acc[u] = mk<V>(T(0), T(0));
        const int j = lane + 32 * u;
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= j) ++n;
        on[u] = n;
        om[u] = j - n * (n + 1) / 2;
    }
    const V *lev = me + lvl_off3(l) * nc;
    for (int qz = (iz >> 1) - 1; qz <= (iz >> 1) + 1; ++qz)
        for (int qy = (iy >> 1) - 1; qy <= (iy >> 1) + 1; ++qy)
            for (int qx = (ix >> 1) - 1; qx <= (ix >> 1) + 1; ++qx) {
                if (qx < 0 || qy < 0 || qz < 0 || qx >= pside || qy >= pside || qz >= pside)
                    continue;
                for (int c = 0; c < 8; ++c) {
                    const int sx = 2 * qx + (c & 1), sy = 2 * qy + ((c >> 1) & 1),
                              sz = 2 * qz + (c >> 2);
                    const int dx = ix - sx, dy = iy - sy, dz = iz - sz;
                    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) continue;
                    const uint32_t sb = morton3(uint32_t(sx), uint32_t(sy), uint32_t(sz));
                    if (box_count3(start, L, l, sb) == 0) continue;
                    __syncwarp();
                    for (int i = lane; i < nc; i += 32) sme[wid][i] = lev[int64_t(sb) * nc + i];
                    __syncwarp();
                    const V *tab = itab + ((dx + 3) + 7 * (dy + 3) + 49 * (dz + 3)) * nci;
#pragma unroll
                    for (int u = 0; u < OUT3; ++u) {
                        if (lane + 32 * u >= nc) continue;
                        const int k = on[u], lo = om[u];
                        V s = mk<V>(T(0), T(0));
                        for (int n = 0; n < p; ++n)
                            for (int m = -n; m <= n; ++m)
                                cmac(s, coef3(sme[wid], n, m), coef3(tab, n + k, m + lo));
                        if (k & 1) {
                            acc[u].x -= s.x;
                            acc[u].y -= s.y;
                        } else {
                            acc[u].x += s.x;
                            acc[u].y += s.y;
                        }
                    }
                }
            }
    V *dst = le + (lvl_off3(l) + b) * nc;
#pragma unroll
    for (int u = 0; u < OUT3; ++u)
        if (lane + 32 * u < nc) dst[lane + 32 * u] = acc[u];
}

// ---------------------------------------------------------------------------
// M2L of the mixed path as GEMMs.  The coefficients of a real potential with
// degrees < p are p^2 real numbers: Re of every stored (n, m), then Im of
// those with m > 0 (Im of m = 0 is zero).  In that basis each offset's
// translation is a fixed real p^2 x p^2 matrix A_delta (built on the host in
// FP64 from the M2L sum, rounded to FP32; stored transposed, k-major, padded
// to NRP = p^2 rounded up to 32); rmap[r] = (coefficient, part) of real index
// r, part 0 = Re, 1 = Im, 2 = Re of an m = 0 coefficient (its Im is zero).  A block takes 64 consecutive parent cells
// (Morton order) of level l - 1 and one target child class c: 64 target rows.
// For each (source class cs, parent offset d) of the interaction list of
// class c (delta = c - cs - 2d, |delta|_inf >= 2), the 64 source rows (parent
// P + d, class cs; zero when outside the domain or empty) are staged k-major
// in shared memory and multiplied by A_delta in K chunks of 32: every thread
// owns 4 rows x NRP / 8 columns, reading its 4 rows with one 16-byte load and
// its columns with 16-byte loads (conflict-free: a warp spans 4 row groups x
// 8 column groups).  Sums in a fixed order; the result is written, the L2L
// that follows adds the parent's part.
// ---------------------------------------------------------------------------
constexpr int MG_ROWS = 64, MG_THREADS = 128, MG_XS = MG_ROWS + 4;
#ifndef MG_PIPE_ROWS
#define MG_PIPE_ROWS 128  // target rows per block of the pipelined M2L (64 or 128)
#endif

__host__ __device__ constexpr int mg_nrp(int p) { return (p * p + 31) / 32 * 32; }
// K chunk of A staged at once: all of it up to 64 rows, else 64 or 32 rows,
// whichever divides NRP (so no chunk reads past its operator)
__host__ __device__ constexpr int mg_kt(int p) {
    return mg_nrp(p) <= 64 ? mg_nrp(p) : (mg_nrp(p) % 64 == 0 ? 64 : 32);
}

template <int P>
__global__ void __launch_bounds__(MG_THREADS) k3_m2l_gemm(int l, int L, const uint32_t *__restrict__ start,
                                                        const float *__restrict__ atab,
                                                        const short2 *__restrict__ rmap,
                                                        const float2 *__restrict__ me,
                                                        float2 *__restrict__ le) {
    constexpr int NC = P * (P + 1) / 2, NR = P * P, NRP = mg_nrp(P), CG = NRP / 8;
    constexpr int KT = mg_kt(P);
    static_assert(NRP % KT == 0 && KT % 4 == 0 && CG % 4 == 0, "chunking");
    constexpr int NLOAD = (MG_ROWS * NC + MG_THREADS - 1) / MG_THREADS;
    extern __shared__ __align__(16) float mg_smem[];
    float *xs = mg_smem;                 // [NRP][MG_XS]: X^T, k-major
    float *as = xs + NRP * MG_XS;        // [KT][NRP]: a K chunk of A^T
    __shared__ int srow[MG_ROWS];
    __shared__ short imr[NC];            // real index of Im of coefficient j (m > 0), else -1
    const int tid = threadIdx.x, rg = tid >> 3, g = tid & 7;
    const int c = int(blockIdx.x & 7);
    const int64_t np = int64_t(1) << (3 * (l - 1));  // parent cells of level l - 1
    const int64_t p0 = int64_t(blockIdx.x >> 3) * MG_ROWS;
    const int pside = 1 << (l - 1);
    for (int i = tid; i < (NRP - NR) * MG_XS; i += MG_THREADS) xs[NR * MG_XS + i] = 0.f;
    for (int j = tid; j < NC; j += MG_THREADS) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= j) ++n;
        // the m > 0 coefficients before j, in order: j - n - 1
        imr[j] = short(j == n * (n + 1) / 2 ? -1 : NC + j - n - 1);
    }
    float acc[4][CG];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[i][j] = 0.f;
    const float2 *lev = me + lvl_off3(l) * NC;
    for (int cs = 0; cs < 8; ++cs)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    // delta = target - source, in box widths
                    const int ex = (c & 1) - (cs & 1) - 2 * dx;
                    const int ey = ((c >> 1) & 1) - ((cs >> 1) & 1) - 2 * dy;
                    const int ez = (c >> 2) - (cs >> 2) - 2 * dz;
                    if (ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1 && ez >= -1 && ez <= 1)
                        continue;  // near field
                    // source rows (the barrier also ends the previous offset's reads)
                    bool have = false;
                    if (tid < MG_ROWS) {
                        int sb = -1;
                        const int64_t pc = p0 + tid;
                        if (pc < np) {
                            const int qx = int(compact3(uint32_t(pc))) + dx,
                                      qy = int(compact3(uint32_t(pc) >> 1)) + dy,
                                      qz = int(compact3(uint32_t(pc) >> 2)) + dz;
                            if (qx >= 0 && qy >= 0 && qz >= 0 && qx < pside && qy < pside &&
                                qz < pside) {
                                const uint32_t b = morton3(uint32_t(qx), uint32_t(qy), uint32_t(qz)) *
                                                       8u + uint32_t(cs);
                                if (box_count3(start, L, l, b)) sb = int(b);
                            }
                        }
                        srow[tid] = sb;
                        have = sb >= 0;
                    }
                    if (!__syncthreads_or(have)) continue;
                    {
                        // every load of the rows in flight at once, then the
                        // k-major scatter (Re to row j, Im to row imr[j])
                        float2 v[NLOAD];
#pragma unroll
                        for (int u = 0; u < NLOAD; ++u) {
                            const int i = tid + u * MG_THREADS;
                            v[u] = make_float2(0.f, 0.f);
                            if (i < MG_ROWS * NC) {
                                const int sb = srow[i / NC];
                                if (sb >= 0) v[u] = lev[int64_t(sb) * NC + i % NC];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < NLOAD; ++u) {
                            const int i = tid + u * MG_THREADS;
                            if (i < MG_ROWS * NC) {
                                const int row = i / NC, j = i % NC;
                                xs[j * MG_XS + row] = v[u].x;
                                if (imr[j] >= 0) xs[imr[j] * MG_XS + row] = v[u].y;
                            }
                        }
                    }
                    const float *at = atab + size_t((ex + 3) + 7 * (ey + 3) + 49 * (ez + 3)) * NRP * NRP;
                    for (int k0 = 0; k0 < NRP; k0 += KT) {
                        __syncthreads();
#pragma unroll
                        for (int u = 0; u < (KT * NRP / 4 + MG_THREADS - 1) / MG_THREADS; ++u) {
                            const int i = tid + u * MG_THREADS;
                            if (i < KT * NRP / 4)
                                reinterpret_cast<float4 *>(as)[i] =
                                    __ldg(reinterpret_cast<const float4 *>(at + size_t(k0) * NRP) + i);
                        }
                        __syncthreads();
#pragma unroll 4
                        for (int kk = 0; kk < KT; ++kk) {
                            const float4 x4 = *reinterpret_cast<const float4 *>(
                                xs + (k0 + kk) * MG_XS + 4 * rg);
                            const float *ar = as + kk * NRP + g * CG;
#pragma unroll
                            for (int j4 = 0; j4 < CG; j4 += 4) {
                                const float4 a4 = *reinterpret_cast<const float4 *>(ar + j4);
                                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                                for (int t = 0; t < 4; ++t) {
                                    acc[0][j4 + t] = fmaf(x4.x, av[t], acc[0][j4 + t]);
                                    acc[1][j4 + t] = fmaf(x4.y, av[t], acc[1][j4 + t]);
                                    acc[2][j4 + t] = fmaf(x4.z, av[t], acc[2][j4 + t]);
                                    acc[3][j4 + t] = fmaf(x4.w, av[t], acc[3][j4 + t]);
                                }
                            }
                        }
                    }
                }
    float *lef = reinterpret_cast<float *>(le + lvl_off3(l) * NC);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t pc = p0 + 4 * rg + i;
        if (pc >= np) continue;
        const int64_t box = pc * 8 + c;
#pragma unroll
        for (int j = 0; j < CG; ++j) {
            const int r = g * CG + j;
            if (r >= NR) continue;
            const short2 mp = rmap[r];
            lef[(box * NC + mp.x) * 2 + (mp.y == 1)] = acc[i][j];
            if (mp.y == 2) lef[(box * NC + mp.x) * 2 + 1] = 0.f;  // Im of m = 0
        }
    }
}

// The same GEMMs with the operands of the next offset in flight: for p <= 8
// (a whole operator is one K chunk) the operator and the source rows of
// offset i + 1 are copied with cp.async (16-byte chunks; 8 when a box's
// coefficients are an odd number of float2; rows of empty or outside boxes
// zero-filled without a read) into the second operator buffer and a raw row
// buffer while offset i multiplies; then the raw rows are split into the
// k-major real layout.  Offsets whose 64 source rows are all empty skip
// their multiply.
__device__ __forceinline__ void cp_async_z(void *dst, const void *src, int bytes, bool pred) {
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    const int n = pred ? bytes : 0;
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n));
}

template <int P, int R>
constexpr size_t mgp_smem_bytes() {
    return size_t(mg_nrp(P) * (R + 4) + 2 * mg_nrp(P) * mg_nrp(P)) * sizeof(float) +
           size_t(R) * (P * (P + 1) / 2) * sizeof(float2);
}

// blocks of level l in an all-levels M2L launch of R-row blocks:
// ceil(8^(l-1) / R) x 8
__host__ __device__ __forceinline__ int64_t mg_blocks(int l, int R) {
    return ((int64_t(1) << (3 * (l - 1))) + R - 1) / R * 8;
}

// R target rows per block (R Morton-consecutive parent cells: 4 x 4 x 4 for
// 64, 8 x 4 x 4 for 128), R / 16 rows per thread.
template <int P, int R>
__global__ void __launch_bounds__(MG_THREADS) k3_m2l_pipe(int L, const uint32_t *__restrict__ start,
                                                        const float *__restrict__ atab,
                                                        const float2 *__restrict__ me,
                                                        float2 *__restrict__ le) {
    // this block's level: levels 2..L one after another in the grid
    int l = 2;
    int64_t bid = blockIdx.x;
    while (l < L && bid >= mg_blocks(l, R)) bid -= mg_blocks(l++, R);
    constexpr int NC = P * (P + 1) / 2, NR = P * P, NRP = mg_nrp(P), CG = NRP / 8;
    static_assert(NRP <= 64, "one K chunk per operator");
    constexpr int XS = R + 4, RT = R / 16;
    constexpr int BITS = R == 128 ? 7 : 6;              // Morton bits of the block's parents
    constexpr int NX = 1 << ((BITS + 2) / 3), NY = 1 << ((BITS + 1) / 3), NZ = 1 << (BITS / 3);
    constexpr int HX = NX + 2, HY = NY + 2, HZ = NZ + 2;
    static_assert(R == 64 || R == 128, "rows per block");
    constexpr int CB = (NC % 2 == 0) ? 16 : 8;          // copy chunk bytes of a row
    constexpr int RCH = NC * 8 / CB;                     // chunks per row
    extern __shared__ __align__(16) float mg_smem[];
    float *xs = mg_smem;                                 // [NRP][XS]
    float *as0 = xs + NRP * XS;                          // 2 x [NRP][NRP]
    float2 *raw = reinterpret_cast<float2 *>(as0 + 2 * NRP * NRP);  // [R][NC]
    __shared__ int srow[2][R];
    __shared__ short imr[NC];
    __shared__ unsigned char offs[216];                  // the class's offsets (cs, d)
    __shared__ int noff;
    // occupied boxes of the parent cells around the block's (one cell of
    // halo), 8 classes each: one bit per class
    __shared__ unsigned char hocc[HX * HY * HZ];
    const int tid = threadIdx.x, rg = tid >> 3, g = tid & 7;
    const int c = int(bid & 7);
    const int64_t np = int64_t(1) << (3 * (l - 1));
    const int64_t p0 = (bid >> 3) * R;
    const int pside = 1 << (l - 1);
    const int hx0 = int(compact3(uint32_t(p0))) - 1, hy0 = int(compact3(uint32_t(p0) >> 1)) - 1,
              hz0 = int(compact3(uint32_t(p0) >> 2)) - 1;
    for (int h = tid; h < HX * HY * HZ; h += MG_THREADS) {
        const int qx = hx0 + h % HX, qy = hy0 + (h / HX) % HY, qz = hz0 + h / (HX * HY);
        unsigned bits = 0;
        if (qx >= 0 && qy >= 0 && qz >= 0 && qx < pside && qy < pside && qz < pside) {
            const uint32_t pb = morton3(uint32_t(qx), uint32_t(qy), uint32_t(qz));
            for (int cs = 0; cs < 8; ++cs)
                if (box_count3(start, L, l, pb * 8u + uint32_t(cs))) bits |= 1u << cs;
        }
        hocc[h] = (unsigned char)bits;
    }
    __syncthreads();
    // a block whose target boxes (class c of its own parent cells) are all
    // empty writes nothing: an empty box's local expansion is never read
    {
        bool mine = false;
        for (int r = tid; r < R; r += MG_THREADS) {
            const int64_t pc = p0 + r;
            if (pc >= np) continue;
            const int qx = int(compact3(uint32_t(pc))), qy = int(compact3(uint32_t(pc) >> 1)),
                      qz = int(compact3(uint32_t(pc) >> 2));
            mine |= (hocc[(qx - hx0) + HX * ((qy - hy0) + HY * (qz - hz0))] >> c) & 1u;
        }
        if (!__syncthreads_or(mine)) return;
    }
    for (int i = tid; i < (NRP - NR) * XS; i += MG_THREADS) xs[NR * XS + i] = 0.f;
    for (int j = tid; j < NC; j += MG_THREADS) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= j) ++n;
        imr[j] = short(j == n * (n + 1) / 2 ? -1 : NC + j - n - 1);
    }
    if (tid == 0) {
        int k = 0;
        for (int o = 0; o < 216; ++o) {
            const int cs = o / 27, d = o % 27;
            const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
            const int ex = (c & 1) - (cs & 1) - 2 * dx, ey = ((c >> 1) & 1) - ((cs >> 1) & 1) - 2 * dy,
                      ez = (c >> 2) - (cs >> 2) - 2 * dz;
            if (ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1 && ez >= -1 && ez <= 1) continue;
            offs[k++] = (unsigned char)o;
        }
        noff = k;
    }
    __syncthreads();
    const float2 *lev = me + lvl_off3(l) * NC;
    // source box of target row `row` for offset entry o (-1: none), from the
    // halo occupancy (no global load)
    auto source = [&](int o, int row) {
        const int cs = o / 27, d = o % 27;
        const int64_t pc = p0 + row;
        if (pc >= np) return -1;
        const int qx = int(compact3(uint32_t(pc))) + d % 3 - 1,
                  qy = int(compact3(uint32_t(pc) >> 1)) + (d / 3) % 3 - 1,
                  qz = int(compact3(uint32_t(pc) >> 2)) + d / 9 - 1;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= pside || qy >= pside || qz >= pside) return -1;
        if (!((hocc[(qx - hx0) + HX * ((qy - hy0) + HY * (qz - hz0))] >> cs) & 1u)) return -1;
        return int(morton3(uint32_t(qx), uint32_t(qy), uint32_t(qz)) * 8u + uint32_t(cs));
    };
    auto slot_of = [&](int o) {
        const int cs = o / 27, d = o % 27;
        const int ex = (c & 1) - (cs & 1) - 2 * (d % 3 - 1),
                  ey = ((c >> 1) & 1) - ((cs >> 1) & 1) - 2 * ((d / 3) % 3 - 1),
                  ez = (c >> 2) - (cs >> 2) - 2 * (d / 9 - 1);
        return (ex + 3) + 7 * (ey + 3) + 49 * (ez + 3);
    };
    auto issue = [&](int i) {  // copies of offset i (srow[i & 1] ready)
        const int o = offs[i];
        const float *at = atab + size_t(slot_of(o)) * NRP * NRP;
        float *asb = as0 + (i & 1) * NRP * NRP;
        for (int q = tid; q < NRP * NRP / 4; q += MG_THREADS)
            cp_async_z(asb + 4 * q, at + 4 * q, 16, true);
        for (int q = tid; q < R * RCH; q += MG_THREADS) {
            const int row = q / RCH, ch = q - row * RCH;
            const int sb = srow[i & 1][row];
            const char *src = reinterpret_cast<const char *>(sb >= 0 ? lev + int64_t(sb) * NC : lev);
            cp_async_z(reinterpret_cast<char *>(raw + row * NC) + ch * CB, src + ch * CB, CB, sb >= 0);
        }
        cp_async_commit();
    };
    float acc[RT][CG];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[i][j] = 0.f;
    const int nof = noff;
    bool have = false;
    if (tid < R) {
        srow[0][tid] = source(offs[0], tid);
        have = srow[0][tid] >= 0;
    }
    bool cur_any = __syncthreads_or(have);
    issue(0);
    for (int i = 0; i < nof; ++i) {
        cp_async_wait_all();
        __syncthreads();
        // split the raw rows of offset i into the k-major real layout, and
        // find the source rows of offset i + 1
        for (int q = tid; q < R * NC; q += MG_THREADS) {
            const int row = q % R, j = q / R;
            const float2 v = raw[row * NC + j];
            xs[j * XS + row] = v.x;
            if (imr[j] >= 0) xs[imr[j] * XS + row] = v.y;
        }
        have = false;
        if (tid < R && i + 1 < nof) {
            srow[(i + 1) & 1][tid] = source(offs[i + 1], tid);
            have = srow[(i + 1) & 1][tid] >= 0;
        }
        const bool next_any = __syncthreads_or(have);
        if (i + 1 < nof) issue(i + 1);
        if (cur_any) {
            const float *asb = as0 + (i & 1) * NRP * NRP;
#pragma unroll 4
            for (int k = 0; k < NRP; ++k) {
                float xv[RT];
#pragma unroll
                for (int i4 = 0; i4 < RT; i4 += 4) {
                    const float4 x4 = *reinterpret_cast<const float4 *>(xs + k * XS + RT * rg + i4);
                    xv[i4] = x4.x;
                    xv[i4 + 1] = x4.y;
                    xv[i4 + 2] = x4.z;
                    xv[i4 + 3] = x4.w;
                }
                const float *ar = asb + k * NRP + g * CG;
#pragma unroll
                for (int j4 = 0; j4 < CG; j4 += 4) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(ar + j4);
                    const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int i = 0; i < RT; ++i)
                            acc[i][j4 + t] = fmaf(xv[i], av[t], acc[i][j4 + t]);
                }
            }
        }
        cur_any = next_any;
    }
    cp_async_wait_all();
    float *lef = reinterpret_cast<float *>(le + lvl_off3(l) * NC);
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int64_t pc = p0 + RT * rg + i;
        if (pc >= np) continue;
        const int64_t box = pc * 8 + c;
#pragma unroll
        for (int j = 0; j < CG; ++j) {
            const int r = g * CG + j;
            if (r >= NR) continue;
            // real index r: Re of coefficient r (r < NC), else Im of the
            // (r - NC)-th coefficient with m > 0
            if (r < NC) {
                lef[(box * NC + r) * 2] = acc[i][j];
                int n = 0;
                while ((n + 1) * (n + 2) / 2 <= r) ++n;
                if (r == n * (n + 1) / 2) lef[(box * NC + r) * 2 + 1] = 0.f;
            }
        }
    }
    // Im parts: thread columns r >= NC map back through imr (search)
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int64_t pc = p0 + RT * rg + i;
        if (pc >= np) continue;
        const int64_t box = pc * 8 + c;
#pragma unroll
        for (int j = 0; j < CG; ++j) {
            const int r = g * CG + j;
            if (r < NC || r >= NR) continue;
            for (int jj = 0; jj < NC; ++jj)
                if (imr[jj] == r) lef[(box * NC + jj) * 2 + 1] = acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// M2L of the mixed path on the 5th-generation tensor cores (p <= 8): the
// same real GEMMs as k3_m2l_pipe with TF32 inputs split into hi and lo
// parts, each rounded to TF32 (a_hi = a to nearest, a_lo = a - a_hi to
// nearest: a - a_hi - a_lo is within about 2^-23 |a|, near an FP32
// rounding; the products a_hi b_hi + a_lo b_hi + a_hi b_lo leave out
// a_lo b_lo, about 2^-24) and FP32 accumulation in tensor memory, spread
// over TC3_SETS accumulator sets that consecutive pairs take in turn, read
// out every TC3_FLUSH pairs and added in registers (round to nearest): a
// chain of MMA additions into one accumulator spans two pairs, 48 steps.  (With one set the potential of a 20k-charge test
// drifted 1.2e-5 from the FP64 path, past the mixed path's 1e-5 budget,
// whether the split truncated or rounded: the error grows with the length
// of the accumulation chain, some 4,500 MMA steps per output here.)  A CTA takes the 128
// Morton-consecutive parent cells of a pipelined-M2L block and two target
// classes c0, c0 + 1: M = 128 rows (TMEM lanes), 2 x NRP accumulator
// columns.  For each (source class cs, parent offset d) pair in a fixed
// order whose operator is not near for one of the two classes and whose
// sources are not all empty, the 128 source rows (the expansion of box
// (P + d) 8 + cs in the real basis, zero for an empty or outside box) are
// split into hi and lo images in shared memory, K-major without swizzle
// (core matrices of 8 rows x 16 bytes: element (m, k) at
// ((k / 4) 128 + m) 16 + (k mod 4) 4 bytes), the two classes' operator
// images (host-built in the same layout, B(n, k) = A_delta[k][n]) are copied
// beside them, and one thread issues the MMAs and commits them to an
// mbarrier that the next pair waits on (bounded) before it overwrites the
// images.  A wait that gives up sets PETFMM_ETIMEOUT and the CTA writes
// nothing.
// ---------------------------------------------------------------------------
constexpr int TC3_STAGERS = 256;  // two threads per row (and per TMEM lane)
constexpr int TC3_THREADS = TC3_STAGERS + 32;  // and a warp that copies and issues
constexpr int TC3_ROWS = 128;
constexpr int TC3_SETS = 4;       // accumulator sets
constexpr int TC3_FLUSH = 8;      // pairs between read-outs of the sets into registers

// coefficient index n (n + 1) / 2 + m of the t-th coefficient with m > 0
template <int P> __host__ __device__ constexpr int tc3_imcoef(int t) {
    int r = 0;
    for (int n = 1; n < P; ++n)
        for (int m = 1; m <= n; ++m) {
            if (r == t) return n * (n + 1) / 2 + m;
            ++r;
        }
    return 0;
}

// v rounded to TF32 (nearest, ties away), in FP32 format
__device__ __forceinline__ float tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// The tensor-core M2L's input (K) basis, coefficient by coefficient: Re of
// coefficient j, then Im of j if its m > 0 (zero padding to NRP), so that
// each half of K covers about half of a row's coefficients and each of the
// two threads staging a row loads about half of it.  The output (N) basis
// stays the one of the M2L matrices (Re of all, then Im of m > 0).
template <int P> struct Tc3Basis {
    int j[mg_nrp(P)];     // coefficient, -1 for padding
    int part[mg_nrp(P)];  // 0 Re, 1 Im
    __host__ __device__ constexpr Tc3Basis() : j(), part() {
        int k = 0;
        for (int n = 0; n < P; ++n)
            for (int m = 0; m <= n; ++m) {
                const int jj = n * (n + 1) / 2 + m;
                j[k] = jj;
                part[k++] = 0;
                if (m > 0) {
                    j[k] = jj;
                    part[k++] = 1;
                }
            }
        for (; k < mg_nrp(P); ++k) {
            j[k] = -1;
            part[k] = 0;
        }
    }
    // the coefficients K half h reads: [lo, hi]
    __host__ __device__ constexpr int jlo(int h) const {
        int r = 1 << 30;
        for (int k = h * (mg_nrp(P) / 2); k < (h + 1) * (mg_nrp(P) / 2); ++k)
            if (j[k] >= 0 && j[k] < r) r = j[k];
        return r == (1 << 30) ? 0 : r;
    }
    __host__ __device__ constexpr int jhi(int h) const {
        int r = -1;
        for (int k = h * (mg_nrp(P) / 2); k < (h + 1) * (mg_nrp(P) / 2); ++k)
            if (j[k] > r) r = j[k];
        return r;
    }
};

// Coefficients a K half reads, and the most either half reads.
template <int P> __host__ __device__ constexpr int tc3_half_j0(int h) { return Tc3Basis<P>{}.jlo(h); }
template <int P> __host__ __device__ constexpr int tc3_half_nw(int h) {
    return Tc3Basis<P>{}.jhi(h) - Tc3Basis<P>{}.jlo(h) + 1;
}
template <int P> __host__ __device__ constexpr int tc3_nw() {
    return tc3_half_nw<P>(0) > tc3_half_nw<P>(1) ? tc3_half_nw<P>(0) : tc3_half_nw<P>(1);
}

// Registers for a half row: from coefficient j0 rounded down to even (so
// that rows with an even coefficient count load 16-byte pieces), one spare.
template <int P> __host__ __device__ constexpr int tc3_nwr() { return tc3_nw<P>() + 2; }

// One K half H of a row of A in the input basis, hi and lo, into the K-major
// images, from the coefficients (j0(H) rounded down to even) .. of the row
// held in w.
template <int P, int H>
__device__ __forceinline__ void tc3_write_half(const float2 (&w)[tc3_nwr<P>()], float *ahi, float *alo,
                                               int row) {
    constexpr int NRP = mg_nrp(P), KH = NRP / 2;
    constexpr Tc3Basis<P> bas{};
    constexpr int J0 = tc3_half_j0<P>(H) & ~1;
#pragma unroll
    for (int g = 0; g < KH / 4; ++g) {
        float v4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = H * KH + 4 * g + e;
            const int jj = bas.j[k];
            v4[e] = jj < 0 ? 0.f : (bas.part[k] ? w[jj - J0].y : w[jj - J0].x);
        }
        float4 h4, l4;
        h4.x = tf32_rna(v4[0]);
        h4.y = tf32_rna(v4[1]);
        h4.z = tf32_rna(v4[2]);
        h4.w = tf32_rna(v4[3]);
        l4 = make_float4(tf32_rna(v4[0] - h4.x), tf32_rna(v4[1] - h4.y), tf32_rna(v4[2] - h4.z),
                         tf32_rna(v4[3] - h4.w));
        const int kg = H * (KH / 4) + g;
        reinterpret_cast<float4 *>(ahi)[kg * TC3_ROWS + row] = h4;
        reinterpret_cast<float4 *>(alo)[kg * TC3_ROWS + row] = l4;
    }
}

template <int P> constexpr size_t tc3_smem_bytes() {
    // one A buffer of hi and lo (128 x NRP each), then four slots of a
    // class's B hi and lo (NRP x NRP each)
    return size_t(2 * TC3_ROWS * mg_nrp(P) + 8 * mg_nrp(P) * mg_nrp(P)) * sizeof(float);
}

// blocks of level l in the all-levels launch: 128 parent cells x 4 class pairs
__host__ __device__ __forceinline__ int64_t tc3_blocks(int l) {
    return ((int64_t(1) << (3 * (l - 1))) + TC3_ROWS - 1) / TC3_ROWS * 4;
}

template <int P>
__global__ void __launch_bounds__(TC3_THREADS, 1) k3_m2l_tc(int L, const uint32_t *__restrict__ start,
                                                          const float *__restrict__ bimg,
                                                          const float2 *__restrict__ me,
                                                          float2 *__restrict__ le,
                                                          long long spin_limit, int *status) {
    constexpr int NC = P * (P + 1) / 2, NR = P * P, NRP = mg_nrp(P), KG = NRP / 4;
    static_assert(NRP <= 64 && NRP % 16 == 0, "tensor-core M2L orders");
    constexpr int HX = 10, HY = 6, HZ = 6;  // the block's 8 x 4 x 4 parent cells and one of halo
    constexpr int AIMG = TC3_ROWS * NRP;    // floats of one A image (hi or lo)
    constexpr int BIMG = 2 * NRP * NRP;     // floats of one class's B images (hi, lo)
    constexpr int NSLOT = 4;                // B slots: step s = 2 pair + class uses slot s mod 4
    extern __shared__ __align__(1024) float tsm[];
    float *ahi = tsm, *alo = ahi + AIMG;    // [KG][128][4] each
    float *bsm = alo + AIMG;                // NSLOT x [hi, lo][KG][NRP][4]
    __shared__ unsigned char hocc[HX * HY * HZ];
    __shared__ unsigned char plist[216];    // the pairs that run: offset entries o
    __shared__ uint32_t pmask[7];           // offsets o with an occupied source row
    __shared__ int npl;
    __shared__ __align__(8) uint64_t mbar[NSLOT], bbar[NSLOT];  // per slot: MMAs done, B landed
    __shared__ uint32_t tslot;
    __shared__ uint32_t set_used;  // bit 2 set + class: that accumulator was written
    int l = 2;
    int64_t bid = blockIdx.x;
    while (l < L && bid >= tc3_blocks(l)) bid -= tc3_blocks(l++);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC3_ROWS - 1), half = (tid / TC3_ROWS) & 1;  // two stagers per row
    const bool stager = tid < TC3_STAGERS;
    const int c0 = 2 * int(bid & 3);
    const int64_t np = int64_t(1) << (3 * (l - 1));
    const int64_t p0 = (bid >> 2) * TC3_ROWS;
    const int pside = 1 << (l - 1);
    const int hx0 = int(compact3(uint32_t(p0))) - 1, hy0 = int(compact3(uint32_t(p0) >> 1)) - 1,
              hz0 = int(compact3(uint32_t(p0) >> 2)) - 1;
    if (tid < 7) pmask[tid] = 0;
    for (int h = tid; h < HX * HY * HZ; h += TC3_THREADS) {
        const int qx = hx0 + h % HX, qy = hy0 + (h / HX) % HY, qz = hz0 + h / (HX * HY);
        unsigned bits = 0;
        if (qx >= 0 && qy >= 0 && qz >= 0 && qx < pside && qy < pside && qz < pside) {
            const uint32_t pb = morton3(uint32_t(qx), uint32_t(qy), uint32_t(qz));
            for (int cs = 0; cs < 8; ++cs)
                if (box_count3(start, L, l, pb * 8u + uint32_t(cs))) bits |= 1u << cs;
        }
        hocc[h] = (unsigned char)bits;
    }
    __syncthreads();
    // this thread's row: parent cell p0 + row, its halo position
    const int64_t pc = p0 + row;
    const bool row_ok = pc < np;
    const int rx = int(compact3(uint32_t(pc))), ry = int(compact3(uint32_t(pc) >> 1)),
              rz = int(compact3(uint32_t(pc) >> 2));
    const unsigned own = row_ok ? hocc[(rx - hx0) + HX * ((ry - hy0) + HY * (rz - hz0))] : 0u;
    // nothing to do if the block's targets of both classes are empty
    if (!__syncthreads_or(int((own >> c0) & 3u))) return;
    // the row's source box for offset entry o (-1: empty or outside)
    auto source = [&](int o) {
        if (!row_ok) return -1;
        const int cs = o / 27, dd = o % 27;
        const int qx = rx + dd % 3 - 1, qy = ry + (dd / 3) % 3 - 1, qz = rz + dd / 9 - 1;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= pside || qy >= pside || qz >= pside) return -1;
        if (!((hocc[(qx - hx0) + HX * ((qy - hy0) + HY * (qz - hz0))] >> cs) & 1u)) return -1;
        return int(morton3(uint32_t(qx), uint32_t(qy), uint32_t(qz)) * 8u + uint32_t(cs));
    };
    // class cc's operator slot for offset entry o, or -1 where it is near
    auto op_slot = [&](int o, int cc) {
        const int c = c0 + cc, cs = o / 27, dd = o % 27;
        const int ex = (c & 1) - (cs & 1) - 2 * (dd % 3 - 1),
                  ey = ((c >> 1) & 1) - ((cs >> 1) & 1) - 2 * ((dd / 3) % 3 - 1),
                  ez = (c >> 2) - (cs >> 2) - 2 * (dd / 9 - 1);
        if (ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1 && ez >= -1 && ez <= 1) return -1;
        return (ex + 3) + 7 * (ey + 3) + 49 * (ez + 3);
    };
    // the pairs that run: an operator for one of the two classes, a source row
    if (stager && half == 0)
        for (int o = 0; o < 216; ++o)
            if (source(o) >= 0) atomicOr(&pmask[o >> 5], 1u << (o & 31));
    __syncthreads();
    if (tid == 0) {
        int k = 0;
        for (int o = 0; o < 216; ++o)
            if (((pmask[o >> 5] >> (o & 31)) & 1u) && (op_slot(o, 0) >= 0 || op_slot(o, 1) >= 0))
                plist[k++] = (unsigned char)o;
        npl = k;
        for (int b = 0; b < NSLOT; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bbar[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        set_used = 0;
    }
    constexpr uint32_t NCOLS = TC3_SETS * 2 * NRP;  // 256 or 512: a power of two
    static_assert(NCOLS <= 512, "TMEM columns");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tslot)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    const int n_pairs = npl;
    // kind::tf32: D F32 (bit 4), A and B TF32 (bits 7, 10), both K-major,
    // N / 8 at bit 17, M / 16 at bit 24
    constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NRP >> 3) << 17) |
                               (uint32_t(TC3_ROWS >> 4) << 24);
    constexpr uint32_t LBO_A = TC3_ROWS * 16, SBO_A = 128, LBO_B = NRP * 16, SBO_B = 128;
    const float2 *lev = me + lvl_off3(l) * NC;
    // Pipeline over the pairs i = 0 .. n_pairs - 1, each two steps s = 2 i +
    // class: ORCH (warp 8, one thread) copies the operator images of pair
    // i + 1 into slots (2 i + 2 + class) mod 4 while pair i multiplies; the
    // stagers hold pair i + 1's source rows in registers, loaded while pair
    // i multiplies, and write them into the single A buffer once ORCH has
    // seen pair i's MMAs done (barrier 1), then ORCH issues pair i + 1's
    // MMAs (barrier 2).  Every step commits once to its slot's mbar (also a
    // near class with no MMA), so mbar[s mod 4] phase s / 4 is "step s done".
    constexpr int ORCH = TC3_STAGERS;
    bool ok = true;
    uint32_t used = 0;        // ORCH: accumulators written
    int ncopy[NSLOT] = {0, 0, 0, 0};  // ORCH: copies into each slot
    int committed = 0;                // ORCH: steps committed
    auto wait_step = [&](int st) {  // ORCH: step st's MMAs done
        if (ok && st >= 0)
            ok = mbar_wait(smem_addr(&mbar[st % NSLOT]), uint32_t(st / NSLOT) & 1u, spin_limit);
    };
    auto copy_pair = [&](int i) {  // ORCH: pair i's images into slots (2 i + class) mod 4
        const int o = plist[i];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int os = op_slot(o, cc);
            const int sl = (2 * i + cc) % NSLOT;
            if (os < 0 || !ok) continue;
            const uint32_t bb = smem_addr(&bbar[sl]);
            mbar_arrive_expect_tx(bb, uint32_t(BIMG * 4));
            bulk_g2s(smem_addr(bsm + sl * BIMG), bimg + size_t(os) * BIMG, uint32_t(BIMG * 4), bb);
            ++ncopy[sl];
        }
    };
    // rows of pair 0 in registers; the images of pair 0 on their way
    // this stager's half of the next pair's row, in registers, from its
    // first coefficient rounded down to even
    constexpr int NWR = tc3_nwr<P>();
    const int j0 = (half ? tc3_half_j0<P>(1) : tc3_half_j0<P>(0)) & ~1;
    const int jend = (half ? tc3_half_j0<P>(1) + tc3_half_nw<P>(1) : tc3_half_j0<P>(0) + tc3_half_nw<P>(0));
    const int nw = jend - j0;  // coefficients wanted, <= NWR
    float2 w[NWR];
    auto load_row = [&](int i) {
        const int sb = (stager && i < n_pairs) ? source(plist[i]) : -1;
        const float2 *src = lev + int64_t(sb < 0 ? 0 : sb) * NC + j0;
        if constexpr (NC % 2 == 0) {
            // 16-byte pieces: the row starts 16-byte aligned and j0 is even
#pragma unroll
            for (int t = 0; t < NWR / 2; ++t) {
                float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (sb >= 0 && 2 * t < nw && j0 + 2 * t + 1 < NC)
                    q4 = reinterpret_cast<const float4 *>(src)[t];
                else if (sb >= 0 && 2 * t < nw)
                    q4 = make_float4(src[2 * t].x, src[2 * t].y, 0.f, 0.f);
                w[2 * t] = make_float2(q4.x, q4.y);
                w[2 * t + 1] = make_float2(q4.z, q4.w);
            }
        } else {
#pragma unroll
            for (int t = 0; t < NWR; ++t) w[t] = (sb >= 0 && t < nw) ? src[t] : make_float2(0.f, 0.f);
        }
    };
    // the stager's class, its row's sums so far (registers, FP32 round to
    // nearest): every TC3_FLUSH pairs the accumulator sets are read out of
    // TMEM, added here, and the next pairs start the sets afresh
    const int my_cc = half;
    float acc[NRP];
#pragma unroll
    for (int k = 0; k < NRP; ++k) acc[k] = 0.f;
    load_row(0);
    if (tid == ORCH && n_pairs > 0) copy_pair(0);
    for (int i = 0; i < n_pairs && ok; ++i) {
        // barrier 1: the A buffer is free (pair i - 1's MMAs done)
        if (tid == ORCH) wait_step(2 * i - 1);
        ok = __syncthreads_and(int(tid != ORCH || ok)) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (stager) {
            // A: the row in the input basis, each of the two stagers of a row
            // writing its half of the K groups
            if (half == 0)
                tc3_write_half<P, 0>(w, ahi, alo, row);
            else
                tc3_write_half<P, 1>(w, ahi, alo, row);
            asm volatile("fence.proxy.async.shared::cta;");
        } else if (tid == ORCH && i + 1 < n_pairs) {
            // pair i + 1's images: its slots last held steps 2 i - 2 and
            // 2 i - 1, done (waited above)
            copy_pair(i + 1);
        }
        // barrier 2: A(i) written
        __syncthreads();
        if (tid == ORCH && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t dah = mma_desc(smem_addr(ahi), LBO_A, SBO_A);
            const uint64_t dal = mma_desc(smem_addr(alo), LBO_A, SBO_A);
            constexpr uint64_t sa = (2 * LBO_A) >> 4, sbk = (2 * LBO_B) >> 4;
            const int set = i % TC3_SETS;
            const int o = plist[i];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int sl = (2 * i + cc) % NSLOT;
                if (op_slot(o, cc) >= 0 && ok) {
                    ok = mbar_wait(smem_addr(&bbar[sl]), uint32_t(ncopy[sl] - 1) & 1u, spin_limit);
                    if (ok) {
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t bh = smem_addr(bsm + sl * BIMG);
                        const uint64_t dbh = mma_desc(bh, LBO_B, SBO_B);
                        const uint64_t dbl = mma_desc(bh + uint32_t(NRP * NRP * 4), LBO_B, SBO_B);
                        const uint32_t dt = tbase + uint32_t((2 * set + cc) * NRP);
                        const uint32_t bit = 1u << (2 * set + cc);
                        const bool was = (used & bit) != 0;
#pragma unroll
                        for (int ks = 0; ks < NRP / 8; ++ks) {
                            mma_tf32(dt, dah + ks * sa, dbh + ks * sbk, idesc,
                                     (was || ks > 0) ? 1u : 0u);
                            mma_tf32(dt, dal + ks * sa, dbh + ks * sbk, idesc, 1u);
                            mma_tf32(dt, dah + ks * sa, dbl + ks * sbk, idesc, 1u);
                        }
                        used |= bit;
                    }
                }
                // one commit per step (also with no MMA)
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&mbar[sl])));
                ++committed;
            }
        }
        // the stagers load pair i + 1's rows while pair i multiplies
        load_row(i + 1);
        if ((i + 1) % TC3_FLUSH == 0 || i + 1 == n_pairs) {
            // flush: every MMA so far done, the sets added into registers
            if (tid == ORCH) {
                wait_step(2 * i + 1);
                set_used = used;
            }
            ok = __syncthreads_and(int(tid != ORCH || ok)) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (stager) {
                const uint32_t su = set_used;
                for (int set = 0; set < TC3_SETS; ++set) {  // the sets in order
                    if (!((su >> (2 * set + my_cc)) & 1u)) continue;  // uniform in the warp
                    const uint32_t taddr = tbase + (uint32_t((warp & 3) * 32) << 16) +
                                           uint32_t((2 * set + my_cc) * NRP);
#pragma unroll
                    for (int q = 0; q < NRP / 16; ++q) {
                        float t16[16];
                        tmem_ld16(taddr + uint32_t(16 * q), t16);
#pragma unroll
                        for (int k = 0; k < 16; ++k) acc[16 * q + k] += t16[k];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (tid == ORCH) used = 0;  // the next MMAs overwrite the sets
        }
    }
    if (tid == ORCH) {
        wait_step(2 * n_pairs - 1);
        if (!ok) {
            set_status(status, ST_ETIMEOUT);
            // the copies and MMAs in flight finish before the memory goes
            // (bounded)
            for (int sl = 0; sl < NSLOT; ++sl)
                if (ncopy[sl] > 0) mbar_wait(smem_addr(&bbar[sl]), uint32_t(ncopy[sl] - 1) & 1u, 1LL << 26);
            if (committed > 0) {  // the last commit covers every earlier MMA
                const int st = committed - 1;
                mbar_wait(smem_addr(&mbar[st % NSLOT]), uint32_t(st / NSLOT) & 1u, 1LL << 26);
            }
        }
    }
    ok = __syncthreads_and(int(tid != ORCH || ok)) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && stager) {
        // warps 0-3 take class c0 (TMEM lanes 32 w ..), warps 4-7 class c0 + 1
        float *lef = reinterpret_cast<float *>(le + lvl_off3(l) * NC);
        const int c = c0 + my_cc;
        const float *v = acc;
        if (row_ok && ((own >> c) & 1u)) {
            float *dst = lef + (pc * 8 + c) * NC * 2;
#pragma unroll
            for (int j = 0; j < NC; ++j) dst[2 * j] = v[j];
            int t = 0;
#pragma unroll
            for (int n = 0; n < P; ++n)
#pragma unroll
                for (int m = 0; m <= n; ++m) {
                    const int j = n * (n + 1) / 2 + m;
                    dst[2 * j + 1] = m == 0 ? 0.f : v[NC + t];
                    t += m > 0 ? 1 : 0;
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS));
}

// ---------------------------------------------------------------------------
// L2L (child level l >= 3): L~'_j^s += 2^-(j+1) sum_{k,l} L~_{j+k}^{s+l}(parent)
// conj(R_k^l(e_c)).  A warp per child box.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(W3 * 32) k3_l2l(int l, int L, int p, const uint32_t *__restrict__ start,
                                                  const typename C3<T>::V *__restrict__ rtab,
                                                  typename C3<T>::V *__restrict__ le) {
    using V = typename C3<T>::V;
    const int lane = threadIdx.x & 31;
    const int64_t cb = int64_t(blockIdx.x) * W3 + (threadIdx.x >> 5);
    if (cb >= (int64_t(1) << (3 * l))) return;
    if (box_count3(start, L, l, uint32_t(cb)) == 0) return;
    const int nc = nc3(p);
    const V *lp = le + (lvl_off3(l - 1) + (cb >> 3)) * nc;
    const V *rt = rtab + int(cb & 7) * nc;
    V *dst = le + (lvl_off3(l) + cb) * nc;
    for (int j0 = lane; j0 < nc; j0 += 32) {
        int j = 0;
        while ((j + 1) * (j + 2) / 2 <= j0) ++j;
        const int s = j0 - j * (j + 1) / 2;
        V acc = mk<V>(T(0), T(0));
        for (int k = 0; j + k < p; ++k)
            for (int ll = -k; ll <= k; ++ll) {
                const int ss = s + ll;
                if (ss < -(j + k) || ss > j + k) continue;
                cmac_conj(acc, coef3(rt, k, ll), coef3(lp, j + k, ss));
            }
        const T sc = T(ldexp(1.0, -(j + 1)));
        V o = dst[j0];
        o.x += acc.x * sc;
        o.y += acc.y * sc;
        dst[j0] = o;
    }
}

// ---------------------------------------------------------------------------
// M2M and L2L of the mixed path for p <= 8 as real matrix-vector products:
// each of the eight child octants has a fixed real P^2 x P^2 operator in the
// real basis of the M2L matrices (the sums of k3_m2m / k3_l2l applied to the
// basis vectors on the host in FP64), staged in shared memory for a block.
// ---------------------------------------------------------------------------
constexpr int TT_MAXP = 8;  // operators of up to 64 x 64 in shared memory

// A warp per parent box of level l: ME = sum over occupied children c of
// A_c x_c, x_c the child's ME in the real basis; lanes over output rows.
template <int P>
__global__ void __launch_bounds__(W3 * 32) k3_m2m_real(int l, int L, const uint32_t *__restrict__ start,
                                                       const float *__restrict__ op,
                                                       const short2 *__restrict__ rmap,
                                                       float2 *__restrict__ me) {
    constexpr int NC = P * (P + 1) / 2, NR = P * P, RL = (NR + 31) / 32;
    __shared__ float sA[NR * NR];  // sA[k_in * NR + r_out]
    __shared__ float sx[W3][NR];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b = int64_t(blockIdx.x) * W3 + wid;
    const bool act = b < (int64_t(1) << (3 * l)) && box_count3(start, L, l, uint32_t(b)) != 0;
    short2 rm[RL];
    float acc[RL];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const int r = lane + 32 * i;
        rm[i] = r < NR ? rmap[r] : make_short2(0, 0);
        acc[i] = 0.f;
    }
    for (int c = 0; c < 8; ++c) {
        __syncthreads();  // the previous operator is no longer read
        for (int t = threadIdx.x; t < NR * NR; t += W3 * 32) sA[t] = op[size_t(c) * NR * NR + t];
        const uint32_t cb = uint32_t(b) * 8u + uint32_t(c);
        const bool use = act && box_count3(start, L, l + 1, cb) != 0;
        if (use) {
            const float2 *mc = me + (lvl_off3(l + 1) + cb) * NC;
#pragma unroll
            for (int i = 0; i < RL; ++i) {
                const int r = lane + 32 * i;
                if (r < NR) {
                    const float2 v = mc[rm[i].x];
                    sx[wid][r] = rm[i].y == 1 ? v.y : v.x;
                }
            }
        }
        __syncthreads();
        if (use)
            for (int k = 0; k < NR; ++k) {
                const float xk = sx[wid][k];
#pragma unroll
                for (int i = 0; i < RL; ++i)
                    if (lane + 32 * i < NR) acc[i] = fmaf(sA[k * NR + lane + 32 * i], xk, acc[i]);
            }
    }
    if (!act) return;
    float *dst = reinterpret_cast<float *>(me + (lvl_off3(l) + b) * NC);
#pragma unroll
    for (int i = 0; i < RL; ++i)
        if (lane + 32 * i < NR) {
            dst[2 * rm[i].x + (rm[i].y == 1 ? 1 : 0)] = acc[i];
            if (rm[i].y == 2) dst[2 * rm[i].x + 1] = 0.f;  // Im of m = 0
        }
}

// L2L: a block per (child octant o, W3 parents of level l - 1), a warp per
// parent; its child of octant o adds B_o y to the local expansion that M2L
// wrote, y the parent's LE in the real basis.
template <int P>
__global__ void __launch_bounds__(W3 * 32) k3_l2l_real(int l, int L, const uint32_t *__restrict__ start,
                                                       const float *__restrict__ op,
                                                       const short2 *__restrict__ rmap,
                                                       float2 *__restrict__ le) {
    constexpr int NC = P * (P + 1) / 2, NR = P * P, RL = (NR + 31) / 32;
    __shared__ float sA[NR * NR];
    __shared__ float sx[W3][NR];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int o = int(blockIdx.x & 7u);
    const int64_t pb = int64_t(blockIdx.x >> 3) * W3 + wid;
    const int64_t cb = pb * 8 + o;
    const bool act = pb < (int64_t(1) << (3 * (l - 1))) && box_count3(start, L, l, uint32_t(cb)) != 0;
    for (int t = threadIdx.x; t < NR * NR; t += W3 * 32) sA[t] = op[size_t(o) * NR * NR + t];
    short2 rm[RL];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const int r = lane + 32 * i;
        rm[i] = r < NR ? rmap[r] : make_short2(0, 0);
        if (act && r < NR) {
            const float2 v = le[(lvl_off3(l - 1) + pb) * NC + rm[i].x];
            sx[wid][r] = rm[i].y == 1 ? v.y : v.x;
        }
    }
    __syncthreads();
    if (!act) return;
    float acc[RL];
#pragma unroll
    for (int i = 0; i < RL; ++i) acc[i] = 0.f;
    for (int k = 0; k < NR; ++k) {
        const float xk = sx[wid][k];
#pragma unroll
        for (int i = 0; i < RL; ++i)
            if (lane + 32 * i < NR) acc[i] = fmaf(sA[k * NR + lane + 32 * i], xk, acc[i]);
    }
    float *dst = reinterpret_cast<float *>(le + (lvl_off3(l) + cb) * NC);
#pragma unroll
    for (int i = 0; i < RL; ++i)
        if (lane + 32 * i < NR) dst[2 * rm[i].x + (rm[i].y == 1 ? 1 : 0)] += acc[i];
}

template <int P>
cudaError_t m2m_l2l_real_p(bool m2m, int l, int L, const uint32_t *start, const float *op,
                           const short2 *rmap, float2 *ex, cudaStream_t st) {
    if (m2m)
        k3_m2m_real<P><<<unsigned(((int64_t(1) << (3 * l)) + W3 - 1) / W3), W3 * 32, 0, st>>>(
            l, L, start, op, rmap, ex);
    else
        k3_l2l_real<P><<<unsigned(8 * (((int64_t(1) << (3 * (l - 1))) + W3 - 1) / W3)), W3 * 32, 0,
                         st>>>(l, L, start, op, rmap, ex);
    return cudaGetLastError();
}

// m2m: level l's parents from level l + 1; else level l's children from l - 1
cudaError_t launch_m2m_l2l_real(bool m2m, int p, int l, int L, const uint32_t *start,
                                const float *op, const short2 *rmap, float2 *ex, cudaStream_t st) {
    switch (p) {
#define TT_CASE(P) case P: return m2m_l2l_real_p<P>(m2m, l, L, start, op, rmap, ex, st);
        TT_CASE(1) TT_CASE(2) TT_CASE(3) TT_CASE(4) TT_CASE(5) TT_CASE(6) TT_CASE(7) TT_CASE(8)
#undef TT_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// L2P in leaf units: phi = sum L~_n^m conj(R_n^m(xi)) and g = grad_xi of it,
// column by column (m >= 0, weight 2 for m > 0: the m and -m terms of a real
// potential are conjugate), with
//   d/dz:  sum conj(R_n^m) L_{n+1}^m
//   d/dx:  sum conj(R_n^m) (L_{n+1}^{m+1} - L_{n+1}^{m-1}) / 2
//   d/dy:  sum conj(R_n^m) (-i / 2) (L_{n+1}^{m+1} + L_{n+1}^{m-1})
// (from d/dz R_n^m = R_{n-1}^m, (d/dx -+ i d/dy) R_n^m = +-R_{n-1}^{m-+1}).
// ---------------------------------------------------------------------------
template <typename T, typename V>
__device__ __forceinline__ void l2p3(const V *lc, int p, T x, T y, T z, T &phi, T &gx, T &gy,
                                     T &gz) {
    const T r2 = x * x + y * y + z * z;
    V rmm = mk<V>(T(1), T(0));
    for (int mu = 0; mu < p; ++mu) {
        if (mu > 0) {
            const T s = T(1) / T(2 * mu);
            rmm = mk<V>((rmm.x * x - rmm.y * y) * s, (rmm.x * y + rmm.y * x) * s);
        }
        const T wgt = mu == 0 ? T(1) : T(2);
        V r1 = rmm, r2v = mk<V>(T(0), T(0));
        for (int n = mu; n < p; ++n) {
            V rn = r1;
            if (n > mu) {
                const T inv = T(1) / T(n * n - mu * mu);
                const T c1 = T(2 * n - 1) * z;
                rn = mk<V>((c1 * r1.x - r2 * r2v.x) * inv, (c1 * r1.y - r2 * r2v.y) * inv);
                r2v = r1;
                r1 = rn;
            }
            const V a = lc[n * (n + 1) / 2 + mu];
            phi += wgt * (a.x * rn.x + a.y * rn.y);  // Re(a conj(rn))
            if (n + 1 < p) {
                const int o = (n + 1) * (n + 2) / 2;
                const V lz = lc[o + mu], lpv = lc[o + mu + 1];
                V lm;
                if (mu >= 1) {
                    lm = lc[o + mu - 1];
                } else {
                    const V l1 = lc[o + 1];
                    lm = mk<V>(-l1.x, l1.y);  // L^-1 = -conj(L^1)
                }
                // Re(conj(rn) A) = rn.x A.x + rn.y A.y
                const T axr = (lpv.x - lm.x) * T(0.5), axi = (lpv.y - lm.y) * T(0.5);
                const T ayr = (lpv.y + lm.y) * T(0.5), ayi = -(lpv.x + lm.x) * T(0.5);
                gx += wgt * (rn.x * axr + rn.y * axi);
                gy += wgt * (rn.x * ayr + rn.y * ayi);
                gz += wgt * (rn.x * lz.x + rn.y * lz.y);
            }
        }
    }
}

template <typename TOut>
__device__ __forceinline__ void store3(void *o, int64_t i, double v) {
    static_cast<TOut *>(o)[i] = TOut(v);
}

// ---------------------------------------------------------------------------
// The near field's work items: leaf b with n_b particles gives ceil(n_b / 32)
// items (b, first sorted rank of the chunk), in leaf order (a hot leaf's
// chunks go to consecutive warps, so they spread over the SMs).
__global__ void __launch_bounds__(256) k3_near_count(const uint32_t *__restrict__ start,
                                                     int64_t nleaf, uint32_t *__restrict__ cnt) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    cnt[b] = (start[b + 1] - start[b] + 31u) / 32u;
}
__global__ void __launch_bounds__(256) k3_near_emit(const uint32_t *__restrict__ start,
                                                    int64_t nleaf, const uint32_t *__restrict__ off,
                                                    const uint32_t *__restrict__ nitems,
                                                    int64_t cap, uint2 *__restrict__ items) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const uint32_t s0 = start[b], k = (start[b + 1] - s0 + 31u) / 32u;
    for (uint32_t c = 0; c < k; ++c) {
        const int64_t o = int64_t(off[b]) + c;
        if (o < cap && o < int64_t(*nitems)) items[o] = make_uint2(uint32_t(b), s0 + 32u * c);
    }
}

// 1/sqrt(x) for a normal x > 0: the PTX approximate reciprocal square root
// with denormal inputs flushed (none reach it: the pairs of two adjacent
// leaves have |d|^2 >= 2^-48).
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Near field + L2P, mixed path: a warp per work item (up to 32 targets of
// one leaf).  An item of k targets gives each target a group of rep lanes,
// rep the largest power of two with k rep <= 32, lane c of a group taking
// sources c, c + rep, ... of every range (a leaf's last, partly filled item
// keeps most lanes busy), the group's partial sums added by shuffles.
// Sources of the leaf and its neighbours in a fixed order (dz, dy, dx, then
// sorted rank), each read once per lane group (one address per group) in
// FP32 leaf units: d = xi_t - (xi_s + offset), 1/|d| from rsqrt, self and
// coincident pairs (|d| = 0, own leaf only: the records are capped below
// 0.5 - 2^-24) skipped.  Output in the caller's order.
template <typename TOut>
__global__ void __launch_bounds__(W3 * 32, 4) k3_near_mixed(int L, int p, double w,
                                                            const uint32_t *__restrict__ start,
                                                            const float4 *__restrict__ rec,
                                                            const float2 *__restrict__ le,
                                                            const uint32_t *__restrict__ perm,
                                                            const uint2 *__restrict__ items,
                                                            const uint32_t *__restrict__ nitems,
                                                            int64_t n, void *phi, void *ex,
                                                            void *ey, void *ez) {
    __shared__ float2 sle[W3][NC3_MAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t it = int64_t(blockIdx.x) * W3 + wid;
    if (it >= int64_t(*nitems)) return;
    // one item: the targets s0 .. s1 - 1 of leaf b
    const uint2 item = items[it];
    const int64_t b = item.x;
    if (!PF_IN(b, int64_t(1) << (3 * L))) return;
    const uint32_t s0 = item.y;
    const uint32_t s1 = min(start[b + 1], s0 + 32u);
    const int k = int(s1 - s0);  // 1..32 (an item holds at least one target)
    int lg = 0;
    while (lg < 5 && (k << (lg + 1)) <= 32) ++lg;
    const uint32_t rep = 1u << lg, c = uint32_t(lane) & (rep - 1u);
    const uint32_t i = s0 + uint32_t(lane >> lg);
    const bool live = i < s1;
    const int nc = nc3(p);
    const bool far = L >= 2;
    if (far)
        for (int t = lane; t < nc; t += 32) sle[wid][t] = le[(lvl_off3(L) + b) * nc + t];
    __syncwarp();
    const int ix = int(compact3(uint32_t(b))), iy = int(compact3(uint32_t(b) >> 1)),
              iz = int(compact3(uint32_t(b) >> 2));
    const int side = 1 << L;
    const float inv_w = float(1.0 / w), inv_w2 = float(1.0 / (w * w));
    const float4 tg = live ? rec[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float f = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int nx = ix + dx, ny = iy + dy, nz = iz + dz;
                if (nx < 0 || ny < 0 || nz < 0 || nx >= side || ny >= side || nz >= side)
                    continue;
                const uint32_t nb = morton3(uint32_t(nx), uint32_t(ny), uint32_t(nz));
                const uint32_t a = start[nb], e = start[nb + 1];
                const float ox = tg.x - float(dx), oy = tg.y - float(dy), oz = tg.z - float(dz);
                // |d| = 0 only within the target's own leaf (self, and
                // coincident particles, which bin to the same leaf); the
                // record cap keeps it from pairs across a leaf face
                auto pair = [&](const float4 sr, bool guard) {
                    const float ddx = ox - sr.x, ddy = oy - sr.y, ddz = oz - sr.z;
                    const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                    float ri = guard ? rsqrtf(r2) : rsqrt_normal(r2);
                    if (guard) ri = r2 > 0.f ? ri : 0.f;
                    const float qr = sr.w * ri;
                    const float qr3 = qr * ri * ri;
                    f += qr;
                    gx = fmaf(qr3, ddx, gx);
                    gy = fmaf(qr3, ddy, gy);
                    gz = fmaf(qr3, ddz, gz);
                };
                // full items (rep = 1) on the plain loop (the strided one
                // measured slower there), both unrolled eight / two deep
                const bool own = dx == 0 && dy == 0 && dz == 0;
                if (rep == 1u) {
                    if (own)
                        for (uint32_t j = a; j < e; ++j) pair(rec[j], true);
                    else {
#pragma unroll 8
                        for (uint32_t j = a; j < e; ++j) pair(rec[j], false);
                    }
                } else {
                    const float4 *sp = rec + a + c, *se = rec + e;
                    if (own)
                        for (; sp < se; sp += rep) pair(*sp, true);
                    else {
#pragma unroll 2
                        for (; sp < se; sp += rep) pair(*sp, false);
                    }
                }
            }
    for (uint32_t o = 1; o < rep; o <<= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, int(o));
        gx += __shfl_xor_sync(0xffffffffu, gx, int(o));
        gy += __shfl_xor_sync(0xffffffffu, gy, int(o));
        gz += __shfl_xor_sync(0xffffffffu, gz, int(o));
    }
    if (c == 0 && live) {
        float ff = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        if (far) l2p3<float, float2>(sle[wid], p, tg.x, tg.y, tg.z, ff, fx, fy, fz);
        const int64_t o = perm[i];
        if (PF_IN(o, n)) {
            store3<TOut>(phi, o, double((f + ff) * inv_w));
            store3<TOut>(ex, o, double((gx - fx) * inv_w2));
            store3<TOut>(ey, o, double((gy - fy) * inv_w2));
            store3<TOut>(ez, o, double((gz - fz) * inv_w2));
        }
    }
}

// The FP64 path: global coordinates, 1/r by division and sqrt.
template <typename TOut>
__global__ void __launch_bounds__(W3 * 32) k3_near_f64(int L, int p, Dom3 d,
                                                       const uint32_t *__restrict__ start,
                                                       const Dbl4 *__restrict__ xs,
                                                       const double2 *__restrict__ le,
                                                       const uint32_t *__restrict__ perm,
                                                       int64_t n, void *phi, void *ex, void *ey,
                                                       void *ez) {
    __shared__ double2 sle[W3][NC3_MAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b = int64_t(blockIdx.x) * W3 + wid;
    if (b >= (int64_t(1) << (3 * L))) return;
    const uint32_t s0 = start[b], s1 = start[b + 1];
    if (s0 == s1) return;
    const int nc = nc3(p);
    const bool far = L >= 2;
    if (far)
        for (int i = lane; i < nc; i += 32) sle[wid][i] = le[(lvl_off3(L) + b) * nc + i];
    __syncwarp();
    const int ix = int(compact3(uint32_t(b))), iy = int(compact3(uint32_t(b) >> 1)),
              iz = int(compact3(uint32_t(b) >> 2));
    const int side = 1 << L;
    const double w = d.width / double(side);
    const double cx = d.x0 + (ix + 0.5) * w, cy = d.y0 + (iy + 0.5) * w,
                 cz = d.z0 + (iz + 0.5) * w;
    for (uint32_t t0 = s0; t0 < s1; t0 += 32) {
        const uint32_t i = t0 + uint32_t(lane);
        const bool valid = i < s1;
        const Dbl4 tg = valid ? xs[i] : Dbl4{cx, cy, cz, 0.0};
        double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nx = ix + dx, ny = iy + dy, nz = iz + dz;
                    if (nx < 0 || ny < 0 || nz < 0 || nx >= side || ny >= side || nz >= side)
                        continue;
                    const uint32_t nb = morton3(uint32_t(nx), uint32_t(ny), uint32_t(nz));
                    const uint32_t a = start[nb], e = start[nb + 1];
                    for (uint32_t j = a; j < e; ++j) {
                        const Dbl4 s = xs[j];
                        const double ddx = tg.x - s.x, ddy = tg.y - s.y, ddz = tg.z - s.z;
                        const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        if (r2 == 0.0) continue;
                        const double ri = 1.0 / sqrt(r2);
                        const double qr = s.w * ri;
                        const double qr3 = qr * ri * ri;
                        f += qr;
                        gx += qr3 * ddx;
                        gy += qr3 * ddy;
                        gz += qr3 * ddz;
                    }
                }
        double ff = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        if (far)
            l2p3<double, double2>(sle[wid], p, (tg.x - cx) / w, (tg.y - cy) / w, (tg.z - cz) / w,
                                  ff, fx, fy, fz);
        if (valid) {
            const int64_t o = perm[i];
            if (!PF_IN(o, n)) continue;
            store3<TOut>(phi, o, f + ff / w);
            store3<TOut>(ex, o, gx - fx / (w * w));
            store3<TOut>(ey, o, gy - fy / (w * w));
            store3<TOut>(ez, o, gz - fz / (w * w));
        }
    }
}

// ---------------------------------------------------------------------------
// Host: operator tables in FP64 from the same recurrences.
// ---------------------------------------------------------------------------
using cd = std::complex<double>;

// R_n^m(v), n < P, m >= 0: out[n (n + 1) / 2 + m]
void host_rec_r(double x, double y, double z, int P, cd *out) {
    const double r2 = x * x + y * y + z * z;
    cd rmm(1.0, 0.0);
    for (int m = 0; m < P; ++m) {
        if (m > 0) rmm *= cd(x, y) / double(2 * m);
        cd r1 = rmm, r0(0.0, 0.0);
        for (int n = m; n < P; ++n) {
            cd rn = r1;
            if (n > m) {
                rn = (double(2 * n - 1) * z * r1 - r2 * r0) / double(n * n - m * m);
                r0 = r1;
                r1 = rn;
            }
            out[n * (n + 1) / 2 + m] = rn;
        }
    }
}

// I_n^m(v), n < P, m >= 0
void host_rec_i(double x, double y, double z, int P, cd *out) {
    const double r2 = x * x + y * y + z * z;
    cd imm(1.0 / std::sqrt(r2), 0.0);
    for (int m = 0; m < P; ++m) {
        if (m > 0) imm *= double(2 * m - 1) * cd(x, y) / r2;
        cd i1 = imm, i0(0.0, 0.0);
        for (int n = m; n < P; ++n) {
            cd in = i1;
            if (n > m) {
                in = (double(2 * n - 1) * z * i1 - double((n - 1) * (n - 1) - m * m) * i0) / r2;
                i0 = i1;
                i1 = in;
            }
            out[n * (n + 1) / 2 + m] = in;
        }
    }
}

// The mixed path's M2L operator for one offset delta in the real basis of a
// real potential's degree-< p coefficients (real index r < p (p + 1) / 2: Re
// of coefficient r = n (n + 1) / 2 + m; r >= p (p + 1) / 2: Im of the
// coefficients with m > 0, in order), from the M2L sum written per stored
// (n, m >= 0) input: L~_k^l gets alpha M~_n^m + beta conj(M~_n^m) with
// alpha = (-1)^k I_{n+k}^{m+l}(delta) and, for m > 0, beta =
// (-1)^(k+m) I_{n+k}^{l-m}(delta) (the -m term).  iv: I_j^s(delta), j < 2p - 1,
// s >= 0; a[k_in * p^2 + r_out] = d(output r_out) / d(input k_in), FP64.
void host_m2l_real(int p, const cd *iv, double *a) {
    const int nc = p * (p + 1) / 2, nr = p * p;
    std::vector<int> imidx(size_t(nc), -1);
    for (int n = 0, r = nc; n < p; ++n)
        for (int m = 1; m <= n; ++m) imidx[size_t(n * (n + 1) / 2 + m)] = r++;
    auto ival = [&](int j, int sg) {  // I_j^sg from the stored s >= 0
        if (sg >= 0) return iv[j * (j + 1) / 2 + sg];
        const cd v = std::conj(iv[j * (j + 1) / 2 - sg]);
        return (sg & 1) ? -v : v;
    };
    std::fill(a, a + size_t(nr) * nr, 0.0);
    for (int k = 0; k < p; ++k)
        for (int lo = 0; lo <= k; ++lo) {
            const int jo = k * (k + 1) / 2 + lo;
            for (int n = 0; n < p; ++n)
                for (int m = 0; m <= n; ++m) {
                    const int ji = n * (n + 1) / 2 + m;
                    const double sk = (k & 1) ? -1.0 : 1.0;
                    const cd al = sk * ival(n + k, m + lo);
                    const cd be =
                        m > 0 ? sk * ((m & 1) ? -1.0 : 1.0) * ival(n + k, lo - m) : cd(0.0, 0.0);
                    // input a (real part): L += (al + be) a; input b (imaginary
                    // part): L += i (al - be) b
                    const cd vr = al + be, vi = cd(0.0, 1.0) * (al - be);
                    a[size_t(ji) * nr + jo] = vr.real();
                    if (lo > 0) a[size_t(ji) * nr + imidx[size_t(jo)]] = vr.imag();
                    if (m > 0) {
                        a[size_t(imidx[size_t(ji)]) * nr + jo] = vi.real();
                        if (lo > 0) a[size_t(imidx[size_t(ji)]) * nr + imidx[size_t(jo)]] = vi.imag();
                    }
                }
        }
}

// v rounded to TF32 (10 mantissa bits; to nearest, ties away from zero)
float host_tf32_rna(float v) {
    uint32_t bits;
    std::memcpy(&bits, &v, 4);
    if ((bits & 0x7F800000u) != 0x7F800000u) bits += 0x1000u;  // finite: round the magnitude
    bits &= 0xFFFFE000u;
    float r;
    std::memcpy(&r, &bits, 4);
    return r;
}

// Coefficient (n, m) of a stored m >= 0 series, m < 0 by symmetry.
cd host_coef(const cd *a, int n, int m) {
    if (m >= 0) return a[n * (n + 1) / 2 + m];
    const cd v = std::conj(a[n * (n + 1) / 2 - m]);
    return (m & 1) ? -v : v;
}

// The M2M sum of k3_m2m for one child (rt: R_k^l of the child's offset):
// out_n^m = sum_k 2^-(n-k) sum_l conj(R_k^l) M_{n-k}^{m-l}.
void host_m2m_one(int p, const cd *rt, const cd *mc, cd *out) {
    for (int n = 0; n < p; ++n)
        for (int m = 0; m <= n; ++m) {
            cd s(0.0, 0.0);
            for (int k = 0; k <= n; ++k) {
                cd sk(0.0, 0.0);
                for (int ll = -k; ll <= k; ++ll) {
                    const int mm = m - ll;
                    if (mm < -(n - k) || mm > n - k) continue;
                    sk += std::conj(host_coef(rt, k, ll)) * host_coef(mc, n - k, mm);
                }
                s += sk * std::ldexp(1.0, -(n - k));
            }
            out[n * (n + 1) / 2 + m] = s;
        }
}

// The L2L sum of k3_l2l for one child: out_j^s = 2^-(j+1) sum_{k, l}
// conj(R_k^l) L_{j+k}^{s+l}.
void host_l2l_one(int p, const cd *rt, const cd *lp, cd *out) {
    for (int j = 0; j < p; ++j)
        for (int s = 0; s <= j; ++s) {
            cd acc(0.0, 0.0);
            for (int k = 0; j + k < p; ++k)
                for (int ll = -k; ll <= k; ++ll) {
                    const int ss = s + ll;
                    if (ss < -(j + k) || ss > j + k) continue;
                    acc += std::conj(host_coef(rt, k, ll)) * host_coef(lp, j + k, ss);
                }
            out[j * (j + 1) / 2 + s] = acc * std::ldexp(1.0, -(j + 1));
        }
}

// The real p^2 x p^2 matrix of a map of real-potential series (the basis
// of host_m2l_real), by applying it to each basis vector:
// a[k_in * p^2 + r_out], FP64.
template <typename F> void host_real_matrix(int p, F apply, double *a) {
    const int nc = p * (p + 1) / 2, nr = p * p;
    // real index -> (coefficient, imaginary part?)
    std::vector<int> jof(static_cast<size_t>(nr)), imof(static_cast<size_t>(nr), 0);
    std::vector<int> imidx(size_t(nc), -1);
    for (int n = 0, r = nc; n < p; ++n)
        for (int m = 0; m <= n; ++m) {
            const int j = n * (n + 1) / 2 + m;
            jof[size_t(j)] = j;
            if (m > 0) {
                imidx[size_t(j)] = r;
                jof[size_t(r)] = j;
                imof[size_t(r++)] = 1;
            }
        }
    std::vector<cd> in(static_cast<size_t>(nc)), out(static_cast<size_t>(nc));
    for (int k = 0; k < nr; ++k) {
        std::fill(in.begin(), in.end(), cd(0.0, 0.0));
        in[size_t(jof[size_t(k)])] = imof[size_t(k)] ? cd(0.0, 1.0) : cd(1.0, 0.0);
        apply(in.data(), out.data());
        for (int j = 0; j < nc; ++j) {
            a[size_t(k) * nr + j] = out[size_t(j)].real();
            if (imidx[size_t(j)] >= 0) a[size_t(k) * nr + imidx[size_t(j)]] = out[size_t(j)].imag();
        }
    }
}

// The real M2M (kind 0: child of the octant -> parent) or L2L (kind 1:
// parent -> child of the octant) operator of order p, FP64.
void host_shift_real(int p, int kind, int octant, double *a) {
    std::vector<cd> ro(static_cast<size_t>(p * (p + 1) / 2));
    host_rec_r((octant & 1) ? 0.25 : -0.25, (octant & 2) ? 0.25 : -0.25,
               (octant & 4) ? 0.25 : -0.25, p, ro.data());
    if (kind == 0)
        host_real_matrix(p, [&](const cd *in, cd *out) { host_m2m_one(p, ro.data(), in, out); }, a);
    else
        host_real_matrix(p, [&](const cd *in, cd *out) { host_l2l_one(p, ro.data(), in, out); }, a);
}

struct DevBuf3 {
    void *p = nullptr;
    size_t cap = 0;
};

int ensure3(DevBuf3 &b, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return PETFMM_OK;
    if (b.p) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return PETFMM_ECUDA;
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return PETFMM_ENOMEM;
    }
    b.cap = bytes;
    return PETFMM_OK;
}

}  // namespace

struct petfmm3d_ctx {
    petfmm_domain3d dom{};
    int L = 0, p = 0, precision = 0, dtype = 0;
    cudaStream_t stream = nullptr;
    DevBuf3 keysA, keysB, valsA, valsB, sortw, start, recu, rec, xs, me, le, status;
    DevBuf3 ncnt, noff, nscan, nitems;  // the mixed near field's work items
    DevBuf3 rtab32, itab32, rtab64, itab64, atab32, rmap;
    DevBuf3 m2m32, l2l32;  // p <= 8: the real M2M / L2L operators of the 8 octants
    DevBuf3 tcimg;  // p <= 8: TF32 hi / lo images of the M2L operators (tensor-core M2L)
    bool m2l_tc = true;  // PETFMM3D_OPT_M2L_TC
    bool timing = false, ev_recorded = false;
    cudaEvent_t ev[PETFMM3D_STAGE_COUNT + 1] = {};
    uint64_t launches = 0, evaluations = 0;
    int64_t last_n = 0;
    bool sorted_in_first = true;
};

namespace {

#define P3_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define P3_CUDA(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { cudaGetLastError(); \
    return e_ == cudaErrorMemoryAllocation ? PETFMM_ENOMEM : PETFMM_ECUDA; } } while (0)

int upload_tables(petfmm3d_ctx *c) {
    const int p = c->p, nc = nc3(p), nci = nci3(p);
    std::vector<cd> rt(size_t(8) * nc), it(size_t(NSLOT3) * nci, cd(0.0, 0.0));
    for (int o = 0; o < 8; ++o)
        host_rec_r((o & 1) ? 0.25 : -0.25, (o & 2) ? 0.25 : -0.25, (o & 4) ? 0.25 : -0.25, p,
                   rt.data() + size_t(o) * nc);
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
                host_rec_i(dx, dy, dz, 2 * p - 1,
                           it.data() + size_t((dx + 3) + 7 * (dy + 3) + 49 * (dz + 3)) * nci);
            }
    // the mixed path's M2L matrices: real index r < nc is Re of coefficient
    // r, r >= nc Im of the coefficients with m > 0 in order
    const int nr = p * p, nrp = mg_nrp(p);
    std::vector<short2> rm(static_cast<size_t>(nr));
    std::vector<int> imidx(size_t(nc), -1);
    for (int n = 0, r = nc; n < p; ++n)
        for (int m = 0; m <= n; ++m) {
            const int j = n * (n + 1) / 2 + m;
            rm[size_t(j)] = make_short2(short(j), short(m == 0 ? 2 : 0));
            if (m > 0) {
                imidx[size_t(j)] = r;
                rm[size_t(r++)] = make_short2(short(j), 1);
            }
        }
    std::vector<float> at(size_t(NSLOT3) * nrp * nrp, 0.f);
    std::vector<double> a64(size_t(nr) * nr);
    for (int slot = 0; slot < NSLOT3; ++slot) {
        const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
        if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
        host_m2l_real(p, it.data() + size_t(slot) * nci, a64.data());
        float *ap = at.data() + size_t(slot) * nrp * nrp;  // ap[k_in * nrp + r_out]
        for (int k = 0; k < nr; ++k)
            for (int r = 0; r < nr; ++r) ap[size_t(k) * nrp + r] = float(a64[size_t(k) * nr + r]);
    }
    if (p <= TT_MAXP) {
        // TF32 hi / lo images of every operator for the tensor-core M2L:
        // [slot][hi, lo][k / 4][n][k mod 4] = A[k][n] (zero padding)
        std::vector<float> img(size_t(NSLOT3) * 2 * nrp * nrp, 0.f);
        // input-basis position k -> row of the M2L matrix (Re of j: j; Im of
        // j: NC + its rank among the m > 0 coefficients)
        std::vector<int> tc3_kin(static_cast<size_t>(nr));
        for (int n = 0, k = 0, t = 0; n < p; ++n)
            for (int m = 0; m <= n; ++m) {
                const int j = n * (n + 1) / 2 + m;
                tc3_kin[size_t(k++)] = j;
                if (m > 0) tc3_kin[size_t(k++)] = nc + t++;
            }
        for (int slot = 0; slot < NSLOT3; ++slot) {
            const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
            if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
            host_m2l_real(p, it.data() + size_t(slot) * nci, a64.data());
            float *hi = img.data() + size_t(slot) * 2 * nrp * nrp, *lo = hi + size_t(nrp) * nrp;
            // K in the input basis of the tensor-core M2L (coefficient by
            // coefficient: Re, then Im if m > 0); N in the M2L matrices' basis
            for (int k = 0; k < nr; ++k) {
                const int kin = tc3_kin[size_t(k)];
                for (int n = 0; n < nr; ++n) {
                    const double a = a64[size_t(kin) * nr + n];
                    const float h = host_tf32_rna(float(a));
                    const size_t o = (size_t(k / 4) * nrp + n) * 4 + size_t(k % 4);
                    hi[o] = h;
                    lo[o] = host_tf32_rna(float(a - double(h)));
                }
            }
        }
        P3_TRY(ensure3(c->tcimg, img.size() * sizeof(float), c->stream));
        P3_CUDA(cudaMemcpy(c->tcimg.p, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    P3_TRY(ensure3(c->atab32, at.size() * sizeof(float), c->stream));
    P3_TRY(ensure3(c->rmap, rm.size() * sizeof(short2), c->stream));
    P3_CUDA(cudaMemcpy(c->atab32.p, at.data(), at.size() * sizeof(float), cudaMemcpyHostToDevice));
    P3_CUDA(cudaMemcpy(c->rmap.p, rm.data(), rm.size() * sizeof(short2), cudaMemcpyHostToDevice));
    std::vector<double2> r64(rt.size()), i64(it.size());
    std::vector<float2> r32(rt.size()), i32(it.size());
    for (size_t i = 0; i < rt.size(); ++i) {
        r64[i] = make_double2(rt[i].real(), rt[i].imag());
        r32[i] = make_float2(float(rt[i].real()), float(rt[i].imag()));
    }
    for (size_t i = 0; i < it.size(); ++i) {
        i64[i] = make_double2(it[i].real(), it[i].imag());
        i32[i] = make_float2(float(it[i].real()), float(it[i].imag()));
    }
    P3_TRY(ensure3(c->rtab64, r64.size() * sizeof(double2), c->stream));
    P3_TRY(ensure3(c->itab64, i64.size() * sizeof(double2), c->stream));
    P3_TRY(ensure3(c->rtab32, r32.size() * sizeof(float2), c->stream));
    P3_TRY(ensure3(c->itab32, i32.size() * sizeof(float2), c->stream));
    P3_CUDA(cudaMemcpy(c->rtab64.p, r64.data(), r64.size() * sizeof(double2), cudaMemcpyHostToDevice));
    P3_CUDA(cudaMemcpy(c->itab64.p, i64.data(), i64.size() * sizeof(double2), cudaMemcpyHostToDevice));
    P3_CUDA(cudaMemcpy(c->rtab32.p, r32.data(), r32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    P3_CUDA(cudaMemcpy(c->itab32.p, i32.data(), i32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if (p <= TT_MAXP) {
        // op[(octant * p^2 + k_in) * p^2 + r_out]
        std::vector<float> mm(size_t(8) * nr * nr), ll(size_t(8) * nr * nr);
        for (int o = 0; o < 8; ++o) {
            host_shift_real(p, 0, o, a64.data());
            for (size_t i = 0; i < size_t(nr) * nr; ++i) mm[size_t(o) * nr * nr + i] = float(a64[i]);
            host_shift_real(p, 1, o, a64.data());
            for (size_t i = 0; i < size_t(nr) * nr; ++i) ll[size_t(o) * nr * nr + i] = float(a64[i]);
        }
        P3_TRY(ensure3(c->m2m32, mm.size() * sizeof(float), c->stream));
        P3_TRY(ensure3(c->l2l32, ll.size() * sizeof(float), c->stream));
        P3_CUDA(cudaMemcpy(c->m2m32.p, mm.data(), mm.size() * sizeof(float), cudaMemcpyHostToDevice));
        P3_CUDA(cudaMemcpy(c->l2l32.p, ll.data(), ll.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return PETFMM_OK;
}

Dom3 make_dom3(const petfmm_domain3d &dom, int L) {
    Dom3 d{};
    d.x0 = dom.x0;
    d.y0 = dom.y0;
    d.z0 = dom.z0;
    d.width = dom.width;
    d.scale = std::ldexp(1.0, L) / dom.width;
    d.x0h = float(d.x0);
    d.x0l = float(d.x0 - double(d.x0h));
    d.y0h = float(d.y0);
    d.y0l = float(d.y0 - double(d.y0h));
    d.z0h = float(d.z0);
    d.z0l = float(d.z0 - double(d.z0h));
    d.sh = float(d.scale);
    d.sl = float(d.scale - double(d.sh));
    return d;
}

void mark3(petfmm3d_ctx *c, int s) {
    if (c->timing) cudaEventRecord(c->ev[s], c->stream);
}

unsigned grid_w(int64_t warps) { return unsigned((warps + W3 - 1) / W3); }

template <int P>
cudaError_t m2l_gemm_p(int l, int L, const uint32_t *start, const float *atab, const short2 *rmap,
                       const float2 *me, float2 *le, cudaStream_t st) {
    if constexpr (mg_nrp(P) <= 64) {
        constexpr int R = MG_PIPE_ROWS;
        constexpr size_t smem = mgp_smem_bytes<P, R>();
        static bool pattr = false;
        if (!pattr) {
            cudaError_t e = cudaFuncSetAttribute(k3_m2l_pipe<P, R>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(smem));
            if (e != cudaSuccess) return e;
            pattr = true;
        }
        if (l != L) return cudaSuccess;  // one launch covers levels 2..L
        int64_t grid = 0;
        for (int k = 2; k <= L; ++k) grid += mg_blocks(k, R);
        k3_m2l_pipe<P, R><<<unsigned(grid), MG_THREADS, smem, st>>>(L, start, atab, me, le);
        return cudaGetLastError();
    }
    const size_t smem = size_t(mg_nrp(P) * MG_XS + mg_kt(P) * mg_nrp(P)) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k3_m2l_gemm<P>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t np = int64_t(1) << (3 * (l - 1));
    const unsigned grid = unsigned((np + MG_ROWS - 1) / MG_ROWS * 8);
    k3_m2l_gemm<P><<<grid, MG_THREADS, smem, st>>>(l, L, start, atab, rmap, me, le);
    return cudaGetLastError();
}

template <int P>
cudaError_t m2l_tc_p(int L, const uint32_t *start, const float *bimg, const float2 *me, float2 *le,
                     int *status, cudaStream_t st) {
    if constexpr (mg_nrp(P) <= 64 && mg_nrp(P) % 16 == 0) {
        constexpr size_t smem = tc3_smem_bytes<P>();
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k3_m2l_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(smem));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        int64_t grid = 0;
        for (int k = 2; k <= L; ++k) grid += tc3_blocks(k);
        k3_m2l_tc<P><<<unsigned(grid), TC3_THREADS, smem, st>>>(L, start, bimg, me, le, 1LL << 26,
                                                                status);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// all levels 2..L in one launch, p <= 8
cudaError_t launch_m2l_tc3(int p, int L, const uint32_t *start, const float *bimg, const float2 *me,
                           float2 *le, int *status, cudaStream_t st) {
    switch (p) {
#define TC3_CASE(P) case P: return m2l_tc_p<P>(L, start, bimg, me, le, status, st);
        TC3_CASE(1) TC3_CASE(2) TC3_CASE(3) TC3_CASE(4) TC3_CASE(5) TC3_CASE(6) TC3_CASE(7)
        TC3_CASE(8)
#undef TC3_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_m2l_gemm(int p, int l, int L, const uint32_t *start, const float *atab,
                            const short2 *rmap, const float2 *me, float2 *le, cudaStream_t st) {
    switch (p) {
#define MG_CASE(P) case P: return m2l_gemm_p<P>(l, L, start, atab, rmap, me, le, st);
        MG_CASE(1) MG_CASE(2) MG_CASE(3) MG_CASE(4) MG_CASE(5) MG_CASE(6) MG_CASE(7) MG_CASE(8)
        MG_CASE(9) MG_CASE(10) MG_CASE(11) MG_CASE(12) MG_CASE(13) MG_CASE(14) MG_CASE(15)
        MG_CASE(16)
#undef MG_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int expansions3(petfmm3d_ctx *c, const uint32_t *start) {
    using V = typename C3<T>::V;
    const int L = c->L, p = c->p;
    cudaStream_t st = c->stream;
    V *me = static_cast<V *>(c->me.p), *le = static_cast<V *>(c->le.p);
    const bool f32 = sizeof(T) == 4;
    const V *rtab = static_cast<const V *>(f32 ? c->rtab32.p : c->rtab64.p);
    const V *itab = static_cast<const V *>(f32 ? c->itab32.p : c->itab64.p);
    const Dom3 d = make_dom3(c->dom, L);
    mark3(c, PETFMM3D_STAGE_P2M);
    if constexpr (sizeof(T) == 4) {
        if (p <= 8)
            P3_CUDA(launch_p2m_lanes(p, L, start, static_cast<const float4 *>(c->rec.p), me, st));
        else
            k3_p2m<T, float4><<<grid_w(int64_t(1) << (3 * L)), W3 * 32, 0, st>>>(
                L, p, d, start, static_cast<const float4 *>(c->rec.p), me);
    } else
        k3_p2m<T, Dbl4><<<grid_w(int64_t(1) << (3 * L)), W3 * 32, 0, st>>>(
            L, p, d, start, static_cast<const Dbl4 *>(c->xs.p), me);
    P3_CUDA(cudaGetLastError());
    c->launches++;
    mark3(c, PETFMM3D_STAGE_M2M);
    // mixed path with p <= 8: M2M and L2L as real matrix-vector products
    const bool real_tt = sizeof(T) == 4 && p <= TT_MAXP;
    for (int l = L - 1; l >= 2; --l) {
        if constexpr (sizeof(T) == 4) {
            if (real_tt) {
                P3_CUDA(launch_m2m_l2l_real(true, p, l, L, start, static_cast<const float *>(c->m2m32.p),
                                            static_cast<const short2 *>(c->rmap.p), me, st));
                c->launches++;
                continue;
            }
        }
        k3_m2m<T><<<grid_w(int64_t(1) << (3 * l)), W3 * 32, 0, st>>>(l, L, p, start, rtab, me);
        P3_CUDA(cudaGetLastError());
        c->launches++;
    }
    mark3(c, PETFMM3D_STAGE_M2L);
    // mixed path with p <= 8: one launch for all levels (launch_m2l_gemm
    // launches at l = L)
    const bool one = sizeof(T) == 4 && mg_nrp(p) <= 64;
    // mixed path, p <= 8, PETFMM3D_OPT_M2L_TC: all levels on the tensor cores
    const bool tc = sizeof(T) == 4 && c->m2l_tc && p <= TT_MAXP;
    if constexpr (sizeof(T) == 4) {
        if (tc) {
            P3_CUDA(launch_m2l_tc3(p, L, start, static_cast<const float *>(c->tcimg.p), me, le,
                                   static_cast<int *>(c->status.p), st));
            c->launches++;
        }
    }
    for (int l = tc ? L + 1 : one ? L : 2; l <= L; ++l) {
        if constexpr (sizeof(T) == 4) {
            P3_CUDA(launch_m2l_gemm(p, l, L, start, static_cast<const float *>(c->atab32.p),
                                    static_cast<const short2 *>(c->rmap.p), me, le, st));
        } else {
            k3_m2l<T><<<grid_w(int64_t(1) << (3 * l)), W3 * 32, 0, st>>>(l, L, p, start, itab,
                                                                          me, le);
        }
        P3_CUDA(cudaGetLastError());
        c->launches++;
    }
    mark3(c, PETFMM3D_STAGE_L2L);
    for (int l = 3; l <= L; ++l) {
        if constexpr (sizeof(T) == 4) {
            if (real_tt) {
                P3_CUDA(launch_m2m_l2l_real(false, p, l, L, start, static_cast<const float *>(c->l2l32.p),
                                            static_cast<const short2 *>(c->rmap.p), le, st));
                c->launches++;
                continue;
            }
        }
        k3_l2l<T><<<grid_w(int64_t(1) << (3 * l)), W3 * 32, 0, st>>>(l, L, p, start, rtab, le);
        P3_CUDA(cudaGetLastError());
        c->launches++;
    }
    return PETFMM_OK;
}

int evaluate3(petfmm3d_ctx *c, int64_t n, const void *x, const void *y, const void *z,
              const void *q, void *phi, void *ex, void *ey, void *ez) {
    cudaStream_t st = c->stream;
    const int L = c->L, p = c->p;
    const bool mixed = c->precision == PETFMM_MIXED, f32 = c->dtype == PETFMM_F32;
    P3_TRY(ensure3(c->status, 16, st));
    P3_CUDA(cudaMemsetAsync(c->status.p, 0, sizeof(int), st));
    c->last_n = n;
    c->ev_recorded = false;
    if (n == 0) return PETFMM_OK;
    const int64_t nleaf = int64_t(1) << (3 * L);
    const int64_t nbox = lvl_off3(L + 1);
    const size_t es = mixed ? sizeof(float2) : sizeof(double2);
    P3_TRY(ensure3(c->keysA, size_t(n) * 4, st));
    P3_TRY(ensure3(c->keysB, size_t(n) * 4, st));
    P3_TRY(ensure3(c->valsA, size_t(n) * 4, st));
    P3_TRY(ensure3(c->valsB, size_t(n) * 4, st));
    P3_TRY(ensure3(c->sortw, size_t(radix_scratch_words(n)) * 4, st));
    P3_TRY(ensure3(c->start, size_t(nleaf + 1) * 4, st));
    P3_TRY(ensure3(c->me, size_t(nbox) * nc3(p) * es, st));
    P3_TRY(ensure3(c->le, size_t(nbox) * nc3(p) * es, st));
    if (mixed) {
        P3_TRY(ensure3(c->recu, size_t(n) * sizeof(float4), st));
        P3_TRY(ensure3(c->rec, size_t(n) * sizeof(float4), st));
    } else {
        P3_TRY(ensure3(c->xs, size_t(n) * sizeof(Dbl4), st));
    }
    uint32_t *kA = static_cast<uint32_t *>(c->keysA.p), *kB = static_cast<uint32_t *>(c->keysB.p);
    uint32_t *vA = static_cast<uint32_t *>(c->valsA.p), *vB = static_cast<uint32_t *>(c->valsB.p);
    uint32_t *start = static_cast<uint32_t *>(c->start.p);
    int *status = static_cast<int *>(c->status.p);
    const Dom3 d = make_dom3(c->dom, L);
    const unsigned gp = unsigned((n + 255) / 256);
    float4 *recu = mixed ? static_cast<float4 *>(c->recu.p) : nullptr;

    mark3(c, PETFMM3D_STAGE_BIN);
    if (f32)
        k3_bin<float><<<gp, 256, 0, st>>>(n, static_cast<const float *>(x), static_cast<const float *>(y),
                                          static_cast<const float *>(z), static_cast<const float *>(q),
                                          d, L, kA, recu, status);
    else
        k3_bin<double><<<gp, 256, 0, st>>>(n, static_cast<const double *>(x), static_cast<const double *>(y),
                                           static_cast<const double *>(z), static_cast<const double *>(q),
                                           d, L, kA, recu, status);
    P3_CUDA(cudaGetLastError());
    c->launches++;
    mark3(c, PETFMM3D_STAGE_SORT);
    bool in_first = true;
    P3_CUDA(radix_sort(kA, vA, kB, vB, n, 3 * L, static_cast<uint32_t *>(c->sortw.p), &in_first, st,
                       &c->launches));
    c->sorted_in_first = in_first;
    const uint32_t *skeys = in_first ? kA : kB;
    const uint32_t *perm = in_first ? vA : vB;
    k3_leaf_start<<<unsigned((nleaf + 1 + 255) / 256), 256, 0, st>>>(skeys, n, nleaf, start);
    P3_CUDA(cudaGetLastError());
    c->launches++;
    mark3(c, PETFMM3D_STAGE_GATHER);
    if (mixed) {
        P3_CUDA(launch_gather_mixed(recu, perm, static_cast<float4 *>(c->rec.p), n, st, &c->launches));
    } else {
        Dbl4 *xs = static_cast<Dbl4 *>(c->xs.p);
        if (f32)
            k3_gather_f64<float><<<gp, 256, 0, st>>>(n, perm, static_cast<const float *>(x),
                                                     static_cast<const float *>(y),
                                                     static_cast<const float *>(z),
                                                     static_cast<const float *>(q), xs);
        else
            k3_gather_f64<double><<<gp, 256, 0, st>>>(n, perm, static_cast<const double *>(x),
                                                      static_cast<const double *>(y),
                                                      static_cast<const double *>(z),
                                                      static_cast<const double *>(q), xs);
        P3_CUDA(cudaGetLastError());
        c->launches++;
    }
    if (L >= 2) {
        if (mixed)
            P3_TRY(expansions3<float>(c, start));
        else
            P3_TRY(expansions3<double>(c, start));
    } else {
        for (int s = PETFMM3D_STAGE_P2M; s <= PETFMM3D_STAGE_L2L; ++s) mark3(c, s);
    }
    mark3(c, PETFMM3D_STAGE_NEAR);
    const unsigned gl = grid_w(nleaf);
    const double w = c->dom.width / double(int64_t(1) << L);
    if (mixed) {
        // work items: ceil(n_b / 32) per leaf, at most min(8^L, n) + n / 32
        const int64_t cap = std::min<int64_t>(nleaf, n) + n / 32 + 1;
        P3_TRY(ensure3(c->ncnt, size_t(nleaf) * 4, st));
        P3_TRY(ensure3(c->noff, size_t(nleaf) * 4 + 16, st));
        P3_TRY(ensure3(c->nscan, size_t(scan_scratch_words(nleaf)) * 4, st));
        P3_TRY(ensure3(c->nitems, size_t(cap) * sizeof(uint2), st));
        uint32_t *cnt = static_cast<uint32_t *>(c->ncnt.p), *off = static_cast<uint32_t *>(c->noff.p);
        uint32_t *nit = off + nleaf;  // the item count, after the offsets
        uint2 *items = static_cast<uint2 *>(c->nitems.p);
        const unsigned gb = unsigned((nleaf + 255) / 256);
        k3_near_count<<<gb, 256, 0, st>>>(start, nleaf, cnt);
        P3_CUDA(cudaGetLastError());
        P3_CUDA(exclusive_scan(cnt, off, nleaf, static_cast<uint32_t *>(c->nscan.p), nit, st,
                               &c->launches));
        k3_near_emit<<<gb, 256, 0, st>>>(start, nleaf, off, nit, cap, items);
        P3_CUDA(cudaGetLastError());
        c->launches += 2;
        const float4 *rec = static_cast<const float4 *>(c->rec.p);
        const float2 *le = static_cast<const float2 *>(c->le.p);
        const unsigned gi = grid_w(cap);
        if (f32)
            k3_near_mixed<float><<<gi, W3 * 32, 0, st>>>(L, p, w, start, rec, le, perm, items,
                                                         nit, n, phi, ex, ey, ez);
        else
            k3_near_mixed<double><<<gi, W3 * 32, 0, st>>>(L, p, w, start, rec, le, perm, items,
                                                          nit, n, phi, ex, ey, ez);
    } else {
        const Dbl4 *xs = static_cast<const Dbl4 *>(c->xs.p);
        const double2 *le = static_cast<const double2 *>(c->le.p);
        if (f32)
            k3_near_f64<float><<<gl, W3 * 32, 0, st>>>(L, p, d, start, xs, le, perm, n, phi, ex, ey, ez);
        else
            k3_near_f64<double><<<gl, W3 * 32, 0, st>>>(L, p, d, start, xs, le, perm, n, phi, ex, ey, ez);
    }
    P3_CUDA(cudaGetLastError());
    c->launches++;
    mark3(c, PETFMM3D_STAGE_COUNT);
    c->ev_recorded = c->timing;
    return PETFMM_OK;
}

}  // namespace

extern "C" {

int petfmm3d_create(const petfmm_domain3d *dom, int levels, int order, int precision, int dtype,
                    void *cuda_stream, petfmm3d_ctx **out) {
    if (!out) return PETFMM_EINVAL;
    *out = nullptr;
    if (!dom || !(dom->width > 0.0) || !std::isfinite(dom->width) || !std::isfinite(dom->x0) ||
        !std::isfinite(dom->y0) || !std::isfinite(dom->z0))
        return PETFMM_EINVAL;
    if (levels < 1 || levels > L3_MAX || order < 1 || order > P3_MAX) return PETFMM_EINVAL;
    if (precision != PETFMM_FP64 && precision != PETFMM_MIXED) return PETFMM_EINVAL;
    if (dtype != PETFMM_F64 && dtype != PETFMM_F32) return PETFMM_EINVAL;
    petfmm3d_ctx *c = new (std::nothrow) petfmm3d_ctx;
    if (!c) return PETFMM_ENOMEM;
    c->dom = *dom;
    c->L = levels;
    c->p = order;
    c->precision = precision;
    c->dtype = dtype;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    int rc = upload_tables(c);
    for (int i = 0; !rc && i <= PETFMM3D_STAGE_COUNT; ++i)
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) rc = PETFMM_ECUDA;
    if (rc) {
        cudaGetLastError();
        petfmm3d_destroy(c);
        return rc;
    }
    *out = c;
    return PETFMM_OK;
}

int petfmm3d_evaluate(petfmm3d_ctx *c, int64_t n, const void *x, const void *y, const void *z,
                      const void *q, void *phi, void *ex, void *ey, void *ez) {
    if (!c || n < 0 || n > int64_t(0xffffffffu) / 4) return PETFMM_EINVAL;
    if (n > 0 && (!x || !y || !z || !q || !phi || !ex || !ey || !ez)) return PETFMM_EINVAL;
    const int rc = evaluate3(c, n, x, y, z, q, phi, ex, ey, ez);
    if (!rc) c->evaluations++;
    return rc;
}

int petfmm3d_sync(petfmm3d_ctx *c) {
    if (!c) return PETFMM_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return PETFMM_ECUDA;
    }
    if (!c->status.p) return PETFMM_OK;
    int s = 0;
    if (cudaMemcpy(&s, c->status.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PETFMM_ECUDA;
    }
    return s;
}

int petfmm3d_set_option(petfmm3d_ctx *c, int option, int64_t value) {
    if (!c) return PETFMM_EINVAL;
    switch (option) {
        case PETFMM3D_OPT_TIMING: c->timing = value != 0; return PETFMM_OK;
        case PETFMM3D_OPT_M2L_TC:
            if (value != 0 && value != 1) return PETFMM_EINVAL;
            c->m2l_tc = value != 0;
            return PETFMM_OK;
        default: return PETFMM_EINVAL;
    }
}

int petfmm3d_stage_times(petfmm3d_ctx *c, float *ms, int cap) {
    if (!c || !ms || cap < 0) return PETFMM_EINVAL;
    if (!c->ev_recorded) return PETFMM_ENOTREADY;
    const int k = std::min(cap, int(PETFMM3D_STAGE_COUNT));
    for (int s = 0; s < k; ++s) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev[s], c->ev[s + 1]) != cudaSuccess) {
            cudaGetLastError();
            return PETFMM_ECUDA;
        }
        ms[s] = t;
    }
    return k;
}

int petfmm3d_debug_tree(petfmm3d_ctx *c, int64_t n, uint32_t *skeys, uint32_t *perm,
                        uint32_t *start) {
    if (!c || n != c->last_n || n <= 0 || !skeys || !perm || !start) return PETFMM_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PETFMM_ECUDA;
    const void *k = c->sorted_in_first ? c->keysA.p : c->keysB.p;
    const void *v = c->sorted_in_first ? c->valsA.p : c->valsB.p;
    const size_t nleaf = size_t(1) << (3 * c->L);
    if (cudaMemcpy(skeys, k, size_t(n) * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(perm, v, size_t(n) * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(start, c->start.p, (nleaf + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PETFMM_ECUDA;
    }
    return PETFMM_OK;
}

uint64_t petfmm3d_launches(const petfmm3d_ctx *c) { return c ? c->launches : 0; }

int petfmm3d_debug_m2l_operator(int order, int dx, int dy, int dz, double *out, int64_t cap) {
    if (order < 1 || order > P3_MAX || !out) return PETFMM_EINVAL;
    if (std::abs(dx) > 3 || std::abs(dy) > 3 || std::abs(dz) > 3 ||
        std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2)
        return PETFMM_EINVAL;
    const int64_t nr = int64_t(order) * order;
    if (cap < nr * nr) return PETFMM_EINVAL;
    std::vector<cd> iv(size_t(nci3(order)));
    host_rec_i(dx, dy, dz, 2 * order - 1, iv.data());
    host_m2l_real(order, iv.data(), out);
    return PETFMM_OK;
}

int petfmm3d_debug_shift_operator(int order, int kind, int octant, double *out, int64_t cap) {
    if (order < 1 || order > P3_MAX || !out) return PETFMM_EINVAL;
    if ((kind != PETFMM3D_SHIFT_M2M && kind != PETFMM3D_SHIFT_L2L) || octant < 0 || octant > 7)
        return PETFMM_EINVAL;
    const int64_t nr = int64_t(order) * order;
    if (cap < nr * nr) return PETFMM_EINVAL;
    host_shift_real(order, kind == PETFMM3D_SHIFT_M2M ? 0 : 1, octant, out);
    return PETFMM_OK;
}

int petfmm3d_destroy(petfmm3d_ctx *c) {
    if (!c) return PETFMM_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    DevBuf3 *bufs[] = {&c->ncnt, &c->noff, &c->nscan, &c->nitems,
                       &c->keysA, &c->keysB, &c->valsA, &c->valsB, &c->sortw, &c->start,
                       &c->recu,  &c->rec,   &c->xs,    &c->me,    &c->le,    &c->status,
                       &c->rtab32, &c->itab32, &c->rtab64, &c->itab64, &c->atab32, &c->rmap,
                       &c->m2m32, &c->l2l32, &c->tcimg};
    for (DevBuf3 *b : bufs)
        if (b->p) cudaFree(b->p);
    for (int i = 0; i <= PETFMM3D_STAGE_COUNT; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    cudaGetLastError();
    delete c;
    return PETFMM_OK;
}

}  // extern "C"
