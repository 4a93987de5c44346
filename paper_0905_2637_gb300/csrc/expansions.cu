// expansions.cu -- the upward and downward sweeps of Sec. 2.2 (Fig. 2):
// P2M, M2M, M2L over the interaction list, L2L.  SIMT kernels, templated on
// the real type (double for the FP64 path, float for the mixed path's
// non-tensor stages).
//
// Series (Cauchy kernel; the paper leaves the mathematics to Greengard-
// Rokhlin, Sec. 2.2).  With z = x + i y, the far field is
// w(z) = sum_j gamma_j / (z - z_j) and (u, v) = (Im w, Re w) / 2pi.  Rescaled
// coefficients, r = width of the box that owns the expansion:
//   P2M  a~_k = sum_j gamma_j zeta_j^k,       zeta_j = (z_j - z_c) / r
//   M2M  a~'_l = 2^-l sum_{k<=l} C(l,k) e^(l-k) a~_k,  e = (child - parent
//        centre) / r_child in {+-1/2 +- i/2}
//   M2L  c^_m = sum_k (-1)^(k+1) C(k+m,k) delta^-(k+m+1) a~_k,  delta = (source
//        - target centre) / r, one of 40 fixed offsets
//   L2L  c^'_n = sum_{m>=n} 2^-(m+1) C(m,n) e^(m-n) c^_m
//   L2P  w(z) = r^-1 sum_m c^_m zeta^m
// Costs (Sec. 5.2): P2M O(N_i p) per leaf, M2M and L2L O(p^2) per child,
// M2L O(p^2 n_IL) per box with n_IL <= 27.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "kernels.cuh"

namespace petfmm {

#define PF_LAUNCHED(n) do { if (launches) *launches += (n); } while (0)

// ----------------------------------------------------------------------------
// Interaction-list table.  For a target of child class c = (cx, cy) the
// sources are the children of the parent's 3x3 neighbourhood that are not
// within one box of the target: per axis dx in [-2, 3] if cx = 0 and [-3, 2]
// if cx = 1 (same for y), minus the 3x3 block around the target -- 27
// offsets.  Each offset maps to one of the 40 vectors of [-3, 3]^2 \ [-1, 1]^2.
// ----------------------------------------------------------------------------
__constant__ IlEntry c_il[4][27];

static int offset_op_index(int dx, int dy) { return m2l_op_index(dx, dy); }

static void il_offsets(int c, IlEntry *out) {
    const int cx = c & 1, cy = c >> 1;
    const int x_lo = cx ? -3 : -2, y_lo = cy ? -3 : -2;
    int n = 0;
    for (int dy = y_lo; dy <= y_lo + 5; ++dy)
        for (int dx = x_lo; dx <= x_lo + 5; ++dx) {
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            out[n].dx = int8_t(dx);
            out[n].dy = int8_t(dy);
            out[n].op = int8_t(offset_op_index(dx, dy));
            out[n].pad = 0;
            ++n;
        }
}

static bool g_il_uploaded = false;

static cudaError_t upload_il() {
    if (g_il_uploaded) return cudaSuccess;
    IlEntry h[4][27];
    for (int c = 0; c < 4; ++c) il_offsets(c, h[c]);
    cudaError_t e = cudaMemcpyToSymbol(c_il, h, sizeof(h));
    if (e == cudaSuccess) g_il_uploaded = true;
    return e;
}

int host_interaction_list(int level, int ix, int iy, int32_t *out) {
    if (level < 0 || level > MAX_L) return -1;
    const int nside = 1 << level;
    if (ix < 0 || iy < 0 || ix >= nside || iy >= nside) return -1;
    if (level < 2) return 0;
    IlEntry e[27];
    il_offsets((ix & 1) | ((iy & 1) << 1), e);
    int n = 0;
    for (int i = 0; i < 27; ++i) {
        const int sx = ix + e[i].dx, sy = iy + e[i].dy;
        if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
        out[2 * n] = sx;
        out[2 * n + 1] = sy;
        ++n;
    }
    return n;
}

int64_t m2l_pair_count(int L) {
    int64_t tot = 0;
    for (int l = 2; l <= L; ++l) {
        const int64_t n = int64_t(1) << l;
        tot += (6 * n - 8) * (6 * n - 8) - (3 * n - 2) * (3 * n - 2);
    }
    return tot;
}

// ----------------------------------------------------------------------------
// Operator tables, built in FP64 on the host.
// ----------------------------------------------------------------------------
struct HC { double re, im; };
static HC hmul(HC a, HC b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

static std::vector<double> binomials(int nmax) {
    // Pascal's triangle, nmax + 1 rows
    std::vector<double> c(size_t(nmax + 1) * (nmax + 1), 0.0);
    for (int n = 0; n <= nmax; ++n) {
        c[size_t(n) * (nmax + 1)] = 1.0;
        for (int k = 1; k <= n; ++k)
            c[size_t(n) * (nmax + 1) + k] =
                c[size_t(n - 1) * (nmax + 1) + k - 1] + (k <= n - 1 ? c[size_t(n - 1) * (nmax + 1) + k] : 0.0);
    }
    return c;
}

void host_m2l_table(int p, double *out) {
    const int nb = 2 * p;
    std::vector<double> C = binomials(nb);
    auto binom = [&](int n, int k) { return C[size_t(n) * (nb + 1) + k]; };
    int op = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
            // powers of 1/delta
            const double den = double(x) * x + double(y) * y;
            const HC inv = {double(x) / den, -double(y) / den};
            std::vector<HC> ip(size_t(2 * p + 1));
            ip[0] = {1.0, 0.0};
            for (int i = 1; i <= 2 * p; ++i) ip[i] = hmul(ip[i - 1], inv);
            for (int k = 0; k < p; ++k)
                for (int m = 0; m < p; ++m) {
                    const double s = ((k & 1) ? 1.0 : -1.0) * binom(k + m, k);
                    const HC t = ip[k + m + 1];
                    double *o = out + ((size_t(op) * p + k) * p + m) * 2;
                    o[0] = s * t.re;
                    o[1] = s * t.im;
                }
            ++op;
        }
}

static void host_m2m_table(int p, double *out /* [c][l][k] */) {
    std::vector<double> C = binomials(p);
    for (int c = 0; c < 4; ++c) {
        const HC e = {(c & 1) - 0.5, (c >> 1) - 0.5};
        std::vector<HC> ep(size_t(p + 1));
        ep[0] = {1.0, 0.0};
        for (int i = 1; i <= p; ++i) ep[i] = hmul(ep[i - 1], e);
        for (int l = 0; l < p; ++l)
            for (int k = 0; k < p; ++k) {
                double *o = out + ((size_t(c) * p + l) * p + k) * 2;
                if (k > l) { o[0] = o[1] = 0.0; continue; }
                const double s = std::ldexp(C[size_t(l) * (p + 1) + k], -l);
                o[0] = s * ep[l - k].re;
                o[1] = s * ep[l - k].im;
            }
    }
}

static void host_l2l_table(int p, double *out /* [c][n][m] */) {
    std::vector<double> C = binomials(p);
    for (int c = 0; c < 4; ++c) {
        const HC e = {(c & 1) - 0.5, (c >> 1) - 0.5};
        std::vector<HC> ep(size_t(p + 1));
        ep[0] = {1.0, 0.0};
        for (int i = 1; i <= p; ++i) ep[i] = hmul(ep[i - 1], e);
        for (int n = 0; n < p; ++n)
            for (int m = 0; m < p; ++m) {
                double *o = out + ((size_t(c) * p + n) * p + m) * 2;
                if (m < n) { o[0] = o[1] = 0.0; continue; }
                const double s = std::ldexp(C[size_t(m) * (p + 1) + n], -(m + 1));
                o[0] = s * ep[m - n].re;
                o[1] = s * ep[m - n].im;
            }
    }
}

// Laplace kernel (log potential), rescaled like the Cauchy series: ME
// a~_0 = a_0, a~_k = a_k / w^k; LE b^_m = b_m w^m (w the box width).  With
// e the child centre's offset from the parent's in child widths and delta the
// source centre's offset from the target's in box widths, the translations
// do not depend on the level, except the constant of M2L, whose a_0 log w
// term the M2L kernel adds.
//   M2M  [c][l][k]: l = 0: a~_0; l >= 1: -a~_0 e^l / (l 2^l)
//                   + sum_{1<=k<=l} C(l-1, k-1) e^(l-k) 2^-l a~_k
//   L2L  [c][n][m]: C(m, n) e^(m-n) 2^-m, m >= n
//   M2L  [op][k][m]: k = 0: m = 0 log(-delta), m >= 1 -1 / (m delta^m);
//                   k >= 1: (-1)^k C(m+k-1, k-1) / delta^(k+m)
static void host_lap_m2m_table(int p, double *out /* [c][l][k] */) {
    std::vector<double> C = binomials(p);
    for (int c = 0; c < 4; ++c) {
        const HC e = {(c & 1) - 0.5, (c >> 1) - 0.5};
        std::vector<HC> ep(size_t(p + 1));
        ep[0] = {1.0, 0.0};
        for (int i = 1; i <= p; ++i) ep[i] = hmul(ep[i - 1], e);
        for (int l = 0; l < p; ++l)
            for (int k = 0; k < p; ++k) {
                double *o = out + ((size_t(c) * p + l) * p + k) * 2;
                o[0] = o[1] = 0.0;
                if (k > l) continue;
                if (l == 0) {
                    o[0] = 1.0;
                } else if (k == 0) {
                    const double s = -std::ldexp(1.0, -l) / double(l);
                    o[0] = s * ep[l].re;
                    o[1] = s * ep[l].im;
                } else {
                    const double s = std::ldexp(C[size_t(l - 1) * (p + 1) + k - 1], -l);
                    o[0] = s * ep[l - k].re;
                    o[1] = s * ep[l - k].im;
                }
            }
    }
}

static void host_lap_l2l_table(int p, double *out /* [c][n][m] */) {
    std::vector<double> C = binomials(p);
    for (int c = 0; c < 4; ++c) {
        const HC e = {(c & 1) - 0.5, (c >> 1) - 0.5};
        std::vector<HC> ep(size_t(p + 1));
        ep[0] = {1.0, 0.0};
        for (int i = 1; i <= p; ++i) ep[i] = hmul(ep[i - 1], e);
        for (int n = 0; n < p; ++n)
            for (int m = 0; m < p; ++m) {
                double *o = out + ((size_t(c) * p + n) * p + m) * 2;
                if (m < n) { o[0] = o[1] = 0.0; continue; }
                const double s = std::ldexp(C[size_t(m) * (p + 1) + n], -m);
                o[0] = s * ep[m - n].re;
                o[1] = s * ep[m - n].im;
            }
    }
}

void host_lap_m2l_table(int p, double *out /* [op][k][m] */) {
    const int nb = 2 * p;
    std::vector<double> C = binomials(nb);
    auto binom = [&](int n, int k) { return C[size_t(n) * (nb + 1) + k]; };
    int op = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
            const double den = double(x) * x + double(y) * y;
            const HC inv = {double(x) / den, -double(y) / den};
            std::vector<HC> ip(size_t(2 * p + 1));
            ip[0] = {1.0, 0.0};
            for (int i = 1; i <= 2 * p; ++i) ip[i] = hmul(ip[i - 1], inv);
            for (int k = 0; k < p; ++k)
                for (int m = 0; m < p; ++m) {
                    double *o = out + ((size_t(op) * p + k) * p + m) * 2;
                    HC t;
                    if (k == 0 && m == 0) {
                        // log(-delta), principal branch (only Re enters the result)
                        t = {0.5 * std::log(den), std::atan2(-double(y), -double(x))};
                    } else if (k == 0) {
                        const double s = -1.0 / double(m);
                        t = {s * ip[m].re, s * ip[m].im};
                    } else {
                        const double s = ((k & 1) ? -1.0 : 1.0) * binom(m + k - 1, k - 1);
                        t = {s * ip[k + m].re, s * ip[k + m].im};
                    }
                    o[0] = t.re;
                    o[1] = t.im;
                }
            ++op;
        }
}

void host_op_table(int p, int kernel, int which, std::vector<double> &out) {
    const bool lap = kernel == KERNEL_LAPLACE;
    out.assign(size_t(which == 2 ? 40 : 4) * p * p * 2, 0.0);
    if (which == 0) (lap ? host_lap_m2m_table : host_m2m_table)(p, out.data());
    else if (which == 1) (lap ? host_lap_l2l_table : host_l2l_table)(p, out.data());
    else (lap ? host_lap_m2l_table : host_m2l_table)(p, out.data());
}

cudaError_t build_op_tables(int p, int kernel, OpTables *t) {
    cudaError_t e = upload_il();
    if (e != cudaSuccess) return e;
    t->p = p;
    const size_t n_m2m = size_t(4) * p * p, n_m2l = size_t(40) * p * p;
    std::vector<double> m2m(2 * n_m2m), l2l(2 * n_m2m), m2l(2 * n_m2l);
    if (kernel == KERNEL_LAPLACE) {
        host_lap_m2m_table(p, m2m.data());
        host_lap_l2l_table(p, l2l.data());
        host_lap_m2l_table(p, m2l.data());
    } else {
        host_m2m_table(p, m2m.data());
        host_l2l_table(p, l2l.data());
        host_m2l_table(p, m2l.data());
    }
    std::vector<float> m2m32(m2m.begin(), m2m.end()), l2l32(l2l.begin(), l2l.end()),
        m2l32(m2l.begin(), m2l.end());
    auto up = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(dst, bytes);
        if (r != cudaSuccess) return r;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    if ((e = up((void **)&t->m2m64, m2m.data(), m2m.size() * 8)) != cudaSuccess) return e;
    if ((e = up((void **)&t->l2l64, l2l.data(), l2l.size() * 8)) != cudaSuccess) return e;
    if ((e = up((void **)&t->m2l64, m2l.data(), m2l.size() * 8)) != cudaSuccess) return e;
    if ((e = up((void **)&t->m2m32, m2m32.data(), m2m32.size() * 4)) != cudaSuccess) return e;
    if ((e = up((void **)&t->l2l32, l2l32.data(), l2l32.size() * 4)) != cudaSuccess) return e;
    if ((e = up((void **)&t->m2l32, m2l32.data(), m2l32.size() * 4)) != cudaSuccess) return e;
    if (((2 * p + 15) & ~15) <= 48) {
        std::vector<float> img;
        host_m2l_tc_images(p, kernel, img);
        if ((e = up((void **)&t->m2l_tc, img.data(), img.size() * 4)) != cudaSuccess) return e;
        host_m2l_tcb_images(p, kernel, img);
        if ((e = up((void **)&t->m2l_tcb, img.data(), img.size() * 4)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void free_op_tables(OpTables *t) {
    cudaFree(t->m2m64); cudaFree(t->l2l64); cudaFree(t->m2l64);
    cudaFree(t->m2m32); cudaFree(t->l2l32); cudaFree(t->m2l32);
    cudaFree(t->m2l_tc);
    cudaFree(t->m2l_tcb);
    *t = OpTables();
}

// ----------------------------------------------------------------------------
// P2M: one warp per occupied leaf.  k_occ_list collects the occupied leaves
// (in no particular order); a persistent grid of warps strides over that
// list, so no block is spent on an empty leaf and the dense leaves of a
// cluster spread over all SMs.  Per leaf, lanes take 32 particles at a time,
// write the gamma * zeta^k powers to shared memory, and lane k sums column k
// in a fixed order: each leaf's expansion does not depend on which warp or
// in which order the leaves were processed.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_occ_list(const Task *__restrict__ tasks, int ntasks,
                                                  const InstDesc *__restrict__ insts,
                                                  const uint32_t *__restrict__ start,
                                                  uint2 *__restrict__ occ, uint32_t *ctrl) {
    const int lane = threadIdx.x & 31;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    bool o = false;
    if (m < t.count) {
        const uint32_t *st = start + insts[t.inst].soff;
        o = st[m + 1] > st[m];
    }
    const uint32_t b = __ballot_sync(0xffffffffu, o);
    uint32_t base = 0;
    if (lane == 0 && b) base = atomicAdd(ctrl + CTRL_NOCC, uint32_t(__popc(b)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (o) occ[base + __popc(b & ((1u << lane) - 1u))] = make_uint2(uint32_t(t.inst), uint32_t(m));
}

cudaError_t launch_occ_list(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                            const uint32_t *start, uint2 *occ, uint32_t *ctrl, cudaStream_t st,
                            uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_occ_list<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, occ, ctrl);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

template <typename R>
__device__ __forceinline__ typename Cplx<R>::T mk2(R a, R b) {
    typename Cplx<R>::T r;
    r.x = a;
    r.y = b;
    return r;
}

template <typename R>
__global__ void __launch_bounds__(P2M_WARPS * 32) k_p2m(
    const uint2 *__restrict__ occ, const uint32_t *ctrl, const InstDesc *__restrict__ insts,
    int pmax, const uint32_t *__restrict__ start, const double *__restrict__ xs,
    const double *__restrict__ ys, const double *__restrict__ gs, const float4 *__restrict__ rec,
    typename Cplx<R>::T *__restrict__ me) {
    using C2 = typename Cplx<R>::T;
    extern __shared__ unsigned char smem_raw[];
    C2 *buf = reinterpret_cast<C2 *>(smem_raw) + size_t(threadIdx.x >> 5) * 32 * pmax;
    const int lane = threadIdx.x & 31;
    const uint32_t nocc = ctrl[CTRL_NOCC];
    const uint32_t nwarps = gridDim.x * P2M_WARPS;
    for (uint32_t i = blockIdx.x * P2M_WARPS + (threadIdx.x >> 5); i < nocc; i += nwarps) {
        const uint2 e = occ[i];
        const InstDesc &d = insts[e.x];
        const int p = d.p, L = d.L;
        const uint32_t m = e.y;
        uint32_t s0 = start[d.soff + m], s1 = start[d.soff + m + 1];
        if (!(PF_IN(m, int64_t(1) << (2 * L)) && PF_IN(int64_t(s0) - d.poff, d.n + 1) &&
              PF_IN(int64_t(s1) - d.poff, d.n + 1)) || s1 < s0)
            s1 = s0;  // checked build: a leaf range outside the instance is skipped
        const uint32_t ix = compact_bits(m), iy = compact_bits(m >> 1);
        const double cx = d.x0 + (double(ix) + 0.5) * d.wleaf;
        const double cy = d.y0 + (double(iy) + 0.5) * d.wleaf;
        C2 acc0 = mk2<R>(R(0), R(0)), acc1 = mk2<R>(R(0), R(0));
        for (uint32_t c0 = s0; c0 < s1; c0 += 32) {
            const uint32_t j = c0 + lane;
            C2 z, w;
            if (j < s1) {
                if (rec) {
                    const float4 r = rec[j];
                    z = mk2<R>(R(r.x), R(r.y));
                    w = mk2<R>(R(r.z), R(0));
                } else {
                    z = mk2<R>(R((xs[j] - cx) * d.scale), R((ys[j] - cy) * d.scale));
                    w = mk2<R>(R(gs[j]), R(0));
                }
            } else {
                z = mk2<R>(R(0), R(0));
                w = mk2<R>(R(0), R(0));
            }
            // vortex: gamma zeta^k; Laplace: q, then -q zeta^k / k
            const bool lap = d.kernel == KERNEL_LAPLACE;
            for (int k = 0; k < p; ++k) {
                C2 wk = w;
                if (lap && k) {
                    const R s = R(-1) / R(k);
                    wk = mk2<R>(w.x * s, w.y * s);
                }
                buf[lane * pmax + k] = wk;
                w = cmul(w, z);
            }
            __syncwarp();
            if (lane < p) {
                for (int q = 0; q < 32; ++q) {
                    const C2 b = buf[q * pmax + lane];
                    acc0.x += b.x;
                    acc0.y += b.y;
                }
            }
            if (lane + 32 < p) {
                for (int q = 0; q < 32; ++q) {
                    const C2 b = buf[q * pmax + lane + 32];
                    acc1.x += b.x;
                    acc1.y += b.y;
                }
            }
            __syncwarp();
        }
        C2 *dst = me + d.eoff + (lvl_off(L) + box_index(L, ix, iy)) * p;
        if (lane < p) dst[lane] = acc0;
        if (lane + 32 < p) dst[lane + 32] = acc1;
    }
}

// Leaves of at most this many blobs are summed by one lane each (k_p2m_reg).
constexpr uint32_t P2M_LANE_MAX = 16;

// Mixed path, p <= PM: each lane keeps the running sums of its particles'
// gamma zeta^k in registers over all chunks of the leaf, and the warp adds
// the 32 lanes' sums once per leaf (transposed through shared memory, lane k
// adding column k: even rows and odd rows separately, then the two).  About a
// third of the instructions of the per-chunk transpose above.
template <int PM>
__global__ void __launch_bounds__(P2M_WARPS * 32) k_p2m_reg(
    const uint2 *__restrict__ occ, const uint32_t *ctrl, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float4 *__restrict__ rec, float2 *__restrict__ me) {
    constexpr int SP = PM | 1;  // odd row stride: conflict-free 8-byte accesses
    __shared__ float2 buf[P2M_WARPS][32 * SP];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nocc = ctrl[CTRL_NOCC];
    const uint32_t gw = blockIdx.x * P2M_WARPS + wid, nwarps = gridDim.x * P2M_WARPS;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // leaf range of occupied-leaf entry i (empty in the checked build when
    // it lies outside its instance)
    auto range = [&](uint32_t i, const InstDesc *&dp, uint32_t &m, uint32_t &s0, uint32_t &s1) {
        const uint2 e = occ[i];
        dp = insts + e.x;
        m = e.y;
        s0 = start[dp->soff + m];
        s1 = start[dp->soff + m + 1];
        if (!(PF_IN(m, int64_t(1) << (2 * dp->L)) && PF_IN(int64_t(s0) - dp->poff, dp->n + 1) &&
              PF_IN(int64_t(s1) - dp->poff, dp->n + 1)) || s1 < s0)
            s1 = s0;
    };
    // 1. Leaves of at most P2M_LANE_MAX blobs, one per lane, 32 entries per
    //    warp at a time: the lane sums its few blobs' series by itself and
    //    writes the p coefficients (a warp and a 32-row reduction per leaf
    //    of one or a few blobs would be mostly idle).
    for (uint32_t base = gw * 32; base < nocc; base += nwarps * 32) {
        const uint32_t i = base + lane;
        if (i >= nocc) continue;
        const InstDesc *dp;
        uint32_t m, s0, s1;
        range(i, dp, m, s0, s1);
        if (s1 - s0 > P2M_LANE_MAX) continue;
        const InstDesc &d = *dp;
        const int p = d.p;
        float2 acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k) acc[k] = make_float2(0.f, 0.f);
        for (uint32_t j = s0; j < s1; ++j) {
            const float4 r = rec[j];
            float2 w = make_float2(r.z, 0.f);
            const float2 z = make_float2(r.x, r.y);
#pragma unroll
            for (int k = 0; k < PM; ++k) {
                if (k < p) {
                    acc[k].x += w.x;
                    acc[k].y += w.y;
                    w = cmul(w, z);
                }
            }
        }
        const uint32_t ix = compact_bits(m), iy = compact_bits(m >> 1);
        float2 *dst = me + d.eoff + (lvl_off(d.L) + box_index(d.L, ix, iy)) * p;
        const bool lap = d.kernel == KERNEL_LAPLACE;
#pragma unroll
        for (int k = 0; k < PM; ++k) {
            if (k < p) {
                // Laplace kernel: a_k = -(1/k) sum q zeta^k for k >= 1
                const float sc = (lap && k) ? -1.0f / float(k) : 1.0f;
                dst[k] = make_float2(sc * acc[k].x, sc * acc[k].y);
            }
        }
    }
    // 2. Larger leaves, one per warp (striding over the entries)
    for (uint32_t i = gw; i < nocc; i += nwarps) {
        const InstDesc *dp;
        uint32_t m, s0, s1;
        range(i, dp, m, s0, s1);
        if (s1 - s0 <= P2M_LANE_MAX) continue;
        const InstDesc &d = *dp;
        const int p = d.p, L = d.L;
        float2 acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k) acc[k] = make_float2(0.f, 0.f);
        // Leaves of more than 32 blobs: two blobs per lane per step (two
        // independent power chains), and the next step's two records
        // requested before this step's arithmetic: up to four 16-byte loads
        // in flight per lane.  Smaller leaves take one step of one blob per
        // lane (a second chain would only add padding).
        if (s1 - s0 <= 32) {
            const float4 r = s0 + lane < s1 ? rec[s0 + lane] : z4;
            float2 w = make_float2(r.z, 0.f);
            const float2 z = make_float2(r.x, r.y);
#pragma unroll
            for (int k = 0; k < PM; ++k) {
                if (k < p) {
                    acc[k].x += w.x;
                    acc[k].y += w.y;
                    w = cmul(w, z);
                }
            }
        }
        float4 na = z4, nb = z4;
        if (s1 - s0 > 32) {
            na = rec[s0 + lane];
            nb = s0 + 32 + lane < s1 ? rec[s0 + 32 + lane] : z4;
        }
        for (uint32_t c0 = s0; s1 - s0 > 32 && c0 < s1; c0 += 64) {
            const float4 ra = na, rb = nb;
            const uint32_t jn = c0 + 64 + lane;
            na = jn < s1 ? rec[jn] : z4;
            nb = jn + 32 < s1 ? rec[jn + 32] : z4;
            float2 wa = make_float2(ra.z, 0.f), wb = make_float2(rb.z, 0.f);
            const float2 za = make_float2(ra.x, ra.y), zb = make_float2(rb.x, rb.y);
#pragma unroll
            for (int k = 0; k < PM; ++k) {
                if (k < p) {
                    acc[k].x += wa.x;
                    acc[k].y += wa.y;
                    acc[k].x += wb.x;
                    acc[k].y += wb.y;
                    wa = cmul(wa, za);
                    wb = cmul(wb, zb);
                }
            }
        }
        float2 *row = buf[wid] + lane * SP;
#pragma unroll
        for (int k = 0; k < PM; ++k)
            if (k < p) row[k] = acc[k];
        __syncwarp();
        if (lane < p) {
            float2 se = make_float2(0.f, 0.f), so = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int q = 0; q < 32; q += 2) {
                const float2 a = buf[wid][q * SP + lane], b = buf[wid][(q + 1) * SP + lane];
                se.x += a.x;
                se.y += a.y;
                so.x += b.x;
                so.y += b.y;
            }
            const uint32_t ix = compact_bits(m), iy = compact_bits(m >> 1);
            // Laplace kernel: a_k = -(1/k) sum q zeta^k for k >= 1
            const float s = (d.kernel == KERNEL_LAPLACE && lane) ? -1.0f / float(lane) : 1.0f;
            me[d.eoff + (lvl_off(L) + box_index(L, ix, iy)) * p + lane] =
                make_float2(s * (se.x + so.x), s * (se.y + so.y));
        }
        __syncwarp();
    }
}

template <int PM, typename C2>
cudaError_t launch_p2m_reg(const uint2 *occ, const uint32_t *ctrl, int64_t max_occ,
                           const InstDesc *insts, const uint32_t *start, const float4 *rec,
                           C2 *me, cudaStream_t st) {
    if constexpr (std::is_same<C2, float2>::value) {
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2m_reg<PM>, P2M_WARPS * 32, 0);
        if (per_sm < 1) per_sm = 1;
        const int64_t grid = std::min<int64_t>((max_occ + P2M_WARPS - 1) / P2M_WARPS,
                                               int64_t(per_sm) * device_sm_count());
        k_p2m_reg<PM><<<unsigned(grid), P2M_WARPS * 32, 0, st>>>(occ, ctrl, insts, start, rec, me);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <typename R>
cudaError_t launch_p2m(const uint2 *occ, const uint32_t *ctrl, int64_t max_occ,
                       const InstDesc *insts, int pmax, const uint32_t *start, const double *xs,
                       const double *ys, const double *gs, const float4 *rec,
                       typename Cplx<R>::T *me, cudaStream_t st, uint64_t *launches) {
    if (max_occ <= 0) return cudaSuccess;
    const size_t smem = size_t(P2M_WARPS) * 32 * pmax * sizeof(typename Cplx<R>::T);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_p2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
    }
    if (rec) {
        // mixed path: the register-accumulating kernel for the smallest
        // compiled bound on p
        cudaError_t e = cudaErrorNotSupported;
        if (pmax <= 8) e = launch_p2m_reg<8>(occ, ctrl, max_occ, insts, start, rec, me, st);
        else if (pmax <= 12) e = launch_p2m_reg<12>(occ, ctrl, max_occ, insts, start, rec, me, st);
        else if (pmax <= 17) e = launch_p2m_reg<17>(occ, ctrl, max_occ, insts, start, rec, me, st);
        else if (pmax <= 24) e = launch_p2m_reg<24>(occ, ctrl, max_occ, insts, start, rec, me, st);
        if (e != cudaErrorNotSupported) {
            PF_LAUNCHED(1);
            return e;
        }
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2m<R>, P2M_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>((max_occ + P2M_WARPS - 1) / P2M_WARPS,
                                           int64_t(per_sm) * device_sm_count());
    k_p2m<R><<<unsigned(grid), P2M_WARPS * 32, smem, st>>>(occ, ctrl, insts, pmax, start, xs, ys,
                                                          gs, rec, me);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// M2M: one thread per (parent box, output coefficient).  Task = (instance,
// parent level l); units = 4^l * p in row-major box order.
// ----------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(EXP_THREADS) k_m2m(const Task *__restrict__ tasks, int ntasks,
                                                     const InstDesc *__restrict__ insts,
                                                     const uint32_t *__restrict__ start,
                                                     typename Cplx<R>::T *__restrict__ me) {
    using C2 = typename Cplx<R>::T;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t u = (int64_t(blockIdx.x) - t.block0) * EXP_THREADS + threadIdx.x;
    if (u >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int p = d.p, l = t.level;
    const int64_t box = u / p;
    const int lp = int(u - box * p);
    const uint32_t ix = uint32_t(box & ((int64_t(1) << l) - 1)), iy = uint32_t(box >> l);
    const uint32_t *st = start + d.soff;
    const uint32_t pm = morton_key(ix, iy);
    if (!box_count(st, d.L, l, pm)) return;
    const C2 *tab = static_cast<const C2 *>(d.t_m2m);
    const int64_t quarter = int64_t(1) << (2 * l);
    const C2 *child = me + d.eoff + (lvl_off(l + 1) + int64_t(iy) * (int64_t(1) << l) + ix) * p;
    C2 s = mk2<R>(R(0), R(0));
    for (int c = 0; c < 4; ++c) {
        // child c of the parent has Morton index 4 pm + c; an empty child has
        // no expansion (it would be zero)
        if (!box_count(st, d.L, l + 1, 4 * pm + uint32_t(c))) continue;
        const C2 *a = child + c * quarter * p;
        const C2 *row = tab + (size_t(c) * p + lp) * p;
        for (int k = 0; k <= lp; ++k) s = cfma(row[k], a[k], s);
    }
    me[d.eoff + (lvl_off(l) + box_index(l, ix, iy)) * p + lp] = s;
}

template <typename R>
cudaError_t launch_m2m(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, typename Cplx<R>::T *me, cudaStream_t st,
                       uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_m2m<R><<<unsigned(nblocks), EXP_THREADS, 0, st>>>(tasks, ntasks, insts, start, me);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// L2L: one thread per (child box, output coefficient); adds the parent's
// local expansion, translated, to the child's.  Task = (instance, child
// level l); units = 4^l * p, row-major.
// ----------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(EXP_THREADS) k_l2l(const Task *__restrict__ tasks, int ntasks,
                                                     const InstDesc *__restrict__ insts,
                                                     const uint32_t *__restrict__ start,
                                                     typename Cplx<R>::T *__restrict__ le) {
    using C2 = typename Cplx<R>::T;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t u = (int64_t(blockIdx.x) - t.block0) * EXP_THREADS + threadIdx.x;
    if (u >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int p = d.p, l = t.level;
    const int64_t box = u / p;
    const int n = int(u - box * p);
    const uint32_t ix = uint32_t(box & ((int64_t(1) << l) - 1)), iy = uint32_t(box >> l);
    if (!box_count(start + d.soff, d.L, l, morton_key(ix, iy))) return;
    const int c = int((ix & 1u) | ((iy & 1u) << 1));
    const C2 *tab = static_cast<const C2 *>(d.t_l2l) + (size_t(c) * p + n) * p;
    const C2 *par = le + d.eoff + (lvl_off(l - 1) + box_index(l - 1, ix >> 1, iy >> 1)) * p;
    C2 s = mk2<R>(R(0), R(0));
    for (int m = n; m < p; ++m) s = cfma(tab[m], par[m], s);
    C2 *dst = le + d.eoff + (lvl_off(l) + box_index(l, ix, iy)) * p + n;
    C2 o = *dst;
    o.x += s.x;
    o.y += s.y;
    *dst = o;
}

template <typename R>
cudaError_t launch_l2l(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, typename Cplx<R>::T *le, cudaStream_t st,
                       uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_l2l<R><<<unsigned(nblocks), EXP_THREADS, 0, st>>>(tasks, ntasks, insts, start, le);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// M2L (SIMT): one warp per target box; lane m owns output coefficient m (and
// m + 32).  The source ME is staged in per-warp shared memory and read as a
// broadcast; operator rows come through L1.  Task = (instance, level l),
// units = 4^l target boxes, row-major.
// ----------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(M2L_WARPS * 32) k_m2l(const Task *__restrict__ tasks,
                                                        int ntasks,
                                                        const InstDesc *__restrict__ insts,
                                                        const uint32_t *__restrict__ start,
                                                        const typename Cplx<R>::T *__restrict__ me,
                                                        typename Cplx<R>::T *__restrict__ le,
                                                        const uint32_t *__restrict__ ucount,
                                                        int dense_pct) {
    using C2 = typename Cplx<R>::T;
    __shared__ C2 sa[M2L_WARPS][MAX_P];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t box0 = ((int64_t(blockIdx.x) - t.block0) * M2L_WARPS + wid) * BOX_RUN;
    if (box0 >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int p = d.p, l = t.level;
    const int nside = 1 << l;
    const uint32_t *st = start + d.soff;
    // the run's target boxes that hold particles and are not left to the
    // tensor cores (levels that also run there leave the dense units to them)
    bool mine = false;
    if (lane < BOX_RUN && box0 + lane < t.count) {
        const int64_t bx = box0 + lane;
        const int jx = int(bx & (nside - 1)), jy = int(bx >> l);
        mine = box_count(st, d.L, l, morton_key(uint32_t(jx), uint32_t(jy))) != 0;
        if (mine && d.tc_unit0[l] >= 0) {
            const int jc = (jx & 1) | ((jy & 1) << 1);
            int nbox;
            const int64_t u = d.tc_unit0[l] + unit_of(d, l, jc, jy >> 1, jx >> 1, &nbox);
            mine = !tc_unit_dense(ucount[u], nbox, dense_pct);
        }
    }
    uint32_t todo = __ballot_sync(0xffffffffu, mine);
    while (todo) {
        const int64_t box = box0 + (__ffs(todo) - 1);
        todo &= todo - 1;
        const int ix = int(box & (nside - 1)), iy = int(box >> l);
        const int c = (ix & 1) | ((iy & 1) << 1);
        const C2 *tab = static_cast<const C2 *>(d.t_m2l);
        const C2 *lev = me + d.eoff + lvl_off(l) * p;
        C2 acc0 = mk2<R>(R(0), R(0)), acc1 = mk2<R>(R(0), R(0));
        for (int e = 0; e < 27; ++e) {
            const IlEntry en = c_il[c][e];
            const int sx = ix + en.dx, sy = iy + en.dy;
            if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
            if (!box_count(st, d.L, l, morton_key(uint32_t(sx), uint32_t(sy)))) continue;
            const C2 *src = lev + box_index(l, uint32_t(sx), uint32_t(sy)) * p;
            if (lane < p) sa[wid][lane] = src[lane];
            if (lane + 32 < p) sa[wid][lane + 32] = src[lane + 32];
            __syncwarp();
            const C2 *T = tab + size_t(en.op) * p * p;
            if (lane < p) {
                for (int k = 0; k < p; ++k) acc0 = cfma(T[k * p + lane], sa[wid][k], acc0);
            }
            if (lane + 32 < p) {
                for (int k = 0; k < p; ++k) acc1 = cfma(T[k * p + lane + 32], sa[wid][k], acc1);
            }
            __syncwarp();
        }
        C2 *dst = le + d.eoff + (lvl_off(l) + box_index(l, uint32_t(ix), uint32_t(iy))) * p;
        if (lane < p) dst[lane] = acc0;
        if (lane + 32 < p) dst[lane + 32] = acc1;
    }
}

template <typename R>
cudaError_t launch_m2l(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, const typename Cplx<R>::T *me,
                       typename Cplx<R>::T *le, const uint32_t *ucount, int dense_pct,
                       cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_m2l<R><<<unsigned(nblocks), M2L_WARPS * 32, 0, st>>>(tasks, ntasks, insts, start, me, le,
                                                          ucount, dense_pct);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Laplace kernel, the level-dependent constant of M2L: the rescaled
// operators carry log(-delta); the a~_0 log w_l part is added here, after all
// M2L kernels of the evaluation: b^_0(t) += log w_l * sum over the occupied
// interaction-list sources s of a~_0(s).  One thread per target box (task =
// instance, level; units = 4^l boxes, row-major), occupied targets only.
// ----------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_m2l_logterm(const Task *__restrict__ tasks, int ntasks,
                                                     const InstDesc *__restrict__ insts,
                                                     const uint32_t *__restrict__ start,
                                                     const typename Cplx<R>::T *__restrict__ me,
                                                     typename Cplx<R>::T *__restrict__ le) {
    using C2 = typename Cplx<R>::T;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t box = (int64_t(blockIdx.x) - t.block0) * 256 + threadIdx.x;
    if (box >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int p = d.p, l = t.level, nside = 1 << l;
    const uint32_t *st = start + d.soff;
    const int ix = int(box & (nside - 1)), iy = int(box >> l);
    if (!box_count(st, d.L, l, morton_key(uint32_t(ix), uint32_t(iy)))) return;
    const int c = (ix & 1) | ((iy & 1) << 1);
    const C2 *lev = me + d.eoff + lvl_off(l) * p;
    R sr = R(0), si = R(0);
    for (int e = 0; e < 27; ++e) {
        const IlEntry en = c_il[c][e];
        const int sx = ix + en.dx, sy = iy + en.dy;
        if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
        if (!box_count(st, d.L, l, morton_key(uint32_t(sx), uint32_t(sy)))) continue;
        const C2 a0 = lev[box_index(l, uint32_t(sx), uint32_t(sy)) * p];
        sr += a0.x;
        si += a0.y;
    }
    const R logw = R(d.logw0 - double(l) * 0.69314718055994530942);
    C2 *dst = le + d.eoff + (lvl_off(l) + box_index(l, uint32_t(ix), uint32_t(iy))) * p;
    C2 o = *dst;
    o.x += logw * sr;
    o.y += logw * si;
    *dst = o;
}

template <typename R>
cudaError_t launch_m2l_logterm(const Task *tasks, int ntasks, int64_t nblocks,
                               const InstDesc *insts, const uint32_t *start,
                               const typename Cplx<R>::T *me, typename Cplx<R>::T *le,
                               cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_m2l_logterm<R><<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, me, le);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}
template cudaError_t launch_m2l_logterm<double>(const Task *, int, int64_t, const InstDesc *,
                                                const uint32_t *, const double2 *, double2 *,
                                                cudaStream_t, uint64_t *);
template cudaError_t launch_m2l_logterm<float>(const Task *, int, int64_t, const InstDesc *,
                                               const uint32_t *, const float2 *, float2 *,
                                               cudaStream_t, uint64_t *);

template cudaError_t launch_p2m<double>(const uint2 *, const uint32_t *, int64_t,
                                        const InstDesc *, int, const uint32_t *, const double *,
                                        const double *, const double *, const float4 *, double2 *,
                                        cudaStream_t, uint64_t *);
template cudaError_t launch_p2m<float>(const uint2 *, const uint32_t *, int64_t, const InstDesc *,
                                       int, const uint32_t *, const double *, const double *,
                                       const double *, const float4 *, float2 *, cudaStream_t,
                                       uint64_t *);
template cudaError_t launch_m2m<double>(const Task *, int, int64_t, const InstDesc *,
                                        const uint32_t *, double2 *, cudaStream_t, uint64_t *);
template cudaError_t launch_m2m<float>(const Task *, int, int64_t, const InstDesc *,
                                       const uint32_t *, float2 *, cudaStream_t, uint64_t *);
template cudaError_t launch_l2l<double>(const Task *, int, int64_t, const InstDesc *,
                                        const uint32_t *, double2 *, cudaStream_t, uint64_t *);
template cudaError_t launch_l2l<float>(const Task *, int, int64_t, const InstDesc *,
                                       const uint32_t *, float2 *, cudaStream_t, uint64_t *);
template cudaError_t launch_m2l<double>(const Task *, int, int64_t, const InstDesc *,
                                        const uint32_t *, const double2 *, double2 *,
                                        const uint32_t *, int, cudaStream_t, uint64_t *);
template cudaError_t launch_m2l<float>(const Task *, int, int64_t, const InstDesc *,
                                       const uint32_t *, const float2 *, float2 *,
                                       const uint32_t *, int, cudaStream_t, uint64_t *);

PF_DEFINE_CHECK_READER(expansions)

}  // namespace petfmm
