// p2p.cu -- evaluation step of Sec. 2.2: the direct near-field sum over the
// leaf and its 8 neighbours with the regularised kernel of Eq. 8, fused with
// L2P of the leaf's local expansion, written back in the caller's order.
//
// Work list.  Every occupied leaf is cut into items of at most TPI targets
// (one warp per item); an item's cost is (targets) x (sources in the 9
// leaves), the n_nd N_i^2 term of the work estimate of Eq. 14.  Warps of a
// persistent grid take items from a queue, so equal-cost items of one leaf
// spread across SMs and the heavy leaves of clustered inputs do not pin one
// SM.  An item with few targets (small leaves: a uniform layout holds about
// 16 blobs per leaf) would leave most lanes idle, so its warp splits into S
// groups of lanes: each group holds all the item's targets and takes every
// S-th source, and the S partial sums of a target are added by a fixed
// butterfly of warp shuffles.  The order of every sum depends only on the
// item's target count: results do not depend on which warp ran the item.
//
// Mixed path (FP32).  Coordinates are leaf-relative in leaf units; with
// rho^2 = |dx|^2 in leaf units and q = kappa rho^2, kappa = w^2 / 2 sigma^2,
//     u_i = w / (4 pi sigma^2) sum_j gamma_j (-d_eta, d_xi) g(q),
//     g(q) = (1 - exp(-q)) / q,
// which is Eq. 8 rearranged (no division, no cancellation at small q).  g is
// evaluated as a polynomial in rho^2 fitted on the host (Chebyshev
// interpolation of g on the range the near field can reach), i.e. on the FMA
// pipe only; if the near field reaches beyond the fitted range the "general"
// variant switches to (1 - exp(-q)) / q from the special-function unit above
// the split.  The self pair has d = 0 and adds exactly zero.
//
// FP64 path: the same loop in FP64 with -expm1(-q) / r^2 (CUDA's expm1).
#include "kernels.cuh"

namespace petfmm {

#define PF_LAUNCHED(n) do { if (launches) *launches += (n); } while (0)

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ----------------------------------------------------------------------------
// Work list
// ----------------------------------------------------------------------------
// log2 of the lanes that hold the targets of an item with nt targets, r per
// lane: the smallest power of two >= ceil(nt / r), at most 32.  The other
// 32 / 2^lw lane groups split the item's sources.
__host__ __device__ __forceinline__ int p2p_group_log2(uint32_t nt, int r) {
    const uint32_t h = (nt + uint32_t(r) - 1) / uint32_t(r);
    int lw = 0;
    while (lw < 5 && (1u << lw) < h) ++lw;
    return lw;
}

__global__ void __launch_bounds__(256) k_p2p_count(const Task *__restrict__ tasks, int ntasks,
                                                   const InstDesc *__restrict__ insts,
                                                   const uint32_t *__restrict__ start, int tpi,
                                                   uint32_t *__restrict__ cnt, uint32_t *ctrl) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    unsigned long long pairs = 0;
    if (m < t.count) {
        const InstDesc &d = insts[t.inst];
        const uint32_t *st = start + d.soff;
        const uint32_t n = st[m + 1] - st[m];
        cnt[d.loff + m] = (n + tpi - 1) / tpi;
        if (n) {
            const int nside = 1 << d.L;
            const int ix = int(compact_bits(uint32_t(m))), iy = int(compact_bits(uint32_t(m) >> 1));
            uint32_t src = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
                    const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
                    src += st[nm + 1] - st[nm];
                }
            pairs = (unsigned long long)n * (src - 1);
        }
    }
    // block reduction of the ordered pair count (for the statistics)
#pragma unroll
    for (int o = 16; o; o >>= 1) pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    __shared__ unsigned long long ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = pairs;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        if (s) atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + CTRL_PAIRS_LO), s);
    }
}

__global__ void __launch_bounds__(256) k_p2p_emit(const Task *__restrict__ tasks, int ntasks,
                                                  const InstDesc *__restrict__ insts,
                                                  const uint32_t *__restrict__ start, int tpi,
                                                  const uint32_t *__restrict__ cnt,
                                                  const uint32_t *__restrict__ off,
                                                  uint4 *__restrict__ items,
                                                  uint32_t *__restrict__ wclass) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (m >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const uint32_t c = cnt[d.loff + m];
    if (!c) return;
    const uint32_t *st = start + d.soff;
    const uint32_t s0 = st[m], s1 = st[m + 1];
    const uint32_t o = off[d.loff + m];
    // sources of the item: the blobs of the leaf and its neighbours
    uint32_t src = 0;
    if (wclass) {
        const int nside = 1 << d.L;
        const int ix = int(compact_bits(uint32_t(m))), iy = int(compact_bits(uint32_t(m) >> 1));
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int sx = ix + dx, sy = iy + dy;
                if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
                const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
                src += st[nm + 1] - st[nm];
            }
    }
    for (uint32_t i = 0; i < c; ++i) {
        const uint32_t f = s0 + i * uint32_t(tpi);
        const uint32_t nt = (s1 - f) < uint32_t(tpi) ? (s1 - f) : uint32_t(tpi);
        items[o + i] = make_uint4(uint32_t(t.inst), uint32_t(m), f, nt);
        // work class of the item (Eq. 14, n_nd N_i^2 term: targets x sources).
        // Every lane of the warp runs the source loop of its group, target
        // slot filled or not, so the cost is the sources per lane group,
        // ceil(src / S) with S groups.  Class = log2(cost) in quarter steps,
        // stored as 127 - class so that an ascending sort is heaviest first.
        if (wclass) {
            const int ns = 5 - p2p_group_log2(nt, tpi / 32);  // log2 S
            const uint32_t cost = (src + (1u << ns) - 1) >> ns;
            const int e = 31 - __clz(int(cost));  // cost >= 1: the leaf's own blobs
            const uint32_t frac = e >= 2 ? (cost >> (e - 2)) & 3u : (cost << (2 - e)) & 3u;
            wclass[o + i] = 127u - (uint32_t(e) * 4u + frac);
        }
    }
}

// Invalid tail of the item array (beyond the device-side count) sorts last.
__global__ void __launch_bounds__(256) k_item_tail(uint32_t *__restrict__ wclass, int64_t cap,
                                                   const uint32_t *ctrl) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < cap && i >= int64_t(ctrl[CTRL_NITEMS])) wclass[i] = 255u;
}

__global__ void __launch_bounds__(256) k_item_permute(const uint4 *__restrict__ in,
                                                      const uint32_t *__restrict__ perm,
                                                      uint4 *__restrict__ out, int64_t cap,
                                                      const uint32_t *ctrl) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r < cap && r < int64_t(ctrl[CTRL_NITEMS])) out[r] = in[perm[r]];
}

cudaError_t launch_p2p_worklist(const Task *tasks, int ntasks, int64_t nblocks,
                                const InstDesc *insts, const uint32_t *start, int64_t nleaves,
                                int tpi, uint32_t *cnt, uint32_t *off, uint32_t *scan_scratch,
                                uint4 *items, uint32_t *ctrl, const P2POrder *order,
                                cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_p2p_count<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, tpi, cnt, ctrl);
    PF_LAUNCHED(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(cnt, off, nleaves, scan_scratch, ctrl + CTRL_NITEMS, st, launches);
    if (e != cudaSuccess) return e;
    uint4 *emit_to = order ? order->items_unsorted : items;
    k_p2p_emit<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, tpi, cnt, off, emit_to,
                                                  order ? order->kA : nullptr);
    PF_LAUNCHED(1);
    if ((e = cudaGetLastError()) != cudaSuccess || !order) return e;
    // heaviest items first: one stable 8-bit radix pass over the work classes
    const int64_t cap = order->cap;
    const unsigned g = unsigned((cap + 255) / 256);
    k_item_tail<<<g, 256, 0, st>>>(order->kA, cap, ctrl);
    PF_LAUNCHED(1);
    bool in_first = true;
    e = radix_sort(order->kA, order->vA, order->kB, order->vB, cap, 8, order->hist, scan_scratch,
                   &in_first, st, launches);
    if (e != cudaSuccess) return e;
    k_item_permute<<<g, 256, 0, st>>>(emit_to, in_first ? order->vA : order->vB, items, cap, ctrl);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Mixed-precision P2P + L2P
// ----------------------------------------------------------------------------
constexpr int P2P_THREADS = 256;

template <int DEG>
__device__ __forceinline__ float poly_eval(const float (&a)[DEG + 1], float s) {
    float g = a[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) g = fmaf(g, s, a[k]);
    return g;
}

template <int DEG, bool GENERAL>
__device__ __forceinline__ float g_of(const float (&a)[DEG + 1], float r2, float kappa, float split) {
    float g = poly_eval<DEG>(a, r2);
    if (GENERAL) {
        const float q = kappa * r2;
        const float ge = __fdividef(1.0f - __expf(-q), q);
        g = r2 < split ? g : ge;
    }
    return g;
}

// One source against the lane's two targets (a, b), both in the source
// leaf's frame.
template <int DEG, bool GENERAL>
__device__ __forceinline__ void pair2(const float4 s, float xa, float ya, float xb, float yb,
                                      const float (&a)[DEG + 1], float kappa, float split,
                                      float &ua, float &va, float &ub, float &vb) {
    const float dxa = xa - s.x, dya = ya - s.y;
    const float dxb = xb - s.x, dyb = yb - s.y;
    const float r2a = fmaf(dxa, dxa, dya * dya);
    const float r2b = fmaf(dxb, dxb, dyb * dyb);
    const float fa = s.z * g_of<DEG, GENERAL>(a, r2a, kappa, split);
    const float fb = s.z * g_of<DEG, GENERAL>(a, r2b, kappa, split);
    ua = fmaf(-dya, fa, ua);
    va = fmaf(dxa, fa, va);
    ub = fmaf(-dyb, fb, ub);
    vb = fmaf(dxb, fb, vb);
}

template <int DEG, bool GENERAL>
__global__ void __launch_bounds__(P2P_THREADS, 5) k_p2p_mixed(
    const uint4 *__restrict__ items, uint32_t *ctrl, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float4 *__restrict__ rec,
    const float2 *__restrict__ le, int dtype_f32, unsigned long long *busy) {
    const int lane = threadIdx.x & 31;
    const uint32_t nitems = *reinterpret_cast<volatile uint32_t *>(ctrl + CTRL_NITEMS);
    const uint64_t t_begin = busy ? global_ns() : 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctrl + CTRL_QUEUE, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const uint4 item = items[it];
        const InstDesc &d = insts[item.x];
        const int L = d.L;
        float a[DEG + 1];
#pragma unroll
        for (int k = 0; k <= DEG; ++k) a[k] = d.poly[k];
        const float kappa = d.kappa, split = d.qsplit_rho2;
        const uint32_t m = item.y;
        const int ix = int(compact_bits(m)), iy = int(compact_bits(m >> 1));
        // lane = (source group grp, target slot k); targets k and k + W
        const int lw = p2p_group_log2(item.w, 2);
        const uint32_t W = 1u << lw, S = 32u >> lw;
        const uint32_t grp = uint32_t(lane) >> lw, k = uint32_t(lane) & (W - 1u);
        const uint32_t ta = item.z + k, tb = item.z + k + W;
        const bool has_a = k < item.w, has_b = k + W < item.w;
        const float4 ra = has_a ? rec[ta] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 rb = has_b ? rec[tb] : make_float4(0.f, 0.f, 0.f, 0.f);
        float ua = 0.f, va = 0.f, ub = 0.f, vb = 0.f;
        const uint32_t *st = start + d.soff;
        const int nside = 1 << L;
        for (int dy = -1; dy <= 1; ++dy) {
            const int sy = iy + dy;
            if (sy < 0 || sy >= nside) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int sx = ix + dx;
                if (sx < 0 || sx >= nside) continue;
                const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
                const uint32_t j0 = st[nm], j1 = st[nm + 1];
                const float xa = ra.x - float(dx), ya = ra.y - float(dy);
                const float xb = rb.x - float(dx), yb = rb.y - float(dy);
                // the stride-1 loop keeps constant load offsets after unrolling
                if (S == 1) {
#pragma unroll 4
                    for (uint32_t j = j0; j < j1; ++j)
                        pair2<DEG, GENERAL>(__ldg(rec + j), xa, ya, xb, yb, a, kappa, split, ua,
                                            va, ub, vb);
                } else {
#pragma unroll 4
                    for (uint32_t j = j0 + grp; j < j1; j += S)
                        pair2<DEG, GENERAL>(__ldg(rec + j), xa, ya, xb, yb, a, kappa, split, ua,
                                            va, ub, vb);
                }
            }
        }
        // add the partial sums of the source groups (fixed butterfly)
        for (uint32_t o = W; o < 32u; o <<= 1) {
            ua += __shfl_xor_sync(0xffffffffu, ua, int(o));
            va += __shfl_xor_sync(0xffffffffu, va, int(o));
            ub += __shfl_xor_sync(0xffffffffu, ub, int(o));
            vb += __shfl_xor_sync(0xffffffffu, vb, int(o));
        }
        // far field: L2P of the leaf's local expansion, w = (1/r) sum c_m zeta^m
        float fua = 0.f, fva = 0.f, fub = 0.f, fvb = 0.f;
        if (L >= 2) {
            const int p = d.p;
            const float2 *c = le + d.eoff + (lvl_off(L) + box_index(L, uint32_t(ix), uint32_t(iy))) * p;
            float2 wa = __ldg(c + p - 1), wb = wa;
            for (int k = p - 2; k >= 0; --k) {
                const float2 ck = __ldg(c + k);
                const float wax = fmaf(wa.x, ra.x, fmaf(-wa.y, ra.y, ck.x));
                const float way = fmaf(wa.x, ra.y, fmaf(wa.y, ra.x, ck.y));
                const float wbx = fmaf(wb.x, rb.x, fmaf(-wb.y, rb.y, ck.x));
                const float wby = fmaf(wb.x, rb.y, fmaf(wb.y, rb.x, ck.y));
                wa = make_float2(wax, way);
                wb = make_float2(wbx, wby);
            }
            fua = d.cfar * wa.y; fva = d.cfar * wa.x;
            fub = d.cfar * wb.y; fvb = d.cfar * wb.x;
        }
        const float cn = d.cnear;
        if (has_a && grp == 0) {
            const int64_t q = int64_t(__float_as_uint(ra.w)) - d.poff;
            const float uo = fmaf(cn, ua, fua), vo = fmaf(cn, va, fva);
            if (dtype_f32) {
                static_cast<float *>(d.u)[q] = uo;
                static_cast<float *>(d.v)[q] = vo;
            } else {
                static_cast<double *>(d.u)[q] = double(uo);
                static_cast<double *>(d.v)[q] = double(vo);
            }
        }
        if (has_b && grp == 0) {
            const int64_t q = int64_t(__float_as_uint(rb.w)) - d.poff;
            const float uo = fmaf(cn, ub, fub), vo = fmaf(cn, vb, fvb);
            if (dtype_f32) {
                static_cast<float *>(d.u)[q] = uo;
                static_cast<float *>(d.v)[q] = vo;
            } else {
                static_cast<double *>(d.u)[q] = double(uo);
                static_cast<double *>(d.v)[q] = double(vo);
            }
        }
    }
    if (busy && lane == 0) {
        const uint64_t t_end = global_ns();
        const size_t gw = size_t(blockIdx.x) * (P2P_THREADS / 32) + (threadIdx.x >> 5);
        busy[2 * gw] = t_begin;
        busy[2 * gw + 1] = t_end;
    }
}

// ----------------------------------------------------------------------------
// FP64 P2P + L2P (one target per lane).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_f64(
    const uint4 *__restrict__ items, uint32_t *ctrl, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const double *__restrict__ xs,
    const double *__restrict__ ys, const double *__restrict__ gs, const uint32_t *__restrict__ perm,
    const double2 *__restrict__ le, int dtype_f32, unsigned long long *busy) {
    const int lane = threadIdx.x & 31;
    const uint32_t nitems = *reinterpret_cast<volatile uint32_t *>(ctrl + CTRL_NITEMS);
    const uint64_t t_begin = busy ? global_ns() : 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctrl + CTRL_QUEUE, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const uint4 item = items[it];
        const InstDesc &d = insts[item.x];
        const int L = d.L;
        const uint32_t m = item.y;
        const int ix = int(compact_bits(m)), iy = int(compact_bits(m >> 1));
        const int lw = p2p_group_log2(item.w, 1);
        const uint32_t W = 1u << lw, S = 32u >> lw;
        const uint32_t grp = uint32_t(lane) >> lw, k = uint32_t(lane) & (W - 1u);
        const bool has = k < item.w;
        const uint32_t ti = item.z + (has ? k : 0u);
        const double x = xs[ti], y = ys[ti];
        const double inv2s2 = d.inv2s2;
        double su = 0.0, sv = 0.0;
        const uint32_t *st = start + d.soff;
        const int nside = 1 << L;
        for (int dy = -1; dy <= 1; ++dy) {
            const int sy = iy + dy;
            if (sy < 0 || sy >= nside) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int sx = ix + dx;
                if (sx < 0 || sx >= nside) continue;
                const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
                const uint32_t j0 = st[nm], j1 = st[nm + 1];
                for (uint32_t j = j0 + grp; j < j1; j += S) {
                    const double ddx = x - __ldg(xs + j), ddy = y - __ldg(ys + j);
                    const double r2 = ddx * ddx + ddy * ddy;
                    if (r2 > 0.0) {
                        const double f = __ldg(gs + j) * (-expm1(-r2 * inv2s2) / r2);
                        su += -ddy * f;
                        sv += ddx * f;
                    }
                }
            }
        }
        for (uint32_t o = W; o < 32u; o <<= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, int(o));
            sv += __shfl_xor_sync(0xffffffffu, sv, int(o));
        }
        double fu = 0.0, fv = 0.0;
        if (L >= 2) {
            const int p = d.p;
            const double cx = d.x0 + (double(ix) + 0.5) * d.wleaf;
            const double cy = d.y0 + (double(iy) + 0.5) * d.wleaf;
            const double zx = (x - cx) * d.scale, zy = (y - cy) * d.scale;
            const double2 *c = le + d.eoff + (lvl_off(L) + box_index(L, uint32_t(ix), uint32_t(iy))) * p;
            double2 w = c[p - 1];
            for (int k = p - 2; k >= 0; --k) {
                const double2 ck = c[k];
                const double wx = w.x * zx - w.y * zy + ck.x;
                const double wy = w.x * zy + w.y * zx + ck.y;
                w = make_double2(wx, wy);
            }
            fu = d.cfar64 * w.y;
            fv = d.cfar64 * w.x;
        }
        if (has && grp == 0) {
            const int64_t q = int64_t(perm[ti]) - d.poff;
            const double uo = su * d.cnear64 + fu, vo = sv * d.cnear64 + fv;
            if (dtype_f32) {
                static_cast<float *>(d.u)[q] = float(uo);
                static_cast<float *>(d.v)[q] = float(vo);
            } else {
                static_cast<double *>(d.u)[q] = uo;
                static_cast<double *>(d.v)[q] = vo;
            }
        }
    }
    if (busy && lane == 0) {
        const uint64_t t_end = global_ns();
        const size_t gw = size_t(blockIdx.x) * (P2P_THREADS / 32) + (threadIdx.x >> 5);
        busy[2 * gw] = t_begin;
        busy[2 * gw + 1] = t_end;
    }
}

// ----------------------------------------------------------------------------
// Launch helpers
// ----------------------------------------------------------------------------
typedef void (*MixedKernel)(const uint4 *, uint32_t *, const InstDesc *, const uint32_t *,
                            const float4 *, const float2 *, int, unsigned long long *);
template <int D>
static MixedKernel pick2(int general) {
    return general ? k_p2p_mixed<D, true> : k_p2p_mixed<D, false>;
}

static MixedKernel pick_mixed(int deg, int general) {
    switch (deg) {
        case 4: return pick2<4>(general);
        case 5: return pick2<5>(general);
        case 6: return pick2<6>(general);
        case 7: return pick2<7>(general);
        case 8: return pick2<8>(general);
        case 9: return pick2<9>(general);
        case 10: return pick2<10>(general);
        case 11: return pick2<11>(general);
        case 12: return pick2<12>(general);
        default: return nullptr;
    }
}

static int g_sms = 0;

int device_sm_count() {
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

int p2p_grid(int precision_mixed, int deg, int general) {
    int per_sm = 1;
    if (precision_mixed) {
        MixedKernel k = pick_mixed(deg, general);
        if (!k) return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, P2P_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p_f64, P2P_THREADS, 0);
    }
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sm_count();
}

cudaError_t launch_p2p_mixed(int grid, int deg, int general, const uint4 *items, uint32_t *ctrl,
                             const InstDesc *insts, const uint32_t *start, const float4 *rec,
                             const float2 *le, int dtype_f32, unsigned long long *busy,
                             cudaStream_t st, uint64_t *launches) {
    MixedKernel k = pick_mixed(deg, general);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, P2P_THREADS, 0, st>>>(items, ctrl, insts, start, rec, le, dtype_f32, busy);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

cudaError_t launch_p2p_f64(int grid, const uint4 *items, uint32_t *ctrl, const InstDesc *insts,
                           const uint32_t *start, const double *xs, const double *ys,
                           const double *gs, const uint32_t *perm, const double2 *le,
                           int dtype_f32, unsigned long long *busy, cudaStream_t st,
                           uint64_t *launches) {
    k_p2p_f64<<<grid, P2P_THREADS, 0, st>>>(items, ctrl, insts, start, xs, ys, gs, perm, le,
                                            dtype_f32, busy);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

}  // namespace petfmm
