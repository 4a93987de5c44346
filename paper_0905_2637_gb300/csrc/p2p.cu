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

// Forward neighbours of a leaf in the pairwise near field (see below).
__constant__ int8_t c_fwd[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};

// A pair of neighbouring leaves is evaluated pairwise when both hold at least
// a warp's worth of blobs; with fewer, most lanes of the 64 x 32 tile would
// idle, and the leaves' own warps sum that neighbour directly instead.  Both
// leaves of a pair decide from the same two counts.
constexpr uint32_t P2P_PAIR_MIN = 32;
__host__ __device__ __forceinline__ bool pairwise(uint32_t na, uint32_t nb) {
    return na >= P2P_PAIR_MIN && nb >= P2P_PAIR_MIN;
}

// A heavy pair is cut into pieces along A, each piece a run of whole
// 128-target chunks holding at most P2P_PAIR_CAPU tiles of 128 targets x 32
// sources, so that no single warp's item outlasts the average share of the
// launch.  Piece 0 writes B's reaction to the pair's slot, piece i >= 1 to a
// scratch run of nb entries; the final pass adds them in piece order.
// Returns the number of pieces; *pc = targets per piece (a multiple of 128).
constexpr uint64_t P2P_PAIR_CAPU = 256;
__host__ __device__ __forceinline__ uint32_t pair_pieces(uint32_t na, uint32_t nb, uint32_t *pc) {
    const uint32_t ca = (na + 127) / 128, cb = (nb + 31) / 32;
    uint64_t np = (uint64_t(ca) * cb + P2P_PAIR_CAPU - 1) / P2P_PAIR_CAPU;
    if (np > ca) np = ca;
    if (np < 1) np = 1;
    const uint32_t per = uint32_t((ca + np - 1) / np);
    *pc = per * 128;
    return (ca + per - 1) / per;
}

// count of the leaf (x, y), 0 outside the domain
__device__ __forceinline__ uint32_t leaf_count(const uint32_t *st, int nside, int x, int y) {
    if (x < 0 || y < 0 || x >= nside || y >= nside) return 0;
    const uint32_t m = morton_key(uint32_t(x), uint32_t(y));
    return st[m + 1] - st[m];
}

// Whether a leaf (n blobs, at ix, iy) has directed near-field work in the
// pairwise mode: its own blobs when it is too small for the pair kernel, or
// an occupied neighbour the pair kernel does not cover.
__device__ __forceinline__ bool directed_work(const uint32_t *st, int nside, int ix, int iy,
                                              uint32_t n) {
    if (!pairwise(n, n)) return n > 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const uint32_t nb = leaf_count(st, nside, ix + dx, iy + dy);
            if (nb && !pairwise(n, nb)) return true;
        }
    return false;
}

// Per-leaf flags of the pairwise mode, read by the final pass: which result
// slots hold this leaf's blobs' sums.
enum : uint32_t {
    LF_FWD = 1u,        // << k: pairs with forward neighbour k (slot k)
    LF_BWD = 16u,       // << k: pairs with backward neighbour k (slot 4 + k)
    LF_SPLIT = 256u,    // << k: ... cut into pieces, partial sums in the scratch
    LF_SELF = 4096u,    // the leaf's own pairs (slot 8)
    LF_DIRECTED = 8192u // directed items (own[])
};

__global__ void __launch_bounds__(256) k_p2p_count(const Task *__restrict__ tasks, int ntasks,
                                                   const InstDesc *__restrict__ insts,
                                                   const uint32_t *__restrict__ start, int tpi,
                                                   int pairs_mode, uint32_t *__restrict__ cnt,
                                                   uint32_t *ctrl) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    unsigned long long pairs = 0;
    if (m < t.count) {
        const InstDesc &d = insts[t.inst];
        const uint32_t *st = start + d.soff;
        const uint32_t n = st[m + 1] - st[m];
        const int nside = 1 << d.L;
        const int ix = int(compact_bits(uint32_t(m))), iy = int(compact_bits(uint32_t(m) >> 1));
        // pairwise mode: items only for the leaves with directed work
        const bool work = pairs_mode ? directed_work(st, nside, ix, iy, n) : n > 0;
        cnt[d.loff + m] = work ? (n + tpi - 1) / tpi : 0u;
        if (n) {
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
__global__ void __launch_bounds__(256) k_item_permute(const uint4 *__restrict__ in,
                                                      const uint32_t *__restrict__ perm,
                                                      uint4 *__restrict__ out, int64_t cap,
                                                      const uint32_t *count) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r < cap && r < int64_t(*count) && PF_IN(perm[r], cap)) out[r] = in[perm[r]];
}

// heaviest items first: one stable 8-bit radix pass over the work classes in
// order->kA, then the items permuted from order->items_unsorted to items
static cudaError_t order_items(const P2POrder *order, uint4 *items, const uint32_t *count,
                               uint32_t *scan_scratch, cudaStream_t st, uint64_t *launches) {
    const int64_t cap = order->cap;
    const unsigned g = unsigned((cap + 255) / 256);
    bool in_first = true;
    cudaError_t e = radix_sort(order->kA, order->vA, order->kB, order->vB, cap, 8, order->hist,
                               &in_first, st, launches, count);
    if (e != cudaSuccess) return e;
    k_item_permute<<<g, 256, 0, st>>>(order->items_unsorted, in_first ? order->vA : order->vB,
                                      items, cap, count);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

cudaError_t launch_p2p_worklist(const Task *tasks, int ntasks, int64_t nblocks,
                                const InstDesc *insts, const uint32_t *start, int64_t nleaves,
                                int tpi, int pairs_mode, uint32_t *cnt, uint32_t *off,
                                uint32_t *scan_scratch, uint4 *items, uint32_t *ctrl,
                                const P2POrder *order, cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_p2p_count<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, tpi, pairs_mode,
                                                   cnt, ctrl);
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
    return order_items(order, items, ctrl + CTRL_NITEMS, scan_scratch, st, launches);
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

// One work item of the directed near field: up to 64 targets of a leaf
// against the leaf and its neighbours (PAIRS: not the neighbours the pair
// kernel covers); the near sum goes to own[] in sorted order, the final pass
// adds the far field.  No L2P here: with few targets per item the lanes of
// all source groups would repeat it.
// Laplace kernel: one source against the lane's two targets, both in the
// source leaf's frame (leaf units): u += q (log rho + log w), i.e. q log r in
// global units; coincident pairs add nothing.
__device__ __forceinline__ void pair2_lap(const float4 s, float xa, float ya, float xb, float yb,
                                          float logw, float &ua, float &ub) {
    const float dxa = xa - s.x, dya = ya - s.y;
    const float dxb = xb - s.x, dyb = yb - s.y;
    const float r2a = fmaf(dxa, dxa, dya * dya);
    const float r2b = fmaf(dxb, dxb, dyb * dyb);
    const float la = r2a > 0.f ? fmaf(0.5f, __logf(r2a), logw) : 0.f;
    const float lb = r2b > 0.f ? fmaf(0.5f, __logf(r2b), logw) : 0.f;
    ua = fmaf(s.z, la, ua);
    ub = fmaf(s.z, lb, ub);
}

template <int DEG, bool GENERAL, bool PAIRS, bool LAP>
__device__ __forceinline__ void directed_item(const uint4 item, const InstDesc *__restrict__ insts,
                                              const uint32_t *__restrict__ start,
                                              const float4 *__restrict__ rec,
                                              float2 *__restrict__ own, int lane) {
    const InstDesc &d = insts[item.x];
    const int L = d.L;
    float a[DEG + 1];
#pragma unroll
    for (int k = 0; k <= DEG; ++k) a[k] = d.poly[k];
    const float kappa = d.kappa, split = d.qsplit_rho2;
    const uint32_t m = item.y;
    // checked build: the item's leaf and target range lie inside the instance
    if (!(PF_IN(m, int64_t(1) << (2 * L)) && PF_IN(int64_t(item.z) - d.poff, d.n + 1) &&
          PF_IN(int64_t(item.z) + item.w - d.poff, d.n + 1)))
        return;
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
    const float logw = LAP ? float(d.logw0 - double(L) * 0.69314718055994530942) : 0.f;
    // The pairwise mode's directed items (small leaves, leftover neighbours)
    // and the Laplace kernel's are mostly short: lanes 0..8 fetch the 9
    // leaves' source ranges at once (lane q: offset (q % 3 - 1, q / 3 - 1)),
    // so an item pays one load latency, not nine.  The directed-only vortex
    // mode (long items) keeps the plain loop, which measured faster there.
    constexpr bool FETCH9 = PAIRS || LAP;
    uint32_t lj0 = 0, lj1 = 0;
    if (FETCH9 && lane < 9) {
        const int sx = ix + lane % 3 - 1, sy = iy + lane / 3 - 1;
        if (sx >= 0 && sy >= 0 && sx < nside && sy < nside) {
            const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
            lj0 = st[nm];
            lj1 = st[nm + 1];
        }
    }
    const uint32_t nme = PAIRS ? st[m + 1] - st[m] : 0u;
    for (int q = 0; q < 9; ++q) {
        const int dx = q % 3 - 1, dy = q / 3 - 1;
        uint32_t j0, j1;
        if (FETCH9) {
            j0 = __shfl_sync(0xffffffffu, lj0, q);
            j1 = __shfl_sync(0xffffffffu, lj1, q);
        } else {
            const int sx = ix + dx, sy = iy + dy;
            if (sx < 0 || sy < 0 || sx >= nside || sy >= nside) continue;
            const uint32_t nm = morton_key(uint32_t(sx), uint32_t(sy));
            j0 = st[nm];
            j1 = st[nm + 1];
        }
        if (j0 == j1) continue;
        {
            // pairwise mode: the leaves the pair kernel covers (the leaf itself
            // included) are skipped
            if (PAIRS && pairwise(nme, j1 - j0)) continue;
            const float xa = ra.x - float(dx), ya = ra.y - float(dy);
            const float xb = rb.x - float(dx), yb = rb.y - float(dy);
            // the stride-1 loop keeps constant load offsets after unrolling
            if (S == 1) {
#pragma unroll 4
                for (uint32_t j = j0; j < j1; ++j) {
                    if constexpr (LAP)
                        pair2_lap(__ldg(rec + j), xa, ya, xb, yb, logw, ua, ub);
                    else
                        pair2<DEG, GENERAL>(__ldg(rec + j), xa, ya, xb, yb, a, kappa, split, ua,
                                            va, ub, vb);
                }
            } else {
#pragma unroll 4
                for (uint32_t j = j0 + grp; j < j1; j += S) {
                    if constexpr (LAP)
                        pair2_lap(__ldg(rec + j), xa, ya, xb, yb, logw, ua, ub);
                    else
                        pair2<DEG, GENERAL>(__ldg(rec + j), xa, ya, xb, yb, a, kappa, split, ua,
                                            va, ub, vb);
                }
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
    const float cn = LAP ? 1.f : d.cnear;
    if (has_a && grp == 0) own[ta] = make_float2(cn * ua, cn * va);
    if (has_b && grp == 0) own[tb] = make_float2(cn * ub, cn * vb);
}

template <int DEG, bool GENERAL, bool PAIRS, bool LAP>
__global__ void __launch_bounds__(P2P_THREADS, 5) k_p2p_mixed(
    const uint4 *__restrict__ items, uint32_t *ctrl, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float4 *__restrict__ rec,
    float2 *__restrict__ own, unsigned long long *busy) {
    const int lane = threadIdx.x & 31;
    const uint32_t nitems = *reinterpret_cast<volatile uint32_t *>(ctrl + CTRL_NITEMS);
    const uint64_t t_begin = busy ? global_ns() : 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctrl + CTRL_QUEUE, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        directed_item<DEG, GENERAL, PAIRS, LAP>(items[it], insts, start, rec, own, lane);
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
        // Laplace kernel: su = sum q_j log|x - x_j| (coincident pairs excluded)
        const bool lap = d.kernel == KERNEL_LAPLACE;
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
                        if (lap) {
                            su += __ldg(gs + j) * (0.5 * log(r2));
                        } else {
                            const double f = __ldg(gs + j) * (-expm1(-r2 * inv2s2) / r2);
                            su += -ddy * f;
                            sv += ddx * f;
                        }
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
            if (lap) {
                fu = w.x;  // the potential is Re of the local expansion
            } else {
                fu = d.cfar64 * w.y;
                fv = d.cfar64 * w.x;
            }
        }
        if (has && grp == 0) {
            const int64_t q = int64_t(perm[ti]) - d.poff;
            const double uo = lap ? su + fu : su * d.cnear64 + fu;
            const double vo = lap ? 0.0 : sv * d.cnear64 + fv;
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
// Pairwise near field between neighbouring leaves (mixed path).
//
// Each unordered pair {A, B} of neighbouring occupied leaves is evaluated
// once, by the item (A, d) with B = A + off[d] one of A's four forward
// neighbours.  One warp holds up to 64 targets of A (two per lane) and 32
// sources of B (one per lane); in 32 steps the sources travel once around
// the warp (shuffles), and for every (target, source) pair the kernel factor
// K(x_a - x_s) is computed once and used twice: gamma_s K for the target and
// -gamma_a K for the source (K is odd, Eq. 8), the latter summed in a register
// that travels with the source.  The sums go to single-owner slots of the
// receiving particle: part[d][a] (from the forward neighbour d) and
// part[4 + d][b] (from the backward neighbour); the 64-target chunks of A
// add to a source's slot one after another in the same warp.  A final pass
// adds, per particle, its own leaf's sum and far field and the slots of its
// occupied neighbours in a fixed order: the result does not depend on which
// warp ran which item.
// ----------------------------------------------------------------------------

// cnt[leaf] = forward neighbours of an occupied leaf that hold particles
__global__ void __launch_bounds__(256) k_pair_count(const Task *__restrict__ tasks, int ntasks,
                                                    const InstDesc *__restrict__ insts,
                                                    const uint32_t *__restrict__ start,
                                                    uint32_t *__restrict__ cnt,
                                                    uint32_t *__restrict__ xcnt,
                                                    uint32_t *ctrl) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    unsigned long long sym = 0;
    if (m < t.count) {
        const InstDesc &d = insts[t.inst];
        const uint32_t *st = start + d.soff;
        uint32_t c = 0, x = 0;
        const uint32_t na = st[m + 1] - st[m];
        if (na >= P2P_PAIR_MIN) {
            const int nside = 1 << d.L;
            const int ix = int(compact_bits(uint32_t(m))), iy = int(compact_bits(uint32_t(m) >> 1));
            for (int k = 0; k < 4; ++k) {
                const uint32_t nb = leaf_count(st, nside, ix + c_fwd[k][0], iy + c_fwd[k][1]);
                if (!pairwise(na, nb)) continue;
                uint32_t pc;
                const uint32_t np = pair_pieces(na, nb, &pc);
                c += np;
                x += (np - 1) * nb;
                sym += (unsigned long long)na * nb;
            }
            // the leaf's own pairs: one item
            c += 1;
            sym += (unsigned long long)na * (na - 1) / 2;
        }
        cnt[d.loff + m] = c;
        xcnt[d.loff + m] = x;
    }
    // block reduction of the unordered pair count (for the statistics)
#pragma unroll
    for (int o = 16; o; o >>= 1) sym += __shfl_down_sync(0xffffffffu, sym, o);
    __shared__ unsigned long long ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sym;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        if (s) atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + CTRL_SYM_LO), s);
    }
}

// items (inst, leaf A, direction d, 0) and their work class (targets x
// sources, log2 in quarter steps, stored as 127 - class: heaviest first)
// Estimated time of nt targets against ns sources in the pair kernel: the
// target chunks it cuts (320/256/128/64/32, see pair_leaves) weighted by
// their measured time per source step (10 and 8 packed, 4 packed, 2 and 1
// targets per lane: 12.1, 10.3, 5.6, 3.4 and 2.5 relative units), times the
// source steps (32 per chunk of 32, 16 for a last chunk of at most 16).
__device__ __forceinline__ uint32_t pair_cost(uint32_t nt, uint32_t ns) {
    uint32_t c = 0;
    for (uint32_t r = nt; r > 0;) {
        if (r >= 257) { c += 121; r = r > 320 ? r - 320 : 0; }
        else if (r >= 192) { c += 103; r = r > 256 ? r - 256 : 0; }
        else if (r >= 96) { c += 56; r = r > 128 ? r - 128 : 0; }
        else if (r >= 33) { c += 34; r = r > 64 ? r - 64 : 0; }
        else { c += 25; r = r > 32 ? r - 32 : 0; }
    }
    const uint32_t tail = ns & 31u;
    return c * ((ns & ~31u) + (tail == 0 ? 0u : tail <= 16 ? 16u : 32u));
}

// work class of an item of `cost` (64-target chunk, 32-source chunk) tiles:
// heaviest first = smallest class, quarter steps of log2
__device__ __forceinline__ uint32_t pair_wclass(uint32_t cost) {
    if (cost < 1) cost = 1;
    const int e = 31 - __clz(int(cost));
    const uint32_t frac = e >= 2 ? (cost >> (e - 2)) & 3u : (cost << (2 - e)) & 3u;
    return 127u - (uint32_t(e) * 4u + frac);
}

__global__ void __launch_bounds__(256) k_pair_emit(const Task *__restrict__ tasks, int ntasks,
                                                   const InstDesc *__restrict__ insts,
                                                   const uint32_t *__restrict__ start,
                                                   const uint32_t *__restrict__ off,
                                                   const uint32_t *__restrict__ xoff,
                                                   const uint32_t *__restrict__ ctrl,
                                                   int64_t xcap, uint32_t *__restrict__ xtab,
                                                   uint32_t *__restrict__ lflags,
                                                   uint4 *__restrict__ items,
                                                   uint32_t *__restrict__ wclass) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t m = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (m >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const uint32_t *st = start + d.soff;
    const uint32_t na = st[m + 1] - st[m];
    const int nside = 1 << d.L;
    const int ix = int(compact_bits(uint32_t(m))), iy = int(compact_bits(uint32_t(m) >> 1));
    // the pieces' scratch runs exist only if all of them fit; else every pair
    // is one piece (decided alike for all pairs, so the result does not depend
    // on which fit)
    const bool split = int64_t(ctrl[CTRL_NXTRA]) <= xcap;
    // this leaf's flags for the final pass
    uint32_t fl = directed_work(st, nside, ix, iy, na) ? LF_DIRECTED : 0u;
    if (na >= P2P_PAIR_MIN) {
        fl |= LF_SELF;
        for (int k = 0; k < 4; ++k) {
            if (pairwise(na, leaf_count(st, nside, ix + c_fwd[k][0], iy + c_fwd[k][1])))
                fl |= LF_FWD << k;
            const uint32_t nbk = leaf_count(st, nside, ix - c_fwd[k][0], iy - c_fwd[k][1]);
            if (pairwise(nbk, na)) {
                fl |= LF_BWD << k;
                uint32_t pc;
                if (split && pair_pieces(nbk, na, &pc) > 1) fl |= LF_SPLIT << k;
            }
        }
    }
    lflags[d.loff + m] = fl;
    if (na < P2P_PAIR_MIN) return;
    uint32_t o = off[d.loff + m], xb = xoff[d.loff + m];
    for (int k = 0; k < 4; ++k) {
        const uint32_t nb = leaf_count(st, nside, ix + c_fwd[k][0], iy + c_fwd[k][1]);
        if (!pairwise(na, nb)) continue;
        uint32_t pc;
        const uint32_t np = pair_pieces(na, nb, &pc);
        const uint32_t base = split ? xb : 0xffffffffu;
        if (np > 1) xtab[(d.loff + m) * 4 + k] = base;
        // a pair in one piece runs with the leaf that pads less as targets
        const uint32_t swap = np == 1 && pair_cost(nb, na) < pair_cost(na, nb) ? 1u : 0u;
        for (uint32_t i = 0; i < np; ++i) {
            items[o] = make_uint4(uint32_t(t.inst), uint32_t(m),
                                  uint32_t(k) | (swap << 3) | (i << 4), base);
            if (wclass) {
                // a warp spends 32 steps per (64-target chunk, 32-source chunk)
                const uint32_t nt = split ? min(pc, na - i * pc) : (i ? 0u : na);
                wclass[o] = pair_wclass(((nt + 63) / 64) * ((nb + 31) / 32));
            }
            ++o;
        }
        xb += (np - 1) * nb;
    }
    // the leaf's own pairs (direction 4): half the tiles of the leaf with itself
    items[o] = make_uint4(uint32_t(t.inst), uint32_t(m), 4u, 0u);
    if (wclass) wclass[o] = pair_wclass(((na + 63) / 64) * ((na + 31) / 32) / 2);
}

// One target (in A's frame) against the travelling source (already in A's
// frame): the target gains gs K, the source -ga K.
template <int DEG, bool GENERAL>
__device__ __forceinline__ void pair_sym(float xa, float ya, float ga, float xs, float ys, float gs,
                                         const float (&a)[DEG + 1], float kappa, float split,
                                         float &ua, float &va, float &bu, float &bv) {
    const float dx = xa - xs, dy = ya - ys;
    const float r2 = fmaf(dx, dx, dy * dy);
    const float g = g_of<DEG, GENERAL>(a, r2, kappa, split);
    const float kx = -dy * g, ky = dx * g;
    ua = fmaf(gs, kx, ua);
    va = fmaf(gs, ky, va);
    bu = fmaf(-ga, kx, bu);
    bv = fmaf(-ga, ky, bv);
}

// placeholders of missing targets / sources: far apart (finite kernel
// values), zero strength (they add nothing and their sums are dropped)
constexpr float kPairFar = 64.f;

// p[0] = w, or p[0] += w
__device__ __forceinline__ void put2(float2 *p, float2 w, bool add) {
    if (add) {
        const float2 o = *p;
        w = make_float2(o.x + w.x, o.y + w.y);
    }
    *p = w;
}

// One pass of a source chunk around the warp: W = 32 sources, one per lane,
// or W = 16 (a tail of at most 16 sources held by both half-warps, each half
// rotating its own copy).  Each step every lane evaluates its TPL targets
// against the source it holds, the source's reaction sum travelling with it;
// after W steps every sum is back at its source's lane (for W = 16 the two
// halves' sums are then added).
template <int DEG, bool GENERAL, int TPL, int W>
__device__ __forceinline__ void source_pass(const float (&tx)[TPL], const float (&ty)[TPL],
                                            const float (&tg)[TPL], float (&u)[TPL],
                                            float (&v)[TPL], const float (&a)[DEG + 1],
                                            float kappa, float split, float xs, float ys,
                                            float gs, float &bu, float &bv, int lane) {
    const int next = (lane & ~(W - 1)) | ((lane + 1) & (W - 1));
    bu = 0.f;
    bv = 0.f;
#pragma unroll 2
    for (int k = 0; k < W; ++k) {
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            pair_sym<DEG, GENERAL>(tx[t], ty[t], tg[t], xs, ys, gs, a, kappa, split, u[t], v[t], bu,
                                   bv);
        xs = __shfl_sync(0xffffffffu, xs, next);
        ys = __shfl_sync(0xffffffffu, ys, next);
        gs = __shfl_sync(0xffffffffu, gs, next);
        bu = __shfl_sync(0xffffffffu, bu, next);
        bv = __shfl_sync(0xffffffffu, bv, next);
    }
    if (W < 32) {
        bu += __shfl_xor_sync(0xffffffffu, bu, 16);
        bv += __shfl_xor_sync(0xffffffffu, bv, 16);
    }
}

// The same pass with 2 H targets per lane held as H pairs and evaluated with
// packed FP32x2 instructions (polynomial near-field factor only): the same
// products per pair as source_pass, each packed instruction doing two of
// them, so half the issue slots.  The reaction sums of a step run in the two
// halves of a pair and are added before the source moves on.  Signs are
// folded out of the loop: the source travels as (-x, -y), the targets keep
// U = -u and the reaction BV = -bv (round-to-nearest is symmetric in sign,
// so the sums are bit for bit the negated ones), which saves the negated
// copies of the strengths and one broadcast per step.
template <int DEG, int H, int W>
__device__ __forceinline__ void source_pass_x2(const float2 (&tx)[H], const float2 (&ty)[H],
                                               const float2 (&tg)[H], float2 (&U)[H],
                                               float2 (&v)[H], const float2 (&a2)[DEG + 1],
                                               float nxs, float nys, float gs, float &bu,
                                               float &BV, int lane) {
    const int next = (lane & ~(W - 1)) | ((lane + 1) & (W - 1));
    bu = 0.f;
    BV = 0.f;
#pragma unroll 2
    for (int k = 0; k < W; ++k) {
        // with K = (-dy, dx) g: u_a += g_s K, reaction u_b -= g_a K
        const float2 nx = make_float2(nxs, nxs), ny = make_float2(nys, nys);
        const float2 g2 = make_float2(gs, gs);
        float2 bu2 = make_float2(bu, 0.f), bv2 = make_float2(BV, 0.f);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float2 dx = __fadd2_rn(tx[h], nx), dy = __fadd2_rn(ty[h], ny);
            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            float2 g = a2[DEG];
#pragma unroll
            for (int q = DEG - 1; q >= 0; --q) g = __ffma2_rn(g, r2, a2[q]);
            const float2 py = __fmul2_rn(dy, g), px = __fmul2_rn(dx, g);
            U[h] = __ffma2_rn(g2, py, U[h]);
            v[h] = __ffma2_rn(g2, px, v[h]);
            bu2 = __ffma2_rn(tg[h], py, bu2);
            bv2 = __ffma2_rn(tg[h], px, bv2);
        }
        bu = bu2.x + bu2.y;
        BV = bv2.x + bv2.y;
        nxs = __shfl_sync(0xffffffffu, nxs, next);
        nys = __shfl_sync(0xffffffffu, nys, next);
        gs = __shfl_sync(0xffffffffu, gs, next);
        bu = __shfl_sync(0xffffffffu, bu, next);
        BV = __shfl_sync(0xffffffffu, BV, next);
    }
    if (W < 32) {
        bu += __shfl_xor_sync(0xffffffffu, bu, 16);
        BV += __shfl_xor_sync(0xffffffffu, BV, 16);
    }
}

// Source chunk bc of B as seen by this lane: the source it starts with (in
// A's frame; placeholders past the end) and whether the chunk is a tail of
// at most 16 (half-warp pass).
struct SourceSlot {
    float xs, ys, gs;
    uint32_t sb;
    bool hs, half;
};
__device__ __forceinline__ SourceSlot source_slot(const float4 *__restrict__ rec, uint32_t b0,
                                                  uint32_t bc, uint32_t nb, int ox, int oy,
                                                  int lane) {
    // the next chunk's records into L1 while this one is evaluated
    if (bc + 32 + uint32_t(lane) < nb)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(rec + b0 + bc + 32 + lane));
    SourceSlot o;
    o.half = nb - bc <= 16;
    o.sb = bc + uint32_t(o.half ? (lane & 15) : lane);
    o.hs = o.sb < nb;
    const float4 s = o.hs ? rec[b0 + o.sb] : make_float4(-kPairFar, -kPairFar, 0.f, 0.f);
    // B's centre is A's plus (ox, oy) leaves
    o.xs = s.x + float(ox);
    o.ys = s.y + float(oy);
    o.gs = s.z;
    return o;
}

// One chunk of a leaf pair: targets ac .. min(ac + 32 TPL, aend) - 1 of leaf A
// (TPL per lane: lane + 32 t) against all nb sources of leaf B, B in chunks
// of 32 sources travelling around the warp with their reaction sums (a last
// chunk of at most 16 in a half-warp pass).  fwd[i]: A's blob i from B;
// bwd[j]: B's blob j from A (bwd_add / fwd_add: the chunk adds to them, else
// writes).
template <int DEG, bool GENERAL, int TPL>
__device__ __noinline__ void pair_chunk(const float4 *__restrict__ rec, uint32_t a0,
                                        uint32_t ac, uint32_t aend, uint32_t b0, uint32_t nb,
                                        int ox, int oy, const float (&a)[DEG + 1], float kappa,
                                        float split, float cn, float2 *fwd, float2 *bwd,
                                        bool bwd_add, bool fwd_add, int lane) {
    float tx[TPL], ty[TPL], tg[TPL], u[TPL], v[TPL];
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const bool h = ac + lane + 32 * t < aend;
        const float4 r =
            h ? rec[a0 + ac + lane + 32 * t] : make_float4(kPairFar, kPairFar, 0.f, 0.f);
        tx[t] = r.x;
        ty[t] = r.y;
        tg[t] = r.z;
        u[t] = v[t] = 0.f;
    }
    for (uint32_t bc = 0; bc < nb; bc += 32) {
        const SourceSlot ss = source_slot(rec, b0, bc, nb, ox, oy, lane);
        float bu, bv;
        if (ss.half)
            source_pass<DEG, GENERAL, TPL, 16>(tx, ty, tg, u, v, a, kappa, split, ss.xs, ss.ys,
                                               ss.gs, bu, bv, lane);
        else
            source_pass<DEG, GENERAL, TPL, 32>(tx, ty, tg, u, v, a, kappa, split, ss.xs, ss.ys,
                                               ss.gs, bu, bv, lane);
        if (ss.hs && (!ss.half || lane < 16))
            put2(bwd + ss.sb, make_float2(cn * bu, cn * bv), bwd_add);
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t)
        if (ac + lane + 32 * t < aend)
            put2(fwd + ac + lane + 32 * t, make_float2(cn * u[t], cn * v[t]), fwd_add);
}

// The same chunk with 2 H targets per lane held as H pairs (targets lane +
// 64 h and lane + 64 h + 32), evaluated by source_pass_x2 (which keeps -u
// and the reaction's -v; the signs are restored on the way out).
template <int DEG, int H>
__device__ __noinline__ void pair_chunk_x2(const float4 *__restrict__ rec, uint32_t a0,
                                           uint32_t ac, uint32_t aend, uint32_t b0, uint32_t nb,
                                           int ox, int oy, const float (&a)[DEG + 1], float cn,
                                           float2 *fwd, float2 *bwd, bool bwd_add, bool fwd_add,
                                           int lane) {
    float2 tx[H], ty[H], tg[H], U[H], v[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const uint32_t i0 = ac + lane + 64 * h, i1 = i0 + 32;
        const float4 r0 = i0 < aend ? rec[a0 + i0] : make_float4(kPairFar, kPairFar, 0.f, 0.f);
        const float4 r1 = i1 < aend ? rec[a0 + i1] : make_float4(kPairFar, kPairFar, 0.f, 0.f);
        tx[h] = make_float2(r0.x, r1.x);
        ty[h] = make_float2(r0.y, r1.y);
        tg[h] = make_float2(r0.z, r1.z);
        U[h] = v[h] = make_float2(0.f, 0.f);
    }
    float2 a2[DEG + 1];
#pragma unroll
    for (int k = 0; k <= DEG; ++k) a2[k] = make_float2(a[k], a[k]);
    for (uint32_t bc = 0; bc < nb; bc += 32) {
        const SourceSlot ss = source_slot(rec, b0, bc, nb, ox, oy, lane);
        float bu, BV;
        if (ss.half)
            source_pass_x2<DEG, H, 16>(tx, ty, tg, U, v, a2, -ss.xs, -ss.ys, ss.gs, bu, BV, lane);
        else
            source_pass_x2<DEG, H, 32>(tx, ty, tg, U, v, a2, -ss.xs, -ss.ys, ss.gs, bu, BV, lane);
        if (ss.hs && (!ss.half || lane < 16))
            put2(bwd + ss.sb, make_float2(cn * bu, -(cn * BV)), bwd_add);
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const uint32_t i0 = ac + lane + 64 * h, i1 = i0 + 32;
        if (i0 < aend) put2(fwd + i0, make_float2(-(cn * U[h].x), cn * v[h].x), fwd_add);
        if (i1 < aend) put2(fwd + i1, make_float2(-(cn * U[h].y), cn * v[h].y), fwd_add);
    }
}

// The pairs of blobs abeg .. aend - 1 of leaf A (from a0) with the nb blobs
// of leaf B (from b0): A in chunks of 320, 256, 128, 64 or 32 targets.  Leaf
// pairs take the largest chunk that the remaining targets fill to at least
// three quarters (for 320: more than 256, where one 320-chunk is faster
// than 256 + a tail chunk); more targets per lane amortise the shuffles of
// a step over more pairs (measured in isolation on GB300: 10 targets per
// lane 0.776 of the FP32 peak, 8 per lane 0.727).  A range of whole 32-blob
// chunks (exact) is cut without padding.  The first chunk writes bwd (unless bwd_add), later ones
// add to it; fwd_add: the chunks add to fwd.
template <int DEG, bool GENERAL>
__device__ __forceinline__ void pair_leaves(const float4 *__restrict__ rec, uint32_t a0,
                                            uint32_t abeg, uint32_t aend, uint32_t b0, uint32_t nb,
                                            int ox, int oy, const float (&a)[DEG + 1],
                                            float kappa, float split, float cn, float2 *fwd,
                                            float2 *bwd, bool bwd_add, bool fwd_add, bool exact,
                                            int lane) {
    const uint32_t t10 = exact ? 320 : 257, t8 = exact ? 256 : 192, t4 = exact ? 128 : 96,
                   t2 = exact ? 64 : 33;
    for (uint32_t ac = abeg; ac < aend; bwd_add = true) {
        const uint32_t rem = aend - ac;
        if (!GENERAL && rem >= t10) {
            pair_chunk_x2<DEG, 5>(rec, a0, ac, aend, b0, nb, ox, oy, a, cn, fwd, bwd, bwd_add,
                                  fwd_add, lane);
            ac += 320;
        } else if (!GENERAL && rem >= t8) {
            pair_chunk_x2<DEG, 4>(rec, a0, ac, aend, b0, nb, ox, oy, a, cn, fwd, bwd, bwd_add,
                                  fwd_add, lane);
            ac += 256;
        } else if (rem >= t4) {
            if (GENERAL)
                pair_chunk<DEG, GENERAL, 4>(rec, a0, ac, aend, b0, nb, ox, oy, a, kappa, split, cn,
                                            fwd, bwd, bwd_add, fwd_add, lane);
            else
                pair_chunk_x2<DEG, 2>(rec, a0, ac, aend, b0, nb, ox, oy, a, cn, fwd, bwd, bwd_add,
                                      fwd_add, lane);
            ac += 128;
        } else if (rem >= t2) {
            pair_chunk<DEG, GENERAL, 2>(rec, a0, ac, aend, b0, nb, ox, oy, a, kappa, split, cn,
                                        fwd, bwd, bwd_add, fwd_add, lane);
            ac += 64;
        } else {
            pair_chunk<DEG, GENERAL, 1>(rec, a0, ac, aend, b0, nb, ox, oy, a, kappa, split, cn,
                                        fwd, bwd, bwd_add, fwd_add, lane);
            ac += 32;
        }
    }
}

// The pairs within one leaf (n >= 32 blobs from a0), each once, summed into
// slf[0 .. n) by one warp in a fixed order.  For each 32-blob sub-chunk j:
// the pairs inside it -- the blobs rotate around the warp for 16 steps, so
// that every lane meets every other lane's blob once (at step 16 the two
// halves of the warp meet each other, so only lanes 0..15 count it), and a
// final shuffle brings each travelling reaction back to its blob -- then its
// pairs with all blobs before it, as a pair range (targets 0 .. 32 j,
// sources the sub-chunk).
template <int DEG, bool GENERAL>
__device__ __forceinline__ void self_leaf(const float4 *__restrict__ rec, uint32_t a0,
                                          uint32_t n, const float (&a)[DEG + 1], float kappa,
                                          float split, float cn, float2 *slf, int lane) {
    const int next = (lane + 1) & 31;
    for (uint32_t s0 = 0; s0 < n; s0 += 32) {
        const uint32_t ns = min(32u, n - s0);
        const bool h = uint32_t(lane) < ns;
        const float4 r = h ? rec[a0 + s0 + lane] : make_float4(kPairFar, kPairFar, 0.f, 0.f);
        float xs = r.x, ys = r.y, gs = r.z, bu = 0.f, bv = 0.f, u = 0.f, v = 0.f;
        for (int k = 1; k <= 16; ++k) {
            xs = __shfl_sync(0xffffffffu, xs, next);
            ys = __shfl_sync(0xffffffffu, ys, next);
            gs = __shfl_sync(0xffffffffu, gs, next);
            bu = __shfl_sync(0xffffffffu, bu, next);
            bv = __shfl_sync(0xffffffffu, bv, next);
            const bool on = k < 16 || lane < 16;
            pair_sym<DEG, GENERAL>(r.x, r.y, on ? r.z : 0.f, xs, ys, on ? gs : 0.f, a, kappa,
                                   split, u, v, bu, bv);
        }
        // lane l holds the reaction of the blob of lane l + 16
        bu = __shfl_sync(0xffffffffu, bu, (lane + 16) & 31);
        bv = __shfl_sync(0xffffffffu, bv, (lane + 16) & 31);
        if (h) slf[s0 + lane] = make_float2(cn * (u + bu), cn * (v + bv));
        __syncwarp();
        if (s0)
            pair_leaves<DEG, GENERAL>(rec, a0, 0, s0, a0 + s0, ns, 0, 0, a, kappa, split, cn, slf,
                                      slf + s0, true, true, true, lane);
        __syncwarp();
    }
}

// One item of the pairwise near field: piece item.z >> 4 of leaf A (item.y)
// with its forward neighbour B, direction item.z & 7 (4: the leaf's own
// pairs, to slot 8); bit 3: B's blobs are the targets (a pair in one piece);
// item.w = the pair's scratch base (all ones: the pair is not split, piece 0
// takes all of it).
template <int DEG, bool GENERAL>
__device__ __forceinline__ void pair_item(const uint4 item, const InstDesc *__restrict__ insts,
                                          const uint32_t *__restrict__ start,
                                          const float4 *__restrict__ rec,
                                          float2 *__restrict__ part, int64_t nslot,
                                          float2 *__restrict__ xs, int64_t xcap, int lane) {
    const InstDesc &d = insts[item.x];
    float a[DEG + 1];
#pragma unroll
    for (int k = 0; k <= DEG; ++k) a[k] = d.poly[k];
    const float kappa = d.kappa, split = d.qsplit_rho2, cn = d.cnear;
    const uint32_t m = item.y;
    const int dir = int(item.z & 7u);
    const bool swap = (item.z >> 3) & 1u;
    const uint32_t piece = item.z >> 4;
    const uint32_t *st = start + d.soff;
    const uint32_t a0 = st[m], na = st[m + 1] - a0;
    // checked build: the leaf and its range lie inside the instance
    if (!(PF_IN(m, int64_t(1) << (2 * d.L)) && PF_IN(int64_t(a0) - d.poff, d.n + 1) &&
          PF_IN(int64_t(a0) + na - d.poff, d.n + 1) && PF_IN(int64_t(a0) + na, nslot + 1)))
        return;
    if (dir == 4) {
        self_leaf<DEG, GENERAL>(rec, a0, na, a, kappa, split, cn, part + 8 * nslot + a0, lane);
        return;
    }
    const int ix = int(compact_bits(m)), iy = int(compact_bits(m >> 1));
    const int ox = c_fwd[dir][0], oy = c_fwd[dir][1];
    const uint32_t mb = morton_key(uint32_t(ix + ox), uint32_t(iy + oy));
    const uint32_t b0 = st[mb], nb = st[mb + 1] - b0;
    if (!(PF_IN(mb, int64_t(1) << (2 * d.L)) && PF_IN(int64_t(b0) - d.poff, d.n + 1) &&
          PF_IN(int64_t(b0) + nb - d.poff, d.n + 1)))
        return;
    float2 *fwd = part + int64_t(dir) * nslot + a0;      // A's particles, from B
    float2 *bwd = part + int64_t(4 + dir) * nslot + b0;  // B's particles, from A
    if (swap) {
        pair_leaves<DEG, GENERAL>(rec, b0, 0, nb, a0, na, -ox, -oy, a, kappa, split, cn, bwd, fwd,
                                  false, false, false, lane);
        return;
    }
    uint32_t abeg = 0, aend = na;
    if (item.w != 0xffffffffu) {
        uint32_t pc;
        pair_pieces(na, nb, &pc);
        abeg = piece * pc;
        aend = min(na, abeg + pc);
        if (piece) {
            if (!PF_IN(int64_t(item.w) + int64_t(piece) * nb - 1, xcap)) return;
            bwd = xs + item.w + int64_t(piece - 1) * nb;
        }
    } else if (piece) {
        return;
    }
    pair_leaves<DEG, GENERAL>(rec, a0, abeg, aend, b0, nb, ox, oy, a, kappa, split, cn, fwd, bwd,
                              false, false, false, lane);
}

// The pair items of the pairwise mode, heaviest first, in one persistent
// launch (64 registers for the four targets per lane: 4 CTAs per SM); the
// directed items of the leaves' own and not-pairwise neighbours follow in
// k_p2p_mixed<.., PAIRS = true> at its higher occupancy.  Measured on GB300,
// one queue over both kinds of item (the directed ones filling the pairs'
// tail) was slower: the directed items ran at this kernel's occupancy.
template <int DEG, bool GENERAL>
__global__ void __launch_bounds__(P2P_THREADS, 3) k_p2p_pairs(
    const uint4 *__restrict__ pitems, uint32_t *ctrl, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float4 *__restrict__ rec, const PairBufs pb,
    unsigned long long *busy) {
    const int lane = threadIdx.x & 31;
    const uint32_t npairs = *reinterpret_cast<volatile uint32_t *>(ctrl + CTRL_NPAIRS);
    const uint64_t t_begin = busy ? global_ns() : 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctrl + CTRL_QUEUE2, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= npairs) break;
        pair_item<DEG, GENERAL>(pitems[it], insts, start, rec, pb.part, pb.nslot, pb.xs, pb.xcap,
                                lane);
    }
    if (busy && lane == 0) {
        const size_t gw = size_t(blockIdx.x) * (P2P_THREADS / 32) + (threadIdx.x >> 5);
        busy[2 * gw] = t_begin;
        busy[2 * gw + 1] = global_ns();
    }
}

// The final pass of the mixed near field, one thread per blob: u, v = its
// leaf's far field (L2P of the local expansion, Sec. 2.2), plus its directly
// summed near part, plus (pairwise mode, pb.part != nullptr) the slots of its
// pairwise neighbours, a split pair's scratch runs after its slot in piece
// order; a fixed order throughout, written at the caller's index.
// blobs per occupied leaf from which the final pass requests every pair
// slot of a blob up front (see k_p2p_final)
constexpr int64_t kEagerBlobsPerLeaf = 48;

__global__ void __launch_bounds__(256, 4) k_p2p_final(
    const Task *__restrict__ tasks, int ntasks, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const uint32_t *__restrict__ skeys,
    const float4 *__restrict__ rec, const float2 *__restrict__ le, const PairBufs pb,
    int dtype_f32, float *__restrict__ stage, int64_t nstage, const uint32_t *__restrict__ ctrl,
    int64_t ntotal) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t j = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (j >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int64_t r = d.poff + j;
    const uint32_t *st = start + d.soff;
    const int nside = 1 << d.L;
    // Where the occupied leaves hold many blobs on average (pair slots
    // nearly everywhere), this blob's near-field parts are requested at once,
    // with its key and record, instead of after its leaf's flags: one latency
    // instead of three on the way to the sum.  The flags still decide which
    // of them are added, in the same order.
    const bool eager = pb.part && int64_t(ntotal) >= kEagerBlobsPerLeaf * int64_t(ctrl[CTRL_NOCC]);
    float2 e_own = make_float2(0.f, 0.f), e_self = e_own, e_fwd[4], e_bwd[4];
    if (eager) {
        e_own = pb.own[r];
        e_self = pb.part[8 * pb.nslot + r];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e_fwd[k] = pb.part[int64_t(k) * pb.nslot + r];
            e_bwd[k] = pb.part[int64_t(4 + k) * pb.nslot + r];
        }
    }
    const uint32_t m = skeys[r] & ((d.L >= 16) ? 0xffffffffu : ((1u << (2 * d.L)) - 1u));
    const int ix = int(compact_bits(m)), iy = int(compact_bits(m >> 1));
    const float4 rr = rec[r];
    float2 w = make_float2(0.f, 0.f);
    if (d.L >= 2) {
        // w = (1/r) sum c_m zeta^m, zeta the offset from the leaf centre
        const int p = d.p;
        const float2 *c =
            le + d.eoff + (lvl_off(d.L) + box_index(d.L, uint32_t(ix), uint32_t(iy))) * p;
        float2 z = __ldg(c + p - 1);
        for (int k = p - 2; k >= 0; --k) {
            const float2 ck = __ldg(c + k);
            z = make_float2(fmaf(z.x, rr.x, fmaf(-z.y, rr.y, ck.x)),
                            fmaf(z.x, rr.y, fmaf(z.y, rr.x, ck.y)));
        }
        // vortex: u - i v = cfar w; Laplace: the potential is Re of the LE
        w = d.kernel == KERNEL_LAPLACE ? make_float2(z.x, 0.f)
                                       : make_float2(d.cfar * z.y, d.cfar * z.x);
    }
    // then the near-field parts this leaf has, in a fixed order
    const uint32_t fl = pb.part ? pb.lflags[d.loff + m] : LF_DIRECTED;
    if (fl & LF_DIRECTED) {
        const float2 o = eager ? e_own : pb.own[r];
        w.x += o.x;
        w.y += o.y;
    }
    if (fl & LF_SELF) {
        const float2 sp = eager ? e_self : pb.part[8 * pb.nslot + r];
        w.x += sp.x;
        w.y += sp.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (fl & (LF_FWD << k)) {
            const float2 p = eager ? e_fwd[k] : pb.part[int64_t(k) * pb.nslot + r];
            w.x += p.x;
            w.y += p.y;
        }
        if (!(fl & (LF_BWD << k))) continue;
        const float2 p = eager ? e_bwd[k] : pb.part[int64_t(4 + k) * pb.nslot + r];
        w.x += p.x;
        w.y += p.y;
        if (fl & (LF_SPLIT << k)) {
            // pieces 1 .. of the pair (A = the backward neighbour, B = this leaf)
            const int ax = ix - c_fwd[k][0], ay = iy - c_fwd[k][1];
            const uint32_t na = leaf_count(st, nside, ax, ay), nme = st[m + 1] - st[m];
            const uint32_t jme = uint32_t(r) - st[m];
            uint32_t pc;
            const uint32_t np = pair_pieces(na, nme, &pc);
            const uint32_t ma = morton_key(uint32_t(ax), uint32_t(ay));
            const uint32_t base = pb.xtab[(d.loff + int64_t(ma)) * 4 + k];
            for (uint32_t i = 1; i < np; ++i) {
                const float2 x = pb.xs[base + int64_t(i - 1) * nme + jme];
                w.x += x.x;
                w.y += x.y;
            }
        }
    }
    if (stage) {
        // sorted order; k_unsort writes the caller's arrays
        stage[r] = w.x;
        stage[nstage + r] = w.y;
        return;
    }
    const int64_t q = int64_t(__float_as_uint(rr.w)) - d.poff;
    if (!PF_IN(q, d.n)) return;  // checked build: the caller's index of the blob
    if (dtype_f32) {
        static_cast<float *>(d.u)[q] = w.x;
        static_cast<float *>(d.v)[q] = w.y;
    } else {
        static_cast<double *>(d.u)[q] = double(w.x);
        static_cast<double *>(d.v)[q] = double(w.y);
    }
}

cudaError_t launch_pair_worklist(const Task *tasks, int ntasks, int64_t nblocks,
                                 const InstDesc *insts, const uint32_t *start, int64_t nleaves,
                                 uint32_t *cnt, uint32_t *off, uint32_t *scan_scratch,
                                 uint4 *items, uint32_t *ctrl, const P2POrder *order,
                                 const PairBufs &pb, cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_pair_count<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, cnt, pb.xcnt,
                                                    ctrl);
    PF_LAUNCHED(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(cnt, off, nleaves, scan_scratch, ctrl + CTRL_NPAIRS, st, launches);
    if (e != cudaSuccess) return e;
    e = exclusive_scan(pb.xcnt, pb.xoff, nleaves, scan_scratch, ctrl + CTRL_NXTRA, st, launches);
    if (e != cudaSuccess) return e;
    uint4 *emit_to = order ? order->items_unsorted : items;
    k_pair_emit<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, off, pb.xoff, ctrl,
                                                   pb.xcap, pb.xtab, pb.lflags, emit_to,
                                                   order ? order->kA : nullptr);
    PF_LAUNCHED(1);
    if ((e = cudaGetLastError()) != cudaSuccess || !order) return e;
    return order_items(order, items, ctrl + CTRL_NPAIRS, scan_scratch, st, launches);
}

// ----------------------------------------------------------------------------
// Launch helpers
// ----------------------------------------------------------------------------
typedef void (*MixedKernel)(const uint4 *, uint32_t *, const InstDesc *, const uint32_t *,
                            const float4 *, float2 *, unsigned long long *);
template <int D>
static MixedKernel pick2(int general, bool pairs) {
    if (pairs)
        return general ? k_p2p_mixed<D, true, true, false> : k_p2p_mixed<D, false, true, false>;
    return general ? k_p2p_mixed<D, true, false, false> : k_p2p_mixed<D, false, false, false>;
}

static MixedKernel pick_mixed(int deg, int general, bool pairs = false, bool lap = false) {
    if (lap) return k_p2p_mixed<4, false, false, true>;  // no polynomial, no pairs
    switch (deg) {
        case 4: return pick2<4>(general, pairs);
        case 5: return pick2<5>(general, pairs);
        case 6: return pick2<6>(general, pairs);
        case 7: return pick2<7>(general, pairs);
        case 8: return pick2<8>(general, pairs);
        case 9: return pick2<9>(general, pairs);
        case 10: return pick2<10>(general, pairs);
        case 11: return pick2<11>(general, pairs);
        case 12: return pick2<12>(general, pairs);
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

int p2p_grid(int precision_mixed, int deg, int general, int laplace) {
    int per_sm = 1;
    if (precision_mixed) {
        MixedKernel k = pick_mixed(deg, general, false, laplace != 0);
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
                             float2 *own, int pairs, int laplace, unsigned long long *busy,
                             cudaStream_t st, uint64_t *launches) {
    MixedKernel k = pick_mixed(deg, general, pairs != 0, laplace != 0);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, P2P_THREADS, 0, st>>>(items, ctrl, insts, start, rec, own, busy);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

typedef void (*PairsKernel)(const uint4 *, uint32_t *, const InstDesc *, const uint32_t *,
                            const float4 *, const PairBufs, unsigned long long *);

template <int D>
static PairsKernel pick_pairs2(int general) {
    return general ? k_p2p_pairs<D, true> : k_p2p_pairs<D, false>;
}

static PairsKernel pick_pairs(int deg, int general) {
    switch (deg) {
        case 4: return pick_pairs2<4>(general);
        case 5: return pick_pairs2<5>(general);
        case 6: return pick_pairs2<6>(general);
        case 7: return pick_pairs2<7>(general);
        case 8: return pick_pairs2<8>(general);
        case 9: return pick_pairs2<9>(general);
        case 10: return pick_pairs2<10>(general);
        case 11: return pick_pairs2<11>(general);
        case 12: return pick_pairs2<12>(general);
        default: return nullptr;
    }
}

int p2p_pairs_grid(int deg, int general) {
    PairsKernel k = pick_pairs(deg, general);
    if (!k) return 0;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, P2P_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sm_count();
}

cudaError_t launch_p2p_pairs(int grid, int deg, int general, const uint4 *pitems, uint32_t *ctrl,
                             const InstDesc *insts, const uint32_t *start, const float4 *rec,
                             const PairBufs &pb, unsigned long long *busy, cudaStream_t st,
                             uint64_t *launches) {
    PairsKernel k = pick_pairs(deg, general);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, P2P_THREADS, 0, st>>>(pitems, ctrl, insts, start, rec, pb, busy);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// The caller's u (comp 0) or v (comp 1) from the sorted-order stage, FP32
// outputs.  One component per launch: its scattered 4-byte writes then fit in
// L2 and leave it as whole sectors, where writing u and v together from the
// final pass evicts partly written sectors (each one read back and written
// again).
__global__ void __launch_bounds__(256) k_unsort_f32(const Task *__restrict__ tasks, int ntasks,
                                                    const InstDesc *__restrict__ insts,
                                                    const uint32_t *__restrict__ perm,
                                                    const float *__restrict__ stage, int comp) {
    // four consecutive sorted ranks per thread (tasks of 1024 per block):
    // four independent scattered stores after two 16-byte loads
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t j0 = ((int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x) * 4;
    if (j0 >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int64_t r0 = d.poff + j0;
    float *out = static_cast<float *>(comp ? d.v : d.u);
    if (j0 + 4 <= t.count && (r0 & 3) == 0) {
        const uint4 q = *reinterpret_cast<const uint4 *>(perm + r0);
        const float4 w = *reinterpret_cast<const float4 *>(stage + r0);
        if (PF_IN(int64_t(q.x) - d.poff, d.n)) out[int64_t(q.x) - d.poff] = w.x;
        if (PF_IN(int64_t(q.y) - d.poff, d.n)) out[int64_t(q.y) - d.poff] = w.y;
        if (PF_IN(int64_t(q.z) - d.poff, d.n)) out[int64_t(q.z) - d.poff] = w.z;
        if (PF_IN(int64_t(q.w) - d.poff, d.n)) out[int64_t(q.w) - d.poff] = w.w;
    } else {
        for (int e = 0; e < 4; ++e)
            if (j0 + e < t.count && PF_IN(int64_t(perm[r0 + e]) - d.poff, d.n))
                out[int64_t(perm[r0 + e]) - d.poff] = stage[r0 + e];
    }
}

cudaError_t launch_p2p_final(const Task *tasks, int ntasks, int64_t nblocks,
                             const InstDesc *insts, const uint32_t *start, const uint32_t *skeys,
                             const float4 *rec, const float2 *le, const PairBufs &pb,
                             int dtype_f32, const uint32_t *perm, float *stage, int64_t nstage,
                             const Task *utasks, int nutasks, int64_t unblocks,
                             const uint32_t *ctrl, int64_t ntotal, cudaStream_t st,
                             uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_p2p_final<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, start, skeys, rec, le, pb,
                                                   dtype_f32, stage, nstage, ctrl, ntotal);
    PF_LAUNCHED(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !stage || unblocks <= 0) return e;
    for (int comp = 0; comp < 2; ++comp) {
        k_unsort_f32<<<unsigned(unblocks), 256, 0, st>>>(utasks, nutasks, insts, perm,
                                                         stage + comp * nstage, comp);
        PF_LAUNCHED(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
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

PF_DEFINE_CHECK_READER(p2p)

}  // namespace petfmm
