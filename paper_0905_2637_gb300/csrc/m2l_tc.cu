// m2l_tc.cu -- M2L (Sec. 2.2, downward sweep) as a dense GEMM on the 5th-
// generation tensor cores (tcgen05, TF32 inputs, FP32 accumulation in TMEM),
// mixed-precision path.
//
// With expansions stored by child class (common.cuh), the interaction list of
// a target of class c at parent cell P is the set of 27 (source class c',
// parent offset (dx, dy)) pairs whose child offset
//     delta = (2 dx + c'x - cx, 2 dy + c'y - cy)
// is not within one box.  Each such pair is one fixed operator T_delta, and
// the translation of all targets of one parent row is
//     LE_c[P] += ME_c'[P + (dx, dy)] T_delta^T
// i.e. a real GEMM with M = targets (128 per MMA), K = 2p source coefficients
// (real parts then imaginary parts) and N = 2p output coefficients, with
// B_delta = [[Tr^T, Ti^T], [-Ti^T, Tr^T]].
//
// Two unit shapes.  Blocks (k_m2l_tcb, the default; below): 8 x 16 parent
// cells with the four target classes side by side in N.  Row units
// (k_m2l_tc, PETFMM_OPT_TC_BLOCKS = 2), described here: a segment of up to
// 512 parent cells of one parent row, for one target class.  For each of the
// 12 (c', dy) source strips the
// CTA stages the strip's source expansions once in shared memory, K-major
// without swizzle (core matrices of 8 rows x 16 bytes; rows 16 B apart inside
// a k-group, so a row offset is a 16-byte shift of the descriptor start), and
// the three dx shifts of the strip are the same staged data read one row
// earlier or later.  Operands are split for 3xTF32: a = a_hi + a_lo with
// a_hi = a with its low 13 mantissa bits cleared; the GEMM accumulates
// a_hi b_hi + a_hi b_lo + a_lo b_hi (relative error about 2^-20).  Units whose
// targets are all empty are skipped, and so are strips whose sources are all
// empty (their expansions would be zero).
//
// One thread issues the MMAs; their completion is tracked with an mbarrier
// (tcgen05.commit); every wait is bounded and reports PETFMM_ETIMEOUT.
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace petfmm {

#define PF_LAUNCHED(n) do { if (launches) *launches += (n); } while (0)

// 256 threads: the first 128 own the TMEM lanes (targets) in the epilogue,
// all of them stage operands (twice the loads in flight of 128 threads)
constexpr int TC_THREADS = 256;
constexpr int TC_MAX_NPAD = 48;

// Operators of the strip (source class cs, parent row offset dyp) for a
// target of class c: bit s of the result is set if the dx shift dxp = s - 1
// is in the interaction list (child offset not within one box), ops[s] its
// operator index.
__device__ __forceinline__ uint32_t tc_strip_ops(int c, int cs, int dyp, int *ops) {
    const int cx = c & 1, cy = c >> 1, csx = cs & 1, csy = cs >> 1;
    uint32_t mask3 = 0;
    for (int dxp = -1; dxp <= 1; ++dxp) {
        const int ddx = 2 * dxp + csx - cx, ddy = 2 * dyp + csy - cy;
        const int ax = ddx < 0 ? -ddx : ddx, ay = ddy < 0 ? -ddy : ddy;
        ops[dxp + 1] = 0;
        if ((ax > ay ? ax : ay) >= 2) {
            mask3 |= 1u << (dxp + 1);
            ops[dxp + 1] = m2l_op_index(ddx, ddy);
        }
    }
    return mask3;
}

// Counts, for every unit of the tensor-core launch (index = the launch's block
// index), how many of its targets hold particles; one warp per unit.  The
// tensor cores take the dense units, the SIMT kernel the boxes of the others.
__global__ void __launch_bounds__(256) k_tc_unit_count(const Task *__restrict__ tasks, int ntasks,
                                                       const InstDesc *__restrict__ insts,
                                                       const uint32_t *__restrict__ start,
                                                       uint32_t *__restrict__ ucount,
                                                       int64_t nunits) {
    const int64_t u = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= nunits) return;
    const Task t = tasks[find_task(tasks, ntasks, u)];
    const InstDesc &d = insts[t.inst];
    const int l = t.level;
    int c, Py0, R = 1, Px0, SEG;
    if ((d.tc_levels >> l) & 1u) {
        tc_unit_decode(l, d.tc_segmax, u - t.block0, &c, &Py0, &Px0, &SEG);
    } else if ((d.tcb_levels >> l) & 1u) {
        // a block: 8 x 16 parent cells, all four classes (i = c 128 + cell)
        tcb_unit_decode(l, u - t.block0, &Py0, &Px0);
        const uint32_t *st = start + d.soff;
        uint32_t cnt = 0;
        for (int i = lane; i < 4 * TCB_BX * TCB_BY; i += 32) {
            const int cc = i >> 7, q = i & 127;
            const uint32_t ix = uint32_t(2 * (Px0 + (q & 7)) + (cc & 1));
            const uint32_t iy = uint32_t(2 * (Py0 + (q >> 3)) + (cc >> 1));
            cnt += box_count(st, d.L, l, morton_key(ix, iy)) != 0;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if (lane == 0) ucount[u] = cnt;
        return;
    } else {
        tile_unit_decode(l, u - t.block0, &c, &Py0, &R, &Px0, &SEG);
    }
    const uint32_t *st = start + d.soff;
    uint32_t cnt = 0;
    for (int i = lane; i < R * SEG; i += 32) {
        const int r = i / SEG, x = i - r * SEG;
        const uint32_t ix = uint32_t(2 * (Px0 + x) + (c & 1)), iy = uint32_t(2 * (Py0 + r) + (c >> 1));
        cnt += box_count(st, d.L, l, morton_key(ix, iy)) != 0;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) ucount[u] = cnt;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(
    const Task *__restrict__ tasks, int ntasks, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float2 *__restrict__ me, float2 *__restrict__ le,
    const uint32_t *__restrict__ ucount, int dense_pct, long long spin_limit, int *status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ uint32_t used_mask;
    // source-box occupancy of every strip of the unit: [strip][row]
    __shared__ uint8_t socc[12][TC_MAX_SEG + 2];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const InstDesc &d = insts[t.inst];
    const int l = t.level, L = d.L, p = d.p;
    const int W = 1 << (l - 1);
    int c, Py, Px0, SEG;
    tc_unit_decode(l, d.tc_segmax, int64_t(blockIdx.x) - t.block0, &c, &Py, &Px0, &SEG);
    const int S = SEG / 128;
    const int cx = c & 1, cy = c >> 1;
    const uint32_t *st = start + d.soff;

    // 1. sparse units are left to the SIMT kernel (same test there)
    if (!tc_unit_dense(ucount[blockIdx.x], SEG, dense_pct)) return;
    // which 128-target sub-tiles hold particles (empty ones issue no MMA)
    uint32_t sub_mask = 0;
    for (int s = 0; s < S; ++s) {
        bool o = false;
        if (tid < 128) {
            const int i = s * 128 + tid;
            const uint32_t ix = uint32_t(2 * (Px0 + i) + cx), iy = uint32_t(2 * Py + cy);
            o = box_count(st, L, l, morton_key(ix, iy)) != 0;
        }
        if (__syncthreads_or(o)) sub_mask |= 1u << s;
    }

    const int K2 = 2 * p;
    const int Kpad = (K2 + 7) & ~7, Npad = (K2 + 15) & ~15;
    const int KG = Kpad / 4, Rs = SEG + 2;
    float *A_hi = reinterpret_cast<float *>(smem);
    float *A_lo = A_hi + size_t(KG) * Rs * 4;
    float *Bsm = A_lo + size_t(KG) * Rs * 4;  // 6 slots of Kpad x Npad floats
    const int bslot = Kpad * Npad;
    // zero the K padding of every staged row once (never overwritten)
    for (int i = tid; i < Rs * (Kpad - K2); i += TC_THREADS) {
        const int r = i / (Kpad - K2), k = K2 + i % (Kpad - K2);
        const size_t o = (size_t(k >> 2) * Rs + r) * 4 + (k & 3);
        A_hi[o] = 0.f;
        A_lo[o] = 0.f;
    }
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;");
        used_mask = 0;
    }
    int ncols = 32;
    while (ncols < S * Npad) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(Npad >> 3) << 17) |
                           (uint32_t(128 >> 4) << 24);
    const uint32_t LBO_A = uint32_t(Rs) * 16, LBO_B = uint32_t(Npad) * 16, SBO = 128;
    const int64_t quarter = int64_t(1) << (2 * (l - 1));
    const float2 *lev = me + d.eoff + lvl_off(l) * p;
    const float *bimg = static_cast<const float *>(d.t_m2l_tc);
    uint32_t phase = 0;
    bool ok = true;
    uint32_t used = 0;  // thread 0's record of initialised accumulators

    // The strips: (source class cs, parent row offset dyp) pairs with at
    // least one interaction-list operator, in a fixed order.  Strip j + 1's
    // source expansions are copied asynchronously (cp.async, empty boxes
    // zero-filled) into a raw buffer while strip j is split into the TF32
    // operand layout and multiplied; its operator images follow as soon as
    // strip j's MMAs have released the B buffer.
    int ncand = 0;
    uint8_t cand[12];
    for (int cs = 0; cs < 4; ++cs)
        for (int dyp = -1; dyp <= 1; ++dyp) {
            const int Pys = Py + dyp;
            if (Pys < 0 || Pys >= W) continue;
            int ops[3];
            if (tc_strip_ops(c, cs, dyp, ops)) cand[ncand++] = uint8_t(cs * 3 + dyp + 1);
        }
    const int total = Rs * p;
    const uint32_t inv_p = ((1u << 20) + uint32_t(p) - 1) / uint32_t(p);
    float2 *raw = reinterpret_cast<float2 *>(Bsm + size_t(6) * bslot);
    // occupancy of all strips' source boxes at once (one round of lookups)
    __shared__ uint32_t sany;
    if (tid == 0) sany = 0;
    __syncthreads();
    for (int i = tid; i < ncand * Rs; i += TC_THREADS) {
        const int jj = i / Rs, r = i - jj * Rs;
        const int cs = cand[jj] / 3, dyp = cand[jj] % 3 - 1;
        const int Px = Px0 - 1 + r, Pys = Py + dyp;
        bool o = false;
        if (Px >= 0 && Px < W)
            o = box_count(st, L, l, morton_key(uint32_t(2 * Px + (cs & 1)),
                                               uint32_t(2 * Pys + (cs >> 1)))) != 0;
        socc[jj][r] = o;
        if (o) atomicOr(&sany, 1u << jj);
    }
    __syncthreads();
    const uint32_t strip_any = sany;
    // first candidate >= j0 with an occupied source box: its raw copy is
    // requested (one commit group); returns ncand if there is none
    auto prepare = [&](int j0) -> int {
        for (int jj = j0; jj < ncand; ++jj) {
            if (!((strip_any >> jj) & 1u)) continue;
            const int cs = cand[jj] / 3, dyp = cand[jj] % 3 - 1, Pys = Py + dyp;
            const float2 *src = lev + (int64_t(cs) * quarter + int64_t(Pys) * W + Px0 - 1) * p;
            for (int e = tid; e < total; e += TC_THREADS) {
                const int r = int((uint32_t(e) * inv_p) >> 20);
                cp_async8(smem_addr(raw + e), src + e, socc[jj][r] ? 8u : 0u);
            }
            cp_async_commit();
            return jj;
        }
        return ncand;
    };
    // the B operators of strip jj's (up to three) dx shifts, hi and lo images
    auto request_b = [&](int jj) {
        int ops[3];
        const uint32_t mask3 = tc_strip_ops(c, cand[jj] / 3, cand[jj] % 3 - 1, ops);
        const int n4 = (2 * bslot) / 4;
        for (int s3 = 0; s3 < 3; ++s3) {
            if (!(mask3 & (1u << s3))) continue;
            const float4 *src = reinterpret_cast<const float4 *>(bimg + size_t(ops[s3]) * 2 * bslot);
            const uint32_t dst = smem_addr(Bsm + size_t(2 * s3) * bslot);
            for (int i = tid; i < n4; i += TC_THREADS) cp_async16(dst + uint32_t(i) * 16, src + i);
        }
        cp_async_commit();
    };

    int j = prepare(0);
    if (j < ncand) request_b(j);
    while (j < ncand && ok) {
        cp_async_wait_all();
        __syncthreads();
        // split the strip: real parts at k < p, imaginary parts at p <= k < 2p;
        // element e of the raw strip is coefficient k of row r, e = r p + k,
        // with r = e * inv_p >> 20 (exact for e < 2^14, p <= 24)
        for (int e = tid; e < total; e += TC_THREADS) {
            const int r = int((uint32_t(e) * inv_p) >> 20), k = e - r * p;
            const float2 v = raw[e];
            const float hr = tf32_hi(v.x), hi_ = tf32_hi(v.y);
            const size_t o_re = (size_t(k >> 2) * Rs + r) * 4 + (k & 3);
            const size_t o_im = (size_t((k + p) >> 2) * Rs + r) * 4 + ((k + p) & 3);
            A_hi[o_re] = hr;
            A_lo[o_re] = v.x - hr;
            A_hi[o_im] = hi_;
            A_lo[o_im] = v.y - hi_;
        }
        __syncthreads();
        int ops[3];
        const uint32_t mask3 = tc_strip_ops(c, cand[j] / 3, cand[j] % 3 - 1, ops);
        const int jn = prepare(j + 1);  // its copy overlaps this strip's MMAs
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ahi = smem_addr(A_hi), alo = smem_addr(A_lo);
            for (int s3 = 0; s3 < 3; ++s3) {
                if (!(mask3 & (1u << s3))) continue;
                const uint32_t bhi = smem_addr(Bsm + size_t(2 * s3) * bslot);
                const uint32_t blo = smem_addr(Bsm + size_t(2 * s3 + 1) * bslot);
                // descriptors step by adding to their start-address field
                // (address / 16 in the low bits; shared addresses stay below
                // 256 KB, so the sum never carries out of the field)
                const uint64_t sa = (2 * LBO_A) >> 4, sb = (2 * LBO_B) >> 4;
                const uint64_t dbh = mma_desc(bhi, LBO_B, SBO), dbl = mma_desc(blo, LBO_B, SBO);
                for (int s = 0; s < S; ++s) {
                    if (!(sub_mask & (1u << s))) continue;  // no target there
                    const uint32_t row0 = uint32_t(s * 128 + 1 + (s3 - 1)) * 16;
                    const uint32_t dt = tbase + uint32_t(s * Npad);
                    const uint64_t dah = mma_desc(ahi + row0, LBO_A, SBO);
                    const uint64_t dal = mma_desc(alo + row0, LBO_A, SBO);
                    for (int ks = 0; ks < Kpad / 8; ++ks) {
                        const uint32_t acc = (used >> s) & 1u;
                        mma_tf32(dt, dah + ks * sa, dbh + ks * sb, idesc, acc);
                        mma_tf32(dt, dah + ks * sa, dbl + ks * sb, idesc, 1u);
                        mma_tf32(dt, dal + ks * sa, dbh + ks * sb, idesc, 1u);
                        used |= 1u << s;
                    }
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
        }
        // wait until the tensor core has consumed the staged operands
        const bool waited = mbar_wait(bar, phase, spin_limit);
        // one decision for the whole CTA (every thread then takes the same barriers)
        if (!__syncthreads_and(waited)) {
            if (tid == 0) set_status(status, ST_ETIMEOUT);
            ok = false;
            // second bounded wait, so that TMEM is not freed under MMAs in flight
            mbar_wait(bar, phase, 1LL << 26);
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (ok && jn < ncand) request_b(jn);
        j = jn;
    }
    // no asynchronous copy may still be writing shared memory past this point
    cp_async_wait_all();
    __syncthreads();
    if (tid == 0) used_mask = used;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t umask = used_mask;
    if (ok && tid < 128) {
        for (int s = 0; s < S; ++s) {
            if (!(sub_mask & (1u << s))) continue;
            const int Px = Px0 + s * 128 + tid;
            float v[TC_MAX_NPAD];
            if (umask & (1u << s)) {
                const uint32_t taddr = tbase + (uint32_t(warp * 32) << 16) + uint32_t(s * Npad);
                for (int c0 = 0; c0 < Npad; c0 += 16) tmem_ld16(taddr + uint32_t(c0), v + c0);
            } else {
#pragma unroll
                for (int i = 0; i < TC_MAX_NPAD; ++i) v[i] = 0.f;
            }
            const uint32_t ix = uint32_t(2 * Px + cx), iy = uint32_t(2 * Py + cy);
            if (box_count(st, L, l, morton_key(ix, iy))) {
                float2 *dst = le + d.eoff + (lvl_off(l) + int64_t(c) * quarter + int64_t(Py) * W + Px) * p;
                for (int m = 0; m < p; ++m) dst[m] = make_float2(v[m], v[p + m]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols));
}

// ----------------------------------------------------------------------------
// Block units: one CTA per block of 8 x 16 parent cells (x, y), all four
// target classes.  The block's 128 parent cells are the MMA's M rows (cell
// row y = core-matrix group y) and the four classes sit side by side in N:
// columns c Npad .. c Npad + 2p - 1 hold class c's coefficients.  The source
// cells of a target class c at parent P are P + (dx, dy) in source class c'
// for every class c (only the operator depends on c), so for each source
// class c' the CTA stages, once, the block's cells plus a one-cell halo
// (10 x 18 cells, empty and out-of-domain boxes as zeros) in the K-major
// layout with a staged row of 10 cells as the group stride (SBO), and each of
// the nine parent offsets (dx, dy) is one 128 x 4Npad x 2p product whose A
// starts dy staged rows and dx cells away and whose B is the four classes'
// operators T_delta, delta = (2 dx + c'x - cx, 2 dy + c'y - cy), side by side
// (zero for a class whose delta is within one box; each class padded to a
// multiple of 8 columns, NW = 2p rounded up).  Wide N amortises each A read
// from shared memory over four operators.
//
// Pipeline.  The offsets run in a fixed order, source class by source class,
// each as S stages: S = 1, its B hi and lo images together (three products);
// S = 2, its B hi image (products A_hi B_hi and A_lo B_hi), then its B lo
// image (A_hi B_lo).  Stage h's images arrive by one bulk asynchronous copy
// into buffer h mod 2 on mbarrier bbar[h mod 2]; its MMAs complete on
// mbar[h mod 2].  Thread 0 issues copies and MMAs and alone waits
// on the barriers, always in stage order, so no barrier runs a phase ahead
// of its waiter: stage h + 1's copy is issued, once stage h - 1's MMAs (the
// last reader of that buffer) are done, before stage h's MMAs, and lands
// while they run.  A new source class is split into A once every MMA so far
// is done.  With S = 2 a CTA holds 109 KB of shared memory at p = 17, so two
// share an SM and one's splits overlap the other's MMAs, at twice the waits
// per offset: the launch takes S = 2 when it has many blocks (a full tree of
// >= 10 levels, a batch) and S = 1 (181 KB, one CTA per SM) otherwise.
// ----------------------------------------------------------------------------
constexpr int TCB_HX = TCB_BX + 2, TCB_HY = TCB_BY + 2;
constexpr int TCB_HALO = TCB_HX * TCB_HY;  // staged cells per source class
constexpr int TCB_M = TCB_BX * TCB_BY;     // parent cells per block

// delta's operator for target class c, source class cs and parent offset
// (dx, dy), or -1 if delta is within one box
__host__ __device__ __forceinline__ int tcb_op(int c, int cs, int dx, int dy) {
    const int ddx = 2 * dx + (cs & 1) - (c & 1), ddy = 2 * dy + (cs >> 1) - (c >> 1);
    const int ax = ddx < 0 ? -ddx : ddx, ay = ddy < 0 ? -ddy : ddy;
    return (ax > ay ? ax : ay) >= 2 ? m2l_op_index(ddx, ddy) : -1;
}

template <int S, bool DA>
__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tcb(
    const Task *__restrict__ tasks, int ntasks, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float2 *__restrict__ me, float2 *__restrict__ le,
    const uint32_t *__restrict__ ucount, int dense_pct, long long spin_limit, int *status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2], bbar[2];
    __shared__ uint32_t tslot;
    __shared__ uint32_t sany;
    __shared__ int s_issued;
    __shared__ uint8_t hocc[4][TCB_HALO];  // occupied halo cells, per source class

    const int tid = threadIdx.x, warp = tid >> 5;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const InstDesc &d = insts[t.inst];
    const int l = t.level, L = d.L, p = d.p;
    const int W = 1 << (l - 1);
    int Py0, Px0;
    tcb_unit_decode(l, int64_t(blockIdx.x) - t.block0, &Py0, &Px0);
    // sparse units are left to the SIMT kernel (same test there)
    if (!tc_unit_dense(ucount[blockIdx.x], 4 * TCB_M, dense_pct)) return;
    const uint32_t *st = start + d.soff;

    const int K2 = 2 * p;
    const int Kpad = (K2 + 7) & ~7, NW = (K2 + 7) & ~7, NC = 4 * NW;
    const int KG = Kpad / 4;
    const size_t aplane = size_t(KG) * TCB_HALO * 4;  // floats of A hi (or lo)
    const size_t bplane = size_t(Kpad) * NC;          // floats of one B image (hi or lo)
    const size_t bstage = size_t(3 - S) * bplane;     // floats of one stage's images
    // DA: two A buffers (a source class is split into one while the other's
    // MMAs run); each holds hi, then lo
    constexpr int NA = DA ? 2 : 1;
    float *A = reinterpret_cast<float *>(smem);       // hi, then lo (then the second buffer)
    float *B = A + NA * 2 * aplane;                   // 2 buffers of one stage
    // zero the K padding of every staged cell once (never overwritten)
    for (int i = tid; i < TCB_HALO * (Kpad - K2); i += TC_THREADS) {
        const int r = i / (Kpad - K2), k = K2 + i % (Kpad - K2);
        const size_t o = (size_t(k >> 2) * TCB_HALO + r) * 4 + (k & 3);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            A[a * 2 * aplane + o] = 0.f;
            A[a * 2 * aplane + aplane + o] = 0.f;
        }
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bbar[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        sany = 0;
    }
    uint32_t ncols = 32;
    while (ncols < uint32_t(NC)) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // occupancy of the halo cells of all four source classes (one round)
    for (int i = tid; i < 4 * TCB_HALO; i += TC_THREADS) {
        const int cs = i / TCB_HALO, q = i - cs * TCB_HALO;
        const int hy = q / TCB_HX, hx = q - hy * TCB_HX;
        const int Px = Px0 - 1 + hx, Py = Py0 - 1 + hy;
        bool o = false;
        if (Px >= 0 && Px < W && Py >= 0 && Py < W)
            o = box_count(st, L, l, morton_key(uint32_t(2 * Px + (cs & 1)),
                                               uint32_t(2 * Py + (cs >> 1)))) != 0;
        hocc[cs][q] = o;
        if (o) atomicOr(&sany, 1u << cs);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NC >> 3) << 17) |
                           (uint32_t(128 >> 4) << 24);
    const uint32_t LBO_A = uint32_t(TCB_HALO) * 16, SBO_A = uint32_t(TCB_HX) * 16;
    const uint32_t LBO_B = uint32_t(NC) * 16, SBO_B = 128;
    const int64_t quarter = int64_t(1) << (2 * (l - 1));
    const float2 *lev = me + d.eoff + lvl_off(l) * p;
    const float *bimg = static_cast<const float *>(d.t_m2l_tcb);

    // the offsets (source class, dy, dx) of occupied source classes with an
    // operator for some target class, as g = cs 9 + (dy + 1) 3 + dx + 1, in a
    // fixed order; the same list in every thread
    const uint32_t cs_any = sany;
    int ng = 0;
    uint8_t gl[36];
    for (int cs = 0; cs < 4; ++cs) {
        if (!((cs_any >> cs) & 1u)) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                bool any = false;
                for (int c = 0; c < 4; ++c) any |= tcb_op(c, cs, dx, dy) >= 0;
                if (any) gl[ng++] = uint8_t(cs * 9 + (dy + 1) * 3 + dx + 1);
            }
    }
    // element e of a staged class is coefficient k of cell q, e = q p + k,
    // with q = e * inv_p >> 20 (exact for e < 2^14, p <= 24); eight loads in
    // flight per thread before the first is used
    const uint32_t inv_p = ((1u << 20) + uint32_t(p) - 1) / uint32_t(p);
    constexpr int SB = 8;
    auto split = [&](int cs, int buf, int t0, int nt) {
        float *hi = A + size_t(buf) * 2 * aplane, *lo = hi + aplane;
        const int total = TCB_HALO * p;
        for (int e0 = t0; e0 < total; e0 += SB * nt) {
            float2 v[SB];
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int e = e0 + u * nt;
                v[u] = make_float2(0.f, 0.f);
                if (e < total) {
                    const int q = int((uint32_t(e) * inv_p) >> 20), k = e - q * p;
                    if (hocc[cs][q]) {
                        const int hy = q / TCB_HX, hx = q - hy * TCB_HX;
                        v[u] = __ldg(lev + (int64_t(cs) * quarter + int64_t(Py0 - 1 + hy) * W +
                                            (Px0 - 1 + hx)) * p + k);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int e = e0 + u * nt;
                if (e >= total) break;
                const int q = int((uint32_t(e) * inv_p) >> 20), k = e - q * p;
                const float hr = tf32_hi(v[u].x), him = tf32_hi(v[u].y);
                const size_t o_re = (size_t(k >> 2) * TCB_HALO + q) * 4 + (k & 3);
                const size_t o_im = (size_t((k + p) >> 2) * TCB_HALO + q) * 4 + ((k + p) & 3);
                hi[o_re] = hr;
                lo[o_re] = v[u].x - hr;
                hi[o_im] = him;
                lo[o_im] = v[u].y - him;
            }
        }
    };
    // thread 0's state: stages whose MMAs are known complete, whose B copy
    // was issued and has landed, MMAs issued, and whether every wait so far
    // ended in time; stage h is offset gl[h / S] (S = 2: image h % 2, hi or lo)
    const int nh = S * ng;
    int done = -1, copied = -1, landed = -1, issued = -1;
    bool ok0 = true;
    auto wait_mma = [&](int k) {  // thread 0 only, in stage order
        for (int kk = done + 1; kk <= k && ok0; ++kk) {
            ok0 = mbar_wait(smem_addr(&mbar[kk & 1]), uint32_t(kk >> 1) & 1u, spin_limit);
            if (ok0) done = kk;
        }
    };
    const uint32_t bbytes = uint32_t(bstage * 4);
    auto copy_b = [&](int k) {  // thread 0 only
        const uint32_t bb = smem_addr(&bbar[k & 1]);
        mbar_arrive_expect_tx(bb, bbytes);
        const size_t src = (size_t(gl[k / S]) * 2 + size_t(S == 2 ? (k & 1) : 0)) * bplane;
        bulk_g2s(smem_addr(B + size_t(k & 1) * bstage), bimg + src, bbytes, bb);
        copied = k;
    };
    bool ok = true;
    if (ng > 0) {
        split(gl[0] / 9, 0, tid, TC_THREADS);
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
    }
    // Thread 0: stage h, its MMAs reading A buffer abuf.  They are issued
    // as soon as stage h's images have landed, queued behind stage h - 1's
    // (so the tensor core does not drain between stages); then, once stage
    // h - 1 is done, stage h + 1's images go to the buffer it read, to land
    // while stage h multiplies.
    auto issue_stage = [&](int h, int abuf) {
        if (h == 0) copy_b(0);
        if (h + 1 < nh && ok0) {
            wait_mma(h - 1);
            if (ok0) copy_b(h + 1);
        }
        if (ok0) {
            ok0 = mbar_wait(smem_addr(&bbar[h & 1]), uint32_t(h >> 1) & 1u, spin_limit);
            if (ok0) landed = h;
        }
        if (ok0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int g = h / S;
            const int dy = (gl[g] % 9) / 3 - 1, dx = gl[g] % 3 - 1;
            const uint32_t ahi = smem_addr(A + size_t(abuf) * 2 * aplane),
                           alo = ahi + uint32_t(aplane * 4);
            const uint32_t bimg_s = smem_addr(B + size_t(h & 1) * bstage);
            const uint64_t sa = (2 * LBO_A) >> 4, sb = (2 * LBO_B) >> 4;
            const uint64_t db = mma_desc(bimg_s, LBO_B, SBO_B);
            const uint64_t dbl = mma_desc(bimg_s + uint32_t(bplane * 4), LBO_B, SBO_B);
            const uint32_t cell0 = uint32_t((1 + dy) * TCB_HX + 1 + dx) * 16;
            const uint64_t dah = mma_desc(ahi + cell0, LBO_A, SBO_A);
            const uint64_t dal = mma_desc(alo + cell0, LBO_A, SBO_A);
            uint32_t acc = issued >= 0 ? 1u : 0u;
            for (int ks = 0; ks < Kpad / 8; ++ks) {
                if (S == 1) {
                    mma_tf32(tbase, dah + ks * sa, db + ks * sb, idesc, acc);
                    mma_tf32(tbase, dah + ks * sa, dbl + ks * sb, idesc, 1u);
                    mma_tf32(tbase, dal + ks * sa, db + ks * sb, idesc, 1u);
                } else {
                    mma_tf32(tbase, dah + ks * sa, db + ks * sb, idesc, acc);
                    if (!(h & 1)) mma_tf32(tbase, dal + ks * sa, db + ks * sb, idesc, 1u);
                }
                acc = 1u;
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&mbar[h & 1])));
            issued = h;
        }
    };
    if constexpr (DA) {
        // One source class at a time: thread 0 issues the class's stages from
        // A buffer cur while warps 1-7 split the next class into the other
        // buffer.  That buffer's last readers are the previous class's MMAs:
        // thread 0 first queues this class's first stage behind them, then
        // waits for them, and only then lets the splitters in.
        int cur = 0;
        for (int h0 = 0; h0 < nh && ok;) {
            int h1 = h0 + S;
            while (h1 < nh && gl[h1 / S] / 9 == gl[h0 / S] / 9) h1 += S;
            if (tid == 0 && ok0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                issue_stage(h0, cur);
                if (ok0) wait_mma(h0 - 1);
            }
            ok = __syncthreads_and(tid != 0 || ok0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                for (int h = h0 + 1; h < h1 && ok0; ++h) issue_stage(h, cur);
            } else if (warp > 0 && h1 < nh) {
                split(gl[h1 / S] / 9, cur ^ 1, tid - 32, TC_THREADS - 32);
                asm volatile("fence.proxy.async.shared::cta;");
            }
            ok = __syncthreads_and(tid != 0 || ok0);
            cur ^= 1;
            h0 = h1;
        }
    }
    for (int h = 0; h < (DA ? 0 : nh) && ok; ++h) {
        if (tid == 0 && ok0) issue_stage(h, 0);
        // a new source class: split it into A once every MMA so far is done
        if (h + 1 < nh && (h + 1) % S == 0 && gl[(h + 1) / S] / 9 != gl[h / S] / 9) {
            if (tid == 0 && ok0) wait_mma(h);
            ok = __syncthreads_and(tid != 0 || ok0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            split(gl[(h + 1) / S] / 9, 0, tid, TC_THREADS);
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
        }
    }
    if (tid == 0 && ok0) wait_mma(issued);
    ok = __syncthreads_and(tid != 0 || ok0) && ok;
    if (!ok) {
        if (tid == 0) {
            set_status(status, ST_ETIMEOUT);
            // let the copies and MMAs in flight finish before the shared
            // memory and TMEM go (bounded, in order)
            for (int kk = landed + 1; kk <= copied; ++kk)
                mbar_wait(smem_addr(&bbar[kk & 1]), uint32_t(kk >> 1) & 1u, 1LL << 26);
            for (int kk = done + 1; kk <= issued; ++kk)
                mbar_wait(smem_addr(&mbar[kk & 1]), uint32_t(kk >> 1) & 1u, 1LL << 26);
        }
        __syncthreads();
    }
    if (tid == 0) s_issued = issued;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // warp w reads TMEM lanes 32 (w mod 4) .. (M rows = cells (m mod 8,
        // m / 8)); warps 0-3 take target classes 0 and 1, warps 4-7 classes 2, 3
        const int m = (warp & 3) * 32 + (tid & 31);
        const int Px = Px0 + (m & 7), Py = Py0 + (m >> 3);
        for (int cc = 0; cc < 2; ++cc) {
            const int c = (warp >> 2) * 2 + cc;
            // class c's columns c NW .. c NW + 2p - 1, read in 16-column chunks
            // from the 16-aligned column at or below c NW
            const int a0 = (c * NW) & ~15, off = c * NW - a0;
            const int nch = (off + K2 + 15) / 16;
            float v[64];
            if (s_issued >= 0) {
                const uint32_t taddr = tbase + (uint32_t((warp & 3) * 32) << 16) + uint32_t(a0);
                for (int q = 0; q < nch; ++q) tmem_ld16(taddr + uint32_t(16 * q), v + 16 * q);
            } else {
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = 0.f;
            }
            const uint32_t ix = uint32_t(2 * Px + (c & 1)), iy = uint32_t(2 * Py + (c >> 1));
            if (box_count(st, L, l, morton_key(ix, iy))) {
                float2 *dst =
                    le + d.eoff + (lvl_off(l) + int64_t(c) * quarter + int64_t(Py) * W + Px) * p;
                for (int k = 0; k < p; ++k) dst[k] = make_float2(v[off + k], v[off + p + k]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols));
}

// stages per offset: 2 for launches of many blocks
constexpr int64_t kTcbTwoStageUnits = 2048;
static int tcb_stages(int64_t nblocks) { return nblocks >= kTcbTwoStageUnits ? 2 : 1; }

static size_t tcb_smem_bytes(int p, int S, bool da = false) {
    const int K2 = 2 * p, Kpad = (K2 + 7) & ~7, NW = (K2 + 7) & ~7;
    // A hi and lo of one staged class (two with da); two buffers of one
    // stage's B images
    return size_t(da ? 4 : 2) * (Kpad / 4) * TCB_HALO * 16 +
           size_t(2) * (3 - S) * Kpad * (4 * NW) * 4;
}

// Most dynamic shared memory a block unit may take (plus the static part).
constexpr size_t kTcbSmemMax = size_t(220) * 1024;

size_t m2l_tcb_smem_bytes(int p) { return tcb_smem_bytes(p, 1); }

bool m2l_tcb_supported(int p, int level) {
    const int Npad = (2 * p + 15) & ~15;
    return level >= 5 && level <= 15 && Npad <= TC_MAX_NPAD &&
           m2l_tcb_smem_bytes(p) <= size_t(220) * 1024;
}

int64_t m2l_tcb_units(int level) {
    const int64_t W = int64_t(1) << (level - 1);
    return (W / TCB_BX) * (W / TCB_BY);
}

// B images of the block units for p: for each (source class c', dy, dx), as
// g = c' 9 + (dy + 1) 3 + dx + 1, hi then lo, each Kpad x 4NW floats (NW = 2p
// rounded up to 8) in the K-major core-matrix layout [k / 4][n][k % 4],
// n = c NW + (column of the row-unit image of class c's operator, zero if
// none).
void host_m2l_tcb_images(int p, int kernel, std::vector<float> &out) {
    const int K2 = 2 * p, Kpad = (K2 + 7) & ~7, Npad = (K2 + 15) & ~15, NW = (K2 + 7) & ~7;
    const int NC = 4 * NW;
    std::vector<float> ops;
    host_m2l_tc_images(p, kernel, ops);
    const size_t oslot = size_t(Kpad) * Npad, bslot = size_t(Kpad) * NC;
    out.assign(size_t(36) * 2 * bslot, 0.0f);
    for (int cs = 0; cs < 4; ++cs)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int g = cs * 9 + (dy + 1) * 3 + dx + 1;
                for (int c = 0; c < 4; ++c) {
                    const int op = tcb_op(c, cs, dx, dy);
                    if (op < 0) continue;
                    for (int hl = 0; hl < 2; ++hl) {
                        const float *src = ops.data() + (size_t(op) * 2 + hl) * oslot;
                        float *dst = out.data() + (size_t(g) * 2 + hl) * bslot;
                        for (int kg = 0; kg < Kpad / 4; ++kg)
                            for (int n = 0; n < NW; ++n)
                                for (int r = 0; r < 4; ++r)
                                    dst[(size_t(kg) * NC + c * NW + n) * 4 + r] =
                                        src[(size_t(kg) * Npad + n) * 4 + r];
                    }
                }
            }
}

cudaError_t launch_m2l_tcb(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                           const uint32_t *start, const float2 *me, float2 *le,
                           const uint32_t *ucount, int dense_pct, int pmax, long long spin_limit,
                           int pipe, int *status, cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    // pipe 2: double-buffered A, one stage per offset (if it fits); 1: the
    // single A, stages by launch size; 0: automatic
    // (measured on GB300, M2L stage: two CTAs per SM with two stages per
    // offset beat one CTA with the double buffer in launches of >= 2048
    // blocks -- Lamb-Oseen 1.05 against 1.16 ms, clustered-16M 0.36 against
    // 0.38 ms -- while in smaller launches, one CTA per SM either way, the
    // double buffer gains: lattice-1M 0.188 -> 0.184 ms)
    const bool da_fits = tcb_smem_bytes(pmax, 1, true) <= kTcbSmemMax;
    const bool da = pipe == 2   ? da_fits
                    : pipe == 1 ? false
                                : da_fits && tcb_stages(nblocks) == 1;
    const int S = da ? 1 : tcb_stages(nblocks);
    const size_t smem_bytes = tcb_smem_bytes(pmax, S, da);
    auto k = da ? k_m2l_tcb<1, true> : S == 2 ? k_m2l_tcb<2, false> : k_m2l_tcb<1, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem_bytes));
    if (e != cudaSuccess) return e;
    k<<<unsigned(nblocks), TC_THREADS, smem_bytes, st>>>(tasks, ntasks, insts, start, me, le, ucount,
                                                         dense_pct, spin_limit, status);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

size_t m2l_tc_smem_bytes(int p, int seg) {
    const int K2 = 2 * p, Kpad = (K2 + 7) & ~7, Npad = (K2 + 15) & ~15;
    // A hi and lo, six B images, the raw strip (seg + 2 rows of p complex)
    return size_t(2) * (Kpad / 4) * (seg + 2) * 16 + size_t(6) * Kpad * Npad * 4 +
           size_t(seg + 2) * p * 8;
}

int m2l_tc_seg(int level, int segmax) { return tc_seg(level, segmax); }

bool m2l_tc_supported(int p, int level, int segmax) {
    const int Npad = (2 * p + 15) & ~15;
    return level >= 8 && level <= 15 && Npad <= TC_MAX_NPAD &&
           m2l_tc_smem_bytes(p, m2l_tc_seg(level, segmax)) <= size_t(220) * 1024;
}

int64_t m2l_tc_units(int level, int segmax) {
    const int64_t W = int64_t(1) << (level - 1);
    return 4 * W * (W / tc_seg(level, segmax));
}

// B images for p: for each of the 40 offsets, hi then lo, each Kpad x Npad
// floats in the K-major core-matrix layout [k / 4][n][k % 4].
void host_m2l_tc_images(int p, int kernel, std::vector<float> &out) {
    const int K2 = 2 * p, Kpad = (K2 + 7) & ~7, Npad = (K2 + 15) & ~15;
    std::vector<double> T(size_t(40) * p * p * 2);
    if (kernel == KERNEL_LAPLACE)
        host_lap_m2l_table(p, T.data());  // [op][k][m] complex
    else
        host_m2l_table(p, T.data());
    const size_t slot = size_t(Kpad) * Npad;
    out.assign(size_t(40) * 2 * slot, 0.0f);
    for (int op = 0; op < 40; ++op) {
        float *hi = out.data() + size_t(op) * 2 * slot;
        float *lo = hi + slot;
        for (int n = 0; n < K2; ++n)
            for (int k = 0; k < K2; ++k) {
                const int m = n < p ? n : n - p, kk = k < p ? k : k - p;
                const double *tc = T.data() + ((size_t(op) * p + kk) * p + m) * 2;
                const double tr = tc[0], tim = tc[1];
                double b;
                if (n < p) b = k < p ? tr : -tim;
                else b = k < p ? tim : tr;
                const float bf = float(b);
                uint32_t bits;
                std::memcpy(&bits, &bf, 4);
                bits &= 0xFFFFE000u;
                float h;
                std::memcpy(&h, &bits, 4);
                const size_t o = (size_t(k >> 2) * Npad + n) * 4 + (k & 3);
                hi[o] = h;
                lo[o] = float(b - double(h));
            }
    }
}

cudaError_t launch_tc_unit_count(const Task *tasks, int ntasks, int64_t nunits,
                                 const InstDesc *insts, const uint32_t *start, uint32_t *ucount,
                                 cudaStream_t st, uint64_t *launches) {
    if (nunits <= 0) return cudaSuccess;
    const int64_t blocks = (nunits * 32 + 255) / 256;
    k_tc_unit_count<<<unsigned(blocks), 256, 0, st>>>(tasks, ntasks, insts, start, ucount, nunits);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                          const uint32_t *start, const float2 *me, float2 *le,
                          const uint32_t *ucount, int dense_pct, size_t smem_bytes,
                          long long spin_limit, int *status, cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem_bytes));
    if (e != cudaSuccess) return e;
    k_m2l_tc<<<unsigned(nblocks), TC_THREADS, smem_bytes, st>>>(tasks, ntasks, insts, start, me, le,
                                                                ucount, dense_pct, spin_limit, status);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

}  // namespace petfmm
