// tree.cu -- the uniform quadtree of Sec. 2.1 on the device: binning with
// z-order keys (Sec. 5.1), a stable LSD radix sort of the keys, the leaf
// ranges, and the gather of the particles into sorted order.
//
// All of it is bandwidth-bound.  Per particle the algorithmic traffic is one
// read of x, y and one key write (binning), one read of the key for the digit
// counts of all passes, then per radix pass one read and one write of
// (key, value), and finally a gather of x, y, gamma into sorted order.
#include <cstdio>

#include "kernels.cuh"

namespace petfmm {

#define PF_LAUNCHED(n) do { if (launches) *launches += (n); } while (0)

// ----------------------------------------------------------------------------
// Binning: t = x - x0; s = t * (2^L / W); ix = floor(s) clamped to [0, 2^L-1].
// The FP64 operations are spelled as round-to-nearest intrinsics so that no
// contraction can change a bit; the host computes 2^L / W once.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bin_coord(double x, double x0, double scale, uint32_t nb) {
    double t = __dsub_rn(x, x0);
    double s = __dmul_rn(t, scale);
    double f = floor(s);
    if (!(f >= 0.0)) return 0u;  // also NaN (reported separately)
    if (f > double(nb - 1)) return nb - 1;
    return uint32_t(f);
}

// Leaf-relative coordinate (x - c) scale, c = x0 + (i + 1/2) w, computed as
// (x - x0) scale - (i + 1/2) in float-float arithmetic (x0 = x0h + x0l,
// scale = sh + sl; two-sum for the difference, an FMA for the product's
// error): the result before its final rounding to FP32 is within about 2^-44
// of the exact value, relative to (x - x0) scale.
__device__ __forceinline__ void split_ff(float x, float *h, float *l) { *h = x; *l = 0.0f; }
__device__ __forceinline__ void split_ff(double x, float *h, float *l) {
    *h = float(x);
    *l = float(x - double(*h));
}
template <typename TIn>
__device__ __forceinline__ float leaf_coord(TIn xin, float x0h, float x0l, float sh, float sl,
                                            uint32_t i) {
    float xh, xl;
    split_ff(xin, &xh, &xl);
    // t = x - x0 = th + tl
    const float th = __fsub_rn(xh, x0h);
    const float bb = __fsub_rn(th, xh);
    float tl = __fadd_rn(__fsub_rn(xh, __fsub_rn(th, bb)), __fsub_rn(-x0h, bb));
    tl = __fadd_rn(tl, __fsub_rn(xl, x0l));
    // s = t scale = p + e
    const float p = __fmul_rn(th, sh);
    float e = __fmaf_rn(th, sh, -p);
    e = __fmaf_rn(th, sl, __fmaf_rn(tl, sh, e));
    return __fadd_rn(__fsub_rn(p, __fadd_rn(float(i), 0.5f)), e);
}

// FP32 shortcut (FP64 arithmetic is slow on this GPU).  With xf, x0f and
// scalef the FP32 roundings of x, x0 and scale, s32 = fl(fl(xf - x0f) scalef)
// differs from the FP64 s above by at most 4 u scale (|x| + |x0|) plus terms
// of order u^2 (u = 2^-24: one rounding each of xf, x0f, scalef, the
// difference and the product); the margin m = 8 u scale (|x| + |x0|) also
// covers the roundings of s32 -/+ m.  If both ends of [s32 - m, s32 + m] fall
// in the same bin and inside (0, nb (1 - 2^-20)), the FP64 value s is in that
// bin too (no clamping) and the point is inside the domain: s > 0 means
// fl(x - x0) > 0, i.e. x > x0; s < nb (1 - 2^-20) bounds x - x0 below
// W (1 - 2^-21), so x <= fl(x0 + W) whenever |x0 + W| <= 2^32 W -- and a
// domain farther from the origin has m > nb, so the test fails there.
// Otherwise (near a bin edge or the domain boundary, NaN, Inf) returns false
// and the caller takes the FP64 path.  The result is therefore bit-identical.
__device__ __forceinline__ bool bin_coord_fast(float xf, float x0f, float scalef, uint32_t nb,
                                               uint32_t *bin) {
    const float s = __fmul_rn(__fsub_rn(xf, x0f), scalef);
    const float m = __fmul_rn(__fmul_rn(__fadd_rn(fabsf(xf), fabsf(x0f)), scalef), 0x1p-21f);
    const float lo = __fsub_rn(s, m), hi = __fadd_rn(s, m);
    if (!(lo > 0.0f && hi < float(nb) * (1.0f - 0x1p-20f))) return false;
    const float f = floorf(lo);
    if (f != floorf(hi)) return false;
    *bin = uint32_t(f);
    return true;
}

// recu != nullptr (mixed path): also the blob's record in input order,
// (xi, eta, gamma, batch index) with (xi, eta) its offset from its leaf's
// centre in leaf widths.
template <typename TIn>
__global__ void __launch_bounds__(256) k_morton(const Task *__restrict__ tasks, int ntasks,
                                                const InstDesc *__restrict__ insts,
                                                uint32_t *__restrict__ keys,
                                                float4 *__restrict__ recu, int *status) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t j = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (j >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const TIn xin = static_cast<const TIn *>(d.x)[j];
    const TIn yin = static_cast<const TIn *>(d.y)[j];
    const uint32_t nb = 1u << d.L;
    uint32_t ix, iy;
    if (!(bin_coord_fast(float(xin), d.x0h, d.sh, nb, &ix) &&
          bin_coord_fast(float(yin), d.y0h, d.sh, nb, &iy))) {
        const double x = double(xin), y = double(yin);
        const double x1 = __dadd_rn(d.x0, d.width), y1 = __dadd_rn(d.y0, d.width);
        if (!(x >= d.x0 && x <= x1 && y >= d.y0 && y <= y1)) set_status(status, ST_EDOMAIN);
        ix = bin_coord(x, d.x0, d.scale, nb);
        iy = bin_coord(y, d.y0, d.scale, nb);
    }
    keys[d.poff + j] = d.key_hi | morton_key(ix, iy);
    if (recu) {
        float4 o;
        o.x = leaf_coord(xin, d.x0h, d.x0l, d.sh, d.sl, ix);
        o.y = leaf_coord(yin, d.y0h, d.y0l, d.sh, d.sl, iy);
        o.z = float(static_cast<const TIn *>(d.g)[j]);
        o.w = __uint_as_float(uint32_t(d.poff + j));
        recu[d.poff + j] = o;
    }
}

cudaError_t launch_morton(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                          int dtype_f32, uint32_t *keys, float4 *recu, int *status,
                          cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    if (dtype_f32)
        k_morton<float><<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, keys, recu, status);
    else
        k_morton<double><<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, keys, recu,
                                                            status);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Exclusive scan (reduce-then-scan, recursive over tiles of 2048).
// ----------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t n = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += n;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = warp ? warp_sums[warp - 1] : 0u;
    *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before + incl - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile_sums(const uint32_t *__restrict__ in,
                                                                 int64_t n,
                                                                 uint32_t *__restrict__ sums) {
    const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + int64_t(k) * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t total;
    block_exclusive_sum(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t *in, uint32_t *out,
                                                             int64_t n,
                                                             const uint32_t *__restrict__ prefix,
                                                             uint32_t *total_out) {
    const int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_sum(s, &total);
    const uint32_t p0 = prefix ? prefix[blockIdx.x] : 0u;
    run += p0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = p0 + total;
}

int64_t scan_scratch_words(int64_t n) {
    int64_t w = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        w += n;
    }
    return w + 1;
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch,
                           uint32_t *total, cudaStream_t st, uint64_t *launches) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    if (n <= SCAN_TILE) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, total);
        PF_LAUNCHED(1);
        return cudaGetLastError();
    }
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t *sums = scratch;
    k_scan_tile_sums<<<unsigned(nt), SCAN_THREADS, 0, st>>>(in, n, sums);
    PF_LAUNCHED(1);
    cudaError_t e = exclusive_scan(sums, sums, nt, scratch + nt, nullptr, st, launches);
    if (e != cudaSuccess) return e;
    k_scan_tiles<<<unsigned(nt), SCAN_THREADS, 0, st>>>(in, out, n, sums, total);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, reduce-then-scan.  Per pass:
// k_radix_counts counts the digits of each tile of RS_TILE consecutive
// elements in digit-major order, count[digit * tiles + tile]; an exclusive
// scan of that gives every (digit, tile) its first output position; then
// k_radix_scatter moves the tile.
//
// Within a tile, warp w owns the consecutive chunk [w * RS_WCHUNK, (w + 1) *
// RS_WCHUNK) and reads it in rounds of 32 (lane order), so (warp, round, lane)
// is the input order.  The ranks within the warp (digit_peers per round)
// become positions in the tile sorted by digit; the tile is sorted in shared
// memory and each digit's run written to its place in the output, consecutive
// threads to consecutive addresses.
// ----------------------------------------------------------------------------
// Lanes of the warp holding the same digit as this lane (bit d of the
// 9-bit value 0..256, 256 = no element): 9 ballots, which run on the ALU
// pipe, where __match_any_sync stalls on a long-latency unit.
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const bool bit = (dg >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

constexpr int RS_THREADS = 512;
constexpr int RS_ITEMS = 8;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_WCHUNK = RS_ITEMS * 32;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
static_assert(RS_WCHUNK <= 256 && RS_ITEMS % 4 == 0 && RS_TILE < 65536,
              "ranks packed as 8-bit fields, warp offsets as 16-bit");
constexpr int RC_THREADS = 256;

int64_t radix_blocks(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

int64_t radix_scratch_words(int64_t n) {
    const int64_t c = 256 * radix_blocks(n);
    return c + scan_scratch_words(c);
}

// n_live (device, may be null): only the first *n_live of the n elements
// take part; tiles past them count nothing and move nothing.
__device__ __forceinline__ int64_t live_count(int64_t n, const uint32_t *n_live) {
    if (!n_live) return n;
    const int64_t m = int64_t(*n_live);
    return m < n ? m : n;
}

// Exclusive sums of (a, b) over the block's NT threads.
template <int NT>
__device__ __forceinline__ void block_exclusive_sum2(uint32_t a, uint32_t b, uint32_t *ea,
                                                     uint32_t *eb, uint2 *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t na = __shfl_up_sync(0xffffffffu, ia, o);
        const uint32_t nb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += na;
            ib += nb;
        }
    }
    if (lane == 31) ws[warp] = make_uint2(ia, ib);
    __syncthreads();
    if (warp == 0) {
        uint2 s = lane < NT / 32 ? ws[lane] : make_uint2(0u, 0u);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t nx = __shfl_up_sync(0xffffffffu, s.x, o);
            const uint32_t ny = __shfl_up_sync(0xffffffffu, s.y, o);
            if (lane >= o) {
                s.x += nx;
                s.y += ny;
            }
        }
        if (lane < NT / 32) ws[lane] = s;
    }
    __syncthreads();
    const uint2 before = warp ? ws[warp - 1] : make_uint2(0u, 0u);
    *ea = before.x + ia - a;
    *eb = before.y + ib - b;
    __syncthreads();
}

// count[d * nblocks + tile]: elements of the tile whose digit
// (key >> shift) & mask is d (tiles past the live elements count zero).
__global__ void __launch_bounds__(RC_THREADS) k_radix_counts(const uint32_t *__restrict__ keys,
                                                             int64_t n, const uint32_t *n_live,
                                                             int shift, uint32_t mask,
                                                             uint32_t *__restrict__ count,
                                                             int64_t nblocks) {
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    n = live_count(n, n_live);
    const int64_t t0 = int64_t(blockIdx.x) * RS_TILE;
    uint32_t k[RS_TILE / RC_THREADS];
#pragma unroll
    for (int u = 0; u < RS_TILE / RC_THREADS; ++u) {
        const int64_t i = t0 + u * RC_THREADS + tid;
        k[u] = i < n ? keys[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < RS_TILE / RC_THREADS; ++u)
        if (t0 + u * RC_THREADS + tid < n) atomicAdd(&h[(k[u] >> shift) & mask], 1u);
    __syncthreads();
    count[int64_t(tid) * nblocks + blockIdx.x] = h[tid];
}

// One pass: digit (key >> shift) & mask; offs: the scanned counts (first
// output position of each digit of each tile).
template <bool FIRST>
__global__ void __launch_bounds__(RS_THREADS, 3) k_radix_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n, const uint32_t *n_live, int shift, uint32_t mask,
    const uint32_t *__restrict__ offs, int64_t nblocks) {
    __shared__ uint16_t wcnt[RS_WARPS][256];  // per-warp digit counts, then warp offsets
    __shared__ uint32_t lstart[256];          // start of each digit's run in the sorted tile
    __shared__ uint32_t gbase[256];           // its start in the output
    __shared__ uint32_t skey[RS_TILE], sval[RS_TILE];
    __shared__ uint2 wsum[RS_WARPS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    n = live_count(n, n_live);
    const int64_t t0 = int64_t(blockIdx.x) * RS_TILE;
    if (t0 >= n) return;
    const int64_t tile_n = n - t0 < RS_TILE ? n - t0 : RS_TILE;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    if (tid < 256) gbase[tid] = offs[int64_t(tid) * nblocks + blockIdx.x];
    __syncthreads();
    // 1. rank within the warp, in input order
    // rk: ranks within the warp (< RS_WCHUNK = 256), four 8-bit fields a word
    uint32_t key[RS_ITEMS], val[RS_ITEMS], rk[RS_ITEMS / 4] = {};
    const int64_t wbase = t0 + int64_t(warp) * RS_WCHUNK;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? (FIRST ? uint32_t(i) : vin[i]) : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const bool valid = wbase + r * 32 + lane < n;
        const uint32_t dg = valid ? (key[r] >> shift) & mask : 0x100u;
        const uint32_t peers = digit_peers(dg);
        const uint32_t below = peers & lt_mask;
        if (valid) rk[r >> 2] |= (wcnt[warp][dg] + __popc(below)) << (8 * (r & 3));
        __syncwarp();
        if (valid && below == 0) wcnt[warp][dg] = uint16_t(wcnt[warp][dg] + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // 2. per digit (thread tid < 256 = digit): the warps' offsets, then the
    //    runs' starts in the sorted tile
    uint32_t cnt = 0;
    if (tid < 256) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = uint16_t(cnt);
            cnt += c;
        }
    }
    uint32_t ls, unused;
    block_exclusive_sum2<RS_THREADS>(cnt, 0u, &ls, &unused, wsum);
    if (tid < 256) lstart[tid] = ls;
    __syncthreads();
    // 3. sort the tile in shared memory
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        if (wbase + r * 32 + lane < n) {
            const uint32_t dg = (key[r] >> shift) & mask;
            const uint32_t pos = lstart[dg] + wcnt[warp][dg] + ((rk[r >> 2] >> (8 * (r & 3))) & 0xffu);
            skey[pos] = key[r];
            sval[pos] = val[r];
        }
    }
    __syncthreads();
    // 4. write the runs
    for (int q = tid; q < tile_n; q += RS_THREADS) {
        const uint32_t k = skey[q];
        const uint32_t dg = (k >> shift) & mask;
        const uint32_t pos = gbase[dg] + (uint32_t(q) - lstart[dg]);
        if (!PF_IN(pos, n)) continue;
        kout[pos] = k;
        vout[pos] = sval[q];
    }
}

cudaError_t radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n,
                       int nbits, uint32_t *scratch, bool *result_in_first, cudaStream_t st,
                       uint64_t *launches, const uint32_t *n_live) {
    *result_in_first = true;
    if (n <= 0) return cudaSuccess;
    const int passes = (nbits + 7) / 8;
    if (passes <= 0 || passes > 4 || n > int64_t(0xffffffffu)) return cudaErrorInvalidValue;
    const int64_t nb = radix_blocks(n);
    uint32_t *count = scratch;
    uint32_t *scan = scratch + 256 * nb;
    uint32_t *kin = k0, *vin = nullptr, *kout = k1, *vout = v1;
    bool in_first = true;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const int bits = nbits - shift < 8 ? nbits - shift : 8;
        const uint32_t mask = (1u << bits) - 1u;
        k_radix_counts<<<unsigned(nb), RC_THREADS, 0, st>>>(kin, n, n_live, shift, mask, count, nb);
        PF_LAUNCHED(1);
        cudaError_t e = exclusive_scan(count, count, 256 * nb, scan, nullptr, st, launches);
        if (e != cudaSuccess) return e;
        if (pass == 0)
            k_radix_scatter<true><<<unsigned(nb), RS_THREADS, 0, st>>>(
                kin, vin, kout, vout, n, n_live, shift, mask, count, nb);
        else
            k_radix_scatter<false><<<unsigned(nb), RS_THREADS, 0, st>>>(
                kin, vin, kout, vout, n, n_live, shift, mask, count, nb);
        PF_LAUNCHED(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        in_first = !in_first;
        if (in_first) {
            kin = k0; vin = v0; kout = k1; vout = v1;
        } else {
            kin = k1; vin = v1; kout = k0; vout = v0;
        }
    }
    *result_in_first = in_first;
    return cudaSuccess;
}

// ----------------------------------------------------------------------------
// Leaf ranges: start[b] = lower_bound(sorted keys of the instance, key_hi | b).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_leaf_start(const Task *__restrict__ tasks, int ntasks,
                                                    const InstDesc *__restrict__ insts,
                                                    const uint32_t *__restrict__ skeys,
                                                    uint32_t *__restrict__ start) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t b = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (b >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int64_t nleaf = int64_t(1) << (2 * d.L);
    uint32_t r;
    if (b >= nleaf) {
        r = uint32_t(d.poff + d.n);
    } else {
        const uint32_t want = d.key_hi | uint32_t(b);
        int64_t lo = d.poff, hi = d.poff + d.n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (skeys[mid] < want) lo = mid + 1; else hi = mid;
        }
        r = uint32_t(lo);
    }
    start[d.soff + b] = r;
}

cudaError_t launch_leaf_start(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                              const uint32_t *skeys, uint32_t *start, cudaStream_t st,
                              uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    k_leaf_start<<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, skeys, start);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Gather into sorted order.  Task units are sorted ranks of one instance.
// ----------------------------------------------------------------------------
template <typename TIn>
__global__ void __launch_bounds__(256) k_gather_f64(const Task *__restrict__ tasks, int ntasks,
                                                    const InstDesc *__restrict__ insts,
                                                    const uint32_t *__restrict__ perm,
                                                    double *__restrict__ xs, double *__restrict__ ys,
                                                    double *__restrict__ gs) {
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const int64_t j = (int64_t(blockIdx.x) - t.block0) * blockDim.x + threadIdx.x;
    if (j >= t.count) return;
    const InstDesc &d = insts[t.inst];
    const int64_t r = d.poff + j;
    const int64_t q = int64_t(perm[r]) - d.poff;
    if (!PF_IN(q, d.n)) return;
    xs[r] = double(static_cast<const TIn *>(d.x)[q]);
    ys[r] = double(static_cast<const TIn *>(d.y)[q]);
    gs[r] = double(static_cast<const TIn *>(d.g)[q]);
}

// Mixed path: the records were built by the binning kernel in input order;
// the gather is one 16-byte permutation (a random read of one sector per
// blob, where reading x, y, gamma separately would touch three).
__global__ void __launch_bounds__(256) k_gather_mixed(const float4 *__restrict__ recu,
                                                      const uint32_t *__restrict__ perm,
                                                      float4 *__restrict__ rec, int64_t n) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r < n) {
        const uint32_t q = perm[r];
        rec[r] = PF_IN(q, n) ? recu[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

cudaError_t launch_gather_f64(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                              int dtype_f32, const uint32_t *perm, double *xs, double *ys,
                              double *gs, cudaStream_t st, uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    if (dtype_f32)
        k_gather_f64<float><<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, perm, xs, ys, gs);
    else
        k_gather_f64<double><<<unsigned(nblocks), 256, 0, st>>>(tasks, ntasks, insts, perm, xs, ys, gs);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_mixed(const float4 *recu, const uint32_t *perm, float4 *rec, int64_t n,
                                cudaStream_t st, uint64_t *launches) {
    if (n <= 0) return cudaSuccess;
    k_gather_mixed<<<unsigned((n + 255) / 256), 256, 0, st>>>(recu, perm, rec, n);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

PF_DEFINE_CHECK_READER(tree)

}  // namespace petfmm
