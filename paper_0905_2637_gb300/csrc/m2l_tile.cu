// m2l_tile.cu -- M2L (Sec. 2.2, downward sweep) as tiled SIMT GEMMs for the
// mixed path, on the levels the tensor cores do not take (parent rows of
// fewer than 128 cells) and for every level when they are switched off.
//
// The unit of work follows the tensor-core kernel's (m2l_tc.cu): one CTA per
// (target child class c, target boxes) -- a segment of 128 parent cells of
// one parent row, or R whole rows of together at most 64 cells where rows
// are shorter -- and it takes
// the unit only if at least dense_pct percent of its targets hold particles
// (the per-box SIMT kernel takes the boxes of the others).  For each of the
// 12 (source class c', parent row offset dy) strips the CTA stages, for each
// of its rows, the source expansions of the segment plus one cell on each
// side once in shared memory (empty or out-of-domain boxes as zeros), and the
// up to three operators T_delta of the strip's dx shifts; the dx shifts read
// the same staged rows one row earlier or later.  Thread t holds target boxes
// t mod 64 and t mod 64 + 64 and one half of the p output coefficients, so a
// step of the k loop is two shared loads of source coefficients, one
// broadcast load of an operator entry per output coefficient and, per (box,
// coefficient), one complex multiply-add as two packed FP32x2 FMAs:
//     (re, im) += (t.x, t.x) (a.x, a.y) + (-t.y, t.y) (a.y, a.x)
// with the operator entry staged as (t.x, t.x, -t.y, t.y), so one 16-byte
// load gives both packed multipliers.  All 32 lanes of every warp work, and
// every operator entry read serves two boxes.
//
//     LE_c[P] = sum over strips and dx of T_delta ME_c'[P + (dx, dy)]
//
// with the rescaled operators of Sec. 2.2 (level independent), accumulated
// in FP32 in a fixed order.
#include "kernels.cuh"

namespace petfmm {

#define PF_LAUNCHED(n) do { if (launches) *launches += (n); } while (0)

constexpr int MT_THREADS = 128;
constexpr int MT_BOXES = M2L_TILE_SEG;  // target boxes per unit
constexpr int MT_MAX_ROWS = 136;        // staged rows: R (SEG + 2) <= 130
constexpr int MT_MAX_P = 24;
// thread t takes boxes t mod 64 and t mod 64 + 64 of a unit
static_assert(MT_BOXES <= 128 && MT_THREADS == 128, "two boxes per thread pair of half-units");

// shared-memory row stride of the staged strip: odd, so that the 8-byte reads
// of 16 consecutive boxes by a half-warp hit distinct banks
__host__ __device__ __forceinline__ int mt_stride(int p) { return p | 1; }

template <int PH>
__global__ void __launch_bounds__(MT_THREADS) k_m2l_tile(
    const Task *__restrict__ tasks, int ntasks, const InstDesc *__restrict__ insts,
    const uint32_t *__restrict__ start, const float2 *__restrict__ me, float2 *__restrict__ le,
    const uint32_t *__restrict__ ucount, int dense_pct) {
    extern __shared__ float2 mt_smem[];
    __shared__ uint8_t rowocc[MT_MAX_ROWS];

    const int tid = threadIdx.x;
    const int ti = find_task(tasks, ntasks, blockIdx.x);
    const Task t = tasks[ti];
    const InstDesc &d = insts[t.inst];
    const int l = t.level, L = d.L, p = d.p;
    const int W = 1 << (l - 1);
    // the unit: parent rows Py0 .. Py0 + R - 1, cells Px0 .. Px0 + SEG - 1
    int c, Py0, R, Px0, SEG;
    tile_unit_decode(l, int64_t(blockIdx.x) - t.block0, &c, &Py0, &R, &Px0, &SEG);
    if (!tc_unit_dense(ucount[blockIdx.x], R * SEG, dense_pct)) return;  // sparse: per-box kernel
    const int cx = c & 1, cy = c >> 1;
    const uint32_t *st = start + d.soff;

    const int SP = mt_stride(p);
    const int Rs = SEG + 2;          // staged rows per parent row
    const int nrows = R * Rs;
    const int psq = p * p;
    float4 *tsm = reinterpret_cast<float4 *>(mt_smem);   // 3 operators, [k][m], packed
    float2 *strip = mt_smem + size_t(6) * psq;             // nrows x SP

    // this thread: boxes b0, b1 of the unit, coefficients m0 .. m0 + mc - 1;
    // box b is cell b % SEG of row b / SEG, staged at row (b / SEG) Rs + b % SEG + 1
    const int half = (p + 1) >> 1;
    const int b0 = tid & 63, b1 = b0 + 64;
    const int m0 = (tid >> 6) * half;
    const int mc = (tid >> 6) ? p - half : half;
    const int nb = R * SEG;
    const bool act0 = b0 < nb, act1 = b1 < nb;
    const int r0 = b0 / SEG, r1 = b1 / SEG;
    const int s0 = r0 * Rs + (b0 - r0 * SEG) + 1, s1 = r1 * Rs + (b1 - r1 * SEG) + 1;

    float2 acc0[PH], acc1[PH];
#pragma unroll
    for (int i = 0; i < PH; ++i) {
        acc0[i] = make_float2(0.f, 0.f);
        acc1[i] = make_float2(0.f, 0.f);
    }
    const int64_t quarter = int64_t(1) << (2 * (l - 1));
    const float2 *lev = me + d.eoff + lvl_off(l) * p;
    const float2 *tab = static_cast<const float2 *>(d.t_m2l);
    const uint32_t inv_p = ((1u << 20) + uint32_t(p) - 1) / uint32_t(p);

    for (int cs = 0; cs < 4; ++cs) {
        const int csx = cs & 1, csy = cs >> 1;
        for (int dyp = -1; dyp <= 1; ++dyp) {
            int ops[3];
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
            if (!mask3) continue;
            // occupancy of the staged source boxes: staged row q is cell
            // Px0 - 1 + q % Rs of parent row Py0 + q / Rs + dyp; empty and
            // out-of-domain boxes (never-written expansions) are staged as zeros
            bool anyr = false;
            for (int q = tid; q < nrows; q += MT_THREADS) {
                const int rr = q / Rs;
                const int Px = Px0 - 1 + (q - rr * Rs), Pys = Py0 + rr + dyp;
                bool o = false;
                if (Px >= 0 && Px < W && Pys >= 0 && Pys < W)
                    o = box_count(st, L, l,
                                  morton_key(uint32_t(2 * Px + csx), uint32_t(2 * Pys + csy))) != 0;
                rowocc[q] = o;
                anyr |= o;
            }
            if (!__syncthreads_or(anyr)) continue;
            // stage the strips (each row's cells are contiguous in the
            // class-split layout); element e = q p + k, q = e / p exactly for
            // e < 2^14 by the multiply-shift (p <= 24, nrows <= MT_MAX_ROWS)
            const int total = nrows * p;
            for (int e = tid; e < total; e += MT_THREADS) {
                const int q = int((uint32_t(e) * inv_p) >> 20), k = e - q * p;
                float2 v = make_float2(0.f, 0.f);
                if (rowocc[q]) {
                    const int rr = q / Rs;
                    const int Px = Px0 - 1 + (q - rr * Rs), Pys = Py0 + rr + dyp;
                    v = __ldg(lev + (int64_t(cs) * quarter + int64_t(Pys) * W + Px) * p + k);
                }
                strip[q * SP + k] = v;
            }
            // ... and the operators of the dx shifts
            for (int s3 = 0; s3 < 3; ++s3) {
                if (!(mask3 & (1u << s3))) continue;
                const float2 *T = tab + size_t(ops[s3]) * psq;
                for (int i = tid; i < psq; i += MT_THREADS) {
                    const float2 tk = __ldg(T + i);
                    tsm[s3 * psq + i] = make_float4(tk.x, tk.x, -tk.y, tk.y);
                }
            }
            __syncthreads();
            for (int s3 = 0; s3 < 3; ++s3) {
                if (!(mask3 & (1u << s3))) continue;
                const float4 *T = tsm + s3 * psq + m0;
                const float2 *a0p = strip + (s0 + s3 - 1) * SP;
                const float2 *a1p = strip + (s1 + s3 - 1) * SP;
                if (act1) {
                    for (int k = 0; k < p; ++k) {
                        const float2 a0 = a0p[k], a1 = a1p[k];
                        const float2 a0s = make_float2(a0.y, a0.x), a1s = make_float2(a1.y, a1.x);
#pragma unroll
                        for (int i = 0; i < PH; ++i) {
                            if (i < mc) {
                                const float4 tk = T[k * p + i];
                                const float2 tl = make_float2(tk.x, tk.y), th = make_float2(tk.z, tk.w);
                                acc0[i] = __ffma2_rn(tl, a0, acc0[i]);
                                acc1[i] = __ffma2_rn(tl, a1, acc1[i]);
                                acc0[i] = __ffma2_rn(th, a0s, acc0[i]);
                                acc1[i] = __ffma2_rn(th, a1s, acc1[i]);
                            }
                        }
                    }
                } else if (act0) {
                    for (int k = 0; k < p; ++k) {
                        const float2 a0 = a0p[k];
                        const float2 a0s = make_float2(a0.y, a0.x);
#pragma unroll
                        for (int i = 0; i < PH; ++i) {
                            if (i < mc) {
                                const float4 tk = T[k * p + i];
                                acc0[i] = __ffma2_rn(make_float2(tk.x, tk.y), a0, acc0[i]);
                                acc0[i] = __ffma2_rn(make_float2(tk.z, tk.w), a0s, acc0[i]);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // write the targets that hold particles (the others' LE is never read)
    for (int j = 0; j < 2; ++j) {
        if (!(j ? act1 : act0)) continue;
        const int b = j ? b1 : b0, rr = j ? r1 : r0;
        const int Px = Px0 + b - rr * SEG, Py = Py0 + rr;
        if (!box_count(st, L, l, morton_key(uint32_t(2 * Px + cx), uint32_t(2 * Py + cy))))
            continue;
        float2 *dst = le + d.eoff + (lvl_off(l) + int64_t(c) * quarter + int64_t(Py) * W + Px) * p;
#pragma unroll
        for (int i = 0; i < PH; ++i)
            if (i < mc) dst[m0 + i] = j ? acc1[i] : acc0[i];
    }
}

bool m2l_tile_supported(int p) { return p >= 1 && p <= MT_MAX_P; }

int64_t m2l_tile_units(int level) { return tile_units(level); }

size_t m2l_tile_smem_bytes(int p, int level) {
    int R, seg;
    tile_geom(level, &R, &seg);
    return (size_t(R) * (seg + 2) * mt_stride(p) + size_t(6) * p * p) * sizeof(float2);
}

cudaError_t launch_m2l_tile(const Task *tasks, int ntasks, int64_t nblocks, int pmax,
                            const InstDesc *insts, const uint32_t *start, const float2 *me,
                            float2 *le, const uint32_t *ucount, int dense_pct, cudaStream_t st,
                            uint64_t *launches) {
    if (nblocks <= 0) return cudaSuccess;
    const size_t smem = (size_t(MT_MAX_ROWS) * mt_stride(pmax) + size_t(6) * pmax * pmax) *
                        sizeof(float2);
    const int ph = (pmax + 1) / 2;
    void (*k)(const Task *, int, const InstDesc *, const uint32_t *, const float2 *, float2 *,
              const uint32_t *, int) = nullptr;
    if (ph <= 4) k = k_m2l_tile<4>;
    else if (ph <= 6) k = k_m2l_tile<6>;
    else if (ph <= 9) k = k_m2l_tile<9>;
    else if (ph <= 12) k = k_m2l_tile<12>;
    else return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
    }
    k<<<unsigned(nblocks), MT_THREADS, smem, st>>>(tasks, ntasks, insts, start, me, le, ucount,
                                                  dense_pct);
    PF_LAUNCHED(1);
    return cudaGetLastError();
}

}  // namespace petfmm
