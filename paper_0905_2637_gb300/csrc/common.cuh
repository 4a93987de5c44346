// common.cuh -- shared definitions of the GB300 vortex-blob FMM kernels.
//
// Data layout in HBM (one batch of instances; a single evaluation is a batch
// of one):
//   particles   keys/vals (uint32) ping-pong pairs for the radix sort, then
//               the sorted particles: FP64 path SoA double x, y, gamma (global
//               coordinates); mixed path float4 (xi, eta, gamma, 0) with
//               (xi, eta) = (x - leaf centre) / leaf width, i.e. leaf-relative
//               coordinates in leaf units (exact for FP32 inputs on a dyadic
//               domain).
//   start       per instance 4^L + 1 uint32 leaf starts (global sorted rank).
//   ME, LE      per instance, per level l, 4^l boxes x p complex coefficients
//               (double2 or float2).  Boxes of a level are stored "by child
//               class": box (ix, iy) at level l >= 1 has class
//               c = (ix & 1) | (iy & 1) << 1 and parent cell P = (ix >> 1,
//               iy >> 1), and index c * 4^(l-1) + Py * 2^(l-1) + Px.  The four
//               children of one parent sit at the same P in four planes, and a
//               fixed (class, parent offset) pair of the interaction list is a
//               constant shift of the parent grid.
//   Expansions are rescaled so that the translation operators do not depend
//   on the level and FP32 cannot overflow: a~_k = a_k / r^k (ME) and
//   c^_m = r^(m+1) b_m (LE), r = box width.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace petfmm {

constexpr int MAX_P = 40;
constexpr int MAX_L = 15;
constexpr int POLY_MAX = 14;

// Device status codes (same values as the PETFMM_E* codes of the ABI).
constexpr int ST_EDOMAIN = -3;
constexpr int ST_ETIMEOUT = -5;

// One FMM problem of a batch.
// The kernels an evaluation can sum (the Evaluator of Sec. 6.1 is
// parameterised by its kernel): the Gaussian-regularised Biot-Savart
// velocity of Eq. 8/9, and the 2D logarithmic potential
// phi_i = sum_{j != i} q_j log|x_i - x_j|.
enum { KERNEL_VORTEX = 0, KERNEL_LAPLACE = 1 };

struct InstDesc {
    double x0, y0, width;   // domain square
    double scale;           // 2^L / width (computed once on the host)
    double wleaf;           // width / 2^L
    double sigma;
    int L, p;
    int64_t n;              // particles
    int64_t poff;           // first particle of this instance in batch arrays
    int64_t soff;           // first entry of its leaf-start array
    int64_t loff;           // first leaf of this instance in batch leaf arrays
    int64_t eoff;           // first box of this instance in ME/LE (box units)
    uint32_t key_hi;        // composite sort key = key_hi | Morton key
    int kernel;             // KERNEL_VORTEX or KERNEL_LAPLACE
    const void *x, *y, *g;  // caller's arrays (storage type of the context)
    void *u, *v;
    const void *t_m2m, *t_l2l, *t_m2l;  // operator tables for this p (path's real type)
    const void *t_m2l_tc;               // tensor-core M2L operator images (mixed path)
    const void *t_m2l_tcb;              // ... side by side for the block units
    int64_t tc_unit0[MAX_L + 1];        // per level: first unit of this (instance, level)
                                        // in the tensor-core M2L launch, or -1
    int tc_segmax;                      // widest tensor-core unit (parent cells)
    uint32_t tc_levels;                 // bit l: level l's dense units run on the tensor
                                        // cores (else, if tc_unit0[l] >= 0, on the
                                        // tiled SIMT kernel)
    uint32_t tcb_levels;                // bit l: ... on the tensor cores in 8 x 16 blocks
                                        // (all four classes per block)
    // mixed-precision P2P constants (leaf units)
    float kappa;            // w^2 / (2 sigma^2): q = kappa * rho^2
    float cnear;            // w / (4 pi sigma^2)
    float cfar;             // 1 / (2 pi w)
    float qsplit_rho2;      // general path: polynomial below this rho^2
    int deg;                // polynomial degree (in rho^2) of g(q) = (1 - e^-q) / q
    int general;            // 1: some near pairs exceed the polynomial range
    float poly[POLY_MAX + 1];
    // FP64 constants
    double inv2s2;          // 1 / (2 sigma^2)
    double cnear64;         // 1 / (2 pi)
    double cfar64;          // 1 / (2 pi w)
    double logw0;           // Laplace kernel: log(domain width); level l boxes are
                            // log(width) - l log 2 wide in log scale
    // float-float copies of the domain: x0 = x0h + x0l, y0 = y0h + y0l,
    // scale = sh + sl (binning shortcut and leaf-relative coordinates in FP32)
    float x0h, x0l, y0h, y0l, sh, sl;
};

// Sets the domain square and the quantities derived from it.
inline void inst_set_domain(InstDesc &d, double x0, double y0, double width, int L) {
    d.x0 = x0;
    d.y0 = y0;
    d.width = width;
    d.scale = std::ldexp(1.0, L) / width;
    d.wleaf = width / std::ldexp(1.0, L);
    d.x0h = float(x0);
    d.x0l = float(x0 - double(d.x0h));
    d.y0h = float(y0);
    d.y0l = float(y0 - double(d.y0h));
    d.sh = float(d.scale);
    d.sl = float(d.scale - double(d.sh));
    d.logw0 = std::log(width);
}

// A range of work units of one kind, for one instance (and level).
struct Task {
    int inst;
    int level;
    int64_t count;    // work units
    int64_t block0;   // first block of the launch assigned to this task
};

__host__ __device__ __forceinline__ int64_t lvl_off(int l) {
    return ((int64_t(1) << (2 * l)) - 1) / 3;
}

// index of box (ix, iy) within its level, class-split layout
__host__ __device__ __forceinline__ int64_t box_index(int l, uint32_t ix, uint32_t iy) {
    if (l == 0) return 0;
    int64_t q = int64_t(1) << (2 * (l - 1));
    int64_t c = (ix & 1u) | ((iy & 1u) << 1);
    return c * q + int64_t(iy >> 1) * (int64_t(1) << (l - 1)) + int64_t(ix >> 1);
}

__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__host__ __device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// z-order key: x bit b -> key bit 2b, y bit b -> key bit 2b + 1
__host__ __device__ __forceinline__ uint32_t morton_key(uint32_t ix, uint32_t iy) {
    return spread_bits(ix) | (spread_bits(iy) << 1);
}

// Particles in box m (Morton index) of level l: the leaves of a box form one
// contiguous Morton range, so this is two reads of the leaf starts st[] of
// an instance with depth L.  Expansions of empty boxes are never computed
// or read (their coefficients would be exactly zero).
__device__ __forceinline__ uint32_t box_count(const uint32_t *st, int L, int l, uint32_t m) {
    const int sh = 2 * (L - l);
    return st[(uint64_t(m) + 1) << sh] - st[uint64_t(m) << sh];
}

// The task of block (or unit) b: the last task with block0 <= b (tasks are
// in ascending block0 order, the first at 0).  A 32-way search by the warp:
// lane i tests candidate lo + i * step, and since block0 ascends the lanes
// that pass are a prefix, so one ballot narrows the range 32-fold (at most
// two rounds of loads for 1024 tasks, against ten dependent loads of a
// binary search).  Every lane of the warp must call it with the same b.
__device__ __forceinline__ int find_task(const Task *tasks, int ntasks, int64_t b) {
    int lo = 0, n = ntasks;
    const int lane = threadIdx.x & 31;
    while (n > 1) {
        const int step = (n + 31) >> 5;
        const int idx = lo + lane * step;
        const bool le = idx < lo + n && tasks[idx].block0 <= b;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const int k = 31 - __clz(int(m | 1u));
        const int end = lo + n;
        lo += k * step;
        n = min(step, end - lo);
    }
    return lo;
}

__device__ __forceinline__ void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

// Bounds-checked build (compiled with -DPETFMM_CHECKS; the library build
// makes it as libpetfmm_checked.so).  PF_IN(i, n) is true when 0 <= i < n;
// otherwise it records the source line of the check in this file's device
// word pf_check_line (the first failure wins) and is false, and the caller
// skips the access (reads a zero, writes nothing).  It never traps, so a bad
// index leaves the context usable and is reported by petfmm_debug_checks().
// In the regular build PF_IN is the constant true and costs nothing.
#ifdef PETFMM_CHECKS
static __device__ unsigned int pf_check_line = 0;
__device__ __forceinline__ bool pf_in_range(int64_t i, int64_t n, unsigned line) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&pf_check_line, 0u, line);
    return false;
}
#define PF_IN(i, n) ::petfmm::pf_in_range(int64_t(i), int64_t(n), __LINE__)
// host: read and clear this file's word (0: no failure)
#define PF_DEFINE_CHECK_READER(name)                                            \
    unsigned pf_checks_##name() {                                               \
        unsigned v = 0, z = 0;                                                  \
        if (cudaMemcpyFromSymbol(&v, pf_check_line, sizeof(v)) != cudaSuccess) \
            cudaGetLastError();                                                 \
        if (cudaMemcpyToSymbol(pf_check_line, &z, sizeof(z)) != cudaSuccess)   \
            cudaGetLastError();                                                 \
        return v;                                                               \
    }
#else
#define PF_IN(i, n) true
#define PF_DEFINE_CHECK_READER(name) \
    unsigned pf_checks_##name() { return 0; }
#endif

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

template <typename T2> __host__ __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T2> __host__ __device__ __forceinline__ T2 cfma(T2 a, T2 b, T2 c) {
    // a * b + c
    T2 r;
    r.x = a.x * b.x - a.y * b.y + c.x;
    r.y = a.x * b.y + a.y * b.x + c.y;
    return r;
}

// Position of the M2L offset (dx, dy) among the 40 vectors of
// [-3, 3]^2 \ [-1, 1]^2, taken row by row (increasing dy, then dx): the index
// of its operator T_delta.
__host__ __device__ __forceinline__ int m2l_op_index(int dx, int dy) {
    const int base = dy <= -1 ? 7 * (dy + 3) : (dy <= 2 ? 14 + 4 * (dy + 1) : 33);
    const int pos = (dy >= -1 && dy <= 1) ? (dx < 0 ? dx + 3 : dx) : dx + 3;
    return base + pos;
}

// Tensor-core M2L units: at level l (parent grid W = 2^(l-1) per side) a unit
// is a segment of SEG = min(W, segmax) parent cells of one parent row, for one
// target child class c; units are numbered ((c W) + Py) (W / SEG) + segment.
// segmax is 128, 256 or 512 (InstDesc::tc_segmax).
constexpr int TC_MAX_SEG = 512;

__host__ __device__ __forceinline__ int tc_seg(int l, int segmax) {
    const int W = 1 << (l - 1);
    return W < segmax ? W : segmax;
}

__host__ __device__ __forceinline__ void tc_unit_decode(int l, int segmax, int64_t unit, int *c,
                                                        int *Py, int *Px0, int *seg) {
    const int W = 1 << (l - 1);
    const int s = tc_seg(l, segmax), nseg = W / s;
    *seg = s;
    *c = int(unit / (int64_t(W) * nseg));
    const int64_t rem = unit - int64_t(*c) * W * nseg;
    *Py = int(rem / nseg);
    *Px0 = int(rem - int64_t(*Py) * nseg) * s;
}

__host__ __device__ __forceinline__ int64_t tc_unit_of(int l, int segmax, int c, int Py, int Px) {
    const int W = 1 << (l - 1);
    const int s = tc_seg(l, segmax), nseg = W / s;
    return (int64_t(c) * W + Py) * nseg + Px / s;
}

// Block units of the tensor-core M2L: 8 x 16 parent cells (x, y), all four
// target classes (512 targets); units are numbered (Py / 16) (W / 8) + Px / 8.
constexpr int TCB_BX = 8, TCB_BY = 16;

__host__ __device__ __forceinline__ void tcb_unit_decode(int l, int64_t unit, int *Py0, int *Px0) {
    const int W = 1 << (l - 1);
    const int nbx = W / TCB_BX;
    *Py0 = int(unit / nbx) * TCB_BY;
    *Px0 = int(unit - (unit / nbx) * nbx) * TCB_BX;
}

// Units of the tiled SIMT M2L: a segment of M2L_TILE_SEG parent cells of one
// parent row, or, where rows are shorter, R whole rows of together at most
// M2L_TILE_ROWS_BOXES target boxes (half a full unit: a shallow level has few
// boxes, and smaller units keep more CTAs in flight).
constexpr int M2L_TILE_SEG = 128;
constexpr int M2L_TILE_ROWS_BOXES = 64;

__host__ __device__ __forceinline__ void tile_geom(int l, int *R, int *seg) {
    const int W = 1 << (l - 1);
    *seg = W < M2L_TILE_SEG ? W : M2L_TILE_SEG;
    const int r = W < M2L_TILE_SEG ? M2L_TILE_ROWS_BOXES / *seg : 1;
    *R = r < 1 ? 1 : r < W ? r : W;
}

__host__ __device__ __forceinline__ int64_t tile_units(int l) {
    const int W = 1 << (l - 1);
    int R, s;
    tile_geom(l, &R, &s);
    return int64_t(4) * (W / R) * (W / s);
}

__host__ __device__ __forceinline__ void tile_unit_decode(int l, int64_t unit, int *c, int *Py0,
                                                          int *R, int *Px0, int *seg) {
    const int W = 1 << (l - 1);
    tile_geom(l, R, seg);
    const int nseg = W / *seg, nrow = W / *R;
    *c = int(unit / (int64_t(nrow) * nseg));
    const int64_t rem = unit - int64_t(*c) * nrow * nseg;
    *Py0 = int(rem / nseg) * *R;
    *Px0 = int(rem - (rem / nseg) * nseg) * *seg;
}

// Unit of box (c, Py, Px) of level l (tensor-core or tiled units) and the
// number of its targets.
__host__ __device__ __forceinline__ int64_t unit_of(const InstDesc &d, int l, int c, int Py,
                                                    int Px, int *nbox) {
    if ((d.tc_levels >> l) & 1u) {
        *nbox = tc_seg(l, d.tc_segmax);
        return tc_unit_of(l, d.tc_segmax, c, Py, Px);
    }
    const int W = 1 << (l - 1);
    if ((d.tcb_levels >> l) & 1u) {
        (void)c;
        *nbox = 4 * TCB_BX * TCB_BY;
        return int64_t(Py / TCB_BY) * (W / TCB_BX) + Px / TCB_BX;
    }
    int R, s;
    tile_geom(l, &R, &s);
    *nbox = R * s;
    return (int64_t(c) * (W / R) + Py / R) * (W / s) + Px / s;
}

// A unit goes to the tensor cores (or the tiled SIMT kernel) when at least
// dense_pct percent of its targets hold particles; the per-box SIMT kernel
// takes the boxes of the others.
__host__ __device__ __forceinline__ bool tc_unit_dense(uint32_t count, int seg, int dense_pct) {
    return count > 0 && 100u * count >= uint32_t(dense_pct) * uint32_t(seg);
}

// Interaction-list table: for child class c, the 27 (dx, dy) offsets of the
// sources relative to the target box and the index (0..39) of the M2L
// operator for that offset.  Filled by the host (expansions.cu).
struct IlEntry {
    int8_t dx, dy;
    int8_t op;
    int8_t pad;
};

}  // namespace petfmm
