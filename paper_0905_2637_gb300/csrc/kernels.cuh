// kernels.cuh -- host-side launchers of the FMM kernels (internal).
#pragma once
#include <vector>

#include "common.cuh"

namespace petfmm {

// Every launcher returns cudaGetLastError() after the launch and adds the
// number of kernels it launched to *launches.

// Bounds-checked build: the first failing PF_IN check's source line in each
// file (0: none), read and cleared (always 0 in the regular build).
unsigned pf_checks_tree();
unsigned pf_checks_expansions();
unsigned pf_checks_p2p();

// ---- tree.cu ---------------------------------------------------------------
// Sec. 2.1 binning + z-order key of every particle (composite key for batches);
// if recu != nullptr also its mixed-path record (see launch_gather_mixed) in
// input order.
cudaError_t launch_morton(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                          int dtype_f32, uint32_t *keys, float4 *recu, int *status,
                          cudaStream_t st, uint64_t *launches);

// Scratch (uint32 words) needed by exclusive_scan for n elements.
int64_t scan_scratch_words(int64_t n);
// out[i] = sum_{j < i} in[j]; in may equal out.  If total != nullptr the sum
// of all elements is written there (device).
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch,
                           uint32_t *total, cudaStream_t st, uint64_t *launches);

// Stable LSD radix sort of (key, value) over the low nbits bits (8-bit
// digits, at most 4 passes, n < 2^32); the initial values are the element
// indices.  Result ends up in (k0, v0) or (k1, v1): *result_in_first tells
// which.  scratch: radix_scratch_words(n) words (per-tile digit counts and
// their scan).  n_live (device, optional): sort only the
// first min(n, *n_live) elements (the grid stays sized for n; tiles past the
// live ones return at once).
int64_t radix_blocks(int64_t n);
int64_t radix_scratch_words(int64_t n);
cudaError_t radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n,
                       int nbits, uint32_t *scratch, bool *result_in_first, cudaStream_t st,
                       uint64_t *launches, const uint32_t *n_live = nullptr);

// start[soff + b] = first sorted rank of leaf b (b = 0..4^L).
cudaError_t launch_leaf_start(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                              const uint32_t *skeys, uint32_t *start, cudaStream_t st,
                              uint64_t *launches);

// Sorted particle arrays.
cudaError_t launch_gather_f64(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                              int dtype_f32, const uint32_t *perm, double *xs, double *ys,
                              double *gs, cudaStream_t st, uint64_t *launches);
// rec[r] = recu[perm[r]]: (xi, eta, gamma, batch index) in sorted order, with
// (xi, eta) the offset from the leaf centre in leaf widths.
cudaError_t launch_gather_mixed(const float4 *recu, const uint32_t *perm, float4 *rec, int64_t n,
                                cudaStream_t st, uint64_t *launches);

// ---- expansions.cu ---------------------------------------------------------
// Operator tables for p (FP64 build, also rounded to FP32), device-resident.
struct OpTables {
    int p = 0;
    double2 *m2m64 = nullptr, *l2l64 = nullptr, *m2l64 = nullptr;
    float2 *m2m32 = nullptr, *l2l32 = nullptr, *m2l32 = nullptr;
    float *m2l_tc = nullptr;  // hi/lo B images for the tensor-core M2L (p <= 24)
    float *m2l_tcb = nullptr; // ... the four target classes side by side (block units)
};
cudaError_t build_op_tables(int p, int kernel, OpTables *out);
// The FP64 table behind them: which = 0 M2M [c][l][k], 1 L2L [c][n][m],
// 2 M2L [op][k][m], complex as (re, im) pairs.
void host_op_table(int p, int kernel, int which, std::vector<double> &out);
void free_op_tables(OpTables *t);
void host_m2l_table(int p, double *out_re_im /* 40 * p * p * 2, [op][k][m] */);
// Interaction list exactly as the kernels enumerate it; returns the count.
int host_interaction_list(int level, int ix, int iy, int32_t *out);
// Number of (target, source) M2L translations of levels 2..L.
int64_t m2l_pair_count(int L);

// occ[0 .. ctrl[CTRL_NOCC]) = (instance, leaf) of every occupied leaf, in no
// particular order (one thread per leaf of the tasks).
cudaError_t launch_occ_list(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                            const uint32_t *start, uint2 *occ, uint32_t *ctrl, cudaStream_t st,
                            uint64_t *launches);
// P2M of the listed leaves by a persistent grid (max_occ bounds the list).
template <typename R>
cudaError_t launch_p2m(const uint2 *occ, const uint32_t *ctrl, int64_t max_occ,
                       const InstDesc *insts, int pmax, const uint32_t *start, const double *xs,
                       const double *ys, const double *gs, const float4 *rec,
                       typename Cplx<R>::T *me, cudaStream_t st, uint64_t *launches);
// M2M, M2L and L2L skip boxes with no particles in their subtree (and M2L
// skips empty sources): their coefficients would be exactly zero and are
// never read.  start = the batch's leaf-start array.
template <typename R>
cudaError_t launch_m2m(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, typename Cplx<R>::T *me, cudaStream_t st,
                       uint64_t *launches);
// For levels that also have tensor-core units (InstDesc::tc_unit0 >= 0) the
// SIMT M2L skips the boxes of dense units (ucount, dense_pct).
template <typename R>
cudaError_t launch_m2l(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, const typename Cplx<R>::T *me,
                       typename Cplx<R>::T *le, const uint32_t *ucount, int dense_pct,
                       cudaStream_t st, uint64_t *launches);
template <typename R>
cudaError_t launch_l2l(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                       const uint32_t *start, typename Cplx<R>::T *le, cudaStream_t st,
                       uint64_t *launches);

// ---- m2l_tc.cu -------------------------------------------------------------
// Tensor-core M2L (mixed path) for levels with at least 128 parent cells per
// row and p <= 24: one CTA per (target class, parent row, segment) unit.
bool m2l_tc_supported(int p, int level, int segmax);
// block units (8 x 16 parent cells, all four target classes), levels >= 5
bool m2l_tcb_supported(int p, int level);
int64_t m2l_tcb_units(int level);
size_t m2l_tcb_smem_bytes(int p);
void host_m2l_tcb_images(int p, int kernel, std::vector<float> &out);
// pmax: the largest order among the launch's units (sizes shared memory)
cudaError_t launch_m2l_tcb(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                           const uint32_t *start, const float2 *me, float2 *le,
                           const uint32_t *ucount, int dense_pct, int pmax, long long spin_limit,
                           int pipe, int *status, cudaStream_t st, uint64_t *launches);
int64_t m2l_tc_units(int level, int segmax);
size_t m2l_tc_smem_bytes(int p, int seg);
int m2l_tc_seg(int level, int segmax);
void host_m2l_tc_images(int p, int kernel, std::vector<float> &out);
void host_lap_m2l_table(int p, double *out_re_im /* 40 * p * p * 2, [op][k][m] */);
// Laplace kernel: the level-dependent constant of M2L, added after every M2L
// kernel (tasks: instance, level; units: 4^l target boxes).
template <typename R>
cudaError_t launch_m2l_logterm(const Task *tasks, int ntasks, int64_t nblocks,
                               const InstDesc *insts, const uint32_t *start,
                               const typename Cplx<R>::T *me, typename Cplx<R>::T *le,
                               cudaStream_t st, uint64_t *launches);
// ucount[u] = targets holding particles in unit u of the launch (tensor-core
// or tiled SIMT units; block index = unit).
cudaError_t launch_tc_unit_count(const Task *tasks, int ntasks, int64_t nunits,
                                 const InstDesc *insts, const uint32_t *start, uint32_t *ucount,
                                 cudaStream_t st, uint64_t *launches);
// Dense units (tc_unit_dense) on the tensor cores; the SIMT launch covers the
// boxes of the other units of the same levels.
cudaError_t launch_m2l_tc(const Task *tasks, int ntasks, int64_t nblocks, const InstDesc *insts,
                          const uint32_t *start, const float2 *me, float2 *le,
                          const uint32_t *ucount, int dense_pct, size_t smem_bytes,
                          long long spin_limit, int *status, cudaStream_t st, uint64_t *launches);

// ---- m2l_tile.cu -----------------------------------------------------------
// Tiled SIMT M2L (mixed path, p <= 24) for the dense units of the levels the
// tensor cores do not take; units as above with M2L_TILE_SEG parent cells.
bool m2l_tile_supported(int p);
int64_t m2l_tile_units(int level);
size_t m2l_tile_smem_bytes(int p, int level);
cudaError_t launch_m2l_tile(const Task *tasks, int ntasks, int64_t nblocks, int pmax,
                            const InstDesc *insts, const uint32_t *start, const float2 *me,
                            float2 *le, const uint32_t *ucount, int dense_pct, cudaStream_t st,
                            uint64_t *launches);

// units of work per block of each expansion kernel (the host plans with them)
constexpr int P2M_WARPS = 4;      // warps per block
constexpr int M2L_WARPS = 4;      // warps per block
// Each warp of the SIMT M2L owns a run of consecutive boxes and skips the
// empty ones after one ballot: at the clustered workload 87% of the leaves
// are empty, and a block per few boxes made the kernel bound by block
// scheduling.
constexpr int BOX_RUN = 8;
constexpr int M2L_BOXES = M2L_WARPS * BOX_RUN;   // target boxes per block
constexpr int EXP_THREADS = 256;  // (box, coefficient) pairs per block for M2M / L2L

// ---- p2p.cu ----------------------------------------------------------------
// Work list: items (inst, leaf, first target rank, target count) for every
// occupied leaf, tpi targets per item.  ctrl[CTRL_NITEMS] receives the count.
enum { CTRL_STATUS = 0, CTRL_NITEMS = 1, CTRL_QUEUE = 2, CTRL_PAIRS_LO = 4, CTRL_NOCC = 6,
       CTRL_NPAIRS = 7, CTRL_QUEUE2 = 8, CTRL_NXTRA = 9, CTRL_SYM_LO = 10, CTRL_WORDS = 16 };
// Buffers for dispatching the items heaviest first (order != nullptr): the
// items are emitted to items_unsorted, sorted by work class (one stable radix
// pass over cap entries) and permuted into the item array.
struct P2POrder {
    int64_t cap;
    uint4 *items_unsorted;
    uint32_t *kA, *kB, *vA, *vB, *hist;  // hist: radix_scratch_words(cap) words
};
// pairs_mode: only the leaves with directed work (leaves under 32 blobs, or
// with a neighbour the pair kernel does not cover) get items.
cudaError_t launch_p2p_worklist(const Task *tasks, int ntasks, int64_t nblocks,
                                const InstDesc *insts, const uint32_t *start, int64_t nleaves,
                                int tpi, int pairs_mode, uint32_t *cnt, uint32_t *off,
                                uint32_t *scan_scratch, uint4 *items, uint32_t *ctrl,
                                const P2POrder *order, cudaStream_t st, uint64_t *launches);
cudaError_t launch_p2p_f64(int grid, const uint4 *items, uint32_t *ctrl, const InstDesc *insts,
                           const uint32_t *start, const double *xs, const double *ys,
                           const double *gs, const uint32_t *perm, const double2 *le,
                           int dtype_f32, unsigned long long *busy, cudaStream_t st,
                           uint64_t *launches);
// Mixed near field, every leaf against all 9 leaves (pairs: not the
// neighbours the pair kernel covers): own[r] = the near sum of sorted blob r
// (launch_p2p_final then adds the far field).
cudaError_t launch_p2p_mixed(int grid, int deg, int general, const uint4 *items, uint32_t *ctrl,
                             const InstDesc *insts, const uint32_t *start, const float4 *rec,
                             float2 *own, int pairs, int laplace, unsigned long long *busy,
                             cudaStream_t st, uint64_t *launches);
// Pairwise near field between neighbouring leaves (mixed path).  Buffers:
// own[N]: each blob's directly summed part (sorted order; the only one used
// by the directed mode, part == nullptr there); part: 9 slots of
// nslot float2 (slot d: A's blobs from forward neighbour d, slot 4 + d: B's
// blobs from A, slot 8: each blob from the other blobs of its leaf); xcnt, xoff: per leaf, the scratch entries of its split pairs
// and their exclusive scan; xtab[4 nleaves]: per (leaf, direction) of a split
// pair its scratch base (all ones: not split); lflags[nleaves]: per leaf,
// which of these hold its blobs' sums; xs[xcap]: the scratch runs of pieces
// 1 .. of split pairs.
struct PairBufs {
    float2 *own, *part;
    int64_t nslot;
    uint32_t *xcnt, *xoff, *xtab, *lflags;
    float2 *xs;
    int64_t xcap;
};
// ... the item list (inst, leaf A, direction | swap << 3 | piece << 4,
// scratch base; direction 4: the leaf's own pairs),
// ctrl[CTRL_NPAIRS] its count, ctrl[CTRL_NXTRA] the scratch entries wanted ...
cudaError_t launch_pair_worklist(const Task *tasks, int ntasks, int64_t nblocks,
                                 const InstDesc *insts, const uint32_t *start, int64_t nleaves,
                                 uint32_t *cnt, uint32_t *off, uint32_t *scan_scratch,
                                 uint4 *items, uint32_t *ctrl, const P2POrder *order,
                                 const PairBufs &pb, cudaStream_t st, uint64_t *launches);
// ... the pair items, one persistent launch (the directed items follow in
// launch_p2p_mixed with pairs = 1) ...
int p2p_pairs_grid(int deg, int general);
cudaError_t launch_p2p_pairs(int grid, int deg, int general, const uint4 *pitems, uint32_t *ctrl,
                             const InstDesc *insts, const uint32_t *start, const float4 *rec,
                             const PairBufs &pb, unsigned long long *busy, cudaStream_t st,
                             uint64_t *launches);
// Either mode's final pass: far field (L2P) + own + pair slots per blob,
// written at the caller's index (tasks over blobs).
cudaError_t launch_p2p_final(const Task *tasks, int ntasks, int64_t nblocks,
                             const InstDesc *insts, const uint32_t *start, const uint32_t *skeys,
                             const float4 *rec, const float2 *le, const PairBufs &pb,
                             int dtype_f32, const uint32_t *perm, float *stage, int64_t nstage,
                             const Task *utasks, int nutasks, int64_t unblocks,
                             const uint32_t *ctrl, int64_t ntotal, cudaStream_t st,
                             uint64_t *launches);
// (stage != nullptr, FP32 outputs: the pass writes u, v in sorted order to
// stage[0 .. nstage) and stage[nstage ..), then one launch per component
// scatters them to the caller's arrays through perm; utasks: the blobs of
// every instance, 1024 per block.)
int p2p_grid(int precision_mixed, int deg, int general, int laplace);
int device_sm_count();
constexpr int P2P_TPI_F64 = 32;
constexpr int P2P_TPI_MIXED = 64;

}  // namespace petfmm
