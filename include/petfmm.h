/*
 * petfmm.h -- C ABI of the GB300 (sm_103a) 2D vortex-blob fast multipole
 * library.
 *
 * One call evaluates the velocity that N Gaussian vortex blobs induce on one
 * another, the N-body sum of Eq. 1 with targets = sources, in the vortex-method
 * form of Sec. 3:
 *
 *     u(x_i) = sum_{j != i} gamma_j K_sigma(x_i - x_j)                  (Eq. 9)
 *     K_sigma(x) = (-x2, x1) (1 - exp(-|x|^2 / 2 sigma^2)) / (2 pi |x|^2) (Eq. 8)
 *
 * accelerated by the fast multipole method of Sec. 2 (Fig. 2): binning into a
 * uniform quadtree with z-order numbering (Sec. 2.1, Sec. 5.1), P2M and M2M
 * (upward sweep), M2L over each box's interaction list and L2L (downward
 * sweep), then L2P plus the direct near-field P2P over the box and its 8
 * neighbours (evaluation step).  The far field uses the expansions of the
 * singular kernel 1/|x|^2 (kernel substitution, end of Sec. 3); the near field
 * uses K_sigma exactly.  Expansions have p terms (k = 0..p-1).
 *
 * Conventions for every entry point:
 *   - Status: 0 (PETFMM_OK) or a negative PETFMM_E* code; nothing else crosses
 *     the ABI (no exceptions, no exit).  petfmm_strerror() names a code.
 *   - Device pointers are CUDA global-memory pointers on the context's device;
 *     host pointers are ordinary (preferably page-locked) host memory.
 *   - x, y, gamma, u, v are dense 1-D arrays of n elements of the context's
 *     storage type (PETFMM_F64: double, PETFMM_F32: float), owned by the caller.
 *   - Kernels are enqueued on the context's CUDA stream; device-side errors
 *     (a particle outside the domain, a bounded wait that ran out) are
 *     recorded in a status word and returned by the next petfmm_sync().
 *   - A context is bound to one stream and one device and is not thread-safe;
 *     the server (petfmm_serve_*) is thread-safe.
 */
#ifndef PETFMM_H
#define PETFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    PETFMM_OK = 0,
    PETFMM_EINVAL = -1,    /* an argument is out of range (checked before any launch) */
    PETFMM_ENOMEM = -2,    /* device or host allocation failed, or over a memory budget */
    PETFMM_EDOMAIN = -3,   /* a particle lies outside the closed domain square, or is NaN */
    PETFMM_ECUDA = -4,     /* a CUDA runtime call failed */
    PETFMM_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    PETFMM_EBUSY = -6,     /* the server has no free slot and the queue is full */
    PETFMM_ENOTREADY = -7  /* a served request has not finished yet */
};

/* Precision mode of the arithmetic. */
enum {
    PETFMM_FP64 = 0,   /* every stage in FP64 */
    PETFMM_MIXED = 1   /* binning/sort exact, P2P and expansions in FP32 with
                          rescaled expansions, M2L on the tensor cores (3xTF32) */
};

/* Storage type of x, y, gamma, u, v. */
enum { PETFMM_F64 = 0, PETFMM_F32 = 1 };

/* Closed square domain [x0, x0 + width] x [y0, y0 + width] (Sec. 2.1). */
typedef struct {
    double x0, y0, width;
} petfmm_domain;

typedef struct petfmm_ctx petfmm_ctx;

/*
 * petfmm_create -- make an evaluation context (Sec. 6.1: the Evaluator over a
 * Quadtree with one Kernel; here the regularised Biot-Savart kernel).
 *   dom        domain square (width > 0, finite).
 *   levels     depth L of the uniform quadtree, 1..15 (leaves = 4^L); the
 *              interaction lists are empty at levels 0 and 1 (Sec. 2.2).
 *   order      p, the number of expansion terms, 1..40 (Sec. 2, Table 1).
 *   sigma      blob core size of Eq. 5 / Eq. 8, > 0.
 *   precision  PETFMM_FP64 or PETFMM_MIXED.
 *   dtype      PETFMM_F64 or PETFMM_F32 (storage type of the caller's arrays).
 *   cuda_stream  a cudaStream_t of the current device, or NULL for the
 *              legacy default stream.
 *   out        receives the context; the library owns it and every buffer
 *              in it until petfmm_destroy().
 * Returns PETFMM_EINVAL for out-of-range arguments, PETFMM_ENOMEM, or
 * PETFMM_ECUDA.
 */
int petfmm_create(const petfmm_domain *dom, int levels, int order, double sigma,
                  int precision, int dtype, void *cuda_stream, petfmm_ctx **out);

/*
 * petfmm_evaluate -- one full FMM velocity evaluation (Sec. 2.2): Morton
 * binning and sort, P2M, M2M, M2L, L2L, L2P + P2P, written back to u, v in
 * the caller's particle order.
 *   n          number of particles, 0 <= n < 2^31.
 *   x, y, gamma  device arrays (positions and circulations gamma_j of Eq. 4).
 *   u, v       device arrays receiving the velocity of Eq. 9 (including the
 *              1/2pi factor); may not alias the inputs.
 * Asynchronous on the context's stream: the arrays must stay valid until
 * petfmm_sync() returns.  Library buffers grow on demand (PETFMM_ENOMEM if
 * that fails).  A particle outside the domain makes the next petfmm_sync()
 * return PETFMM_EDOMAIN; u, v are then unspecified.
 */
int petfmm_evaluate(petfmm_ctx *ctx, int64_t n, const void *x, const void *y,
                    const void *gamma, void *u, void *v);

/*
 * petfmm_evaluate_host -- the same evaluation with HOST arrays: copies x, y,
 * gamma to the device, evaluates, copies u, v back, and waits.  Pinned host
 * memory gives the fastest copies.  Returns the evaluation's status.
 */
int petfmm_evaluate_host(petfmm_ctx *ctx, int64_t n, const void *x, const void *y,
                         const void *gamma, void *u, void *v);

/* petfmm_sync -- wait for the context's stream; returns the first deferred
 * device status since the previous sync (and clears it). */
int petfmm_sync(petfmm_ctx *ctx);

/* petfmm_destroy -- wait for outstanding work and free the context. */
int petfmm_destroy(petfmm_ctx *ctx);

/*
 * Batched evaluation: many independent FMM problems of uneven size in one
 * pass of batched kernels (every stage launches once for all instances, or
 * once per tree level).
 *   levels <= 0 asks the library to choose L: a level rule installed in the
 *   context (petfmm_set_level_rules, petfmm_tune_batch) if one matches, else
 *   the work model of Sec. 5.2 (Eq. 14), always under the kernel-substitution
 *   guard exp(-r_L^2 / 2 sigma^2) <= 1e-8 for the leaf width r_L.
 * The context supplies precision, storage type, stream and workspace; its own
 * domain, L, p, sigma are not used.  Arrays are device pointers; the call is
 * asynchronous like petfmm_evaluate().  Each instance's result is bit-for-bit
 * the one it gets alone, except that with PETFMM_OPT_TC_BLOCKS = 0 (default) a
 * batch with enough trees runs M2L levels 5 to 7 on the tensor cores where a
 * tree alone would not (the two differ by FP32 rounding; with the option at 1
 * or 2 the equality is exact).
 */
typedef struct {
    petfmm_domain domain;
    int levels;          /* L, or <= 0 for automatic */
    int order;           /* p, 1..40 */
    double sigma;        /* > 0 */
    int64_t n;           /* particles, >= 0 */
    const void *x, *y, *gamma;
    void *u, *v;
} petfmm_instance;

int petfmm_evaluate_batch(petfmm_ctx *ctx, int n_inst, const petfmm_instance *inst);

/*
 * petfmm_choose_levels -- the automatic L of petfmm_evaluate_batch for one
 * problem: minimises the Sec. 5.2 work estimate (Eq. 13 for the upper levels,
 * Eq. 14 for the leaves, uniform occupancy assumed) under the guard above.
 * Returns L >= 1, or PETFMM_EINVAL.
 */
int petfmm_choose_levels(int64_t n, int order, double sigma, const petfmm_domain *dom);

/* ---------------------------------------------------------------------- */
/* Autotuning of batches (tree depth and M2L shape, seeded by Sec. 5.2).   */
/* ---------------------------------------------------------------------- */
/*
 * A level rule: instances of this order whose particle count n has
 * floor(log2 n) == log2n get `levels` as their automatic tree depth (levels
 * <= 0 in petfmm_evaluate_batch) instead of the work model's.  With a
 * uniform quadtree the depth also fixes the leaf size (n / 4^L on average),
 * so this is the leaf-size choice too.  ms: the time the tuner measured for
 * the rule's sub-batch (informational).
 */
typedef struct {
    int32_t order, log2n, levels;
    float ms;
} petfmm_level_rule;

/*
 * petfmm_rule_levels -- the automatic L of one problem (n particles, order,
 * sigma, domain) under the given rules: the matching rule's L if there is
 * one and it satisfies the kernel-substitution guard of
 * petfmm_choose_levels, else petfmm_choose_levels.  Host only; rules may be
 * NULL when nrules = 0.  Returns L >= 1 or PETFMM_EINVAL.
 */
int petfmm_rule_levels(const petfmm_level_rule *rules, int nrules, int64_t n, int order,
                       double sigma, const petfmm_domain *dom);

/*
 * petfmm_set_level_rules -- install (copy) rules in the context: its
 * automatic L (petfmm_evaluate_batch with levels <= 0) follows
 * petfmm_rule_levels from then on.  nrules = 0 clears them.  Host only.
 * Returns PETFMM_OK or PETFMM_EINVAL (a rule with order outside 1..40,
 * log2n outside 0..62 or levels outside 1..15).
 */
int petfmm_set_level_rules(petfmm_ctx *ctx, const petfmm_level_rule *rules, int nrules);

typedef struct {
    int tc_blocks;      /* the PETFMM_OPT_TC_BLOCKS it chose (set on the context) */
    int tc_dense_pct;   /* the PETFMM_OPT_TC_DENSE it chose (set on the context) */
    int nrules;         /* rules written to out_rules (one per (order, log2n) class) */
    int changed;        /* rules whose L differs from the work model's */
    int evaluations;    /* evaluations run while tuning (warm-up ones included) */
    float ms_model;     /* the whole batch, work-model L, the context's options on entry */
    float ms_tuned;     /* the whole batch, tuned L and options */
} petfmm_tune_report;

/*
 * petfmm_tune_batch -- the autotuner for petfmm_evaluate_batch.  Seeded by
 * the work model of Sec. 5.2 (Eq. 13/14, petfmm_choose_levels), it times on
 * the GPU, with CUDA events on the context's stream, the median of `reps`
 * evaluations (after one warm-up) of:
 *   1. per class of instances (same order, same floor(log2 n)), the class
 *      as a sub-batch (with an empty instance at the batch's deepest level,
 *      so the launch sequence is the whole batch's) at L_model, L_model - 1
 *      and L_model + 1 (those the guard allows), keeping the fastest L as
 *      the class's rule -- another L than the model's only if it is at least
 *      2% faster;
 *   2. the whole batch under those rules with the context's options on
 *      entry and then every PETFMM_OPT_TC_BLOCKS in {0, 1, 2} with
 *      PETFMM_OPT_TC_DENSE in {1, 5}, keeping the fastest pair if it beats
 *      the entry options by 2%.
 * It installs the rules (petfmm_set_level_rules) and the two options in the
 * context, writes up to cap rules to out_rules (may be NULL with cap 0) and
 * fills *report.  The instances' levels fields are ignored; their u, v
 * receive the results of the tuning evaluations (the last one is the tuned
 * batch).  Synchronous.  Returns PETFMM_OK, PETFMM_EINVAL, PETFMM_ENOMEM,
 * PETFMM_ECUDA, or the first failing evaluation's status.
 */
int petfmm_tune_batch(petfmm_ctx *ctx, int n_inst, const petfmm_instance *inst, int reps,
                      petfmm_level_rule *out_rules, int cap, petfmm_tune_report *report);

/* ---------------------------------------------------------------------- */
/* Sharding one evaluation over several GPUs: the tree cut of Sec. 4 with  */
/* the work and communication model of Sec. 5.1-5.2 (host only).           */
/* ---------------------------------------------------------------------- */
/*
 * The quadtree of depth L is cut at level k (0 <= k <= L) into a root tree
 * and 4^k subtrees, one per level-k box (Morton index s); leaf_counts[m] is
 * the number of particles in leaf m (Morton order, 4^L entries).
 *
 * petfmm_shard_weights -- work[s] of every subtree: Eq. 13 for each of its
 *   (4^(L-k) - 1) / 3 non-leaf boxes plus Eq. 14 for each of its leaves with
 *   that leaf's particle count (the reading of Eq. 15), with n_c = 4,
 *   n_IL = 27, n_nd = 9.
 * petfmm_shard_comm -- expansion terms exchanged (both directions) between
 *   two lateral neighbour subtrees (Eq. 11: sum over n = k+1..L of
 *   alpha 2^(n-k) 4) and two diagonal neighbour subtrees (alpha 8 (L - k):
 *   the corner boxes, four per level each way, as the interaction lists give
 *   them; Eq. 12's printed form is garbled).  alpha: terms per box, e.g. p
 *   complex numbers.
 * petfmm_shard_partition -- assign the subtrees to nranks ranks
 *   (1 <= nranks <= 4^k) as contiguous runs of their z-order, with the
 *   largest run work as small as a contiguous split allows; owner[s] = rank.
 *   ranks[r] summarises rank r: work, particles, subtrees, its Morton range
 *   [first_subtree, last_subtree) and comm = the model's expansion terms
 *   (alpha = 1) over the edges it cuts.
 * petfmm_shard_halo -- what rank `rank` must receive from other ranks: the
 *   leaves (Morton, level L) adjacent to its leaves that other ranks own (their
 *   particles, for the near field), and the boxes (level, Morton) at levels
 *   k+1..L in the interaction lists of its boxes that other ranks own (their
 *   multipole expansions).  The level-k expansions of all subtrees are
 *   all-gathered and the root tree evaluated by every rank, so they are not
 *   listed.  Writes at most leaf_cap leaves and box_cap (level, box) pairs
 *   and sets *nleaves, *nboxes to the full counts (call with caps 0 first to
 *   size the arrays).
 * All return PETFMM_OK or PETFMM_EINVAL.
 */
typedef struct {
    double work;            /* Eq. 13-15 work of its subtrees */
    double comm;            /* model expansion terms over its cut edges (alpha = 1) */
    int64_t particles;
    int32_t subtrees;
    int32_t first_subtree;  /* its z-order run of level-k boxes: [first, last) */
    int32_t last_subtree;
} petfmm_shard_rank;

int petfmm_shard_weights(int L, int k, int order, const uint32_t *leaf_counts, double *work);
int petfmm_shard_comm(int L, int k, double alpha, double *lateral, double *diagonal);
int petfmm_shard_partition(int L, int k, int order, const uint32_t *leaf_counts, int nranks,
                           int32_t *owner, petfmm_shard_rank *ranks);
int petfmm_shard_halo(int L, int k, const int32_t *owner, int rank, int32_t *leaves,
                      int64_t leaf_cap, int32_t *boxes, int64_t box_cap, int64_t *nleaves,
                      int64_t *nboxes);

/* ---------------------------------------------------------------------- */
/* Serving: a thread-safe request loop with continuous batching.           */
/* ---------------------------------------------------------------------- */
typedef struct petfmm_server petfmm_server;

/*
 * One request = n_steps midpoint-RK2 steps (2 velocity evaluations each) of
 * the Lagrangian vortex method of Sec. 3 (Eq. 6: blobs move with their
 * velocity, gamma is carried unchanged).  x, y, gamma are HOST arrays copied
 * at submit time.  The domain is a square 1.25 times the blobs' bounding box;
 * after every evaluation the bounding box is reduced on the device and, if a
 * blob has left the square, the square is refitted before the next one.
 */
typedef struct {
    int64_t n;
    const double *x, *y, *gamma;  /* host, FP64, copied at submit */
    int levels, order;            /* levels <= 0: automatic */
    double sigma, dt;
    int n_steps;                  /* RK2 steps (evaluations = 2 * n_steps) */
    int precision;                /* PETFMM_FP64 or PETFMM_MIXED */
} petfmm_request;

typedef struct {
    int status;            /* PETFMM_OK or the request's error */
    double latency_ms;     /* submit -> completion */
    double queue_ms;       /* submit -> admission */
    int64_t n;
    double *x, *y;         /* host arrays owned by the server: final positions
                              (valid until petfmm_serve_release or destroy) */
    int32_t rounds;        /* scheduler rounds the request took part in */
    int32_t max_shared;    /* most requests resident in one of those rounds
                              (itself included): > 1 means its evaluations
                              ran batched with other requests' */
} petfmm_result;

/* hbm_budget_bytes: device memory the server may hold for admitted requests;
 * max_slots: most requests resident at once; max_queue: most waiting. */
int petfmm_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue,
                        petfmm_server **out);
/* Queue a request; PETFMM_EBUSY if the queue is full, PETFMM_EINVAL,
 * PETFMM_EDOMAIN if a position is not finite, or PETFMM_ENOMEM if the
 * request alone exceeds the budget.  The host arrays are copied and the
 * initial domain fitted here, in the caller's thread. */
int petfmm_serve_submit(petfmm_server *s, const petfmm_request *req, uint64_t *ticket);
/* PETFMM_ENOTREADY until the request is done; then fills *out. */
int petfmm_serve_poll(petfmm_server *s, uint64_t ticket, petfmm_result *out);
/* Free a finished request's result arrays. */
int petfmm_serve_release(petfmm_server *s, uint64_t ticket);
/* Stop the scheduler thread (finishing admitted work) and free everything. */
int petfmm_serve_destroy(petfmm_server *s);
/* Server counters since creation (a snapshot). */
typedef struct {
    uint64_t rounds;      /* scheduler rounds run (one batched evaluation each) */
    uint64_t submitted, admitted, completed;
    int32_t queued;       /* requests waiting now */
    int32_t max_active;   /* most requests resident in one round */
    double mean_active;   /* mean requests resident per round */
    double busy_ms;       /* scheduler-thread time spent in rounds */
    double up_ms;         /* time since petfmm_serve_create */
    /* scheduler-thread time by phase: admitting requests (device state,
     * copies in), launching rounds, waiting for the GPU, and the work after
     * a round (statuses, refitted domains, finished requests copied out) */
    double admit_ms, launch_ms, wait_ms, post_ms;
    double gpu_ms;        /* device time of the rounds: CUDA events on the
                             server's stream around each round's work (from
                             its start, after the admitted copies, to the
                             copy of its bounding boxes) */
} petfmm_serve_counters;
int petfmm_serve_stats(petfmm_server *s, petfmm_serve_counters *out);
/* Per-round trace: for the first min(cap, count) rounds since creation, the
 * round's start time (ms since creation) and the requests queued and
 * resident at that moment.  Returns the number of rounds recorded, or
 * PETFMM_EINVAL.  Host only. */
int petfmm_serve_trace(petfmm_server *s, double *t_ms, int32_t *queued, int32_t *active, int cap);
/* Per-request device-memory estimate used for admission (Table 1 adapted). */
size_t petfmm_serve_estimate_bytes(int64_t n, int levels, int order, int precision);

/* ---------------------------------------------------------------------- */
/* Inspection (the verification dump of Sec. 6.2) and instrumentation.    */
/* ---------------------------------------------------------------------- */

/* Bounds checks (the library built with -DPETFMM_CHECKS, libpetfmm_checked.so:
 * every index read from device data -- permutation, leaf ranges, work items,
 * the caller index of a blob, split-pair scratch bases -- is checked before
 * use; a bad one is skipped and its check's source line recorded, never a
 * trap).  Writes the first failing line of tree.cu, expansions.cu and p2p.cu
 * (0: none) to lines[0..2] and clears them; call after petfmm_sync().
 * Returns 3 in the checked build, 0 in the regular one (lines all 0), or
 * PETFMM_EINVAL for a NULL pointer.  Section 6.2's verification support;
 * the paper has no counterpart of the checks themselves. */
int petfmm_debug_checks(uint32_t *lines);

/* Tree of the last petfmm_evaluate (after petfmm_sync): host arrays
 * keys[n] (Morton key of each particle, input order), perm[n] (input index
 * of each sorted rank) and start[4^L + 1] (first rank of each leaf).
 * Any pointer may be NULL. */
int petfmm_debug_tree(petfmm_ctx *ctx, uint32_t *keys, uint32_t *perm, uint32_t *start);

/* Expansions of level `level` (2..L) of the last evaluation, copied to the
 * host as FP64 complex pairs out[(m * p + k) * 2 + {0,1}], m = Morton index.
 * which = 0: multipole (ME), scaled a_k / r^k; which = 1: local (LE), scaled
 * r^(k+1) b_k; r = box width at that level.  Only boxes with particles in
 * them are computed (an empty box's ME is exactly zero and its LE is never
 * evaluated); the values of the other boxes are unspecified. */
int petfmm_debug_expansions(petfmm_ctx *ctx, int level, int which, double *out);

/* Interaction list of box (level, ix, iy) as the device kernels enumerate it:
 * out[2 * i], out[2 * i + 1] = source box coordinates (at most 27 entries);
 * returns the count, or PETFMM_EINVAL. */
int petfmm_debug_interaction_list(int level, int ix, int iy, int32_t *out);

/* The mixed path's near-field factor of Eq. 8, g(q) = (1 - e^-q) / q with
 * q = kappa rho^2 (rho in leaf widths, kappa = w^2 / (2 sigma^2)), as the
 * host fits it for blob size sigma, leaf width w and relative tolerance tol
 * (the relative tolerance itself, e.g. 2.5e-6: the value that
 * PETFMM_OPT_NEAR_TOL sets, times 1e-9); host only, no GPU needed.  out[0] = degree,
 * out[1] = 1 if near pairs reach beyond the polynomial (the kernels then use
 * (1 - e^-q) / q there), out[2] = kappa and out[3] = the largest rho^2 the
 * polynomial covers, both as the kernels hold them (FP32), out[4 + k] = the
 * FP32 coefficient of rho^(2k), k = 0..14 (zero above the degree).  Returns
 * PETFMM_OK or PETFMM_EINVAL. */
int petfmm_debug_near_fit(double sigma, double wleaf, double tol, double *out);

/* The FP64 translation operators of Sec. 2.2 for order p (1..40) and kernel,
 * in the rescaled coefficients (box width r: ME a~_k = a_k / r^k; LE
 * r^(m+1) b_m for the vortex kernel, r^m b_m for the Laplace kernel), as the
 * host builds them for both precisions; host only, no GPU needed.  Complex
 * entries as (re, im) pairs:
 *   which = 0  M2M [c][l][k]: parent a~'_l += M[c][l][k] a~_k of child class c
 *              (c = (ix & 1) | (iy & 1) << 1; the child's centre is
 *              ((c & 1) - 1/2, (c >> 1) - 1/2) child widths from the parent's);
 *   which = 1  L2L [c][n][m]: child c^'_n += L[c][n][m] c^_m of the parent;
 *   which = 2  M2L [o][k][m]: target c^_m += T[o][k][m] a~_k for the source
 *              at offset delta_o (box widths), o as in petfmm_debug_m2l_images.
 * (For the Laplace kernel the M2L constant a_0 log r is added separately.)
 * Returns the number of doubles; copies them to out when cap is at least
 * that; PETFMM_EINVAL for bad arguments. */
int petfmm_debug_op_table(int order, int kernel, int which, double *out, int64_t cap);

/* Operator images of the tensor-core M2L (Sec. 2.2's M2L with the rescaled
 * coefficients: c^_m = sum_k T_delta[k][m] a~_k), as the host builds them
 * for order p (1..24) and kernel (PETFMM_KERNEL_VORTEX / _LAPLACE); host
 * only, no GPU needed.  Each image is the real 2p x 2p matrix
 * B = [[Re T, Im T], [-Im T, Re T]] (rows k: real parts of a~ then imaginary
 * parts; columns n: real parts of c^ then imaginary parts) split for 3xTF32
 * into hi (low 13 mantissa bits cleared) and lo = B - hi, padded with zeros
 * to Kpad = 2p rounded up to 8 rows, stored K-major as [k / 4][n][k % 4].
 *   blocks = 0: for each of the 40 offsets delta of [-3, 3]^2 \ [-1, 1]^2 in
 *     row order (increasing dy, then dx), hi then lo, Npad = 2p rounded up to
 *     16 columns.
 *   blocks = 1: for each (source class c', dy, dx), as
 *     g = c' 9 + (dy + 1) 3 + dx + 1, hi then lo, 4 NW columns (NW = 2p
 *     rounded up to 8): target class c's operator for delta = (2 dx + c'x -
 *     cx, 2 dy + c'y - cy) in columns c NW .., zeros where delta is within one
 *     box.
 * Returns the number of floats; copies them to out when cap is at least
 * that (out may be NULL with cap 0 to ask for the size); PETFMM_EINVAL for
 * bad arguments. */
int petfmm_debug_m2l_images(int order, int kernel, int blocks, float *out, int64_t cap);

/* Launch plan of a batch, built on the host without touching the device
 * (pointers in inst are not dereferenced).  Each task is written as five
 * int64 {range, instance, level, units, first block}; range 0 the scatter of
 * staged FP32 outputs to the caller's order (1024 blobs per block),
 * 1 leaf starts, 2 gather, 3 P2M, 4 P2P work list, 5 M2L (SIMT, units =
 * target boxes), 6 M2L on the tensor cores (units = CTAs), 7 tiled SIMT M2L
 * (units = CTAs), 100 + r the r-th M2M launch, 200 + r the r-th L2L launch,
 * as a context with default options would launch them.  Writes at most cap
 * tasks and returns the total count, or PETFMM_EINVAL. */
int petfmm_debug_plan(int precision, int n_inst, const petfmm_instance *inst, int64_t *out, int cap);

/* Options. */
enum {
    PETFMM_OPT_TIMING = 1,     /* 1: record per-stage CUDA events each evaluation */
    PETFMM_OPT_SPIN_LIMIT = 2, /* iteration limit of device-side waits (0 = default 2^26;
                                  < 0: no iterations, so the first wait of the tensor-core
                                  M2L reports PETFMM_ETIMEOUT -- for testing the report;
                                  that evaluation's u, v are then unspecified) */
    PETFMM_OPT_P2P_MODE = 3,   /* order in which the persistent P2P warps take the work
                                  items from their queue: 0 (default) heaviest first by
                                  the targets x sources cost of Eq. 14, 1 leaf (Morton)
                                  order; the results are identical */
    PETFMM_OPT_POISON = 4,     /* 1: fill the expansion buffers with NaN bytes before each
                                  evaluation (testing: a read of a never-written
                                  coefficient then shows up as NaN in u, v) */
    PETFMM_OPT_M2L_TC = 5,     /* mixed path: 1 (default) M2L of levels >= 8 on the tensor
                                  cores (3xTF32; see PETFMM_OPT_TC_BLOCKS), 0 all levels
                                  on the FP32 SIMT kernels */
    PETFMM_OPT_TC_DENSE = 6,   /* percent (0..100, default 1) of a tensor-core (or
                                  tiled) unit's targets that must hold particles for the
                                  unit to run there; sparser units use the per-box SIMT
                                  kernel */
    PETFMM_OPT_TC_SEG = 8,     /* widest tensor-core M2L unit in parent cells: 128
                                  (default), 256 or 512 */
    PETFMM_OPT_NEAR_TOL = 9,   /* mixed path: relative tolerance of the polynomial that
                                  evaluates Eq. 8's factor (1 - e^-q)/q, in units of
                                  1e-9 (1 .. 1000000; default 2500 = 2.5e-6, a quarter
                                  of the 1e-5 budget against FP64; 100 = 1e-7 is the
                                  FP32 rounding level).  Applies from the next
                                  evaluation. */
    PETFMM_OPT_GRAPH = 10,     /* 1: run an evaluation's launch sequence as a CUDA graph,
                                  captured on the first evaluation of a launch shape
                                  (sizes, tree depths, orders, options; the caller's
                                  arrays may change) and replayed while it repeats;
                                  0 (default) plain launches.  Results are identical.
                                  The context's stream must not be capturing. */
    PETFMM_OPT_P2P_PAIRS = 11, /* mixed path: 1 (default) each pair of blobs in the same
                                  or neighbouring leaves that both hold >= 32 blobs is
                                  evaluated once, its kernel value serving both blobs
                                  (K of Eq. 8 is odd);
                                  heavy pairs are cut into pieces for load balance.
                                  0: every leaf sums its 9 leaves directly.  Both
                                  deterministic; they differ by FP32 rounding of the
                                  sums.  Extra device memory in mode 1: 88 bytes per
                                  blob and 28 per leaf. */
    PETFMM_OPT_TC_BLOCKS = 13, /* mixed path, with PETFMM_OPT_M2L_TC = 1: the shape of
                                  the tensor-core M2L.  0 (default): blocks of 8 x 16
                                  parent cells (all four child classes) at levels >= 8,
                                  and at levels 5 to 7 when the evaluation has at least
                                  512 blocks there (a batch; a single tree runs those
                                  levels on the tiled SIMT kernel in FP32); 1: blocks at every
                                  level >= 5; 2: row units (one child class, a segment
                                  of a parent row) at levels >= 8 and no blocks.
                                  Results differ by FP32 rounding only. */
    PETFMM_OPT_TC_PIPE = 14,   /* mixed path, block tensor-core M2L: 1: one staging buffer
                                  for the source expansions (a source class is split after
                                  every MMA so far is done; two stages per offset, two CTAs
                                  per SM, in launches of >= 2048 blocks); 2: two staging
                                  buffers, the next class split while the current one
                                  multiplies (one stage per offset, one CTA per SM; p <= 20);
                                  0 (default): 2 in launches under 2048 blocks where it
                                  fits, else 1.  The two differ by FP32 rounding when the
                                  stages per offset differ. */
    PETFMM_OPT_OVERLAP = 15,   /* mixed path: 1 (default) run the record gather and the
                                  expansion chain (P2M, M2M, M2L, L2L) on a second
                                  stream of the context, overlapping the near field:
                                  its work lists need only the leaf starts, the pair
                                  and directed kernels wait for the gather only; the
                                  final pass waits for both.  0: one stream.  Results
                                  identical. */
    PETFMM_OPT_KERNEL = 12     /* the sum the context evaluates (the kernel parameter of
                                  the paper's Evaluator, Sec. 6.1):
                                  PETFMM_KERNEL_VORTEX (default) the blob velocity of
                                  Eq. 8/9; PETFMM_KERNEL_LAPLACE the 2D logarithmic
                                  potential u_i = sum_{j != i} g_j log|x_i - x_j|
                                  (coincident pairs excluded; sigma unused), v = 0,
                                  by the same FMM with the series of the complex
                                  logarithm (p terms, the log counted as one).  Both
                                  precisions; the mixed path sums the near field
                                  directly (PETFMM_OPT_P2P_PAIRS applies to the
                                  vortex kernel only). */
};
enum { PETFMM_KERNEL_VORTEX = 0, PETFMM_KERNEL_LAPLACE = 1 };
int petfmm_set_option(petfmm_ctx *ctx, int option, int64_t value);

/* Stages reported by petfmm_stage_times (milliseconds, last evaluation).
 * PAIRS: the pairwise near-field kernel (mixed path, PETFMM_OPT_P2P_PAIRS = 1;
 * about zero otherwise); P2P: the directed near field (and, on the FP64 path,
 * L2P and the output in the same kernel); FINAL: the mixed path's final pass
 * (L2P, the sum of the near-field parts, the output in the caller's order;
 * about zero on the FP64 path).  With PETFMM_OPT_OVERLAP the stages
 * GATHER..L2L run beside WORKLIST..P2P, so the times overlap (their sum
 * exceeds the evaluation's), WORKLIST also holds any wait for the end of the
 * gather and P2P any wait for the end of L2L. */
enum {
    PETFMM_STAGE_MORTON = 0, PETFMM_STAGE_SORT, PETFMM_STAGE_GATHER, PETFMM_STAGE_P2M,
    PETFMM_STAGE_M2M, PETFMM_STAGE_M2L, PETFMM_STAGE_L2L, PETFMM_STAGE_WORKLIST,
    PETFMM_STAGE_PAIRS, PETFMM_STAGE_P2P, PETFMM_STAGE_FINAL, PETFMM_STAGE_COUNT
};
int petfmm_stage_times(petfmm_ctx *ctx, float *ms, int cap);

typedef struct {
    uint64_t kernel_launches;  /* kernels this context has launched */
    uint64_t evaluations;
    int64_t p2p_pairs;         /* ordered near-field pairs of the last evaluation */
    int64_t m2l_pairs;         /* (target, source) M2L translations of the last evaluation */
    int64_t p2p_items;         /* P2P work items of the last evaluation */
    float p2p_load_balance;    /* min / max CTA busy time of the last P2P (Eq. 20) */
    int64_t p2p_pair_items;    /* pairwise mode: (leaf pair, piece) items of the last evaluation */
    int64_t p2p_split_entries; /* pairwise mode: scratch entries the split pairs wanted (pairs
                                  are split only when these fit in one entry per blob) */
    int64_t p2p_sym_pairs;     /* pairwise mode: unordered blob pairs the pair kernel
                                  evaluated (each serves two of the ordered p2p_pairs) */
    float pairs_load_balance;  /* pairwise mode: min / max CTA busy time of the pair kernel */
    int64_t occupied_leaves;   /* leaves holding at least one particle in the last
                                  evaluation (all instances) */
} petfmm_stats;
/* Counters; p2p_pairs, m2l_pairs, p2p_items and the load balances need
 * PETFMM_OPT_TIMING and a petfmm_sync() after the evaluation. */
int petfmm_get_stats(petfmm_ctx *ctx, petfmm_stats *out);

/*
 * petfmm_tree_noalloc -- the quadtree build alone (binning, stable z-order
 * sort, leaf ranges: the same results petfmm_debug_tree reports after an
 * evaluation) without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * call cudaMalloc -- a host application whose own caching allocator already
 * holds the GPU's memory, code with a fixed device-memory budget, or loops
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause.  All intermediate buffers live in one static device array sized for
 * PETFMM_NOALLOC_MAX_N particles (about 16.3 MB, held on every GPU that loads
 * the library until the process exits).
 *   dom, levels  domain square and depth L (1..15), as for petfmm_create.
 *   dtype        PETFMM_F64 or PETFMM_F32 storage of x, y.
 *   n            particles, 0 <= n <= PETFMM_NOALLOC_MAX_N; larger n returns
 *                PETFMM_ENOMEM without launching anything.
 *   x, y         device arrays of n positions.
 *   keys         device array of n Morton keys in input order, or NULL.
 *   perm         device array: perm[r] = input index of sorted rank r.
 *   start        device array of 4^L + 1 leaf starts.
 * Runs on cuda_stream (a cudaStream_t, NULL for the legacy default stream)
 * and waits for it before returning (so it cannot be called while that
 * stream is capturing).  Returns PETFMM_OK, PETFMM_EDOMAIN (a particle
 * outside the domain or NaN; outputs unspecified; the next call is
 * unaffected), PETFMM_EINVAL, PETFMM_ENOMEM (n above the maximum, or the
 * device had no room for the static array when it was created) or
 * PETFMM_ECUDA.  The first call in a CUDA context (for the primary context:
 * the first call on a device) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Lookups are cached per context ID, so a context
 * made after cudaDeviceReset gets a fresh lookup.  The array is created when
 * the library's device code is loaded onto the device (the first lookup,
 * under lazy module loading).  Every call uses the same array, so calls that
 * overlap on the GPU (other streams or host threads) race with each other;
 * serialise them.  n = 0 writes start[] as all zeros.
 */
#define PETFMM_NOALLOC_MAX_N 1048576
int petfmm_tree_noalloc(const petfmm_domain *dom, int levels, int dtype, int64_t n, const void *x,
                        const void *y, uint32_t *keys, uint32_t *perm, uint32_t *start,
                        void *cuda_stream);

/* Measured pipe rates of the current device, for quoting roofline fractions
 * (Sec. 5.2 costs the steps by operation counts; the paper has no
 * counterpart of the measurement itself).  Runs microbenchmarks on every SM
 * for tens of milliseconds on a private stream and waits for them:
 *   fp32_ops      FP32 FFMA instructions per second x 32 lanes (one op each)
 *   fp64_ops      FP64 DFMA, counted the same way
 *   mufu_rcp_ops  special-function unit, rcp.approx
 *   mufu_ex2_ops  special-function unit, ex2.approx
 *   tf32_flops    dense TF32 MMA on the tensor cores (tcgen05 kind::tf32,
 *                 M = 128, N = 256, K = 8 from shared memory), 2 flops per MAC
 *   sms           streaming multiprocessors used
 * Returns PETFMM_OK, PETFMM_EINVAL (out NULL), PETFMM_ENOMEM, PETFMM_ECUDA or
 * PETFMM_ETIMEOUT (the tensor-core wait gave up; tf32_flops then
 * unspecified).  Allocates and frees a few MB of device memory. */
typedef struct {
    double fp32_ops, fp64_ops, mufu_rcp_ops, mufu_ex2_ops, tf32_flops;
    int sms;
} petfmm_peaks;
int petfmm_measure_peaks(petfmm_peaks *out);

const char *petfmm_strerror(int code);
int petfmm_version(void);

/* ------------------------------------------------------------------------
 * Three dimensions: the Laplace potential and field of point charges by the
 * FMM on a uniform octree -- the extension the paper names first (Sec. 8:
 * tree, work model and partition unchanged; a new kernel with its 3D series
 * and translation operators).  For every particle i
 *     phi_i = sum_{j != i} q_j / |x_i - x_j|,
 *     E_i   = -grad phi_i = sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3,
 * self and coincident pairs contributing 0.  Series: solid harmonics of the
 * 1/r kernel with p terms (degrees 0..p-1, p (p + 1) / 2 complex
 * coefficients per box), rescaled by the box width; near domain = the leaf
 * and its up to 26 neighbours; interaction list = the children of the
 * parent's neighbours that are not neighbours of the box (at most 189),
 * levels >= 2.  Binning and z-order as in 2D with three interleaved
 * coordinates (bit b of ix, iy, iz to bits 3b, 3b + 1, 3b + 2).
 * ------------------------------------------------------------------------ */
typedef struct petfmm3d_ctx petfmm3d_ctx;
typedef struct {
    double x0, y0, z0, width; /* closed cube [x0, x0 + W] x [y0, y0 + W] x [z0, z0 + W] */
} petfmm_domain3d;
#define PETFMM3D_MAX_L 8
#define PETFMM3D_MAX_P 16

/* levels 1..PETFMM3D_MAX_L (8^L leaves), order p 1..PETFMM3D_MAX_P;
 * precision PETFMM_FP64 (every step in FP64) or PETFMM_MIXED (expansions,
 * translations, near field and L2P in FP32 on leaf-relative coordinates;
 * binning in FP64); dtype PETFMM_F64 or PETFMM_F32 storage of x, y, z, q and
 * of the outputs; cuda_stream: the cudaStream_t every launch goes to (NULL:
 * the legacy default stream).  Uploads the operator tables (synchronous).
 * Returns PETFMM_OK, PETFMM_EINVAL, PETFMM_ENOMEM or PETFMM_ECUDA. */
int petfmm3d_create(const petfmm_domain3d *dom, int levels, int order, int precision, int dtype,
                    void *cuda_stream, petfmm3d_ctx **out);
/* One evaluation of n particles, asynchronous on the context's stream.
 * x, y, z, q: device arrays of n values (dtype of the context), read only;
 * phi, ex, ey, ez: device arrays of n values, written in the caller's order.
 * The caller owns all eight and keeps them valid until petfmm3d_sync returns.
 * A particle outside the closed cube (or NaN) is reported as PETFMM_EDOMAIN
 * by petfmm3d_sync (outputs unspecified).  Grows the context's buffers when n
 * or the tree needs it (cudaMalloc; PETFMM_ENOMEM if that fails).  Returns
 * PETFMM_OK, PETFMM_EINVAL (n < 0 or above 2^30, a null array), PETFMM_ENOMEM
 * or PETFMM_ECUDA. */
int petfmm3d_evaluate(petfmm3d_ctx *ctx, int64_t n, const void *x, const void *y, const void *z,
                      const void *q, void *phi, void *ex, void *ey, void *ez);
/* Waits for the stream; returns the device status of the last evaluation
 * (PETFMM_OK or PETFMM_EDOMAIN) or PETFMM_ECUDA. */
int petfmm3d_sync(petfmm3d_ctx *ctx);
enum {
    PETFMM3D_OPT_TIMING = 1, /* 1: record CUDA events per stage */
    PETFMM3D_OPT_M2L_TC = 2  /* mixed path, p <= 8: 1 (default) run M2L on the
                                tensor cores (tcgen05, TF32 hi/lo split, FP32
                                accumulation); 0 the SIMT GEMM kernel.  Results
                                differ by FP32-level rounding. */
};
int petfmm3d_set_option(petfmm3d_ctx *ctx, int option, int64_t value);
enum {
    PETFMM3D_STAGE_BIN = 0, PETFMM3D_STAGE_SORT, PETFMM3D_STAGE_GATHER, PETFMM3D_STAGE_P2M,
    PETFMM3D_STAGE_M2M, PETFMM3D_STAGE_M2L, PETFMM3D_STAGE_L2L, PETFMM3D_STAGE_NEAR,
    PETFMM3D_STAGE_COUNT
};
/* milliseconds per stage of the last evaluation (SORT includes the leaf
 * starts; NEAR is the near field with L2P and the output); returns the
 * number written, PETFMM_ENOTREADY without a timed evaluation. */
int petfmm3d_stage_times(petfmm3d_ctx *ctx, float *ms, int cap);
/* Host copies of the last evaluation's sorted keys and permutation (n each;
 * perm[r] = input index of sorted rank r) and its 8^L + 1 leaf starts. */
int petfmm3d_debug_tree(petfmm3d_ctx *ctx, int64_t n, uint32_t *skeys, uint32_t *perm,
                        uint32_t *start);
/* kernels this context has launched */
uint64_t petfmm3d_launches(const petfmm3d_ctx *ctx);
/* Host only (no device work): the mixed path's M2L operator for the offset
 * (dx, dy, dz) between same-level boxes (target minus source, in box widths;
 * |each| <= 3, max >= 2) and order p, in the real basis of a real
 * potential's coefficients (real index r < p (p + 1) / 2: Re of coefficient
 * n (n + 1) / 2 + m; then Im of the coefficients with m > 0, in order), for
 * expansions scaled by the box width.  out[k * p^2 + r] = d(output r) /
 * d(input k), FP64 (the library rounds it to FP32); cap >= p^4 doubles. */
int petfmm3d_debug_m2l_operator(int order, int dx, int dy, int dz, double *out, int64_t cap);
/* kinds of petfmm3d_debug_shift_operator */
enum { PETFMM3D_SHIFT_M2M = 0, PETFMM3D_SHIFT_L2L = 1 };
/* Host only (no device work): the mixed path's M2M (child of the octant to
 * its parent) or L2L (parent to its child of the octant) operator of order
 * p <= 16 (the library uses them for p <= 8), in the real basis of
 * petfmm3d_debug_m2l_operator, for expansions scaled by each box's own
 * width (the Sec. 8 octree: a child is half its parent's width).  Octant
 * bit 0/1/2 set: the child lies on the +x/+y/+z side of the parent's
 * centre.  out[k * p^2 + r] = d(output r) / d(input k), FP64 (the library
 * rounds it to FP32); cap >= p^4 doubles; PETFMM_EINVAL for a bad kind,
 * octant, order or cap. */
int petfmm3d_debug_shift_operator(int order, int kind, int octant, double *out, int64_t cap);
int petfmm3d_destroy(petfmm3d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PETFMM_H */
