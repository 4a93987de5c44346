// engine.cu -- the evaluation context and the C ABI of include/petfmm.h.
//
// One evaluation (Sec. 2.2, Fig. 2) is this sequence of launches on the
// context's stream, every one of them covering all instances of the batch:
//   binning -> radix sort (ceil(bits / 8) passes) -> leaf starts -> gather
//   -> P2M -> M2M (one launch per level, bottom-up) -> M2L (all levels in one
//   launch) -> L2L (one launch per level, top-down) -> P2P work list
//   -> P2P + L2P.
// The host only plans (task tables, offsets) and launches; nothing is read
// back until petfmm_sync().
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/petfmm.h"
#include "kernels.cuh"

using namespace petfmm;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// Grows `b` to at least `bytes` (waits for the stream first: the old buffer
// may still be in use).  Returns PETFMM_OK or PETFMM_ENOMEM / PETFMM_ECUDA.
int ensure(DevBuf &b, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return PETFMM_OK;
    if (b.p) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return PETFMM_ECUDA;
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 8;
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return PETFMM_ENOMEM;
        }
        want = bytes;
    }
    b.cap = want;
    return PETFMM_OK;
}

// The tasks of one launch.  Kernels binary-search their block in a
// contiguous slice of the uploaded task array, so each range keeps its own
// list while planning and the lists are laid out one after another at the
// end (flatten_tasks).
struct TaskRange {
    int first = 0;
    int count = 0;
    int64_t nblocks = 0;
    std::vector<Task> list;
};

struct Plan {
    std::vector<InstDesc> inst;
    std::vector<Task> tasks;
    TaskRange outscatter, start, particles, leaves_p2m, leaves_wl, m2l, m2l_tc, m2l_tcb, m2l_log;
    // tiled SIMT M2L, one launch per order class (p <= 8, 12, 18, 24): each
    // launch's kernel is specialised for its class's largest order
    static constexpr int kTileClasses = 4;
    TaskRange m2l_tile[kTileClasses];
    int tile_pmax[kTileClasses] = {};
    int64_t tile_blocks() const {
        int64_t b = 0;
        for (const TaskRange &r : m2l_tile) b += r.nblocks;
        return b;
    }
    std::vector<TaskRange> m2m, l2l;  // in launch order
    int64_t N = 0, nleaves = 0, nstart = 0, ncoef = 0, items_cap = 0;
    int nbits = 0, pmax = 1, Lmax = 0;
    int deg = 0, general = 0;          // mixed P2P variant (max over instances)
    size_t tc_smem = 0;                // dynamic shared memory of the tensor-core M2L
    int tcb_pmax = 0;                  // largest order among the block units
};

struct Problem {
    petfmm_domain dom;
    int L, p;
    double sigma;
    int64_t n;
    const void *x, *y, *g;
    void *u, *v;
};

}  // namespace

namespace {
// default relative tolerance of the near-field polynomial (PETFMM_OPT_NEAR_TOL)
constexpr double kNearTolDefault = 2.5e-6;
// default widest tensor-core M2L unit (PETFMM_OPT_TC_SEG)
constexpr int kTcSegDefault = 128;
}  // namespace

struct petfmm_ctx {
    petfmm_domain dom{};
    int L = 0, p = 0;
    double sigma = 0.0;
    int precision = 0, dtype = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool timing = false;
    int p2p_mode = 0;  // 0: work items heaviest first (Eq. 14 weights), 1: Morton order
    bool p2p_pairs = true;  // mixed path: neighbouring leaves pairwise (PETFMM_OPT_P2P_PAIRS)
    int kernel = KERNEL_VORTEX;  // PETFMM_OPT_KERNEL
    int tc_blocks = 0;           // PETFMM_OPT_TC_BLOCKS: 0 automatic, 1 always, 2 never
    int tc_pipe = 0;             // PETFMM_OPT_TC_PIPE: 0 automatic, 1 single A, 2 double A
    bool poison = false;
    bool m2l_tc = true;
    // measured on GB300 (clustered 16M and lattice 1M blobs): 128-cell units
    // with a 25% occupancy threshold gave the fastest M2L on both
    int tc_dense_pct = 1;
    int tc_segmax = kTcSegDefault;
    double near_tol = kNearTolDefault;
    int64_t spin_limit = 0;
    uint64_t launches = 0, evaluations = 0;

    DevBuf keysA, keysB, valsA, valsB, hist, scratch, start, xs, ys, gs, rec, me, le, cnt, off,
        items, ctrl, plan_dev, busy, ucount, recu, occ, items_u, ikA, ikB, ivA, ivB, ihist, own,
        part, pitems, pxtra, pxs, ustage;
    DevBuf hx, hy, hg, hu, hv;  // device staging for petfmm_evaluate_host
    std::map<int, OpTables> tables;

    // plan upload
    std::vector<unsigned char> last_upload;
    void *pinned = nullptr;
    size_t pinned_cap = 0;
    cudaEvent_t upload_done = nullptr;
    bool upload_pending = false;

    // last evaluation (for inspection)
    Plan plan;
    bool sorted_in_first = true;
    int p2p_grid = 0, pairs_grid = 0;  // CTAs of the persistent near-field launches
    // CUDA-graph replay of the launch sequence (PETFMM_OPT_GRAPH)
    bool use_graph = false;
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;  // captures run here (the legacy stream cannot)
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey = 0, glaunches = 0;
    // stage events: ev[s] starts stage s, ev[COUNT] ends the evaluation and
    // ev[COUNT + 1] ends the L2L stage (its stream may be aux)
    cudaEvent_t ev[PETFMM_STAGE_COUNT + 2] = {};
    // the expansion chain's stream on the mixed path, and its fork / join
    bool overlap = true;  // PETFMM_OPT_OVERLAP
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_gathered = nullptr;
    bool ev_recorded = false;
    // level rules of the automatic L (petfmm_set_level_rules / petfmm_tune_batch)
    std::vector<petfmm_level_rule> rules;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int check_problem(const petfmm_domain *dom, int L, int p, double sigma) {
    if (!dom) return PETFMM_EINVAL;
    if (!(dom->width > 0.0) || !std::isfinite(dom->width) || !std::isfinite(dom->x0) ||
        !std::isfinite(dom->y0))
        return PETFMM_EINVAL;
    if (L < 1 || L > MAX_L) return PETFMM_EINVAL;
    if (p < 1 || p > MAX_P) return PETFMM_EINVAL;
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return PETFMM_EINVAL;
    return PETFMM_OK;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PETFMM_OK;
    if (e == cudaErrorMemoryAllocation) return PETFMM_ENOMEM;
    return PETFMM_ECUDA;
}

// ---------------------------------------------------------------------------
// Near-field polynomial: Chebyshev interpolation of g(q) = (1 - e^-q) / q on
// [0, Q], converted to monomials in rho^2 (q = kappa rho^2).  The smallest
// degree (at least 4) whose relative error on a fine grid stays below the
// context's tolerance is taken: by default 2.5e-6, a quarter of the 1e-5
// budget of the mixed path against FP64 (each pair's factor g is then within
// 2.5e-6 of exact, before FP32 rounding); 1e-7 reaches the FP32 rounding of
// the Horner evaluation itself.
// ---------------------------------------------------------------------------
double g_exact(double q) { return q == 0.0 ? 1.0 : -std::expm1(-q) / q; }

bool solve_dense(std::vector<double> &A, std::vector<double> &b, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return true;
}

// Fits on q in [0, Q]; returns degree (0 on failure) and coefficients in rho^2.
int fit_near_poly(double Q, double kappa, double tol, float *coef) {
    for (int d = 4; d <= 12; ++d) {
        const int n = d + 1;
        std::vector<double> A(size_t(n) * n), b(n);
        for (int j = 0; j < n; ++j) {
            const double t = 0.5 * (1.0 - std::cos(M_PI * (j + 0.5) / n));  // in [0, 1]
            double pw = 1.0;
            for (int k = 0; k < n; ++k) {
                A[size_t(j) * n + k] = pw;
                pw *= t;
            }
            b[j] = g_exact(t * Q);
        }
        if (!solve_dense(A, b, n)) continue;
        // coefficients in rho^2: a_k = b_k (kappa / Q)^k
        double a[16];
        const double r = kappa / Q;
        double rp = 1.0;
        for (int k = 0; k < n; ++k) {
            a[k] = b[k] * rp;
            rp *= r;
        }
        double err = 0.0;
        const double smax = Q / kappa;
        for (int i = 0; i <= 4000; ++i) {
            const double s = smax * i / 4000.0;
            double v = a[d];
            for (int k = d - 1; k >= 0; --k) v = v * s + a[k];
            err = std::max(err, std::fabs(v - g_exact(kappa * s)) / g_exact(kappa * s));
        }
        if (err < tol) {
            for (int k = 0; k <= POLY_MAX; ++k) coef[k] = k <= d ? float(a[k]) : 0.0f;
            return d;
        }
    }
    return 0;
}

// Largest q the polynomial alone may cover.
constexpr double kPolyQMax = 2.0;

void fill_p2p_constants(InstDesc &d, double tol) {
    const double w = d.wleaf;
    const double kappa = w * w / (2.0 * d.sigma * d.sigma);
    d.kappa = float(kappa);
    d.cnear = float(w / (4.0 * M_PI * d.sigma * d.sigma));
    d.cfar = float(1.0 / (2.0 * M_PI * w));
    d.inv2s2 = 1.0 / (2.0 * d.sigma * d.sigma);
    d.cnear64 = 1.0 / (2.0 * M_PI);
    d.cfar64 = 1.0 / (2.0 * M_PI * w);
    // The fit depends on kappa alone; evaluations of the same problem shape
    // (a served request's every round, a repeated batch) reuse it.
    struct Fit {
        int general, deg;
        float split;
        float poly[POLY_MAX + 1];
    };
    static std::mutex mu;
    static std::map<std::pair<double, double>, Fit> cache;
    const std::pair<double, double> key(kappa, tol);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            d.general = it->second.general;
            d.deg = it->second.deg;
            d.qsplit_rho2 = it->second.split;
            std::memcpy(d.poly, it->second.poly, sizeof(d.poly));
            return;
        }
    }
    // near pairs are at most 2 leaf widths apart per axis: rho^2 <= 8
    const double rho2max = 8.0 * (1.0 + 1e-6);
    const double qmax = kappa * rho2max;
    if (qmax <= kPolyQMax) {
        d.general = 0;
        d.deg = fit_near_poly(qmax, kappa, tol, d.poly);
        d.qsplit_rho2 = float(rho2max);
    } else {
        d.general = 1;
        d.deg = fit_near_poly(1.0, kappa, tol, d.poly);
        d.qsplit_rho2 = float(1.0 / kappa);
    }
    Fit f;
    f.general = d.general;
    f.deg = d.deg;
    f.split = d.qsplit_rho2;
    std::memcpy(f.poly, d.poly, sizeof(f.poly));
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() > 4096) cache.clear();
    cache[key] = f;
}

OpTables *get_tables(petfmm_ctx *c, int p, int kernel, int *err) {
    const int key = p | (kernel << 16);
    auto it = c->tables.find(key);
    if (it != c->tables.end()) return &it->second;
    OpTables t;
    cudaError_t e = build_op_tables(p, kernel, &t);
    if (e != cudaSuccess) {
        free_op_tables(&t);
        *err = cuda_status(e);
        return nullptr;
    }
    return &(c->tables[key] = t);
}

void add_task(TaskRange &r, int inst, int level, int64_t count, int64_t per_block) {
    if (count <= 0) return;
    Task t;
    t.inst = inst;
    t.level = level;
    t.count = count;
    t.block0 = r.nblocks;
    r.list.push_back(t);
    r.count++;
    r.nblocks += (count + per_block - 1) / per_block;
}

void flatten_tasks(Plan &pl) {
    pl.tasks.clear();
    auto put = [&](TaskRange &r) {
        r.first = int(pl.tasks.size());
        pl.tasks.insert(pl.tasks.end(), r.list.begin(), r.list.end());
    };
    put(pl.outscatter);
    put(pl.start);
    put(pl.particles);
    put(pl.leaves_p2m);
    put(pl.leaves_wl);
    put(pl.m2l);
    put(pl.m2l_tc);
    put(pl.m2l_tcb);
    for (TaskRange &r : pl.m2l_tile) put(r);
    put(pl.m2l_log);
    for (TaskRange &r : pl.m2m) put(r);
    for (TaskRange &r : pl.l2l) put(r);
}

// order class of the tiled M2L launches: p <= 8, 12, 18, 24
// Fewest block units at levels 5 to 7 for which those levels run as blocks
// rather than on the tiled SIMT kernel (a batch of 512 trees has 3,260; one
// tree, at most 42).
constexpr int64_t kTcbShallowMinUnits = 512;

int tile_class(int p) { return p <= 8 ? 0 : p <= 12 ? 1 : p <= 18 ? 2 : 3; }

int build_plan(int precision, int kernel, bool use_tc, int tc_blocks, int tc_segmax, double near_tol,
               const std::vector<Problem> &probs, Plan &pl) {
    pl = Plan();
    const int ni = int(probs.size());
    int inst_bits = 0;
    while ((1 << inst_bits) < ni) ++inst_bits;
    int Lmax = 0, pmax = 1;
    for (const auto &pb : probs) {
        Lmax = std::max(Lmax, pb.L);
        pmax = std::max(pmax, pb.p);
    }
    pl.Lmax = Lmax;
    pl.pmax = pmax;
    pl.nbits = 2 * Lmax + inst_bits;
    if (pl.nbits > 32) return PETFMM_EINVAL;
    int64_t poff = 0, loff = 0, eoff = 0;
    for (int i = 0; i < ni; ++i) {
        const Problem &pb = probs[i];
        InstDesc d;
        std::memset(&d, 0, sizeof(d));
        inst_set_domain(d, pb.dom.x0, pb.dom.y0, pb.dom.width, pb.L);
        d.kernel = kernel;
        d.sigma = pb.sigma;
        d.L = pb.L;
        d.p = pb.p;
        d.n = pb.n;
        d.poff = poff;
        d.loff = loff;
        d.soff = loff + i;
        d.eoff = eoff;
        d.key_hi = inst_bits ? (uint32_t(i) << (2 * Lmax)) : 0u;
        d.x = pb.x;
        d.y = pb.y;
        d.g = pb.g;
        d.u = pb.u;
        d.v = pb.v;
        fill_p2p_constants(d, near_tol);
        if (precision == PETFMM_MIXED && d.deg == 0) return PETFMM_EINVAL;
        pl.deg = std::max(pl.deg, d.deg);
        pl.general |= d.general;
        pl.inst.push_back(d);
        const int64_t nleaf = int64_t(1) << (2 * pb.L);
        poff += pb.n;
        loff += nleaf;
        eoff += lvl_off(pb.L + 1) * pb.p;
    }
    pl.N = poff;
    pl.nleaves = loff;
    pl.nstart = loff + ni;
    pl.ncoef = eoff;
    if (pl.N >= (int64_t(1) << 31)) return PETFMM_EINVAL;

    const int tpi = precision == PETFMM_MIXED ? P2P_TPI_MIXED : P2P_TPI_F64;
    int64_t items_cap = 0;
    for (int i = 0; i < ni; ++i) {
        InstDesc &d = pl.inst[i];
        const int64_t nleaf = int64_t(1) << (2 * d.L);
        for (int l = 0; l <= MAX_L; ++l) d.tc_unit0[l] = -1;
        d.tc_segmax = tc_segmax;
        d.tc_levels = 0;
        d.tcb_levels = 0;
        add_task(pl.outscatter, i, d.L, d.n, 1024);  // output scatter: 4 blobs per thread
        add_task(pl.start, i, d.L, nleaf + 1, 256);
        add_task(pl.particles, i, d.L, d.n, 256);
        add_task(pl.leaves_p2m, i, d.L, nleaf, 256);
        add_task(pl.leaves_wl, i, d.L, nleaf, 256);
        for (int l = 2; l <= d.L; ++l) {
            // levels the tensor cores can take get both launches: the tensor
            // cores translate the dense units, the SIMT kernel the boxes of the
            // sparse ones (a data-dependent split made on the device)
            // (row units: only when blocks are switched off, PETFMM_OPT_TC_BLOCKS = 2)
            if (precision == PETFMM_MIXED && use_tc && tc_blocks == 2 &&
                m2l_tc_supported(d.p, l, tc_segmax)) {
                d.tc_unit0[l] = pl.m2l_tc.nblocks;  // one unit per block
                d.tc_levels |= 1u << l;
                add_task(pl.m2l_tc, i, l, m2l_tc_units(l, tc_segmax), 1);
                pl.tc_smem = std::max(pl.tc_smem, m2l_tc_smem_bytes(d.p, m2l_tc_seg(l, tc_segmax)));
            }
            add_task(pl.m2l, i, l, int64_t(1) << (2 * l), M2L_BOXES);
            if (kernel == KERNEL_LAPLACE) add_task(pl.m2l_log, i, l, int64_t(1) << (2 * l), 256);
        }
        items_cap += d.n / tpi + std::min<int64_t>(d.n, nleaf) + 1;
    }
    // the other levels of the mixed path: dense units on the tensor cores in
    // blocks of 8 x 16 parent cells (levels >= 8; levels 5 to 7 too when the
    // plan has many blocks), the rest on the tiled SIMT kernel (their units
    // follow the row units in the unit-count array: blocks, then the tile
    // classes one by one)
    if (precision == PETFMM_MIXED) {
        int64_t base = pl.m2l_tc.nblocks;
        // levels 5 to 7: a batch fills the GPU with blocks; a single tree has
        // few, and runs them on the tiled SIMT kernel (also in FP32, where
        // the blocks' 3xTF32 adds about 1e-6 to the rel-L2 error)
        int64_t blocks = 0;
        for (int i = 0; i < ni; ++i)
            for (int l = 2; l <= std::min(pl.inst[i].L, 7); ++l)
                if (!((pl.inst[i].tc_levels >> l) & 1u) && m2l_tcb_supported(pl.inst[i].p, l))
                    blocks += m2l_tcb_units(l);
        const bool shallow = tc_blocks == 1 || (tc_blocks == 0 && blocks >= kTcbShallowMinUnits);
        if (use_tc && tc_blocks != 2) {
            for (int i = 0; i < ni; ++i) {
                InstDesc &d = pl.inst[i];
                for (int l = 2; l <= d.L; ++l) {
                    if (((d.tc_levels >> l) & 1u) || !m2l_tcb_supported(d.p, l)) continue;
                    if (l < 8 && !shallow) continue;
                    d.tc_unit0[l] = base + pl.m2l_tcb.nblocks;
                    d.tcb_levels |= 1u << l;
                    add_task(pl.m2l_tcb, i, l, m2l_tcb_units(l), 1);
                    pl.tcb_pmax = std::max(pl.tcb_pmax, d.p);
                }
            }
        }
        base += pl.m2l_tcb.nblocks;
        for (int cls = 0; cls < Plan::kTileClasses; ++cls) {
            TaskRange &tr = pl.m2l_tile[cls];
            for (int i = 0; i < ni; ++i) {
                InstDesc &d = pl.inst[i];
                if (!m2l_tile_supported(d.p) || tile_class(d.p) != cls) continue;
                for (int l = 2; l <= d.L; ++l) {
                    if (((d.tc_levels | d.tcb_levels) >> l) & 1u) continue;
                    d.tc_unit0[l] = base + tr.nblocks;
                    add_task(tr, i, l, m2l_tile_units(l), 1);
                    pl.tile_pmax[cls] = std::max(pl.tile_pmax[cls], d.p);
                }
            }
            base += tr.nblocks;
        }
    }
    // M2M rounds: round r computes level L_i - 1 - r (>= 2) of every instance.
    for (int r = 0; r + 3 <= Lmax; ++r) {
        TaskRange tr;
        for (int i = 0; i < ni; ++i) {
            const int l = pl.inst[i].L - 1 - r;
            if (l >= 2) add_task(tr, i, l, (int64_t(1) << (2 * l)) * pl.inst[i].p, EXP_THREADS);
        }
        if (tr.count) pl.m2m.push_back(tr);
    }
    // L2L rounds: round r translates level 2 + r into level 3 + r.
    for (int r = 0; r + 3 <= Lmax; ++r) {
        TaskRange tr;
        for (int i = 0; i < ni; ++i) {
            const int l = 3 + r;
            if (l <= pl.inst[i].L)
                add_task(tr, i, l, (int64_t(1) << (2 * l)) * pl.inst[i].p, EXP_THREADS);
        }
        if (tr.count) pl.l2l.push_back(tr);
    }
    pl.items_cap = items_cap;
    flatten_tasks(pl);
    return PETFMM_OK;
}

// Operator tables (device pointers) of every instance's p.
int attach_tables(petfmm_ctx *c, Plan &pl) {
    for (InstDesc &d : pl.inst) {
        int err = PETFMM_OK;
        OpTables *t = get_tables(c, d.p, c->kernel, &err);
        if (!t) return err;
        if (c->precision == PETFMM_FP64) {
            d.t_m2m = t->m2m64; d.t_l2l = t->l2l64; d.t_m2l = t->m2l64;
        } else {
            d.t_m2m = t->m2m32; d.t_l2l = t->l2l32; d.t_m2l = t->m2l32;
            d.t_m2l_tc = t->m2l_tc;
            d.t_m2l_tcb = t->m2l_tcb;
        }
    }
    return PETFMM_OK;
}

// Uploads InstDesc[] followed by Task[] to c->plan_dev (skipped when equal to
// the previous upload).
int upload_plan(petfmm_ctx *c, const Plan &pl) {
    const size_t ib = pl.inst.size() * sizeof(InstDesc);
    const size_t tb = pl.tasks.size() * sizeof(Task);
    const size_t total = align_up(ib) + tb;
    std::vector<unsigned char> blob(total, 0);
    std::memcpy(blob.data(), pl.inst.data(), ib);
    if (tb) std::memcpy(blob.data() + align_up(ib), pl.tasks.data(), tb);
    if (blob == c->last_upload && c->plan_dev.p) return PETFMM_OK;
    int rc = ensure(c->plan_dev, total, c->stream);
    if (rc) return rc;
    if (c->pinned_cap < total) {
        if (c->pinned) {
            cudaEventSynchronize(c->upload_done);
            cudaFreeHost(c->pinned);
            c->pinned = nullptr;
        }
        if (cudaMallocHost(&c->pinned, total) != cudaSuccess) {
            cudaGetLastError();
            c->pinned = nullptr;
            c->pinned_cap = 0;
            return PETFMM_ENOMEM;
        }
        c->pinned_cap = total;
        c->upload_pending = false;
    }
    if (c->upload_pending) cudaEventSynchronize(c->upload_done);
    std::memcpy(c->pinned, blob.data(), total);
    cudaError_t e = cudaMemcpyAsync(c->plan_dev.p, c->pinned, total, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    cudaEventRecord(c->upload_done, c->stream);
    c->upload_pending = true;
    c->last_upload.swap(blob);
    return PETFMM_OK;
}

#define PF_TRY(expr)                         \
    do {                                     \
        int rc_ = (expr);                    \
        if (rc_ != PETFMM_OK) return rc_;    \
    } while (0)
#define PF_CUDA(expr) PF_TRY(cuda_status(expr))

// FNV-1a over everything a kernel argument of the launch sequence depends on.
struct KeyHash {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
    template <typename T> void put(const T &v) { add(&v, sizeof(v)); }
};

uint64_t graph_key(const petfmm_ctx *c, const Plan &pl, int grid) {
    KeyHash k;
    if (!pl.tasks.empty()) k.add(pl.tasks.data(), pl.tasks.size() * sizeof(Task));
    auto range = [&](const TaskRange &r) { k.put(r.first); k.put(r.count); k.put(r.nblocks); };
    for (const TaskRange *r : {&pl.outscatter, &pl.start, &pl.particles, &pl.leaves_p2m, &pl.leaves_wl,
                               &pl.m2l, &pl.m2l_tc, &pl.m2l_tcb, &pl.m2l_log})
        range(*r);
    for (const TaskRange &r : pl.m2l_tile) range(r);
    for (int cls = 0; cls < Plan::kTileClasses; ++cls) k.put(pl.tile_pmax[cls]);
    for (const TaskRange &r : pl.m2m) range(r);
    for (const TaskRange &r : pl.l2l) range(r);
    k.put(pl.m2m.size()); k.put(pl.l2l.size());
    k.put(pl.N); k.put(pl.nleaves); k.put(pl.nstart); k.put(pl.ncoef); k.put(pl.items_cap);
    k.put(pl.nbits); k.put(pl.pmax); k.put(pl.deg); k.put(pl.general);
    k.put(pl.tc_smem); k.put(pl.tcb_pmax); k.put(grid);
    k.put(c->precision); k.put(c->dtype); k.put(c->timing); k.put(c->p2p_mode); k.put(c->poison);
    k.put(c->tc_dense_pct); k.put(c->spin_limit); k.put(c->p2p_pairs); k.put(c->kernel);
    k.put(c->tc_blocks); k.put(c->tc_pipe); k.put(c->overlap);
    for (const DevBuf *b : {&c->keysA, &c->keysB, &c->valsA, &c->valsB, &c->hist, &c->scratch,
                            &c->start, &c->xs, &c->ys, &c->gs, &c->rec, &c->me, &c->le, &c->cnt,
                            &c->off, &c->items, &c->ctrl, &c->plan_dev, &c->busy, &c->ucount,
                            &c->recu, &c->occ, &c->items_u, &c->ikA, &c->ikB, &c->ivA, &c->ivB,
                            &c->ihist, &c->own, &c->part, &c->pitems, &c->pxtra, &c->pxs,
                            &c->ustage})
        k.put(b->p);
    return k.h;
}

void stage_mark_on(petfmm_ctx *c, int stage, cudaStream_t s) {
    if (!c->timing) return;
    // inside a capture the record must become an event node of the graph
    if (c->capturing)
        cudaEventRecordWithFlags(c->ev[stage], s, cudaEventRecordExternal);
    else
        cudaEventRecord(c->ev[stage], s);
}

void stage_mark(petfmm_ctx *c, int stage) { stage_mark_on(c, stage, c->stream); }

// blobs of one instance from which the final pass stages FP32 results
// (2 x 4 B x n > 64 MB)
constexpr int64_t kUnsortStageMin = int64_t(8) << 20;

int run(petfmm_ctx *c, const std::vector<Problem> &probs) {
    Plan &pl = c->plan;
    PF_TRY(build_plan(c->precision, c->kernel, c->m2l_tc, c->tc_blocks, c->tc_segmax, c->near_tol,
                      probs, pl));
    PF_TRY(attach_tables(c, pl));
    cudaStream_t st = c->stream;  // the launch sequence's stream (a capture swaps it)
    const bool mixed = c->precision == PETFMM_MIXED;
    const int64_t N = pl.N;
    // buffers
    PF_TRY(ensure(c->ctrl, CTRL_WORDS * sizeof(uint32_t), st));
    if (c->evaluations == 0 && c->launches == 0) PF_CUDA(cudaMemsetAsync(c->ctrl.p, 0, CTRL_WORDS * 4, st));
    PF_TRY(upload_plan(c, pl));
    if (N == 0) {
        c->evaluations++;
        c->ev_recorded = false;
        return PETFMM_OK;
    }
    PF_TRY(ensure(c->keysA, N * 4, st));
    PF_TRY(ensure(c->keysB, N * 4, st));
    PF_TRY(ensure(c->valsA, N * 4, st));
    PF_TRY(ensure(c->valsB, N * 4, st));
    PF_TRY(ensure(c->hist, size_t(radix_scratch_words(N)) * 4, st));
    // pairwise near field (mixed path): at most 4 forward neighbours per leaf,
    // a pair cut into at most ceil(na / 128) pieces, and the leaf's own pairs
    // (the pairwise near field is the vortex kernel's)
    const bool pairs = mixed && c->p2p_pairs && c->kernel == KERNEL_VORTEX;
    const int64_t pair_cap =
        pairs ? 5 * std::min<int64_t>(pl.nleaves, N) + 4 * (N / 128) + 1 : 0;
    const int64_t order_cap = std::max<int64_t>(pl.items_cap, pair_cap);
    const int64_t scan_n = pl.nleaves;
    PF_TRY(ensure(c->scratch, size_t(scan_scratch_words(scan_n)) * 4, st));
    PF_TRY(ensure(c->start, size_t(pl.nstart) * 4, st));
    if (mixed) {
        PF_TRY(ensure(c->rec, size_t(N) * sizeof(float4), st));
        PF_TRY(ensure(c->recu, size_t(N) * sizeof(float4), st));
        PF_TRY(ensure(c->me, size_t(pl.ncoef) * sizeof(float2), st));
        PF_TRY(ensure(c->le, size_t(pl.ncoef) * sizeof(float2), st));
    } else {
        PF_TRY(ensure(c->xs, size_t(N) * 8, st));
        PF_TRY(ensure(c->ys, size_t(N) * 8, st));
        PF_TRY(ensure(c->gs, size_t(N) * 8, st));
        PF_TRY(ensure(c->me, size_t(pl.ncoef) * sizeof(double2), st));
        PF_TRY(ensure(c->le, size_t(pl.ncoef) * sizeof(double2), st));
    }
    PF_TRY(ensure(c->cnt, size_t(pl.nleaves) * 4, st));
    PF_TRY(ensure(c->occ, size_t(pl.nleaves) * sizeof(uint2), st));
    PF_TRY(ensure(c->off, size_t(pl.nleaves) * 4, st));
    PF_TRY(ensure(c->items, size_t(pl.items_cap) * sizeof(uint4), st));
    PF_TRY(ensure(c->ucount,
                  size_t(pl.m2l_tc.nblocks + pl.m2l_tcb.nblocks + pl.tile_blocks()) * sizeof(uint32_t),
                  st));
    if (mixed) PF_TRY(ensure(c->own, size_t(N) * sizeof(float2), st));
    if (pairs) {
        PF_TRY(ensure(c->part, size_t(9) * N * sizeof(float2), st));
        PF_TRY(ensure(c->pitems, size_t(pair_cap) * sizeof(uint4), st));
        PF_TRY(ensure(c->pxtra, size_t(7) * pl.nleaves * sizeof(uint32_t), st));
        PF_TRY(ensure(c->pxs, size_t(N) * sizeof(float2), st));
    }
    PairBufs pb{};
    if (mixed) pb.own = static_cast<float2 *>(c->own.p);
    if (pairs) {
        pb.part = static_cast<float2 *>(c->part.p);
        pb.nslot = N;
        pb.xcnt = static_cast<uint32_t *>(c->pxtra.p);
        pb.xoff = pb.xcnt + pl.nleaves;
        pb.xtab = pb.xoff + pl.nleaves;
        pb.lflags = pb.xtab + 4 * pl.nleaves;
        pb.xs = static_cast<float2 *>(c->pxs.p);
        pb.xcap = N;  // scratch of split pairs; more wanted: no pair is split
    }
    P2POrder order{}, porder{};
    if (c->p2p_mode == 0) {
        const size_t cap = size_t(order_cap);
        PF_TRY(ensure(c->items_u, cap * sizeof(uint4), st));
        PF_TRY(ensure(c->ikA, cap * 4, st));
        PF_TRY(ensure(c->ikB, cap * 4, st));
        PF_TRY(ensure(c->ivA, cap * 4, st));
        PF_TRY(ensure(c->ivB, cap * 4, st));
        PF_TRY(ensure(c->ihist, size_t(radix_scratch_words(order_cap)) * 4, st));
        order.cap = pl.items_cap;
        order.items_unsorted = static_cast<uint4 *>(c->items_u.p);
        order.kA = static_cast<uint32_t *>(c->ikA.p);
        order.kB = static_cast<uint32_t *>(c->ikB.p);
        order.vA = static_cast<uint32_t *>(c->ivA.p);
        order.vB = static_cast<uint32_t *>(c->ivB.p);
        order.hist = static_cast<uint32_t *>(c->ihist.p);
        porder = order;
        porder.cap = pair_cap;
    }
    const bool lap = c->kernel == KERNEL_LAPLACE;
    const int grid = p2p_grid(mixed, pl.deg, pl.general, lap ? 1 : 0);
    if (grid <= 0) return PETFMM_EINVAL;
    const int pgrid = pairs ? p2p_pairs_grid(pl.deg, pl.general) : 0;
    if (pairs && pgrid <= 0) return PETFMM_EINVAL;
    // busy times: the directed kernel's CTAs, then the pair kernel's
    c->p2p_grid = grid;
    c->pairs_grid = pgrid;
    unsigned long long *busy = nullptr, *pbusy = nullptr;
    if (c->timing) {
        PF_TRY(ensure(c->busy, size_t(grid + pgrid) * 8 * 2 * sizeof(unsigned long long), st));
        busy = static_cast<unsigned long long *>(c->busy.p);
        if (pairs) pbusy = busy + size_t(grid) * 8 * 2;
    }

    const InstDesc *dinst = static_cast<const InstDesc *>(c->plan_dev.p);
    const Task *dtask = reinterpret_cast<const Task *>(static_cast<unsigned char *>(c->plan_dev.p) +
                                                       align_up(pl.inst.size() * sizeof(InstDesc)));
    uint32_t *ctrl = static_cast<uint32_t *>(c->ctrl.p);
    uint32_t *kA = static_cast<uint32_t *>(c->keysA.p), *kB = static_cast<uint32_t *>(c->keysB.p);
    uint32_t *vA = static_cast<uint32_t *>(c->valsA.p), *vB = static_cast<uint32_t *>(c->valsB.p);
    uint32_t *start = static_cast<uint32_t *>(c->start.p);
    uint32_t *scratch = static_cast<uint32_t *>(c->scratch.p);
    const int f32 = c->dtype == PETFMM_F32;
    uint64_t *lc = &c->launches;

    // the launch sequence (the only part of an evaluation a graph replays)
    // FP32 outputs larger than half the L2: the final pass stages them in
    // sorted order, then one scatter per component (see k_unsort_f32)
    float *stage = nullptr;
    int64_t nmax = 0;  // an instance's scatter stays within its own arrays
    for (const InstDesc &d : pl.inst) nmax = std::max(nmax, d.n);
    if (mixed && f32 && nmax >= kUnsortStageMin) {
        PF_TRY(ensure(c->ustage, size_t(2) * N * sizeof(float), st));
        stage = static_cast<float *>(c->ustage.p);
    }
    auto launch_all = [&]() -> int {
    if (c->poison) {
        const size_t es = mixed ? sizeof(float2) : sizeof(double2);
        PF_CUDA(cudaMemsetAsync(c->me.p, 0xff, size_t(pl.ncoef) * es, st));
        PF_CUDA(cudaMemsetAsync(c->le.p, 0xff, size_t(pl.ncoef) * es, st));
    }
    // per-evaluation control words (the status word survives until sync)
    PF_CUDA(cudaMemsetAsync(ctrl + 1, 0, (CTRL_WORDS - 1) * 4, st));

    stage_mark(c, PETFMM_STAGE_MORTON);
    float4 *recu = mixed ? static_cast<float4 *>(c->recu.p) : nullptr;
    const float4 *srec = mixed ? static_cast<const float4 *>(c->rec.p) : nullptr;  // sorted
    PF_CUDA(launch_morton(dtask + pl.particles.first, pl.particles.count, pl.particles.nblocks,
                          dinst, f32, kA, recu, reinterpret_cast<int *>(ctrl + CTRL_STATUS), st,
                          lc));
    stage_mark(c, PETFMM_STAGE_SORT);
    bool in_first = true;
    PF_CUDA(radix_sort(kA, vA, kB, vB, N, pl.nbits, static_cast<uint32_t *>(c->hist.p), &in_first,
                       st, lc));
    c->sorted_in_first = in_first;
    const uint32_t *skeys = in_first ? kA : kB;
    const uint32_t *perm = in_first ? vA : vB;
    PF_CUDA(launch_leaf_start(dtask + pl.start.first, pl.start.count, pl.start.nblocks, dinst, skeys,
                              start, st, lc));
    // The record gather and the expansion chain (P2M, M2M, M2L, L2L) run on
    // a second stream on the mixed path: the near-field work lists need only
    // the leaf starts and run beside the gather, the pair and directed
    // kernels wait for the gathered blobs only, and the final pass joins
    // the two streams (PETFMM_OPT_OVERLAP).
    cudaStream_t xs = st;
    const bool fork = mixed && c->overlap;
    if (fork) {
        PF_CUDA(cudaEventRecord(c->ev_fork, st));
        PF_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
        xs = c->aux;
    }
    stage_mark_on(c, PETFMM_STAGE_GATHER, xs);
    if (mixed)
        PF_CUDA(launch_gather_mixed(recu, perm, static_cast<float4 *>(c->rec.p), N, xs, lc));
    else
        PF_CUDA(launch_gather_f64(dtask + pl.particles.first, pl.particles.count,
                                  pl.particles.nblocks, dinst, f32, perm,
                                  static_cast<double *>(c->xs.p), static_cast<double *>(c->ys.p),
                                  static_cast<double *>(c->gs.p), st, lc));
    if (fork) PF_CUDA(cudaEventRecord(c->ev_gathered, xs));
    stage_mark_on(c, PETFMM_STAGE_P2M, xs);
    uint2 *occ = static_cast<uint2 *>(c->occ.p);
    PF_CUDA(launch_occ_list(dtask + pl.leaves_p2m.first, pl.leaves_p2m.count, pl.leaves_p2m.nblocks,
                            dinst, start, occ, ctrl, xs, lc));
    if (mixed)
        PF_CUDA(launch_p2m<float>(occ, ctrl, pl.nleaves, dinst, pl.pmax, start, nullptr, nullptr,
                                  nullptr, srec,
                                  static_cast<float2 *>(c->me.p), xs, lc));
    else
        PF_CUDA(launch_p2m<double>(occ, ctrl, pl.nleaves, dinst, pl.pmax, start,
                                   static_cast<const double *>(c->xs.p),
                                   static_cast<const double *>(c->ys.p),
                                   static_cast<const double *>(c->gs.p), nullptr,
                                   static_cast<double2 *>(c->me.p), xs, lc));
    stage_mark_on(c, PETFMM_STAGE_M2M, xs);
    for (const TaskRange &tr : pl.m2m) {
        if (mixed)
            PF_CUDA(launch_m2m<float>(dtask + tr.first, tr.count, tr.nblocks, dinst, start,
                                      static_cast<float2 *>(c->me.p), xs, lc));
        else
            PF_CUDA(launch_m2m<double>(dtask + tr.first, tr.count, tr.nblocks, dinst, start,
                                       static_cast<double2 *>(c->me.p), xs, lc));
    }
    stage_mark_on(c, PETFMM_STAGE_M2L, xs);
    uint32_t *ucount = nullptr;
    if (pl.m2l_tc.count || pl.m2l_tcb.count || pl.tile_blocks()) {
        ucount = static_cast<uint32_t *>(c->ucount.p);
        if (pl.m2l_tc.count)
            PF_CUDA(launch_tc_unit_count(dtask + pl.m2l_tc.first, pl.m2l_tc.count,
                                         pl.m2l_tc.nblocks, dinst, start, ucount, xs, lc));
        if (pl.m2l_tcb.count)
            PF_CUDA(launch_tc_unit_count(dtask + pl.m2l_tcb.first, pl.m2l_tcb.count,
                                         pl.m2l_tcb.nblocks, dinst, start,
                                         ucount + pl.m2l_tc.nblocks, xs, lc));
        int64_t base = pl.m2l_tc.nblocks + pl.m2l_tcb.nblocks;
        for (const TaskRange &tr : pl.m2l_tile) {
            if (tr.count)
                PF_CUDA(launch_tc_unit_count(dtask + tr.first, tr.count, tr.nblocks, dinst, start,
                                             ucount + base, xs, lc));
            base += tr.nblocks;
        }
    }
    if (pl.m2l.count) {
        if (mixed)
            PF_CUDA(launch_m2l<float>(dtask + pl.m2l.first, pl.m2l.count, pl.m2l.nblocks, dinst,
                                      start, static_cast<const float2 *>(c->me.p),
                                      static_cast<float2 *>(c->le.p), ucount, c->tc_dense_pct,
                                      xs, lc));
        else
            PF_CUDA(launch_m2l<double>(dtask + pl.m2l.first, pl.m2l.count, pl.m2l.nblocks, dinst,
                                       start, static_cast<const double2 *>(c->me.p),
                                       static_cast<double2 *>(c->le.p), nullptr, 0, xs, lc));
    }
    if (pl.m2l_tc.count) {
        // spin_limit < 0: zero-iteration budget (tests the timeout report)
        const long long spin = c->spin_limit > 0 ? c->spin_limit : c->spin_limit < 0 ? 0 : (1LL << 26);
        PF_CUDA(launch_m2l_tc(dtask + pl.m2l_tc.first, pl.m2l_tc.count, pl.m2l_tc.nblocks, dinst,
                              start, static_cast<const float2 *>(c->me.p),
                              static_cast<float2 *>(c->le.p), ucount, c->tc_dense_pct,
                              pl.tc_smem, spin, reinterpret_cast<int *>(ctrl + CTRL_STATUS), xs,
                              lc));
    }
    if (pl.m2l_tcb.count) {
        const long long spin = c->spin_limit > 0 ? c->spin_limit : c->spin_limit < 0 ? 0 : (1LL << 26);
        PF_CUDA(launch_m2l_tcb(dtask + pl.m2l_tcb.first, pl.m2l_tcb.count, pl.m2l_tcb.nblocks,
                               dinst, start, static_cast<const float2 *>(c->me.p),
                               static_cast<float2 *>(c->le.p), ucount + pl.m2l_tc.nblocks,
                               c->tc_dense_pct, pl.tcb_pmax, spin, c->tc_pipe,
                               reinterpret_cast<int *>(ctrl + CTRL_STATUS), xs, lc));
    }
    {
        int64_t base = pl.m2l_tc.nblocks + pl.m2l_tcb.nblocks;
        for (int cls = 0; cls < Plan::kTileClasses; ++cls) {
            const TaskRange &tr = pl.m2l_tile[cls];
            if (tr.count)
                PF_CUDA(launch_m2l_tile(dtask + tr.first, tr.count, tr.nblocks, pl.tile_pmax[cls],
                                        dinst, start, static_cast<const float2 *>(c->me.p),
                                        static_cast<float2 *>(c->le.p), ucount + base,
                                        c->tc_dense_pct, xs, lc));
            base += tr.nblocks;
        }
    }
    if (pl.m2l_log.count) {
        if (mixed)
            PF_CUDA(launch_m2l_logterm<float>(dtask + pl.m2l_log.first, pl.m2l_log.count,
                                              pl.m2l_log.nblocks, dinst, start,
                                              static_cast<const float2 *>(c->me.p),
                                              static_cast<float2 *>(c->le.p), xs, lc));
        else
            PF_CUDA(launch_m2l_logterm<double>(dtask + pl.m2l_log.first, pl.m2l_log.count,
                                               pl.m2l_log.nblocks, dinst, start,
                                               static_cast<const double2 *>(c->me.p),
                                               static_cast<double2 *>(c->le.p), xs, lc));
    }
    stage_mark_on(c, PETFMM_STAGE_L2L, xs);
    for (const TaskRange &tr : pl.l2l) {
        if (mixed)
            PF_CUDA(launch_l2l<float>(dtask + tr.first, tr.count, tr.nblocks, dinst, start,
                                      static_cast<float2 *>(c->le.p), xs, lc));
        else
            PF_CUDA(launch_l2l<double>(dtask + tr.first, tr.count, tr.nblocks, dinst, start,
                                       static_cast<double2 *>(c->le.p), xs, lc));
    }
    stage_mark_on(c, PETFMM_STAGE_COUNT + 1, xs);  // end of the L2L stage
    if (fork) PF_CUDA(cudaEventRecord(c->ev_join, xs));
    stage_mark(c, PETFMM_STAGE_WORKLIST);
    const int tpi = mixed ? P2P_TPI_MIXED : P2P_TPI_F64;
    PF_CUDA(launch_p2p_worklist(dtask + pl.leaves_wl.first, pl.leaves_wl.count, pl.leaves_wl.nblocks,
                                dinst, start, pl.nleaves, tpi, pairs ? 1 : 0,
                                static_cast<uint32_t *>(c->cnt.p),
                                static_cast<uint32_t *>(c->off.p), scratch,
                                static_cast<uint4 *>(c->items.p), ctrl,
                                c->p2p_mode == 0 ? &order : nullptr, st, lc));
    if (pairs)
        PF_CUDA(launch_pair_worklist(dtask + pl.leaves_wl.first, pl.leaves_wl.count,
                                     pl.leaves_wl.nblocks, dinst, start, pl.nleaves,
                                     static_cast<uint32_t *>(c->cnt.p),
                                     static_cast<uint32_t *>(c->off.p), scratch,
                                     static_cast<uint4 *>(c->pitems.p), ctrl,
                                     c->p2p_mode == 0 ? &porder : nullptr, pb, st, lc));
    if (fork) PF_CUDA(cudaStreamWaitEvent(st, c->ev_gathered, 0));
    stage_mark(c, PETFMM_STAGE_PAIRS);
    // pairwise mode: the neighbouring leaves pairwise
    if (pairs)
        PF_CUDA(launch_p2p_pairs(pgrid, pl.deg, pl.general, static_cast<const uint4 *>(c->pitems.p),
                                 ctrl, dinst, start, srec, pb,
                                 pbusy, st, lc));
    stage_mark(c, PETFMM_STAGE_P2P);
    if (mixed) {
        // near sums of the own leaf and the directed neighbours, then far
        // field and the sum
        PF_CUDA(launch_p2p_mixed(grid, pl.deg, pl.general, static_cast<const uint4 *>(c->items.p),
                                 ctrl, dinst, start, srec, pb.own,
                                 pairs, lap ? 1 : 0, busy, st, lc));
        if (fork) PF_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
        stage_mark(c, PETFMM_STAGE_FINAL);
        PF_CUDA(launch_p2p_final(dtask + pl.particles.first, pl.particles.count,
                                 pl.particles.nblocks, dinst, start, skeys, srec,
                                 static_cast<const float2 *>(c->le.p), pb, f32, perm, stage, N,
                                 dtask + pl.outscatter.first, pl.outscatter.count,
                                 pl.outscatter.nblocks, ctrl, N, st, lc));
    } else
        PF_CUDA(launch_p2p_f64(grid, static_cast<const uint4 *>(c->items.p), ctrl, dinst, start,
                               static_cast<const double *>(c->xs.p),
                               static_cast<const double *>(c->ys.p),
                               static_cast<const double *>(c->gs.p), perm,
                               static_cast<const double2 *>(c->le.p), f32, busy, st, lc));
    if (!mixed) stage_mark(c, PETFMM_STAGE_FINAL);
    stage_mark(c, PETFMM_STAGE_COUNT);
    return PETFMM_OK;
    };

    if (!c->use_graph) {
        PF_TRY(launch_all());
    } else {
        // Every kernel argument is a function of the launch shape, the
        // library's buffers and the options (the plan itself, including the
        // caller's arrays, is read from device memory): replay the captured
        // graph while they are unchanged, capture a new one otherwise.
        const uint64_t key = graph_key(c, pl, grid);
        if (!(c->gexec && c->gkey == key)) {
            if (c->gexec) {
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
            if (!c->cap_stream &&
                cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                c->cap_stream = nullptr;
                return PETFMM_ECUDA;
            }
            const cudaStream_t user = c->stream;
            PF_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            c->stream = st = c->cap_stream;
            c->capturing = true;
            const uint64_t l0 = c->launches;
            const int rc = launch_all();
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
            c->capturing = false;
            c->stream = st = user;
            if (rc != PETFMM_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                c->launches = l0;
                return rc != PETFMM_OK ? rc : PETFMM_ECUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                cudaGetLastError();
                c->gexec = nullptr;
                c->launches = l0;
                return PETFMM_ECUDA;
            }
            c->gkey = key;
            c->glaunches = c->launches - l0;
            c->launches = l0;
        }
        PF_CUDA(cudaGraphLaunch(c->gexec, st));
        c->launches += c->glaunches;
    }
    c->ev_recorded = c->timing;
    c->evaluations++;
    return PETFMM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int petfmm_version(void) { return 1; }

const char *petfmm_strerror(int code) {
    switch (code) {
        case PETFMM_OK: return "ok";
        case PETFMM_EINVAL: return "invalid argument";
        case PETFMM_ENOMEM: return "out of memory";
        case PETFMM_EDOMAIN: return "particle outside the domain";
        case PETFMM_ECUDA: return "CUDA error";
        case PETFMM_ETIMEOUT: return "device wait timed out";
        case PETFMM_EBUSY: return "server busy";
        case PETFMM_ENOTREADY: return "not ready";
        default: return "unknown status";
    }
}

int petfmm_create(const petfmm_domain *dom, int levels, int order, double sigma, int precision,
                  int dtype, void *cuda_stream, petfmm_ctx **out) {
    if (!out) return PETFMM_EINVAL;
    *out = nullptr;
    int rc = check_problem(dom, levels, order, sigma);
    if (rc) return rc;
    if (precision != PETFMM_FP64 && precision != PETFMM_MIXED) return PETFMM_EINVAL;
    if (dtype != PETFMM_F64 && dtype != PETFMM_F32) return PETFMM_EINVAL;
    petfmm_ctx *c = new (std::nothrow) petfmm_ctx();
    if (!c) return PETFMM_ENOMEM;
    c->dom = *dom;
    c->L = levels;
    c->p = order;
    c->sigma = sigma;
    c->precision = precision;
    c->dtype = dtype;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PETFMM_ECUDA;
    }
    if (cudaEventCreateWithFlags(&c->upload_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PETFMM_ECUDA;
    }
    for (auto &e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            petfmm_destroy(c);
            return PETFMM_ECUDA;
        }
    }
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_gathered, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        petfmm_destroy(c);
        return PETFMM_ECUDA;
    }
    int err = PETFMM_OK;
    if (!get_tables(c, order, KERNEL_VORTEX, &err)) {
        petfmm_destroy(c);
        return err;
    }
    *out = c;
    return PETFMM_OK;
}

int petfmm_destroy(petfmm_ctx *c) {
    if (!c) return PETFMM_EINVAL;
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->keysA, &c->keysB, &c->valsA, &c->valsB, &c->hist, &c->scratch,
                      &c->start, &c->xs, &c->ys, &c->gs, &c->rec, &c->me, &c->le, &c->cnt,
                      &c->off, &c->items, &c->ctrl, &c->plan_dev, &c->busy, &c->ucount, &c->recu, &c->occ, &c->items_u, &c->ikA, &c->ikB, &c->ivA, &c->ivB, &c->ihist, &c->own, &c->part, &c->pitems, &c->pxtra, &c->pxs, &c->ustage, &c->hx, &c->hy,
                      &c->hg, &c->hu, &c->hv};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto &kv : c->tables) free_op_tables(&kv.second);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->upload_done) cudaEventDestroy(c->upload_done);
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaStreamDestroy(c->aux);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_gathered) cudaEventDestroy(c->ev_gathered);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete c;
    return PETFMM_OK;
}

int petfmm_evaluate(petfmm_ctx *c, int64_t n, const void *x, const void *y, const void *gamma,
                    void *u, void *v) {
    if (!c || n < 0) return PETFMM_EINVAL;
    if (n > 0 && (!x || !y || !gamma || !u || !v)) return PETFMM_EINVAL;
    std::vector<Problem> probs(1);
    probs[0] = Problem{c->dom, c->L, c->p, c->sigma, n, x, y, gamma, u, v};
    return run(c, probs);
}

int petfmm_evaluate_host(petfmm_ctx *c, int64_t n, const void *x, const void *y, const void *gamma,
                         void *u, void *v) {
    if (!c || n < 0) return PETFMM_EINVAL;
    if (n > 0 && (!x || !y || !gamma || !u || !v)) return PETFMM_EINVAL;
    const size_t es = c->dtype == PETFMM_F32 ? 4 : 8;
    const size_t bytes = size_t(n) * es;
    cudaStream_t st = c->stream;
    PF_TRY(ensure(c->hx, bytes, st));
    PF_TRY(ensure(c->hy, bytes, st));
    PF_TRY(ensure(c->hg, bytes, st));
    PF_TRY(ensure(c->hu, bytes, st));
    PF_TRY(ensure(c->hv, bytes, st));
    if (n > 0) {
        PF_CUDA(cudaMemcpyAsync(c->hx.p, x, bytes, cudaMemcpyHostToDevice, st));
        PF_CUDA(cudaMemcpyAsync(c->hy.p, y, bytes, cudaMemcpyHostToDevice, st));
        PF_CUDA(cudaMemcpyAsync(c->hg.p, gamma, bytes, cudaMemcpyHostToDevice, st));
    }
    int rc = petfmm_evaluate(c, n, c->hx.p, c->hy.p, c->hg.p, c->hu.p, c->hv.p);
    if (rc) return rc;
    if (n > 0) {
        PF_CUDA(cudaMemcpyAsync(u, c->hu.p, bytes, cudaMemcpyDeviceToHost, st));
        PF_CUDA(cudaMemcpyAsync(v, c->hv.p, bytes, cudaMemcpyDeviceToHost, st));
    }
    return petfmm_sync(c);
}

int petfmm_sync(petfmm_ctx *c) {
    if (!c) return PETFMM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return PETFMM_ECUDA;
    if (!c->ctrl.p) return PETFMM_OK;
    int status = 0;
    e = cudaMemcpy(&status, c->ctrl.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return PETFMM_ECUDA;
    if (status) {
        e = cudaMemset(c->ctrl.p, 0, sizeof(int));
        if (e != cudaSuccess) return PETFMM_ECUDA;
    }
    return status;
}

static int problems_from(int n_inst, const petfmm_instance *inst, std::vector<Problem> &probs,
                         const std::vector<petfmm_level_rule> *rules = nullptr) {
    probs.resize(static_cast<size_t>(n_inst));
    for (int i = 0; i < n_inst; ++i) {
        const petfmm_instance &s = inst[i];
        int L = s.levels;
        if (L <= 0) {
            L = rules && !rules->empty()
                    ? petfmm_rule_levels(rules->data(), int(rules->size()), s.n, s.order, s.sigma,
                                         &s.domain)
                    : petfmm_choose_levels(s.n, s.order, s.sigma, &s.domain);
            if (L < 0) return L;
        }
        int rc = check_problem(&s.domain, L, s.order, s.sigma);
        if (rc) return rc;
        if (s.n < 0 || (s.n > 0 && (!s.x || !s.y || !s.gamma || !s.u || !s.v))) return PETFMM_EINVAL;
        probs[i] = Problem{s.domain, L, s.order, s.sigma, s.n, s.x, s.y, s.gamma, s.u, s.v};
    }
    return PETFMM_OK;
}

int petfmm_evaluate_batch(petfmm_ctx *c, int n_inst, const petfmm_instance *inst) {
    if (!c || n_inst < 0 || (n_inst > 0 && !inst)) return PETFMM_EINVAL;
    std::vector<Problem> probs;
    int rc = problems_from(n_inst, inst, probs, &c->rules);
    if (rc) return rc;
    return run(c, probs);
}

// ---------------------------------------------------------------------------
// Autotuner (petfmm_tune_batch): the work model seeds L, the GPU decides.
// ---------------------------------------------------------------------------
namespace {

int floor_log2(int64_t n) {
    int e = 0;
    while (n > 1) {
        n >>= 1;
        ++e;
    }
    return e;
}

// fraction by which a candidate must beat the work model's choice (or the
// entry options) to replace it
constexpr float kTuneMargin = 0.02f;

// Median of `reps` timed evaluations of the problems (after one warm-up,
// which also captures the graph of a new launch shape), CUDA events on the
// context's stream.
int time_batch(petfmm_ctx *c, const std::vector<Problem> &probs, int reps, float *ms, int *nevals) {
    int rc = run(c, probs);
    if (rc) return rc;
    ++*nevals;
    if ((rc = petfmm_sync(c))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return PETFMM_ECUDA;
    }
    std::vector<float> t;
    for (int r = 0; r < reps && rc == PETFMM_OK; ++r) {
        cudaEventRecord(e0, c->stream);
        rc = run(c, probs);
        cudaEventRecord(e1, c->stream);
        if (rc) break;
        ++*nevals;
        if ((rc = petfmm_sync(c))) break;
        float x = 0.f;
        if (cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            rc = PETFMM_ECUDA;
            break;
        }
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms = t.empty() ? 0.f : t[t.size() / 2];
    return PETFMM_OK;
}

}  // namespace

int petfmm_rule_levels(const petfmm_level_rule *rules, int nrules, int64_t n, int order,
                       double sigma, const petfmm_domain *dom) {
    const int Lm = petfmm_choose_levels(n, order, sigma, dom);
    if (Lm < 0 || nrules <= 0 || !rules) return Lm;
    const int e = floor_log2(n);
    const double rmin = sigma * std::sqrt(2.0 * std::log(1e8));
    for (int i = 0; i < nrules; ++i) {
        const petfmm_level_rule &r = rules[i];
        if (r.order != order || r.log2n != e) continue;
        if (r.levels < 1 || r.levels > MAX_L) return Lm;
        // the kernel-substitution guard of petfmm_choose_levels
        if (dom->width / std::ldexp(1.0, r.levels) < rmin) return Lm;
        return r.levels;
    }
    return Lm;
}

int petfmm_set_level_rules(petfmm_ctx *c, const petfmm_level_rule *rules, int nrules) {
    if (!c || nrules < 0 || (nrules > 0 && !rules)) return PETFMM_EINVAL;
    for (int i = 0; i < nrules; ++i)
        if (rules[i].order < 1 || rules[i].order > MAX_P || rules[i].log2n < 0 ||
            rules[i].log2n > 62 || rules[i].levels < 1 || rules[i].levels > MAX_L)
            return PETFMM_EINVAL;
    c->rules.assign(rules, rules + nrules);
    return PETFMM_OK;
}

int petfmm_tune_batch(petfmm_ctx *c, int n_inst, const petfmm_instance *inst, int reps,
                      petfmm_level_rule *out_rules, int cap, petfmm_tune_report *report) {
    if (!c || n_inst < 0 || (n_inst > 0 && !inst) || reps < 1 || cap < 0 ||
        (cap > 0 && !out_rules) || !report)
        return PETFMM_EINVAL;
    std::memset(report, 0, sizeof(*report));
    report->tc_blocks = c->tc_blocks;
    report->tc_dense_pct = c->tc_dense_pct;
    if (n_inst == 0) return PETFMM_OK;
    // whole batch at the work model's L, options as on entry
    const std::vector<petfmm_level_rule> none;
    std::vector<Problem> probs;
    int rc = problems_from(n_inst, inst, probs, &none);
    if (rc) return rc;
    int nev = 0;
    rc = time_batch(c, probs, reps, &report->ms_model, &nev);
    if (rc) return rc;
    // 1. per class (order, floor(log2 n)): the class alone at L_model - 1,
    //    L_model, L_model + 1
    std::map<std::pair<int, int>, std::vector<int>> classes;
    for (int i = 0; i < n_inst; ++i)
        if (inst[i].n > 0) classes[{inst[i].order, floor_log2(inst[i].n)}].push_back(i);
    // Each class is timed with an empty anchor instance at the batch's
    // deepest level, so that every candidate runs the launch sequence of the
    // whole batch (one M2M/L2L launch per level, ...): the comparison then
    // sees the class's work, not the launches a shallower tree would drop
    // when alone but not inside the batch.
    int Ldeep = 1;
    for (const Problem &q : probs) Ldeep = std::max(Ldeep, q.L);
    std::vector<petfmm_level_rule> rules;
    for (const auto &kv : classes) {
        const std::vector<int> &members = kv.second;
        std::vector<petfmm_instance> sub;
        for (int i : members) sub.push_back(inst[i]);
        petfmm_instance anchor{};
        anchor.domain = petfmm_domain{0.0, 0.0, 1.0};
        anchor.levels = Ldeep;
        anchor.order = kv.first.first;
        anchor.sigma = 1.0;
        anchor.n = 0;
        sub.push_back(anchor);
        const petfmm_instance &f = sub.front();
        const int Lm = petfmm_choose_levels(f.n, f.order, f.sigma, &f.domain);
        if (Lm < 0) return Lm;
        petfmm_level_rule best{kv.first.first, kv.first.second, Lm, -1.f};
        float model_ms = -1.f;
        for (int L : {Lm, Lm - 1, Lm + 1}) {
            if (L < 1 || L > MAX_L) continue;
            const petfmm_level_rule cand{kv.first.first, kv.first.second, L, 0.f};
            const std::vector<petfmm_level_rule> one{cand};
            std::vector<Problem> sp;
            if ((rc = problems_from(int(sub.size()), sub.data(), sp, &one))) return rc;
            bool applies = false;  // the guard may send every member back to the model
            for (size_t q = 0; q + 1 < sp.size(); ++q) applies |= sp[q].L == L;
            if (!applies) continue;
            float ms = 0.f;
            if ((rc = time_batch(c, sp, reps, &ms, &nev))) return rc;
            if (L == Lm) model_ms = ms;
            // another depth must beat the model's by kTuneMargin (timing noise
            // is not a reason to leave the model)
            const bool better = L == Lm ? best.ms < 0.f || ms < best.ms
                                        : ms < best.ms && (model_ms < 0.f ||
                                                           ms < (1.f - kTuneMargin) * model_ms);
            if (best.ms < 0.f || better) {
                best.levels = L;
                best.ms = ms;
            }
        }
        if (best.levels != Lm) report->changed++;
        rules.push_back(best);
    }
    // 2. the M2L shape for the whole batch under those rules (the entry
    //    options first; another pair must beat them by kTuneMargin)
    if ((rc = problems_from(n_inst, inst, probs, &rules))) return rc;
    const int blocks0 = c->tc_blocks, dense0 = c->tc_dense_pct;
    float best_ms = -1.f, entry_ms = -1.f;
    int best_blocks = blocks0, best_dense = dense0;
    std::vector<std::pair<int, int>> shapes{{blocks0, dense0}};
    for (int blocks = 0; blocks <= 2; ++blocks)
        for (int dense : {1, 5})
            if (!(blocks == blocks0 && dense == dense0)) shapes.push_back({blocks, dense});
    for (const auto &sh : shapes) {
        c->tc_blocks = sh.first;
        c->tc_dense_pct = sh.second;
        float ms = 0.f;
        rc = time_batch(c, probs, reps, &ms, &nev);
        if (rc) {
            c->tc_blocks = blocks0;
            c->tc_dense_pct = dense0;
            return rc;
        }
        if (entry_ms < 0.f) entry_ms = ms;
        if (best_ms < 0.f || (ms < best_ms && ms < (1.f - kTuneMargin) * entry_ms)) {
            best_ms = ms;
            best_blocks = sh.first;
            best_dense = sh.second;
        }
    }
    c->tc_blocks = best_blocks;
    c->tc_dense_pct = best_dense;
    c->rules = rules;
    // the tuned batch once more, so the caller's u, v hold its result
    if ((rc = run(c, probs))) return rc;
    ++nev;
    if ((rc = petfmm_sync(c))) return rc;
    report->tc_blocks = best_blocks;
    report->tc_dense_pct = best_dense;
    report->nrules = int(rules.size());
    report->evaluations = nev;
    report->ms_tuned = best_ms;
    for (int i = 0; i < std::min(cap, int(rules.size())); ++i) out_rules[i] = rules[i];
    return PETFMM_OK;
}

int petfmm_debug_plan(int precision, int n_inst, const petfmm_instance *inst, int64_t *out, int cap) {
    if (n_inst < 0 || (n_inst > 0 && !inst) || cap < 0 || (cap > 0 && !out)) return PETFMM_EINVAL;
    if (precision != PETFMM_FP64 && precision != PETFMM_MIXED) return PETFMM_EINVAL;
    std::vector<Problem> probs;
    int rc = problems_from(n_inst, inst, probs);
    if (rc) return rc;
    Plan pl;
    rc = build_plan(precision, KERNEL_VORTEX, true, 0, kTcSegDefault, kNearTolDefault, probs, pl);
    if (rc) return rc;
    int n = 0;
    auto emit = [&](int64_t id, const TaskRange &r) {
        for (int i = 0; i < r.count; ++i) {
            const Task &t = pl.tasks[size_t(r.first + i)];
            if (n < cap) {
                int64_t *o = out + 5 * size_t(n);
                o[0] = id; o[1] = t.inst; o[2] = t.level; o[3] = t.count; o[4] = t.block0;
            }
            ++n;
        }
    };
    emit(0, pl.outscatter);
    emit(1, pl.start);
    emit(2, pl.particles);
    emit(3, pl.leaves_p2m);
    emit(4, pl.leaves_wl);
    emit(5, pl.m2l);
    emit(6, pl.m2l_tc);
    emit(7, pl.m2l_tcb);
    for (int cls = 0; cls < Plan::kTileClasses; ++cls) emit(70 + cls, pl.m2l_tile[cls]);
    for (size_t r = 0; r < pl.m2m.size(); ++r) emit(100 + int64_t(r), pl.m2m[r]);
    for (size_t r = 0; r < pl.l2l.size(); ++r) emit(200 + int64_t(r), pl.l2l[r]);
    return n;
}

int petfmm_choose_levels(int64_t n, int order, double sigma, const petfmm_domain *dom) {
    if (n < 0 || order < 1 || order > MAX_P || !(sigma > 0.0) || !dom || !(dom->width > 0.0))
        return PETFMM_EINVAL;
    // Kernel-substitution guard: the far field starts one leaf away, so the
    // leaf width must keep exp(-r^2 / 2 sigma^2) <= 1e-8.
    const double rmin = sigma * std::sqrt(2.0 * std::log(1e8));
    const double p = order, p2 = double(order) * order;
    // Relative GPU costs of the units of Eq. 13 / 14 (one P2P pair, one
    // complex multiply-add of an expansion translation, one P2M/L2P term).
    const double c_pair = 1.0, c_mac = 0.35, c_term = 1.0;
    int best = 1;
    double best_cost = -1.0;
    for (int L = 1; L <= 12; ++L) {
        if (dom->width / std::ldexp(1.0, L) < rmin) break;
        const double nleaf = std::ldexp(1.0, 2 * L);
        const double s = double(n) / nleaf;
        double cost = nleaf * (c_term * 2.0 * s * p + c_mac * p2 * 27.0 + c_pair * 9.0 * s * s);
        for (int l = 2; l < L; ++l) cost += std::ldexp(1.0, 2 * l) * c_mac * p2 * (2.0 * 4.0 + 27.0);
        if (best_cost < 0.0 || cost < best_cost) {
            best_cost = cost;
            best = L;
        }
    }
    return best;
}

int petfmm_set_option(petfmm_ctx *c, int option, int64_t value) {
    if (!c) return PETFMM_EINVAL;
    switch (option) {
        case PETFMM_OPT_TIMING: c->timing = value != 0; return PETFMM_OK;
        case PETFMM_OPT_SPIN_LIMIT: c->spin_limit = value; return PETFMM_OK;
        case PETFMM_OPT_P2P_MODE: if (value < 0 || value > 1) return PETFMM_EINVAL; c->p2p_mode = int(value); return PETFMM_OK;
        case PETFMM_OPT_POISON: c->poison = value != 0; return PETFMM_OK;
        case PETFMM_OPT_M2L_TC: c->m2l_tc = value != 0; return PETFMM_OK;
        case PETFMM_OPT_TC_SEG:
            if (value != 128 && value != 256 && value != 512) return PETFMM_EINVAL;
            c->tc_segmax = int(value);
            return PETFMM_OK;
        case PETFMM_OPT_GRAPH: c->use_graph = value != 0; return PETFMM_OK;
        case PETFMM_OPT_P2P_PAIRS: c->p2p_pairs = value != 0; return PETFMM_OK;
        case PETFMM_OPT_TC_BLOCKS:
            if (value < 0 || value > 2) return PETFMM_EINVAL;
            c->tc_blocks = int(value);
            return PETFMM_OK;
        case PETFMM_OPT_TC_PIPE:
            if (value < 0 || value > 2) return PETFMM_EINVAL;
            c->tc_pipe = int(value);
            return PETFMM_OK;
        case PETFMM_OPT_OVERLAP: c->overlap = value != 0; return PETFMM_OK;
        case PETFMM_OPT_KERNEL:
            if (value != PETFMM_KERNEL_VORTEX && value != PETFMM_KERNEL_LAPLACE)
                return PETFMM_EINVAL;
            c->kernel = int(value);
            return PETFMM_OK;
        case PETFMM_OPT_NEAR_TOL:
            if (value < 1 || value > 1000000) return PETFMM_EINVAL;
            c->near_tol = double(value) * 1e-9;
            return PETFMM_OK;
        case PETFMM_OPT_TC_DENSE: if (value < 0 || value > 100) return PETFMM_EINVAL; c->tc_dense_pct = int(value); return PETFMM_OK;
        default: return PETFMM_EINVAL;
    }
}

int petfmm_stage_times(petfmm_ctx *c, float *ms, int cap) {
    if (!c || !ms || cap < 0) return PETFMM_EINVAL;
    if (!c->ev_recorded) return PETFMM_ENOTREADY;
    const int n = std::min(cap, int(PETFMM_STAGE_COUNT));
    for (int s = 0; s < n; ++s) {
        float t = 0.f;
        const cudaEvent_t end = s == PETFMM_STAGE_L2L ? c->ev[PETFMM_STAGE_COUNT + 1] : c->ev[s + 1];
        if (cudaEventElapsedTime(&t, c->ev[s], end) != cudaSuccess) {
            cudaGetLastError();
            return PETFMM_ECUDA;
        }
        ms[s] = t;
    }
    return n;
}

int petfmm_get_stats(petfmm_ctx *c, petfmm_stats *out) {
    if (!c || !out) return PETFMM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->kernel_launches = c->launches;
    out->evaluations = c->evaluations;
    for (const InstDesc &d : c->plan.inst) out->m2l_pairs += m2l_pair_count(d.L);
    if (c->ctrl.p && c->evaluations) {
        uint32_t w[CTRL_WORDS];
        if (cudaMemcpy(w, c->ctrl.p, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return PETFMM_ECUDA;
        out->p2p_items = w[CTRL_NITEMS];
        out->occupied_leaves = w[CTRL_NOCC];
        unsigned long long pairs;
        std::memcpy(&pairs, w + CTRL_PAIRS_LO, sizeof(pairs));
        out->p2p_pairs = int64_t(pairs);
        if (c->p2p_pairs && c->precision != PETFMM_FP64) {
            out->p2p_pair_items = w[CTRL_NPAIRS];
            out->p2p_split_entries = w[CTRL_NXTRA];
            unsigned long long sym;
            std::memcpy(&sym, w + CTRL_SYM_LO, sizeof(sym));
            out->p2p_sym_pairs = int64_t(sym);
        }
    }
    if (c->timing && c->busy.p && c->p2p_grid > 0 && c->ev_recorded) {
        const int warps = 8;
        const bool pairs = c->p2p_pairs && c->precision != PETFMM_FP64 && c->pairs_grid > 0;
        const size_t nblk = size_t(c->p2p_grid) + (pairs ? size_t(c->pairs_grid) : 0);
        std::vector<unsigned long long> b(nblk * warps * 2);
        if (cudaMemcpy(b.data(), c->busy.p, b.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return PETFMM_ECUDA;
        // Eq. 20 over the CTAs of one persistent launch: min / max busy span
        auto lb = [&](size_t b0, size_t nb) {
            double lo = 0, hi = 0;
            for (size_t blk = b0; blk < b0 + nb; ++blk) {
                unsigned long long s = ~0ull, e = 0;
                for (int w = 0; w < warps; ++w) {
                    s = std::min(s, b[(blk * warps + w) * 2]);
                    e = std::max(e, b[(blk * warps + w) * 2 + 1]);
                }
                const double span = double(e - s);
                if (blk == b0) lo = hi = span;
                lo = std::min(lo, span);
                hi = std::max(hi, span);
            }
            return hi > 0 ? float(lo / hi) : 1.0f;
        };
        out->p2p_load_balance = lb(0, size_t(c->p2p_grid));
        if (pairs) out->pairs_load_balance = lb(size_t(c->p2p_grid), size_t(c->pairs_grid));
    }
    return PETFMM_OK;
}

int petfmm_debug_checks(uint32_t *lines) {
    if (!lines) return PETFMM_EINVAL;
    lines[0] = pf_checks_tree();
    lines[1] = pf_checks_expansions();
    lines[2] = pf_checks_p2p();
#ifdef PETFMM_CHECKS
    return 3;
#else
    return 0;
#endif
}

int petfmm_debug_tree(petfmm_ctx *c, uint32_t *keys, uint32_t *perm, uint32_t *start) {
    if (!c) return PETFMM_EINVAL;
    if (c->plan.inst.size() != 1) return PETFMM_EINVAL;
    const int64_t n = c->plan.N;
    const InstDesc &d = c->plan.inst[0];
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PETFMM_ECUDA;
    std::vector<uint32_t> sk(static_cast<size_t>(n)), pm(static_cast<size_t>(n));
    if (n > 0) {
        const void *skp = c->sorted_in_first ? c->keysA.p : c->keysB.p;
        const void *pmp = c->sorted_in_first ? c->valsA.p : c->valsB.p;
        if (cudaMemcpy(sk.data(), skp, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PETFMM_ECUDA;
        if (cudaMemcpy(pm.data(), pmp, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PETFMM_ECUDA;
    }
    if (perm) std::memcpy(perm, pm.data(), size_t(n) * 4);
    if (keys)
        for (int64_t r = 0; r < n; ++r) keys[pm[r]] = sk[r];
    if (start) {
        const size_t ns = (size_t(1) << (2 * d.L)) + 1;
        if (n > 0) {
            if (cudaMemcpy(start, c->start.p, ns * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PETFMM_ECUDA;
        } else {
            std::memset(start, 0, ns * 4);
        }
    }
    return PETFMM_OK;
}

int petfmm_debug_expansions(petfmm_ctx *c, int level, int which, double *out) {
    if (!c || !out || (which != 0 && which != 1)) return PETFMM_EINVAL;
    if (c->plan.inst.size() != 1 || c->plan.N == 0) return PETFMM_EINVAL;
    const InstDesc &d = c->plan.inst[0];
    if (level < 2 || level > d.L) return PETFMM_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PETFMM_ECUDA;
    const int p = d.p;
    const int64_t nb = int64_t(1) << (2 * level);
    const DevBuf &src = which == 0 ? c->me : c->le;
    const bool mixed = c->precision == PETFMM_MIXED;
    const size_t es = mixed ? sizeof(float2) : sizeof(double2);
    std::vector<unsigned char> h(size_t(nb) * p * es);
    const unsigned char *base = static_cast<const unsigned char *>(src.p) + (d.eoff + lvl_off(level) * p) * es;
    if (cudaMemcpy(h.data(), base, h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return PETFMM_ECUDA;
    for (int64_t m = 0; m < nb; ++m) {
        const uint32_t ix = compact_bits(uint32_t(m)), iy = compact_bits(uint32_t(m) >> 1);
        const int64_t b = box_index(level, ix, iy);
        for (int k = 0; k < p; ++k) {
            double re, im;
            if (mixed) {
                const float2 *f = reinterpret_cast<const float2 *>(h.data()) + b * p + k;
                re = f->x; im = f->y;
            } else {
                const double2 *f = reinterpret_cast<const double2 *>(h.data()) + b * p + k;
                re = f->x; im = f->y;
            }
            out[(m * p + k) * 2] = re;
            out[(m * p + k) * 2 + 1] = im;
        }
    }
    return PETFMM_OK;
}

int petfmm_debug_interaction_list(int level, int ix, int iy, int32_t *out) {
    if (!out) return PETFMM_EINVAL;
    const int n = host_interaction_list(level, ix, iy, out);
    return n < 0 ? PETFMM_EINVAL : n;
}

int petfmm_debug_near_fit(double sigma, double wleaf, double tol, double *out) {
    if (!(sigma > 0.0) || !(wleaf > 0.0) || !(tol > 0.0) || !out) return PETFMM_EINVAL;
    InstDesc d{};
    d.sigma = sigma;
    d.wleaf = wleaf;
    fill_p2p_constants(d, tol);
    out[0] = d.deg;
    out[1] = d.general;
    out[2] = d.kappa;
    out[3] = d.qsplit_rho2;
    for (int k = 0; k <= POLY_MAX; ++k) out[4 + k] = d.poly[k];
    return PETFMM_OK;
}

int petfmm_debug_op_table(int order, int kernel, int which, double *out, int64_t cap) {
    if (order < 1 || order > MAX_P || (kernel != KERNEL_VORTEX && kernel != KERNEL_LAPLACE) ||
        which < 0 || which > 2 || cap < 0 || (cap > 0 && !out))
        return PETFMM_EINVAL;
    std::vector<double> t;
    host_op_table(order, kernel, which, t);
    const int64_t n = int64_t(t.size());
    if (out && cap >= n) std::memcpy(out, t.data(), size_t(n) * sizeof(double));
    return int(n);
}

int petfmm_debug_m2l_images(int order, int kernel, int blocks, float *out, int64_t cap) {
    if (order < 1 || order > 24 || (kernel != KERNEL_VORTEX && kernel != KERNEL_LAPLACE) ||
        blocks < 0 || blocks > 1 || cap < 0 || (cap > 0 && !out))
        return PETFMM_EINVAL;
    std::vector<float> img;
    if (blocks) host_m2l_tcb_images(order, kernel, img);
    else host_m2l_tc_images(order, kernel, img);
    const int64_t n = int64_t(img.size());
    if (out && cap >= n) std::memcpy(out, img.data(), size_t(n) * sizeof(float));
    return int(n);
}

}  // extern "C"
