// shard.cu -- the tree cut of Sec. 4 and the work / communication model of
// Sec. 5.1-5.2, for sharding one evaluation over several GPUs (host code).
//
// The quadtree is cut at level k: a root tree (levels 0..k) and 4^k local
// subtrees, each rooted at a level-k box and holding levels k..L below it.
// Each subtree is a vertex weighted by its work (Eq. 13 for its non-leaf
// boxes, Eq. 14 for its leaves with their actual particle counts: the
// reading of Eq. 15's leaf term); two subtrees that touch are joined by an
// edge weighted by the expansion terms their interaction lists exchange
// (Eq. 11 for lateral neighbours, the diagonal count below for corner
// neighbours).  The paper hands this graph to ParMETIS; here the subtrees are
// cut into contiguous runs of their z-order (Sec. 5.1 uses the same
// numbering to find neighbours), with the largest run weight as small as a
// contiguous split allows -- a space-filling-curve partition, whose runs are
// spatially compact, so the cut edges stay few.
//
// For a rank, the halo is what it must receive before evaluating its
// subtrees' particles: the particles of the other ranks' leaves adjacent to
// its leaves (near field, Sec. 2.2's evaluation step), and the multipole
// expansions of the other ranks' boxes at levels k+1..L that lie in the
// interaction lists of its boxes.  The level-k expansions of all subtrees
// are exchanged by every rank (all-gather), and the root tree (levels <= k)
// is then evaluated by each rank for itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/petfmm.h"
#include "kernels.cuh"

using namespace petfmm;

namespace {

constexpr int kNC = 4;    // children of a quadtree box
constexpr int kNIL = 27;  // interaction-list members of an interior box
constexpr int kNND = 9;   // near-domain leaves (the leaf and its 8 neighbours)

bool bad_cut(int L, int k) { return L < 1 || L > MAX_L || k < 0 || k > L; }

// Morton index of the level-k ancestor of leaf m (level L).
inline uint32_t ancestor(uint32_t m, int L, int k) { return m >> (2 * (L - k)); }

inline uint32_t ix_of(uint32_t m) { return compact_bits(m); }
inline uint32_t iy_of(uint32_t m) { return compact_bits(m >> 1); }

}  // namespace

extern "C" {

int petfmm_shard_weights(int L, int k, int order, const uint32_t *leaf_counts, double *work) {
    if (bad_cut(L, k) || order < 1 || order > MAX_P || !leaf_counts || !work) return PETFMM_EINVAL;
    const double p = order, p2 = double(order) * order;
    const int64_t nsub = int64_t(1) << (2 * k);
    const int64_t per = int64_t(1) << (2 * (L - k));  // leaves per subtree
    // Eq. 13 per non-leaf box of a subtree (levels k .. L-1 inside it; a
    // subtree of depth L - k has (4^(L-k) - 1) / 3 of them)
    const double nonleaf = double((per - 1) / 3);
    for (int64_t s = 0; s < nsub; ++s) {
        double w = nonleaf * p2 * (2.0 * kNC + kNIL);
        // Eq. 14 per leaf, with the leaf's own particle count
        for (int64_t j = 0; j < per; ++j) {
            const double ni = leaf_counts[s * per + j];
            w += 2.0 * ni * p + p2 * kNIL + kNND * ni * ni;
        }
        work[s] = w;
    }
    return PETFMM_OK;
}

int petfmm_shard_comm(int L, int k, double alpha, double *lateral, double *diagonal) {
    if (bad_cut(L, k) || !(alpha >= 0.0) || !lateral || !diagonal) return PETFMM_EINVAL;
    // Eq. 11: expansion terms between two lateral neighbours (both
    // directions: 2^(n-k) boxes on each side of the shared edge, two layers
    // each way)
    double lat = 0.0;
    for (int n = k + 1; n <= L; ++n) lat += alpha * std::ldexp(1.0, n - k) * 4.0;
    // diagonal neighbours: only the corner boxes, four per level each way
    // (Eq. 12 is garbled in the text; this is the count the interaction lists
    // give, see petfmm_shard_halo)
    *lateral = lat;
    *diagonal = alpha * 8.0 * double(L - k);
    return PETFMM_OK;
}

int petfmm_shard_partition(int L, int k, int order, const uint32_t *leaf_counts, int nranks,
                           int32_t *owner, petfmm_shard_rank *ranks) {
    if (bad_cut(L, k) || order < 1 || order > MAX_P || !leaf_counts || nranks < 1 || !owner ||
        !ranks)
        return PETFMM_EINVAL;
    const int64_t nsub = int64_t(1) << (2 * k);
    if (nranks > nsub) return PETFMM_EINVAL;  // every rank gets at least one subtree
    std::vector<double> w(size_t(nsub), 0.0);
    int rc = petfmm_shard_weights(L, k, order, leaf_counts, w.data());
    if (rc) return rc;
    // Smallest largest-run weight of a split into nranks contiguous runs
    // (non-empty): bisection on the bound, a greedy fill checking it.
    auto runs_needed = [&](double cap) {
        int runs = 1;
        double acc = 0.0;
        for (int64_t s = 0; s < nsub; ++s) {
            if (w[size_t(s)] > cap) return nranks + 1;
            if (acc + w[size_t(s)] > cap) {
                ++runs;
                acc = 0.0;
            }
            acc += w[size_t(s)];
        }
        return runs;
    };
    double lo = *std::max_element(w.begin(), w.end()), hi = 0.0;
    for (double x : w) hi += x;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (runs_needed(mid) <= nranks) hi = mid; else lo = mid;
    }
    // fill greedily under the bound, keeping enough subtrees for the ranks
    // still to come (so no rank is left empty)
    int r = 0;
    double acc = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const int64_t left = nsub - s;           // subtrees not yet assigned
        const int ranks_after = nranks - 1 - r;  // ranks after the current one
        if (r < nranks - 1 && acc > 0.0 && (acc + w[size_t(s)] > hi || left <= ranks_after)) {
            ++r;
            acc = 0.0;
        }
        owner[s] = r;
        acc += w[size_t(s)];
    }
    // per-rank summary: work, particles, runs, and the Eq. 11 / diagonal
    // communication of its cut edges (alpha = 1: expansion terms)
    double lat = 0.0, diag = 0.0;
    petfmm_shard_comm(L, k, 1.0, &lat, &diag);
    const int64_t per = int64_t(1) << (2 * (L - k));
    const int side = 1 << k;
    for (int q = 0; q < nranks; ++q) std::memset(&ranks[q], 0, sizeof(ranks[q]));
    for (int q = 0; q < nranks; ++q) ranks[q].first_subtree = -1;
    for (int64_t s = 0; s < nsub; ++s) {
        petfmm_shard_rank &R = ranks[owner[s]];
        R.work += w[size_t(s)];
        R.subtrees++;
        if (R.first_subtree < 0) R.first_subtree = int32_t(s);
        R.last_subtree = int32_t(s + 1);
        for (int64_t j = 0; j < per; ++j) R.particles += leaf_counts[s * per + j];
        const int sx = int(ix_of(uint32_t(s))), sy = int(iy_of(uint32_t(s)));
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int nx = sx + dx, ny = sy + dy;
                if (nx < 0 || ny < 0 || nx >= side || ny >= side) continue;
                const uint32_t t = morton_key(uint32_t(nx), uint32_t(ny));
                if (owner[t] == owner[s]) continue;
                R.comm += (dx && dy) ? diag : lat;
            }
    }
    return PETFMM_OK;
}

int petfmm_shard_halo(int L, int k, const int32_t *owner, int rank, int32_t *leaves,
                      int64_t leaf_cap, int32_t *boxes, int64_t box_cap, int64_t *nleaves,
                      int64_t *nboxes) {
    if (bad_cut(L, k) || !owner || rank < 0 || leaf_cap < 0 || box_cap < 0 ||
        (leaf_cap > 0 && !leaves) || (box_cap > 0 && !boxes) || !nleaves || !nboxes)
        return PETFMM_EINVAL;
    const int64_t nleaf = int64_t(1) << (2 * L);
    const int nside = 1 << L;
    // near field: other ranks' leaves adjacent to this rank's leaves
    std::vector<char> mark(size_t(nleaf), 0);
    for (int64_t m = 0; m < nleaf; ++m) {
        if (owner[ancestor(uint32_t(m), L, k)] != rank) continue;
        const int ix = int(ix_of(uint32_t(m))), iy = int(iy_of(uint32_t(m)));
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = ix + dx, y = iy + dy;
                if (x < 0 || y < 0 || x >= nside || y >= nside) continue;
                const uint32_t t = morton_key(uint32_t(x), uint32_t(y));
                if (owner[ancestor(t, L, k)] != rank) mark[t] = 1;
            }
    }
    int64_t nl = 0;
    for (int64_t m = 0; m < nleaf; ++m)
        if (mark[size_t(m)]) {
            if (nl < leaf_cap) leaves[nl] = int32_t(m);
            ++nl;
        }
    // far field: other ranks' boxes at levels k+1..L in the interaction lists
    // of this rank's boxes (the same interaction lists the kernels use)
    int64_t nb = 0;
    int32_t il[2 * 27];
    for (int l = k + 1; l <= L; ++l) {
        const int64_t n = int64_t(1) << (2 * l);
        std::vector<char> need(size_t(n), 0);
        for (int64_t m = 0; m < n; ++m) {
            if (owner[ancestor(uint32_t(m), l, k)] != rank) continue;
            const int cnt = host_interaction_list(l, int(ix_of(uint32_t(m))), int(iy_of(uint32_t(m))), il);
            for (int i = 0; i < cnt; ++i) {
                const uint32_t t = morton_key(uint32_t(il[2 * i]), uint32_t(il[2 * i + 1]));
                if (owner[ancestor(t, l, k)] != rank) need[t] = 1;
            }
        }
        for (int64_t m = 0; m < n; ++m)
            if (need[size_t(m)]) {
                if (nb < box_cap) {
                    boxes[2 * nb] = l;
                    boxes[2 * nb + 1] = int32_t(m);
                }
                ++nb;
            }
    }
    *nleaves = nl;
    *nboxes = nb;
    return PETFMM_OK;
}

}  // extern "C"
