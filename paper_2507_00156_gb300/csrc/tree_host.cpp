// Treecode far field (Sec. 3.4), host side: the octree of the surface's nodes, its upload, and
// the parameter rule of Eq. (optimal_params).
//
// The nodes are partitioned recursively: a cluster of more than N0 nodes is split at the midpoint
// of its bounding box into octants (a node goes to the upper half of axis a when x_a > (lo_a +
// hi_a)/2; empty octants are dropped; a box without extent stays a leaf).  Every cluster keeps
// the bounding box of its own nodes, centre c = (lo + hi)/2, half-widths (hi - lo)/2 and radius
// r_c = half the box diagonal.  Clusters are numbered level by level (breadth first), so the
// children of a cluster are contiguous; the octant partition is stable, so the node order of
// the leaves does not depend on the numbering.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tree.h"

namespace ers {

void treecode_defaults(double h, double *theta, int *n0, int *p) {
    // Eq. (optimal_params): theta = 0.6; N0 = 2000, p = 6 at h = 1/64, N0 doubling and p growing
    // by 2 with every halving of h.  Below h = 1/64 the rule is held at N0 >= 1000 and p >= 6, the
    // values Table 2 uses at h = 1/16 and 1/32.
    const double L = std::round(std::log2(1.0 / (64.0 * h)));
    const double n = 2000.0 * std::exp2(L);
    *theta = 0.6;
    *n0 = (int)std::fmax(1000.0, std::fmin(n, 1.0e9));
    *p = (int)std::fmax(6.0, std::fmin(6.0 + 2.0 * L, (double)TREE_PMAX));
}

namespace {

struct Pending {
    int64_t start, count;
    int level;
};

TreeCluster make_cluster(const std::vector<double> &x, const std::vector<int> &perm, int64_t s, int64_t e,
                         int level) {
    TreeCluster C{};
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = s; i < e; ++i)
        for (int a = 0; a < 3; ++a) {
            const double v = x[3 * (size_t)perm[i] + a];
            lo[a] = v < lo[a] ? v : lo[a];
            hi[a] = v > hi[a] ? v : hi[a];
        }
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        C.c[a] = 0.5 * (lo[a] + hi[a]);
        C.hw[a] = 0.5 * (hi[a] - lo[a]);
        const double ext = hi[a] - lo[a];
        const double e2 = ext * ext;
        diag2 = diag2 + e2;
    }
    C.rc = 0.5 * std::sqrt(diag2);
    C.start = (int)s;
    C.count = (int)(e - s);
    C.level = level;
    C.first_child = -1;
    C.nchild = 0;
    return C;
}

// The octree of nodes x (canonical order, [N][3]) for leaf size n0: clusters numbered level by
// level, perm = tree position -> canonical node; returns the depth.
int build_octree(const std::vector<double> &x, int64_t N, int n0, std::vector<TreeCluster> &cl, std::vector<int> &perm) {
    perm.resize(N);
    std::vector<int> tmp(N);
    for (int64_t i = 0; i < N; ++i) perm[i] = (int)i;
    cl.clear();
    std::vector<Pending> cur{{0, N, 0}}, next;
    if (N == 0) cur.clear();
    int depth = 0;
    // level by level: every cluster of the level is created, then split (if it must be) into
    // children that are appended, contiguously, to the next level
    while (!cur.empty()) {
        const size_t base = cl.size();
        for (const Pending &q : cur) cl.push_back(make_cluster(x, perm, q.start, q.start + q.count, q.level));
        next.clear();
        for (size_t i = 0; i < cur.size(); ++i) {
            TreeCluster &C = cl[base + i];
            const double ext2 = C.hw[0] * C.hw[0] + C.hw[1] * C.hw[1] + C.hw[2] * C.hw[2];
            if (C.count <= n0 || !(ext2 > 0.0)) continue;
            const int64_t s0 = C.start, e0 = (int64_t)C.start + C.count;
            int64_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            auto octant = [&](int node) {
                const double *pp = &x[3 * (size_t)node];
                return (pp[0] > C.c[0] ? 1 : 0) | (pp[1] > C.c[1] ? 2 : 0) | (pp[2] > C.c[2] ? 4 : 0);
            };
            for (int64_t k = s0; k < e0; ++k) ++cnt[octant(perm[k])];
            int64_t off[8], pos[8];
            off[0] = s0;
            for (int o = 1; o < 8; ++o) off[o] = off[o - 1] + cnt[o - 1];
            std::memcpy(pos, off, sizeof pos);
            for (int64_t k = s0; k < e0; ++k) tmp[pos[octant(perm[k])]++] = perm[k];
            std::memcpy(&perm[s0], &tmp[s0], sizeof(int) * (size_t)(e0 - s0));
            C.first_child = (int)(base + cur.size() + next.size());
            for (int o = 0; o < 8; ++o) {
                if (cnt[o] == 0) continue;
                next.push_back({off[o], cnt[o], C.level + 1});
                ++C.nchild;
            }
        }
        if (!next.empty()) depth = cur[0].level + 1;
        cur.swap(next);
    }
    return depth;
}

// Morton (Z-order) code of a cell: the bits of ix, iy, iz interleaved.
uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
    uint64_t k = 0;
    for (int bit = 0; bit < 21; ++bit) {
        k |= (uint64_t)((ix >> bit) & 1u) << (3 * bit);
        k |= (uint64_t)((iy >> bit) & 1u) << (3 * bit + 1);
        k |= (uint64_t)((iz >> bit) & 1u) << (3 * bit + 2);
    }
    return k;
}

void free_dev(TreeCache *t) {
    void *ptrs[] = {t->cl, t->leaf_ids, t->inner_ids, t->tsrt, t->tleaf, t->trec, t->trec32, t->W, t->W32,
                    t->stats};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

std::vector<int> morton_cell_rank(const Grid &G) {
    // targets ordered by cell with the cells in Morton order: the 32 targets of a warp are
    // compact, so they share near nodes in the caches and decide alike at tree clusters
    std::vector<int> cell_rank((size_t)G.ncell);
    if (G.ncell <= ((int64_t)1 << 26)) {
        std::vector<std::pair<uint64_t, int>> mk((size_t)G.ncell);
        for (int64_t c = 0; c < G.ncell; ++c) {
            const uint32_t ix = (uint32_t)(c % G.nc[0]), iy = (uint32_t)((c / G.nc[0]) % G.nc[1]);
            const uint32_t iz = (uint32_t)(c / ((int64_t)G.nc[0] * G.nc[1]));
            mk[c] = {morton3(ix, iy, iz), (int)c};
        }
        std::sort(mk.begin(), mk.end());
        for (int64_t r = 0; r < G.ncell; ++r) cell_rank[mk[r].second] = (int)r;
    } else {
        for (int64_t c = 0; c < G.ncell; ++c) cell_rank[c] = (int)c;
    }
    return cell_rank;
}

void tree_free(ers_surface *s) {
    if (!s || !s->tree) return;
    free_dev(s->tree);
    delete s->tree;
    s->tree = nullptr;
}

int tree_build(ers_surface *s, int n0) {
    if (s->tree && s->tree->n0 == n0) return ERS_OK;
    tree_free(s);
    const int64_t N = s->N;
    if (N > INT32_MAX / 2) return fail(ERS_E_UNSUPPORTED, "treecode: more than 2^30 nodes");
    std::vector<double> x(3 * (size_t)N);
    std::vector<int> sperm(N);  // cell-sorted index -> canonical index
    cudaError_t e = cudaMemcpy(x.data(), s->x, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sperm.data(), s->perm, sizeof(int) * N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "treecode: download of the nodes");
    std::vector<int> srt_of(N);  // canonical -> cell-sorted
    for (int64_t j = 0; j < N; ++j) srt_of[sperm[j]] = (int)j;

    std::vector<int> perm;
    std::vector<TreeCluster> cl;
    const int depth = build_octree(x, N, n0, cl, perm);

    TreeCache *t = new TreeCache();
    t->n0 = n0;
    t->ncl = (int)cl.size();
    t->depth = depth;
    t->host_cl = cl;
    std::vector<int> leaves, inner;
    t->inner_off.assign(depth + 2, 0);
    for (int l = 0; l <= depth; ++l) {
        t->inner_off[l] = (int)inner.size();
        for (int c = 0; c < t->ncl; ++c) {
            if (cl[c].level != l) continue;
            if (cl[c].nchild == 0) leaves.push_back(c);
            else inner.push_back(c);
        }
    }
    t->inner_off[depth + 1] = (int)inner.size();
    t->nleaf = (int)leaves.size();
    std::vector<int> tsrt(N), tleaf(N);
    for (int64_t i = 0; i < N; ++i) tsrt[i] = srt_of[perm[i]];
    for (int c : leaves)
        for (int i = cl[c].start; i < cl[c].start + cl[c].count; ++i) tleaf[i] = c;

    auto alloc = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes ? bytes : 16);
    };
    alloc((void **)&t->cl, sizeof(TreeCluster) * cl.size());
    alloc((void **)&t->leaf_ids, sizeof(int) * leaves.size());
    alloc((void **)&t->inner_ids, sizeof(int) * inner.size());
    alloc((void **)&t->tsrt, sizeof(int) * N);
    alloc((void **)&t->tleaf, sizeof(int) * N);
    alloc((void **)&t->trec, sizeof(double) * REC * N);
    alloc((void **)&t->trec32, sizeof(float) * 12 * N);
    alloc((void **)&t->stats, sizeof(unsigned long long) * 3);
    if (e == cudaSuccess) e = cudaMemcpy(t->cl, cl.data(), sizeof(TreeCluster) * cl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !leaves.empty())
        e = cudaMemcpy(t->leaf_ids, leaves.data(), sizeof(int) * leaves.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !inner.empty())
        e = cudaMemcpy(t->inner_ids, inner.data(), sizeof(int) * inner.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->tsrt, tsrt.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->tleaf, tleaf.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_dev(t);
        delete t;
        return fail(ERS_E_NOMEM, std::string("treecode: device allocation/upload: ") + cudaGetErrorString(e));
    }
    s->tree = t;
    return ERS_OK;
}

}  // namespace ers

// Test hook (not in the public header): the octree of nodes x ([N][3], host) for leaf size n0,
// host only.  Per cluster: geom[c][7] = centre, half-widths, r_c; info[c][5] = start, count,
// first child, children, level; perm[N] = tree position -> node.  Returns the number of clusters,
// or minus the number needed when cap is smaller.
extern "C" int64_t ers_debug_octree(const double *x, int64_t N, int n0, int64_t cap, double *geom, int *info,
                                    int *perm) {
    if (!x || N < 0 || n0 < 1) return 0;
    std::vector<double> xv(x, x + 3 * N);
    std::vector<ers::TreeCluster> cl;
    std::vector<int> pv;
    ers::build_octree(xv, N, n0, cl, pv);
    const int64_t n = (int64_t)cl.size();
    if (n > cap) return -n;
    for (int64_t c = 0; c < n; ++c) {
        const ers::TreeCluster &C = cl[c];
        for (int a = 0; a < 3; ++a) {
            geom[7 * c + a] = C.c[a];
            geom[7 * c + 3 + a] = C.hw[a];
        }
        geom[7 * c + 6] = C.rc;
        int *o = info + 5 * c;
        o[0] = C.start;
        o[1] = C.count;
        o[2] = C.first_child;
        o[3] = C.nchild;
        o[4] = C.level;
    }
    if (perm) std::memcpy(perm, pv.data(), sizeof(int) * (size_t)N);
    return n;
}

namespace ers {

int tree_stats(ers_surface *s, int64_t out[5]) {
    for (int i = 0; i < 5; ++i) out[i] = 0;
    TreeCache *t = s->tree;
    if (!t) return ERS_OK;
    out[0] = t->ncl;
    out[1] = t->nleaf;
    out[2] = t->depth;
    if (t->stats_valid) {
        unsigned long long h[3] = {0, 0, 0};
        cudaError_t e = cudaMemcpy(h, t->stats, sizeof h, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "treecode statistics");
        out[3] = (int64_t)h[0];
        out[4] = (int64_t)h[1];
        if (h[2]) return fail(ERS_E_TIMEOUT, "treecode: a staging wait ran out; the last result is invalid");
    }
    return ERS_OK;
}

}  // namespace ers
