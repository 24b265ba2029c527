// Treecode far field (Sec. 3.4): the per-surface cache shared by the host tree build
// (tree_host.cpp) and the kernels (k_tree.cu).
#pragma once

#include "ers_internal.h"

namespace ers {

// cos(k pi / p), k = 0..p: the Chebyshev points of the second kind on [-1, 1]
struct Cheb {
    double cosk[TREE_PMAX + 1];
    int p;
};

struct TreeCache {
    int n0 = 0;  // leaf size the tree was built for (0: none)
    int ncl = 0, nleaf = 0, depth = 0;
    std::vector<TreeCluster> host_cl;
    std::vector<int> inner_off;  // inner (non-leaf) clusters of level l: inner_ids[inner_off[l] .. inner_off[l+1])
    TreeCluster *cl = nullptr;   // [ncl]
    int *leaf_ids = nullptr;     // [nleaf]
    int *inner_ids = nullptr;    // [ncl - nleaf], grouped by level
    int *tsrt = nullptr;         // [N] tree position -> cell-sorted node index
    int *tleaf = nullptr;        // [N] tree position -> its leaf
    double *trec = nullptr;      // [N][REC] tree-ordered records of the current densities
    float *trec32 = nullptr;     // [N][12] FP32: x - leaf centre, w f, w n, q
    uint64_t rec_version = ~0ull;
    // modified weights of degree p for the densities of version w_version
    int p = 0;
    uint64_t w_version = ~0ull;
    bool have_w32 = false;
    bool w_fp64 = false;  // the weights were built with FP64 products (else good for the mixed path only)
    double *W = nullptr;   // [ncl][(p+1)^3][TREE_WS]
    float *W32 = nullptr;  // [ncl][(p+1)^3][TREE_WS]
    size_t w_cap = 0, w32_cap = 0;
    Cheb ch{};
    unsigned long long *stats = nullptr;  // [3]: approximated (target, cluster) pairs, far pairs summed directly, wait ran out
    bool stats_valid = false;
};

// Build the octree of the surface's nodes for leaf size n0 (host), upload it; ERS_OK or an error.
int tree_build(ers_surface *s, int n0);

}  // namespace ers
