/*
 * FP64 CPU oracle of the kernel-independent treecode far field (Siebor & Tlupova, Sec. 3.4,
 * Eqs. (MAC), (particle-cluster), (particle-cluster-KITC), (mod_weights)).
 *
 * TEST INFRASTRUCTURE ONLY, like ers_oracle.c (which it is linked with): the plain reference
 * that the GPU treecode is checked against.  It shares no code with the GPU library.
 *
 * The steps, in the paper's order:
 *  1. the nodes are partitioned into an octree: a cluster with more than N0 nodes is split
 *     into the eight octants of its box, until every leaf holds at most N0 nodes;
 *  2. the modified weights of every cluster, Eq. (mod_weights), for the 15 densities that the
 *     subtracted sums need: f w (3), n w (3) and q_j n_k w (9);
 *  3. for each target, a recursive walk from the root: a cluster that meets the MAC r_c/R <=
 *     theta (Eq. (MAC)) is summed by Eq. (particle-cluster-KITC) with the unregularized
 *     Stokeslet and stresslet at its Chebyshev points; otherwise its children are visited, and a
 *     leaf is summed directly, with the regularized kernels for the K deltas at the nodes within
 *     Rc = tc delta_K and the plain kernels beyond (Sec. 3.3);
 *  4. the extrapolation of Eq. (extrap_eqn) (ers_oracle.c:ora_extrapolate_k).
 *
 * Readings (where the text leaves a choice):
 *  - the box of a cluster is the bounding box of its nodes; a cluster is split at the midpoint
 *    of its box, a node going to the upper half of axis a when x_a > (lo_a + hi_a)/2; empty
 *    octants are dropped, the others are visited in octant order (bit a of the octant index =
 *    upper half of axis a); a cluster whose box has no extent is a leaf;
 *  - r_c = half the diagonal of the box, R = |y - box centre|;
 *  - Chebyshev points of the second kind s_k = c_a + h_a cos(k pi / p) (k = 0..p, c_a and h_a the
 *    centre and half-width of the box along axis a) with the barycentric weights (-1)^k d_k,
 *    d_0 = d_p = 1/2, else 1 (Berrut & Trefethen, SIAM Review 46 (2004)); L_k(x) = 1 when
 *    x equals s_k, the first such k in index order;
 *  - a cluster is approximated only if, besides the MAC, every node it can hold lies beyond the
 *    near radius with a relative margin: R - r_c > (1 + 1e-4) Rc.  The near sums then see exactly
 *    the nodes within Rc, as in the direct evaluation, and the treecode changes only the far
 *    sum (without this, a cluster that meets the MAC could hold nodes where the regularization
 *    still acts, which the paper's walk would sum unregularized);
 *  - targets with |b| > Rc take plain, unsubtracted sums (no node is within Rc), as in
 *    ora_eval_k.
 *
 * Parity status: pinned by tests/test_oracle_treecode.py (the tree's invariants; the
 * interpolation basis: partition of unity, L_k(s_j) = delta_kj, exact for polynomials of degree
 * <= p; moments of the modified weights up to degree p equal the nodes' moments; theta -> 0 gives
 * the direct evaluation of ora_eval_k; spectral decay of the error with p; the error of the full
 * method on the sphere closed form is unchanged at the paper's parameters).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_TC_PI 3.14159265358979323846

/* from ers_oracle.c */
void ora_sl_term(const double d[3], double r, double delta, double tc, const double g[3], double w,
                 double acc[3], int sharp);
void ora_dl_term(double r, double delta, double tc, double b, const double nrm0[3], const double xh[3],
                 const double Q[3], const double nx[3], double w, double acc[3], int sharp);
void ora_sl_plain(const double d[3], double r, const double g[3], double w, double acc[3]);
void ora_dl_plain(const double d[3], double r, const double Q[3], const double nx[3], double w, double acc[3]);
int ora_extrapolate_k(int K, const double *rho, double b, double h, const double *U, int nrhs, double *out);

#define NW 15 /* modified-weight densities per Chebyshev point: f w (3), n w (3), q_j n_k w (9, j major) */

typedef struct {
    double lo[3], hi[3], c[3], hw[3]; /* box, centre, half-widths */
    double rc;                        /* half the diagonal */
    int64_t start, count;             /* nodes perm[start .. start+count) */
    int64_t child[8];
    int nchild, level;
} ora_clu;

typedef struct {
    ora_clu *cl;
    int64_t ncl, cap;
    int64_t *perm;
    int depth;
} ora_tree;

static int64_t tree_new_cluster(ora_tree *T) {
    if (T->ncl == T->cap) {
        T->cap = T->cap ? 2 * T->cap : 64;
        T->cl = (ora_clu *)realloc(T->cl, sizeof(ora_clu) * T->cap);
    }
    memset(&T->cl[T->ncl], 0, sizeof(ora_clu));
    return T->ncl++;
}

/* Step 1: the cluster of nodes perm[s .. e), then its octants (recursively). */
static int64_t tree_build_rec(ora_tree *T, const double *x, int64_t s, int64_t e, int64_t N0, int level,
                              int64_t *tmp) {
    int64_t id = tree_new_cluster(T);
    ora_clu C;
    memset(&C, 0, sizeof C);
    for (int a = 0; a < 3; ++a) { C.lo[a] = INFINITY; C.hi[a] = -INFINITY; }
    for (int64_t i = s; i < e; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * T->perm[i] + a];
            if (v < C.lo[a]) C.lo[a] = v;
            if (v > C.hi[a]) C.hi[a] = v;
        }
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        C.c[a] = 0.5 * (C.lo[a] + C.hi[a]);
        C.hw[a] = 0.5 * (C.hi[a] - C.lo[a]);
        double ext = C.hi[a] - C.lo[a];
        diag2 += ext * ext;
    }
    C.rc = 0.5 * sqrt(diag2);
    C.start = s;
    C.count = e - s;
    C.level = level;
    if (level > T->depth) T->depth = level;
    if (e - s > N0 && diag2 > 0.0) {
        /* stable partition into the 8 octants */
        int64_t cnt[8] = {0}, off[8];
        for (int64_t i = s; i < e; ++i) {
            const double *p = x + 3 * T->perm[i];
            int o = (p[0] > C.c[0]) | ((p[1] > C.c[1]) << 1) | ((p[2] > C.c[2]) << 2);
            cnt[o]++;
        }
        off[0] = s;
        for (int o = 1; o < 8; ++o) off[o] = off[o - 1] + cnt[o - 1];
        int64_t pos[8];
        memcpy(pos, off, sizeof pos);
        for (int64_t i = s; i < e; ++i) {
            const double *p = x + 3 * T->perm[i];
            int o = (p[0] > C.c[0]) | ((p[1] > C.c[1]) << 1) | ((p[2] > C.c[2]) << 2);
            tmp[pos[o]++] = T->perm[i];
        }
        memcpy(T->perm + s, tmp + s, sizeof(int64_t) * (e - s));
        for (int o = 0; o < 8; ++o) {
            if (cnt[o] == 0) continue;
            int64_t ch = tree_build_rec(T, x, off[o], off[o] + cnt[o], N0, level + 1, tmp);
            C.child[C.nchild++] = ch;
        }
    }
    T->cl[id] = C;
    return id;
}

static void tree_build(ora_tree *T, const double *x, int64_t N, int64_t N0) {
    memset(T, 0, sizeof *T);
    T->perm = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) T->perm[i] = i;
    if (N > 0) tree_build_rec(T, x, 0, N, N0, 0, tmp);
    free(tmp);
}

static void tree_free(ora_tree *T) {
    free(T->cl);
    free(T->perm);
}

/* Chebyshev points of the second kind on [-1, 1]: s_k = cos(k pi / p), k = 0..p. */
void ora_cheb_points(int p, double *s) {
    for (int k = 0; k <= p; ++k) s[k] = cos(k * ORA_TC_PI / p);
}

/*
 * Lagrange basis of degree p at the Chebyshev points of the interval centre c, half-width hw,
 * evaluated at x by the barycentric formula L_k(x) = (w_k/(x - s_k)) / sum_j w_j/(x - s_j)
 * with w_k = (-1)^k d_k (d_0 = d_p = 1/2, else 1); L_k(x) = 1 where x equals s_k.
 */
void ora_lagrange(int p, double c, double hw, double x, double *L) {
    double s[32];
    for (int k = 0; k <= p; ++k) s[k] = c + hw * cos(k * ORA_TC_PI / p);
    for (int k = 0; k <= p; ++k) {
        if (x == s[k]) {
            for (int j = 0; j <= p; ++j) L[j] = (j == k) ? 1.0 : 0.0;
            return;
        }
    }
    double den = 0.0;
    for (int k = 0; k <= p; ++k) {
        double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);
        L[k] = wk / (x - s[k]);
        den += L[k];
    }
    for (int k = 0; k <= p; ++k) L[k] /= den;
}

/* The densities of Eq. (mod_weights) at node j: f w, n w, q_j n_k w. */
static void node_densities(const double *nrm, const double *w, const double *f, const double *q, int64_t j,
                           double g[NW]) {
    for (int i = 0; i < 3; ++i) {
        g[i] = f[3 * j + i] * w[j];
        g[3 + i] = nrm[3 * j + i] * w[j];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g[6 + 3 * a + b] = q[3 * j + a] * nrm[3 * j + b] * w[j];
}

/* Step 2: modified weights of cluster C, Eq. (mod_weights): W[k][i] = sum_{x_j in C} L_k1(x_j1)
 * L_k2(x_j2) L_k3(x_j3) g_i(x_j), k = (k1 (p+1) + k2) (p+1) + k3. */
static void modified_weights(const ora_tree *T, const ora_clu *C, int p, const double *x, const double *nrm,
                             const double *w, const double *f, const double *q, double *W) {
    const int P1 = p + 1, NK = P1 * P1 * P1;
    memset(W, 0, sizeof(double) * NK * NW);
    double L[3][32], g[NW];
    for (int64_t i = C->start; i < C->start + C->count; ++i) {
        int64_t j = T->perm[i];
        for (int a = 0; a < 3; ++a) ora_lagrange(p, C->c[a], C->hw[a], x[3 * j + a], L[a]);
        node_densities(nrm, w, f, q, j, g);
        for (int k1 = 0; k1 <= p; ++k1)
            for (int k2 = 0; k2 <= p; ++k2)
                for (int k3 = 0; k3 <= p; ++k3) {
                    double Lk = L[0][k1] * L[1][k2] * L[2][k3];
                    double *Wk = W + (int64_t)((k1 * P1 + k2) * P1 + k3) * NW;
                    for (int c = 0; c < NW; ++c) Wk[c] += Lk * g[c];
                }
    }
}

typedef struct {
    const double *x, *nrm, *w, *f, *q;
    const ora_tree *T;
    const double *W; /* [ncl][NK][NW] */
    int p;
    double theta, Rc, Racc; /* Racc = (1 + 1e-4) Rc */
    int K;
    const double *rho;
    double h, tc;
} tc_ctx;

typedef struct {
    const double *y, *x0, *n0, *q0;
    double b, fn0;  /* signed distance, f(x0).n0 (0 for plain sums) */
    int subtract;   /* 0: plain sums (|b| > Rc) */
    double far_u[3], far_v[3];
    double near_u[4][3], near_v[4][3];
    int64_t n_approx, n_covered, n_direct, n_near;
} tc_target;

/* Eq. (particle-cluster-KITC): the unregularized Stokeslet and stresslet at the Chebyshev
 * points of C against the modified weights (subtracted as in Eqs. (Stokes_SL1), (Stokes_DL1)). */
static void approx_cluster(const tc_ctx *X, const ora_clu *C, int64_t cid, tc_target *t) {
    const int P1 = X->p + 1, NK = P1 * P1 * P1;
    const double *W = X->W + cid * (int64_t)NK * NW;
    double s[3][32];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k <= X->p; ++k) s[a][k] = C->c[a] + C->hw[a] * cos(k * ORA_TC_PI / X->p);
    for (int k1 = 0; k1 <= X->p; ++k1)
        for (int k2 = 0; k2 <= X->p; ++k2)
            for (int k3 = 0; k3 <= X->p; ++k3) {
                const double *Wk = W + (int64_t)((k1 * P1 + k2) * P1 + k3) * NW;
                double d[3] = {t->y[0] - s[0][k1], t->y[1] - s[1][k2], t->y[2] - s[2][k3]};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                /* single layer: g = f w - (f(x0).n0) n w */
                double g[3];
                for (int i = 0; i < 3; ++i) g[i] = Wk[i] - t->fn0 * Wk[3 + i];
                ora_sl_plain(d, r, g, 1.0, t->far_u);
                /* double layer: -6 d_i d_j d_k (q_j n_k w - q0_j n_k w) / r^5 */
                double r5 = r * r * r * r * r, s2 = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double G = Wk[6 + 3 * a + b] - (t->subtract ? t->q0[a] * Wk[3 + b] : 0.0);
                        s2 += d[a] * d[b] * G;
                    }
                for (int i = 0; i < 3; ++i) t->far_v[i] += -6.0 * d[i] * s2 / r5;
            }
    t->n_approx += 1;
    t->n_covered += C->count;
}

/* A leaf that fails the MAC: direct sums, regularized for the K deltas within Rc (Sec. 3.3). */
static void direct_leaf(const tc_ctx *X, const ora_clu *C, tc_target *t) {
    for (int64_t i = C->start; i < C->start + C->count; ++i) {
        int64_t j = X->T->perm[i];
        const double *xj = X->x + 3 * j, *nj = X->nrm + 3 * j;
        double d[3] = {t->y[0] - xj[0], t->y[1] - xj[1], t->y[2] - xj[2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double g[3], Q[3], xh[3];
        for (int a = 0; a < 3; ++a) {
            g[a] = X->f[3 * j + a] - t->fn0 * nj[a];
            Q[a] = X->q[3 * j + a] - (t->subtract ? t->q0[a] : 0.0);
            xh[a] = xj[a] - (t->subtract ? t->x0[a] : 0.0);
        }
        if (!t->subtract || r > X->Rc) {
            ora_sl_plain(d, r, g, X->w[j], t->far_u);
            ora_dl_plain(d, r, Q, nj, X->w[j], t->far_v);
            t->n_direct += 1;
            continue;
        }
        for (int k = 0; k < X->K; ++k) {
            double delta = X->rho[k] * X->h;
            ora_sl_term(d, r, delta, X->tc, g, X->w[j], t->near_u[k], 0);
            ora_dl_term(r, delta, X->tc, t->b, t->n0, xh, Q, nj, X->w[j], t->near_v[k], 0);
        }
        t->n_near += 1;
    }
}

/* Step 3: the walk from cluster cid. */
static void visit(const tc_ctx *X, int64_t cid, tc_target *t) {
    const ora_clu *C = &X->T->cl[cid];
    double dx = t->y[0] - C->c[0], dy = t->y[1] - C->c[1], dz = t->y[2] - C->c[2];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    if (C->rc <= X->theta * R && R - C->rc > X->Racc) {
        approx_cluster(X, C, cid, t);
        return;
    }
    if (C->nchild == 0) {
        direct_leaf(X, C, t);
        return;
    }
    for (int c = 0; c < C->nchild; ++c) visit(X, C->child[c], t);
}

/*
 * The method with the far sums by the treecode: same arguments and conventions as ora_eval_k
 * (K deltas rho[0..K-1], localized at Rc = tc rho[K-1] h), plus theta, N0, p.  stats (may be
 * NULL): [M][4] per target: clusters approximated, nodes in them, far pairs summed directly,
 * near pairs.
 * Returns the number of failed solves.
 */
int64_t ora_eval_tree(int K, const double *x, const double *nrm, const double *w, const double *f,
                      const double *q, int64_t N, const double *y, const double *x0, const double *n0,
                      const double *b, const double *f0, const double *q0, int64_t M, double h, const double *rho,
                      double tc, double theta, int64_t N0, int p, double *u, double *v, int64_t *stats) {
    const double inv8pi = 1.0 / (8.0 * ORA_TC_PI);
    ora_tree T;
    tree_build(&T, x, N, N0);
    const int P1 = p + 1, NK = P1 * P1 * P1;
    double *W = (double *)malloc(sizeof(double) * (size_t)T.ncl * NK * NW);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < T.ncl; ++c) modified_weights(&T, &T.cl[c], p, x, nrm, w, f, q, W + c * (int64_t)NK * NW);
    tc_ctx X = {x, nrm, w, f, q, &T, W, p, theta, 0.0, 0.0, K, rho, h, tc};
    X.Rc = tc * rho[K - 1] * h;
    X.Racc = (1.0 + 1e-4) * X.Rc;
    int64_t nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nfail)
    for (int64_t m = 0; m < M; ++m) {
        tc_target t;
        memset(&t, 0, sizeof t);
        t.y = y + 3 * m;
        t.x0 = x0 + 3 * m;
        t.n0 = n0 + 3 * m;
        t.q0 = q0 + 3 * m;
        t.b = b[m];
        t.subtract = !(fabs(b[m]) > X.Rc);
        const double *fm0 = f0 + 3 * m;
        t.fn0 = t.subtract ? fm0[0] * t.n0[0] + fm0[1] * t.n0[1] + fm0[2] * t.n0[2] : 0.0;
        if (N > 0) visit(&X, 0, &t);
        if (stats) {
            stats[4 * m] = t.n_approx;
            stats[4 * m + 1] = t.n_covered;
            stats[4 * m + 2] = t.n_direct;
            stats[4 * m + 3] = t.n_near;
        }
        if (!t.subtract) {
            for (int i = 0; i < 3; ++i) { u[3 * m + i] = t.far_u[i] * inv8pi; v[3 * m + i] = t.far_v[i] * inv8pi; }
            continue;
        }
        double chi = (t.b < 0.0) ? 1.0 : ((t.b > 0.0) ? 0.0 : 0.5);
        double U[4][6], out[6];
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < 3; ++i) {
                U[k][i] = (t.far_u[i] + t.near_u[k][i]) * inv8pi;
                U[k][3 + i] = (t.far_v[i] + t.near_v[k][i]) * inv8pi + chi * t.q0[i];
            }
        if (ora_extrapolate_k(K, rho, t.b, h, &U[0][0], 6, out) != 0) nfail += 1;
        for (int i = 0; i < 3; ++i) { u[3 * m + i] = out[i]; v[3 * m + i] = out[3 + i]; }
    }
    free(W);
    tree_free(&T);
    return nfail;
}

/*
 * The octree of step 1, for the tests: returns the number of clusters (or -(needed) when cap is
 * too small).  Per cluster c: box lo/hi [c][3] each, centre/half-width are derived; start, count,
 * level, nchild, parent (-1 for the root); perm[N] = the node order of the leaves.
 */
int64_t ora_tree_info(const double *x, int64_t N, int64_t N0, int64_t cap, double *lo, double *hi, double *rc,
                      int64_t *start, int64_t *count, int64_t *level, int64_t *nchild, int64_t *parent,
                      int64_t *perm) {
    ora_tree T;
    tree_build(&T, x, N, N0);
    int64_t n = T.ncl;
    if (n > cap) {
        tree_free(&T);
        return -n;
    }
    for (int64_t c = 0; c < n; ++c) parent[c] = -1;
    for (int64_t c = 0; c < n; ++c) {
        const ora_clu *C = &T.cl[c];
        for (int a = 0; a < 3; ++a) { lo[3 * c + a] = C->lo[a]; hi[3 * c + a] = C->hi[a]; }
        rc[c] = C->rc;
        start[c] = C->start;
        count[c] = C->count;
        level[c] = C->level;
        nchild[c] = C->nchild;
        for (int k = 0; k < C->nchild; ++k) parent[C->child[k]] = c;
    }
    memcpy(perm, T.perm, sizeof(int64_t) * N);
    tree_free(&T);
    return n;
}

/* Modified weights of every cluster (step 2), [ncl][(p+1)^3][15], for the tests; returns ncl
 * (or -(needed clusters) when cap is too small). */
int64_t ora_tree_weights(const double *x, const double *nrm, const double *w, const double *f, const double *q,
                         int64_t N, int64_t N0, int p, int64_t cap, double *W) {
    ora_tree T;
    tree_build(&T, x, N, N0);
    int64_t n = T.ncl;
    if (n > cap) {
        tree_free(&T);
        return -n;
    }
    const int P1 = p + 1, NK = P1 * P1 * P1;
    for (int64_t c = 0; c < n; ++c) modified_weights(&T, &T.cl[c], p, x, nrm, w, f, q, W + c * (int64_t)NK * NW);
    tree_free(&T);
    return n;
}
