/*
 * ers.h -- C ABI of the GB300 library for the localized extrapolated-regularization method
 * for nearly singular Stokes single- and double-layer integrals (Siebor & Tlupova,
 * "Localized evaluation and fast summation in the extrapolated regularization method for
 * integrals in Stokes flow").
 *
 * What the library computes, for a closed surface Gamma and targets y:
 *   u_i(y) = 1/(8 pi) int S_ij(y,x) f_j(x) dS(x)            (Eq. (Stokes_SL), Stokeslet Eq. (Stokeslet))
 *   v_i(y) = 1/(8 pi) int T_ijk(y,x) q_j(x) n_k(x) dS(x)    (Eq. (Stokes_DL), stresslet Eq. (Stresslet))
 * discretised with the lattice-crossing quadrature of Sec. 2.2 (Eq. (quadrature)).  For a
 * target within Rc = cutoff_t * delta_3 of Gamma it uses the subtracted densities of
 * Eqs. (Stokes_SL1), (Stokes_DL1), the regularized kernels of Eqs. (Sreg), (Treg) with the
 * smoothing functions of Eqs. (s1)-(s3) for three delta_k = rho_k h, and the extrapolation of
 * Eq. (extrap_eqn) with I0, I2 of Eqs. (I0), (I2); the regularization is applied only where
 * r/delta_k <= cutoff_t (Sec. 3.2), and the unregularized far part (nodes with r > Rc) is
 * evaluated once and shared by the three delta_k (Eq. (near_far), Sec. 3.3).  Targets
 * farther than Rc from Gamma get the plain sums of Eqs. (Stokes_SL), (Stokes_DL).
 *
 * Conventions for every entry point:
 *  - Arrays are contiguous, row-major, IEEE double precision unless stated; "dev" arrays are
 *    CUDA device pointers owned by the caller (the library never frees them); points and
 *    vectors are (count, 3).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously on it; results are ready when the stream reaches that point.
 *  - Return value: ERS_OK (0), a positive warning, or a negative ERS_E_* code.  The calling
 *    thread's last message is available from ers_last_error().  No entry point aborts or
 *    throws across the ABI.
 *  - One evaluation at a time per surface: calls that use the same surface on different
 *    streams concurrently race on the surface's work buffers.
 */
#ifndef ERS_H
#define ERS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ERS_OK 0
#define ERS_W_CUTOFF 1        /* warning: cutoff_t < 6 (regularization truncated earlier than Sec. 3.2) */
#define ERS_W_NOT_CONVERGED 2 /* warning: ers_gmres stopped at maxit above the tolerance */
#define ERS_E_INVAL (-1)      /* bad argument (NULL, size, non-finite, unsorted rho, ...) */
#define ERS_E_NOMEM (-2)      /* device or host allocation failed */
#define ERS_E_CUDA (-3)       /* a CUDA call failed; message holds the CUDA error string */
#define ERS_E_TIMEOUT (-4)    /* a bounded device-side wait expired */
#define ERS_E_UNSUPPORTED (-5)/* valid but not supported by the library (e.g. cutoff_t > 8) */
#define ERS_E_STATE (-6)      /* call out of order (e.g. eval before set_density) */

#define ERS_LAYER_SL 1
#define ERS_LAYER_DL 2

#define ERS_OPT_CONCURRENT 1 /* ers_params.options, ERS_PREC_MIXED only: run the far field (FP32
                                pipe) on a second stream of the surface, concurrently with the near
                                field (FP64 pipe), instead of one after the other (see ers_eval) */

#define ERS_OPT_SHARP 2   /* ers_params.options: targets ON the surface (b = 0, see ers_closest_point) use
                             the modified smoothing functions s#_p of Sec. 2.1 with one delta# =
                             rho_sharp h and no extrapolation (single layer: Eq. (Sreg) with s#_1, s#_2;
                             double layer: the stresslet -6 d d d s#_3/r^5), localized at
                             cutoff_t delta#; targets off the surface are unchanged */

#define ERS_OPT_FOUR_DELTA 4 /* ers_params.options: the O(delta^7) variant of the extrapolation that
                                Sec. 1 mentions, with a fourth delta_3 = rho4 h and the error model
                                u^delta = u + c1 rho I0 + c2 rho^3 I2 + c3 rho^5 I4 + O(delta^7),
                                I4(lambda) = (2/15)((3 - 2 lambda^2 + 4 lambda^4) e^{-lambda^2}/sqrt(pi)
                                - 4 |lambda|^5 erfc|lambda|) (the k = 2 moment int_lambda^inf erfc(r)
                                (r^2 - lambda^2)^k dr, of which I0, I2 are k = 0, 1); near radius
                                cutoff_t delta_3.  Not available in the batched, no-allocation and
                                closure paths (ERS_E_UNSUPPORTED) */

#define ERS_OPT_TREECODE 8 /* ers_params.options: the far sums by the kernel-independent treecode of
                              Sec. 3.4 instead of the direct sum: an octree of the nodes (leaves of at
                              most tree_n0), clusters that meet the MAC r_c/R <= tree_theta and lie
                              beyond the near radius (R - r_c > (1 + 1e-4) Rc) summed by barycentric
                              Lagrange interpolation of degree tree_p at Chebyshev points (modified
                              weights of w f, w n, q_j w n_k), other leaves summed directly over their
                              nodes beyond Rc.  The near sums and the extrapolation are unchanged.  The
                              tree is built on the host at the first use for a given tree_n0 and kept
                              with the surface (that call synchronizes the device and allocates: make
                              it before any stream capture); the modified weights are recomputed on
                              `stream` after every ers_set_density or change of tree_p (allocating when
                              tree_p grows).  ERS_OPT_CONCURRENT is ignored.
                              Not available in the batched, no-allocation and closure paths */

#define ERS_PREC_FP64 0   /* far field in FP64; local sums at FP64-level accuracy (pair geometry in
                             FP64, kernel factors and contractions in float-pair arithmetic,
                             ~1e-14 relative), closest point and 3x3 solve in FP64 */
#define ERS_PREC_MIXED 1  /* far field with FP32 operands and FP64 accumulation per source tile;
                             local sums, closest point and 3x3 solve as in ERS_PREC_FP64 */

typedef struct ers_surface ers_surface; /* opaque, library-owned */

/* Ellipsoid sum(((x - center)/axes)^2) = 1; a sphere when the three axes are equal. */
typedef struct {
    double center[3];
    double axes[3];
} ers_shape;

typedef struct {
    double rho[3];    /* delta_k = rho_k h, strictly increasing, > 0 (Sec. 2: typically 3,4,5 or 2,3,4) */
    double cutoff_t;  /* regularize only where r/delta <= cutoff_t; 6 in Sec. 3.2; range (0, 8] */
    int precision;    /* ERS_PREC_FP64 or ERS_PREC_MIXED */
    int layers;       /* bitmask of ERS_LAYER_SL, ERS_LAYER_DL */
    int options;      /* bitmask of ERS_OPT_*; 0 for the defaults */
    double rho_sharp; /* ERS_OPT_SHARP: delta# = rho_sharp h (> 0), or 0 for rho[1] */
    double rho4;      /* ERS_OPT_FOUR_DELTA: delta_3 = rho4 h (> rho[2]), or 0 for 2 rho[2] - rho[1] */
    double tree_theta; /* ERS_OPT_TREECODE: MAC parameter in (0, 1), or 0 for ers_treecode_defaults */
    int tree_n0;       /* ERS_OPT_TREECODE: leaf size >= 1, or 0 for ers_treecode_defaults */
    int tree_p;        /* ERS_OPT_TREECODE: interpolation degree 1..16, or 0 for ers_treecode_defaults */
} ers_params;

/*
 * Build the quadrature of Sec. 2.2 on an ellipsoid with lattice spacing h (> 0): nodes where
 * lattice lines parallel to e_k, through (i h, j h) in the other two coordinates, cross the
 * surface, kept when |n_k| >= cos 70 deg, with weights w = psi_k(n)/|n_k| h^2 from the
 * partition of unity psi_k = beta_k / sum beta_j, beta_j = b(arccos|n_j| / theta),
 * b(r) = exp(2 r^2/(r^2 - 1)) for |r| < 1 (Eq. (quadrature)).  Nodes are in the canonical order
 * k = 1,2,3; first remaining lattice index; second remaining index; lower root first.
 * Allocates device memory on the current device; *out receives the handle.
 * Errors: ERS_E_INVAL (NULL, h <= 0, axes <= 0, non-finite), ERS_E_NOMEM, ERS_E_CUDA.
 */
int ers_build_surface(const ers_shape *shape, double h, ers_surface **out);

/* Release a surface and its device memory; NULL is accepted.  Returns ERS_OK. */
int ers_surface_free(ers_surface *s);

/*
 * Node data in canonical order: *N nodes; *x, *n (N,3) dev, *w (N) dev (pointers remain owned
 * by the surface and valid until ers_surface_free).  Any output pointer may be NULL.
 */
int ers_surface_info(const ers_surface *s, int64_t *N, double *h, const double **x, const double **n,
                     const double **w);

/*
 * Set the densities at the nodes, in canonical order: f for the single layer, q for the
 * double layer, each (N,3) dev; either may be NULL to leave it unchanged.  Copies the data
 * (the caller may free or reuse the arrays once the stream reaches this point).
 */
int ers_set_density(ers_surface *s, const double *f, const double *q, void *stream);

/*
 * Closest point x0 on the surface, outward unit normal n0 there and signed distance b for M
 * targets y (Sec. 2: y = x0 + b n0, b < 0 inside).  |b| <= 1e-12 * (largest semi-axis) is
 * returned as b = 0 (on the surface, chi = 1/2 in Eq. (Stokes_DL1)).  y, x0, n0 (M,3) and
 * b (M) dev.  On the medial set of an ellipsoid one valid closest point is returned.
 * Errors: ERS_E_INVAL, ERS_E_CUDA.
 */
int ers_closest_point(const ers_surface *s, const double *y, int64_t M, double *x0, double *n0, double *b,
                      void *stream);

/*
 * Evaluate the layers selected by p->layers at M targets y (M,3) dev.
 *   x0, n0, b : closest-point data from ers_closest_point (dev), or all three NULL to have
 *               them computed inside this call;
 *   f0, q0    : the densities f and q at the closest points (M,3) dev, as in
 *               Eqs. (Stokes_SL1), (Stokes_DL1); read only for targets with |b| <= Rc and only
 *               for the selected layers (may be NULL when the layer is not selected);
 *   u, v      : outputs (M,3) dev for the single and double layer (NULL when not selected).
 * Requires ers_set_density for the selected layers.  M = 0 is a no-op.
 * All work is ordered after earlier work on `stream` and before later work on it.  With
 * ERS_PREC_MIXED and ERS_OPT_CONCURRENT the far field runs on a second stream owned by the
 * surface, forked from and joined back to `stream` with events (also under stream capture);
 * such calls on one surface must not run concurrently from several streams.
 * Returns ERS_OK, ERS_W_CUTOFF (cutoff_t < 6), or ERS_E_INVAL / ERS_E_STATE / ERS_E_NOMEM /
 * ERS_E_CUDA / ERS_E_UNSUPPORTED.
 */
int ers_eval(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
             const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
             void *stream);

/* Single layer only: ers_eval with layers = ERS_LAYER_SL (p->layers is ignored). */
int ers_eval_SL(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                const double *n0, const double *b, const double *f0, double *u, void *stream);

/* Double layer only: ers_eval with layers = ERS_LAYER_DL (p->layers is ignored). */
int ers_eval_DL(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                const double *n0, const double *b, const double *q0, double *v, void *stream);

/*
 * ers_eval with HOST arrays (any host memory; pinned memory gives faster copies): copies y,
 * f0, q0 (and x0, n0, b when given) to library-owned device buffers on `stream`, evaluates,
 * copies u, v back and synchronizes the stream before returning.
 */
int ers_eval_host(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                  const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                  void *stream);

/*
 * Counts of the most recent ers_eval on this surface, for throughput reporting: number of
 * targets with |b| <= Rc, number of (target, node) pairs in their local (r <= Rc) sums, and
 * the number of far-field pairs.  Synchronizes the stream of that call.
 */
int ers_last_counts(ers_surface *s, int64_t *near_targets, int64_t *near_pairs, int64_t *far_pairs);

/*
 * Per-kernel timing of the following ers_eval calls on this surface: when enabled, CUDA events
 * are recorded on the call's stream around the closest-point, far-field and near-field
 * kernels.  enable = 0 turns it off.  Creates the events on first use (ERS_E_CUDA on failure).
 */
int ers_profile(ers_surface *s, int enable);

/*
 * Kernel durations in milliseconds of the most recent profiled ers_eval on this surface
 * (closest point; far field; near field + extrapolation).  Synchronizes that call's stream.
 * A kernel that did not run reports 0.  When the far and near fields ran concurrently
 * (ERS_OPT_CONCURRENT) both durations are measured from the common start, so they overlap.  ERS_E_STATE if no profiled call happened.
 */
int ers_last_profile(ers_surface *s, double *ms_closest, double *ms_far, double *ms_near);

/*
 * Densities of nrhs right-hand sides at once (nrhs = 1, 2, 4 or 8), canonical node order:
 * f, q (nrhs, N, 3) dev (either may be NULL: that layer's density is then zero).  Used by the
 * batched evaluation; independent of ers_set_density.  Errors: ERS_E_INVAL, ERS_E_NOMEM,
 * ERS_E_CUDA.
 */
int ers_set_density_multi(ers_surface *s, const double *f, const double *q, int nrhs, void *stream);

/*
 * One problem of a batched evaluation: the layers of surface s (densities from
 * ers_set_density_multi) at M targets.  All arrays dev, row-major:
 *   y, x0, n0 (M,3), b (M): targets and their closest-point data on s (ers_closest_point);
 *   f0, q0 (nrhs, M, 3): the densities of each right-hand side at x0 (Eqs. (Stokes_SL1),
 *   (Stokes_DL1)); u, v (nrhs, M, 3): outputs.
 * Several problems may share a surface (e.g. one surface evaluated at its own nodes and at the
 * nodes of a nearby surface); outputs of different problems must not overlap.
 */
typedef struct {
    ers_surface *s;
    int64_t M;
    const double *y, *x0, *n0, *b;
    const double *f0, *q0;
    double *u, *v;
} ers_problem;

typedef struct ers_batch ers_batch; /* opaque plan: work list, device copies, CUDA graph */

/*
 * Plan a batched evaluation of nprob problems with nrhs densities each, sharing the parameters
 * p (p->precision must be ERS_PREC_MIXED: far field with FP32 operands and FP64 accumulation;
 * near sums, closest point data and the solve in FP64, as in ers_eval).  The whole evaluation
 * runs as ONE persistent kernel launch: each work item is (problem, block of 128 targets) and
 * is computed end to end (far field, near field for the three delta_k, extrapolation) by one
 * CTA; CTAs take items from an atomic counter, largest first.  The launch (and the reset of the
 * counter) is captured into a CUDA graph here; ers_batch_launch replays it.  The plan records
 * the pointers of every problem: change the data behind them (new densities through
 * ers_set_density_multi with the same nrhs, new f0, q0) and relaunch, but do not free or move
 * them while the plan exists.  Errors: ERS_E_INVAL, ERS_E_STATE (densities not set with this
 * nrhs), ERS_E_UNSUPPORTED (precision, ERS_OPT_SHARP), ERS_E_NOMEM, ERS_E_CUDA.
 */
int ers_batch_create(const ers_problem *probs, int nprob, const ers_params *p, int nrhs, ers_batch **out);

/* Replay the plan's graph on stream (asynchronous).  ERS_E_INVAL on a NULL plan or another device. */
int ers_batch_launch(ers_batch *b, void *stream);

/* Number of work items and the persistent grid size of a plan. */
int ers_batch_info(const ers_batch *b, int *nitems, int *grid);

/* Release a plan (NULL accepted).  The problems' arrays are not touched. */
int ers_batch_free(ers_batch *b);

/*
 * Learned closure of the near field (a growth item on top of the paper's method).
 *
 * Eq. (extrap_eqn) models the regularized value as u^delta = u + c1 rho I0(lambda) +
 * c2 rho^3 I2(lambda) + O(delta^5) with c1, c2 independent of delta.  The closure evaluates fewer
 * regularized sums over a smaller near set and predicts what they miss:
 *   ndelta = 1: the single sum u^{delta_0} (near set r <= cutoff_t delta_0, a quarter of the
 *     pairs for rho = (2,3,4)); predicted: the whole correction u - u^{delta_0};
 *   ndelta = 2: the two smaller deltas (near set r <= cutoff_t delta_1) combined with weights
 *     beta (sum beta = 1, sum beta rho I0 = 0) into u + gamma c2 (gamma = sum beta rho^3 I2);
 *     predicted: c2.
 * c1 and c2 are linear in the density and fixed by the surface and the density near the closest
 * point x0, so the prediction is a linear map from density jets at x0 whose coefficients a
 * network computes from the local geometry:
 *   frame: t1, t2 the principal directions at x0 (where the principal curvatures agree to 1e-6,
 *     as on a sphere: t1 = n0 x a / |n0 x a|, a = e_x, or e_y when |n0_x| >= 0.9), n0;
 *   geometry (the network's input): lambda_0 = b / delta_0, kappa_1 h >= kappa_2 h (principal
 *     curvatures, positive on a convex surface), rho_0, rho_1;
 *   jets: derivatives of the density's components along t1, t2, n0 with respect to the
 *     tangent-plane coordinates ((x - x0).t1, (x - x0).t2) / h, taken from the least-squares
 *     polynomial of total degree <= 4 fitted to the node values (ers_set_density) within 3.5 h of
 *     x0; single layer: orders 0..2 (18 values, component-major, within a component the
 *     monomial order 1, xi, eta, xi^2, xi eta, eta^2), double layer: orders 1..3 (27 values:
 *     xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta, xi eta^2, eta^3); divided by their largest
 *     magnitude S;
 *   output: c (3 components in the frame) = sum_j A_ej jet_j, the correction divided by S h^p
 *     (p = 1 single layer, p = 0 double layer); for ndelta = 2 the correction is -gamma c2.
 * Network: an MLP 16 -> 64 -> 64 -> 64 -> 96 with GELU (5 inputs and 3 J outputs used, J = 18
 * single, 27 double layer), BF16 weights and activations, FP32 accumulation, on the tensor cores
 * (tcgen05), the head's contraction in FP32.  One network per layer (0 = single, 1 = double).
 * A sample record is 48 floats: [geometry (5) | 0 (11) | jets (J) | 0]; outputs are 4 floats (c, 0).
 * The density jets need targets within cutoff_t delta_{ndelta-1} of the surface (only those carry
 * a correction) and at least 15 nodes within 3.5 h of x0.
 */
typedef struct ers_closure ers_closure;

/* Create the two networks: He-uniform hidden weights drawn from `seed`, zero biases and a zero
 * last layer (an untrained network predicts no correction). */
int ers_closure_create(uint64_t seed, ers_closure **out);
int ers_closure_free(ers_closure *c);

/*
 * Read (get != NULL) and/or replace (set != NULL) the FP32 parameters of one network, host
 * arrays of count = 15648 floats: W1 (64x16), b1 (64), W2 (64x64), b2, W3 (64x64), b3, W4 (96x64),
 * b4 (96), weights row-major [out][in]; rows 3 J..95 of W4 and b4 are unused.
 */
int ers_closure_params(ers_closure *c, int layer, float *get, const float *set, int64_t count);

/* Outputs Y (n, 4) floats dev (c, 0) for sample records X (n, 48) floats dev, on the tensor
 * cores.  A tensor-core wait that expires sets a flag read by ers_closure_status. */
int ers_closure_infer(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream);

/* The same network evaluated with FP32 CUDA-core arithmetic and the same BF16 rounding (a check of
 * the tensor-core kernel; not used by the evaluation path). */
int ers_closure_infer_reference(ers_closure *c, int layer, const float *X, int64_t n, float *Y, void *stream);

/* *timed_out = 1 if a bounded tensor-core wait expired in an inference call (synchronous). */
int ers_closure_status(ers_closure *c, int *timed_out);

/*
 * The extent of the geometry one network was trained on: get and/or set host arrays of 10 floats,
 * lo[5] then hi[5], one pair per input (lambda_0, the two principal curvatures times h, rho_0,
 * rho_1).  ers_closure_train widens the extent to cover every record it trains on (non-finite
 * values are skipped); set replaces it (lo <= hi for every input, else ERS_E_INVAL).  *have (may
 * be NULL) = 1 once the extent is known, 0 before.  Synchronous.
 */
int ers_closure_range(ers_closure *c, int layer, float *get, const float *set, int *have);

/*
 * With the check enabled (the default), ers_eval_learned evaluates every corrected target whose
 * geometry leaves the extent of a network that has one (each input widened by 5 % of its width
 * plus 1e-3 of its magnitude plus 1e-6) with the three-delta method instead of the network: the
 * network is not used where it was not trained (the jets enter linearly and are not checked).
 * enabled = 0 turns the check off.
 */
int ers_closure_set_range_check(ers_closure *c, int enabled);

/* *n = the number of targets of the last ers_eval_learned call that left the extent. */
int ers_closure_last_out_of_range(ers_closure *c, int64_t *n);

/* Loss L = (1/n) sum_s w_s/2 |c_s - t_s|^2 (c_s the network's output for record s, T (n, 4) =
 * (t_s, w_s)) and its gradient G (15648 floats dev) with respect to the FP32 parameters (BF16
 * rounding in the forward pass, straight-through in the backward pass).  X (n,48), T (n,4) floats
 * dev; *loss (host) may be NULL.  Synchronizes when loss is requested. */
int ers_closure_grad(ers_closure *c, int layer, const float *X, const float *T, int64_t n, float *G, double *loss,
                     void *stream);

/* `steps` Adam steps (lr with cosine decay over the call) on minibatches of `batch` samples drawn
 * from (X, T) with a counter-based generator seeded by the closure seed; *final_loss (host, may
 * be NULL) receives the loss of the last minibatch. */
int ers_closure_train(ers_closure *c, int layer, const float *X, const float *T, int64_t n, int steps, int batch,
                      float lr, double *final_loss, void *stream);

/*
 * Training data from the method itself: runs the sums with ndelta deltas (1: delta_0 alone;
 * 2: delta_0, delta_1 with the two-delta weights) at M targets and writes the sample records Xs,
 * Xd (M,48) and targets Ts, Td (M,4) of both networks: the target c in the frame divided by S h^p
 * (p = 1 single layer, 0 double layer) and a sample weight:
 *   ndelta = 1: c = u3 - (one-delta value), weight 1;
 *   ndelta = 2: c = c2 = ((two-delta value) - u3) / gamma, weight (gamma / gamma(0))^2, so that the
 *     loss measures gamma c2, the error of the two-delta value; 0 where |gamma| < 1 % of
 *     |gamma(0)| (there the c2 term vanishes and dividing by gamma only amplifies rounding);
 * weight 0 (and no correction) beyond the reduced near radius or without a density fit.  u3, v3
 * (M,3) dev are the values of ers_eval (three deltas) at the same targets.  valid (M) ints: 1 for
 * targets with a positive weight in either layer.  x0, n0, b from ers_closest_point; both
 * densities must have been set.  ERS_OPT_FOUR_DELTA, ERS_OPT_TREECODE and ERS_OPT_SHARP give
 * ERS_E_UNSUPPORTED.
 */
int ers_closure_data(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                     const double *n0, const double *b, const double *f0, const double *q0, const double *u3,
                     const double *v3, int ndelta, float *Xs, float *Xd, float *Ts, float *Td, int *valid,
                     void *stream);

/*
 * Both layers with the learned closure: far field (precision of p) + one- or two-delta near sums +
 * the networks' correction; targets whose geometry leaves the training extent (ers_closure_range,
 * ers_closure_set_range_check) take the three-delta method instead.  Then a validation: every
 * vstride-th target is also given the three-delta method's value and, per layer, the error
 * max|value - method| / max|method| over that sample is measured with and without the network's
 * correction; a layer keeps the correction only where it lowers that error (else the correction
 * is taken back), and if the lower of the two errors exceeds tol for either layer, the whole call
 * falls back to ers_eval (*fell_back = 1).  val_err[2] (host, may be NULL) receives the errors of
 * the kept values; ers_closure_last_gate reports both errors and the choice.  Synchronizes the
 * stream (to read the validation).  The method's value at the sample and at the targets outside
 * the extent is the closure's sums without the correction plus the difference of the near-field
 * sums with three and with ndelta deltas over the three-delta near radius (the far field is the
 * same in both; at targets between the two near radii the two-delta sums carry the plain sum, so
 * the quadrature error of the subtraction identity there, below 1e-8 of the values, remains).
 * Errors as ers_eval, plus ERS_E_TIMEOUT when a tensor-core wait expired and ERS_E_STATE when a
 * density is missing; ERS_OPT_FOUR_DELTA, ERS_OPT_TREECODE and ERS_OPT_SHARP give
 * ERS_E_UNSUPPORTED.
 */
int ers_eval_learned(ers_surface *s, ers_closure *c, const ers_params *p, const double *y, int64_t M,
                     const double *x0, const double *n0, const double *b, const double *f0, const double *q0,
                     int ndelta, double *u, double *v, double tol, int vstride, double *val_err, int *fell_back,
                     void *stream);

/* The validation of the last ers_eval_learned call (host arrays of 2, layer 0 single, 1 double;
 * any may be NULL): used[l] = 1 if layer l kept the network's correction; err_with[l],
 * err_without[l] = the sample's error with and without it. */
int ers_closure_last_gate(ers_closure *c, int used[2], double err_with[2], double err_without[2]);

/*
 * ers_eval for callers that cannot allocate device memory while they evaluate (a solver that
 * owns a fixed memory pool, a plugin running where cudaMalloc is forbidden or too slow to risk,
 * a real-time loop).  The paper has no counterpart; this is a deployment variant of ers_eval.
 *
 * Same arguments and results as ers_eval, except:
 *  - x0, n0 and b are required (fill them with ers_closest_point, which writes into the
 *    caller's arrays and allocates nothing);
 *  - M must not exceed 524,288 targets per call: the far-field partial sums (6 doubles per
 *    target and source chunk) live in a fixed 24 MiB device array inside the library, and larger
 *    M is rejected with ERS_E_INVAL and a message naming the limit (split the targets across
 *    calls); the sources are split into chunks as in ers_eval, but into at most 524,288 / M;
 *  - ers_last_counts is not updated;
 *  - the far and near fields run one after the other on `stream` (ERS_OPT_CONCURRENT is ignored);
 *  - ERS_OPT_SHARP is rejected with ERS_E_UNSUPPORTED.
 * The call performs no cudaMalloc, cudaFree or other allocating call.  The fixed array (24 MiB
 * of scratch plus the 55 KB smoothing-function table) is part of the library's device image:
 * every GPU on which this entry point is used holds it until the process exits.  The first call
 * on a device does a one-time set-up with that device current (it looks up the array's device
 * address and copies the table into it synchronously); make that first call before any stream
 * capture.  Every call on a device shares the same scratch array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU (different streams, or concurrent host
 * threads) race and give wrong results; serialize them.  The surface itself is built
 * beforehand with ers_build_surface and ers_set_density.
 */
int ers_eval_noalloc(ers_surface *s, const ers_params *p, const double *y, int64_t M, const double *x0,
                     const double *n0, const double *b, const double *f0, const double *q0, double *u, double *v,
                     void *stream);

/*
 * Treecode parameters of Eq. (optimal_params) for lattice spacing h (> 0): theta = 0.6, and
 * N0 = 2000, p = 6 at h = 1/64 with N0 doubling and p growing by 2 per halving of h, held at
 * N0 >= 1000 and 6 <= p <= 16 (Table 2 uses N0 = 1000, p = 6 at h = 1/16 and 1/32).  Host only;
 * any output may be NULL.  ERS_E_INVAL for h <= 0 or non-finite.
 */
int ers_treecode_defaults(double h, double *theta, int *n0, int *p);

/*
 * Treecode statistics of the surface: out[0] clusters, out[1] leaves, out[2] depth of the last
 * tree built (0 if none); out[3] (target, cluster) pairs approximated and out[4] far pairs summed
 * directly by the last ERS_OPT_TREECODE evaluation (synchronizes with it).  n >= 5.
 * ERS_E_TIMEOUT if a bounded wait of that evaluation's staging copies ran out (its result is then
 * invalid).
 */
int ers_tree_stats(ers_surface *s, int64_t *out, int n);

/*
 * Value at M points x0 on the surface (device (M,3), with their unit normals n0) of a density
 * known at the nodes (vals: device (N,3), canonical node order): the least-squares polynomial of
 * total degree <= 4 in tangent-plane coordinates fitted to the node values within 3.5 h of the
 * point, evaluated at the point (an O(h^5) approximation; exact for that polynomial space).  This
 * supplies q(x0) of Eq. (Stokes_DL1) when a density is known only at the nodes, as for the
 * velocity of the other drop in Eq. (IE-2Surf).  out: device (M,3); a point with fewer than 15
 * nodes within 3.5 h (or a singular fit) gets NaN.  Asynchronous on `stream`.
 */
int ers_node_interp(const ers_surface *s, const double *vals, const double *x0, const double *n0, int64_t M,
                    double *out, void *stream);

/* y = a x + b y for device vectors of length n (asynchronous on `stream`). */
int ers_vec_axpby(int64_t n, double a, const double *x, double b, double *y, void *stream);

/*
 * GMRES (Saad & Schultz 1986) without restart for A x = b with device vectors of length n,
 * starting from x = 0: Arnoldi with modified Gram-Schmidt (inner products by a deterministic
 * two-stage reduction), the least-squares problem by Givens rotations.  A(ctx, v, w, stream)
 * must write A v into w (both device, length n) on `stream` and return 0 (or a negative
 * ERS_E_* code, which ends the solve).  Stops when ||b - A x|| <= tol ||b|| or after maxit
 * iterations; *iters and *relres (may be NULL) receive the iterations and the relative residual
 * of the least-squares problem.  Workspace (maxit + 2) n doubles is allocated and freed inside.
 * Returns ERS_OK, ERS_W_NOT_CONVERGED, or an error code; synchronizes `stream`.
 */
typedef int (*ers_matvec_fn)(void *ctx, const double *x, double *y, void *stream);
int ers_gmres(int64_t n, ers_matvec_fn A, void *ctx, const double *b, double *x, double tol, int maxit, int *iters,
              double *relres, void *stream);

/* Message of the last error on the calling thread ("" if none).  Never NULL. */
const char *ers_last_error(void);

/* Library version string. */
const char *ers_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ERS_H */
