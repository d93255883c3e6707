/*
 * vpx.h -- C ABI of the GB300 library for the particular-solution stage of the
 * FMM-accelerated Poisson solver with function extension (Fryklund &
 * Greengard, arXiv 2211.14537):
 *
 *   (a) extension of the source f from the interior of Omega to the
 *       boundary-cut leaves and their extension lists (Sections 3.2, 4.1);
 *   (b) the volume potential  V[f^e](x) = (1/2pi) int_E log|x-y| f^e(y) dy
 *       (eq. volinte) at every leaf node of an adaptive, level-restricted
 *       quad-tree and at the Gauss-Legendre nodes of the boundary panels
 *       (Section 4.1, last paragraph; Section 5, boundary nodes y_ij).
 *
 * Conventions shared by every call
 *   - Every function returns an int status: VPX_OK (0) or a negative
 *     VPX_ERR_* code; nothing throws across the ABI.  vpx_error_string()
 *     names a code; vpx_last_error_message() gives detail for this thread.
 *   - D = [-0.5, 0.5]^2 is the root box (Section 4: Omega and the support E
 *     of f^e lie inside the unit square centred at the origin).
 *   - Points are interleaved (x, y) doubles.  Leaves are listed in Z-order
 *     (depth first, children SW, SE, NW, NE); the K*K nodes of a leaf are
 *     Gauss-Legendre tensor nodes, node (a, b) at index b*K + a (x varies
 *     fastest).
 *   - Right-hand sides are columns: column r of an input/output array starts
 *     at ptr + r*ld.  Device pointers are raw CUDA device addresses; the
 *     caller allocates and owns them.  `stream` is a cudaStream_t (NULL =
 *     legacy default stream).  Device calls are asynchronous on `stream`;
 *     kernel-side errors are latched in a device status word that
 *     vpx_sync_status() reads after synchronising the stream.
 *   - A plan owns every device buffer it allocates (tree, lists, tables,
 *     extension operators, workspace) and frees them in vpx_plan_destroy().
 *   - A plan is used by one host thread at a time.
 */
#ifndef VPX_H
#define VPX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define VPX_OK             0
#define VPX_ERR_ARG       -1  /* invalid argument (null pointer, bad size, bad option) */
#define VPX_ERR_CUDA      -2  /* a CUDA runtime call failed */
#define VPX_ERR_NOMEM     -3  /* host or device allocation failed */
#define VPX_ERR_STENCIL   -4  /* the extension stencil cannot be formed (a cut leaf without interior points;
                                 ext_mode 1: a ray point outside Omega or at the origin) */
#define VPX_ERR_DOMAIN    -5  /* the extension square of a cut leaf leaves D */
#define VPX_ERR_LEVEL     -6  /* refinement would exceed the compiled maximum level */
#define VPX_ERR_TIMEOUT   -7  /* a bounded device wait gave up */
#define VPX_ERR_NAN       -8  /* non-finite value detected in input or output */
#define VPX_ERR_CALLBACK  -9  /* a user callback returned non-zero */
#define VPX_ERR_STATE    -10  /* call not valid for this plan (e.g. host-only plan) */
#define VPX_ERR_NODEV    -11  /* no CUDA device available */

/* ----------------------------------------------------------------- options */
#define VPX_PREC_FP64   0   /* every step in FP64 */
#define VPX_PREC_MIXED  1   /* near-field and M2L contractions on tensor cores with exact bf16 slices */

#define VPX_PLAN_HOST_ONLY 1u /* build tree, lists and stencil on the host only; no device work */

typedef struct {
    int    K;            /* leaf nodes per dimension (Gauss-Legendre), 4..16, even */
    int    min_level;    /* every box above this level is split (uniform base) */
    int    max_level;    /* no box is split below this level (<= 15) */
    double refine_tol;   /* resolution tolerance (0: uniform tree at min_level) */
    double f_scale;      /* tolerance is relative to this magnitude of f (> 0) */
    int    p;            /* multipole / local expansion order (terms 0..p), 8..60 */
    int    precision;    /* VPX_PREC_FP64 or VPX_PREC_MIXED */
    int    max_rhs;      /* largest nrhs a later vpx_execute may pass */
    int    n_quad_bdry;  /* Gauss-Legendre nodes per boundary panel (default 16) */
    double rbf_eps;      /* shape parameter of the Gaussians on the unit box (Section 3.1): 0 (default)
                            = their flat limit, the polynomial interpolant at G; up to 1e-3 otherwise
                            (the paper uses ~1e-5), K = 6, 8 or 16 */
    int    ext_mode;     /* 0 (default): universal-stencil extension (Section 3.2); 1: extension along
                            lines through the origin (Section 6.4: Floater-Hormann, degree 3, eight
                            points per line over one leaf side); Omega must be star-shaped about the
                            origin, else plan creation fails with VPX_ERR_STENCIL.  With ext_mode 0 a
                            cut leaf whose interior points do not determine P_q (fewer than N_G of
                            them, or a rank-deficient A_I) takes the minimum-norm least-squares fit:
                            singular values below 1e-13 of the largest are dropped */
} vpx_options;

/* ---------------------------------------------------------------- callbacks
 * All return 0 on success; non-zero aborts plan creation with VPX_ERR_CALLBACK.
 *   vpx_points_cb: out[i] = f(xy[2i], xy[2i+1]) for i < n  (the source used
 *                  for adaptive refinement; may be called outside Omega).
 *   vpx_inside_cb: inside[i] = 1 iff point i lies strictly inside Omega.
 *   vpx_curve_cb : for panel `panel` (0-based) and n parameters t[k] in [-1,1],
 *                  xy[2k..] = gamma_panel(t[k]), dxy[2k..] = gamma_panel'(t[k]).
 */
typedef int (*vpx_points_cb)(const double *xy, int64_t n, double *out, void *ctx);
typedef int (*vpx_inside_cb)(const double *xy, int64_t n, uint8_t *inside, void *ctx);
typedef int (*vpx_curve_cb)(int panel, const double *t, int n, double *xy, double *dxy, void *ctx);

typedef struct vpx_plan *vpx_plan_t;

/* Fill `opt` with defaults (K=8, levels 4/4, p=44, FP64, max_rhs=1, 16 boundary nodes). */
int vpx_default_options(vpx_options *opt);

/*
 * Build the plan for one geometry (Section 4): the adaptive quad-tree
 * (resolution and cut-size refinement, 2:1 level restriction, extension
 * restriction), leaf classification and extension lists, the universal
 * stencil of every cut leaf and its least-squares extension operator
 * (Section 3.2), the near-field, expansion and translation tables of the box
 * FMM, the interaction lists (built on the host and uploaded), and the
 * boundary nodes.
 * n_panels may be 0 (no boundary: every leaf must then be regular).
 * flags: 0 or VPX_PLAN_HOST_ONLY.  On success *out owns all resources.
 */
int vpx_plan_create(const vpx_options *opt, int n_panels, vpx_curve_cb curve, vpx_inside_cb inside,
                    vpx_points_cb refine_f, void *ctx, unsigned flags, vpx_plan_t *out);

/* Sizes: leaves, leaf nodes (n_leaves*K*K), stencil points (length of the f
 * input column), boundary nodes (n_panels * n_quad_bdry).  Any pointer may be NULL. */
int vpx_plan_sizes(vpx_plan_t plan, int64_t *n_leaves, int64_t *n_leaf_nodes, int64_t *n_stencil,
                   int64_t *n_bdry);

/* Host copies of the leaf table, each of length n_leaves (any may be NULL):
 * level, ix, iy (box = [-0.5+ix*s, -0.5+(ix+1)*s] x ..., s = 2^-level),
 * cls (0 regular, 1 cut, 2 exterior), owner (exterior leaves: the leaf index
 * of the cut leaf whose extension list holds it, else -1). */
int vpx_plan_leaves(vpx_plan_t plan, int32_t *level, int32_t *ix, int32_t *iy, int32_t *cls, int32_t *owner);

/* Host array of 2*n_stencil doubles: every point where f must be supplied --
 * the K*K nodes of each regular leaf (leaf order), then for each cut leaf
 * (leaf order) its interior stencil points X_S^I, X_Sbar^I, G^I (Section 3.2). */
int vpx_stencil_points(vpx_plan_t plan, double *xy);

/* Host array of 2*n_leaf_nodes doubles: all target nodes, leaf-major. */
int vpx_leaf_nodes(vpx_plan_t plan, double *xy);

/* Host array of 2*n_bdry doubles: boundary nodes gamma_i(t_j), j fastest. */
int vpx_boundary_nodes(vpx_plan_t plan, double *xy);

/* Interaction-list counts of the plan (host): near pairs, M2L (list i)
 * pairs, S2L (list i+) pairs, M2T (list i-) pairs, boxes, levels.  Any may be NULL. */
int vpx_plan_list_counts(vpx_plan_t plan, int64_t *near, int64_t *m2l, int64_t *s2l, int64_t *m2t,
                         int64_t *n_boxes, int32_t *n_levels);

/* Host copies of the fixed-slot interaction lists (-1 = empty slot), for
 * inspection and tests: near (n_leaves x 33: the source leaf of each of the
 * 9 colleague, 12 coarse and 12 fine configurations), list i (n_boxes x 40
 * offsets), list i+ (n_boxes x 20), list i- (n_leaves x 20), and the boxes
 * (level, ix, iy, leaf index or -1), n_boxes each.  Any pointer may be NULL. */
int vpx_plan_lists(vpx_plan_t plan, int32_t *near, int32_t *vlist, int32_t *xlist, int32_t *wlist,
                   int32_t *box_level, int32_t *box_ix, int32_t *box_iy, int32_t *box_leaf);

/* The universal extension operator A_{X,G} = Phi_{X,G} Phi_{G,G}^{-1}
 * (Section 3.1, eq. defA) that plans of leaf order K and shape parameter
 * rbf_eps use, on the reference extension square [-1,1]^2: *nx x *ng doubles,
 * row-major (rows X_S, X_Sbar, G; columns G), written to `out` when non-NULL.
 * rbf_eps = 0 is the flat limit; rbf_eps > 0 adds (rbf_eps / 2)^2 A2, the
 * eps^2 term of the Gaussian operator, from a table precomputed in
 * multiprecision (unit box of side 1 = half the reference square).  Host only;
 * no plan needed.  Errors: VPX_ERR_ARG (bad K or rbf_eps, null nx / ng). */
int vpx_universal_matrix(int K, double rbf_eps, double *out, int64_t *nx, int64_t *ng);

/* The operator of the extension along lines (ext_mode 1, Section 6.4), for
 * inspection and tests: one entry per exterior grid point of every cut leaf,
 * *n_ray in all.  ray_c: the cut leaf's index among the cut leaves; ray_g: the
 * grid index by*Kbar + ax; ray_src: position of the first of its eight line
 * points in the f column; coef (8 per entry): the grid value is
 * sum_q coef[q] f[ray_src + q].  Pass NULL arrays to get *n_ray first.
 * Errors: VPX_ERR_ARG (null plan or n_ray), VPX_ERR_STATE (ext_mode 0). */
int vpx_plan_ray_operator(vpx_plan_t plan, int64_t *n_ray, int32_t *ray_c, int32_t *ray_g, int64_t *ray_src,
                          double *coef);

/* Host copy of the near-field tables (33 x K*K x K*K doubles): entry
 * [c][i][j] = int over the source box [-1,1]^2 of log|x_i - y| l_j(y) dy, x_i the
 * i-th target node of configuration c in source reference coordinates
 * (Section 4, near-neighbour tables).  Device plans only. */
int vpx_plan_near_tables(vpx_plan_t plan, double *out);

/*
 * The hot path: the extension of Section 3.2 on the cut leaves and their
 * extension lists (f^e at every leaf node), then the box FMM of Section 4.1,
 * V[f^e] (eq. volinte) at every leaf node and boundary node.
 * f_stencil: device, nrhs columns of n_stencil values in vpx_stencil_points
 * order (ld_f >= n_stencil).  v_leaf: device, nrhs columns of n_leaf_nodes
 * values, leaf-major (ld_v >= n_leaf_nodes).  v_bdry: device, nrhs columns of
 * n_bdry values (ld_b >= n_bdry); may be NULL.  The caller owns all three.
 * Asynchronous on `stream`; the first call with a given set of pointers,
 * strides, nrhs and stream captures a CUDA graph, later calls replay it.
 * Errors: VPX_ERR_ARG (null plan or buffer, nrhs outside 1..opt.max_rhs,
 * short leading dimension; nothing is launched), VPX_ERR_STATE (host-only
 * plan), VPX_ERR_CUDA.  Non-finite output (VPX_ERR_NAN) and a bounded wait
 * that gave up (VPX_ERR_TIMEOUT) are latched on the device and returned by
 * vpx_sync_status.
 */
int vpx_execute(vpx_plan_t plan, const double *f_stencil, int nrhs, int64_t ld_f,
                double *v_leaf, int64_t ld_v, double *v_bdry, int64_t ld_b, void *stream);

/*
 * Many trees at once (uneven batches): vpx_execute for n plans, captured into
 * one CUDA graph on `stream` and replayed while the plans and buffers stay the
 * same.  Each plan's passes run on that plan's own streams, forked from and
 * joined back to `stream`, so small and large trees overlap.  Arrays have n
 * entries each; entry i has the meaning of the same argument of vpx_execute
 * for plans[i] (v_bdry[i] may be NULL).  The paper solves one tree at a time;
 * batching is this library's.  Errors: VPX_ERR_ARG (null arrays, n < 1, a plan
 * listed twice, a bad entry: nothing is launched), VPX_ERR_STATE (host-only
 * plan), VPX_ERR_CUDA.  A NULL stream runs the plans one after the other
 * without a graph.
 */
int vpx_execute_batch(int n, vpx_plan_t const *plans, const double *const *f_stencil, const int *nrhs,
                      const int64_t *ld_f, double *const *v_leaf, const int64_t *ld_v, double *const *v_bdry,
                      const int64_t *ld_b, void *stream);

/*
 * Autotuner: picks, for every mixed-form pass that two engines or two tile
 * widths can run, the choice that makes the whole step fastest on this
 * plan's own data (the near field on tcgen05 or on mma.sync; 8 or 32 pairs per
 * mma.sync tile).  It runs one execute on f_stencil (device, nrhs columns,
 * ld_f) into internal buffers and records the pass calls.  It checks every
 * candidate against the default choice to 1e-12 of the maximum, with outputs
 * in scratch memory.  Then, pass by pass, it times replays of the captured
 * execute graph under each candidate and keeps the fastest (one sweep of
 * coordinate descent; a candidate replaces the current choice only if its step
 * is at least 3 % shorter).  Choices are cached per pass-shape signature for the
 * process, and later executes and graphs use them.  Synchronises `stream`;
 * allocates and frees device scratch.  *n_passes and *n_changed (either may
 * be NULL) receive the passes tuned and those whose choice differs from the
 * default.  The paper has no counterpart: schedules and tile shapes are this
 * library's.  Errors: VPX_ERR_ARG; VPX_ERR_STATE (a host-only plan, or a
 * candidate that disagrees with the default, in which case the defaults are
 * kept); VPX_ERR_CUDA; VPX_ERR_NOMEM.  An FP64-form plan has nothing to tune
 * (VPX_OK, 0 passes).
 */
int vpx_autotune(vpx_plan_t plan, const double *f_stencil, int nrhs, int64_t ld_f, void *stream, int *n_passes,
                 int *n_changed);

/*
 * The same for a batch (arrays of n entries, as in vpx_execute_batch): each
 * pass role, meaning the same pass of every plan (near field, M2L, ...), gets
 * one choice for all plans.  The choice is timed on replays of the batch
 * graph, so that it suits trees that run side by side.  Not cached.
 */
int vpx_autotune_batch(int n, vpx_plan_t const *plans, const double *const *f_stencil, const int *nrhs,
                       const int64_t *ld_f, void *stream, int *n_passes, int *n_changed);

/* Extension only (Section 3.2): f^e at all leaf nodes (device, nrhs columns,
 * ld_fe >= n_leaf_nodes; f_stencil as in vpx_execute).  Errors as in vpx_execute. */
int vpx_extend(vpx_plan_t plan, const double *f_stencil, int nrhs, int64_t ld_f,
               double *fe_leaf, int64_t ld_fe, void *stream);

/* Volume potential only (the box FMM of Section 4.1, eq. volinte) for given
 * leaf-node values fe_leaf (device, nrhs columns of n_leaf_nodes values,
 * leaf-major, ld_fe >= n_leaf_nodes); outputs as in vpx_execute.  Errors as in
 * vpx_execute. */
int vpx_potential(vpx_plan_t plan, const double *fe_leaf, int nrhs, int64_t ld_fe,
                  double *v_leaf, int64_t ld_v, double *v_bdry, int64_t ld_b, void *stream);

/* Volume potential with no device allocation at call time (no counterpart in
 * the paper: a deployment variant of vpx_potential).  Same arguments and
 * result as vpx_potential, but the multipole and local expansions live in a
 * file-scope device array of VPX_STATIC_SCRATCH_DOUBLES doubles (16 MiB) that
 * every GPU loading the library holds until exit, instead of the plan's
 * workspace.  For callers that cannot call cudaMalloc at this point (a pool
 * allocator owns the device, or an allocation or its failure is unacceptable
 * mid-run).  The first call on a device looks up the array's device address
 * (once per device); make that first call before any stream capture.
 * Returns VPX_ERR_ARG, before any device work, when nrhs is outside
 * [1, max_rhs] (the mixed form's slice buffers are plan workspace sized by
 * max_rhs) or when nrhs * n_boxes * 4 * (p + 1) exceeds the array.  The
 * passes zero both expansion arrays at the start of every call.
 * All calls share the array: calls that overlap on the GPU (any stream, any
 * plan) race and must be serialised by the caller. */
#define VPX_STATIC_SCRATCH_DOUBLES (2 * 1024 * 1024)
int vpx_potential_static(vpx_plan_t plan, const double *fe_leaf, int nrhs, int64_t ld_fe,
                         double *v_leaf, int64_t ld_v, double *v_bdry, int64_t ld_b, void *stream);

/* ------------------------------------------------ boundary correction (host part)
 * Dirichlet problem (Section 5): u = V[f^e] + D[sigma] (+ the log terms of
 * multiply connected and exterior domains, Section 2), with D the double
 * layer of eqs. dlpot / dblker discretised on the panels' Gauss-Legendre
 * nodes (eq. discdblpotpanel).  The panels form closed curves, each
 * counter-clockwise, numbered curve by curve; D uses each curve's outward
 * normal, so the limit from Omega is -1/2 sigma + D sigma on Omega's outer
 * boundary and +1/2 sigma + D sigma on a curve that Omega surrounds (a hole,
 * or an inclusion of an exterior problem).
 *
 * vpx_bie_setup computes, once per plan, the Nystrom geometry, the curves and
 * the side of Omega at each (one call of `inside` at a point just off every
 * curve), and the product-integration corrections (Helsing-Ojala, Section 5)
 * for every leaf node within reach of a panel (|zeta| < 2 in the panel's
 * coordinates).  Host work only; threads on all cores.  Errors: VPX_ERR_ARG
 * (null argument), VPX_ERR_CALLBACK, VPX_ERR_STATE (no panels; panel ends
 * that do not close into curves; a clockwise curve; two outer curves).  A
 * leaf node exactly on the boundary has no defined correction. */
int vpx_bie_setup(vpx_plan_t plan, vpx_inside_cb inside, void *ctx);

/* The curves found by vpx_bie_setup: their number, the outer one (-1 for an
 * exterior problem), and per boundary node its curve and jump (+-1/2).
 * curve_of_node and jump may be NULL.  Errors: VPX_ERR_ARG, VPX_ERR_STATE. */
int vpx_bie_topology(vpx_plan_t plan, int *n_curves, int *outer_curve, int32_t *curve_of_node, double *jump);

/* The log terms: one per curve that Omega surrounds, centred at the curve's
 * area centroid (which must lie outside Omega); n_unknowns = n_bdry + n_log,
 * the length of the solution vector of vpx_bie_solve.  curve (n_log) and
 * centre (2 n_log) may be NULL.  Errors: VPX_ERR_ARG, VPX_ERR_STATE. */
int vpx_bie_log_terms(vpx_plan_t plan, int *n_log, int32_t *curve, double *centre, int64_t *n_unknowns);

/* Solve for the density and the log coefficients (device plans; the system
 * was assembled and inverted on the device by vpx_bie_setup, Gauss-Jordan
 * with partial pivoting):  boundary rows  jump sigma + D sigma
 * [+ (1/2pi) int sigma, exterior] + sum_k A_k log|y - s_k| = g - vb;  one
 * zero-circulation row per hole (for an exterior problem per inclusion but
 * the last) and, for an exterior problem, sum_k A_k = growth, the coefficient
 * of log|x| that u - V must have at infinity (A - Q, Section 2).
 *   g, vb  device, n_bdry doubles: Dirichlet data and V at the boundary nodes
 *   sol    device, n_unknowns doubles, written: sigma (panel-major), then A_k
 * One right-hand side; two launches on `stream`.  The plan holds one
 * right-hand-side buffer: calls on one plan must be serialised (one stream).
 * Errors: VPX_ERR_ARG, VPX_ERR_STATE (host-only plan, no setup). */
int vpx_bie_solve(vpx_plan_t plan, const double *g, const double *vb, double growth, double *sol, void *stream);

/* u = V + D[sigma] + sum_k A_k log|x - s_k| [+ (1/2pi) int sigma, exterior]
 * at every leaf node: the kernel summed over all boundary nodes in FP64, plus
 * the product-integration corrections of the panels near each node.  At leaf
 * nodes outside Omega the value is that of the same formula there, not u.
 *   sol    device, n_unknowns doubles (vpx_bie_solve's output)
 *   v_leaf device, n_leaf_nodes doubles (V, e.g. vpx_potential's output)
 *   u_leaf device, n_leaf_nodes doubles, written (may equal v_leaf)
 * Errors: VPX_ERR_ARG, VPX_ERR_STATE. */
int vpx_bie_eval(vpx_plan_t plan, const double *sol, const double *v_leaf, double *u_leaf, void *stream);

/* Each boundary node's double-layer term (density 1) as a multipole of the
 * leaf that holds it, in the box FMM's scaled form: for a leaf of side L and
 * centre c, Phi(z) = a_0 log(z - c) + sum_{k>=1} at_k (L / (z - c))^k with
 * (1/2pi) Re Phi the potential; here a_0 = 0 and at_k = -i gamma'(t_j) w_j
 * (1/L) ((y - c) / L)^(k-1) (complex, stored Re, Im).  *n_coef = 2(p + 1)
 * doubles per node; out (n_bdry x n_coef, row-major) may be NULL.  These are
 * the source terms through which the density enters the FMM passes.
 * Errors: VPX_ERR_ARG, VPX_ERR_STATE (vpx_bie_setup has not run). */
int vpx_bie_dipole_multipoles(vpx_plan_t plan, int *n_coef, double *out);

/* Per boundary node (n_bdry of them, panel-major): the outward unit normal
 * (nu, 2 doubles), s*w = |gamma_i'(t_j)| times the Gauss-Legendre weight, and
 * the signed curvature (gamma'' from differentiating the degree-(nq-1)
 * interpolant of gamma' on the panel).  Host arrays; any may be NULL.
 * Errors: VPX_ERR_ARG, VPX_ERR_STATE (vpx_bie_setup has not run). */
int vpx_bie_geometry(vpx_plan_t plan, double *nu, double *sw, double *kappa);

/* The corrections in CSR form over the leaf nodes: *n_corr entries; off
 * (n_leaf_nodes + 1), panel (n_corr) and w (n_corr x nq, row-major) may each
 * be NULL (call once with all NULL for the count).  For leaf node q,
 * D[sigma](x_q) = sum_b K(x_q, y_b) s_b w_b sigma_b
 *               + sum_{e in [off[q], off[q+1])} sum_j w[e][j] sigma[panel[e] * nq + j],
 * K the kernel of eq. dblker.  Errors: VPX_ERR_ARG, VPX_ERR_STATE. */
int vpx_bie_corrections(vpx_plan_t plan, int64_t *n_corr, int64_t *off, int32_t *panel, double *w);

/* Net charge of the extended source (Section 6.2): A^e = the integral of f^e
 * over its support, by each leaf's tensor Gauss-Legendre rule.  Far from D the
 * potential V[f^e] grows like (A^e / 2 pi) log|x|, which an exterior solver
 * takes out of its condition at infinity.
 *   fe_leaf  device, leaf values in the layout vpx_extend writes (column r at
 *            fe_leaf + r * ld_fe, ld_fe >= n_leaf_nodes); read only
 *   charge   device, nrhs doubles, written
 * Two launches on `stream`, no synchronisation; the summation order is fixed,
 * so equal inputs give bit-equal results.  Errors: VPX_ERR_ARG (null pointer,
 * nrhs outside [1, max_rhs], ld_fe too small), VPX_ERR_STATE (host-only plan). */
int vpx_net_charge(vpx_plan_t plan, const double *fe_leaf, int nrhs, int64_t ld_fe, double *charge, void *stream);

/* End to end with HOST buffers (contiguous columns of n_stencil, n_leaf_nodes
 * and n_bdry doubles; v_bdry_host may be NULL): copies f in, runs vpx_execute
 * on the plan's own stream, copies V out and synchronises.  Errors as in
 * vpx_execute; the latched device status (VPX_ERR_NAN, VPX_ERR_TIMEOUT) is
 * read by a following vpx_sync_status. */
int vpx_execute_host(vpx_plan_t plan, const double *f_stencil_host, int nrhs,
                     double *v_leaf_host, double *v_bdry_host);

/* Synchronise the plan's last stream and return the latched device status
 * (VPX_OK, VPX_ERR_NAN, VPX_ERR_TIMEOUT, ...); clears it. */
int vpx_sync_status(vpx_plan_t plan);

/* Per-pass device times (ms) of the last vpx_execute when timing is enabled
 * (vpx_set_timing(plan, 1)); n <= VPX_N_PASSES entries are written. */
#define VPX_N_PASSES 8
int vpx_set_timing(vpx_plan_t plan, int enable);
int vpx_get_timings(vpx_plan_t plan, double *ms, int n);

/* Names of the passes timed by vpx_get_timings, in order. */
const char *vpx_pass_name(int i);

/* Number of kernel launches in the CUDA graph that vpx_execute captured for
 * its last buffer set (0 before the first captured call, or when the calls
 * run without a graph).  The paper has no counterpart: it reports what one
 * execute launches, for measurement.  Errors: VPX_ERR_ARG for a null
 * argument. */
int vpx_graph_kernel_count(vpx_plan_t plan, int64_t *kernels);

/* Exercise the bounded-wait path of the tensor-core engines on device 0's
 * current context: a kernel waits on a barrier that nothing completes, gives up
 * after 20 ms of wall-clock time and latches VPX_ERR_TIMEOUT, which is
 * returned in *status (VPX_ERR_TIMEOUT expected).  The paper has no
 * counterpart; it is the library's self-check of its failure detection.  Errors:
 * VPX_ERR_ARG for a null argument, VPX_ERR_CUDA / VPX_ERR_NODEV. */
int vpx_check_bounded_wait(int *status);

/* Invert the n x n row-major host matrix a into inv (host, n x n) with the
 * device Gauss-Jordan elimination that vpx_bie_setup runs on the Nystrom
 * system (partial pivoting, one pivot column per step), on the current
 * device.  *status receives 0, or VPX_ERR_STATE when a pivot column is zero
 * or not a number (a singular matrix): the elimination then stops, and inv
 * holds no inverse.  The paper has no counterpart; it is the library's
 * self-check of its inversion and of that stop.  Errors: VPX_ERR_ARG (a null
 * argument, n < 1), VPX_ERR_CUDA, VPX_ERR_NODEV, VPX_ERR_NOMEM. */
int vpx_check_gauss_jordan(int n, const double *a, double *inv, int *status);

const char *vpx_error_string(int code);
const char *vpx_last_error_message(void);

void vpx_plan_destroy(vpx_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* VPX_H */
