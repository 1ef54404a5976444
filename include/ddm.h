/*
 * ddm.h - C ABI of the GB300 (sm_103a) fast multipole, fully coupled
 * poroelastic displacement discontinuity method (2D, constant spatial and
 * constant temporal elements).
 *
 * The library computes the matrix-free influence product of paper
 * Eqs. (2.3)-(2.5) - stress (sigma_s, sigma_n) and pore pressure p at every
 * element midpoint caused by shear DD, normal DD and fluid source on every
 * element - with the black-box (Chebyshev) fast multipole method of paper
 * Sec. 3, and uses it in the two places of the paper's algorithm (Sec. 4):
 * the time-marching history sum and the GMRES solve of each time step.
 *
 * Conventions (all calls):
 *   - SI units; tension-positive stress; pore pressure positive.
 *   - Element e runs from (x0[e], y0[e]) to (x1[e], y1[e]); its tangent t
 *     points from the first to the second end point, its normal n is t
 *     rotated by +90 degrees.  D = u(+) - u(-), + face on the side n points
 *     to; D_n > 0 opens the crack.  D_q is the fluid source strength per unit
 *     element length (m^2/s per m).
 *   - Unknown vectors have 3N doubles in blocks [Ds(N), Dn(N), Dq(N)];
 *     result vectors have 3N doubles [sigma_s(N), sigma_n(N), p(N)], each at
 *     the element midpoint, stresses resolved in that element's (t, n) frame.
 *   - K(tau) is the response to a source switched on at time 0 and held,
 *     observed at time tau (K(tau <= 0) = 0).  A source held constant over
 *     the time element (t_a, t_b] seen at time t_obs contributes
 *     [K(t_obs - t_a) - K(t_obs - t_b)] x.
 *
 * Memory and streams:
 *   - Every d_* pointer is DEVICE memory on the context's device, owned by
 *     the caller, contiguous, 8-byte aligned, and must stay valid until the
 *     enqueued work has finished.  Every h_* pointer is host memory read
 *     before the call returns.
 *   - Trees, workspaces, Chebyshev expansions and Krylov bases are owned by
 *     the library.
 *   - Work is enqueued on the stream given to ddm_create and calls return
 *     without synchronising, except where a call's comment says it
 *     synchronises (tree build and GMRES read small values back).
 *
 * Errors: no C++ exception crosses this boundary.  Invalid arguments give
 * DDM_EINVAL, allocation failures DDM_ENOMEM, CUDA runtime errors DDM_ECUDA;
 * ddm_last_error() returns a message for the last failing call on a context.
 */
#ifndef DDM_GB300_H
#define DDM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DDM_OK = 0,
    DDM_EINVAL = 1,
    DDM_ENOMEM = 2,
    DDM_ENOTCONV = 3,   /* GMRES did not reach tol; solution and residual still written */
    DDM_ETIMEOUT = 4,   /* a bounded device wait expired */
    DDM_ECUDA = 5,
    DDM_PENDING = 6,    /* ddm_poll: request still running */
    DDM_ECANCELED = 7   /* ddm_poll: request cancelled (ddm_server_cancel) */
} ddm_status;

/* Poroelastic rock (paper Table 1 quantities): shear modulus G, drained and
 * undrained Poisson ratios, Skempton B, permeability k (m^2) and fluid
 * viscosity mu (Pa s).  Biot alpha, M and the diffusivity c follow from
 * these (Biot / Rice-Cleary plane strain). */
typedef struct {
    double G, nu, nu_u, B, perm, visc;
} ddm_material;

/* FMM controls (paper Sec. 3): n_cheb = Chebyshev nodes per dimension
 * (n^2 per cell; even, 2..16), leaf_size = the "prescribed number" of elements above
 * which a cell is split, max_depth fixes the quadtree depth cap (0 =
 * automatic: the deepest depth allowed by leaf_size, then, for a uniform
 * tree, the depth that minimises a cost model of the product measured on
 * GB300).  quad_near = Gauss points per element for the fluid-source near
 * field (0 = 6).
 * adaptive = 0: a uniform tree, every leaf at one depth (empty cells
 * dropped).  adaptive = 1: the quadtree of paper Sec. 3.1 as stated, every
 * cell holding more than leaf_size elements split into four, recursively,
 * so leaves sit at different levels (a cell whose elements are longer than a
 * quarter of its children's width is not split).  Two leaves then interact
 * directly when their ancestors at the coarser leaf's level share a vertex
 * (or coincide); every other pair goes through the M2L of the first level at
 * which their ancestors are apart, as in the uniform tree.  The same calls
 * and kernels serve both.
 * adaptive = 2: both trees are built and the one with the lower value of the
 * measured cost model of a product (near pairs, interaction pairs scaled by
 * (n/8)^4, cells: the model that picks the uniform tree's depth) is kept;
 * the build takes about twice as long, and ddm_tree_get_info reports the
 * kind kept. */
typedef struct {
    int n_cheb;
    int leaf_size;
    int max_depth;
    int quad_near;
    int adaptive;
} ddm_fmm_params;

typedef struct ddm_ctx ddm_ctx;
typedef struct ddm_tree ddm_tree;

/* Create a context bound to the current CUDA device and the given stream
 * (a cudaStream_t, or NULL for the legacy default stream). */
ddm_status ddm_create(ddm_ctx **out, const ddm_material *mat, const ddm_fmm_params *prm,
                      void *cuda_stream);
void ddm_destroy(ddm_ctx *ctx);
const char *ddm_last_error(const ddm_ctx *ctx);

/* Kernels that wait on the GPU (tensor-core pipelines) give up after a
 * bounded number of polls and raise a device word on the context instead of
 * hanging.  ddm_device_check synchronises the context stream, returns
 * DDM_ETIMEOUT (and clears the word) if any such wait expired since the last
 * check, else DDM_OK.  No counterpart in the paper. */
ddm_status ddm_device_check(ddm_ctx *ctx);

/* Poll limit of the grid barriers in the GMRES orthogonalisation kernel
 * (cooperative launch, every block resident): a block that has polled this
 * many times gives up, raises the error word and carries on, so a wait never
 * hangs.  polls = 0 restores the default (2^22 polls of about 64 ns).  A very
 * small limit makes the waits give up on purpose (a test of the failure
 * path: the solve then returns DDM_ETIMEOUT).  No counterpart in the paper. */
ddm_status ddm_set_wait_limit(ddm_ctx *ctx, int64_t polls);

/* Compressed M2L operators (the SVD compression of black-box FMM operators
 * that paper Sec. 3 cites as the further step of the Chebyshev FMM; the
 * paper applies the full operators).  Per tree level and time window the
 * (4n^2 x 4n^2) operators of all cell offsets are replaced by shared bases
 * of rank k and k x k cores, built on the device from the window's full
 * operators (randomized range finder on the component-equilibrated
 * operators, FP32) and cached per (tree, window) like the operators.
 *   rank: 0 for the default k = 64 + 4 (n - 8), else a multiple of 8 up to
 *         512 (capped at 4n^2); a new rank drops the tree's cached sets.
 *   mode 0: never; the M2L applies the full operators.
 *   mode 1: for every order n >= 8, from a window's first product.
 *   mode 2 (default): for orders n >= 10, once a window's full operators
 *           have served 128 products (the set-up costs tens of products, so
 *           only a window that keeps being applied pays for it).
 * Products of FMM mode (ddm_matvec, the operator of ddm_gmres_solve, history
 * windows) take it; batched problems keep the full operators.  A stream in
 * CUDA-graph capture never starts a set-up.  Errors: DDM_EINVAL for another
 * mode or rank.  No counterpart in the paper. */
ddm_status ddm_set_m2l_compression(ddm_ctx *ctx, int mode, int rank);

/* Build the quadtree of paper Sec. 3.1 over the element midpoints: level-0
 * square covering all midpoints, uniform depth (smallest depth whose leaves
 * hold <= leaf_size elements, capped so that no element is longer than a
 * quarter of a leaf), empty ("zero") cells dropped, children in Z order,
 * neighbour and interaction lists of paper Sec. 3.1.  Built on the device
 * (Morton keys + radix sort).  d_xy: 4N doubles [x0(N), y0(N), x1(N), y1(N)].
 * Below the occupancy depth, the depth minimising a measured cost model of
 * near pairs, interaction pairs and cells is taken (unless max_depth is set).
 * Synchronises the stream.  The tree keeps its own copy of the geometry.
 * DDM_EINVAL (nothing allocated, the context stays usable) for n <= 0,
 * n > 2^30, a null pointer, or an element of zero length or with a
 * non-finite end point. */
ddm_status ddm_build_tree(ddm_ctx *ctx, const double *d_xy, int64_t n, ddm_tree **out);
/* The same with the tree's own FMM parameters (Chebyshev order, leaf size,
 * depth cap, near-field rule, tree kind; n_cheb, leaf_size and quad_near
 * <= 0 take the context's, max_depth and adaptive are taken as given): every
 * product, history sum and solve on this tree uses them.  Lets one context
 * serve problems of different sizes at the order and leaf size that suit
 * each (see ddm_autotune).  DDM_EINVAL for an odd or out-of-range order. */
ddm_status ddm_build_tree_params(ddm_ctx *ctx, const double *d_xy, int64_t n, const ddm_fmm_params *prm,
                                 ddm_tree **out);
void ddm_tree_destroy(ddm_tree *tree);

typedef struct {
    int64_t n_elements;
    int depth;             /* deepest level (the leaf level of a uniform tree) */
    int64_t n_cells;       /* non-empty cells, all levels */
    int64_t n_leaves;
    int64_t n_m2l_pairs;   /* interaction-list entries, all levels */
    int64_t n_p2p_pairs;   /* (target element, source element) near pairs */
    double root_half_width;
    int leaf_level_min;    /* coarsest leaf level (= depth for a uniform tree) */
    int adaptive;          /* the kind built: 0 uniform, 1 adaptive */
    int max_leaf_records;  /* most direct-interaction element ranges of one leaf
                              (<= 9 in a uniform tree) */
} ddm_tree_info;
ddm_status ddm_tree_get_info(const ddm_tree *tree, ddm_tree_info *info);

#define DDM_MODE_FMM 0     /* Chebyshev FMM (paper Sec. 3) */
#define DDM_MODE_DENSE 1   /* every pair evaluated on the fly (conventional PDDM) */
#define DDM_MODE_PRECISE 16 /* OR-ed flag for accurate residuals.  With
                               DDM_MODE_FMM: the DD part of every directly
                               summed pair in FP64.  With DDM_MODE_DENSE: the
                               whole product in FP64 from the caller's FP64
                               geometry, every pair's DD part by its exact
                               element integral (a dislocation pair) and its
                               fluid source by an 8-point Gauss rule, O(N^2)
                               FP64 work */

/* d_y = [K(tau_hi) - K(tau_lo)] d_x  (paper Eqs. 2.3-2.5, left-hand sums for
 * tau_lo = 0, tau_hi = dt; one history term otherwise).  0 <= tau_lo < tau_hi.
 * d_x, d_y: 3N doubles, caller element order, must not overlap. */
ddm_status ddm_matvec(ddm_ctx *ctx, const ddm_tree *tree, double tau_lo, double tau_hi,
                      const double *d_x, double *d_y, int mode);

/* Time-history double sum of paper Eqs. (2.3)-(2.5) (applied with FMM as in
 * paper Sec. 4):  d_rhs -= sum_{eta=1}^{H} [K(t_{H+1} - t_{eta-1})
 *                                          - K(t_{H+1} - t_eta)] D^eta
 * d_hist: H x 3N doubles, row eta-1 = D^eta (caller element order);
 * h_times: H + 2 host doubles t_0 < t_1 < ... < t_{H+1} (t_{H+1} = the
 * current observation time).  With history compression on (below) and
 * H > exact_steps, the older steps take the compressed sum. */
ddm_status ddm_history_apply(ddm_ctx *ctx, const ddm_tree *tree, const double *d_hist,
                             const double *h_times, int H, double *d_rhs, int mode);

/* Time-compressed history sum (an extension: the paper sums every past step
 * exactly, Sec. 4).  The exact_steps most recent steps stay exact; older
 * steps are grouped by their window start lo = t_{H+1} - t_eta into blocks
 * [tau_E ratio^b, tau_E ratio^(b+1)) (tau_E: lo of the newest compressed
 * step), and over each block the response K(tau) is interpolated in
 * log tau at `nodes` Chebyshev points alpha_m:
 *   sum_{eta in block} [K(hi_eta) - K(lo_eta)] D^eta
 *     ~ sum_{m != m*} [K(alpha_m) - K(alpha_m*)] M_m,
 *   M_m = sum_eta [l_m(log hi_eta) - l_m(log lo_eta)] D^eta  (FP64 on the device),
 * alpha_m* the largest node (the weights sum to zero, so the instantaneous
 * part cancels exactly).  Products per step: exact_steps + (nodes - 1) x
 * (number of blocks) instead of H; with a constant step the node windows
 * are the same at every step (cached operators).  Measured against the
 * exact FP64 sum (oracle) on 100 steps of random D: nodes = 8 and ratio 2
 * give 5e-6 of the history's block maxima, nodes = 10 better.
 *   exact_steps = 0: off (default).  Otherwise nodes 2..16, ratio in
 *   [1.5, 16].  Errors: DDM_EINVAL.  The setting belongs to the context and
 *   applies to every later ddm_history_apply on it. */
ddm_status ddm_set_history_compression(ddm_ctx *ctx, int exact_steps, int nodes, double ratio);

#define DDM_SYS_PRESSURE 0     /* unknowns Ds, Dn, Dq; rows sigma_s, sigma_n, p (3N) */
#define DDM_SYS_IMPERMEABLE 1  /* unknowns Ds, Dn (Dq given); rows sigma_s, sigma_n (2N) */
#define DDM_SYS_RATE 2         /* unknowns Ds, Dn (Dq given); rows sigma_s, sigma_n + p (2N) */

/* Known right-hand side of the first step (paper Sec. 4): far-field stresses
 * transformed to each element face and added to the hydraulic load.
 * sigma_H along x and sigma_h along y are compression positive.  With p_f the
 * fracture fluid pressure and p0 the initial pore pressure:
 *   PRESSURE:    [-tau_inf, -(p_f - s_nn_inf), p_f - p0]
 *   IMPERMEABLE: [-tau_inf, -(p_f - s_nn_inf), 0]
 *   RATE:        [-tau_inf, -(p0 - s_nn_inf), 0]   (second row is sigma_n + p)
 * d_pf: N doubles of per-element fluid pressure, or NULL to use p_f. */
typedef struct {
    double sigma_H, sigma_h, p_f, p0;
    int system;
} ddm_loads;
ddm_status ddm_rhs(ddm_ctx *ctx, const ddm_tree *tree, const ddm_loads *loads, const double *d_pf,
                   double *d_rhs);

typedef struct {
    int system;        /* DDM_SYS_* */
    int restart;       /* Krylov basis size before restart (default 50) */
    int max_iters;     /* total iterations (default 1000) */
    double tol;        /* relative residual ||b - A x|| / ||b|| (default 1e-6, paper Sec. 5) */
    int mode;          /* DDM_MODE_FMM or DDM_MODE_DENSE for the products */
} ddm_gmres_params;
typedef struct {
    int iterations;
    int restarts;
    double rel_residual;   /* residual of the returned x, recomputed with the last residual operator */
    int converged;
} ddm_gmres_info;

/* Solve [K(dt)] x = rhs restricted to the chosen system with restarted GMRES
 * (paper Sec. 4, "modified GMRES with FMM products") in FP64, right
 * preconditioned by block Jacobi over fracture chains: elements that share
 * end points are cut into blocks of <= 64 elements whose own influence
 * matrices are inverted on the device (FP32) once per (dt, system); an
 * element on no chain is a block of its own.
 * d_rhs: 3N doubles of row values [sigma_s, sigma_n, p]; rows not in the
 * system are ignored, and for RATE the second system row is
 * d_rhs[N:2N] + d_rhs[2N:3N] (sigma_n + p: a history term subtracted from
 * all three rows stays complete).  d_x: 3N doubles,
 * in: initial guess (and the prescribed Dq for 2N systems), out: solution.
 * Precision escalates on stalls: at first every product (Arnoldi steps and
 * the residual recomputed at each restart) uses the requested mode, and
 * each restart's inner solve runs to 0.3 tol ||b||.  A restart that fails
 * to reduce the recomputed residual by 10% switches the residuals (and the
 * convergence test) to an accurate operator (problems of <= 16,384
 * elements: DDM_MODE_DENSE | DDM_MODE_PRECISE, once per restart; larger
 * ones: the requested mode with DDM_MODE_PRECISE), inner solves then
 * running to max(0.3 tol ||b||, 1e-4 of the restart's residual); a further
 * such restart makes the Arnoldi products precise as well (the requested
 * mode with DDM_MODE_PRECISE), and one more, for problems of <= 10,000
 * elements, makes them the exact FP64 dense product.  Returns DDM_ENOTCONV (x and
 * info still written) when max_iters is reached or three further restarts
 * in a row fail to reduce the residual by 10%.
 * Arnoldi orthogonalisation, Givens rotations, the residual estimate and the
 * least-squares solve run on the device in FP64; the host reads one status
 * triple per Arnoldi step (live flag, residual estimate, the context's
 * error word) and one norm per restart, so the call synchronises the
 * stream.  DDM_ETIMEOUT when a grid barrier of the orthogonalisation gave
 * up (see ddm_set_wait_limit): x is then invalid, and the barrier and the
 * error word are reset before the call returns, so the context stays
 * usable. */
ddm_status ddm_gmres_solve(ddm_ctx *ctx, const ddm_tree *tree, double dt, const double *d_rhs,
                           double *d_x, const ddm_gmres_params *prm, ddm_gmres_info *info);

/* Stress intensity factors from the tip element DDs (paper Eq. 2.6, Olson):
 * K = 0.806 E / (4 (1 - nu^2)) sqrt(pi / (2 a)) D, a = half-length of the tip
 * element, (E, nu) drained.  d_tip: n element indices; d_KI, d_KII: n doubles. */
ddm_status ddm_sif(ddm_ctx *ctx, const ddm_tree *tree, const double *d_x, const int64_t *d_tip,
                   int n, double *d_KI, double *d_KII);

/* One fracture growth step (the propagation check of paper Sec. 4's
 * time-marching algorithm; the paper gives no criterion, this is the
 * reading): for every tip, given by its element d_tip[i] and the end
 * d_tip_end[i] (0: (x0, y0), 1: (x1, y1)) that is the fracture tip,
 * K_I and K_II by Olson's formula (as ddm_sif, drained E and nu) in the
 * crack-tip frame (x outward along the fracture, y = x turned by +90
 * degrees), the maximum tangential stress criterion (Erdogan and Sih):
 *   theta = 2 atan((K_I - sqrt(K_I^2 + 8 K_II^2)) / (4 K_II))  (0 if K_II = 0),
 *   K_eq  = cos(theta/2) (K_I cos^2(theta/2) - 1.5 K_II sin(theta)),
 * and a tip with K_I > 0 and K_eq >= K_Ic grows by one element of its tip
 * element's length, from the tip along x rotated by theta.
 *   d_xy, n, d_x: the current geometry (4N, caller order) and solution (3N);
 *   d_xy_out: room for 4 (n + n_tips) doubles (not overlapping d_xy); it
 *     receives the grown geometry, the n old elements then the new ones
 *     (rows of stride *n_out);
 *   d_tip, d_tip_end: updated in place (a grown tip becomes the new
 *     element, end 1);
 *   d_theta, d_keq (device, n_tips, may be null): kink angle and K_eq.
 * The history of a march extends with zeros for the new elements (they did
 * not exist before).  Errors: DDM_EINVAL, DDM_ENOMEM, DDM_ECUDA. */
ddm_status ddm_grow(ddm_ctx *ctx, const double *d_xy, int64_t n, const double *d_x, int64_t *d_tip,
                    int *d_tip_end, int n_tips, double K_Ic, double *d_xy_out, int64_t *n_out,
                    double *d_theta, double *d_keq);

/* Batches of independent problems (no counterpart in the paper; many
 * uneven fracture sets solved together).  A batch refers to P trees (which
 * must outlive it); vectors of a batch are the problems' 3N vectors
 * concatenated in the order of `trees`.  Products of all problems are one
 * CUDA graph launch on the context stream (captured on the first call and
 * again whenever dt, mode or the buffers change).  All problems share dt,
 * system and GMRES parameters. */
typedef struct ddm_batch ddm_batch;
ddm_status ddm_batch_create(ddm_ctx *ctx, ddm_tree *const *trees, int n, ddm_batch **out);
void ddm_batch_destroy(ddm_batch *batch);
/* d_y_p = [K(dt)] d_x_p for every problem p. */
ddm_status ddm_batch_matvec(ddm_ctx *ctx, ddm_batch *batch, double dt, const double *d_x, double *d_y,
                            int mode);
/* Lockstep restarted GMRES of every problem (FP64 Arnoldi with per-problem
 * reductions; preconditioner, precision and stopping as ddm_gmres_solve).
 * infos: n entries.  Returns DDM_ENOTCONV if any problem did not converge
 * (its x and info are still written).  Synchronises the stream. */
ddm_status ddm_batch_gmres_solve(ddm_ctx *ctx, ddm_batch *batch, double dt, const double *d_rhs,
                                 double *d_x, const ddm_gmres_params *prm, ddm_gmres_info *infos);

/* Request loop with continuous batching (no counterpart in the paper; a
 * serving front end for many fracture-set solves).  ddm_server_create
 * starts a server thread with its own context and CUDA stream on the
 * context's device, material and FMM parameters.  Requests queue in
 * arrival order; the server admits them while the estimated device
 * footprint of the admitted ones (tree, M2L operators, solution history,
 * Krylov arena) stays within hbm_budget_bytes (0 = 64 GiB) and at most
 * max_active run.  Each round advances every admitted request by one time
 * step (history sum of its past steps, right-hand side from its loads, one
 * lockstep batched GMRES of all admitted requests with the same dt and
 * system, tolerance tol); finished requests leave and queued ones join the
 * next round.  A request's d_xy and d_x must stay valid until ddm_poll
 * reports completion; the solution of the last step is written to d_x
 * (3N doubles).  ddm_submit does not block (DDM_ENOMEM if the request alone
 * exceeds the budget); ddm_poll returns DDM_PENDING until the request is
 * done, then its final status. */
typedef struct ddm_server ddm_server;
typedef struct {
    int64_t n;              /* elements */
    const double *d_xy;     /* 4N geometry (device) */
    ddm_loads loads;        /* loads and system */
    double dt;              /* time step */
    int steps;              /* number of time steps */
    double *d_x;            /* out: 3N solution of the last step (device) */
} ddm_request;
typedef struct {
    int status;             /* DDM_PENDING, DDM_OK or the failure */
    int iterations;         /* GMRES iterations over all steps */
    int steps_done;
    double rel_residual;    /* last step */
    double queue_ms;        /* submit -> admission (host clock), -1 before */
    double latency_ms;      /* submit -> completion, -1 before */
} ddm_result;
ddm_status ddm_server_create(ddm_ctx *ctx, size_t hbm_budget_bytes, int max_active, double tol,
                             ddm_server **out);
ddm_status ddm_submit(ddm_server *server, const ddm_request *req, uint64_t *ticket);
ddm_status ddm_poll(ddm_server *server, uint64_t ticket, ddm_result *result);
/* Cancel every request not finished: queued ones leave the queue, active
 * ones stop before their next time step (a round in flight completes);
 * their status becomes DDM_ECANCELED and their x_out holds no result.
 * Later submissions are served as usual.  ddm_server_destroy alone waits
 * for every submitted request to finish. */
ddm_status ddm_server_cancel(ddm_server *server);

/* Where the server thread's time went since its start (host clock, ms):
 * rounds, time-step solves done, admission (tree builds), history sums and
 * right-hand sides, batch set-up, batched GMRES, and the rest. */
typedef struct {
    int64_t rounds;
    int64_t solves;
    double ms_admit;
    double ms_history;
    double ms_setup;
    double ms_solve;
    double ms_other;
} ddm_server_stats;
ddm_status ddm_server_get_stats(ddm_server *server, ddm_server_stats *stats);

/* Product mode of the server's later rounds (history sums and GMRES):
 * DDM_MODE_FMM (default) or DDM_MODE_DENSE (the conventional DDM, for a
 * comparison on the same request stream).  Errors: DDM_EINVAL. */
ddm_status ddm_server_set_mode(ddm_server *server, int mode);
void ddm_server_destroy(ddm_server *server);

/* Dense influence product that allocates nothing (no counterpart in the
 * paper).  For callers that cannot allocate device memory where they need a
 * product - e.g. a real-time loop that forbids allocation after start-up,
 * or code running inside another framework's fixed memory budget or while
 * that framework holds its allocator.  Same result as ddm_matvec with
 * DDM_MODE_DENSE, but needs no tree: d_xy is the 4N geometry
 * [x0, y0, x1, y1] (device, caller order), d_x / d_y 3N vectors (device,
 * must not overlap); d_y is overwritten.
 * Scratch: a device array inside the library for DDM_STATIC_MAX_ELEMENTS
 * elements (about 3 MB, held by every GPU that loads the library until the
 * process exits); n outside [1, DDM_STATIC_MAX_ELEMENTS] gives DDM_EINVAL.
 * The call uses no cudaMalloc/cudaFree or other allocating routine.  The
 * context's device must be current (else DDM_EINVAL).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (other
 * streams, other threads) race, so serialise them.  Each call rewrites the
 * entries it reads; nothing needs clearing.  d_x and d_y ranges that overlap
 * give DDM_EINVAL.  The geometry is checked on the device without
 * synchronising: an element of zero length or with a non-finite end point
 * makes every output NaN (ddm_matvec rejects such geometry at the tree
 * build instead). */
#define DDM_STATIC_MAX_ELEMENTS 65536
ddm_status ddm_matvec_dense_static(ddm_ctx *ctx, const double *d_xy, int64_t n, double tau_lo,
                                   double tau_hi, const double *d_x, double *d_y);

/* Autotuner (no counterpart in the paper): for a representative problem of
 * a size bucket (d_xy: 4N geometry, d_x: a 3N vector, both device; dt the
 * time step), build a tree for every candidate Chebyshev order (orders,
 * n_orders; NULL = 4, 6, 8, 10, 12), leaf size (leaves, n_leaves;
 * NULL = 16, 32, 64) and tree kind (uniform and adaptive, see
 * ddm_fmm_params), time its FMM product on the device (CUDA events,
 * after a warm-up that builds the window caches) and measure its error
 * against the on-the-fly dense product (max over the output blocks of
 * max|y - y_dense| / max|y_dense|).  *best receives the fastest candidate
 * whose error is <= max_rel_err (n_cheb, leaf_size and adaptive; the other
 * fields from the context, max_depth 0), with its
 * time per product and error.  DDM_ENOTCONV when no candidate meets the
 * bound.  Synchronises the stream; allocates and frees its own trees. */
ddm_status ddm_autotune(ddm_ctx *ctx, const double *d_xy, int64_t n, const double *d_x, double dt,
                        const int *orders, int n_orders, const int *leaves, int n_leaves, double max_rel_err,
                        ddm_fmm_params *best, double *best_ms, double *best_err);

/* Stage timing for profiling (no counterpart in the paper): when enabled,
 * CUDA events bracket each stage on the context stream.  ddm_profile_read
 * synchronises the stream and returns, per stage, the summed milliseconds
 * (ms[DDM_NSTAGES]) and the number of kernel launches (counted whether or
 * not timing is enabled) since the last read, then resets both.
 * Stages: 0 charges + own elements (dense path, trees below depth 2),
 * 1 own-element blocks of a new time window, 2 upward pass (charges, own
 * elements, P2M, M2M), 3 M2L operators of a new time window, 4 M2L,
 * 5 downward pass (L2L), 6 leaf (L2P + P2P), 7 dense product, 8 GMRES
 * vector kernels, 9 tree build. */
#define DDM_NSTAGES 10
ddm_status ddm_profile(ddm_ctx *ctx, int enable);
ddm_status ddm_profile_read(ddm_ctx *ctx, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* DDM_GB300_H */
