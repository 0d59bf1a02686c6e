/*
 * bie.h -- C ABI of the GB300 (sm_103a) periodized Stokes boundary-integral
 * library: the mobility problem of rigid bodies in a doubly periodic, sheared
 * two-dimensional Stokes flow, after Wang, Nazockdast & Barnett,
 * arXiv 1912.04501.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - All floating-point data are IEEE double unless stated otherwise.
 *  - Nodes are numbered body by body; on body i the nodes are the periodic
 *    trapezoidal nodes t_k = 2*pi*k/N_i, k = 0..N_i-1, of the parametrisation
 *    x(t) = x^c + R(theta) (a cos t, b sin t), counter-clockwise (Sec. 6, first
 *    paragraph).  N is the total node count.
 *  - A density or a traction is a vector of 2N doubles, node-major:
 *    (v_x[0], v_y[0], v_x[1], v_y[1], ...).
 *  - Pointers flagged `on_device` are device pointers on the context's GPU;
 *    otherwise they are host pointers (pageable or pinned).  The caller owns
 *    every array it passes; the library reads or writes it only during the
 *    call.  The library owns the device memory it allocates in bie_init.
 *  - Every function returns BIE_OK (0) or a negative BIE_E* code; the text of
 *    the last error is available from bie_last_error.  A context is not
 *    thread-safe: calls on one context must not overlap.
 *  - A context holds one unit cell (bie_init) or a batch of independent unit
 *    cells (bie_init_batch; the paper has no batches -- it is how many
 *    independent suspensions share one GPU).  Nodes and bodies of all cells
 *    are numbered cell after cell, so a density is still 2N doubles; every
 *    per-cell output (mu_eff, e2) has one entry per cell in cell order.
 */
#ifndef BIE_H
#define BIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BIE_OK 0
#define BIE_EINVAL (-1)   /* bad argument, size or geometry */
#define BIE_ENOCONV (-2)  /* solver stopped above its tolerance; outputs hold the last iterate */
#define BIE_ECOLLIDE (-3) /* two bodies closer than the allowed minimum gap */
#define BIE_ENUMERIC (-4) /* NaN or Inf met in a residual */
#define BIE_ECUDA (-5)    /* a CUDA runtime call failed */
#define BIE_ENOMEM (-6)   /* device allocation failed */

#define BIE_FP64 0  /* every pair sum in double precision */
#define BIE_MIXED 1 /* pair sums in single precision inside FP64 iterative refinement */
#define BIE_DF64 2  /* near pair sums in double-float arithmetic (pairs of floats, ~48-bit
                       significands) on the FP32 pipe; everything else in double */

typedef struct bie_ctx bie_ctx;
typedef struct bie_net bie_net;

#define BIE_NET_FEATURES 13 /* node features of the warm-start network (bie_features) */
#define BIE_NET_HIDDEN 64   /* its hidden width */

/* Lattice vectors e1, e2 and the centre of the unit cell U (Sec. 2). */
typedef struct {
    double e1[2];
    double e2[2];
    double center[2];
} bie_lattice;

/* One rigid body with centre xc and angle theta, discretised by n_nodes
 * trapezoidal nodes (n_nodes even, 8 <= n_nodes <= 16384), of one of two
 * shapes, given in the body frame and rotated by theta:
 *   shape 0, ellipse: (a cos t, b sin t), a = p[0], b = p[1];
 *   shape 1, star (Sec. 8 Examples 4-5): r(t) (cos t, sin t) with
 *            r(t) = r0 (1 + eps cos(k t)), r0 = p[0] > 0, 0 <= eps = p[1] < 1,
 *            k = p[2] an integer in 1..64.
 * xc is the reference point of the rigid motion (velocities are reported
 * there); for ellipses and stars with k >= 2 it is the boundary's arc-length
 * centroid (Sec. 2). */
typedef struct {
    int32_t n_nodes;
    int32_t shape;
    double p[4];
    double xc[2];
    double theta;
} bie_body;

/* One unit cell of a batch: lattice, viscosity mu, shear rate gamma and the
 * number of its bodies (the next n_bodies entries of the bodies array). */
typedef struct {
    bie_lattice lattice;
    double mu;
    double gamma;
    int32_t n_bodies;
} bie_cell;

/* Numerical parameters.  bie_default_opts fills every field. */
typedef struct {
    int32_t precision;    /* BIE_FP64, BIE_MIXED or BIE_DF64 (solver and time step) */
    int32_t n_proxy;      /* M proxy Stokeslets on a circle about the cell centre (Sec. 6.1), 4..256 */
    double proxy_radius;  /* radius of that circle */
    int32_t n_coll;       /* m Gauss-Legendre collocation points per wall (Sec. 6.1), 2..128 */
    double lam_rel;       /* Tikhonov parameter of the proxy least-squares fit, relative to ||Q||_F */
    double gmres_tol;     /* target relative residual ||b - A sigma|| / ||b|| (FP64 operator) */
    int32_t gmres_max;    /* maximum Krylov dimension of one GMRES cycle, 1..1000 */
    double inner_tol;     /* relative tolerance of each single-precision inner solve (BIE_MIXED) */
    int32_t max_refine;   /* maximum outer refinement sweeps (BIE_MIXED) */
    int32_t warm_start;   /* bie_step start: 0 = zero; 1 = previous step's density as the initial
                             guess; 2 = zero start, first GMRES cycle augmented with the previous
                             density, its last change and the warm-start network's direction
                             (bie_set_warm_net); with BIE_MIXED the second refinement sweep is
                             augmented with the previous step's second-sweep correction (the
                             single-precision operator's error changes little per step);
                             3 = as 2 without the network */
    double min_gap;       /* bie_step fails with BIE_ECOLLIDE below this body gap (node-sampled); 0 = off */
    int32_t device;       /* CUDA device ordinal */
    double close_factor;  /* close-evaluation zone in units of the source body's node spacing
                             h_b = perimeter / N_b (Sec. 6.3 remark: 10); 0 disables the correction */
    int32_t close_capacity; /* maximum (target, body image) close pairs stored; 0 = no limit
                             * (the storage grows with the geometry) */
    int32_t residual;     /* BIE_MIXED refinement residual: BIE_FP64 (native double) or BIE_DF64 */
    int32_t autotune;     /* 1: at bie_init, time the single-precision near-sum tile shapes on the
                             context's own cells and keep the fastest (bie_near_shape); the shape sets
                             the source splits, so results then agree across contexts to single-
                             precision rounding only.  0: the default shape (bit-reproducible) */
    int32_t graph;        /* 1: single-precision operator applications replay CUDA graphs captured
                             once per geometry (same kernels, same results); 0: direct launches
                             (the default: on GB300 the replay's extra copies cost about what the
                             launches it saves do) */
    int32_t precond;      /* 1: right-precondition GMRES with the inverse of the dense operator block
                             on the nodes inside another curve's close-evaluation zone (at most
                             1024, the closest kept; I/2 elsewhere), rebuilt with every geometry:
                             for nearly touching bodies (single-cell contexts only).  0: none */
    int32_t n_images;     /* near-image set of the periodizer.  9: the 3 x 3 lattice translates of
                             every body, proxies on a circle of radius proxy_radius about the cell
                             centre.  4: the paper's own periodizer (Def. Gnear, Sec. 6.1 remark after
                             Eq. W): each node's four lattice images inside the doubled cell U~ (same
                             centre, twice the size), chosen per node by its lattice coordinates, n_proxy
                             proxies (a multiple of 4) on the walls of U~, and the periodic sums taken at
                             each node's lattice translate inside U (Sec. 6.2); 4N sources per near sum
                             instead of 9N.  Bodies must be small enough that every close-evaluation pair
                             sees whole body images (BIE_EINVAL otherwise); autotune must be 0 */
    int32_t close_rule;   /* how each close-evaluation block (the integral of G^t times the trigonometric
                             interpolant of the nodal density over the exact curve, Sec. 6.3) is built.
                             0: the fine trapezoidal rule on rho N_b points of the interpolant (rho from the
                             target's distance, up to 4096).  1: the paper's special quadrature: compensated
                             barycentric rules for the Cauchy integrals the single-layer traction reduces to
                             (exterior boundary values by the Plemelj formula), O(N_b^2) per block whatever
                             the distance; exact for the interpolant of sigma / tau rather than of sigma, so
                             the two rules agree on smooth densities (to ~1e-12) and differ on rough ones */
} bie_opts;

typedef struct {
    int32_t iterations;   /* Krylov iterations, all cycles and sweeps */
    int32_t refinements;  /* outer refinement sweeps (BIE_MIXED), else GMRES cycles */
    int32_t applies64;    /* FP64 operator applications */
    int32_t applies32;    /* single-precision operator applications */
    double rel_residual;  /* final ||b - A sigma|| / ||b||, FP64 operator (batches: the
                             largest over the cells, each cell's norms taken over its own nodes) */
} bie_solve_info;

/* Fill *opts with the defaults: BIE_MIXED, M = 48, radius 1.5, m = 24,
 * lam_rel 1e-8, gmres_tol 1e-10, gmres_max 200, inner_tol 1e-5, max_refine 8,
 * warm_start 3, min_gap 0, device 0, close_factor 10, close_capacity 0,
 * residual BIE_DF64, autotune 0, graph 0, precond 0, n_images 9. */
void bie_default_opts(bie_opts* opts);

/* Create a context for one unit cell: lattice, viscosity mu, shear rate
 * gamma (background flow u0 = (gamma x2, 0), Sec. 3) and n_bodies bodies.
 * Copies the inputs, allocates the device buffers, discretises the bodies on
 * the GPU and builds the proxy fit.  opts may be NULL (defaults).
 * Errors: BIE_EINVAL (sizes, degenerate lattice, non-positive axes),
 * BIE_ENOMEM, BIE_ECUDA.  On error *ctx is set to NULL. */
int bie_init(bie_ctx** ctx, const bie_lattice* lattice, double mu, double gamma,
             int32_t n_bodies, const bie_body* bodies, const bie_opts* opts);

/* Create a context for n_cells independent unit cells (1..4096) solved
 * together: one kernel launch serves every cell (the near-sum work of all
 * cells is split into even waves across the SMs), the GMRES iterations of the
 * cells run in lockstep with per-cell Arnoldi processes and convergence tests,
 * and a converged cell drops out of the near sums.  bodies holds the bodies of
 * cell 0, then of cell 1, and so on.  opts applies to every cell.  Each cell
 * gives the same results (up to rounding order in the reductions) as a
 * context of its own.  Errors as bie_init. */
int bie_init_batch(bie_ctx** ctx, int32_t n_cells, const bie_cell* cells, const bie_body* bodies,
                   const bie_opts* opts);

/* Batch layout and the last solve per cell: n_cells; node_offset and
 * body_offset (n_cells + 1 entries each: first node / body of every cell and
 * the totals); last_solve (n_cells) the last bie_solve's or bie_step's
 * statistics per cell (iterations and sweeps the cell took part in, its own
 * relative residual).  Any pointer may be NULL; host pointers. */
int bie_cells(const bie_ctx* ctx, int32_t* n_cells, int32_t* node_offset, int32_t* body_offset,
              bie_solve_info* last_solve);

void bie_destroy(bie_ctx* ctx);
const char* bie_last_error(const bie_ctx* ctx);

/* Total node count N and body count. */
int bie_size(const bie_ctx* ctx, int32_t* n_nodes, int32_t* n_bodies);

/* Make the library launch on the given cudaStream_t (NULL = legacy default). */
int bie_set_stream(bie_ctx* ctx, void* stream);

/* Copy the current discretisation to the caller: positions x (2N), outward
 * unit normals n (2N), trapezoidal weights w (N), curvature kappa (N).  Any
 * pointer may be NULL.  Host pointers unless on_device. */
int bie_nodes(bie_ctx* ctx, double* x, double* n, double* w, double* kappa, int32_t on_device);

/* out = A sigma, the discretised operator of Eq. (BIEdiscretized) completed
 * by L (Eq. BIEPerturbed2) with the pressure fix of Sec. 6.2:
 *   out_i = sigma_i/2 + T_i + alpha n_i + F_b + (x_i - x^c_b)^perp tau_b,
 *   T = 3x3 near image sum of G^t (Eq. Gt) with the on-curve diagonal limit
 *       + proxy-Stokeslet correction fitted to the wall discrepancy (Sec. 6.2
 *       steps 1-4) + close-evaluation correction (Sec. 6.3): for targets within
 *       close_factor * h_b of a body image, the smooth rule is replaced by the
 *       integral of the trigonometric interpolant of the density over the exact
 *       ellipse;  alpha = -T_0 . n_0.
 * precision: BIE_FP64, BIE_MIXED (single-precision pair sums) or BIE_DF64
 * (double-float near pair sums, FP64-class accuracy at FP32-pipe speed).
 * sigma and out: 2N doubles each, must not overlap. */
int bie_apply(bie_ctx* ctx, const double* sigma, double* out, int32_t precision, int32_t on_device);

/* The right-hand side -T(u0, p0) = -mu gamma (n_2, n_1) of Eq. (BIEPerturbed)
 * at every node (2N doubles). */
int bie_rhs(bie_ctx* ctx, double* b, int32_t on_device);

/* Solve A sigma = b to opts.gmres_tol (relative FP64 residual) by GMRES on
 * the native-double operator (opts.precision = BIE_FP64), on the double-float
 * operator (BIE_DF64), or by single-precision GMRES inside FP64 iterative
 * refinement (BIE_MIXED; the residual in the precision opts.residual names).
 * A refinement sweep that reaches its inner tolerance yet reduces the
 * residual less than tenfold (an operator too ill-conditioned for single-
 * precision pairs, e.g. bodies ~1e-5 apart) switches the remaining sweeps to
 * GMRES on the double-float operator to the final tolerance; those
 * applications count as applies64.  If the double-float sweeps stall the
 * same way, the residual is at the double-float operator's own accuracy and
 * is taken in native FP64 from then on.
 * rhs NULL means -T(u0, p0).  sigma holds
 * the initial guess on entry when use_guess != 0 and the solution on exit
 * (2N doubles).  info may be NULL.  Returns BIE_ENOCONV if the tolerance was
 * not met (sigma then holds the best iterate), BIE_ENUMERIC on NaN/Inf. */
int bie_solve(bie_ctx* ctx, const double* rhs, double* sigma, int32_t use_guess, int32_t on_device,
              bie_solve_info* info);

/* Rigid-body velocities and effective viscosity from a density sigma (2N):
 * v (2 n_bodies) = (u + u0) at each centroid, omega (n_bodies) = half the
 * vorticity there, u the periodic single layer with its free constant fixed
 * by a zero proxy velocity at the cell centre; mu_eff (one per cell) the
 * particle-stress average mu - (1/(gamma |U|)) sum_b int (x_2 - x^c_2) sigma_1 ds.
 * Outputs may be NULL; they are host pointers unless on_device. */
int bie_velocities(bie_ctx* ctx, const double* sigma, double* v, double* omega, double* mu_eff,
                   int32_t on_device);

/* Effective viscosity per cell by the contour-deformation formula of
 * Sec. 6.4 (Eq. contourdef): the shear force per unit shear through a contour
 * from L to R below every body, moved by Gauss' law to the walls
 * D - e2, D - e1 - e2, R - e2 and L - e1 - e2 (each at least half a cell from
 * every source, so the trapezoidal quadrature is never evaluated near a
 * curve) with the density's near sum taken from each curve's quadrant pieces
 * translated by -e1 (right half) and -e2 (upper half), minus the net force of
 * the upper pieces, plus the proxy correction's traction on D; 32-point
 * Gauss-Legendre rules per wall.  Unlike Eq. (mueff) on D it holds when
 * bodies cross D, and it agrees with the particle-stress average of
 * bie_velocities to discretisation accuracy.  Needs opts.n_images = 4
 * (BIE_EINVAL otherwise).  sigma: 2N doubles; mu_eff: one per cell; host
 * pointers unless on_device. */
int bie_mu_eff_contour(bie_ctx* ctx, const double* sigma, double* mu_eff, int32_t on_device);

/* Advance n_steps forward-Euler steps of size dt (Sec. 7): solve, extract
 * (v, omega, mu_eff), move and rotate the bodies, shear the lattice
 * e2(t) = (gamma t L2 reduced by the nearest multiple of e1, L2) and re-wrap
 * the centres into the cell.  Requires e1 = (L1, 0).  The density of the
 * last solve stays in the context as the next warm start.  mu_eff_out, if not
 * NULL, receives n_steps x n_cells host doubles (step-major); info (host) the
 * last solve's info.  Every cell of a batch steps with the same dt.
 * Returns BIE_ECOLLIDE if opts.min_gap > 0 and a gap falls below it. */
int bie_step(bie_ctx* ctx, double dt, int32_t n_steps, double* mu_eff_out, bie_solve_info* info);

/* Checkpoint: time t, current e2 (2 per cell), centroids xc (2 n_bodies),
 * angles theta (n_bodies), last density sigma (2N, may be NULL).  Host pointers. */
int bie_get_state(bie_ctx* ctx, double* t, double* e2, double* xc, double* theta, double* sigma);

/* Restore a checkpoint taken from a context with the same bodies and node
 * counts; re-discretises and rebuilds the proxy fit.  sigma may be NULL
 * (warm start cleared).  Clears the history below. */
int bie_set_state(bie_ctx* ctx, double t, const double* e2, const double* xc, const double* theta,
                  const double* sigma);

/* The rest of a checkpoint for warm starts 2 and 3: the density of the solve
 * before the last, the last solve's second-sweep correction (BIE_MIXED), both
 * 2N host doubles (zeros when not kept), the last time step, and which of the
 * two are kept (bit 0: sigma_prev2, bit 1: d2).  Restoring them with
 * bie_set_history after bie_set_state makes warm_start 3 resume bit for bit
 * (warm_start 2 also reads the previous geometry's gaps, which a restored
 * context recomputes only from its next step on).  NULL pointers clear them. */
int bie_get_history(bie_ctx* ctx, double* sigma_prev2, double* d2, double* dt_prev, int32_t* have);
int bie_set_history(bie_ctx* ctx, const double* sigma_prev2, const double* d2, double dt_prev);

/* bie_apply_static: the same operator application as
 * bie_apply(ctx, sigma, out, BIE_MIXED, 1), but it allocates no device memory
 * at all and does not touch the per-call buffers that bie_init allocated.  It
 * has no counterpart in the paper; it exists for callers that may not call
 * cudaMalloc -- for instance code running inside a host application whose own
 * memory manager owns the device heap and forbids other allocations -- yet
 * need the operator on their own device buffers.  Like every call on a
 * context it must not overlap another call on the same context (it launches
 * on the context's stream, counts its launches in the context, and records
 * the profiler's events when bie_profile is on).
 *   sigma, out: device pointers, 2N doubles each (node-major), on the
 *   context's GPU; they must not overlap.  The call is asynchronous on the
 *   context's stream (unless bie_profile is on: the profiler may then wait
 *   for the stream to fold its events); out is ready when that stream
 *   reaches the end of it.
 * Its per-call scratch is one static device array of 4 MiB inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  Contexts with more than 8192 nodes (or whose buffers would not fit
 * the 4 MiB) are rejected with BIE_EINVAL and a message.  All calls share
 * that array and it keeps the last call's contents; each call writes every
 * buffer it reads, so nothing needs clearing, but calls that overlap on the
 * GPU (two streams, two contexts on one device) race on it.  The first call
 * on each device looks up the array's device address; make that first call
 * before any stream capture. */
int bie_apply_static(bie_ctx* ctx, const double* sigma, double* out);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper).  A per-node multilayer
 * perceptron, x (BIE_NET_FEATURES) -> tanh(W1 x + b1) -> tanh(W2 . + b2) ->
 * W3 . + b3 (2 outputs), hidden width BIE_NET_HIDDEN, maps local features
 * (bie_features) to a density direction in units of mu |gamma| dt; the
 * shipped parameters are trained on the density change over one time step.  Parameters: one float array, W1 (row-major), b1, W2, b2,
 * W3, b3.  The kernels read bfloat16 weights; layers 1 and 2 and the weight
 * gradients are tensor-core products of bfloat16 operands (the inputs and
 * the first hidden layer rounded to bfloat16, and in the gradient the
 * back-propagated errors too) with FP32 accumulation; tanh, the last layer
 * and the bias sums are FP32.  Training keeps FP32 master weights and Adam
 * moments.  BIE_ECUDA also reports a tensor-core completion wait that timed
 * out (the kernels never wait without a limit).  With warm_start = 2, bie_step
 * adds the prediction to the directions of the first GMRES cycle's search
 * space (see bie_opts.warm_start), so the GMRES residual test at gmres_tol
 * still decides convergence.
 * ---------------------------------------------------------------------- */

/* Create a network with n_in inputs (1..16) on a device; parameters are zero
 * until bie_net_set_params.  Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA. */
int bie_net_init(bie_net** net, int32_t n_in, int32_t device);
void bie_net_destroy(bie_net* net);
const char* bie_net_last_error(const bie_net* net);
/* inputs, hidden width and parameter count */
int bie_net_size(const bie_net* net, int32_t* n_in, int32_t* hidden, int32_t* n_params);
int bie_net_set_stream(bie_net* net, void* stream);
/* Host float arrays of n_params entries; set also clears the Adam state. */
int bie_net_set_params(bie_net* net, const float* params);
int bie_net_get_params(bie_net* net, float* params);
/* Y (N x 2) = net(X (N x n_in)); device pointers, row-major floats. */
int bie_net_forward(bie_net* net, const float* X, int32_t N, float* Y);
/* Loss L = sum_i W_i |net(X_i) - T_i|^2 / sum_i W_i over N nodes (device
 * pointers: X N x n_in, T N x 2, W N) and its gradient.  grad (host, n_params
 * floats) may be NULL; the gradient is kept for bie_net_adam_step; loss (host)
 * may be NULL. */
int bie_net_loss_grad(bie_net* net, const float* X, const float* T, const float* W, int32_t N, float* grad,
                      double* loss);
/* One Adam step (Kingma & Ba, bias-corrected) with the last gradient. */
int bie_net_adam_step(bie_net* net, double lr, double beta1, double beta2, double eps);

/* The context's BIE_NET_FEATURES node features (N x BIE_NET_FEATURES floats,
 * row-major) for the current geometry and the stored densities of the last
 * two solves: normal (2), curvature x h_b, (x - x^c) / max(a, b) (2), last
 * density / (mu |gamma|) (2), its last change / (mu |gamma| dt) (2, dt the
 * last bie_step's step), log(d / h_b) with d the distance to the nearest
 * other curve within the close zone (else the zone's edge), the unit vector
 * towards it (2), and log(d_prev / d) / (|gamma| dt) (0 if unknown).  Host
 * pointer unless on_device.  The network's outputs are read as the density
 * change over the next step in units of mu |gamma| dt. */
int bie_features(bie_ctx* ctx, float* X, int32_t on_device);

/* Attach (or detach with NULL) the warm-start network used by warm_start = 2.
 * It must take BIE_NET_FEATURES inputs and live on the context's device; the
 * caller keeps ownership and must not destroy it while attached. */
int bie_set_warm_net(bie_ctx* ctx, const bie_net* net);

/* Tile shapes of the single-precision near sum (packed = two lattice images
 * per f32x2 instruction; targets per thread; resident CTAs per SM):
 * 0 packed 2/5 (the default), 1 packed 1/8, 2 packed 3/4, 3 scalar 3/4,
 * 4 scalar 2/5.  *shape receives the one in use; ms (BIE_NEAR32_SHAPES
 * floats, may be NULL) the median launch time of each in milliseconds as
 * opts.autotune measured it (0 where not measured). */
#define BIE_NEAR32_SHAPES 5
int bie_near_shape(bie_ctx* ctx, int32_t* shape, float* ms);

/* Close-evaluation bookkeeping of the current geometry: number of stored
 * (target, body image) pairs, and pairs closer to the curve than the finest
 * rule (4096-fold upsampling) resolves to double precision (their correction
 * is then less accurate).  The upsampling factor of a pair is the smallest
 * power of two rho >= 2 with (rho - 1/2) d >= 6.4 h (d its distance to the
 * curve, h the local node spacing); tables for the factors in use are built
 * when a geometry first needs them. */
int bie_close_info(bie_ctx* ctx, int32_t* n_pairs, int32_t* under_resolved);

/* Profiling aid (no counterpart in the paper: it instruments the kernels
 * above).  bie_profile(ctx, 1) starts recording a CUDA event pair on the
 * context stream around every near-image-sum launch and counting every kernel
 * the library launches; bie_profile(ctx, 0) stops.  bie_profile_read
 * synchronises the stream, returns the totals since the last read and resets
 * them. */
typedef struct {
    int64_t launches;        /* all kernels launched by the library */
    int32_t near32_launches; /* single-precision near-sum launches */
    double near32_ms;        /* their summed device time (CUDA events) */
    int32_t near64_launches; /* double-precision near-sum launches */
    double near64_ms;
    int32_t neardf_launches; /* double-float near-sum launches */
    double neardf_ms;
} bie_profile_info;

int bie_profile(bie_ctx* ctx, int32_t enable);
int bie_profile_read(bie_ctx* ctx, bie_profile_info* info);

/* Target partition for a solve sharded across processes, one GPU each
 * (Sec. 6.2: the near sum, the dominant cost, splits by target).  Every
 * process holds the whole cell (geometry, proxy fit and density are
 * replicated) and owns the targets of bodies [body_begin, body_end) (whole
 * bodies, so each close-evaluation row stays with its target).  Every
 * operator application -- bie_apply, and each one inside bie_solve and
 * bie_step -- then evaluates the near sum only for its own targets (and node
 * 0, whose traction fixes the pressure constant), and calls exchange(y, 2N,
 * user) with the device vector y once its own rows are final and the stream
 * is synchronised; exchange must fill every other process's rows (an
 * all-gather of the slices) before returning, and return 0 (non-zero makes
 * the call fail with BIE_ECUDA).  The rest of the solve (wall discrepancy,
 * proxy fit, GMRES, extraction) runs replicated and bit-identical on every
 * process, so no other collective is needed.  The whole range (0, n_bodies)
 * with exchange NULL switches partitioning off.  Single-cell contexts only.
 * The paper has no multi-process design; this is the hot path's data split. */
int bie_set_partition(bie_ctx* ctx, int32_t body_begin, int32_t body_end,
                      int (*exchange)(double* y, int64_t n2, void* user), void* user);

/* Streaming multiprocessors of the context's device, as queried at bie_init
 * (the near-sum work items are sized for them). */
int bie_device_sms(const bie_ctx* ctx, int32_t* sms);

/* Measurement aid (no counterpart in the paper): the CUDA-core FMA
 * throughput of a device, the roofline denominators of the pair sums.
 * Launches full-occupancy grids of independent FMA chains -- scalar
 * fma.rn.f32, packed fma.rn.f32x2, then fma.rn.f64 -- on the given
 * cudaStream_t (NULL = legacy default stream), a few milliseconds each, and
 * returns the best of three timed launches of each in TFLOP/s (2 flops per
 * FMA lane).  Synchronises the stream.  Outputs (host) may be NULL.
 * Errors: BIE_EINVAL, BIE_ENOMEM, BIE_ECUDA. */
int bie_alu_peak(int32_t device, void* stream, double* ffma_tflops, double* ffma2_tflops, double* dfma_tflops);

#ifdef __cplusplus
}
#endif

#endif /* BIE_H */
