/*
 * lbm_solid.h -- C ABI of the B300 (sm_103a) solid lattice Boltzmann library:
 * primal LBM sweep, discrete adjoint (ALBM) sweep and gradient for the inverse
 * problems of arXiv 2609.31347 (linear-elastic solids, D2Q8 moment-space MRT).
 *
 * Method references (sections / equations of the paper):
 *   primal collide + stream ......... Section 3.1, Eqs. local_collide, local_stream,
 *                                     moments_c, moments_eq, forcing, Table A.1
 *   objective ....................... Section 3.2, Eqs. node_J, discrete_J
 *   adjoint fixed point ............. Section 3.3.2, Eqs. adjoint_streaming,
 *                                     adjoint_collision, adjoint_iteration, Algorithm 1
 *   gradient ........................ Eq. optimality, Table 1 control maps,
 *                                     Eq. zero_mean_projection
 *   convergence monitor ............. Eqs. convergence, convergence_crit
 *
 * Conventions
 *   - Lattice: nx * ny nodes, node n = y*nx + x.  Periodic grids wrap in both
 *     directions; bounded grids (elliptic plate) mark active nodes and give a
 *     boundary rule for every link whose source node is not active.
 *   - Populations are SoA: population k of node n at [k*N + n], k in the D2Q8 order
 *     Q = ((1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)), N = nx*ny.
 *     Two-component fields (force, displacement, gradient) are SoA [i*N + n].
 *   - Storage is IEEE binary64 (populations, fields, controls, results); lattice
 *     units with dt = dx^2 (Section 3.1), lattice force g = dx^2 F.
 *   - Arithmetic of the sweeps (lbm_solid_desc.kernel):
 *       LBM_KERNEL_FP64: every operation in binary64 (relative rounding 2^-53 per
 *         operation).
 *       LBM_KERNEL_AUTO (default): the collision of each node (periodic nodes, interior
 *         nodes of bounded grids, and boundary nodes whose gamma-modified constants are
 *         below 1/2 in magnitude; constant or per-node modulus) runs in 64-bit fixed
 *         point scaled to the node's largest input: the ten inputs of the node (8
 *         populations, 2 force or adjoint-source values) are converted to integers at
 *         the scale 2^-56 of that largest input, combined exactly with integer adds and
 *         62-bit fixed-point constants, and rounded back to binary64.  Every output is
 *         within 4 * 2^-56 of the node's largest input of the exact value.  This is
 *         tighter than binary64 for values near the node's maximum, but a value much
 *         smaller than its node's maximum keeps fewer relative bits (a population 2^-40
 *         of the node's largest input keeps about 16).  On periodic lattices the
 *         objective pass (e = d - d*) and the force gradient (r/2 - (dC/dg)^T phi_S)
 *         form their per-node differences the same way (twelve and ten inputs, within
 *         a few 2^-56 of the node's largest input) before binary64 products and sums.
 *         Nodes whose largest input lies outside [2^-923, 2^57) (subnormal-only nodes,
 *         Inf and NaN), the boundary rules, reductions, plate objectives and the
 *         modulus gradients use binary64; a node whose inputs are all zero maps to
 *         zero exactly.
 *   - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA tensors) on
 *     the handle's device; *_host are host pointers; desc arrays are host arrays.
 *     All caller pointers are borrowed for the duration of the call only.
 *   - Calls are stream-ordered on the stream given to lbm_solid_create.  Calls that
 *     return host scalars (objective, solves that test convergence, gradients of
 *     scalar controls written to host) synchronise that stream.
 *   - Errors are return codes; the library never aborts or exits.  After
 *     LBM_ERR_CUDA the handle is unusable except for lbm_solid_destroy.
 *     lbm_solid_last_error gives a one-line description of the last failure.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef LBM_SOLID_H
#define LBM_SOLID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_solid lbm_solid; /* opaque; owns all device state of one lattice */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,           /* invalid argument, size or inconsistent description */
  LBM_ERR_CUDA = 2,          /* CUDA runtime error (handle unusable afterwards)   */
  LBM_ERR_OOM = 3,           /* device allocation failed                         */
  LBM_ERR_STATE = 4,         /* call out of order (e.g. adjoint before primal)    */
  LBM_ERR_NOT_CONVERGED = 5, /* max_steps reached before the stopping rule held   */
  LBM_ERR_DIVERGED = 6       /* NaN/Inf detected in the monitored quantity        */
} lbm_status;

/* Control maps (Table 1 of the paper plus the scalar/field modulus variants). */
typedef enum {
  LBM_CTRL_FORCE_FIELD = 0,  /* alpha = nodal force F_n, 2N values (benchmark 2)       */
  LBM_CTRL_FORCE_BASIS2 = 1, /* F = alpha_1 Phi_1 + alpha_2 Phi_2, 2 values; alpha o F*
                                (benchmark 1) is Phi_1 = (F*_1,0), Phi_2 = (0,F*_2)    */
  LBM_CTRL_YOUNG_SCALAR = 2, /* E = alpha^2, 1 value (benchmark 3, Eq. E_substitution) */
  LBM_CTRL_YOUNG_FIELD = 3   /* E_n = alpha_n^2 per node, N values                     */
} lbm_control_kind;

/* Link rule codes for bounded grids (per node and direction, host array). */
enum { LBM_LINK_REGULAR = 0, LBM_LINK_DIRICHLET = 1, LBM_LINK_NEUMANN = 2 };

/* Arithmetic of the sweep kernels. */
enum {
  LBM_KERNEL_AUTO = 0, /* bulk collisions in 64-bit fixed point (see Conventions) */
  LBM_KERNEL_FP64 = 1  /* every operation in binary64 on the FP64 pipe           */
};

typedef struct {
  int nx, ny;               /* nodes per direction, >= 3 each                            */
  double dx;                /* grid spacing (periodic unit square: 1/nx)                 */
  int periodic;             /* 1 periodic (Section 4.2), 0 bounded (Section 4.3)         */
  double E, nu;             /* Young's modulus (> 0) and Poisson ratio (-1 < nu < 1);
                               YOUNG_* controls override E                              */
  const uint8_t *node_mask; /* host, N: 1 active, 0 outside; NULL = all active.
                               Must be NULL (or all 1) for periodic grids               */
  const uint8_t *link_bc;   /* host, 8N SoA [k*N+n]: LBM_LINK_* for each active node and
                               incoming direction k; non-regular exactly where the
                               source node n - c_k is outside.  NULL for periodic grids  */
  const double *wall_d;     /* host, 2N: Dirichlet displacement at nodes with Dirichlet
                               links (Eq. disp_Dirichlet), or NULL if none               */
  const double *wall_T;     /* host, 2N: traction T at nodes with Neumann links
                               (Eq. disp_Neumann), or NULL if none                       */
  const double *wall_n;     /* host, 2N: outward unit normal at Neumann nodes, or NULL   */
  const double *obs_mask;   /* host, N: weight of Omega^J (1/0); NULL = all active nodes  */
  int control;              /* lbm_control_kind                                          */
  const double *force;      /* host, 2N: fixed physical body force for YOUNG_* controls
                               (NULL = zero); ignored for force controls                 */
  const double *force_basis;/* host, 4N: (Phi_1 [2N], Phi_2 [2N]) for FORCE_BASIS2       */
  int kernel;               /* LBM_KERNEL_*                                              */
} lbm_solid_desc;

typedef struct {
  long max_steps;   /* cap on collide+stream sweeps (>= 1)                               */
  double tol;       /* tolerance of the stopping rule                                    */
  int criterion;    /* 0: coefficient of variation of c(t) over a trailing window
                          (Eq. convergence_crit);
                       1: residual max|f_C(t)-f_C(t-1)| / max|f_C(t)| < tol             */
  long window;      /* criterion 0: number of samples in the window (>= 2)              */
  long check_every; /* sweeps between monitor samples (>= 1).  With criterion 1 and an
                       even check_every the chunks and their tests run on the device
                       (no host round trip per test); the stopping sweep and the state
                       are the same as those of the rule evaluated on the host            */
  int fixed_steps;  /* nonzero: run exactly max_steps sweeps, no stopping test           */
} lbm_solve_opts;

typedef struct {
  long steps;         /* sweeps performed                                              */
  double last_metric; /* last CV (criterion 0) or residual (criterion 1); 0 if fixed   */
  double seconds;     /* host wall time of the call                                     */
} lbm_solve_info;

/* Create a handle for one lattice: validates desc, uploads the geometry, allocates
   ping-pong population buffers (primal and adjoint), and sets f_S(0) = 0 and a zero
   control.  stream: cudaStream_t (NULL = legacy default stream). */
lbm_status lbm_solid_create(const lbm_solid_desc *desc, void *stream, lbm_solid **out);
lbm_status lbm_solid_destroy(lbm_solid *h);

/* Control alpha on the device: n = 2N (FORCE_FIELD), 2 (FORCE_BASIS2), 1
   (YOUNG_SCALAR) or N (YOUNG_FIELD).  For YOUNG_* the modulus is alpha^2 (must be
   > 0).  Resets the primal state to f_S = 0 (Section 4.2.1: zero initial state at
   every optimisation step) unless keep_state is nonzero (warm start). */
lbm_status lbm_solid_set_control(lbm_solid *h, const double *alpha_dev, size_t n,
                                 int keep_state);

/* Target displacement d* on the device (2N); computes Cbar of Eq. node_J. */
lbm_status lbm_solid_set_target(lbm_solid *h, const double *dstar_dev);

/* Primal solve (Algorithm 2, the primal step): sweeps from the current f_S until opts'
   rule holds.  Returns LBM_ERR_NOT_CONVERGED / LBM_ERR_DIVERGED accordingly (the
   state is kept either way).  info may be NULL. */
lbm_status lbm_solid_primal_solve(lbm_solid *h, const lbm_solve_opts *opts,
                                  lbm_solve_info *info);

/* Objective J of Eq. discrete_J at the current primal state (needs a target). */
lbm_status lbm_solid_objective(lbm_solid *h, double *J_host);

/* Adjoint solve (Algorithm 1): phi_C(0) = 0 (or the phi_C given by
   set_populations(which = 2) since the last adjoint solve), iterate Eq.
   adjoint_iteration at the current primal state.  Needs set_target and a primal solve
   after the last set_control. */
lbm_status lbm_solid_adjoint_solve(lbm_solid *h, const lbm_solve_opts *opts,
                                   lbm_solve_info *info);

/* The nodal adjoint source field r = (dx^2 / Cbar) w (d - d*) of the current primal
   state (2N values, device; the adjoint's constant term is j_k = r . c_k, Eq. j of
   Algorithm 1).  Needs set_target.  Used to warm-start the adjoint. */
lbm_status lbm_solid_adjoint_source(lbm_solid *h, double *r_dev);

/* Gradient dJ/dalpha (Eq. optimality) from the current primal and adjoint states,
   written to grad_dev (device, n values as in set_control).  project_zero_mean
   subtracts the per-component mean over active nodes (Eq. zero_mean_projection;
   FORCE_FIELD only). */
lbm_status lbm_solid_gradient(lbm_solid *h, double *grad_dev, size_t n,
                              int project_zero_mean);

/* Forward-mode derivative (f-AD, Eq. fAD) of J along a control direction, at the
   current (converged) primal state: the tangent populations are iterated from zero with
   the differentiated collide + stream step (the primal state held fixed) until opts'
   rule holds, then dJ = sum_n obs (d - d*) . d-dot dx^2 / Cbar is written to dJ_host.
   seed_dev: device direction with n = 2N (FORCE_FIELD), 2 (FORCE_BASIS2) or 1
   (YOUNG_SCALAR, direction in alpha; E = alpha^2).  Not built for YOUNG_FIELD
   (LBM_ERR_ARG).  Needs set_target and a primal solve (LBM_ERR_STATE); allocates two
   population buffers on first use.  An independent check of the adjoint gradient: one
   tangent solve per control direction. */
lbm_status lbm_solid_tangent(lbm_solid *h, const double *seed_dev, size_t n,
                             const lbm_solve_opts *opts, double *dJ_host,
                             lbm_solve_info *info);

/* Populations: which = 0 primal f_S, 1 adjoint phi_S, 2 adjoint phi_C; 8N device
   doubles.  set_populations(0) sets f_S (warm start / checkpoint restore; the next
   primal solve continues from it).  set_populations(2) sets phi_C as the initial state
   of the next adjoint solve only; every other adjoint solve starts from rest (and
   set_control / primal_solve discard a pending one). */
lbm_status lbm_solid_get_populations(lbm_solid *h, int which, double *dst_dev);
lbm_status lbm_solid_set_populations(lbm_solid *h, int which, const double *src_dev);

/* Displacement d = (m10 + g_x/2, m01 + g_y/2) of the primal state (2N device). */
lbm_status lbm_solid_displacement(lbm_solid *h, double *d_dev);

/* Number of kernel launches this handle has issued (for launch accounting). */
long lbm_solid_launch_count(const lbm_solid *h);

/* Monitor samples of the last primal or adjoint solve that used criterion 0 (Eqs.
   convergence, convergence_crit), in order.  Sweeps run in chunks of check_every; a
   chunk that ends after s >= 2 sweeps in total (and is not just the first sweep from an
   explicit f_S) contributes one sample: c of Eq. (convergence) over the active nodes for
   the state its last sweep collided, f_S(s - 1) for the primal and
   phi_S(s - 1) = S'^T phi_C(s - 1) for the adjoint, whose displacement is
   (sum_k c_kx phi_S,k, sum_k c_ky phi_S,k).  The stopping test is applied to these
   samples.  Copies min(count, cap) values to dst_host (host, may be NULL) and returns
   the count; -1 for a NULL handle. */
long lbm_solid_monitor_samples(const lbm_solid *h, double *dst_host, long cap);

/* ---- Batches of periodic lattices -------------------------------------------------
 * Many periodic instances of uneven size (e.g. independent identifications, or the
 * node-wise finite-difference perturbations of one problem) advanced together: every
 * sweep is ONE kernel launch over all instances' tiles, and runs of sweeps are replayed
 * from CUDA graphs.  Same collision, adjoint and gradient as the single-lattice path
 * (Section 3.1, Eq. adjoint_iteration, Eq. optimality for the nodal force control), so
 * an instance reproduces a single-lattice handle with the same kernel variant bit for
 * bit.  One material (E, nu) for the whole batch.
 *
 * Layout: instance i owns nodes [off_i, off_i + nx_i*ny_i) of the concatenated node
 * range (off_i = lbm_batch_offset(b, i); lbm_batch_offset(b, count) = total nodes);
 * population k of its node n at [8 off_i + k N_i + n], two-component fields (force,
 * target, gradient) at [2 off_i + c N_i + n].  All arrays are device arrays borrowed
 * for the call; calls are stream-ordered on `stream` and do not synchronise except
 * create, set_target and tune.  Errors: LBM_ERR_ARG (bad sizes / NULL), LBM_ERR_STATE
 * (objective or adjoint before set_target, gradient before adjoint), LBM_ERR_OOM,
 * LBM_ERR_CUDA. */
typedef struct lbm_batch lbm_batch;
/* dx: per-instance grid spacing, or NULL for 1/nx_i (unit square).  kernel: LBM_KERNEL_*.
   Allocates 4 population buffers and 3 two-component fields over the total nodes. */
lbm_status lbm_batch_create(int count, const int *nx, const int *ny, const double *dx,
                            double E, double nu, int kernel, void *stream, lbm_batch **out);
lbm_status lbm_batch_destroy(lbm_batch *b);
long lbm_batch_offset(const lbm_batch *b, int i); /* node offset of instance i; -1 if bad */
/* Physical body force of every instance (2 * total values); resets every f_S to 0. */
lbm_status lbm_batch_set_force(lbm_batch *b, const double *F_dev);
/* Target displacement of every instance; computes each instance's Cbar (Eq. node_J). */
lbm_status lbm_batch_set_target(lbm_batch *b, const double *dstar_dev);
/* `sweeps` collide+stream sweeps of every instance (fixed count, no stopping test). */
lbm_status lbm_batch_primal(lbm_batch *b, long sweeps);
/* J of every instance (count values, device) at the current primal state. */
lbm_status lbm_batch_objective(lbm_batch *b, double *J_dev);
/* Adjoint from phi_C = 0: `sweeps` iterations of Eq. adjoint_iteration per instance. */
lbm_status lbm_batch_adjoint(lbm_batch *b, long sweeps);
/* dJ/dF_n of every instance (2 * total values, device). */
lbm_status lbm_batch_gradient(lbm_batch *b, double *grad_dev);
/* which = 0: f_S, 2: phi_C of every instance (8 * total values, device). */
lbm_status lbm_batch_get_populations(lbm_batch *b, int which, double *dst_dev);
/* Autotuner: times `sweeps` primal sweeps for tile widths 32, 64, 128 and 256 (tile =
   width x 256/width nodes) and keeps the fastest, then does the same for the adjoint
   sweep, which keeps its own width; the primal and adjoint states are restored.
   best_bx (may be NULL) receives the primal sweep's width.  Allocates two
   population-sized scratch buffers for the duration of the call. */
lbm_status lbm_batch_tune(lbm_batch *b, int sweeps, int *best_bx);

/* ---- Batches of one bounded geometry ---------------------------------------------
 * count instances of the same bounded lattice (geometry, wall data, body force, kernel
 * variant: one lbm_solid_desc with control LBM_CTRL_YOUNG_FIELD), each with its own
 * per-node Young's modulus E_n = alpha_n^2 (Eq. E_substitution), advanced together: every
 * sweep is ONE launch of the bounded grid's compact sweep over all instances (the same
 * per-node arithmetic as a single handle), and runs of sweeps are replayed from CUDA
 * graphs.  Used to generate many steady states of one plate (e.g. training states of a
 * learned warm start) and for batches of perturbed moduli.
 *
 * Layout: instance i's control at [i N + n], its populations at [8 i N + k N + n].  All
 * arrays are device arrays borrowed for the call; calls are stream-ordered on `stream`
 * and return without synchronising, except create and set_control (which validate the
 * moduli on the host).  Errors: LBM_ERR_ARG (NULL, a description that is periodic or not
 * YOUNG_FIELD, count outside 1..65535, a modulus that gives an invalid material),
 * LBM_ERR_OOM, LBM_ERR_CUDA; create also returns the errors of lbm_solid_create. */
typedef struct lbm_plate_batch lbm_plate_batch;
/* Allocates 2 population buffers and the per-node constants of count instances; every
   instance starts at rest with the description's modulus E. */
lbm_status lbm_plate_batch_create(const lbm_solid_desc *desc, int count, void *stream,
                                  lbm_plate_batch **out);
lbm_status lbm_plate_batch_destroy(lbm_plate_batch *b);
/* count * N controls (E_n = alpha_n^2; values at inactive nodes are ignored); every
   instance is reset to f_S = 0. */
lbm_status lbm_plate_batch_set_control(lbm_plate_batch *b, const double *alpha_dev);
/* `sweeps` collide + stream sweeps of every instance (fixed count, no stopping test). */
lbm_status lbm_plate_batch_primal(lbm_plate_batch *b, long sweeps);
/* f_S of every instance (count * 8N values; zero at inactive nodes). */
lbm_status lbm_plate_batch_get_populations(lbm_plate_batch *b, double *dst_dev);

/* ---- Learned warm start ------------------------------------------------------------
 * The paper has no counterpart: this network only supplies the initial populations of
 * an iteration (Eq. adjoint_iteration or the primal sweep) that then runs to the same
 * residual tolerance as from a cold start, so it changes iteration counts, never the
 * fixed point.  A linear U-Net: `levels` levels of C_l = base * 2^l channels; per level
 * two 3x3 convolutions with circular padding and bias, 2x2 average pooling between
 * levels; decoder: bilinear 2x upsampling (periodic, coarse values at the centres of
 * their 2x2 blocks), concatenation [upsampled, skip], two 3x3
 * convolutions; a 1x1 head to 8 channels.  Input 2 channels, output 8.  BF16 weights
 * and activations, FP32 accumulation on the tensor cores (3x3 convolutions: tcgen05.mma
 * with the accumulator in tensor memory; 1x1 head and weight gradients: mma.sync), FP32
 * master weights and Adam.
 *
 * Layout: x (B, H, W, 2) and y, t (B, H, W, 8) FP32 NHWC device arrays borrowed for
 * the call; parameters are one FP32 vector, per layer in execution order (encoder
 * level 0..levels-1: conv a, conv b; decoder level levels-2..0: conv a, conv b; head)
 * the weights [ky][kx][cin][cout] then the bias [cout].  All calls are stream-ordered
 * on the create-time stream and return without synchronising, except create and
 * destroy.  Errors: LBM_ERR_ARG (NULL, base not a positive multiple of 16, levels not
 * in 1..5, base * 2^(levels-1) > 256, H not divisible by 2^(levels-1), W not divisible
 * by 16 * 2^(levels-1)), LBM_ERR_OOM, LBM_ERR_CUDA. */
typedef struct lbm_unet lbm_unet;
/* Allocates parameters, Adam moments and every activation for batch size `batch` at
   H x W; weights N(0, 1/fan_in) from `seed`, zero biases. */
lbm_status lbm_unet_create(int base, int levels, int batch, int H, int W,
                           unsigned long long seed, void *stream, lbm_unet **out);
lbm_status lbm_unet_destroy(lbm_unet *u);
long lbm_unet_param_count(const lbm_unet *u); /* -1 for NULL */
/* Synchronises the stream; LBM_ERR_CUDA if a tensor-core convolution of this network
   gave up waiting for its own matrix operations since the last call (its outputs were
   then set to NaN).  Reading the flag clears it. */
lbm_status lbm_unet_status(lbm_unet *u);
/* Copies the parameter vector (which = 0) or the last gradient (which = 1) into dst. */
lbm_status lbm_unet_get_params(lbm_unet *u, float *dst_dev, int which);
/* Replaces the parameter vector (Adam moments are kept). */
lbm_status lbm_unet_set_params(lbm_unet *u, const float *src_dev);
/* y = net(x); y_dev may be NULL (the output then stays internal).  exact_acts = 0:
   BF16 activations, as in training.  exact_acts = 1: FP32 activations, each product
   taken as two BF16 products (high and low part of the activation), so that apart from
   the FP32 sums the network is the exact linear map of its BF16 weights; BF16 rounding
   of activations adds broadband noise (about 1e-3 relative, at every wavevector), which
   a warm start must not carry into the slowly decaying modes.  The FP32 activation
   buffers are allocated on the first such call (LBM_ERR_OOM if that fails). */
lbm_status lbm_unet_forward(lbm_unet *u, const float *x_dev, float *y_dev, int exact_acts);
/* Forward, loss L = (1/2) mean (y - t)^2 into loss_dev (may be NULL), gradient of L
   w.r.t. every parameter (readable with get_params(which = 1)), then one Adam step
   (beta 0.9 / 0.999, eps 1e-8) with learning rate lr if lr > 0. */
lbm_status lbm_unet_train_step(lbm_unet *u, const float *x_dev, const float *t_dev, float lr,
                               float *loss_dev);

/* Conversions between solver states and the network's tensors, for `count` samples
 * of one size N = nx * ny laid out like a batch of equal lattices (two-component field
 * of sample b at [2 b N + c N + n], populations at [8 b N + k N + n]).  The network
 * sees a resolution-free form of a steady state (Appendix A.1 moments, theta = 1/3):
 *   mode 1 (primal f_S):  z = (m10, m01, m11/dx, m_s/dx, m_d/dx,
 *                              (m12 - theta m10)/dx^2, (m21 - theta m01)/dx^2, m22/dx),
 *     whose sizes do not depend on dx at steady state;
 *   mode 2 (adjoint phi_C): dx^2 times the same with (1 - theta) for theta (at the
 *     adjoint fixed point m12 = (1 - theta) m10 and m21 = (1 - theta) m01 exactly, and
 *     phi grows as 1/dx^2 for a source r = (dx^2/Cbar) w (d - d*));
 *   mode 0: the plain moments.
 * Every sample is divided by the RMS s_b of its input field (the states are linear in
 * it), every channel by a constant c_i (chan_dev, 8 floats, NULL = 1; c_i = 0 marks a
 * channel that is not predicted: target 0, decoded as 0).  All arrays are device arrays
 * borrowed for the call; stream-ordered, no synchronisation; no allocation.
 * LBM_ERR_ARG for bad sizes, mode or NULL, LBM_ERR_CUDA if a launch fails. */
/* x (count, ny/factor, nx/factor, 2) = factor x factor block means of (field - ref) / s_b,
   s_b the RMS of field - ref (ref_dev NULL = 0: the state of the field itself; else the
   state of the change, which is added to the reference's state by decode's accumulate,
   the states being linear); scale_dev receives s_b (count floats). */
lbm_status lbm_warm_encode(int count, int nx, int ny, int factor, const double *field_dev,
                           const double *ref_dev, float *x_dev, float *scale_dev, void *stream);
/* t (count, ny, nx, 8) = network coordinates of the populations / (s_b c_i); t_dev
   16-byte aligned.  mode 3: as mode 1 (bounded grids). */
lbm_status lbm_warm_targets(int count, int nx, int ny, double dx, int mode,
                            const double *pop_dev, const float *scale_dev,
                            const float *chan_dev, float *t_dev, void *stream);
/* Populations (count, 8, hc*factor, wc*factor) from network output y (count, hc, wc, 8):
   periodic bilinear interpolation to the fine nodes (coarse node j = centre of its
   block), times s_b c_i, moments rescaled with the fine spacing dx_fine, inverted;
   written to pop_dev, or added to it if accumulate is nonzero.  For modes 1 and 2 the
   result's Fourier components at the wavevectors (nx/2, 0) and (0, ny/2) are then removed
   from every population plane (even sizes): the primal and adjoint steps have the
   eigenvalue -1 there, so an initial error in them would never decay, and the steady
   state of a smooth field has none.  Last, the conserved k = 0 components (the mean
   displacement: mean m10, m01 of f_S for mode 1, the matching adjoint invariants for
   mode 2) are set to zero, their value when iterating from rest with a zero-mean force
   or source; otherwise the iteration would settle on a rigidly shifted state.  Mode 3
   (bounded grids) is mode 1 without these two periodic steps. */
lbm_status lbm_warm_decode(int count, int wc, int hc, int factor, double dx_fine, int mode,
                           const float *y_dev, const float *scale_dev, const float *chan_dev,
                           double *pop_dev, int accumulate, void *stream);
/* Bounded grids: the state of one plate geometry as a function of its Young's modulus,
 * with the network on a w x h crop of the nx_box x ny_box box (the crop holds the whole
 * domain).  Mode 3 of lbm_warm_targets / lbm_warm_decode is mode 1 without the periodic
 * steps (no Fourier components removed, no means set to zero).
 * x (count, h/factor, w/factor, 2): block means over factor x factor crop nodes of
 * mask_n E_ref / E_n (the compliance: the steady displacement of a uniform modulus is
 * proportional to it when the loads do not depend on E, so a linear network can represent
 * that dependence) and of mask_n, E_n = alpha_n^2 (per_node: alpha_dev holds
 * count * nx_box * ny_box values) or alpha_b^2 (otherwise: count values); mask_dev
 * (nx_box * ny_box uint8) marks active nodes. */
lbm_status lbm_warm_encode_modulus(int count, int nx_box, int ny_box, int per_node,
                                   const double *alpha_dev, const uint8_t *mask_dev, double E_ref,
                                   int w, int h, int factor, float *x_dev, void *stream);
/* Populations between the box layout (count, 8, ny_box, nx_box) and the crop layout
   (count, 8, h, w): to_box = 0 copies the crop out of the box; to_box = 1 writes the box,
   zero outside the crop and where mask_dev (may be NULL) is 0.  src and dst must differ. */
lbm_status lbm_warm_crop(int count, int nx_box, int ny_box, int w, int h, int to_box,
                         const uint8_t *mask_dev, const double *src_dev, double *dst_dev,
                         void *stream);
/* rms_i of channel i of an (pixels, 8) tensor over its first min(pixels, 2^22) rows. */
lbm_status lbm_warm_channel_rms(const float *t_dev, long pixels, float *rms_dev, void *stream);

/* ---- Initial states from the history of an optimisation loop ----------------------
 * The paper has no counterpart (every solve there starts from rest).  An optimisation
 * loop keeps its last few steady states; the next solve starts from a combination of
 * them, e.g. the Lagrange extrapolation of the primal state in 1/E for a Young's-modulus
 * control (the steady displacement scales with 1/E for loads that do not depend on E),
 * or, for the adjoint, the combination of previous adjoint states whose sources best
 * fit the new source in least squares (the adjoint steady state is linear in its
 * source).  The solver then iterates to the same tolerance, so only iteration counts
 * change.  These two calls do the vector arithmetic.
 *
 * dst[i] = sum_{j < count} w[j] * src_dev[j][i] for i < n.  1 <= count <= 4; w and
 * src_dev are host arrays of count weights and count device pointers to n doubles; dst
 * (device, n doubles) may be one of the sources.  Stream-ordered, no synchronisation.
 * Errors: LBM_ERR_ARG (count out of range, n < 1, a NULL pointer), LBM_ERR_CUDA. */
lbm_status lbm_warm_combine(int count, long n, const double *w, const double *const *src_dev,
                            double *dst_dev, void *stream);
/* Doubles of device scratch that lbm_warm_dots needs. */
long lbm_warm_dot_work_size(void);
/* Inner products of m device vectors of n doubles (1 <= m <= 5): out_host[a*m + b] =
 * sum_i v_dev[a][i] * v_dev[b][i], summed in a fixed order (repeatable bit for bit).
 * work_dev: caller-owned device scratch of lbm_warm_dot_work_size() doubles, not used
 * by another call at the same time.  Synchronises the stream (the result is on the
 * host).  Errors: LBM_ERR_ARG (m out of range, n < 1, a NULL pointer), LBM_ERR_CUDA. */
lbm_status lbm_warm_dots(int m, long n, const double *const *v_dev, double *work_dev,
                         double *out_host, void *stream);

/* Objective without any device allocation.
 *
 * The paper has no counterpart to this entry point: it exists for callers that cannot
 * allocate device memory, and so cannot create a handle (lbm_solid_create allocates).
 * Examples: a host application that gives all device memory to its own pool and
 * forbids other allocations, or a loop that must not pay the device-wide
 * synchronisation that cudaFree implies.  It computes the objective of a state from
 * caller-owned device arrays and calls no cudaMalloc, cudaFree or other allocating
 * routine:
 *
 *   J = (1/2) sum_n w_n |d_n - d*_n|^2 / sum_n w_n |d*_n|^2,  d_n = (m10 + dx^2 F_x / 2,
 *       m01 + dx^2 F_y / 2) of the node's populations  (the dx^2 factors of the sum and
 *       of its normalisation cancel),
 *
 * which is the value lbm_solid_objective returns for the same state, target and
 * weights.  Every node of the nx x ny box is summed: on a bounded grid pass weights that
 * are zero outside the domain (for instance the node mask as doubles), since the handle
 * only sums the domain's nodes.
 *
 *   fS_dev    8N post-streaming populations, SoA [k*N + n] (e.g. from
 *             lbm_solid_get_populations(h, 0, ...))
 *   F_dev     2N physical body force, SoA
 *   dstar_dev 2N target displacement, SoA
 *   obs_dev   N weights w_n, or NULL: w_n = 1 on every node of the box
 *   J_dev     1 double, written with J; NaN if sum_n w_n |d*_n|^2 is zero
 *   stream    cudaStream_t the two kernels are enqueued on (NULL = legacy stream);
 *             the call returns without synchronising.
 *
 * Scratch: per-block partial sums live in one fixed file-scope __device__ array of
 * 2 * LBM_NOALLOC_MAX_NODES / 256 doubles (64 KiB), which every GPU that loads this
 * library holds until the process exits.  Grids with nx * ny > LBM_NOALLOC_MAX_NODES
 * are rejected with LBM_ERR_ARG before anything is launched.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with the device
 * current and keeps it for the life of the process; make that first call before any
 * stream capture, and do not call this entry point again on a device after
 * cudaDeviceReset (the kept address then belongs to a destroyed context).  All calls on
 * a device share the array and every call rewrites the partials it reads, but calls
 * that overlap on the GPU (other streams, other host threads) race on it: serialise
 * them.  Returns LBM_ERR_ARG for invalid sizes or NULL arrays, LBM_ERR_CUDA if the
 * address lookup or a launch fails. */
#define LBM_NOALLOC_MAX_NODES (1L << 20)
lbm_status lbm_objective_noalloc(int nx, int ny, double dx, const double *fS_dev,
                                 const double *F_dev, const double *dstar_dev,
                                 const double *obs_dev, double *J_dev, void *stream);

const char *lbm_status_string(lbm_status s);
const char *lbm_solid_last_error(const lbm_solid *h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_SOLID_H */
