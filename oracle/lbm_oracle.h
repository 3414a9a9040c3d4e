/*
 * CPU reference ("oracle") for the solid lattice Boltzmann method, its discrete
 * adjoint and the gradient of the inverse problems of arXiv 2609.31347
 * ("gradient-based optimisation with an LBM constraint for linear elastic solids").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this library; only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark script do.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Everything here is plain, slow FP64 (plus a forward-mode dual-number type for
 * f-AD), written step by step in the order of the paper:
 *   - D2Q8 stencil in the order Q of Eq. (direction_order), Section 3.1
 *   - moment matrix M (Appendix A.1, Eqs. moments, moment_s, moment_d, moment_f)
 *   - equilibrium m^eq = N (m10bar, m01bar) (Eq. moments_eq), relaxation
 *     (Eqs. moments_c, relaxation, Table A.1), half/half forcing
 *     (Eqs. moments_bar_1/2, moments_c_10/01), collision + streaming
 *     (Eqs. local_collide, local_stream)
 *   - objective (Eqs. node_J, discrete_J), convergence monitor (Eq. convergence)
 *   - adjoint fixed point (Eqs. adjoint_streaming, adjoint_collision,
 *     adjoint_iteration, adjoint_init) and optimality (Eq. optimality)
 *   - f-AD (Eq. fAD) as a dual-number run of the same primal code.
 *
 * Layout: SoA, population k of node n at [k*N + n], node n = y*nx + x.
 * Two-component fields (force, displacement, wall data) are SoA: [i*N + n].
 * All functions return 0 on success and a negative code on bad input.
 *
 * Parity status: every function is pinned by the tests (closed forms, the paper's
 * printed EOCs and matrix, f-AD vs adjoint, the dot-product identity, finite
 * differences); the bounded-domain boundary rules are the builder's own reading
 * (the paper defers them to other work) and are pinned only by the transpose and
 * f-AD identities and by the first-order plate convergence.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny;                    /* nodes per direction; N = nx*ny                         */
  int periodic;                  /* 1: periodic wrap (Section 4.2); 0: bounded domain       */
  double dx;                     /* grid spacing Delta x; Delta t = dx^2 (Section 3.1)      */
  double nu;                     /* Poisson ratio                                          */
  const unsigned char *node_type;/* N: 0 outside, 1 interior, 2 boundary; NULL = all 1     */
  const unsigned char *link;     /* 8N [k*N+n]: 0 regular, 1 Dirichlet-missing,
                                    2 Neumann-missing (incoming population k at n whose
                                    source node n - c_k is outside); NULL = all regular   */
  const double *wall_d;          /* 2N: Dirichlet displacement at boundary nodes, or NULL   */
  const double *wall_T;          /* 2N: Neumann traction at boundary nodes, or NULL         */
  const double *wall_n;          /* 2N: outward unit normal at Neumann nodes, or NULL       */
} orc_grid;

/* M(gamma) row-major 8x8 and its inverse (Gauss-Jordan). Returns -1 if singular. */
int orc_moment_matrix(double gamma, double *M, double *Minv);

/* omega for beta in (11, s, d, 12, 21, f) and the boundary gamma (Eq. gamma, tau_f=1/2).
   Returns -1 if E <= 0, nu outside (-1,1) or tau_s == tau_f (gamma singular). */
int orc_material(double E, double nu, double *omega6, double *gamma_b);

/* One local collision (Eq. local_collide) with lattice force (gx, gy). */
int orc_collide(double E, double nu, int boundary_node, const double *fS8, double gx,
                double gy, double *fC8);

/* Primal: f_S(0) = fS0 (NULL = 0, Section 4.2 zero initial state), then `steps`
   collide+stream steps.  E_node: N moduli.  F: 2N physical body force.
   Writes f_S(steps) (8N) and, if fC_out != NULL, f_C(steps-1) (8N). */
int orc_primal(const orc_grid *g, const double *E_node, const double *F, const double *fS0,
               long steps, double *fS_out, double *fC_out);

/* Forward-mode AD (Eq. fAD): the primal above run in dual numbers with seeds
   Edot (N, NULL = 0) and Fdot (2N, NULL = 0); fS0 tangent is zero. */
int orc_primal_tangent(const orc_grid *g, const double *E_node, const double *Edot,
                       const double *F, const double *Fdot, long steps, double *fS_out,
                       double *fSdot_out);

/* Objective (Eqs. node_J, discrete_J) on f_S; obs: N indicator of Omega^J
   (NULL = all active nodes). Returns J and Cbar. */
int orc_objective(const orc_grid *g, const double *fS, const double *F, const double *dstar,
                  const double *obs, double *J, double *Cbar);
/* Tangent of the objective for a dual state (fS, fSdot) and force tangent Fdot. */
int orc_objective_tangent(const orc_grid *g, const double *fS, const double *fSdot,
                          const double *F, const double *Fdot, const double *dstar,
                          const double *obs, double *J, double *Jdot);

/* d_n = (m10 + gx/2, m01 + gy/2) of f_S (Eq. disp_from_moments), 2N. */
int orc_displacement(const orc_grid *g, const double *fS, const double *F, double *d_out);
/* Physical Cauchy stress (sigma11, sigma22, sigma12) per node, 3N, from bared
   moments (Eq. stress_from_moments) scaled by 1/dx to physical units. */
int orc_stress(const orc_grid *g, const double *E_node, const double *fS, const double *F,
               double *sigma_out);
/* c(t) = (1/N_active) sum ||d_n||^2 (Eq. convergence). */
int orc_monitor(const orc_grid *g, const double *fS, const double *F, double *c);
/* c(t) of Eq. (convergence) for t = 0 .. steps of the primal from f_S(0) = 0:
   c_out[t] = orc_monitor of f_S(t) (steps + 1 values). */
int orc_primal_trace(const orc_grid *g, const double *E_node, const double *F, long steps,
                     double *c_out);
/* c of Eq. (convergence) for the adjoint displacement d^phi_n = (sum_k c_kx phi_S,k,
   sum_k c_ky phi_S,k) of phi_S(i) = S'^T phi_C(i), i = 0 .. steps, along the iteration of
   orc_adjoint (steps + 1 values). */
int orc_adjoint_trace(const orc_grid *g, const double *E_node, const double *F,
                      const double *fS, const double *dstar, const double *obs, long steps,
                      double *c_out);
/* Stopping rule of Eq. (convergence_crit) on a sequence of samples c[0..n): the first
   index i >= window - 1 at which the trailing window c[i-window+1 .. i] has
   std / mean < tol, with std the population standard deviation (divided by window)
   and CV = 0 for a constant zero window; -1 if it never holds (-2 on bad input).
   metric receives the last CV evaluated. */
long orc_cv_stop(const double *c, long n, long window, double tol, double *metric);

/* OpenMP threads of the node loops (n <= 0: all processors); returns the count in use.
   Results do not depend on it. */
int orc_set_threads(int n);
int orc_threads(void);

/* Homogeneous step operators for the dot-product identity:
   P x = S' L x (collide without force, stream without wall sources), and P^T y. */
int orc_apply_step(const orc_grid *g, const double *E_node, const double *x, double *y);
int orc_apply_step_transpose(const orc_grid *g, const double *E_node, const double *y,
                             double *x);

/* Adjoint (Algorithm 1): phi_C(0)=0, `steps` iterations of Eq. adjoint_iteration at
   the primal state fS.  Writes phi_C(steps) and phi_S = S'^T phi_C(steps) (8N each). */
int orc_adjoint(const orc_grid *g, const double *E_node, const double *F, const double *fS,
                const double *dstar, const double *obs, long steps, double *phiC_out,
                double *phiS_out);

/* Eq. optimality for the nodal force control F_n: dJ/dF (2N). */
int orc_gradient_force(const orc_grid *g, const double *E_node, const double *F,
                       const double *fS, const double *phiS, const double *dstar,
                       const double *obs, double *grad_out);

/* Eq. optimality for the Young's modulus: per-node dJ/dE_n (N) and their sum
   (the scalar-E derivative).  Needs f_S, phi_S and phi_C at the fixed point. */
int orc_gradient_young(const orc_grid *g, const double *E_node, const double *F,
                       const double *fS, const double *phiS, const double *phiC,
                       double *grad_node, double *grad_total);

#ifdef __cplusplus
}
#endif
#endif
