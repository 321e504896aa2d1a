/* FP64 CPU oracle for the explicit staggered-grid Navier-Stokes time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  The CUDA path shares no
 * code with it.
 *
 * Method (paper Sec. 4.1, Eq. 1-2): incompressible Navier-Stokes with
 * modified pressure phi = p / rho, body force f = 0, rho = 1, finite
 * differences on a regular rectangular staggered grid, advanced by an
 * explicit Runge-Kutta Method of Lines (Sec. 1) with ghost regions of
 * run-time width filled from neighbours or from boundary conditions
 * (Sec. 1.1).  The paper leaves the discretisation open; the readings used
 * here (MAC placement, advective form, Heun RK2 with a Jacobi pressure
 * projection per stage) are listed in the design notes.
 *
 * Arrays: one double array per field, shape (nz+2g, ny+2g, nx+2g), x fastest,
 * no padding; cell (i,j,k), -g <= i < nx+g, is element
 * ((k+g)*(ny+2g) + (j+g))*(nx+2g) + (i+g).
 */
#ifndef CFD_ORACLE_H
#define CFD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_U = 0, ORA_V = 1, ORA_W = 2, ORA_P = 3 };
enum { ORA_PERIODIC = 0, ORA_WALL = 1 };

typedef struct {
  int n[3];          /* interior cells nx, ny, nz */
  int g;             /* ghost width (1 or 2) */
  double h[3];       /* cell size hx, hy, hz */
  int bc[6];         /* per face -x,+x,-y,+y,-z,+z: ORA_PERIODIC or ORA_WALL */
  double wall[6][3]; /* wall velocity per face (tangential part used) */
  double nu;         /* kinematic viscosity */
  double omega;      /* Jacobi weight */
  int order;         /* 2 or 4 (4 needs g = 2) */
  int form;          /* advection term: ORA_ADVECTIVE or ORA_FLUX (order 2) */
} ora_grid;

/* Advection term of the momentum equation (Sec. 4.1, Eq. 1): the advective
 * form (u . grad) u_c, or, using div u = 0 (Eq. 2), the conservative form
 * div(u u_c) as face-flux differences.  The adjoint functions below
 * linearise either form. */
enum { ORA_ADVECTIVE = 0, ORA_FLUX = 1 };

/* Ghost fill of one field (kind ORA_U..ORA_P), axis passes x, y, z over the
 * full extent of the other two axes, so a later pass wins on edges/corners. */
void ora_ghost_fill(const ora_grid* G, double* f, int kind);

/* F_c(u) = -(u . grad) u_c + nu * lap u_c (form ORA_ADVECTIVE) or
 * F_c(u) = -div(u u_c) + nu * lap u_c (form ORA_FLUX) for c = u, v, w at
 * every interior point of each component.  Inputs need filled ghosts. */
void ora_rhs(const ora_grid* G, const double* u, const double* v, const double* w,
             double* fu, double* fv, double* fw);

/* out_c = a * x_c + b * y_c + c * F_c(y) on the interior; wall-normal faces
 * are set to 0.  x may be NULL when a == 0. */
void ora_stage(const ora_grid* G, double a, const double* const x[3], double b,
               const double* const y[3], double c, double* const out[3]);

/* r = (D w) / c_dt at cell centres (c_dt = 1 gives the plain divergence). */
void ora_divergence(const ora_grid* G, const double* const w[3], double c_dt, double* r);

/* One weighted Jacobi sweep of the 7-point Poisson operator L p = r:
 * p_out = p + omega * ((sum_d (p_{+d} + p_{-d}) / h_d^2 - r) / (sum_d 2/h_d^2) - p),
 * then ghost fill of p_out.  p needs filled ghosts. */
void ora_jacobi_sweep(const ora_grid* G, const double* p, const double* r, double* p_out);

/* iters sweeps starting from p (ghosts filled), result in p (tmp is scratch). */
void ora_jacobi(const ora_grid* G, double* p, const double* r, double* tmp, int iters);

/* u_out = w - c_dt * G p on the interior (G p at d-faces = (p_{+d} - p)/h_d);
 * wall-normal faces set to 0. */
void ora_project(const ora_grid* G, const double* const w[3], const double* p, double c_dt,
                 double* const u_out[3]);

/* One Heun RK2 step with a Jacobi projection per stage, in place on
 * u (3 arrays) and p (warm start and result).  scratch: 8 arrays of the same
 * size.  Ghosts of u and p must be filled on entry and are filled on exit. */
void ora_rk2_step(const ora_grid* G, double* const u[3], double* p, double dt, int iters,
                  double* const scratch[8]);

/* FP64 global quantities over the interior:
 * ke = 1/2 sum (u^2+v^2+w^2) hx hy hz, umax = max |u_d|, divmax = max |D u|. */
void ora_reduce(const ora_grid* G, const double* const u[3], double* ke, double* umax,
                double* divmax);

/* ||L p - r||_2 over interior cells (p ghosts filled). */
double ora_residual(const ora_grid* G, const double* p, const double* r);

/* Host threads used by the OpenMP loops (results do not depend on it);
 * n <= 0 restores the default.  Returns the count in effect. */
int ora_set_threads(int n);

/* The 7-point operator itself: lp = L p on the interior (test helper). */
void ora_laplace_p(const ora_grid* G, const double* p, double* lp);

/* ---- geometric multigrid for L p = r (cfd_oracle_mg.c) ---- */

typedef struct {
  int levels;    /* coarse levels below the grid, 1 .. ora_mg_max_levels */
  int nu1, nu2;  /* weighted Jacobi sweeps before and after the coarse correction */
  int ncoarse;   /* sweeps on the coarsest level (>= 1) */
  double omega;  /* Jacobi weight of every sweep of the cycle */
} ora_mg;

/* Coarse levels available: halvings while every n_d is even and >= 4. */
int ora_mg_max_levels(const ora_grid* G);

/* The next coarser level: n / 2, 2 h, same faces, ghost width and order. */
void ora_mg_coarse_grid(const ora_grid* F, ora_grid* C);

/* rc(I) = mean over the 8 fine cells of coarse cell I of (r - L p); p ghosts
 * filled; rc is a coarse array (ghosts set to 0). */
void ora_mg_restrict_residual(const ora_grid* F, const double* p, const double* r, double* rc);

/* p += trilinear interpolation of the coarse correction ec (ghosts filled)
 * at the fine cell centres (weights 3/4, 1/4 per axis), then ghost fill of p. */
void ora_mg_prolong_add(const ora_grid* F, const double* ec, double* p);

/* One V-cycle on p (ghosts filled) for L p = r: nu1 sweeps, restriction of
 * the residual, the same cycle on the coarse level from a zero correction
 * (ncoarse sweeps on the coarsest), prolongation, nu2 sweeps. */
void ora_mg_vcycle(const ora_grid* G, const ora_mg* M, double* p, const double* r);

/* ora_rk2_step with each stage's pressure solve replaced by 'cycles'
 * V-cycles (warm start from the last pressure).  scratch: 7 arrays. */
void ora_rk2_step_mg(const ora_grid* G, double* const u[3], double* p, double dt,
                     const ora_mg* M, int cycles, double* const scratch[8]);

/* ---- discrete adjoint (cfd_oracle_adjoint.c) ---- */

/* Transpose of ora_ghost_fill's linear part: ghost values are added onto
 * their sources (passes z, y, x) and cleared. */
void ora_ghost_fold(const ora_grid* G, double* f, int kind);

/* Transpose of ora_stage linearised at y: xbar += a outbar,
 * ybar += b outbar + c (dF/dy)^T outbar, *nubar += c <outbar, lap y>;
 * outbar is cleared.  xbar may be NULL when a == 0. */
void ora_adj_stage(const ora_grid* G, double a, double* const xbar[3], double b,
                   const double* const y[3], double c, double* const ybar[3],
                   double* const outbar[3], double* nubar);

/* Transpose of ora_rk2_step linearised at the step's stored states u^n
 * (start of the step) and u1 (after the stage-1 projection), both with
 * filled ghosts.  On entry ubar, pbar hold dL/d(u, p) after the step
 * (interior, ghosts 0); on exit dL/d(u, p) before it.  *nubar accumulates
 * dL/dnu.  scratch: 11 arrays. */
void ora_adj_rk2_step(const ora_grid* G, double* const un[3], double* const u1[3], double dt,
                      int iters, double* const ubar[3], double* pbar, double* nubar,
                      double* const scratch[11]);

#ifdef __cplusplus
}
#endif
#endif
