/* FP64 CPU oracle: forward time step.  TEST INFRASTRUCTURE ONLY (see the
 * header).  Plain loops over (k, j, i); OpenMP, when enabled, only splits the
 * rows (k, j) of point-wise updates, each of which writes its own outputs
 * (so a grid of a single plane still uses every core), and every sum is
 * taken in a fixed order, so results do not depend on the thread count.
 *
 * Scheme (readings of Sec. 4.1, Eq. 1-2 and the Method of Lines of Sec. 1):
 *  - MAC grid: p at cell centres, u/v/w on the +x/+y/+z faces of cell (i,j,k).
 *  - Advective form (u . grad) u with central differences; the transverse
 *    velocity at a face point is the 4-point (order 2) or 4x4-point cubic
 *    (order 4) interpolation of the neighbouring faces.
 *  - Or (order 2) the conservative form div(u u_c): around the point of u_c
 *    the flux of c-momentum through the side normal to d is the product of
 *    u_c and u_d, each the mean of its two nearest values on that side
 *    (Eq. 2 makes the two forms agree for the continuous field).
 *  - Viscous term: 3-point (order 2) or 5-point (order 4) Laplacian per axis.
 *  - Pressure: 7-point Poisson operator L = D G, weighted Jacobi sweeps.
 *  - Time: Heun RK2; each stage is projected: w = stage value,
 *    r = D w / (c dt), p <- Jacobi^K(p, r), u = w - c dt G p.
 *  - Boundaries (Sec. 1.1 ghost regions): periodic, or a wall carrying a
 *    tangential velocity (no-slip / moving lid); wall-normal faces are held at
 *    zero and p takes a zero-gradient ghost.
 */
#include "cfd_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

static inline long ext(const ora_grid* G, int a) { return (long)G->n[a] + 2L * G->g; }

static inline size_t at(const ora_grid* G, int i, int j, int k) {
  return ((size_t)(k + G->g) * (size_t)ext(G, 1) + (size_t)(j + G->g)) * (size_t)ext(G, 0) +
         (size_t)(i + G->g);
}

static inline size_t at3(const ora_grid* G, const int q[3]) { return at(G, q[0], q[1], q[2]); }

static size_t total(const ora_grid* G) { return (size_t)ext(G, 0) * ext(G, 1) * ext(G, 2); }

/* ---------------------------------------------------------------- ghosts */

/* Value written into ghost index q[a] (outside 0..n-1) of field kind on the
 * face 'face' (2a for the low side, 2a+1 for the high side).  m = 1..g is the
 * distance of the ghost layer from the interior. */
static double ghost_value(const ora_grid* G, const double* f, int kind, int a, int face, int m,
                          const int q[3]) {
  const int N = G->n[a];
  int s[3] = {q[0], q[1], q[2]};
  const int low = (face == 2 * a);
  if (G->bc[face] == ORA_PERIODIC) {
    s[a] = low ? N - m : m - 1;           /* f[-m] = f[N-m],  f[N-1+m] = f[m-1] */
    return f[at3(G, s)];
  }
  s[a] = low ? m - 1 : N - m;             /* mirror image across the wall */
  if (kind == ORA_P) return f[at3(G, s)]; /* zero normal gradient */
  if (kind == a) return 0.0;              /* no flow through the wall */
  return 2.0 * G->wall[face][kind] - f[at3(G, s)]; /* wall value is the mean */
}

void ora_ghost_fill(const ora_grid* G, double* f, int kind) {
  const int g = G->g;
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    /* within the pass along a, every write is a ghost layer of a and every
     * read an interior index of a (dims >= 2g), so the rows are independent */
#pragma omp parallel for collapse(2) schedule(static)
    for (int qc = -g; qc < G->n[c] + g; ++qc)
      for (int qb = -g; qb < G->n[b] + g; ++qb)
        for (int m = 1; m <= g; ++m) {
          int q[3];
          q[b] = qb;
          q[c] = qc;
          q[a] = -m;
          f[at3(G, q)] = ghost_value(G, f, kind, a, 2 * a, m, q);
          q[a] = G->n[a] - 1 + m;
          f[at3(G, q)] = ghost_value(G, f, kind, a, 2 * a + 1, m, q);
        }
  }
}

/* ------------------------------------------------------------------- RHS */

static inline double val(const ora_grid* G, const double* f, const int p[3], int d1, int o1,
                         int d2, int o2) {
  int q[3] = {p[0], p[1], p[2]};
  q[d1] += o1;
  q[d2] += o2;
  return f[at3(G, q)];
}

/* Transverse velocity f_d interpolated to the point of component c (d != c).
 * Along c the point lies between offsets 0 and +1 of f_d, along d between
 * offsets -1 and 0. */
static double interp(const ora_grid* G, const double* fd, int c, int d, const int p[3]) {
  if (G->order == 2) {
    double s = 0.0;
    for (int oc = 0; oc <= 1; ++oc)
      for (int od = -1; od <= 0; ++od) s += val(G, fd, p, c, oc, d, od);
    return 0.25 * s;
  }
  static const double wgt[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
  double s = 0.0;
  for (int ac = 0; ac < 4; ++ac)
    for (int ad = 0; ad < 4; ++ad) s += wgt[ac] * wgt[ad] * val(G, fd, p, c, ac - 1, d, ad - 2);
  return s;
}

/* Flux of c-momentum in direction d through the side of the control volume
 * of f_c that lies between the points q and q + e_d of f_c (for d = c: the
 * cell centre between them; otherwise the cell edge).  There f_c is the mean
 * of f_c(q) and f_c(q + e_d), and f_d the mean of f_d(q) and f_d(q + e_c). */
static double flux_cd(const ora_grid* G, const double* const f[3], int c, int d, const int q[3]) {
  const double fc = 0.5 * (val(G, f[c], q, d, 0, d, 0) + val(G, f[c], q, d, 1, d, 0));
  const double fd = 0.5 * (val(G, f[d], q, c, 0, c, 0) + val(G, f[d], q, c, 1, c, 0));
  return fc * fd;
}

/* F_c = -sum_d vel_d * d(f_c)/dx_d + nu * sum_d d2(f_c)/dx_d^2 at point p,
 * or, in the flux form, F_c = -sum_d (flux_cd(p) - flux_cd(p - e_d)) / h_d
 * + nu * sum_d d2(f_c)/dx_d^2. */
static double rhs_point(const ora_grid* G, const double* const f[3], int c, const int p[3]) {
  const double* fc = f[c];
  const double f0 = fc[at3(G, p)];
  double adv = 0.0, lap = 0.0;
  if (G->form == ORA_FLUX) {
    for (int d = 0; d < 3; ++d) {
      const double h = G->h[d];
      const double p1 = val(G, fc, p, d, 1, d, 0), m1 = val(G, fc, p, d, -1, d, 0);
      int pm[3] = {p[0], p[1], p[2]};
      pm[d] -= 1;
      adv += (flux_cd(G, f, c, d, p) - flux_cd(G, f, c, d, pm)) / h;
      lap += (p1 - 2.0 * f0 + m1) / (h * h);
    }
    return -adv + G->nu * lap;
  }
  for (int d = 0; d < 3; ++d) {
    const double h = G->h[d];
    const double p1 = val(G, fc, p, d, 1, d, 0), m1 = val(G, fc, p, d, -1, d, 0);
    double deriv, second;
    if (G->order == 2) {
      deriv = (p1 - m1) / (2.0 * h);
      second = (p1 - 2.0 * f0 + m1) / (h * h);
    } else {
      const double p2 = val(G, fc, p, d, 2, d, 0), m2 = val(G, fc, p, d, -2, d, 0);
      deriv = (-p2 + 8.0 * p1 - 8.0 * m1 + m2) / (12.0 * h);
      second = (-p2 + 16.0 * p1 - 30.0 * f0 + 16.0 * m1 - m2) / (12.0 * h * h);
    }
    const double vel = (d == c) ? f0 : interp(G, f[d], c, d, p);
    adv += vel * deriv;
    lap += second;
  }
  return -adv + G->nu * lap;
}

void ora_rhs(const ora_grid* G, const double* u, const double* v, const double* w, double* fu,
             double* fv, double* fw) {
  const double* f[3] = {u, v, w};
  double* out[3] = {fu, fv, fw};
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        for (int c = 0; c < 3; ++c) out[c][at3(G, p)] = rhs_point(G, f, c, p);
      }
}

/* A face of component c that lies on a wall (index n_c - 1 with a wall on
 * the high side of axis c). */
static inline int wall_face(const ora_grid* G, int c, const int p[3]) {
  return G->bc[2 * c + 1] == ORA_WALL && p[c] == G->n[c] - 1;
}

void ora_stage(const ora_grid* G, double a, const double* const x[3], double b,
               const double* const y[3], double c, double* const out[3]) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        const size_t q = at3(G, p);
        for (int m = 0; m < 3; ++m) {
          if (wall_face(G, m, p)) {
            out[m][q] = 0.0;
            continue;
          }
          double s = b * y[m][q] + c * rhs_point(G, y, m, p);
          if (a != 0.0) s += a * x[m][q];
          out[m][q] = s;
        }
      }
}

/* ------------------------------------------------------------- pressure */

void ora_divergence(const ora_grid* G, const double* const w[3], double c_dt, double* r) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        double s = 0.0;
        for (int d = 0; d < 3; ++d)
          s += (w[d][at3(G, p)] - val(G, w[d], p, d, -1, d, 0)) / G->h[d];
        r[at3(G, p)] = s / c_dt;
      }
}

void ora_jacobi_sweep(const ora_grid* G, const double* p, const double* r, double* p_out) {
  double diag = 0.0;
  for (int d = 0; d < 3; ++d) diag += 2.0 / (G->h[d] * G->h[d]);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int q[3] = {i, j, k};
        double nb = 0.0;
        for (int d = 0; d < 3; ++d)
          nb += (val(G, p, q, d, 1, d, 0) + val(G, p, q, d, -1, d, 0)) / (G->h[d] * G->h[d]);
        const double pc = p[at3(G, q)];
        p_out[at3(G, q)] = pc + G->omega * ((nb - r[at3(G, q)]) / diag - pc);
      }
  ora_ghost_fill(G, p_out, ORA_P);
}

void ora_jacobi(const ora_grid* G, double* p, const double* r, double* tmp, int iters) {
  double* src = p;
  double* dst = tmp;
  for (int it = 0; it < iters; ++it) {
    ora_jacobi_sweep(G, src, r, dst);
    double* t = src;
    src = dst;
    dst = t;
  }
  if (src != p) memcpy(p, src, total(G) * sizeof(double));
}

void ora_project(const ora_grid* G, const double* const w[3], const double* p, double c_dt,
                 double* const u_out[3]) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int q[3] = {i, j, k};
        const size_t o = at3(G, q);
        for (int d = 0; d < 3; ++d) {
          if (wall_face(G, d, q)) {
            u_out[d][o] = 0.0;
            continue;
          }
          const double grad = (val(G, p, q, d, 1, d, 0) - p[o]) / G->h[d];
          u_out[d][o] = w[d][o] - c_dt * grad;
        }
      }
}

/* ------------------------------------------------------------- RK2 step */

void ora_rk2_step(const ora_grid* G, double* const u[3], double* p, double dt, int iters,
                  double* const scratch[8]) {
  double* const W[3] = {scratch[0], scratch[1], scratch[2]};
  double* const U1[3] = {scratch[3], scratch[4], scratch[5]};
  double* R = scratch[6];
  double* T = scratch[7];
  const double* cu[3] = {u[0], u[1], u[2]};
  const double* cW[3] = {W[0], W[1], W[2]};
  const double* cU1[3] = {U1[0], U1[1], U1[2]};

  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, u[c], c);
  ora_ghost_fill(G, p, ORA_P);

  /* stage 1: w = u^n + dt F(u^n), projected with c dt = dt */
  ora_stage(G, 0.0, NULL, 1.0, cu, dt, W);
  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, W[c], c);
  ora_divergence(G, cW, dt, R);
  ora_jacobi(G, p, R, T, iters);
  ora_project(G, cW, p, dt, U1);
  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, U1[c], c);

  /* stage 2: w = 1/2 u^n + 1/2 u1 + 1/2 dt F(u1), projected with c dt = dt/2 */
  ora_stage(G, 0.5, cu, 0.5, cU1, 0.5 * dt, W);
  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, W[c], c);
  ora_divergence(G, cW, 0.5 * dt, R);
  ora_jacobi(G, p, R, T, iters);
  ora_project(G, cW, p, 0.5 * dt, u);
  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, u[c], c);
}

/* ------------------------------------------------------------ reductions */

void ora_reduce(const ora_grid* G, const double* const u[3], double* ke, double* umax,
                double* divmax) {
  const int nz = G->n[2];
  double* part = (double*)calloc((size_t)nz * 3, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k) {
    double s = 0.0, m = 0.0, dm = 0.0;
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int q[3] = {i, j, k};
        const size_t o = at3(G, q);
        double div = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double x = u[d][o];
          s += x * x;
          if (fabs(x) > m) m = fabs(x);
          div += (x - val(G, u[d], q, d, -1, d, 0)) / G->h[d];
        }
        if (fabs(div) > dm) dm = fabs(div);
      }
    part[3 * k] = s;
    part[3 * k + 1] = m;
    part[3 * k + 2] = dm;
  }
  double s = 0.0, m = 0.0, dm = 0.0;
  for (int k = 0; k < nz; ++k) {
    s += part[3 * k];
    if (part[3 * k + 1] > m) m = part[3 * k + 1];
    if (part[3 * k + 2] > dm) dm = part[3 * k + 2];
  }
  free(part);
  if (ke) *ke = 0.5 * s * G->h[0] * G->h[1] * G->h[2];
  if (umax) *umax = m;
  if (divmax) *divmax = dm;
}

void ora_laplace_p(const ora_grid* G, const double* p, double* lp) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int q[3] = {i, j, k};
        const double pc = p[at3(G, q)];
        double s = 0.0;
        for (int d = 0; d < 3; ++d)
          s += (val(G, p, q, d, 1, d, 0) - 2.0 * pc + val(G, p, q, d, -1, d, 0)) /
               (G->h[d] * G->h[d]);
        lp[at3(G, q)] = s;
      }
}

double ora_residual(const ora_grid* G, const double* p, const double* r) {
  const int nz = G->n[2];
  double* part = (double*)calloc((size_t)nz, sizeof(double));
  double* lp = (double*)calloc(total(G), sizeof(double));
  ora_laplace_p(G, p, lp);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k) {
    double s = 0.0;
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const size_t o = at(G, i, j, k);
        const double e = lp[o] - r[o];
        s += e * e;
      }
    part[k] = s;
  }
  double s = 0.0;
  for (int k = 0; k < nz; ++k) s += part[k];
  free(part);
  free(lp);
  return sqrt(s);
}

int ora_set_threads(int n) {
#ifdef _OPENMP
  static int dflt = 0;
  if (dflt == 0) dflt = omp_get_max_threads();
  omp_set_num_threads(n > 0 ? n : dflt);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
