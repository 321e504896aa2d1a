/* FP64 CPU oracle: discrete adjoint of the RK2 projection step.
 * TEST INFRASTRUCTURE ONLY (see cfd_oracle.h).
 *
 * The adjoint is the transpose of the forward oracle's own statements,
 * taken in reverse order, in scatter form: every forward assignment
 * y = sum_k a_k x_k becomes xbar_k += a_k ybar followed by ybar = 0, and a
 * ghost fill g = A + S src becomes srcbar += S gbar, gbar = 0 (the passes
 * z, y, x in that order, the reverse of the fill).  Nonlinear terms are
 * linearised at the stored forward states u^n and u1 of the step.  The
 * viscosity enters F linearly, so dL/dnu = sum over stages of
 * c dt <wbar, lap(y)>.  Sequential loops (scatter updates overlap).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "cfd_oracle.h"

static inline long ext(const ora_grid* G, int a) { return (long)G->n[a] + 2L * G->g; }
static inline size_t at3(const ora_grid* G, const int q[3]) {
  return ((size_t)(q[2] + G->g) * (size_t)ext(G, 1) + (size_t)(q[1] + G->g)) * (size_t)ext(G, 0) +
         (size_t)(q[0] + G->g);
}
static size_t total(const ora_grid* G) { return (size_t)ext(G, 0) * ext(G, 1) * ext(G, 2); }
static inline size_t off(const ora_grid* G, const int p[3], int d1, int o1, int d2, int o2) {
  int q[3] = {p[0], p[1], p[2]};
  q[d1] += o1;
  q[d2] += o2;
  return at3(G, q);
}
static inline int wall_face(const ora_grid* G, int c, const int p[3]) {
  return G->bc[2 * c + 1] == ORA_WALL && p[c] == G->n[c] - 1;
}

/* ------------------------------------------------------- ghost fill, transposed */

/* Forward: ghost = A + S * f[src] (ghost_value in cfd_oracle.c).  Returns S
 * and the source index. */
static double ghost_coef(const ora_grid* G, int kind, int a, int face, int m, const int q[3],
                         int s[3]) {
  const int N = G->n[a];
  const int low = (face == 2 * a);
  s[0] = q[0];
  s[1] = q[1];
  s[2] = q[2];
  if (G->bc[face] == ORA_PERIODIC) {
    s[a] = low ? N - m : m - 1;
    return 1.0;
  }
  s[a] = low ? m - 1 : N - m;
  if (kind == ORA_P) return 1.0;
  if (kind == a) return 0.0;
  return -1.0;
}

void ora_ghost_fold(const ora_grid* G, double* f, int kind) {
  const int g = G->g;
  for (int a = 2; a >= 0; --a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    for (int qc = -g; qc < G->n[c] + g; ++qc)
      for (int qb = -g; qb < G->n[b] + g; ++qb)
        for (int m = 1; m <= g; ++m) {
          for (int side = 0; side < 2; ++side) {
            int q[3], s[3];
            q[b] = qb;
            q[c] = qc;
            q[a] = side == 0 ? -m : G->n[a] - 1 + m;
            const double S = ghost_coef(G, kind, a, 2 * a + side, m, q, s);
            const size_t gi = at3(G, q);
            f[at3(G, s)] += S * f[gi];
            f[gi] = 0.0;
          }
        }
  }
}

/* ------------------------------------------------------ RHS stage, transposed */

static const double W4[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};

/* Scatter of w * dF_c(y)/dy for the conservative (flux) form, order 2:
 * F_c(p) = -sum_d (E(p) - E(p - e_d)) / h_d + nu lap y_c with
 * E(q) = A(q) B(q) / 4, A = y_c(q) + y_c(q + e_d), B = y_d(q) + y_d(q + e_c);
 * dE = (B dA + A dB) / 4 (for d = c, A = B and both terms add).  Returns
 * sum_d second_d(y_c). */
static double rhs_point_adj_flux(const ora_grid* G, const double* const y[3], int c,
                                 const int p[3], double w, double* const ybar[3]) {
  const double* fc = y[c];
  const double f0 = fc[at3(G, p)];
  double lap = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double h = G->h[d];
    const double p1 = fc[off(G, p, d, 1, d, 0)], m1 = fc[off(G, p, d, -1, d, 0)];
    lap += (p1 - 2.0 * f0 + m1) / (h * h);
    const double v = w * G->nu / (h * h);
    ybar[c][off(G, p, d, 1, d, 0)] += v;
    ybar[c][off(G, p, d, -1, d, 0)] += v;
    ybar[c][at3(G, p)] += -2.0 * v;
    for (int side = 0; side < 2; ++side) {  /* E(p) with -1/h_d, E(p - e_d) with +1/h_d */
      int q[3] = {p[0], p[1], p[2]};
      q[d] -= side;
      const double wq = (side == 0 ? -w : w) / h;
      const double A = y[c][at3(G, q)] + y[c][off(G, q, d, 1, d, 0)];
      const double B = y[d][at3(G, q)] + y[d][off(G, q, c, 1, c, 0)];
      ybar[c][at3(G, q)] += 0.25 * wq * B;
      ybar[c][off(G, q, d, 1, d, 0)] += 0.25 * wq * B;
      ybar[d][at3(G, q)] += 0.25 * wq * A;
      ybar[d][off(G, q, c, 1, c, 0)] += 0.25 * wq * A;
    }
  }
  return lap;
}

/* Scatter of w * dF_c(y)/dy into ybar at point p; returns sum_d second_d(y_c)
 * (the nu-derivative of F_c) for the viscosity gradient. */
static double rhs_point_adj(const ora_grid* G, const double* const y[3], int c, const int p[3],
                            double w, double* const ybar[3]) {
  if (G->form == ORA_FLUX) return rhs_point_adj_flux(G, y, c, p, w, ybar);
  const double* fc = y[c];
  const double f0 = fc[at3(G, p)];
  double lap = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double h = G->h[d];
    /* value of the derivative and of the transverse velocity */
    double deriv, vel;
    const double p1 = fc[off(G, p, d, 1, d, 0)], m1 = fc[off(G, p, d, -1, d, 0)];
    if (G->order == 2) {
      deriv = (p1 - m1) / (2.0 * h);
      lap += (p1 - 2.0 * f0 + m1) / (h * h);
    } else {
      const double p2 = fc[off(G, p, d, 2, d, 0)], m2 = fc[off(G, p, d, -2, d, 0)];
      deriv = (-p2 + 8.0 * p1 - 8.0 * m1 + m2) / (12.0 * h);
      lap += (-p2 + 16.0 * p1 - 30.0 * f0 + 16.0 * m1 - m2) / (12.0 * h * h);
    }
    if (d == c) {
      vel = f0;
    } else if (G->order == 2) {
      vel = 0.0;
      for (int oc = 0; oc <= 1; ++oc)
        for (int od = -1; od <= 0; ++od) vel += 0.25 * y[d][off(G, p, c, oc, d, od)];
    } else {
      vel = 0.0;
      for (int ac = 0; ac < 4; ++ac)
        for (int ad = 0; ad < 4; ++ad) vel += W4[ac] * W4[ad] * y[d][off(G, p, c, ac - 1, d, ad - 2)];
    }
    /* F_c = -vel * deriv + nu * second: scatter the partial derivatives */
    double* fb = ybar[c];
    if (G->order == 2) {
      const double a = -w * vel / (2.0 * h), v = w * G->nu / (h * h);
      fb[off(G, p, d, 1, d, 0)] += a + v;
      fb[off(G, p, d, -1, d, 0)] += -a + v;
      fb[at3(G, p)] += -2.0 * v;
    } else {
      const double a = -w * vel / (12.0 * h), v = w * G->nu / (12.0 * h * h);
      fb[off(G, p, d, 2, d, 0)] += -a - v;
      fb[off(G, p, d, 1, d, 0)] += 8.0 * a + 16.0 * v;
      fb[off(G, p, d, -1, d, 0)] += -8.0 * a + 16.0 * v;
      fb[off(G, p, d, -2, d, 0)] += a - v;
      fb[at3(G, p)] += -30.0 * v;
    }
    const double dv = -w * deriv; /* d(-vel * deriv)/d vel */
    if (d == c) {
      fb[at3(G, p)] += dv;
    } else if (G->order == 2) {
      for (int oc = 0; oc <= 1; ++oc)
        for (int od = -1; od <= 0; ++od) ybar[d][off(G, p, c, oc, d, od)] += 0.25 * dv;
    } else {
      for (int ac = 0; ac < 4; ++ac)
        for (int ad = 0; ad < 4; ++ad) ybar[d][off(G, p, c, ac - 1, d, ad - 2)] += W4[ac] * W4[ad] * dv;
    }
  }
  return lap;
}

/* Transpose of ora_stage (out = a x + b y + c F(y), wall faces 0):
 * xbar += a outbar, ybar += b outbar + c (dF/dy)^T outbar (into ghosts too),
 * *nubar += c <outbar, lap y>; outbar is cleared. */
void ora_adj_stage(const ora_grid* G, double a, double* const xbar[3], double b,
                   const double* const y[3], double c, double* const ybar[3],
                   double* const outbar[3], double* nubar) {
  double nb = 0.0;
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        const size_t q = at3(G, p);
        for (int m = 0; m < 3; ++m) {
          const double ob = outbar[m][q];
          outbar[m][q] = 0.0;
          if (wall_face(G, m, p)) continue;
          if (a != 0.0) xbar[m][q] += a * ob;
          ybar[m][q] += b * ob;
          nb += c * ob * rhs_point_adj(G, y, m, p, c * ob, ybar);
        }
      }
  if (nubar) *nubar += nb;
}

/* ------------------------------------------------- pressure steps, transposed */

/* Transpose of r = D w / c_dt. */
static void adj_divergence(const ora_grid* G, double* const wbar[3], double c_dt, double* rbar) {
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        const size_t q = at3(G, p);
        const double rb = rbar[q];
        rbar[q] = 0.0;
        for (int d = 0; d < 3; ++d) {
          wbar[d][q] += rb / (G->h[d] * c_dt);
          wbar[d][off(G, p, d, -1, d, 0)] -= rb / (G->h[d] * c_dt);
        }
      }
}

/* Transpose of one sweep dst = J(src, r) followed by ghost_fill(dst). */
static void adj_sweep(const ora_grid* G, double* srcbar, double* rbar, double* dstbar) {
  double diag = 0.0;
  for (int d = 0; d < 3; ++d) diag += 2.0 / (G->h[d] * G->h[d]);
  ora_ghost_fold(G, dstbar, ORA_P);
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        const size_t q = at3(G, p);
        const double db = dstbar[q];
        dstbar[q] = 0.0;
        srcbar[q] += (1.0 - G->omega) * db;
        for (int d = 0; d < 3; ++d) {
          const double wgt = G->omega / (diag * G->h[d] * G->h[d]);
          srcbar[off(G, p, d, 1, d, 0)] += wgt * db;
          srcbar[off(G, p, d, -1, d, 0)] += wgt * db;
        }
        rbar[q] += -G->omega / diag * db;
      }
}

/* Transpose of ora_jacobi (iters sweeps on p, ping-pong, result in p). */
static void adj_jacobi(const ora_grid* G, double* pbar, double* rbar, double* tmp, int iters) {
  /* forward buffers: sweep m reads buf[m%2] and writes buf[(m+1)%2], with
   * buf[0] = p, buf[1] = tmp; an odd count ends with a copy tmp -> p */
  double* buf[2] = {pbar, tmp};
  memset(tmp, 0, total(G) * sizeof(double));
  if (iters % 2) { /* transpose of the final copy tmp -> p */
    memcpy(tmp, pbar, total(G) * sizeof(double));
    memset(pbar, 0, total(G) * sizeof(double));
  }
  for (int m = iters - 1; m >= 0; --m) adj_sweep(G, buf[m % 2], rbar, buf[(m + 1) % 2]);
}

/* Transpose of u_out = w - c_dt G p (wall faces 0). */
static void adj_project(const ora_grid* G, double* const wbar[3], double* pbar, double c_dt,
                        double* const ubar[3]) {
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        const int p[3] = {i, j, k};
        const size_t q = at3(G, p);
        for (int d = 0; d < 3; ++d) {
          const double ub = ubar[d][q];
          ubar[d][q] = 0.0;
          if (wall_face(G, d, p)) continue;
          wbar[d][q] += ub;
          pbar[off(G, p, d, 1, d, 0)] -= c_dt / G->h[d] * ub;
          pbar[q] += c_dt / G->h[d] * ub;
        }
      }
}

/* --------------------------------------------------------- one step, transposed */

void ora_adj_rk2_step(const ora_grid* G, double* const un[3], double* const u1[3], double dt,
                      int iters, double* const ubar[3], double* pbar, double* nubar,
                      double* const scratch[11]) {
  const size_t n = total(G);
  double* Wb[3] = {scratch[0], scratch[1], scratch[2]};
  double* U1b[3] = {scratch[3], scratch[4], scratch[5]};
  double* Uin[3] = {scratch[6], scratch[7], scratch[8]};
  double* Rb = scratch[9];
  double* T = scratch[10];
  for (int s = 0; s < 11; ++s) memset(scratch[s], 0, n * sizeof(double));
  const double* cun[3] = {un[0], un[1], un[2]};
  const double* cu1[3] = {u1[0], u1[1], u1[2]};

  /* stage 2, reversed: u = W - dt/2 G p; ghost(u) */
  for (int c = 0; c < 3; ++c) ora_ghost_fold(G, ubar[c], c);
  adj_project(G, Wb, pbar, 0.5 * dt, ubar);
  adj_jacobi(G, pbar, Rb, T, iters);
  adj_divergence(G, Wb, 0.5 * dt, Rb);
  for (int c = 0; c < 3; ++c) ora_ghost_fold(G, Wb[c], c);
  ora_adj_stage(G, 0.5, Uin, 0.5, cu1, 0.5 * dt, U1b, Wb, nubar);

  /* stage 1, reversed: U1 = W - dt G p; ghost(U1) */
  for (int c = 0; c < 3; ++c) ora_ghost_fold(G, U1b[c], c);
  adj_project(G, Wb, pbar, dt, U1b);
  adj_jacobi(G, pbar, Rb, T, iters);
  adj_divergence(G, Wb, dt, Rb);
  for (int c = 0; c < 3; ++c) ora_ghost_fold(G, Wb[c], c);
  ora_adj_stage(G, 0.0, NULL, 1.0, cun, dt, Uin, Wb, nubar);

  /* ghost fills at the start of the step */
  for (int c = 0; c < 3; ++c) ora_ghost_fold(G, Uin[c], c);
  ora_ghost_fold(G, pbar, ORA_P);
  for (int c = 0; c < 3; ++c) memcpy(ubar[c], Uin[c], n * sizeof(double));
}
