/* FP64 CPU oracle: geometric multigrid V-cycle for the pressure equation
 * L p = r.  TEST INFRASTRUCTURE ONLY (see the header).
 *
 * The paper solves the pressure equation of Sec. 4.1 but fixes no solver;
 * the residual-controlled solve is taken to convergence here by the
 * textbook cell-centred multigrid V-cycle (the correction scheme of
 * Briggs, Henson & McCormick, "A Multigrid Tutorial", Ch. 3, with the
 * cell-centred transfers of Wesseling, "An Introduction to Multigrid
 * Methods", Sec. 5): each level halves every axis (coarse cell I covers
 * fine cells 2I and 2I + 1, cell size doubles) and keeps the faces' kinds;
 * the operator on every level is the same 7-point L with that level's
 * cell size; the smoother is weighted Jacobi (ora_jacobi_sweep with the
 * cycle's weight); restriction averages the residual r - L p over the
 * eight fine cells of a coarse cell; prolongation interpolates the coarse
 * correction trilinearly to the fine cell centres, which lie a quarter of
 * a coarse cell from the nearest coarse centre along each axis (weights
 * 3/4 and 1/4), reading the coarse ghost layer at the faces.
 */
#include "cfd_oracle.h"

#include <stdlib.h>
#include <string.h>

static long ext(const ora_grid* G, int a) { return (long)G->n[a] + 2L * G->g; }

static size_t cells(const ora_grid* G) { return (size_t)ext(G, 0) * ext(G, 1) * ext(G, 2); }

static size_t idx(const ora_grid* G, int i, int j, int k) {
  return ((size_t)(k + G->g) * (size_t)ext(G, 1) + (size_t)(j + G->g)) * (size_t)ext(G, 0) +
         (size_t)(i + G->g);
}

int ora_mg_max_levels(const ora_grid* G) {
  int n[3] = {G->n[0], G->n[1], G->n[2]};
  int levels = 0;
  while (levels < 16 && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] >= 4 &&
         n[1] >= 4 && n[2] >= 4) {
    for (int a = 0; a < 3; ++a) n[a] /= 2;
    ++levels;
  }
  return levels;
}

void ora_mg_coarse_grid(const ora_grid* F, ora_grid* C) {
  *C = *F;
  for (int a = 0; a < 3; ++a) {
    C->n[a] = F->n[a] / 2;
    C->h[a] = 2.0 * F->h[a];
  }
}

void ora_mg_restrict_residual(const ora_grid* F, const double* p, const double* r, double* rc) {
  ora_grid C;
  ora_mg_coarse_grid(F, &C);
  double* lp = (double*)calloc(cells(F), sizeof(double));
  ora_laplace_p(F, p, lp);
  memset(rc, 0, cells(&C) * sizeof(double));
  for (int K = 0; K < C.n[2]; ++K)
    for (int J = 0; J < C.n[1]; ++J)
      for (int I = 0; I < C.n[0]; ++I) {
        double s = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              const size_t q = idx(F, 2 * I + a, 2 * J + b, 2 * K + c);
              s += r[q] - lp[q];
            }
        rc[idx(&C, I, J, K)] = s / 8.0;
      }
  free(lp);
}

void ora_mg_prolong_add(const ora_grid* F, const double* ec, double* p) {
  ora_grid C;
  ora_mg_coarse_grid(F, &C);
  const double w[2] = {0.75, 0.25};  /* nearest coarse centre, next one */
  for (int k = 0; k < F->n[2]; ++k)
    for (int j = 0; j < F->n[1]; ++j)
      for (int i = 0; i < F->n[0]; ++i) {
        /* the fine centre sits below the coarse centre for an even index */
        const int I = i / 2, J = j / 2, K = k / 2;
        const int oi = (i % 2) ? 1 : -1, oj = (j % 2) ? 1 : -1, ok = (k % 2) ? 1 : -1;
        double e = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
              e += w[a] * w[b] * w[c] * ec[idx(&C, I + a * oi, J + b * oj, K + c * ok)];
        p[idx(F, i, j, k)] += e;
      }
  ora_ghost_fill(F, p, ORA_P);
}

static void vcycle(const ora_grid* G, const ora_mg* M, int depth, double* p, const double* r) {
  ora_grid S = *G;
  S.omega = M->omega;
  double* tmp = (double*)calloc(cells(G), sizeof(double));
  if (depth == M->levels) {
    ora_jacobi(&S, p, r, tmp, M->ncoarse);
    free(tmp);
    return;
  }
  ora_jacobi(&S, p, r, tmp, M->nu1);
  ora_grid C;
  ora_mg_coarse_grid(G, &C);
  double* rc = (double*)calloc(cells(&C), sizeof(double));
  double* ec = (double*)calloc(cells(&C), sizeof(double)); /* zero guess, ghosts included */
  ora_mg_restrict_residual(G, p, r, rc);
  vcycle(&C, M, depth + 1, ec, rc);
  ora_mg_prolong_add(G, ec, p);
  ora_jacobi(&S, p, r, tmp, M->nu2);
  free(ec);
  free(rc);
  free(tmp);
}

void ora_mg_vcycle(const ora_grid* G, const ora_mg* M, double* p, const double* r) {
  vcycle(G, M, 0, p, r);
}

void ora_rk2_step_mg(const ora_grid* G, double* const u[3], double* p, double dt,
                     const ora_mg* M, int cycles, double* const scratch[8]) {
  double* const W[3] = {scratch[0], scratch[1], scratch[2]};
  double* const U1[3] = {scratch[3], scratch[4], scratch[5]};
  double* R = scratch[6];
  const double* cu[3] = {u[0], u[1], u[2]};
  const double* cW[3] = {W[0], W[1], W[2]};
  const double* cU1[3] = {U1[0], U1[1], U1[2]};
  for (int c = 0; c < 3; ++c) ora_ghost_fill(G, u[c], c);
  ora_ghost_fill(G, p, ORA_P);
  /* the two projected Heun stages of ora_rk2_step, each pressure solve
   * being 'cycles' V-cycles from the last pressure */
  for (int stage = 1; stage <= 2; ++stage) {
    const double cdt = stage == 1 ? dt : 0.5 * dt;
    if (stage == 1)
      ora_stage(G, 0.0, NULL, 1.0, cu, dt, W);
    else
      ora_stage(G, 0.5, cu, 0.5, cU1, 0.5 * dt, W);
    for (int c = 0; c < 3; ++c) ora_ghost_fill(G, W[c], c);
    ora_divergence(G, cW, cdt, R);
    for (int k = 0; k < cycles; ++k) ora_mg_vcycle(G, M, p, R);
    double* const* out = stage == 1 ? U1 : u;
    ora_project(G, cW, p, cdt, out);
    for (int c = 0; c < 3; ++c) ora_ghost_fill(G, out[c], c);
  }
}
