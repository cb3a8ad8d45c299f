/*
 * flip_oracle.c — plain FP64 CPU oracle of one FLIP time step.
 *
 * TEST INFRASTRUCTURE ONLY: called by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Every function follows
 * one passage of Centeno & Pereira, "Fluid Implicit Particle Simulation for CPU
 * and GPU" (arXiv 2404.01931), cited beside it, in the paper's order and with
 * no blocking, fusion or reordering beyond what the passage states.  OpenMP
 * only splits independent loops (and sums dot products per thread).
 *
 * Parity status: every function here is pinned by the tests in
 * tests/test_oracle_pins.py (closed forms, invariants, a brute-force gather and
 * dense solves); see the header of that file for which pin covers which part.
 */
#include "flip_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int64_t oracle_n_cells(const oracle_params* P) {
  return (int64_t)P->n[0] * P->n[1] * P->n[2];
}

/* Face-array extent of component comp along axis ax: one more node along the
 * component's own axis (MAC grid, Section 3.1.1). */
static int64_t face_dim(const oracle_params* P, int comp, int ax) {
  return (int64_t)P->n[ax] + (ax == comp ? 1 : 0);
}

int64_t oracle_n_faces(const oracle_params* P, int comp) {
  return face_dim(P, comp, 0) * face_dim(P, comp, 1) * face_dim(P, comp, 2);
}

static int64_t face_index(const oracle_params* P, int comp, int64_t a, int64_t b, int64_t c) {
  return a + face_dim(P, comp, 0) * (b + face_dim(P, comp, 1) * c);
}

static int64_t cell_index(const oracle_params* P, int64_t i, int64_t j, int64_t k) {
  return i + (int64_t)P->n[0] * (j + (int64_t)P->n[1] * k);
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

static double clampd(double v, double lo, double hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

/* Eq. 4b: h(r) = 1 - |r| on [-1, 1], 0 outside. */
double oracle_hat(double r) {
  if (r >= 0.0 && r <= 1.0) return 1.0 - r;
  if (r >= -1.0 && r < 0.0) return 1.0 + r;
  return 0.0;
}

/* Cell index of a point (Section 3.1.5 "raw index"; the paper's 16-bit hash
 * formula in Section 3.2.2 is garbled, the reading is floor(x/dx) per axis,
 * taken here as floor(x * (1/dx)) in FP64 and clamped to the grid). */
void oracle_cell_of(const oracle_params* P, double x, double y, double z, int64_t cell[3]) {
  const double inv = 1.0 / P->dx;
  const double pos[3] = {x, y, z};
  for (int ax = 0; ax < 3; ++ax)
    cell[ax] = clampi((int64_t)floor(pos[ax] * inv), 0, P->n[ax] - 1);
}

/* Grid coordinate of a point relative to the face nodes of component comp:
 * the node of index a sits at (a + off)*dx with off = 0 along the component's
 * own axis and 1/2 along the other two (MAC layout).  The coordinate is clamped
 * to the node range, so a point between a wall and the first node samples the
 * first node only (the paper does not say how transfers treat the half cell
 * next to a wall; this keeps all eight nodes inside the grid and the weights a
 * partition of unity). */
static double sample_coord(const oracle_params* P, int comp, int ax, double pos) {
  const double off = (ax == comp) ? 0.0 : 0.5;
  return clampd(pos / P->dx - off, 0.0, (double)(face_dim(P, comp, ax) - 1));
}

/* Eq. 4a: k(x_P - x_node) = h(.)h(.)h(.) in units of dx. */
double oracle_weight(const oracle_params* P, int comp, int64_t a, int64_t b, int64_t c,
                     double x, double y, double z) {
  const double pos[3] = {x, y, z};
  const int64_t node[3] = {a, b, c};
  double w = 1.0;
  for (int ax = 0; ax < 3; ++ax) w *= oracle_hat(sample_coord(P, comp, ax, pos[ax]) - (double)node[ax]);
  return w;
}

/* Section 3.1.5, Fig. 4: compute each particle's raw cell index, sort the
 * particles by it, and record per cell the offset and count of its particles
 * (the "space hash").  A stable counting sort: particles keep their relative
 * order inside a cell. */
void oracle_bin(const oracle_params* P, int64_t np, const double* x, const double* y,
                const double* z, int64_t* start, int64_t* order) {
  const int64_t nc = oracle_n_cells(P);
  int64_t* cellid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  memset(start, 0, sizeof(int64_t) * (size_t)(nc + 1));
  for (int64_t p = 0; p < np; ++p) {
    int64_t c3[3];
    oracle_cell_of(P, x[p], y[p], z[p], c3);
    cellid[p] = cell_index(P, c3[0], c3[1], c3[2]);
    start[cellid[p] + 1] += 1;
  }
  for (int64_t c = 0; c < nc; ++c) start[c + 1] += start[c];
  for (int64_t c = 0; c < nc; ++c) cursor[c] = start[c];
  for (int64_t p = 0; p < np; ++p) order[cursor[cellid[p]]++] = p;
  free(cellid);
  free(cursor);
}

/* Section 3.1.6: gather form of the particle-to-grid transfer.  For every face
 * node, loop over the particles that can reach it and form
 *     u_node = sum_P u_P k(x_P - x_node) / sum_P k(x_P - x_node)
 * (0 where no particle reaches the node).  A particle reaches a node only if
 * its sample coordinate is within one node spacing on every axis; with the
 * half-cell staggering that confines it to cells node-1..node along the
 * component's own axis and node-1..node+1 along the other two. */
void oracle_p2g(const oracle_params* P, int comp, const double* x, const double* y,
                const double* z, const double* vel, const int64_t* start,
                const int64_t* order, double* grid, double* wsum) {
  const int64_t fx = face_dim(P, comp, 0), fy = face_dim(P, comp, 1), fz = face_dim(P, comp, 2);
  const int64_t nf = fx * fy * fz;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t node[3] = {f % fx, (f / fx) % fy, f / (fx * fy)};
    int64_t lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) {
      lo[ax] = clampi(node[ax] - 1, 0, P->n[ax] - 1);
      hi[ax] = clampi(ax == comp ? node[ax] : node[ax] + 1, 0, P->n[ax] - 1);
    }
    double swu = 0.0, sw = 0.0;
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
      for (int64_t j = lo[1]; j <= hi[1]; ++j)
        for (int64_t i = lo[0]; i <= hi[0]; ++i) {
          const int64_t c = cell_index(P, i, j, k);
          for (int64_t q = start[c]; q < start[c + 1]; ++q) {
            const int64_t p = order[q];
            const double wt = oracle_weight(P, comp, node[0], node[1], node[2], x[p], y[p], z[p]);
            swu += wt * vel[p];
            sw += wt;
          }
        }
    grid[f] = sw > 0.0 ? swu / sw : 0.0;
    if (wsum) wsum[f] = sw;
  }
}

/* Section 3.1.5: a cell holds fluid when its particle count is above zero. */
void oracle_cell_types(const oracle_params* P, const int64_t* start, uint8_t* type) {
  const int64_t nc = oracle_n_cells(P);
  for (int64_t c = 0; c < nc; ++c) type[c] = (start[c + 1] > start[c]) ? 1 : 0;
}

/* Eq. 1 / Section 2.1.3 splitting: the force step adds g*dt to the grid
 * velocity; then the solid-wall condition (Section 3.1.7) sets the normal
 * velocity on the six domain planes to zero. */
void oracle_forces_walls(const oracle_params* P, int comp, const double* u_old, double* u_star) {
  const int64_t fx = face_dim(P, comp, 0), fy = face_dim(P, comp, 1), fz = face_dim(P, comp, 2);
  const int64_t nf = fx * fy * fz;
  const double dv = P->gravity[comp] * P->dt;
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t node[3] = {f % fx, (f / fx) % fy, f / (fx * fy)};
    const int wall = (node[comp] == 0) || (node[comp] == P->n[comp]);
    u_star[f] = wall ? 0.0 : u_old[f] + dv;
  }
}

/* Eq. 6 with central differences on the MAC grid (Section 3.1.7):
 * b = -div u* in each fluid cell. */
void oracle_divergence(const oracle_params* P, const double* const u[3], const uint8_t* type,
                       double* b) {
  const int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  const int64_t nc = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    if (!type[c]) { b[c] = 0.0; continue; }
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const double du = u[0][face_index(P, 0, i + 1, j, k)] - u[0][face_index(P, 0, i, j, k)];
    const double dv = u[1][face_index(P, 1, i, j + 1, k)] - u[1][face_index(P, 1, i, j, k)];
    const double dw = u[2][face_index(P, 2, i, j, k + 1)] - u[2][face_index(P, 2, i, j, k)];
    b[c] = -(du + dv + dw) / P->dx;
  }
}

/* Number of a cell's six neighbours that are not solid walls (the domain
 * planes are the only solids). */
static int nonsolid_neighbours(const oracle_params* P, int64_t i, int64_t j, int64_t k) {
  const int64_t idx[3] = {i, j, k};
  int cnt = 0;
  for (int ax = 0; ax < 3; ++ax) {
    if (idx[ax] > 0) ++cnt;
    if (idx[ax] < P->n[ax] - 1) ++cnt;
  }
  return cnt;
}

/* Section 3.1.7: row of the seven-point Laplacian for fluid cell c,
 *   (A p)_c = dt/(rho dx^2) * ( n_c p_c - sum_{fluid neighbours m} p_m ),
 * n_c = number of non-solid neighbours (air neighbours carry p = 0, the free
 * surface condition; solid neighbours drop out, the wall condition). */
void oracle_apply_A(const oracle_params* P, const uint8_t* type, const double* p, double* Ap) {
  const int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  const int64_t nc = nx * ny * nz;
  const double s = P->dt / (P->rho * P->dx * P->dx);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    if (!type[c]) { Ap[c] = 0.0; continue; }
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    double off = 0.0;
    if (i > 0 && type[c - 1]) off += p[c - 1];
    if (i < nx - 1 && type[c + 1]) off += p[c + 1];
    if (j > 0 && type[c - nx]) off += p[c - nx];
    if (j < ny - 1 && type[c + nx]) off += p[c + nx];
    if (k > 0 && type[c - nx * ny]) off += p[c - nx * ny];
    if (k < nz - 1 && type[c + nx * ny]) off += p[c + nx * ny];
    Ap[c] = s * ((double)nonsolid_neighbours(P, i, j, k) * p[c] - off);
  }
}

static double dot_fluid(int64_t nc, const uint8_t* type, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t c = 0; c < nc; ++c)
    if (type[c]) s += a[c] * b[c];
  return s;
}

/* Section 3.1.7: preconditioned conjugate gradient on A p = b (the paper's
 * CPU solver; it defers the preconditioner to Bridson, read here as the
 * diagonal (Jacobi) one).  Start p = 0; stop when the recursive residual
 * satisfies ||r||_2 <= tol * ||b||_2.  Returns the number of A-applications,
 * or -1 when max_iter is reached first. */
int oracle_pcg(const oracle_params* P, const uint8_t* type, const double* b, double tol,
               int max_iter, double* x, double* rel_res) {
  const int64_t nx = P->n[0], ny = P->n[1];
  const int64_t nc = oracle_n_cells(P);
  const double s = P->dt / (P->rho * P->dx * P->dx);
  double* r = (double*)malloc(sizeof(double) * (size_t)nc);
  double* zz = (double*)malloc(sizeof(double) * (size_t)nc);
  double* d = (double*)malloc(sizeof(double) * (size_t)nc);
  double* q = (double*)malloc(sizeof(double) * (size_t)nc);
  double* minv = (double*)malloc(sizeof(double) * (size_t)nc);
  int result = -1;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    x[c] = 0.0;
    r[c] = type[c] ? b[c] : 0.0;
    minv[c] = type[c] ? 1.0 / (s * (double)nonsolid_neighbours(P, i, j, k)) : 0.0;
    zz[c] = minv[c] * r[c];
    d[c] = zz[c];
  }
  const double bnorm = sqrt(dot_fluid(nc, type, r, r));
  double rz = dot_fluid(nc, type, r, zz);
  double rnorm = bnorm;
  if (bnorm == 0.0 || rnorm <= tol * bnorm) {
    result = 0;
  } else {
    for (int it = 1; it <= max_iter; ++it) {
      oracle_apply_A(P, type, d, q);
      const double alpha = rz / dot_fluid(nc, type, d, q);
#pragma omp parallel for schedule(static)
      for (int64_t c = 0; c < nc; ++c)
        if (type[c]) {
          x[c] += alpha * d[c];
          r[c] -= alpha * q[c];
        }
      rnorm = sqrt(dot_fluid(nc, type, r, r));
      if (rnorm <= tol * bnorm) { result = it; break; }
#pragma omp parallel for schedule(static)
      for (int64_t c = 0; c < nc; ++c) zz[c] = minv[c] * r[c];
      const double rz_new = dot_fluid(nc, type, r, zz);
      const double beta = rz_new / rz;
      rz = rz_new;
#pragma omp parallel for schedule(static)
      for (int64_t c = 0; c < nc; ++c)
        if (type[c]) d[c] = zz[c] + beta * d[c];
    }
  }
  if (rel_res) *rel_res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(r); free(zz); free(d); free(q); free(minv);
  return result;
}

/* Eq. 5: u_new = u* - dt/rho * (p_{+} - p_{-})/dx on faces with a fluid cell on
 * at least one side (air cells carry p = 0); wall faces stay 0; faces between
 * two air cells keep u*. */
void oracle_project(const oracle_params* P, int comp, const double* u_star, const double* p,
                    const uint8_t* type, double* u_new) {
  const int64_t fx = face_dim(P, comp, 0), fy = face_dim(P, comp, 1), fz = face_dim(P, comp, 2);
  const int64_t nf = fx * fy * fz;
  const double scale = P->dt / (P->rho * P->dx);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nf; ++f) {
    int64_t node[3] = {f % fx, (f / fx) % fy, f / (fx * fy)};
    if (node[comp] == 0 || node[comp] == P->n[comp]) { u_new[f] = 0.0; continue; }
    const int64_t cp = cell_index(P, node[0], node[1], node[2]);
    node[comp] -= 1;
    const int64_t cm = cell_index(P, node[0], node[1], node[2]);
    if (type[cp] || type[cm])
      u_new[f] = u_star[f] - scale * ((type[cp] ? p[cp] : 0.0) - (type[cm] ? p[cm] : 0.0));
    else
      u_new[f] = u_star[f];
  }
}

/* Section 3.1.8: trilinear interpolation from the eight face nodes around the
 * point, with the Eq. 4 weights (the same weights the transfer to the grid
 * uses). */
double oracle_interp(const oracle_params* P, int comp, const double* field, double x, double y,
                     double z) {
  const double pos[3] = {x, y, z};
  int64_t base[3], dim[3];
  for (int ax = 0; ax < 3; ++ax) {
    dim[ax] = face_dim(P, comp, ax);
    base[ax] = clampi((int64_t)floor(sample_coord(P, comp, ax, pos[ax])), 0,
                      dim[ax] >= 2 ? dim[ax] - 2 : 0);
  }
  double acc = 0.0;
  for (int dc = 0; dc < 2; ++dc)
    for (int db = 0; db < 2; ++db)
      for (int da = 0; da < 2; ++da) {
        const int64_t a = base[0] + da, b = base[1] + db, c = base[2] + dc;
        if (a >= dim[0] || b >= dim[1] || c >= dim[2]) continue;
        acc += oracle_weight(P, comp, a, b, c, x, y, z) * field[face_index(P, comp, a, b, c)];
      }
  return acc;
}

/* Section 3.1.8 then Section 3.1.3.  First the change of the grid velocity,
 * du = u_new - u_old, is formed and stored; then for each particle the new grid
 * velocity U and the change dU are interpolated and blended:
 *     v_P <- r (v_P + dU) + (1 - r) U          (FLIP share r, Section 2.1.4)
 * Then forward Euler x_P <- x_P + v dt (v = the blended particle velocity, or U
 * when advect_source = 1) and the clamp back into the domain by the skin width
 * along each axis. */
void oracle_g2p(const oracle_params* P, int64_t np, double* x, double* y, double* z, double* u,
                double* v, double* w, const double* const u_old[3],
                const double* const u_new[3]) {
  double* du[3];
  for (int comp = 0; comp < 3; ++comp) {
    const int64_t nf = oracle_n_faces(P, comp);
    du[comp] = (double*)malloc(sizeof(double) * (size_t)nf);
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < nf; ++f) du[comp][f] = u_new[comp][f] - u_old[comp][f];
  }
  const double r = P->flip_ratio;
  double* vel[3] = {u, v, w};
  double* pos[3] = {x, y, z};
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; ++p) {
    double U[3], Vb[3];
    for (int comp = 0; comp < 3; ++comp) {
      U[comp] = oracle_interp(P, comp, u_new[comp], x[p], y[p], z[p]);
      const double dU = oracle_interp(P, comp, du[comp], x[p], y[p], z[p]);
      Vb[comp] = r * (vel[comp][p] + dU) + (1.0 - r) * U[comp];
    }
    for (int ax = 0; ax < 3; ++ax) {
      vel[ax][p] = Vb[ax];
      const double adv = (P->advect_source == 1) ? U[ax] : Vb[ax];
      const double hi = (double)P->n[ax] * P->dx - P->skin;
      pos[ax][p] = clampd(pos[ax][p] + adv * P->dt, P->skin, hi);
    }
  }
  for (int comp = 0; comp < 3; ++comp) free(du[comp]);
}

double oracle_div_norm(const oracle_params* P, const double* const u[3], const uint8_t* type) {
  const int64_t nc = oracle_n_cells(P);
  double* d = (double*)malloc(sizeof(double) * (size_t)nc);
  oracle_divergence(P, u, type, d);
  const double s = sqrt(dot_fluid(nc, type, d, d));
  free(d);
  return s;
}

/* One FLIP step (Section 3 order; gravity enters after the transfer to the
 * grid, per the force-advect-project splitting of Section 2.1.3):
 *   bin -> P2G -> cell types -> gravity + walls -> b = -div u* -> PCG ->
 *   Eq. 5 projection -> G2P blend -> forward Euler + clamp. */
static int step_with_dt(const oracle_params* P, int64_t np, double* x, double* y, double* z,
                        double* u, double* v, double* w, oracle_fields* out,
                        oracle_stats* stats);

/* Sec. 3.1.4: with a CFL number alpha > 0 the step takes
 * dt = min(dt_max, alpha dx / max_p |v_p|) from the particle velocities at its
 * start (dt_max when every particle rests). */
double oracle_cfl_dt(const oracle_params* P, int64_t np, const double* u, const double* v,
                     const double* w) {
  if (!(P->cfl > 0.0)) return P->dt;
  double vmax = 0.0;
  for (int64_t q = 0; q < np; ++q) {
    const double s = sqrt(u[q] * u[q] + v[q] * v[q] + w[q] * w[q]);
    if (s > vmax) vmax = s;
  }
  if (vmax <= 0.0) return P->dt;
  const double dt = P->cfl * P->dx / vmax;
  return dt < P->dt ? dt : P->dt;
}

int oracle_step(const oracle_params* P, int64_t np, double* x, double* y, double* z, double* u,
                double* v, double* w, oracle_fields* out, oracle_stats* stats) {
  oracle_params Q = *P;
  Q.dt = oracle_cfl_dt(P, np, u, v, w);
  if (stats) stats->dt = Q.dt;
  return step_with_dt(&Q, np, x, y, z, u, v, w, out, stats);
}

static int step_with_dt(const oracle_params* P, int64_t np, double* x, double* y, double* z,
                        double* u, double* v, double* w, oracle_fields* out,
                        oracle_stats* stats) {
  const int64_t nc = oracle_n_cells(P);
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  double* uo[3];
  double* us[3];
  double* un[3];
  for (int d = 0; d < 3; ++d) {
    const size_t nf = (size_t)oracle_n_faces(P, d);
    uo[d] = (double*)malloc(sizeof(double) * nf);
    us[d] = (double*)malloc(sizeof(double) * nf);
    un[d] = (double*)malloc(sizeof(double) * nf);
  }
  double* p = (double*)malloc(sizeof(double) * (size_t)nc);
  double* b = (double*)malloc(sizeof(double) * (size_t)nc);
  uint8_t* type = (uint8_t*)malloc((size_t)nc);
  int status = 0;
  if (!start || !order || !p || !b || !type) status = 3;
  for (int d = 0; d < 3; ++d)
    if (!uo[d] || !us[d] || !un[d]) status = 3;
  if (status == 0) {
    oracle_bin(P, np, x, y, z, start, order);
    const double* pv[3] = {u, v, w};
    for (int d = 0; d < 3; ++d) oracle_p2g(P, d, x, y, z, pv[d], start, order, uo[d], NULL);
    oracle_cell_types(P, start, type);
    for (int d = 0; d < 3; ++d) oracle_forces_walls(P, d, uo[d], us[d]);
    const double* usc[3] = {us[0], us[1], us[2]};
    oracle_divergence(P, usc, type, b);
    int64_t nfluid = 0;
    for (int64_t c = 0; c < nc; ++c) nfluid += type[c];
    /* A is singular exactly when a connected fluid region has no air
     * neighbour; with the domain planes as the only solids such a region is
     * closed under adjacency, i.e. it is the whole grid. */
    if (nfluid == nc && nc > 0) status = 2;
    double rel = 0.0;
    int iters = 0;
    if (status == 0) {
      if (P->preconditioner == 1)
        iters = oracle_pcg_mg(P, type, b, P->cg_tol, P->cg_max_iter, P->mg_nu, P->mg_omega, p, &rel);
      else if (P->preconditioner == 2)
        iters = oracle_rbgs(P, type, b, P->cg_tol, P->cg_max_iter, p, &rel);
      else
        iters = oracle_pcg(P, type, b, P->cg_tol, P->cg_max_iter, p, &rel);
      if (iters < 0) status = 1;
      for (int d = 0; d < 3; ++d) oracle_project(P, d, us[d], p, type, un[d]);
      const double* unc[3] = {un[0], un[1], un[2]};
      const double* uoc[3] = {uo[0], uo[1], uo[2]};
      const double d0 = oracle_div_norm(P, usc, type);
      const double d1 = oracle_div_norm(P, unc, type);
      if (stats) {
        stats->cg_iterations = iters;
        stats->cg_rel_residual = rel;
        stats->rel_divergence = d0 > 0.0 ? d1 / d0 : 0.0;
        stats->n_fluid = nfluid;
      }
      oracle_g2p(P, np, x, y, z, u, v, w, uoc, unc);
      if (out) {
        for (int d = 0; d < 3; ++d) {
          const size_t nb = sizeof(double) * (size_t)oracle_n_faces(P, d);
          if (out->u_old[d]) memcpy(out->u_old[d], uo[d], nb);
          if (out->u_star[d]) memcpy(out->u_star[d], us[d], nb);
          if (out->u_new[d]) memcpy(out->u_new[d], un[d], nb);
        }
        if (out->pressure) memcpy(out->pressure, p, sizeof(double) * (size_t)nc);
        if (out->rhs) memcpy(out->rhs, b, sizeof(double) * (size_t)nc);
        if (out->type) memcpy(out->type, type, (size_t)nc);
      }
    }
  }
  free(start); free(order); free(p); free(b); free(type);
  for (int d = 0; d < 3; ++d) { free(uo[d]); free(us[d]); free(un[d]); }
  return status;
}

/* ------------------------------------------------------------------------
 * Multigrid V-cycle preconditioner (red-black Gauss-Seidel smoothing, Sec. 3.2.3)
 * ------------------------------------------------------------------------ */

typedef struct {
  int64_t n[3];
  double s;       /* dt / (rho h_l^2) */
  uint8_t* t;     /* fluid flags */
  double* x;
  double* b;
} mg_level;

int oracle_mg_levels(const oracle_params* P, int32_t dims[][3]) {
  int64_t n[3] = {P->n[0], P->n[1], P->n[2]};
  int L = 0;
  for (;;) {
    for (int a = 0; a < 3; ++a) dims[L][a] = (int32_t)n[a];
    ++L;
    const int64_t m = n[0] > n[1] ? (n[0] > n[2] ? n[0] : n[2]) : (n[1] > n[2] ? n[1] : n[2]);
    if (m <= 4 || L == ORACLE_MG_MAX_LEVELS) break;
    for (int a = 0; a < 3; ++a) n[a] = (n[a] + 1) / 2;
  }
  return L;
}

static int64_t lv_idx(const mg_level* v, int64_t i, int64_t j, int64_t k) {
  return i + v->n[0] * (j + v->n[1] * k);
}

static int lv_nonsolid(const mg_level* v, int64_t i, int64_t j, int64_t k) {
  const int64_t idx[3] = {i, j, k};
  int cnt = 0;
  for (int ax = 0; ax < 3; ++ax) cnt += (idx[ax] > 0) + (idx[ax] < v->n[ax] - 1);
  return cnt;
}

/* sum of x over the fluid neighbours of cell (i,j,k) */
static double lv_nbr_sum(const mg_level* v, const double* x, int64_t i, int64_t j, int64_t k) {
  const int64_t di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
  double s = 0.0;
  for (int q = 0; q < 6; ++q) {
    const int64_t a = i + di[q], b = j + dj[q], c = k + dk[q];
    if (a < 0 || b < 0 || c < 0 || a >= v->n[0] || b >= v->n[1] || c >= v->n[2]) continue;
    const int64_t m = lv_idx(v, a, b, c);
    if (v->t[m]) s += x[m];
  }
  return s;
}

/* One Gauss-Seidel half-sweep over the fluid cells of one colour (i+j+k even =
 * red = 0): x_c <- (b_c + s sum_fluid-neighbours x_n) / (s n_c).  Cells of one
 * colour only have neighbours of the other colour, so the order inside a colour
 * does not matter. */
static void lv_half_sweep(mg_level* v, int colour) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < v->n[2]; ++k)
    for (int64_t j = 0; j < v->n[1]; ++j)
      for (int64_t i = 0; i < v->n[0]; ++i) {
        if (((i + j + k) & 1) != colour) continue;
        const int64_t c = lv_idx(v, i, j, k);
        if (!v->t[c]) continue;
        v->x[c] = (v->b[c] + v->s * lv_nbr_sum(v, v->x, i, j, k)) /
                  (v->s * (double)lv_nonsolid(v, i, j, k));
      }
}

static void mg_vcycle_level(mg_level* lv, int l, int L, int nu, double omega) {
  mg_level* v = &lv[l];
  const int64_t nc = v->n[0] * v->n[1] * v->n[2];
  for (int64_t c = 0; c < nc; ++c) v->x[c] = 0.0;
  if (l == L - 1) {
    for (int s = 0; s < ORACLE_MG_COARSE_SWEEPS; ++s) { lv_half_sweep(v, 0); lv_half_sweep(v, 1); }
    for (int s = 0; s < ORACLE_MG_COARSE_SWEEPS; ++s) { lv_half_sweep(v, 1); lv_half_sweep(v, 0); }
    return;
  }
  for (int s = 0; s < nu; ++s) { lv_half_sweep(v, 0); lv_half_sweep(v, 1); }
  /* residual of the fine level, restricted: b_{l+1} = (1/16) sum of fluid children.
   * 1/8 averages the children; the extra 1/2 matches the coarse equation to the
   * Galerkin operator P^T A P / 8, which for piecewise-constant P is twice the
   * 7-point operator rediscretised at spacing 2h. */
  mg_level* w = &lv[l + 1];
  const int64_t ncc = w->n[0] * w->n[1] * w->n[2];
  for (int64_t c = 0; c < ncc; ++c) w->b[c] = 0.0;
  for (int64_t k = 0; k < v->n[2]; ++k)
    for (int64_t j = 0; j < v->n[1]; ++j)
      for (int64_t i = 0; i < v->n[0]; ++i) {
        const int64_t c = lv_idx(v, i, j, k);
        if (!v->t[c]) continue;
        const double ax = v->s * ((double)lv_nonsolid(v, i, j, k) * v->x[c] - lv_nbr_sum(v, v->x, i, j, k));
        w->b[lv_idx(w, i / 2, j / 2, k / 2)] += (v->b[c] - ax) / 16.0;
      }
  mg_vcycle_level(lv, l + 1, L, nu, omega);
  /* correction: each fluid cell adds omega times its parent's value */
  for (int64_t k = 0; k < v->n[2]; ++k)
    for (int64_t j = 0; j < v->n[1]; ++j)
      for (int64_t i = 0; i < v->n[0]; ++i) {
        const int64_t c = lv_idx(v, i, j, k);
        if (v->t[c]) v->x[c] += omega * w->x[lv_idx(w, i / 2, j / 2, k / 2)];
      }
  for (int s = 0; s < nu; ++s) { lv_half_sweep(v, 1); lv_half_sweep(v, 0); }
}

static int mg_build(const oracle_params* P, const uint8_t* type, mg_level* lv) {
  int32_t dims[ORACLE_MG_MAX_LEVELS][3];
  const int L = oracle_mg_levels(P, dims);
  for (int l = 0; l < L; ++l) {
    for (int a = 0; a < 3; ++a) lv[l].n[a] = dims[l][a];
    const double h = P->dx * (double)(1 << l);
    lv[l].s = P->dt / (P->rho * h * h);
    const size_t nc = (size_t)(lv[l].n[0] * lv[l].n[1] * lv[l].n[2]);
    lv[l].t = (uint8_t*)calloc(nc, 1);
    lv[l].x = (double*)calloc(nc, sizeof(double));
    lv[l].b = (double*)calloc(nc, sizeof(double));
  }
  const int64_t nc0 = lv[0].n[0] * lv[0].n[1] * lv[0].n[2];
  for (int64_t c = 0; c < nc0; ++c) lv[0].t[c] = type[c] == 1;
  for (int l = 1; l < L; ++l) {
    const mg_level* f = &lv[l - 1];
    for (int64_t k = 0; k < f->n[2]; ++k)
      for (int64_t j = 0; j < f->n[1]; ++j)
        for (int64_t i = 0; i < f->n[0]; ++i)
          if (f->t[lv_idx(f, i, j, k)]) lv[l].t[lv_idx(&lv[l], i / 2, j / 2, k / 2)] = 1;
  }
  return L;
}

static void mg_free(mg_level* lv, int L) {
  for (int l = 0; l < L; ++l) { free(lv[l].t); free(lv[l].x); free(lv[l].b); }
}

static void mg_apply(mg_level* lv, int L, int nu, double omega, const double* r, double* z) {
  const int64_t nc0 = lv[0].n[0] * lv[0].n[1] * lv[0].n[2];
  for (int64_t c = 0; c < nc0; ++c) lv[0].b[c] = lv[0].t[c] ? r[c] : 0.0;
  mg_vcycle_level(lv, 0, L, nu, omega);
  for (int64_t c = 0; c < nc0; ++c) z[c] = lv[0].t[c] ? lv[0].x[c] : 0.0;
}

void oracle_mg_vcycle(const oracle_params* P, const uint8_t* type, const double* r, double* z,
                      int nu, double omega) {
  mg_level lv[ORACLE_MG_MAX_LEVELS];
  const int L = mg_build(P, type, lv);
  mg_apply(lv, L, nu, omega, r, z);
  mg_free(lv, L);
}

/* PCG with the V-cycle as M^{-1}; the same iteration and stopping rule as
 * oracle_pcg (p0 = 0, ||r|| <= tol ||b||). */
int oracle_pcg_mg(const oracle_params* P, const uint8_t* type, const double* b, double tol,
                  int max_iter, int nu, double omega, double* x, double* rel_res) {
  const int64_t nc = oracle_n_cells(P);
  mg_level lv[ORACLE_MG_MAX_LEVELS];
  const int L = mg_build(P, type, lv);
  double* r = (double*)malloc(sizeof(double) * (size_t)nc);
  double* zz = (double*)malloc(sizeof(double) * (size_t)nc);
  double* d = (double*)malloc(sizeof(double) * (size_t)nc);
  double* q = (double*)malloc(sizeof(double) * (size_t)nc);
  int result = -1;
  for (int64_t c = 0; c < nc; ++c) {
    x[c] = 0.0;
    r[c] = type[c] ? b[c] : 0.0;
  }
  mg_apply(lv, L, nu, omega, r, zz);
  for (int64_t c = 0; c < nc; ++c) d[c] = zz[c];
  const double bnorm = sqrt(dot_fluid(nc, type, r, r));
  double rz = dot_fluid(nc, type, r, zz);
  double rnorm = bnorm;
  if (bnorm == 0.0) {
    result = 0;
  } else {
    for (int it = 1; it <= max_iter; ++it) {
      oracle_apply_A(P, type, d, q);
      const double alpha = rz / dot_fluid(nc, type, d, q);
      for (int64_t c = 0; c < nc; ++c)
        if (type[c]) { x[c] += alpha * d[c]; r[c] -= alpha * q[c]; }
      rnorm = sqrt(dot_fluid(nc, type, r, r));
      if (rnorm <= tol * bnorm) { result = it; break; }
      mg_apply(lv, L, nu, omega, r, zz);
      const double rz_new = dot_fluid(nc, type, r, zz);
      const double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t c = 0; c < nc; ++c)
        if (type[c]) d[c] = zz[c] + beta * d[c];
    }
  }
  if (rel_res) *rel_res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(r); free(zz); free(d); free(q);
  mg_free(lv, L);
  return result;
}

/* Sec. 3.2.3, the paper's GPU solver: red-black Gauss-Seidel sweeps on A x = b
 * from x = 0 (red half-sweep, then black), the residual ||b - A x|| checked
 * after every ORACLE_RBGS_CHECK sweep pairs against tol ||b||; at most max_pairs
 * sweep pairs.  Returns the sweep pairs taken, or -1 at the cap. */
int oracle_rbgs(const oracle_params* P, const uint8_t* type, const double* b, double tol,
                int max_pairs, double* x, double* rel_res) {
  const int64_t nc = oracle_n_cells(P);
  mg_level lv[ORACLE_MG_MAX_LEVELS];
  const int L = mg_build(P, type, lv);
  mg_level* v = &lv[0];
  double* ax = (double*)malloc(sizeof(double) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) {
    v->b[c] = type[c] ? b[c] : 0.0;
    v->x[c] = 0.0;
  }
  const double bnorm = sqrt(dot_fluid(nc, type, v->b, v->b));
  double rnorm = bnorm;
  int pairs = 0, result = 0;
  if (bnorm > 0.0) {
    result = -1;
    while (pairs < max_pairs || pairs == 0) {
      for (int s = 0; s < ORACLE_RBGS_CHECK; ++s) {
        lv_half_sweep(v, 0);
        lv_half_sweep(v, 1);
      }
      pairs += ORACLE_RBGS_CHECK;
      oracle_apply_A(P, type, v->x, ax);
      double rr = 0.0;
      for (int64_t c = 0; c < nc; ++c)
        if (type[c]) rr += (v->b[c] - ax[c]) * (v->b[c] - ax[c]);
      rnorm = sqrt(rr);
      if (rnorm <= tol * bnorm) { result = pairs; break; }
    }
  }
  for (int64_t c = 0; c < nc; ++c) x[c] = type[c] ? v->x[c] : 0.0;
  if (rel_res) *rel_res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(ax);
  mg_free(lv, L);
  return result;
}

/* Sec. 4, Fig. 10: kinetic plus potential energy, summed particle by particle. */
void oracle_energy(int64_t np, const double* x, const double* y, const double* z,
                   const double* u, const double* v, const double* w, const double g[3],
                   double m, double out[3]) {
  double ke = 0.0, pe = 0.0;
  for (int64_t p = 0; p < np; ++p) {
    ke += 0.5 * m * (u[p] * u[p] + v[p] * v[p] + w[p] * w[p]);
    pe -= m * (g[0] * x[p] + g[1] * y[p] + g[2] * z[p]);
  }
  out[0] = ke;
  out[1] = pe;
  out[2] = ke + pe;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output number `counter` of
 * the stream that starts at seed * G. */
static uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  uint64_t z = seed * G + (counter + 1u) * G;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* coordinate of a new particle on axis ax of cell index i (see oracle_step_ex) */
static double spawn_coordinate(const oracle_params* P, int ax, int64_t i, double U) {
  float xf = (float)(((double)i + U) * P->dx);
  int64_t cell[3];
  for (;;) {
    const double q[3] = {ax == 0 ? xf : 0.0, ax == 1 ? xf : 0.0, ax == 2 ? xf : 0.0};
    oracle_cell_of(P, q[0], q[1], q[2], cell);
    if (cell[ax] > i) xf = nextafterf(xf, 0.0f);
    else if (cell[ax] < i) xf = nextafterf(xf, 3.0e38f);
    else break;
  }
  const float lo = (float)P->skin, hi = (float)((double)P->n[ax] * P->dx - P->skin);
  xf = fminf(fmaxf(xf, lo), hi);
  return (double)xf;
}

int oracle_step_ex(const oracle_params* P, int64_t* np_io, int64_t capacity, double* x, double* y,
                   double* z, double* u, double* v, double* w, oracle_fields* out,
                   oracle_stats* stats) {
  int64_t np = *np_io;
  const int64_t nc = oracle_n_cells(P);
  oracle_params Q = *P;
  Q.dt = oracle_cfl_dt(P, np, u, v, w);
  int64_t removed = 0, added = 0;
  double* arr[6] = {x, y, z, u, v, w};
  if (P->ppc_max > 0 && np > 0) {
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)np);
    char* keep = (char*)malloc((size_t)np);
    oracle_bin(P, np, x, y, z, start, order);
    for (int64_t c = 0; c < nc; ++c)
      for (int64_t t = start[c]; t < start[c + 1]; ++t) keep[order[t]] = (t - start[c]) < P->ppc_max;
    int64_t m = 0;
    for (int64_t q = 0; q < np; ++q)
      if (keep[q]) {
        for (int a = 0; a < 6; ++a) arr[a][m] = arr[a][q];
        ++m;
      }
    removed = np - m;
    np = m;
    free(start);
    free(order);
    free(keep);
  }
  /* the step, keeping u_new for the new particles' velocities */
  oracle_fields F;
  memset(&F, 0, sizeof(F));
  if (out) F = *out;
  double* un_own[3] = {NULL, NULL, NULL};
  for (int d = 0; d < 3; ++d)
    if (!F.u_new[d]) {
      un_own[d] = (double*)malloc(sizeof(double) * (size_t)oracle_n_faces(P, d));
      F.u_new[d] = un_own[d];
    }
  oracle_stats S;
  memset(&S, 0, sizeof(S));
  int status = step_with_dt(&Q, np, x, y, z, u, v, w, &F, &S);
  if (status == 0 && P->ppc_min > 0) {
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    oracle_bin(P, np, x, y, z, start, order);
    const double* un[3] = {F.u_new[0], F.u_new[1], F.u_new[2]};
    for (int64_t c = 0; c < nc && status == 0; ++c) {
      const int64_t cnt = start[c + 1] - start[c];
      if (cnt == 0 || cnt >= P->ppc_min) continue;
      const int64_t ijk[3] = {c % P->n[0], (c / P->n[0]) % P->n[1], c / ((int64_t)P->n[0] * P->n[1])};
      for (int64_t s = 0; s < P->ppc_min - cnt; ++s) {
        if (np >= capacity) {
          status = 4;
          break;
        }
        const uint64_t ctr =
            (((uint64_t)P->reseed_step * (uint64_t)nc + (uint64_t)c) * 64u + (uint64_t)(cnt + s)) * 3u;
        double pos[3];
        for (int a = 0; a < 3; ++a) {
          const double U = (double)(splitmix64(P->reseed_seed, ctr + (uint64_t)a) >> 11) * 0x1.0p-53;
          pos[a] = spawn_coordinate(P, a, ijk[a], U);
        }
        x[np] = pos[0];
        y[np] = pos[1];
        z[np] = pos[2];
        u[np] = oracle_interp(P, 0, un[0], pos[0], pos[1], pos[2]);
        v[np] = oracle_interp(P, 1, un[1], pos[0], pos[1], pos[2]);
        w[np] = oracle_interp(P, 2, un[2], pos[0], pos[1], pos[2]);
        ++np;
        ++added;
      }
    }
    free(start);
    free(order);
  }
  for (int d = 0; d < 3; ++d) free(un_own[d]);
  S.dt = Q.dt;
  S.added = added;
  S.removed = removed;
  if (stats) *stats = S;
  *np_io = np;
  return status;
}
