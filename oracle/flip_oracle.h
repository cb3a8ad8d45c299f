/*
 * flip_oracle.h — plain FP64 CPU oracle of one FLIP time step.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct
 * statement of what the FLIP step of Centeno & Pereira, "Fluid Implicit
 * Particle Simulation for CPU and GPU" (arXiv 2404.01931) computes.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Conventions (MAC grid, Section 3.1.1, Figs. 1-2):
 *   - nx, ny, nz cells of edge dx; domain [0, n_a*dx) per axis; y is up.
 *   - Cell (i,j,k) has linear index i + nx*(j + ny*k) (x fastest).
 *   - Component d of the velocity lives on the faces normal to axis d:
 *       u[i,j,k] at (i*dx, (j+1/2)dx, (k+1/2)dx), i in [0,nx], index i + (nx+1)*(j + ny*k)
 *       v[i,j,k] at ((i+1/2)dx, j*dx, (k+1/2)dx), j in [0,ny], index i + nx*(j + (ny+1)*k)
 *       w[i,j,k] at ((i+1/2)dx, (j+1/2)dx, k*dx), k in [0,nz], index i + nx*(j + ny*k)
 *   - The six domain planes are solid walls; every other boundary of the fluid
 *     is a free surface (pressure 0 in air cells).
 *   - Cell types: 1 = fluid (holds at least one particle), 0 = air.
 *
 * Readings of points the paper leaves open are stated beside each function.
 */
#ifndef FLIP_ORACLE_H
#define FLIP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n[3];        /* cells per axis */
  double dx;           /* cell edge (the paper's Delta tau) */
  double dt;           /* time step */
  double gravity[3];   /* body acceleration, e.g. (0, -9.81, 0) */
  double rho;          /* fluid density */
  double flip_ratio;   /* FLIP share of the PIC/FLIP blend, in [0,1] */
  double skin;         /* clamp distance from the walls */
  double cg_tol;       /* PCG stop: ||r||_2 <= cg_tol * ||b||_2 */
  int32_t cg_max_iter; /* PCG iteration cap */
  int32_t advect_source; /* 0: advect with the blended particle velocity; 1: with the grid velocity */
  int32_t preconditioner; /* 0: Jacobi (oracle_pcg); 1: multigrid V-cycle (oracle_pcg_mg);
                             2: red-black Gauss-Seidel as the solver (oracle_rbgs) */
  int32_t mg_nu;          /* multigrid: red-black sweep pairs before and after the correction */
  double mg_omega;        /* multigrid: over-correction of the coarse correction */
  double cfl;             /* Sec. 3.1.4 CFL number; 0: fixed dt */
  int32_t ppc_min;        /* Sec. 3.1.2 reseeding: refill cells below this (0: off) */
  int32_t ppc_max;        /* cells above this lose the excess at the step start (0: off) */
  uint64_t reseed_seed;   /* SplitMix64 seed of the new particles' positions */
  int64_t reseed_step;    /* the step's index (part of the generator's counter) */
} oracle_params;

typedef struct {
  int32_t cg_iterations;   /* A-applications the PCG took; -1 when it hit the cap */
  double cg_rel_residual;  /* recursive ||r||/||b|| at exit */
  double rel_divergence;   /* ||div u_new||_2 / ||div u*||_2 over fluid cells */
  int64_t n_fluid;         /* fluid cells this step */
  double dt;               /* time step taken */
  int64_t added, removed;  /* reseeding: particles created / dropped */
} oracle_stats;

/* Optional outputs of oracle_step; any pointer may be NULL. */
typedef struct {
  double* u_old[3];  /* P2G result, before forces (the FLIP "old" grid velocity) */
  double* u_star[3]; /* after gravity and wall conditions (projection input) */
  double* u_new[3];  /* projected velocity */
  double* pressure;  /* n_cells, 0 in air */
  double* rhs;       /* n_cells, b = -div u* in fluid cells, 0 elsewhere */
  uint8_t* type;     /* n_cells */
} oracle_fields;

int64_t oracle_n_cells(const oracle_params* P);
int64_t oracle_n_faces(const oracle_params* P, int comp);

/* Eq. 4b: the 1-D hat function. */
double oracle_hat(double r);

/* Cell holding a point: floor(x * (1/dx)) per axis, clamped to the grid. */
void oracle_cell_of(const oracle_params* P, double x, double y, double z, int64_t cell[3]);

/* Eq. 4a on the clamped sample coordinate: weight of a particle at (x,y,z) on
 * face node (a,b,c) of component comp. */
double oracle_weight(const oracle_params* P, int comp, int64_t a, int64_t b, int64_t c,
                     double x, double y, double z);

/* Section 3.1.5: stable counting sort of particles by cell.  start has
 * n_cells+1 entries (start[c]..start[c+1] are the particles of cell c, in
 * order[]).  */
void oracle_bin(const oracle_params* P, int64_t np, const double* x, const double* y,
                const double* z, int64_t* start, int64_t* order);

/* Section 3.1.6: gather-form P2G of one component. */
void oracle_p2g(const oracle_params* P, int comp, const double* x, const double* y,
                const double* z, const double* vel, const int64_t* start,
                const int64_t* order, double* grid, double* wsum);

void oracle_cell_types(const oracle_params* P, const int64_t* start, uint8_t* type);

/* Forces (gravity) then solid-wall conditions, one component. */
void oracle_forces_walls(const oracle_params* P, int comp, const double* u_old, double* u_star);

/* Eq. 6: b = -div u* in fluid cells (0 elsewhere). */
void oracle_divergence(const oracle_params* P, const double* const u[3], const uint8_t* type,
                       double* b);

/* Matrix-free 7-point Laplacian of Section 3.1.7 (rows of fluid cells only). */
void oracle_apply_A(const oracle_params* P, const uint8_t* type, const double* p, double* Ap);

/* Jacobi-preconditioned CG on A p = b, p0 = 0.  Returns iterations, or -1 at the cap. */
int oracle_pcg(const oracle_params* P, const uint8_t* type, const double* b, double tol,
               int max_iter, double* p, double* rel_res);

/* Multigrid V-cycle preconditioner for the PCG of Sec. 3.1.7, with the
 * red-black Gauss-Seidel of Sec. 3.2.3 as its smoother.  Levels: level 0 is the
 * cell grid; level l+1 has ceil(n_l/2) cells per axis, a coarse cell is fluid
 * when any of its (up to 8) children is, and coarsening stops once the largest
 * extent is <= 4 (at most ORACLE_MG_MAX_LEVELS levels).  Level l carries the
 * 7-point operator with scale dt/(rho (2^l dx)^2).  A V-cycle from a zero guess:
 * nu (red, black) half-sweep pairs, residual, restriction b_{l+1} = (1/16) sum of
 * the fluid children's residuals (Galerkin scaling for piecewise-constant
 * prolongation), coarse V-cycle, correction x += omega * x_{l+1}(parent)
 * on fluid cells, nu (black, red) pairs.  The coarsest level does
 * ORACLE_MG_COARSE_SWEEPS (red, black) pairs then as many (black, red) pairs.
 * The operator is symmetric positive definite for any omega > 0 (symmetrised
 * smoother plus a positively scaled SPD coarse term); omega = 1 is the
 * Galerkin-consistent cycle, omega > 1 over-corrects, which piecewise-constant
 * prolongation needs to converge fast. */
#define ORACLE_MG_MAX_LEVELS 12
#define ORACLE_MG_COARSE_SWEEPS 2
int oracle_mg_levels(const oracle_params* P, int32_t dims[][3]);
void oracle_mg_vcycle(const oracle_params* P, const uint8_t* type, const double* r, double* z,
                      int nu, double omega);
/* PCG with the V-cycle preconditioner; same stopping rule as oracle_pcg. */
int oracle_pcg_mg(const oracle_params* P, const uint8_t* type, const double* b, double tol,
                  int max_iter, int nu, double omega, double* x, double* rel_res);

/* The paper's GPU solver (Sec. 3.2.3): red-black Gauss-Seidel sweeps from x = 0,
 * ||b - A x|| <= tol ||b|| checked every ORACLE_RBGS_CHECK sweep pairs, at most
 * max_pairs pairs (oracle_params.preconditioner == 2 in oracle_step).  Returns the
 * pairs taken, or -1 at the cap. */
#define ORACLE_RBGS_CHECK 8
int oracle_rbgs(const oracle_params* P, const uint8_t* type, const double* b, double tol,
                int max_pairs, double* x, double* rel_res);

/* Eq. 5: pressure update of one component. */
void oracle_project(const oracle_params* P, int comp, const double* u_star, const double* p,
                    const uint8_t* type, double* u_new);

/* Trilinear interpolation of one face field at a point (Section 3.1.8). */
double oracle_interp(const oracle_params* P, int comp, const double* field, double x, double y,
                     double z);

/* Section 3.1.8 + 3.1.3: PIC/FLIP blend, forward Euler, wall clamp. */
void oracle_g2p(const oracle_params* P, int64_t np, double* x, double* y, double* z, double* u,
                double* v, double* w, const double* const u_old[3],
                const double* const u_new[3]);

/* ||div u||_2 over fluid cells (FP64). */
double oracle_div_norm(const oracle_params* P, const double* const u[3], const uint8_t* type);

/* One full step, in place on the particle arrays (kept in their given order).
 * Returns 0, or 1 when the PCG hit its cap, or 2 when a fluid region touches no
 * air (A singular), or 3 on allocation failure. */
int oracle_step(const oracle_params* P, int64_t np, double* x, double* y, double* z, double* u,
                double* v, double* w, oracle_fields* out, oracle_stats* stats);

/* Total mechanical energy of a particle set (Sec. 4, Fig. 10), each particle of
 * mass m: out[0] = m/2 sum |v|^2, out[1] = -m sum g . x (zero at the origin),
 * out[2] = out[0] + out[1].  Plain sequential FP64 sums. */
void oracle_energy(int64_t np, const double* x, const double* y, const double* z,
                   const double* u, const double* v, const double* w, const double g[3],
                   double m, double out[3]);

/* Surface reconstruction (Sec. 3.3), surface_oracle.c.  Sampling corners
 * (i,j,k) in [0,n[0]] x [0,n[1]] x [0,n[2]] at origin + h*(i,j,k), x fastest. */
double oracle_blobby_kernel(double s);
void oracle_sdf(int64_t np, const double* x, const double* y, const double* z,
                const int32_t n[3], const double origin[3], double h, double r, double R,
                double* phi);
/* Vertex count (returned) and triangle count of the marching-cubes mesh. */
int64_t oracle_mc_count(const int32_t n[3], const double* phi, double iso, int64_t* n_triangles);
/* The mesh: vert[3 nv], vedge[nv] (3 * corner + axis), tri[3 nt], nrm[3 nv]. */
void oracle_mc(const int32_t n[3], const double origin[3], double h, const double* phi,
               double iso, double* vert, int64_t* vedge, int32_t* tri, double* nrm);

/* Sec. 3.1.4: the step's dt for a CFL number P->cfl (P->dt when cfl is 0). */
double oracle_cfl_dt(const oracle_params* P, int64_t np, const double* u, const double* v,
                     const double* w);

/* One step with reseeding (Sec. 3.1.2).  The arrays hold `capacity` entries
 * and *np particles, updated in place:
 *   1. (ppc_max > 0) a cell holding more than ppc_max particles at the step
 *      start keeps the ppc_max of lowest index (the CFL dt is taken before this);
 *   2. the step of oracle_step;
 *   3. (ppc_min > 0) each cell holding 1..ppc_min-1 particles after the
 *      advection gets ppc_min - c new ones, cells in x-fastest order, appended:
 *      slot q = c + s, counter ((reseed_step * n_cells + cell) * 64 + q) * 3 +
 *      axis into SplitMix64(reseed_seed), U = top 53 bits * 2^-53, coordinate
 *      (i + U) dx rounded to float, moved by one float at a time back into the
 *      cell, clamped to [skin, n dx - skin] in float; velocity = the projected
 *      grid velocity interpolated there (oracle_interp of u_new).
 * Returns oracle_step's codes, or 4 when capacity stopped the reseeding. */
int oracle_step_ex(const oracle_params* P, int64_t* np, int64_t capacity, double* x, double* y,
                   double* z, double* u, double* v, double* w, oracle_fields* out,
                   oracle_stats* stats);

int oracle_num_threads(void);
/* Threads of the calling thread's later parallel regions (n > 0; timing only). */
void oracle_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
