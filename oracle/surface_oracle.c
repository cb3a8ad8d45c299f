/*
 * surface_oracle.c — plain FP64 CPU oracle of the surface reconstruction of
 * Sec. 3.3 (scalar field, marching cubes, vertex normals).
 *
 * TEST INFRASTRUCTURE ONLY (see flip_oracle.h).  It shares no code or table
 * with the CUDA library: every cube is polygonised here from its corner signs
 * directly, with no case table.
 *
 * Sampling grid: corners (i,j,k), 0 <= i <= n[0] etc., at origin + h*(i,j,k),
 * index i + (n[0]+1)*(j + (n[1]+1)*k).
 *
 * Readings (the paper states the formulas, not these details):
 *   - phi at a corner with no particle closer than R is R - r.
 *   - A corner is inside when phi < iso.
 *   - On a cube face whose inside corners are diagonal, each inside corner is
 *     cut off by its own segment.
 *   - A polygon is wound so that the Newell normal of its edge midpoints points
 *     along the sum over its edges of (outside end - inside end), and is fanned
 *     from its edge of lowest local number among the edges on no cube face that
 *     holds four of the polygon's edges (else from its lowest edge), so that no
 *     triangle lies inside a cube face.  Local numbers: the edge along axis
 *     a whose lower corner has bits (b_lo, b_hi) on the other two axes (in
 *     ascending axis order) is 4a + b_lo + 2 b_hi; local corner q sits at
 *     (q & 1, (q >> 1) & 1, q >> 2).  Polygons of a cube are listed in the order
 *     of their lowest local edge number.
 *   - A triangle of zero area adds nothing to its vertices' normals; a vertex
 *     whose triangles all have zero area gets a zero normal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "flip_oracle.h"

/* ------------------------------------------------------------ scalar field */

/* Sec. 3.3.1: k(s) = max(0, (1 - s^2)^3). */
double oracle_blobby_kernel(double s) {
  const double t = 1.0 - s * s;
  return t > 0.0 ? t * t * t : 0.0;
}

/* Sec. 3.3.1: phi(x) = |x - sum_i w_i x_i| - sum_i w_i r_i with
 * w_i = k(|x - x_i| / R) / sum_j k(|x - x_j| / R), all r_i = r.  Particles are
 * found through a grid of bins of edge R (counting sort): every particle closer
 * than R to a corner lies in the 3x3x3 bins around the corner's bin. */
void oracle_sdf(int64_t np, const double* x, const double* y, const double* z,
                const int32_t n[3], const double origin[3], double h, double r, double R,
                double* phi) {
  int64_t nb[3], nbins = 1;
  double bo[3];
  for (int a = 0; a < 3; ++a) {
    bo[a] = origin[a] - R;
    nb[a] = (int64_t)ceil((n[a] * h + 2.0 * R) / R) + 1;
    nbins *= nb[a];
  }
  int64_t* start = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
  int64_t* bin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  for (int64_t p = 0; p < np; ++p) {
    const double q[3] = {x[p], y[p], z[p]};
    int64_t b[3];
    int ok = 1;
    for (int a = 0; a < 3; ++a) {
      b[a] = (int64_t)floor((q[a] - bo[a]) / R);
      if (b[a] < 0 || b[a] >= nb[a]) ok = 0;
    }
    bin[p] = ok ? b[0] + nb[0] * (b[1] + nb[1] * b[2]) : -1;
    if (ok) start[bin[p] + 1]++;
  }
  for (int64_t b = 0; b < nbins; ++b) start[b + 1] += start[b];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbins);
    memcpy(fill, start, sizeof(int64_t) * (size_t)nbins);
    for (int64_t p = 0; p < np; ++p)
      if (bin[p] >= 0) order[fill[bin[p]]++] = p;
    free(fill);
  }
  const int64_t cx = n[0] + 1, cy = n[1] + 1, cz = n[2] + 1;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cx * cy * cz; ++c) {
    const int64_t idx[3] = {c % cx, (c / cx) % cy, c / (cx * cy)};
    double X[3], kb[3];
    for (int a = 0; a < 3; ++a) {
      X[a] = origin[a] + h * (double)idx[a];
      kb[a] = floor((X[a] - bo[a]) / R);
    }
    double sk = 0.0, sd[3] = {0.0, 0.0, 0.0};
    for (int64_t bz = (int64_t)kb[2] - 1; bz <= (int64_t)kb[2] + 1; ++bz)
      for (int64_t by = (int64_t)kb[1] - 1; by <= (int64_t)kb[1] + 1; ++by)
        for (int64_t bx = (int64_t)kb[0] - 1; bx <= (int64_t)kb[0] + 1; ++bx) {
          if (bx < 0 || by < 0 || bz < 0 || bx >= nb[0] || by >= nb[1] || bz >= nb[2]) continue;
          const int64_t b = bx + nb[0] * (by + nb[1] * bz);
          for (int64_t s = start[b]; s < start[b + 1]; ++s) {
            const int64_t p = order[s];
            const double d[3] = {x[p] - X[0], y[p] - X[1], z[p] - X[2]};
            const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (dist >= R) continue;
            const double k = oracle_blobby_kernel(dist / R);
            sk += k;
            for (int a = 0; a < 3; ++a) sd[a] += k * d[a];
          }
        }
    if (sk > 0.0) {
      /* x - xbar = -(sum_i k_i (x_i - x)) / sum_i k_i */
      phi[c] = sqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]) / sk - r;
    } else {
      phi[c] = R - r;
    }
  }
  free(start);
  free(bin);
  free(order);
}

/* ------------------------------------------------------------ marching cubes */

typedef struct {
  int32_t n[3];
  int64_t c[3];      /* corners per axis */
  const double* phi;
  double iso;
} mc_grid;

static int64_t corner_index(const mc_grid* G, int64_t i, int64_t j, int64_t k) {
  return i + G->c[0] * (j + G->c[1] * k);
}

static int inside(const mc_grid* G, int64_t c) { return G->phi[c] < G->iso; }

/* the two axes other than a, ascending */
static void other_axes(int a, int* lo, int* hi) {
  *lo = (a == 0) ? 1 : 0;
  *hi = (a == 2) ? 1 : 2;
}

/* local edge number of the edge from local corner q along axis a */
static int local_edge(int q, int a) {
  int lo, hi;
  other_axes(a, &lo, &hi);
  return 4 * a + ((q >> lo) & 1) + 2 * ((q >> hi) & 1);
}

/* does the grid edge (corner c, axis a) cross the level set? */
static int edge_crosses(const mc_grid* G, int64_t i, int64_t j, int64_t k, int a) {
  const int64_t ijk[3] = {i, j, k};
  if (ijk[a] >= G->n[a]) return 0;
  const int64_t c0 = corner_index(G, i, j, k);
  const int64_t c1 = corner_index(G, i + (a == 0), j + (a == 1), k + (a == 2));
  return inside(G, c0) != inside(G, c1);
}

/* Polygons of the cube whose lowest corner is (i,j,k), as lists of local edge
 * numbers, wound and rotated as stated in the file header.  Returns the number
 * of polygons; len[p] is the length of polygon p. */
static int cube_polygons(const mc_grid* G, int64_t i, int64_t j, int64_t k, int poly[6][12],
                         int len[6]) {
  int in[8];
  for (int q = 0; q < 8; ++q)
    in[q] = inside(G, corner_index(G, i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2)));
  /* neighbours of each crossing edge through the faces of the cube */
  int nbr[12][2], deg[12];
  for (int e = 0; e < 12; ++e) deg[e] = 0;
  for (int a = 0; a < 3; ++a)
    for (int side = 0; side < 2; ++side) {
      int u, v;
      other_axes(a, &u, &v);
      /* the face's corners in cyclic order: (0,0), (1,0), (1,1), (0,1) in (u, v) */
      const int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
      int corner[4], edge[4], cross[4];
      for (int t = 0; t < 4; ++t) corner[t] = (side << a) | (cu[t] << u) | (cv[t] << v);
      int ncross = 0;
      for (int t = 0; t < 4; ++t) {
        const int p = corner[t], q = corner[(t + 1) % 4];
        const int along = (p ^ q) == (1 << u) ? u : v;
        edge[t] = local_edge(p < q ? p : q, along);
        cross[t] = in[p] != in[q];
        ncross += cross[t];
      }
      int pairs[2][2], npairs = 0;
      if (ncross == 2) {
        int first = -1;
        for (int t = 0; t < 4; ++t)
          if (cross[t]) {
            if (first < 0) first = t;
            else {
              pairs[0][0] = edge[first];
              pairs[0][1] = edge[t];
              npairs = 1;
            }
          }
      } else if (ncross == 4) {
        for (int t = 0; t < 4; ++t)
          if (in[corner[t]]) {
            /* the two face edges meeting at this inside corner */
            pairs[npairs][0] = edge[(t + 3) % 4];
            pairs[npairs][1] = edge[t];
            npairs++;
          }
      }
      for (int s = 0; s < npairs; ++s) {
        const int e0 = pairs[s][0], e1 = pairs[s][1];
        nbr[e0][deg[e0]++] = e1;
        nbr[e1][deg[e1]++] = e0;
      }
    }
  int seen[12] = {0}, npoly = 0;
  for (int e = 0; e < 12; ++e) {
    if (deg[e] != 2 || seen[e]) continue;
    int *P = poly[npoly], L = 0, prev = -1, cur = e;
    while (1) {
      P[L++] = cur;
      seen[cur] = 1;
      const int next = (nbr[cur][0] == prev) ? nbr[cur][1] : nbr[cur][0];
      prev = cur;
      cur = next;
      if (cur == e) break;
    }
    /* winding */
    double mid[12][3], dir[3] = {0, 0, 0}, N[3] = {0, 0, 0};
    for (int t = 0; t < L; ++t) {
      const int a = P[t] / 4;
      int lo, hi;
      other_axes(a, &lo, &hi);
      int q0 = ((P[t] & 1) << lo) | (((P[t] >> 1) & 1) << hi);
      int q1 = q0 | (1 << a);
      for (int d = 0; d < 3; ++d) {
        const double p0 = (q0 >> d) & 1, p1 = (q1 >> d) & 1;
        mid[t][d] = 0.5 * (p0 + p1);
        dir[d] += in[q0] ? p1 - p0 : p0 - p1;
      }
    }
    for (int t = 0; t < L; ++t) {
      const double* A = mid[t];
      const double* B = mid[(t + 1) % L];
      N[0] += (A[1] - B[1]) * (A[2] + B[2]);
      N[1] += (A[2] - B[2]) * (A[0] + B[0]);
      N[2] += (A[0] - B[0]) * (A[1] + B[1]);
    }
    if (N[0] * dir[0] + N[1] * dir[1] + N[2] * dir[2] < 0.0)
      for (int t = 0; t < L / 2; ++t) {
        const int tmp = P[t];
        P[t] = P[L - 1 - t];
        P[L - 1 - t] = tmp;
      }
    /* start at the lowest edge number among the edges that lie on no cube face
       holding four edges of this polygon (else at the lowest edge number) */
    int face_count[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int t = 0; t < L; ++t) {
      const int a = P[t] / 4;
      int lo, hi;
      other_axes(a, &lo, &hi);
      face_count[lo][P[t] & 1]++;
      face_count[hi][(P[t] >> 1) & 1]++;
    }
    int m = -1;
    for (int t = 0; t < L; ++t) {
      const int a = P[t] / 4;
      int lo, hi;
      other_axes(a, &lo, &hi);
      const int free_edge = face_count[lo][P[t] & 1] < 4 && face_count[hi][(P[t] >> 1) & 1] < 4;
      if (free_edge && (m < 0 || P[t] < P[m])) m = t;
    }
    if (m < 0) {
      m = 0;
      for (int t = 1; t < L; ++t)
        if (P[t] < P[m]) m = t;
    }
    int R[12];
    for (int t = 0; t < L; ++t) R[t] = P[(m + t) % L];
    memcpy(P, R, sizeof(int) * (size_t)L);
    len[npoly++] = L;
  }
  return npoly;
}

int64_t oracle_mc_count(const int32_t n[3], const double* phi, double iso, int64_t* n_triangles) {
  mc_grid G = {{n[0], n[1], n[2]}, {n[0] + 1, n[1] + 1, n[2] + 1}, phi, iso};
  int64_t nv = 0, nt = 0;
  for (int64_t k = 0; k < G.c[2]; ++k)
    for (int64_t j = 0; j < G.c[1]; ++j)
      for (int64_t i = 0; i < G.c[0]; ++i) {
        for (int a = 0; a < 3; ++a) nv += edge_crosses(&G, i, j, k, a);
        if (i < n[0] && j < n[1] && k < n[2]) {
          int poly[6][12], len[6];
          const int np = cube_polygons(&G, i, j, k, poly, len);
          for (int p = 0; p < np; ++p) nt += len[p] - 2;
        }
      }
  if (n_triangles) *n_triangles = nt;
  return nv;
}

/* Sec. 3.3.2.  Vertices: one per crossing grid edge, in edge-id order (edge id
 * 3 * corner + axis), at t = (iso - phi_a) / (phi_b - phi_a) from the lower
 * corner.  Triangles: per cube in corner order, each polygon fanned.  Normals:
 * sum over a vertex's triangles of (unit normal) / (area), normalised. */
void oracle_mc(const int32_t n[3], const double origin[3], double h, const double* phi,
               double iso, double* vert, int64_t* vedge, int32_t* tri, double* nrm) {
  mc_grid G = {{n[0], n[1], n[2]}, {n[0] + 1, n[1] + 1, n[2] + 1}, phi, iso};
  const int64_t ncorner = G.c[0] * G.c[1] * G.c[2];
  /* vertex index of each crossing edge (-1 elsewhere) */
  int64_t* vid = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncorner * 3);
  int64_t nv = 0;
  for (int64_t k = 0; k < G.c[2]; ++k)
    for (int64_t j = 0; j < G.c[1]; ++j)
      for (int64_t i = 0; i < G.c[0]; ++i) {
        const int64_t c = corner_index(&G, i, j, k);
        for (int a = 0; a < 3; ++a) {
          vid[3 * c + a] = -1;
          if (!edge_crosses(&G, i, j, k, a)) continue;
          const int64_t c1 = corner_index(&G, i + (a == 0), j + (a == 1), k + (a == 2));
          const double t = (iso - phi[c]) / (phi[c1] - phi[c]);
          const double ijk[3] = {(double)i, (double)j, (double)k};
          for (int d = 0; d < 3; ++d)
            vert[3 * nv + d] = origin[d] + h * (ijk[d] + (d == a ? t : 0.0));
          vedge[nv] = 3 * c + a;
          vid[3 * c + a] = nv++;
        }
      }
  int64_t nt = 0;
  for (int64_t k = 0; k < n[2]; ++k)
    for (int64_t j = 0; j < n[1]; ++j)
      for (int64_t i = 0; i < n[0]; ++i) {
        int poly[6][12], len[6];
        const int np = cube_polygons(&G, i, j, k, poly, len);
        for (int p = 0; p < np; ++p) {
          int64_t V[12];
          for (int t = 0; t < len[p]; ++t) {
            const int e = poly[p][t], a = e / 4;
            int lo, hi;
            other_axes(a, &lo, &hi);
            int64_t off[3] = {0, 0, 0};
            off[lo] = e & 1;
            off[hi] = (e >> 1) & 1;
            V[t] = vid[3 * corner_index(&G, i + off[0], j + off[1], k + off[2]) + a];
          }
          for (int t = 1; t + 1 < len[p]; ++t) {
            tri[3 * nt] = (int32_t)V[0];
            tri[3 * nt + 1] = (int32_t)V[t];
            tri[3 * nt + 2] = (int32_t)V[t + 1];
            ++nt;
          }
        }
      }
  for (int64_t v = 0; v < 3 * nv; ++v) nrm[v] = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    const double* A = vert + 3 * (int64_t)tri[3 * t];
    const double* B = vert + 3 * (int64_t)tri[3 * t + 1];
    const double* Cc = vert + 3 * (int64_t)tri[3 * t + 2];
    const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double e2[3] = {Cc[0] - A[0], Cc[1] - A[1], Cc[2] - A[2]};
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                          e1[0] * e2[1] - e1[1] * e2[0]};
    const double len2 = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
    if (len2 <= 0.0) continue;
    /* unit normal cr/|cr| over area |cr|/2 */
    const double area = 0.5 * sqrt(len2);
    for (int q = 0; q < 3; ++q)
      for (int d = 0; d < 3; ++d) nrm[3 * (int64_t)tri[3 * t + q] + d] += cr[d] / sqrt(len2) / area;
  }
  for (int64_t v = 0; v < nv; ++v) {
    double* N = nrm + 3 * v;
    const double l = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    if (l > 0.0)
      for (int d = 0; d < 3; ++d) N[d] /= l;
  }
  free(vid);
}
