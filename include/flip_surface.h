/*
 * flip_surface.h — surface reconstruction of a FLIP fluid on the GPU (sm_103a).
 *
 * Section 3.3 of Centeno & Pereira, "Fluid Implicit Particle Simulation for CPU
 * and GPU" (arXiv 2404.01931): a scalar field from the particles (Sec. 3.3.1,
 * the "improved blobbies" signed distance), then a triangle mesh of one of its
 * level sets by marching cubes with per-vertex normals (Sec. 3.3.2).
 *
 * Sampling grid: (n[0]+1) x (n[1]+1) x (n[2]+1) corners at origin + h*(i,j,k),
 * x fastest (corner index i + (n[0]+1)*(j + (n[1]+1)*k)); its resolution is
 * independent of the simulation grid (Sec. 3.3.2).
 *
 * Scalar field (Sec. 3.3.1), for a corner x and the particles x_i with
 * |x - x_i| < R (R = search_radius), all of radius r:
 *   k(s)  = max(0, (1 - s^2)^3)
 *   w_i   = k(|x - x_i| / R) / sum_j k(|x - x_j| / R)
 *   phi   = |x - sum_i w_i x_i| - sum_i w_i r  =  |x - xbar| - r
 * A corner with no particle closer than R gets phi = R - r, the limit of a
 * lone particle leaving its support (so such corners are outside for r < R).
 *
 * Marching cubes (Sec. 3.3.2): a corner is inside when phi < iso.  Each cube
 * with inside and outside corners gets polygons through the crossing edges:
 * on every cube face the crossings are joined in pairs (on a face with two
 * diagonal inside corners, each inside corner is cut off by its own segment,
 * so the two cubes sharing a face always agree and the mesh is closed), the
 * segments of the six faces are chained into loops, each loop is wound so its
 * normal points from the inside corners to the outside ones and is fanned into
 * triangles from its lowest-numbered edge among those lying on no cube face
 * that the loop crosses twice (else its lowest-numbered edge), so no triangle
 * lies inside a cube face and the mesh is a closed, consistently wound surface
 * wherever the sampling box's boundary corners are outside.  The case table is generated from
 * the cube's topology when the library loads.  A vertex sits on each crossing
 * grid edge at the linear interpolation t = (iso - phi_a) / (phi_b - phi_a),
 * and vertices are shared by all triangles on that edge.
 *
 * Vertex normals (Sec. 3.3.2): the unit normals of the triangles sharing the
 * vertex, each weighted by the inverse of the triangle's area, summed and
 * normalised (a zero vector when every such triangle is degenerate).
 *
 * Output order is deterministic: vertices by grid edge id (3 * corner + axis),
 * triangles by cube (the index of its lowest corner) and then table order.
 *
 * Ownership: a surface object owns its device memory; reads copy into
 * caller-owned memory.  Errors follow include/flip.h (status codes,
 * flip_last_error()).
 */
#ifndef FLIP_SURFACE_GB300_H
#define FLIP_SURFACE_GB300_H

#include <stddef.h>
#include <stdint.h>

#include "flip.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flip_surface flip_surface;

typedef struct {
  int32_t n[3];          /* sampling cells per axis, each in [1, 1024] */
  double origin[3];      /* position of corner (0,0,0) */
  double h;              /* corner spacing (> 0) */
  double radius;         /* particle radius r (>= 0, < search_radius) */
  double search_radius;  /* kernel support R (> 0); the particle bins (edge R/2 over the
                            sampling box widened by R per side) must number under 2^31,
                            else flip_surface_create returns FLIP_E_ARG */
  double iso;            /* level set meshed (0: the surface phi = 0) */
} flip_surface_params;

typedef enum {
  FLIP_SURF_FIELD = 0,     /* float32[corners]: phi */
  FLIP_SURF_VERTICES = 1,  /* float32[n_vertices][3] */
  FLIP_SURF_NORMALS = 2,   /* float32[n_vertices][3], unit length or zero */
  FLIP_SURF_TRIANGLES = 3, /* int32[n_triangles][3] vertex indices */
  FLIP_SURF_VERTEX_EDGE = 4 /* int64[n_vertices]: grid edge id 3 * corner + axis */
} flip_surface_field;

/* Sampling grid equal to the simulation grid of p (corners on the cell
 * corners), r = dx / 2, R = 2 dx, iso = 0. */
void flip_surface_default_params(const flip_params* p, flip_surface_params* out);

/* Validates sp and allocates the field; stream (cudaStream_t, nullable: a new
 * non-blocking stream) orders the surface's work.  FLIP_E_ARG on bad
 * parameters, FLIP_E_OOM / FLIP_E_CUDA on allocation failure. */
int flip_surface_create(const flip_surface_params* sp, void* stream, flip_surface** out);

/* phi at every corner from the current particles of a simulation handle (after
 * the handle's queued work; the handle is not modified).  Asynchronous. */
int flip_surface_sdf(flip_surface* s, flip_handle* h);

/* phi at every corner from the caller: float32[corners], host or device.
 * Synchronous with respect to the source. */
int flip_surface_set_field(flip_surface* s, const float* phi, int32_t src_is_device);

/* Marching cubes over the current phi plus vertex normals.  Grows the output
 * buffers as needed and returns their sizes.  Synchronous.  FLIP_E_SIZE when
 * the mesh has 2^29 or more vertices (its triangles, at most 4 per vertex, must
 * stay below 2^31 for int32 indices). */
int flip_surface_mesh(flip_surface* s, int64_t* n_vertices, int64_t* n_triangles);

/* Bytes of a field at the current sizes (0 for an unknown field). */
size_t flip_surface_bytes(const flip_surface* s, flip_surface_field which);

/* Copies a field into caller memory; bytes must equal flip_surface_bytes
 * (FLIP_E_SIZE otherwise).  Synchronous. */
int flip_surface_read(flip_surface* s, flip_surface_field which, void* dst, size_t bytes,
                      int32_t dst_is_device);

void flip_surface_destroy(flip_surface* s);

/* The marching-cubes case table the library generates (host memory, no GPU
 * needed): for corner pattern c (bit q set when local corner q, at offset
 * (q & 1, (q >> 1) & 1, q >> 2), is inside), ntri[c] triangles given as local
 * edge numbers tri[(c * FLIP_SURF_MAX_TRI + t) * 3 + v]; the edge along axis a
 * whose lower corner has bits (b_lo, b_hi) on the other two axes (ascending)
 * is 4a + b_lo + 2 b_hi.  Returns FLIP_OK, or FLIP_E_CUDA if generation failed. */
#define FLIP_SURF_MAX_TRI 12
int flip_surface_case_table(uint8_t ntri[256], uint8_t* tri);

#ifdef __cplusplus
}
#endif
#endif /* FLIP_SURFACE_GB300_H */
