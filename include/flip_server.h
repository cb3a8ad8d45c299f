/*
 * flip_server.h — continuous-batching step server over resident FLIP scenes
 * (part of libflip_gb300.so).  The paper steps one scene at a time; serving many
 * scenes is this library's deployment layer and has no counterpart in it.
 *
 * The server keeps scenes resident on the current device, admits them by their
 * device footprint (flip_footprint_bytes) within a byte budget, and runs step
 * requests on worker threads.  Each request asks for one FLIP step of one scene
 * and carries an arrival time.  Two batches can be in flight at once: while the
 * GPU runs one, the launcher forms the next from the requests that have arrived
 * for scenes not in flight, one per scene, up to max_batch scenes, oldest first,
 * and enqueues it behind the first (the batch stepping of flip_batch_step: the
 * scenes of a batch share one solve launch).  Requests that arrive while batches
 * run join later batches (continuous batching); the next batch's binning and P2G
 * overlap the previous batch's G2P on the device, and the solve launches of the
 * two batches run one after the other.  A completer thread finishes each request
 * as soon as its own scene's step is done on the device (an event on the scene's
 * stream), not when its whole batch is. 
 *
 * Times are seconds on the server's clock (steady clock, 0 at creation).
 * Functions return FLIP_* status codes (include/flip.h) and are safe to call
 * from any thread; a scene's handle may be read only while the scene has no
 * pending request (for instance after flip_server_drain).
 */
#ifndef FLIP_GB300_SERVER_H
#define FLIP_GB300_SERVER_H

#include "flip.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flip_server flip_server;

typedef struct {
  int32_t scene;
  int32_t status;         /* FLIP_OK, or the step's condition (e.g. FLIP_E_NOT_CONVERGED) */
  double t_arrival;       /* when the request became eligible */
  double t_start;         /* when its batch was formed and enqueued */
  double t_done;          /* when its scene's step had finished on the GPU */
  int32_t batch_size;     /* scenes in the batch that served it */
  int32_t reserved;
} flip_request_info;

/* A server with a device-memory budget for resident scenes and a batch width.
 * max_batch in [1, 4096].  Starts the worker thread. */
int flip_server_create(size_t budget_bytes, int32_t max_batch, flip_server** out);

/* Registers a scene (the particle arrays are copied to host memory).  It becomes
 * resident as soon as its footprint fits in the budget next to the scenes
 * already resident (first come, first admitted); until then its requests wait.
 * A scene larger than the whole budget is refused with FLIP_E_OOM. */
int flip_server_add_scene(flip_server* s, const flip_params* params, const float* x,
                          const float* y, const float* z, const float* u, const float* v,
                          const float* w, int64_t np, int32_t* scene_id);

/* Queues one step of a scene, eligible from t_arrival (t_arrival < 0: now).
 * *ticket identifies the request. */
int flip_server_submit(flip_server* s, int32_t scene, double t_arrival, int64_t* ticket);

/* Blocks until the request is done; fills *info (nullable), then forgets the
 * ticket.  Returns the request's status, the two warnings (FLIP_E_NOT_CONVERGED,
 * FLIP_E_CAPACITY: the step is committed) as FLIP_OK with info->status keeping
 * them, or FLIP_E_ARG for an unknown ticket or one another caller has already
 * collected. */
int flip_server_wait(flip_server* s, int64_t ticket, flip_request_info* info);

/* Blocks until every submitted request is done. */
int flip_server_drain(flip_server* s);

/* enable = 1 (the default): the next batch is formed and enqueued as soon as the
 * previous batch's solve has finished, overlapping that batch's G2P.  enable = 0:
 * one batch at a time; the next is formed when the previous one has completed. */
int flip_server_set_overlap(flip_server* s, int32_t enable);

/* The batches' form (flip_batch_set_fused): 0 (default) per-scene launches on the
 * scenes' streams, each scene completing as its own G2P ends; 1 fused, one launch
 * per step kernel for all the batch's scenes, which then complete together.  Set
 * it while no request is queued. */
int flip_server_set_fused(flip_server* s, int32_t enable);

/* Seconds since the server was created. */
double flip_server_now(const flip_server* s);

/* Scenes resident now and their total footprint in bytes. */
int flip_server_usage(flip_server* s, int32_t* resident, size_t* bytes);

/* The handle of a resident scene, for reads between requests (see above);
 * FLIP_E_ARG when the scene is unknown or not resident yet. */
int flip_server_scene_handle(flip_server* s, int32_t scene, flip_handle** h);

/* Frees a scene once its pending requests are done; its memory then admits
 * waiting scenes. */
int flip_server_remove_scene(flip_server* s, int32_t scene);

/* Stops the worker after the queued requests and frees every scene. */
void flip_server_destroy(flip_server* s);

#ifdef __cplusplus
}
#endif
#endif
