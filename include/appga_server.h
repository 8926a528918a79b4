/*
 * appga_server.h -- continuous-batching reconstruction server over the
 * batched APPGA kernels (appga.h).
 *
 * The paper reconstructs one slice at a time (Sec. 4); it has no serving
 * layer.  This interface runs a stream of independent reconstruction
 * requests, each one APPGA problem of Eq. APPGAiter with its own sinogram,
 * background and parameters, on one GPU:
 *
 *  - Geometries.  Each image/sinogram size has its own system matrix
 *    (appga_matrix, created by the caller and kept alive until the server is
 *    destroyed).  appga_server_add_geometry registers one and returns its id.
 *  - Pools.  Requests of one geometry run in pools of `slots_per_pool` slots
 *    (or, with slots_per_pool 0, of 32, 64 or 128 slots: each new pool the
 *    narrowest that holds the geometry's demand, its waiting requests plus
 *    those running in its pools, and admission fills
 *    the narrowest pool with a free slot first -- narrow pools step faster at
 *    light load, wide pools read the matrix once for more slices under heavy
 *    load) that share the matrix: one pool is one batched solver (the slot-minor
 *    SpMM kernels of appga_reconstruct_batched) whose iterates, momentum
 *    scalars, objective values and counters stay in device memory for the
 *    whole life of each request.  A pool steps `steps_per_launch` APPGA maps
 *    per replay of a captured CUDA graph.
 *  - Admission.  A waiting request takes a free slot of a pool of its
 *    geometry at the next step boundary, while the pool's other slots keep
 *    iterating (continuous batching).  A new pool is created only when its
 *    device memory fits both the free device memory minus hbm_reserve_bytes
 *    and hbm_budget_bytes minus what the server's pools already hold; when it
 *    does not, empty pools of other geometries are released first, and
 *    otherwise the request waits until memory frees up.
 *  - Retirement.  A slot whose problem reached max_iters maps or its
 *    relative-objective stopping test is copied out at the step boundary
 *    where the host sees it finished, and the slot is free again.
 *  - Latency.  Each request records submission, admission and completion
 *    times (host steady clock, seconds since server creation);
 *    appga_server_get_summary reports p50/p99 latency and slice-iterations.
 *
 * A request's result does not depend on which slot it runs in, on the other
 * requests of its pool, or on when it was admitted: every slot runs the same
 * per-slot arithmetic, so the same request gives the same image alone and in
 * any mix with the same pool width and precision.  (With adaptive widths a
 * request's pool width depends on the load, and images of the same request
 * agree to FP32 rounding across widths.)
 *
 * Streams: every pool has its own stream, so the replays of different pools
 * (and geometries) overlap on the device.  A scheduling round
 * (appga_server_step) handles the pools whose last replay has landed --
 * retiring their finished slots, admitting waiting requests into them and
 * starting their next replay -- and leaves running pools alone; it blocks
 * only when no pool's work landed and none started.  A retirement copies the
 * finished images out asynchronously and completes (state DONE) in a later
 * round.
 *
 * Threading: a server is driven by one host thread at a time.  Pointers
 * named *_host are host memory; the server copies what it needs during the
 * call.
 */
#ifndef APPGA_SERVER_H
#define APPGA_SERVER_H

#include "appga.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct appga_server appga_server;

typedef struct {
  int32_t slots_per_pool;    /* 32, 64 or 128 slots per pool; 0: adaptive (above) */
  int32_t steps_per_launch;  /* APPGA maps per graph replay, >= 1 */
  int32_t a_precision;       /* APPGA_PREC_FP32 or APPGA_PREC_BF16 (the
                                matrix needs its BF16 copy) for every pool */
  int32_t max_pools;         /* cap on live pools over all geometries; 0 = none */
  int64_t hbm_budget_bytes;  /* cap on device bytes held by pools; 0 = none */
  int64_t hbm_reserve_bytes; /* device memory a new pool must leave free */
  int32_t max_pools_per_geometry; /* cap on live pools of one geometry; 0 = none.
                                     Under load more pools of a geometry stream its
                                     matrix more often and contend for the device;
                                     requests beyond the cap wait for free slots */
  int32_t pad;
} appga_server_config;

/* Defaults: 64 slots per pool, 8 maps per launch, FP32, no pool cap, no
 * budget, 1 GiB reserve, 2 pools per geometry. */
void appga_server_config_default(appga_server_config* cfg);

/* Request states. */
#define APPGA_REQ_WAITING 0 /* submitted, not yet in a slot */
#define APPGA_REQ_RUNNING 1 /* iterating in a slot */
#define APPGA_REQ_DONE 2    /* result ready for appga_server_collect */

typedef struct {
  int32_t state;          /* APPGA_REQ_* */
  int32_t iters;          /* APPGA maps applied to produce the result */
  int32_t result_k;       /* iterate index of the result (f^{result_k}) */
  int32_t stopped_early;  /* 1 if the relative-objective test fired */
  int32_t flags;          /* APPGA_FLAG_* seen by the request's pool */
  int32_t phi_k;          /* index of the last iterate whose Phi was evaluated */
  int64_t guard_hits;     /* guarded bins over the request's iterations */
  double phi_last;        /* Phi(f^{phi_k}) in FP64 (NaN before the first) */
  double t_submit, t_admit, t_done; /* seconds since server creation (NaN if not yet) */
} appga_request_stats;

typedef struct {
  int64_t submitted, completed, waiting, running;
  int64_t slice_iters;   /* APPGA maps over all completed requests */
  int32_t pools;         /* live pools */
  int32_t pad;
  int64_t device_bytes;  /* device memory held by live pools */
  double p50_latency_s, p99_latency_s; /* completion minus submission (nearest rank) */
  double mean_latency_s, max_latency_s;
  double mean_queue_s;   /* admission minus submission, mean over completed */
  /* occupancy: slot-steps the pools ran (pool width x maps per replay, over
   * every replay) and, of those, the slot-steps of slots holding a request
   * when the replay started; device seconds of the replays (each from its
   * start to its slot-state copy, summed over pools, so overlapping replays
   * of different pools add up) */
  int64_t pool_slot_steps, live_slot_steps;
  double replay_seconds;
} appga_server_summary;

/* appga_server_create: EINVAL for a bad config (slots_per_pool not 0, 32, 64
 * or 128; steps_per_launch < 1; negative sizes). */
appga_status appga_server_create(appga_ctx* ctx, const appga_server_config* cfg,
                                 appga_server** out);
/* Frees every pool; requests not collected are dropped. */
appga_status appga_server_destroy(appga_server* srv);

/* Registers a geometry (its matrix must come from the server's context and
 * outlive the server).  EINVAL if it belongs to another context, if the
 * config asks for BF16 and the matrix has no BF16 copy, or if max(m, d)
 * times the widest pool the server may create (slots_per_pool, or 128 when
 * widths are adaptive) reaches 2^31 (the batched kernels' 32-bit offsets). */
appga_status appga_server_add_geometry(appga_server* srv, const appga_matrix* mat,
                                       int32_t* geometry_out);

/* Queues one request.  g_host: float[m] counts (finite, >= 0); gamma_host:
 * float[m] background (finite, > 0); f_init_host: float[d] initial image
 * (finite, >= 0) or NULL for TMC * 1_disk (Sec. 4.1); params: as in
 * appga.h (lambda1, lambda2, eps, omega, a, b, beta, max_iters,
 * rel_obj_tol, precond_freeze_iter, momentum are per request; a_precision,
 * track_objective and graph_iters are set by the server: the objective is
 * always evaluated on the device each iteration).  The inputs are copied
 * before the call returns.  EINVAL (bad geometry id, parameters) or
 * EDOMAIN (input values) with nothing queued. */
appga_status appga_server_submit(appga_server* srv, int32_t geometry, const float* g_host,
                                 const float* gamma_host, const float* f_init_host,
                                 const appga_params* params, int64_t* request_out);

/* One scheduling round: admit waiting requests into free slots (creating
 * pools as memory allows), run one graph replay (steps_per_launch maps) of
 * every pool that holds requests, and retire finished requests.  Returns
 * when the round's device work has finished.  pending_out (may be NULL):
 * requests waiting or running after the round. */
appga_status appga_server_step(appga_server* srv, int32_t* pending_out);

/* State and statistics of a request.  EINVAL for an unknown (or already
 * collected) id. */
appga_status appga_server_poll(const appga_server* srv, int64_t request,
                               appga_request_stats* stats_out);

/* Copies a finished request's image (float[d], host) and statistics, then
 * forgets the request.  EBUSY if it is not finished; EINVAL if unknown. */
appga_status appga_server_collect(appga_server* srv, int64_t request, float* f_out_host,
                                  appga_request_stats* stats_out);

appga_status appga_server_get_summary(const appga_server* srv, appga_server_summary* out);

#ifdef __cplusplus
}
#endif

#endif /* APPGA_SERVER_H */
