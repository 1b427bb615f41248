/*
 * hps_serve.h -- a request loop over the solver of hps.h: continuous batching
 * of factorisation builds and multi-right-hand-side solves on one GPU.
 *
 * The paper has no counterpart: it describes one build followed by solves
 * (Section 1.2: a built solution operator is applied to many boundary data
 * sets, Algorithm 2).  The server keeps built operators resident and serves a
 * stream of requests:
 *
 *   - a build request factors one problem (hps_build) and leaves its operator
 *     resident under the request's id;
 *   - a solve request applies a resident operator to nrhs Dirichlet data sets
 *     (hps_solve); solves waiting on the same operator are coalesced into one
 *     call of up to max_rhs_per_solve right-hand sides.  Every right-hand side
 *     is eliminated and refined on its own, so a coalesced result has the same
 *     bits as the same request served alone.
 *
 * Requests run on `workers` threads, each with its own CUDA stream, so the
 * device overlaps the work of different operators.  A request starts when a
 * worker is free and its device memory (hps_estimate_bytes) fits in
 * hbm_budget next to the resident operators, the running requests and the
 * results not yet released; builds start in arrival order, and when the oldest
 * waiting build does not fit, idle operators are evicted, least recently used
 * first.  A solve on an evicted or failed operator completes with HPS_ENOMEM
 * or the build's status.
 *
 * Inputs are copied at submission; results stay on the device until copied out
 * (hps_server_result) and released (hps_server_release).  All calls are
 * thread-safe.  Return value: HPS_OK or a negative status of hps.h.
 */
#ifndef HPS_SERVE_H
#define HPS_SERVE_H

#include <stdint.h>

#include "hps.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_server_s* hps_server;

typedef struct {
  int64_t hbm_budget;      /* device bytes the server may hold; 0: 90% of the free memory */
  int workers;             /* concurrent device jobs, one stream each (default 4) */
  int max_rhs_per_solve;   /* most right-hand sides coalesced into one solve (default 256) */
  int device;              /* CUDA device ordinal (default 0) */
} hps_server_options;

typedef struct {
  int status;              /* HPS_OK, a negative status, or 1 while pending or running */
  int kind;                /* 0 build, 1 solve */
  int64_t op;              /* operator id (the build request's id) */
  int nrhs;                /* right-hand sides of a solve request */
  int batch_rhs;           /* right-hand sides of the solve call that served it */
  int iterations;          /* refinement corrections of that call (mixed mode) */
  double t_submit, t_start, t_end;  /* seconds on the server's clock */
  int64_t device_bytes;    /* build: bytes the resident operator holds */
} hps_request_info;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t builds, solves, solve_calls, rhs_solved;
  int64_t resident_ops, evicted_ops;
  int64_t bytes_in_use, peak_bytes_in_use, budget;
} hps_server_stats;

void hps_server_default_options(hps_server_options* opt);

/* Start the workers.  HPS_EDEVICE without a usable device. */
int hps_server_create(const hps_server_options* opt, hps_server* out);

/* Finish every submitted request, then free all operators, results and
 * threads.  NULL is accepted. */
int hps_server_destroy(hps_server s);

/* Queue a build of one problem (host coefficient arrays, copied here; the
 * options' device_ptrs and stream are ignored).  Returns the request id,
 * which is also the operator id, or a negative status: HPS_ENOMEM when the
 * build's estimated peak (hps_estimate_bytes) exceeds hbm_budget, since it
 * could never start. */
int64_t hps_server_submit_build(hps_server s, const hps_problem* prob, const hps_options* opt);

/* Queue a solve on operator `op` of nrhs data sets f (host, nrhs * nbnd in
 * the layout of hps_solve, copied here).  Returns the request id or a
 * negative status (HPS_EINVAL for an unknown operator).  A solve whose
 * workspace and result do not fit in hbm_budget next to its own resident
 * operator completes with HPS_ENOMEM instead of waiting. */
int64_t hps_server_submit_solve(hps_server s, int64_t op, const double* f, int nrhs);

/* Wait until request `req` completes or timeout_s seconds pass (< 0: no
 * limit); fills *info (may be NULL).  Returns the request's status, or 1 on
 * timeout. */
int hps_server_wait(hps_server s, int64_t req, double timeout_s, hps_request_info* info);

/* Copy a completed solve's u (nrhs * nx*ny*p*p doubles, layout of hps_solve)
 * to host memory. */
int hps_server_result(hps_server s, int64_t req, double* u);

/* Drop a completed request and its result (its device memory returns to the
 * budget).  A build request's operator stays resident. */
int hps_server_release(hps_server s, int64_t req);

/* Evict an operator once its queued solves have run. */
int hps_server_release_operator(hps_server s, int64_t op);

int hps_server_get_stats(hps_server s, hps_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif
