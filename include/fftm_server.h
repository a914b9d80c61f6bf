/*
 * fftm_server.h -- serving runtime over one GPU for the solver of fftm.h.
 *
 * No counterpart in the paper (whose solver runs one problem per job): a request
 * queue for many independent solves of different grid sizes, boundary conditions
 * and laws.  Up to `max_slots` solves are resident at once, each on its own CUDA
 * stream, so their fixed-point iterations (Algorithm 1) interleave on the device;
 * a queued request is admitted, first fit in arrival order, as soon as a slot is
 * free and its device memory (fftm_problem_workspace_bytes + 64 MiB) fits in the
 * remaining budget.  A resident solve keeps its fields and acceleration history on
 * the device until its last load step, then frees them.
 *
 * A result does not depend on which other requests were resident: every solve runs
 * the kernels and launch shapes it runs alone, and none uses atomics (bitwise equal
 * results, checked by the tests).
 *
 * Threads: the server owns `max_slots` host threads; submit/poll/pending may be
 * called from any thread.  Every function returns an fftm status code.
 */
#ifndef FFTM_SERVER_H
#define FFTM_SERVER_H

#include <stddef.h>

#include "fftm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftm_server fftm_server;

typedef struct fftm_request {
  const fftm_problem_desc* desc; /* HOST, copied at submit (with its phase map and
                                    materials); the caller keeps ownership         */
  const fftm_load* loads;        /* HOST, n_loads load steps, copied at submit      */
  int n_loads;                   /* >= 1                                           */
  void* u_out;                   /* HOST buffer for the final u^f (dense node layout
                                    of FFTM_FIELD_U), or NULL; must stay valid until
                                    the request's result has been polled          */
  size_t u_out_bytes;            /* fftm_field_bytes(FFTM_FIELD_U) of the problem   */
} fftm_request;

typedef struct fftm_result {
  long long id;          /* as returned by fftm_server_submit                      */
  int status;            /* FFTM_OK, FFTM_NOT_CONVERGED (a step hit max_iter) or an
                            error code of the failing call                         */
  int steps;             /* load steps run                                         */
  int converged_steps;
  int iterations;        /* Green applications summed over the steps               */
  double err;            /* final equilibrium error of the last step               */
  double mean_P[6];      /* volume mean stress of the last step                    */
  double t_submit, t_start, t_end; /* host monotonic clock, seconds               */
  char message[160];     /* fftm_last_error() of the failing call, or ""           */
} fftm_result;

/* Start a server on `device` with `max_slots` (1..64) resident solves and a device
   memory budget in bytes (0: nine tenths of the memory free at creation).  Returns
   after every worker has started or failed to start (its CUDA stream or library
   context could not be created); FFTM_E_CUDA, with no server, if none started.  A
   server whose workers have all stopped fails its queued requests with FFTM_E_CUDA
   and refuses new ones. */
int fftm_server_create(int device, size_t memory_budget, int max_slots, fftm_server** out);

/* Queue a request; *id (may be NULL) receives its id.  FFTM_E_NOMEM if the request
   alone exceeds the budget, the descriptor's own status if it is invalid. */
int fftm_server_submit(fftm_server* s, const fftm_request* req, long long* id);

/* Move up to max_results finished results to `out` (HOST) in completion order;
   *n_out receives their number.  With wait_for_one, block until at least one result
   is available or nothing is queued or running. */
int fftm_server_poll(fftm_server* s, fftm_result* out, int max_results, int wait_for_one, int* n_out);

/* Requests queued, solves resident, device bytes reserved by resident solves. */
int fftm_server_pending(fftm_server* s, int* queued, int* active, size_t* bytes_in_use);

/* An fftm_set_option call (include/fftm.h, enum fftm_option) that every request submitted
   afterwards gets on its problem, e.g. FFTM_OPT_CUDA_GRAPH 1; a value the problem refuses
   fails that request with the option's status.  FFTM_E_INVALID for an unknown option. */
int fftm_server_set_option(fftm_server* s, int option, int value);

/* Finish every queued request, join the threads, free the server. */
int fftm_server_destroy(fftm_server* s);

/* Test hook (host only, no device work): the next `count` workers started by
   fftm_server_create fail at start-up as if their stream or context could not be
   created.  With count >= max_slots the create call needs no device at all. */
int fftm_server_inject_start_failures(int count);

#ifdef __cplusplus
}
#endif
#endif /* FFTM_SERVER_H */
