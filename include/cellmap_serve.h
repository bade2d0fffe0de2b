/*
 * cellmap_serve.h -- request server over the cell-list pair map: many
 * independent analysis or energy/force requests of uneven particle counts and
 * box shapes served from one GPU with continuous batching.
 *
 * The paper (Sec. 2.7-2.8) maps one function over one system at a time and
 * parallelises inside that system; it has no server. This layer applies the
 * same map to a stream of systems: a request is a set of positions, a box
 * with cutoff (Sec. 2.5) and a task (energy, forces or distance histogram:
 * Code 5, Code 7, Code 10).
 *
 * Scheduling (a host thread inside the library):
 *  - admission: queued requests are admitted in arrival order while the
 *    device arena (one allocation made at creation) has room for their
 *    positions, cell list, stencil and outputs and fewer than max_inflight
 *    requests are resident; a request larger than the whole arena fails with
 *    CL_ERR_OOM without blocking the others;
 *  - build: each admitted request copies its positions in and builds its cell
 *    list on one of several build streams, overlapping with sweeps in flight;
 *  - batch: all admitted requests not yet swept form one batch, swept by ONE
 *    persistent kernel launch whose CTAs take (request, tile) items from a
 *    device work counter; at most two batches are in flight, so requests that
 *    arrive while a batch runs join the next one (continuous batching);
 *  - completion: per-request fixed-order FP64 reduction, results copied to
 *    the caller's host buffers, arena space released.
 * Each request's result does not depend on what it was batched with: the same
 * kernels, stencil and reduction order run for it alone or in a mix (FP32
 * sums may differ in the last bits when the cell list's slot order differs).
 *
 * Host buffers should be page-locked (e.g. cudaMallocHost or torch
 * pin_memory) for the copies to be asynchronous; pageable buffers work but
 * their copies serialise. Buffers must stay valid until the ticket completes.
 */
#ifndef CELLMAP_SERVE_H
#define CELLMAP_SERVE_H

#include "cellmap.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CL_TASK_ENERGY 0  /* shifted-force energy (half shell) -> energy_host */
#define CL_TASK_FORCES 1  /* energy, forces F = -dE/dx, virial (full shell) -> energy, forces, virial */
#define CL_TASK_HIST 2    /* nbins distance histogram over [0, rmax) (half shell) -> hist_host */

typedef struct {
  const double* pos_host;          /* (n, dim) FP64, host */
  long long n;                     /* 0 <= n < 2^31 */
  cl_box box;                      /* dim, lattice rows, cutoff, lcell */
  int task;                        /* CL_TASK_* */
  int nbins;                       /* CL_TASK_HIST: 1..4096 */
  double rmax;                     /* CL_TASK_HIST: <= 0 means the cutoff */
  double* energy_host;             /* 1 value (ENERGY, FORCES) */
  float* forces_host;              /* n*dim (FORCES) */
  double* virial_host;             /* dim*dim (FORCES), may be NULL */
  unsigned long long* hist_host;   /* nbins (HIST) */
} cl_request;

typedef struct cl_server cl_server;

/* Create a server on `device` with a device arena of arena_bytes and at most
 * max_inflight resident requests (1..1024). Starts the scheduling thread. */
int cl_serve_create(long long arena_bytes, int max_inflight, int device, cl_server** out);

/* Queue a request (thread-safe, returns at once). *ticket identifies it. The
 * request's box is checked here: an invalid box or cutoff returns its error
 * code and queues nothing. */
int cl_serve_submit(cl_server* s, const cl_request* req, long long* ticket);

/* Status of a ticket: 1 = pending, 0 = done, negative = failed with that
 * error code (CL_ERR_CUDA when a copy or kernel launch of its batch failed).
 * Non-blocking. */
int cl_serve_poll(cl_server* s, long long ticket);

/* Wait up to timeout_s seconds for a ticket; returns its status (1 on timeout). */
int cl_serve_wait(cl_server* s, long long ticket, double timeout_s);

/* Host timestamps of a ticket in seconds on the server's steady clock:
 * times[0] submitted, [1] admitted, [2] batch launched, [3] completed. */
int cl_serve_times(cl_server* s, long long ticket, double* times);

/* Counters: stats[0] batches launched, [1] requests completed, [2] requests
 * failed, [3] largest batch, [4] arena bytes in use, [5] arena bytes. */
int cl_serve_stats(cl_server* s, long long* stats);

/* The server's steady clock now, in seconds (same origin as cl_serve_times). */
double cl_serve_clock(cl_server* s);

/* Forget a finished ticket. A ticket's status and timestamps (under 1 KB
 * of host memory; its CUDA event is freed when it completes) are kept until
 * this call or cl_serve_free, so a long-running server should release each
 * ticket once it has read them. Returns CL_OK, 1 when the ticket is still
 * pending (nothing is released), or CL_ERR_INVALID_ARG for an unknown or
 * already released ticket, which later calls also report. */
int cl_serve_release(cl_server* s, long long ticket);

/* Stop the thread after the queued work completes and release everything. */
void cl_serve_free(cl_server* s);

#ifdef __cplusplus
}
#endif

#endif /* CELLMAP_SERVE_H */
