/*
 * rgf_server.h - multi-device transmission server (batching and serving).
 *
 * Same computation as rgf.h (T(E) of a block-tridiagonal nonorthogonal
 * device between two periodic leads, mixed precision), for many devices of
 * different lengths, block sizes and energy windows at once.  The paper
 * evaluates one transmission spectrum per device with an O(N_z M_b^3) RGF
 * per energy point (Results, the scaling paragraph); it has no batching or
 * serving layer.  This interface packs the (device, energy) work items of
 * all requests into shared launches:
 *
 *   - block sizes are padded up to a multiple of class_step with decoupled
 *     orbitals (H = -1 and S = 0 on the padded diagonal, zero couplings), so
 *     that z S - H is the identity there for every z and T is unchanged;
 *     one engine per padded size runs on its own CUDA stream;
 *   - an engine owns `slots` energy slots; each slot carries one (device,
 *     energy) item through the sweep at its own layer, and a slot whose
 *     device is finished is refilled from the next lead-decimated items, so
 *     devices of different lengths share every launch (continuous batching);
 *   - lead decimation and self-energies run for up to 148 items at a time,
 *     ahead of the slots that take them;
 *   - from its third step on, an engine replays its step as a captured CUDA
 *     graph (every kernel of the step launched, masks select the entries;
 *     RGF_NO_GRAPHS=1 in the environment launches the kernels directly);
 *   - requests are admitted in arrival order while their resident bytes
 *     (device blocks in double-float, FP64 lead blocks, energies and
 *     results) fit under capacity_bytes; a request that can never fit is
 *     rejected at submission.
 *
 * Numerics are those of RGF_MIXED in rgf.h (tensor-core slice products,
 * Newton-Schulz-refined inverses, FP64-class decimation); the per-energy
 * err and flags outputs mean the same.  Every (device, energy) item is
 * computed by the same sequence of per-entry operations whatever else is in
 * flight, so a request's result does not depend on the mix it ran in.
 *
 * Threads: one admission thread plus one host thread per engine.  All calls
 * are thread-safe.  Orientation and layout of the blocks: as in rgf.h.
 */
#ifndef RGF_SERVER_H
#define RGF_SERVER_H

#include "rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rgf_server_s* rgf_server_t;

typedef struct {
    double dec_tol;         /* decimation tolerance (as rgf_options); default 1e-14 */
    int dec_max_iter;       /* default 100 */
    int ns_steps;           /* most Newton-Schulz steps per inverse; default 6 */
    int slots;              /* energy slots per block-size engine; default 148 */
    int class_step;         /* block sizes are padded to a multiple of this; default 32 */
    size_t capacity_bytes;  /* cap on the admitted requests' resident bytes;
                               0 = 150e9 or 55% of free device memory, whichever is less */
} rgf_server_options;

/* One transport solve.  Block pointers as rgf_set_device_blocks and
 * rgf_set_leads (lead[side][k], k = H00, S00, H10, S10, Hc, Sc); E has n_E
 * energies; all pointers in memory space `mem`.  The server reads these
 * arrays after rgf_server_submit returns (when the request is admitted):
 * the caller keeps them valid and unchanged until the ticket completes. */
typedef struct {
    int n_layers;   /* >= 1 */
    int b;          /* 1 <= b <= 512 */
    double eta;     /* broadening; > 0 */
    const double* H_diag;
    const double* S_diag;
    const double* H_lower;  /* may be NULL when n_layers == 1 */
    const double* S_lower;
    const double* lead[2][6];
    const double* E;
    int n_E;        /* >= 1 */
    int mem;        /* RGF_MEM_HOST or RGF_MEM_DEVICE */
} rgf_request;

typedef struct {
    long long submitted, completed, rejected;
    long long energies_done;
    long long steps;        /* sweep steps over all engines */
    long long decimations;  /* decimation batches over all engines */
    long long fp64_reseeds;
    int engines;            /* block-size engines created */
    size_t resident_bytes;       /* admitted requests now */
    size_t peak_resident_bytes;
    size_t workspace_bytes;      /* engines' fixed workspace */
    double busy_s;          /* first submission to last completion */
    double latency_p50_ms;  /* over completed requests: submission to completion */
    double latency_p99_ms;
    double latency_max_ms;
} rgf_server_stats;

void rgf_server_options_default(rgf_server_options* opt);

/* Create a server on the current CUDA device.  opt may be NULL. */
rgf_status rgf_server_create(rgf_server_t* server, const rgf_server_options* opt);

/* Per-class settings, normally from the autotuner
 * (paper_2609_37058_b300/autotune.py): for requests whose padded block size
 * is block_class, use `slots` energy slots (0 = the server default), tile_n
 * real output columns per tensor-core CTA (64, 80 or 96; 0 = 96) and a
 * Gauss-Jordan panel width of `panel` columns for the FP32 seed inverse
 * (16 or 32; 0 = default).  Must precede the first request of that class
 * (RGF_E_STATE otherwise); RGF_E_INVALID for values out of range. */
rgf_status rgf_server_set_class(rgf_server_t server, int block_class, int slots, int tile_n, int panel);

/* Queue a request; returns at once with a ticket.  RGF_E_INVALID for bad
 * sizes or pointers, RGF_E_REJECTED if its resident bytes exceed the
 * capacity on their own. */
rgf_status rgf_server_submit(rgf_server_t server, const rgf_request* req, rgf_ticket_t* ticket);

/* Wait for a ticket (timeout_us as rgf_poll: 0 = poll, < 0 = wait) and copy
 * its n_E results into T, err, flags (host or device memory, any of err,
 * flags, latency_ms may be NULL).  latency_ms receives the time from
 * submission to completion.  The first call that returns RGF_OK releases
 * the ticket.  A request that failed on the device returns that error. */
rgf_status rgf_server_poll(rgf_server_t server, rgf_ticket_t ticket, double* T, double* err, int* flags,
                           double* latency_ms, int timeout_us);

/* Counters and latency percentiles so far. */
rgf_status rgf_server_stats_get(rgf_server_t server, rgf_server_stats* stats);

/* Stop the threads, wait for in-flight work and free everything.  Tickets
 * not yet polled are lost. */
rgf_status rgf_server_destroy(rgf_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* RGF_SERVER_H */
