/* tpcca.h — C ABI of the GB300 TPC sector tracker.
 *
 * Implements the sector tracker of Rohr et al., "ALICE HLT TPC Tracking of
 * Pb-Pb Events on GPUs": clusters measured on the 159 pad rows of each of the
 * 36 TPC sectors go in (Section 1: "reconstructed clusters are sent to the
 * sector tracker which reconstructs the tracks in each TPC sector
 * individually"); per-track parameters, covariances and the list of the
 * clusters of each track come out (Section 3.3: the sector tracker "outputs a
 * list of clusters for each track").  Between them run the steps of Section 1
 * (neighbours finder, evolution, tracklets from chains of one-to-one links,
 * Kalman tracklet construction, tracklet selection) with the cluster weight of
 * Section 3.1, the track sorting of Section 3.2 and the 30-cluster minimum of
 * Section 5, all as CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Every function returns an int status (TPC_OK = 0) unless stated otherwise;
 *    nothing throws across this boundary.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary (or pinned) host memory.
 *  - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *    default stream).  All device work of a call is ordered on that stream.
 *  - Cluster input layout (SoA): y[i], z[i] float32 (cm, sector-local frame:
 *    x along the sector centre, y in r-phi, z global), row[i] uint8 pad row.
 *    Clusters are grouped by sector, then by row: counts[s * n_rows + r] is the
 *    number of clusters of sector s on row r, and they follow each other in
 *    that order.  Order inside one (sector, row) group is free.
 *  - Track parameters are (y, z, sin phi, tan lambda, q/pT) at the plane x of
 *    the track's innermost cluster, in its sector's frame; curvature is
 *    -kappa * Bz * q/pT with kappa = 2.99792458e-3 GeV/(T cm).  Covariances are
 *    15 floats: the lower triangle, row-major, of the 5x5 matrix in that order.
 */
#ifndef TPCCA_H
#define TPCCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    TPC_OK = 0,
    TPC_ERR_INVALID_ARG = 1,   /* bad pointer, counts not summing to n, a cluster on the wrong row */
    TPC_ERR_CAPACITY = 2,      /* a device pool overflowed; tpc_last_error_detail says where */
    TPC_ERR_BUDGET = 3,        /* the call would exceed the tracker's HBM budget */
    TPC_ERR_TIMEOUT = 4,       /* a bounded device-side wait expired */
    TPC_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    TPC_ERR_STATE = 6,         /* wrong call order (e.g. reading a result before it was produced) */
    TPC_ERR_CHECK = 7          /* an index bounds check of the checked build failed (internal error) */
};

/* Pipeline stages, as reported by tpc_last_error_detail. */
enum {
    TPC_STAGE_NONE = 0,
    TPC_STAGE_INGEST = 1,      /* A1 cluster ingest and per-row grids */
    TPC_STAGE_NEIGHBOURS = 2,  /* A2 */
    TPC_STAGE_EVOLUTION = 3,   /* A3 + A4 */
    TPC_STAGE_CONSTRUCTION = 4,/* A5 */
    TPC_STAGE_SELECTION = 5,   /* A6 */
    TPC_STAGE_OUTPUT = 6,      /* A7 */
    TPC_STAGE_GLOBAL = 7,      /* global tracking (Section 5), between A6 and A7 */
    TPC_STAGE_MERGE = 8        /* track merger with refit, after A7 */
};

/* Detector geometry (Section 1: two volumes of 18 trapezoidal sectors, 159 pad rows).
 * row_x: host array of n_rows row positions (cm), strictly increasing, copied at create.
 * n_sectors: 36 (z >= 0 for sectors 0-17, z < 0 for 18-35) or 1 (one phi sector
 * spanning both z halves). */
typedef struct {
    int n_rows;
    const float *row_x;
    float tan_half;            /* tan of the sector half-opening, tan(10 deg) */
    float z_max;               /* half-length of the drift volume (cm) */
    int n_sectors;
} tpc_geometry;

/* Tracker constants.  alpha = 6 (Section 3.1) and min_clusters = 30 (Section 5)
 * are the paper's; every other default is a reading of a point the paper leaves
 * open (see tpc_params_default). */
typedef struct {
    float sigma_y, sigma_z;    /* cluster errors (cm) */
    float nb_ty, nb_tz;        /* neighbours finder window: |dy| <= ty*dx, |dz| <= tz*dx */
    float nb_gate;             /* straight-line gate: score <= nb_gate * (1 + wd^2 + wu^2) */
    int min_chain;             /* clusters in a chain of one-to-one links to start a tracklet */
    float seed_cov[5];         /* diagonal of the seed covariance */
    float win_nsigma;          /* construction search window half-width in sigmas */
    float chi2_max;            /* 2-dof chi2 gate for a cluster */
    int max_miss;              /* consecutive rows without a cluster that end a pass */
    float edge_margin;         /* a pass ends when |y| > x * tan_half + edge_margin */
    float sin_max;             /* a pass ends when |sin phi| reaches sin_max */
    float alpha, beta;         /* cluster weight w = n * (alpha - (chi2/ndf) / beta) */
    int min_clusters;          /* minimum clusters of a track */
    float qpt_max;             /* low-momentum cut: |q/pT| <= qpt_max */
    int global_tracking;       /* 1: prolong every track into the neighbouring sectors (Section 5); only
                                  with 36 sectors, ignored otherwise; 0 by default */
    int merge;                 /* 1: track merger with refit (Sections 1 and 3.3): every track is refitted
                                  from its clusters alone and tracks continuing each other across a sector
                                  border (azimuth neighbours, or the other z half) are merged; only with 36
                                  sectors; 0 by default.  The result then holds the merged tracks. */
    float merge_chi2;          /* 5-parameter chi2 gate of a merge */
    float merge_gap;           /* largest radial gap (cm) between the merged ends */
    float merge_qpt_nsigma;    /* q/pT gate of a merge, in combined sigmas */
} tpc_params;

/* Launch and grid choices.  None of them changes any result (every search
 * enumerates all grid cells that overlap its window and applies the exact window
 * test), so the autotuner may pick them freely. */
typedef struct {
    float bin_occupancy;       /* target clusters per grid cell (>0) */
    int neighbours_block;      /* threads per CTA of the neighbours finder (multiple of 32, <= 256) */
    int construct_block;       /* threads per CTA of the tracklet constructor (multiple of 32, <= 128) */
    int construct_ctas_per_sm; /* persistent CTAs per SM of the work-queue constructor (0 = occupancy limit) */
    int construct_mode;        /* 0: one lane per tracklet from a work queue; 1: per-sector row sweep with rows
                                  staged in shared memory.  Same visits, same arithmetic, same results. */
    int stage_rows;            /* form of the neighbours finder: 0 one thread per cluster, rows k-1, k+1 read from
                                  global memory; 1 the same with the rows staged into shared memory by bulk
                                  copies (default); 2 warp-cooperative search on the staged rows (candidates
                                  and pairs of 32 clusters spread over the lanes).  Same links in every form. */
    int tracklet_capacity;     /* 0: n/4 + 64 per call; > 0: store at most this many tracklets (a capacity
                                  knob: more start hits make the call fail with TPC_ERR_CAPACITY) */
    int use_graph;             /* 1: every call's copies, clears and kernels are captured into a CUDA graph
                                  (on a stream of the tracker's own) that updates the tracker's executable
                                  graph in place and is launched on the call's stream as one unit (default);
                                  0: plain stream launches.  Same work, same results. */
    int seed_kernel;           /* 1: a separate launch computes every seed first (default); 0: each
                                  constructor lane walks its tracklet's chain for the seed when it takes the
                                  tracklet; -1: chosen by the call's size (1 above 40 clusters per lane of
                                  5 CTAs per SM).  Same seeds, same results. */
    int order_group;           /* cluster slots per group of the constructor's work order (a call with many
                                  events builds one group's tracklets before the next group's, so that the
                                  rows being searched stay in L2); 0: one group.  At most 6144 / kb groups
                                  per call, kb = 2 n_rows + 2 rounded up to a multiple of 32 (19 groups for
                                  159 rows; larger groups when the call holds more). */
} tpc_tuning;

typedef struct tpc_tracker tpc_tracker;
typedef struct tpc_result tpc_result;

/* Read-only view of a finished result.  All pointers are device pointers owned by
 * the result; they stay valid until tpc_result_release.  Track m's clusters are
 * hits[first[m] .. first[m] + nhits[m]), ordered from the innermost to the
 * outermost row, given as indices into the call's input arrays (for a batch: into
 * the concatenated input).  Tracks are sorted by (event, sector, row and input
 * index of their innermost cluster) (Section 3.2). */
typedef struct {
    int64_t n_tracks;
    int64_t n_hits;
    const float *par;          /* [n_tracks * 5] */
    const float *cov;          /* [n_tracks * 15] */
    const float *x_ref;        /* [n_tracks] x of the innermost cluster */
    const float *alpha;        /* [n_tracks] sector centre azimuth (rad) */
    const float *chi2;         /* [n_tracks] sum of the Kalman update chi2 */
    const int32_t *ndf;        /* [n_tracks] 2 * fitted clusters - 5 */
    const int32_t *nhits;      /* [n_tracks] clusters kept by the track */
    const int32_t *first;      /* [n_tracks] offset into hits */
    const int32_t *sector;     /* [n_tracks] sector within its event */
    const int32_t *event;      /* [n_tracks] event within the batch */
    const int32_t *hits;       /* [n_hits] input cluster indices */
} tpc_track_view;

/* Fill *p with the default constants.  Never fails. */
void tpc_params_default(tpc_params *p);

/* Fill *t with the default launch choices (measured on a GB300): bin_occupancy 0.5,
 * neighbours_block 256, construct_block 64 with construct_ctas_per_sm 11, construct_mode 0,
 * stage_rows 1, tracklet_capacity 0, use_graph 1, seed_kernel 1, order_group 3 << 20.
 * Never fails. */
void tpc_tuning_default(tpc_tuning *t);

/* Create a tracker on the current CUDA device.
 * geometry: host struct, copied.  bz_tesla: solenoid field.
 * params: host struct or NULL for tpc_params_default.
 * hbm_budget: bytes of device memory the tracker may hold (workspace plus live
 *   results); 0 = no limit.  Work that would exceed it fails with TPC_ERR_BUDGET.
 * *out receives the handle (owned by the caller; free with tpc_tracker_destroy).
 * Errors: TPC_ERR_INVALID_ARG (NULL out/geometry, n_rows outside 3..255, row_x not
 * increasing, n_sectors not 1 or 36), TPC_ERR_CUDA. */
int tpc_tracker_create(const tpc_geometry *geometry, float bz_tesla, const tpc_params *params,
                       size_t hbm_budget, tpc_tracker **out);

/* Replace the launch choices (host struct, copied).  Results are unchanged. */
int tpc_tracker_set_tuning(tpc_tracker *tr, const tpc_tuning *t);

/* Pre-size the device workspace and the pinned host staging of the per-row metadata for
 * batches of up to max_clusters clusters and max_events events, so that later calls of that
 * size allocate nothing but their result (see tpc_tracker_reserve_results for those).
 * Errors: TPC_ERR_BUDGET, TPC_ERR_CUDA. */
int tpc_tracker_reserve(tpc_tracker *tr, int64_t max_clusters, int max_events);

/* Preallocate the device memory of `depth` results, each sized for the workspace reserved
 * with tpc_tracker_reserve (its clusters and events), so that tracking calls allocate nothing
 * at all: every call takes one of these result buffers and tpc_result_release gives it back.
 * This is the preallocated output pool of a tracker that serves a stream of events (Section 2
 * keeps the output buffers of each sector resident for the same reason; Section 6 reports a
 * run that failed when a noisy sector exhausted device memory, which a fixed pool turns into a
 * refusal instead).  Results held by the caller count against it: a call made while all
 * `depth` results are held returns TPC_ERR_BUDGET and enqueues nothing.  A released result's
 * buffers are reused by a later call only after the work enqueued on the released result's
 * stream up to the release (e.g. the caller's copies of it) has finished.  A call larger than
 * the reserved workspace grows the workspace and the buffer it takes (synchronously).
 * depth = 0 returns to one allocation per call (buffers still held are freed at their release);
 * a smaller depth than before frees the surplus.
 * Errors: TPC_ERR_STATE (depth > 0 before any tpc_tracker_reserve), TPC_ERR_INVALID_ARG
 * (depth < 0 or > 4096), TPC_ERR_BUDGET (the buffers exceed the HBM budget), TPC_ERR_CUDA. */
int tpc_tracker_reserve_results(tpc_tracker *tr, int depth);

/* Track one event (Section 1; all 36 sectors).  y, z, row: device arrays of n
 * clusters, owned by the caller, which must keep them valid until the stream has
 * passed this call's work.  counts: HOST array of n_sectors * n_rows counts in
 * the grouped order described above; it is read before the call returns.
 * The work is enqueued on `stream`; *out receives a result handle whose data is
 * valid once tpc_result_sync_counts has returned TPC_OK.
 * Calls on one tracker are ordered: a call waits (on the device) for the previous
 * call's use of the shared workspace.
 * Errors: TPC_ERR_INVALID_ARG (counts not summing to n, n < 0, NULL pointers with
 * n > 0), TPC_ERR_BUDGET, TPC_ERR_CUDA.  Device-side errors (a cluster on the
 * wrong row, pool overflow, timeout) are reported by tpc_result_sync_counts. */
int tpc_track_event(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                    const int32_t *counts, int64_t n, void *stream, tpc_result **out);

/* Track n_events events in one pass of every stage (each stage is one launch over
 * all sectors of all events).  The events' clusters are concatenated in y, z,
 * row (device, n_total clusters); counts (host) holds n_events * n_sectors *
 * n_rows counts, event-major.  Results are identical to one call per event.
 * Errors as tpc_track_event. */
int tpc_track_batch(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                    const int32_t *counts, int n_events, int64_t n_total, void *stream,
                    tpc_result **out);

/* Same as tpc_track_event, but y, z, row are HOST arrays: the call copies them to
 * the device on `stream` (from pinned memory when the caller's buffers are
 * pinned) before tracking. */
int tpc_track_event_host(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                         const int32_t *counts, int64_t n, void *stream, tpc_result **out);

/* Same as tpc_track_batch, but y, z, row are HOST arrays (n_total clusters of
 * n_events events, concatenated), copied to the device on `stream` first. */
int tpc_track_batch_host(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                         const int32_t *counts, int n_events, int64_t n_total, void *stream,
                         tpc_result **out);

/* Wait for the result's work and return its track and hit counts (either pointer
 * may be NULL).  Returns the device-side status of the call: TPC_OK,
 * TPC_ERR_INVALID_ARG (a cluster's row byte disagrees with counts),
 * TPC_ERR_CAPACITY, TPC_ERR_TIMEOUT, or TPC_ERR_CUDA. */
int tpc_result_sync_counts(tpc_result *res, int64_t *n_tracks, int64_t *n_hits);

/* Non-blocking completion test: 1 if the result's work has finished (a following
 * tpc_result_sync_counts returns at once), 0 if it is still running, or a negative
 * TPC_ERR_* value (-TPC_ERR_CUDA) if the query failed. */
int tpc_result_ready(tpc_result *res);

/* Fill *view with device pointers to the result.  Requires a successful
 * tpc_result_sync_counts first (TPC_ERR_STATE otherwise). */
int tpc_result_get(tpc_result *res, tpc_track_view *view);

/* Copy the whole result to host buffers sized from tpc_result_sync_counts
 * (any pointer may be NULL to skip that array).  Synchronous: returns when the result's call
 * has finished and its arrays are in the host buffers.  The copies run on a stream of the
 * tracker's own, so they do not wait for later calls queued on the call's stream. */
int tpc_result_copy_to_host(tpc_result *res, float *par, float *cov, float *x_ref, float *alpha,
                            float *chi2, int32_t *ndf, int32_t *nhits, int32_t *first,
                            int32_t *sector, int32_t *event, int32_t *hits);

/* Release a result and its device memory (stream-ordered on the call's stream).
 * NULL is ignored. */
void tpc_result_release(tpc_result *res);

/* Destroy a tracker after its outstanding work finishes; its device workspace is freed at
 * once.  Results it created that the caller still holds must still be released with
 * tpc_result_release (the last release frees the tracker's remaining host state).  NULL
 * and repeated calls are ignored. */
void tpc_tracker_destroy(tpc_tracker *tr);

/* Static text for a status code; never NULL. */
const char *tpc_status_string(int status);

/* Where the last device-side error of the tracker happened (each pointer may be
 * NULL): event index in the batch, sector, and TPC_STAGE_* of the stage.
 * Returns that error's status (TPC_OK if none). */
int tpc_last_error_detail(tpc_tracker *tr, int *event, int *sector, int *stage);

/* Statistics of one call.  ms[] holds device milliseconds per stage, measured with
 * CUDA events on the call's stream when timing was enabled for the call (zeros
 * otherwise): ms[0] set-up copies and clears, ms[TPC_STAGE_INGEST .. TPC_STAGE_MERGE]
 * the stages.  The counts are the work units the roofline figures are based on. */
typedef struct {
    float ms[10];
    int kernel_launches;           /* kernels this library launched for the call */
    int64_t clusters;              /* input clusters */
    int64_t tracklets;             /* start hits = tracklets built (A4, A5) */
    int64_t row_visits;            /* A5 row visits (searches), both passes */
    int64_t candidates;            /* A5 clusters read inside the searched grid cells */
    int64_t tracks;                /* output tracks (after the merger when it runs) */
    int64_t hits;                  /* output clusters */
    int64_t global_found;          /* clusters found by the global-tracking prolongations (before claims) */
    int64_t graph_builds;          /* executable graphs the tracker instantiated up to this call (graph mode) */
    int64_t sector_tracks;         /* tracks before the merger (= tracks when it does not run) */
    int64_t tracklet_hits;         /* A6 clusters of the tracklets that claim clusters */
} tpc_call_stats;

/* Host-side fault injection for failure tests; no GPU fault is involved.  what = 0: off;
 * 1: with rows staged (stage_rows 1 or 2), after the neighbours finder's shared-memory
 * staging of sector 0's middle row has completed
 * (no asynchronous copy is outstanding), its CTA also waits on a barrier that nothing completes,
 * so that bounded wait (1 s of device time) expires and the call reports TPC_ERR_TIMEOUT with
 * stage TPC_STAGE_NEIGHBOURS.  Returns TPC_ERR_INVALID_ARG otherwise. */
int tpc_tracker_inject(tpc_tracker *tr, int what);

/* Enable (1) or disable (0) per-stage event timing for the following calls. */
int tpc_tracker_set_timing(tpc_tracker *tr, int enable);

/* Fill *st for the call that produced res; waits for that call to finish.
 * Errors: TPC_ERR_INVALID_ARG, TPC_ERR_CUDA. */
int tpc_result_stats(tpc_result *res, tpc_call_stats *st);

/* Largest event tpc_find_links_noalloc accepts: clusters, and row units
 * (n_sectors * n_rows of one event). */
#define TPC_NOALLOC_MAX_CLUSTERS 1048576
#define TPC_NOALLOC_MAX_UNITS (36 * 255)

/* Neighbours finder and evolution (the cellular-automaton links) of one event,
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, for instance code
 * that runs inside a framework which hands all device memory to its own
 * allocator at start-up, or a real-time process that must not allocate (nor
 * synchronise the device the way cudaMalloc can) once data taking has started.
 *
 * Inputs as for tpc_track_event: y, z, row device arrays of n clusters, counts a
 * HOST array of n_sectors * n_rows counts.  Outputs (device, caller-owned):
 * up[i], dn[i] = input index of the cluster linked to cluster i on the next /
 * previous row after the evolution step, -1 for none.  status (device, may be
 * NULL) receives 4 ints: device-side status, event, sector, stage (as
 * tpc_last_error_detail).  All work is ordered on `stream`.
 *
 * The intermediate data (binned clusters, grids, raw links) live in one static
 * device array of about 31 MB sized for TPC_NOALLOC_MAX_CLUSTERS clusters; it is
 * reserved on each GPU whose copy of this part of the library has been loaded
 * and stays there until the process exits.  Every call uses the same array and
 * it keeps the previous call's contents, so calls whose GPU work overlaps (two
 * streams, two threads, two trackers) race and corrupt each other: order them on
 * one stream or synchronise between them.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.
 * Errors (returned): TPC_ERR_INVALID_ARG (NULL pointers with n > 0, counts not
 * summing to n, n > TPC_NOALLOC_MAX_CLUSTERS, more row units than
 * TPC_NOALLOC_MAX_UNITS), TPC_ERR_CUDA. */
int tpc_find_links_noalloc(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                           const int32_t *counts, int64_t n, int32_t *up, int32_t *dn,
                           int32_t *status, void *stream);

/* Intermediate buffers of the tracker's last call, for per-stage checks.  Device
 * pointers into the tracker's workspace; valid until its next call.  Cluster
 * slots are "sorted" positions: slot j of row unit u = (event * n_sectors +
 * sector) * n_rows + row is sorted_offset[u] + j for j < count[u].  */
typedef struct {
    int64_t n_units;               /* events * n_sectors * n_rows */
    int64_t n_slots;               /* size of the slot arrays */
    int64_t n_tracklets;           /* tracklets (start hits) of the last call */
    int64_t tracklet_capacity;
    const int32_t *unit_meta;      /* [n_units * 4] input offset, count, sorted offset, cell offset */
    const int32_t *unit_cells;     /* [n_units * 2] cells along y and z */
    const float *unit_grid;        /* [n_units * 4] ymin, zmin, 1/dy, 1/dz */
    const int32_t *cell_start;     /* cell starts, [cell offset + c], relative to the row's first slot */
    const float *yz;               /* [n_slots * 2] y, z in slot order */
    const int32_t *orig;           /* [n_slots] input index of each slot */
    const int32_t *up_raw, *dn_raw;/* [n_slots] A2 links (slots, -1 none) */
    const int32_t *up, *dn;        /* [n_slots] A3 kept links */
    const int32_t *starts;         /* [n_tracklets * 4] first slot, -1, -1, (sector << 16) | (chain length, counted up to 4 or min_chain, << 8) | row */
    const int32_t *tl_nhits;       /* [capacity] */
    const int32_t *tl_hits;        /* [capacity * n_rows] slots, outer to inner */
    const float *tl_par;           /* [5 * capacity] component-major */
    const float *tl_cov;           /* [15 * capacity] component-major */
    const float *tl_x, *tl_chi2, *tl_w; /* [capacity] */
    const int32_t *tl_nowned;      /* [capacity] */
    const uint64_t *cluster_key;   /* [n_slots] winning weight key per slot */
} tpc_debug_view;

/* Fill *v from the tracker's last call (synchronises the device first). */
int tpc_tracker_debug_view(tpc_tracker *tr, tpc_debug_view *v);

/* ---------------------------------------------------------------------------------------
 * Serving loop with continuous batching (the HLT requirement of the abstract: more than 200
 * central events per second; it replaces the paper's CPU/GPU pipeline of Section 2).
 *
 * A server owns `lanes` trackers, each with its own stream, device input buffers and workspace
 * reserved for lane_clusters clusters and max_batch events.  Events are submitted from any
 * thread; a server thread forms a batch whenever a lane is free (up to max_batch events that
 * fit the lane), copies the events' clusters from the caller's buffers, tracks the batch with
 * one tpc_track_batch call, copies the result back and splits it per event.  Results are the
 * same as for the event tracked alone.  The paper has no counterpart of this interface.
 * --------------------------------------------------------------------------------------- */
typedef struct tpc_server tpc_server;

typedef struct {
    int lanes;                 /* trackers working concurrently (>= 1) */
    int max_batch;             /* events per batch (>= 1) */
    int64_t lane_clusters;     /* clusters reserved per lane; larger events are refused */
    size_t hbm_budget;         /* device bytes for all lanes together (0: no limit) */
} tpc_server_config;

/* One finished event.  Host pointers owned by the server, valid until tpc_server_release.
 * Tracks in canonical order; hits are indices into the event's own input arrays. */
typedef struct {
    int status;                /* TPC_OK, or the error of this event (its batch was retried alone) */
    int64_t n_tracks, n_hits;
    const float *par, *cov, *x_ref, *alpha, *chi2;
    const int32_t *ndf, *nhits, *first, *sector, *hits;
    int64_t t_submit_ns, t_launch_ns, t_done_ns;   /* tpc_server_now_ns clock */
    int batch_size;            /* events in the batch that carried it */
} tpc_server_result;

/* Create a server on the current device.  params: NULL for the defaults.  Returns
 * TPC_ERR_BUDGET if a lane's buffers do not fit hbm_budget / lanes. */
int tpc_server_create(const tpc_geometry *geometry, float bz_tesla, const tpc_params *params,
                      const tpc_server_config *config, tpc_server **out);

/* Queue one event: y, z, row are HOST arrays of n clusters (page-locked memory makes the copy
 * asynchronous) that must stay valid until the event is reported done; counts is a host array
 * of n_sectors * n_rows entries (copied).  *id receives the event's id.  Errors:
 * TPC_ERR_BUDGET if n > lane_clusters, TPC_ERR_INVALID_ARG if the counts do not sum to n. */
int tpc_server_submit(tpc_server *server, const float *y, const float *z, const uint8_t *row,
                      const int32_t *counts, int64_t n, int64_t *id);

/* Ids of events finished since the last call (at most max_ids; *n_done receives the count). */
int tpc_server_poll(tpc_server *server, int64_t *ids, int max_ids, int *n_done);

/* Result of a finished event (TPC_ERR_STATE if it is not finished yet). */
int tpc_server_get(tpc_server *server, int64_t id, tpc_server_result *out);

/* Free a finished event's result. */
int tpc_server_release(tpc_server *server, int64_t id);

/* The server's steady clock in nanoseconds. */
int64_t tpc_server_now_ns(void);

/* Finish the queued events, then free everything. */
void tpc_server_destroy(tpc_server *server);

#ifdef __cplusplus
}
#endif
#endif
