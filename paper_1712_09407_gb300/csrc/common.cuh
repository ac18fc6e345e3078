// Internal definitions shared by the kernels and the host side of the tracker library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct tpc_tracker;

namespace tpc {

constexpr int kMaxRows = 255;       // row index is a uint8
constexpr int kMaxSectors = 36;
constexpr int kCellMax = 1024;      // grid cells per row unit (host clamps)
constexpr int kSlotAlign = 8;       // sorted row segments start on 8-element (32 B) boundaries
constexpr int kCellAlign = 4;       // cell-start segments start on 16 B boundaries
constexpr unsigned kFull = 0xffffffffu;
constexpr int kOrderCursors = 6144; // buckets of the constructor's grouped order, at least one group of
                                    // 2 kMaxRows + 2 expected-work keys (the scatter holds two arrays
                                    // of them in 48 KB of shared memory); cursors follow them

// Error word layout in the workspace: [0] status, [1] event, [2] sector, [3] stage.
enum { ERR_STATUS = 0, ERR_EVENT = 1, ERR_SECTOR = 2, ERR_STAGE = 3 };

// Counters in the workspace.
enum {
    CNT_STARTS = 0,     // tracklets found by A4
    CNT_QUEUE = 1,      // A5 work-queue head
    CNT_TRACKS = 2,     // accepted tracks (A7)
    CNT_HITS = 3,       // output hits (A7)
    CNT_VISITS = 4,     // A5 row visits (statistics)
    CNT_CANDS = 5,      // A5 clusters read inside the enumerated grid cells (statistics)
    CNT_SW_CHUNKS = 6,  // chunks of the sector-sweep constructor
    CNT_GPOOL = 7,      // global tracking: entries appended to the prolongation pool
    CNT_GLIST = 8,      // global tracking: prolongations of the call (2 per tracklet)
    CNT_STRACKS = 9,    // merger: sector tracks (CNT_TRACKS then counts the merged tracks)
    CNT_SHITS = 10,     // merger: clusters of the sector tracks
    CNT_GEDGE = 11,     // global tracking: prolongations past the edge test
    CNT_TLHITS = 12,    // A6: clusters of the tracklets that claim (statistics)
    CNT_COUNT = 13
};

// Constants of one tracker, passed by value to every kernel (kernel parameter space).
struct DevConst {
    float row_x[kMaxRows + 1];
    float sec_alpha[kMaxSectors];
    int nr;             // rows
    int ns;             // sectors per event
    float th;           // tan of the sector half-opening
    float margin;       // edge margin of the construction
    float smax;         // |sin phi| limit
    float sy2, sz2;     // sigma_y^2, sigma_z^2
    float isy2, isz2;   // 1 / sigma^2
    float ty, tz;       // neighbours window slopes
    float gate9;        // neighbours gate factor
    float cov0[5];      // seed covariance diagonal
    float nsig;         // search window in sigmas
    float chi2max;      // cluster gate
    float alpha, beta;  // cluster weight constants
    float qptmax;       // low-momentum cut
    float kB;           // curvature per unit q/pT: -kappa * Bz
    int max_miss;
    int min_chain;
    int min_clusters;
    int inject;         // host-side test hook (0 = off): 1 makes one bounded wait of the neighbours finder expire
    int global;         // global tracking on (Section 5)
    float c20, s20;     // cos, sin of the 20 degree sector pitch
    int merge;          // track merger with refit
    float crot[18], srot[18];   // cos, sin of d * 20 degrees (d = 0..17, read as -160..180)
    float mchi2, mgap, mq2;     // merger gates: chi2, radial gap, (q/pT sigmas)^2
};

struct OutBuffers {
    float *par, *cov, *x, *alpha, *chi2;
    int32_t *ndf, *nhits, *first, *sector, *event, *hits;
    int64_t mcap, hcap;    // tracks and hits the buffers hold
};

// Per row unit metadata (host-computed): input offset, count, sorted offset, cell offset.
// A row unit is one pad row of one sector of one event: u = (event * ns + sector) * nr + row.
struct Workspace {
    // per row unit
    int4 *meta;            // {in_off, n, s_off, cell_off}
    int2 *dims;            // {ny, nz}
    float4 *grid;          // {ymin, zmin, 1/dy, 1/dz}
    int4 *rgi;             // {s_off, cell_off, ny, nz}: what a row search needs, in one 16 B load
    int32_t *cell;         // cell starts relative to the row's first slot
    // per cluster slot (sorted order, padded per row unit)
    float2 *yz;
    int32_t *orig;
    int32_t *up_raw, *dn_raw, *up, *dn;
    unsigned long long *ckey;   // A6 claims
    // per tracklet
    int4 *starts;          // {first, -1, -1, (sector << 16) | (chain length up to max(4, min_chain) << 8) | row}
    int32_t *order;        // tracklets in the order the sweep constructor takes them
    float4 *seeds;         // [2 * tcap] per work-queue position: {p0, p1, p2, p3}, {p4, tracklet (-1 - t if
                           // the seed failed), packed start word, input index of the start cluster}
    int32_t *buckets;      // [2 * kOrderCursors] histogram / cursors of the ordering sort
    int32_t *sw_sec;       // [2 * sectors] tracklets per sector, scatter cursors (sweep constructor)
    int4 *sw_chunks;       // {sector, first position in order, count, 0} per chunk (sweep constructor)
    int32_t *tl_n;
    int32_t *tl_hits;      // [tcap * nr]
    float *tl_par;         // [5 * tcap]
    float *tl_cov;         // [15 * tcap]
    float *tl_x, *tl_chi2, *tl_w;
    unsigned long long *tl_key;
    int32_t *tl_nowned;
    uint32_t *tl_own;      // [tcap * ((nr + 31) / 32)] bit i of word i / 32: the tracklet owns its hit i
    int32_t *tl_inner;     // input index of the innermost owned cluster, -1 if rejected
    // global tracking (Section 5)
    float *tl_opar, *tl_ocov, *tl_ox;   // outward pass's state at its last cluster [5|15|1][tcap]
    uint8_t *used;         // [slots] cluster of an accepted track
    unsigned long long *gkey;   // [slots] prolongation claims
    int4 *gent;            // [gpool_cap] unordered pool: {slot, prolongation, position in it, 0}
    int32_t *gpool;        // [gpool_cap] clusters found, per prolongation in search order at g_off
    int64_t gpool_cap;
    int32_t *g_off, *g_n, *g_own;       // [2 * tcap] per prolongation p = 2 * tracklet + (0 in, 1 out)
    float *g_chi;          // [2 * tcap]
    float *g_par, *g_cov, *g_x;         // inward prolongation's last state [5|15|1][tcap]
    int32_t *g_sec;        // [tcap] sector (within the event) of that state
    int32_t *g_list;       // [2 * tcap] prolongations past the edge test
    // track merger
    int32_t *in_sec;       // [input clusters] sector (index within the call)
    OutBuffers st;         // sector tracks (A7 output) when the merger runs after them
    int32_t *rf_ok, *rf_sin, *rf_sout;  // [tcap] refit of every sector track
    float *rf_P, *rf_C, *rf_oP, *rf_oC; // [5|15][tcap] states at the innermost / outermost cluster
    float *rf_xin, *rf_xout, *rf_rin, *rf_rout, *rf_chi2;
    int32_t *mg_sec_cnt, *mg_sec_first, *mg_sec_cur;   // [sectors + 1] tracks per inner sector
    int32_t *mg_by_sec;    // [tcap] tracks grouped by inner sector
    int32_t *mg_best, *mg_next, *mg_prev, *mg_head, *mg_cnt, *mg_idx, *mg_first;   // [tcap]
    unsigned long long *mg_bkey;        // [tcap] best outer end for every inner end
    int32_t *mg_nseg, *mg_headof;       // [tcap] per merged track
    // output ordering
    uint32_t *bits;        // bitmap over input indices of innermost clusters
    int32_t *word_off;     // exclusive prefix of popcounts
    int32_t *rank_trk;     // tracklet of each output rank
    int32_t *rank_first;   // hit offset of each output rank
    int32_t *scan_tmp;     // scratch for block partials
    int32_t *counters;     // [CNT_COUNT]
    int32_t *err;          // [4]
    int64_t ncap, pcap, ccap, tcap, rcap, wcap;
    int64_t tlim;          // tracklets that may be stored (<= tcap, the stride of the per-tracklet arrays)
};

// Number of tracklets of the current call that were stored.
__device__ __forceinline__ int n_tracklets(const Workspace &w)
{
    const int s = w.counters[CNT_STARTS];
    return s < (int)w.tlim ? s : (int)w.tlim;
}

// Device wall clock (ns) for waits bounded in time.
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t kWaitNs = 1000000000ull;   // every device wait gives up after 1 s

// --------------------------------------------------------------------------------------------
// device helpers
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void set_error(int32_t *err, int status, int unit, const DevConst &c, int stage)
{
    if (atomicCAS(&err[ERR_STATUS], 0, status) == 0) {
        int sec = unit / c.nr;
        err[ERR_EVENT] = sec / c.ns;
        err[ERR_SECTOR] = sec % c.ns;
        err[ERR_STAGE] = stage;
    }
}

// Index checks of the checked build (-DTPC_CHECKED, the library built next to the release one):
// an index outside its pool records TPC_ERR_CHECK with the stage and the access is skipped.  The
// release build compiles them to `true`.
#ifdef TPC_CHECKED
__device__ __forceinline__ bool idx_ok(int64_t i, int64_t n, int32_t *err, int stage)
{
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&err[ERR_STATUS], 0, 7) == 0) err[ERR_STAGE] = stage;
    return false;
}
#define TPC_IDX(i, n, err, c, stage) ::tpc::idx_ok((int64_t)(i), (int64_t)(n), (err), (stage))
#else
#define TPC_IDX(i, n, err, c, stage) true
#endif

// Monotone map of a float to an unsigned integer (larger float -> larger integer).
__device__ __forceinline__ uint32_t ordered_bits(float f)
{
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Claim key of global-tracking prolongation (t, d) (d = 0 inward, 1 outward): the track's weight,
// then the lower input index of its start cluster, then the inward end.
__device__ __forceinline__ unsigned long long prolong_key(const Workspace &w, int t, int d)
{
    const uint32_t hi = ordered_bits(w.tl_w[t]);
    const uint32_t o = (uint32_t)w.orig[w.starts[t].x];
    const uint32_t lo = ((0x7fffffffu - o) << 1) | (uint32_t)(1 - d);
    return ((unsigned long long)hi << 32) | lo;
}

// Grid cell along one axis; monotone non-decreasing in v.
__device__ __forceinline__ int cell1(float v, float vmin, float inv, int nb)
{
    float t = (v - vmin) * inv;
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)nb) return nb - 1;
    return (int)t;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive warp scan.
__device__ __forceinline__ int warp_incl_scan(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Bin range slack: windows are widened by this much (cm) before the cell lookup so
// that rounding can never hide a cluster that passes the exact window test.
constexpr float kBinSlack = 1e-3f;

}  // namespace tpc

// Launchers (host side), one per stage; defined next to their kernels.
namespace tpc {
struct LaunchCfg {
    int num_sms;
    int neighbours_block;
    int construct_block;
    int construct_ctas_per_sm;
    int construct_mode;        // 0: per-lane work queue, 1: sector sweep
    int stage_rows;
    int neighbours_smem_max;   // bytes of dynamic shared memory for staged rows
    int seed_kernel;           // -1: by the call's size, 0: seeds walked by the constructor, 1: k_seed
    int64_t n_clusters;        // clusters in the call
    int64_t n_slots;           // cluster slots in the call (rows padded)
    int64_t order_group;       // slots per group of the constructor's order (0: one group)
    int max_row_clusters;      // largest row unit of the call (the cooperative neighbours search packs
                               // row-relative input indices in 16 bits)
};
int launch_ingest(const DevConst &c, const Workspace &w, const float *y, const float *z, const uint8_t *row,
                   int64_t R, cudaStream_t s);
int launch_neighbours(const DevConst &c, const Workspace &w, int64_t R, int smem_bytes, const LaunchCfg &lc,
                       cudaStream_t s);
int launch_evolve(const DevConst &c, const Workspace &w, int64_t R, cudaStream_t s);
int launch_construct(const DevConst &c, const Workspace &w, const LaunchCfg &lc, cudaStream_t s);
int launch_construct_sweep(const DevConst &c, const Workspace &w, int n_sec, const LaunchCfg &lc, cudaStream_t s);
int launch_select(const DevConst &c, const Workspace &w, int64_t n_input, const LaunchCfg &lc, cudaStream_t s);
int launch_output(const DevConst &c, const Workspace &w, const OutBuffers &o, int64_t n_input,
                   const LaunchCfg &lc, cudaStream_t s);
int launch_global(const DevConst &c, const Workspace &w, int64_t n_slots, const LaunchCfg &lc, cudaStream_t s);
int launch_merge(const DevConst &c, const Workspace &w, const OutBuffers &o, const float *y, const float *z,
                 const uint8_t *row, int64_t R, const LaunchCfg &lc, cudaStream_t s);
// Exclusive scan of min(n, *n_dev) int32 values (n_dev may be null); total to *total_out if given.
// partials needs n / 4096 + 64 ints.  Returns the kernels launched.
int launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, const int32_t *n_dev, int32_t *partials,
                    int32_t *total_out, cudaStream_t s);
int neighbours_smem_limit();

// Read-only view of a tracker's constants for entry points defined outside api.cu.
struct TrackerInfo {
    const DevConst *dc;
    const float *row_x;
    int n_rows, n_sectors, num_sms;
    float tan_half, z_max;
    float bin_occupancy;
    int neighbours_block, stage_rows;
};
bool tracker_info(const struct ::tpc_tracker *tr, TrackerInfo *out);
}  // namespace tpc
