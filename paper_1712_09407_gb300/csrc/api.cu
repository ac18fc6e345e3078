// Host side of the C ABI declared in include/tpcca.h: tracker lifetime, device workspace,
// per-call staging and the stage launches, results.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "../../include/tpcca.h"

using namespace tpc;

namespace {
// NVTX range for the host side of a call (visible in nsys/ncu timelines; free when no tool listens).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

constexpr int kStaging = 24;            // ring of pinned staging buffers (calls of one tracker in flight)
constexpr int kCountWords = CNT_COUNT + 4;

struct Staging {
    int4 *meta = nullptr;
    int2 *dims = nullptr;
    int64_t cap = 0;
    cudaEvent_t consumed = nullptr;     // recorded after the H2D copy that reads this buffer
    bool pending = false;
};

struct Alloc {
    void *base = nullptr;
    size_t bytes = 0;
    size_t used = 0;
    template <class T>
    T *take(int64_t count)
    {
        size_t b = ((size_t)(count > 0 ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
        T *p = (T *)((char *)base + used);
        used += b;
        return p;
    }
};

}  // namespace

struct tpc_tracker {
    int device = 0;
    int num_sms = 0;
    DevConst dc{};
    tpc_params params{};
    tpc_tuning tuning{};
    int n_rows = 0, n_sectors = 0;
    float row_x[kMaxRows + 1]{};
    float tan_half = 0.0f, z_max = 0.0f;
    size_t budget = 0;
    size_t bytes_ws = 0, bytes_results = 0;
    // workspace
    void *ws_base = nullptr;
    Workspace w{};
    int64_t cap_n = -1, cap_units = -1;
    // device copy of host inputs for tpc_track_event_host
    void *in_base = nullptr;
    int64_t in_cap = 0;
    cudaEvent_t ws_done = nullptr;
    bool ws_used = false;
    Staging staging[kStaging];
    int next_staging = 0;
    std::vector<int4> meta;
    std::vector<int2> dims;
    std::vector<tpc_result *> free_results;   // released results, reused without new pinned allocations
    int64_t live_results = 0;                 // results handed out and not yet released
    // result ring (tpc_tracker_reserve_results): result buffers allocated once, reused call after call
    std::vector<tpc_result *> ring_free;      // ring results not held by the caller
    int ring_depth = 0;                       // ring size asked for (0: every call allocates its result)
    int ring_count = 0;                       // ring results in existence, free or held
    size_t bytes_ring = 0;
    bool destroyed = false;                   // tpc_tracker_destroy was called; delete at the last release
    // last call
    int64_t last_units = 0, last_slots = 0, last_n = 0;
    bool timing = false;
    int last_err[4] = {0, 0, 0, 0};
    // graph mode (tuning.use_graph)
    cudaStream_t cap_stream = nullptr;
    // copies of finished results to the host (tpc_result_copy_to_host): a stream of their own, so
    // that a copy waits only for its own call and not for the later calls queued on the call's
    // stream; created at the first copy, freed with the tracker object
    cudaStream_t copy_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_builds = 0;
    std::mutex mu;
};

struct tpc_result {
    tpc_tracker *tr = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    OutBuffers out{};
    int32_t *h_counts = nullptr;        // pinned: counters then error word
    bool synced = false;
    int status = TPC_OK;
    int64_t n_tracks = 0, n_hits = 0;
    int64_t n_clusters = 0;
    int launches = 0;
    int64_t graph_builds = 0;            // the tracker's graph instantiations up to this call
    bool timed = false;
    cudaEvent_t stage_ev[10] = {};
    // ring results only: device buffers sized once for cap_t tracks and cap_h hits; `reusable` is
    // recorded on the call's stream at release, and the next call using the buffers waits for it
    bool ring = false;
    int64_t cap_t = 0, cap_h = 0;
    cudaEvent_t reusable = nullptr;
    bool reuse_pending = false;
};

bool tpc::tracker_info(const tpc_tracker *tr, TrackerInfo *out)
{
    if (!tr || !out) return false;
    out->dc = &tr->dc;
    out->row_x = tr->row_x;
    out->n_rows = tr->n_rows;
    out->n_sectors = tr->n_sectors;
    out->num_sms = tr->num_sms;
    out->tan_half = tr->tan_half;
    out->z_max = tr->z_max;
    out->bin_occupancy = tr->tuning.bin_occupancy;
    out->neighbours_block = tr->tuning.neighbours_block;
    out->stage_rows = tr->tuning.stage_rows;
    return true;
}

static int cuda_fail(cudaError_t e)
{
    if (e != cudaSuccess) {
        fprintf(stderr, "tpcca: CUDA error %s\n", cudaGetErrorString(e));
        return TPC_ERR_CUDA;
    }
    return TPC_OK;
}

#define TPC_CUDA(x)                                      \
    do {                                                 \
        int _s = cuda_fail(x);                           \
        if (_s != TPC_OK) return _s;                     \
    } while (0)

extern "C" void tpc_params_default(tpc_params *p)
{
    if (!p) return;
    p->sigma_y = 0.08f;
    p->sigma_z = 0.1f;
    p->nb_ty = 1.0f;
    p->nb_tz = 2.0f;
    p->nb_gate = 9.0f;
    p->min_chain = 3;
    p->seed_cov[0] = (float)(0.08 * 0.08);
    p->seed_cov[1] = (float)(0.1 * 0.1);
    p->seed_cov[2] = 0.01f;
    p->seed_cov[3] = 0.01f;
    p->seed_cov[4] = 1.0f;
    p->win_nsigma = 3.0f;
    p->chi2_max = 16.0f;
    p->max_miss = 10;
    p->edge_margin = 2.0f;
    p->sin_max = 0.99f;
    p->alpha = 6.0f;            // Section 3.1
    p->beta = 1.0f;
    p->min_clusters = 30;       // Section 5
    p->qpt_max = 20.0f;
    p->global_tracking = 0;
    p->merge = 0;
    p->merge_chi2 = 25.0f;
    p->merge_gap = 40.0f;
    p->merge_qpt_nsigma = 5.0f;
}

extern "C" void tpc_tuning_default(tpc_tuning *t)
{
    if (!t) return;
    // picked by the autotuner on the central-like event on a GB300
    t->bin_occupancy = 0.5f;
    t->neighbours_block = 256;
    // constructor: 11 CTAs of 64 threads per SM, 22 of the 24 warps its registers allow, so that a
    // call in flight on another stream finds room during this call's queue drain (measured
    // streamed: 818 against 784 events/s with 6 CTAs of 128 threads)
    t->construct_block = 64;
    t->construct_ctas_per_sm = 11;
    t->construct_mode = 0;
    t->stage_rows = 1;
    t->tracklet_capacity = 0;
    t->use_graph = 1;
    // the seed launch and the pre-seeded constructor were as fast or faster on every workload measured
    // (one sector 0.82 -> 0.71 ms, one 36-sector 4000-track event 1.22 -> 1.20 ms per event)
    t->seed_kernel = 1;
    t->order_group = 3 << 20;
}

extern "C" const char *tpc_status_string(int s)
{
    switch (s) {
    case TPC_OK: return "ok";
    case TPC_ERR_INVALID_ARG: return "invalid argument";
    case TPC_ERR_CAPACITY: return "device pool capacity exceeded";
    case TPC_ERR_BUDGET: return "HBM budget exceeded";
    case TPC_ERR_TIMEOUT: return "bounded device wait expired";
    case TPC_ERR_CUDA: return "CUDA runtime error";
    case TPC_ERR_STATE: return "invalid call order";
    case TPC_ERR_CHECK: return "index bounds check failed (checked build)";
    default: return "unknown status";
    }
}

static void fill_const(tpc_tracker *tr, float bz)
{
    DevConst &c = tr->dc;
    const tpc_params &p = tr->params;
    memset(&c, 0, sizeof c);
    for (int r = 0; r < tr->n_rows; r++) c.row_x[r] = tr->row_x[r];
    for (int s = 0; s < tr->n_sectors; s++)
        c.sec_alpha[s] = (float)((20.0 * (s % 18) + 10.0) * M_PI / 180.0);
    c.nr = tr->n_rows;
    c.ns = tr->n_sectors;
    c.th = tr->tan_half;
    c.margin = p.edge_margin;
    c.smax = p.sin_max;
    c.sy2 = p.sigma_y * p.sigma_y;
    c.sz2 = p.sigma_z * p.sigma_z;
    c.isy2 = 1.0f / c.sy2;
    c.isz2 = 1.0f / c.sz2;
    c.ty = p.nb_ty;
    c.tz = p.nb_tz;
    c.gate9 = p.nb_gate;
    for (int i = 0; i < 5; i++) c.cov0[i] = p.seed_cov[i];
    c.nsig = p.win_nsigma;
    c.chi2max = p.chi2_max;
    c.alpha = p.alpha;
    c.beta = p.beta;
    c.qptmax = p.qpt_max;
    c.kB = (float)(-2.99792458e-3 * (double)bz);
    c.max_miss = p.max_miss;
    c.min_chain = p.min_chain;
    c.min_clusters = p.min_clusters;
    c.global = (p.global_tracking && tr->n_sectors == 36) ? 1 : 0;
    c.c20 = (float)std::cos(20.0 * 3.14159265358979323846 / 180.0);
    c.s20 = (float)std::sin(20.0 * 3.14159265358979323846 / 180.0);
    c.merge = (p.merge && tr->n_sectors == 36) ? 1 : 0;
    for (int d = 0; d < 18; d++) {
        const int deg = d <= 9 ? 20 * d : 20 * (d - 18);     // -160 .. 180
        const double a = (double)(deg < 0 ? -deg : deg) * 3.14159265358979323846 / 180.0;
        c.crot[d] = (float)std::cos(a);
        c.srot[d] = deg < 0 ? -(float)std::sin(a) : (float)std::sin(a);
    }
    c.mchi2 = p.merge_chi2;
    c.mgap = p.merge_gap;
    c.mq2 = (float)((double)p.merge_qpt_nsigma * (double)p.merge_qpt_nsigma);
}

extern "C" int tpc_tracker_create(const tpc_geometry *g, float bz, const tpc_params *params, size_t budget,
                                  tpc_tracker **out)
{
    if (!out || !g || !g->row_x) return TPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (g->n_rows < 3 || g->n_rows > kMaxRows) return TPC_ERR_INVALID_ARG;
    if (g->n_sectors != 1 && g->n_sectors != 36) return TPC_ERR_INVALID_ARG;
    for (int r = 1; r < g->n_rows; r++)
        if (!(g->row_x[r] > g->row_x[r - 1])) return TPC_ERR_INVALID_ARG;
    tpc_tracker *tr = new (std::nothrow) tpc_tracker();
    if (!tr) return TPC_ERR_CUDA;
    if (cudaGetDevice(&tr->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&tr->num_sms, cudaDevAttrMultiProcessorCount, tr->device) != cudaSuccess) {
        delete tr;
        return TPC_ERR_CUDA;
    }
    tr->n_rows = g->n_rows;
    tr->n_sectors = g->n_sectors;
    memcpy(tr->row_x, g->row_x, sizeof(float) * g->n_rows);
    tr->tan_half = g->tan_half;
    tr->z_max = g->z_max;
    tr->budget = budget;
    if (params)
        tr->params = *params;
    else
        tpc_params_default(&tr->params);
    tpc_tuning_default(&tr->tuning);
    fill_const(tr, bz);
    if (cudaEventCreateWithFlags(&tr->ws_done, cudaEventDisableTiming) != cudaSuccess) {
        delete tr;
        return TPC_ERR_CUDA;
    }
    for (auto &s : tr->staging) cudaEventCreateWithFlags(&s.consumed, cudaEventDisableTiming);
    // keep freed result memory in the stream-ordered pool instead of returning it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, tr->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = tr;
    return TPC_OK;
}

extern "C" int tpc_tracker_set_tuning(tpc_tracker *tr, const tpc_tuning *t)
{
    if (!tr || !t) return TPC_ERR_INVALID_ARG;
    if (!(t->bin_occupancy >= 0.5f) || t->neighbours_block < 32 || t->neighbours_block > 256 ||
        t->neighbours_block % 32 || t->construct_block < 32 || t->construct_block > 128 ||
        t->construct_block % 32 || t->construct_ctas_per_sm < 0 || t->construct_mode < 0 || t->construct_mode > 1 ||
        t->stage_rows < 0 || t->stage_rows > 2 ||
        t->tracklet_capacity < 0 || t->use_graph < 0 || t->use_graph > 1 || t->seed_kernel < -1 ||
        t->seed_kernel > 1 || t->order_group < 0)
        return TPC_ERR_INVALID_ARG;
    tr->tuning = *t;
    return TPC_OK;
}

// Sizes of the workspace for n clusters in `events` events.
struct WsSizes {
    int64_t R, P, C, T, W;
};

static WsSizes ws_sizes(const tpc_tracker *tr, int64_t n, int64_t events)
{
    WsSizes s;
    s.R = events * tr->n_sectors * tr->n_rows;
    s.P = n + s.R * kSlotAlign + 64;
    s.C = (int64_t)std::ceil((double)n / 0.5) + s.R * (kCellAlign + 1) + 64;
    s.T = n / 4 + 64;
    s.W = n / 32 + 4;
    return s;
}

static size_t carve(tpc_tracker *tr, const WsSizes &s, Alloc &a)
{
    Workspace &w = tr->w;
    w.meta = a.take<int4>(s.R);
    w.dims = a.take<int2>(s.R);
    w.grid = a.take<float4>(s.R);
    w.rgi = a.take<int4>(s.R);
    w.cell = a.take<int32_t>(s.C);
    w.yz = a.take<float2>(s.P);
    w.orig = a.take<int32_t>(s.P);
    w.up_raw = a.take<int32_t>(s.P);
    w.dn_raw = a.take<int32_t>(s.P);
    w.up = a.take<int32_t>(s.P);
    w.dn = a.take<int32_t>(s.P);
    w.ckey = a.take<unsigned long long>(s.P);
    w.starts = a.take<int4>(s.T);
    w.order = a.take<int32_t>(s.T);
    w.seeds = a.take<float4>(2 * s.T);
    w.buckets = a.take<int32_t>(2 * kOrderCursors);
    w.sw_sec = a.take<int32_t>(2 * (s.R / tr->n_rows) + 64);
    w.sw_chunks = a.take<int4>(s.T / 32 + s.R / tr->n_rows + 64);
    w.tl_n = a.take<int32_t>(s.T);
    w.tl_hits = a.take<int32_t>(s.T * tr->n_rows);
    w.tl_par = a.take<float>(5 * s.T);
    w.tl_cov = a.take<float>(15 * s.T);
    w.tl_x = a.take<float>(s.T);
    w.tl_chi2 = a.take<float>(s.T);
    w.tl_w = a.take<float>(s.T);
    w.tl_key = a.take<unsigned long long>(s.T);
    w.tl_nowned = a.take<int32_t>(s.T);
    w.tl_own = a.take<uint32_t>(s.T * ((tr->n_rows + 31) / 32));
    w.tl_inner = a.take<int32_t>(s.T);
    if (tr->dc.global) {
        w.tl_opar = a.take<float>(5 * s.T);
        w.tl_ocov = a.take<float>(15 * s.T);
        w.tl_ox = a.take<float>(s.T);
        w.used = a.take<uint8_t>(s.P);
        w.gkey = a.take<unsigned long long>(s.P);
        w.gent = a.take<int4>(s.P);
        w.gpool = a.take<int32_t>(s.P);
        w.gpool_cap = s.P;
        w.g_off = a.take<int32_t>(2 * s.T);
        w.g_n = a.take<int32_t>(2 * s.T);
        w.g_own = a.take<int32_t>(2 * s.T);
        w.g_chi = a.take<float>(2 * s.T);
        w.g_par = a.take<float>(5 * s.T);
        w.g_cov = a.take<float>(15 * s.T);
        w.g_x = a.take<float>(s.T);
        w.g_sec = a.take<int32_t>(s.T);
        w.g_list = a.take<int32_t>(2 * s.T);
    } else {
        w.tl_opar = w.tl_ocov = w.tl_ox = w.g_chi = w.g_par = w.g_cov = w.g_x = nullptr;
        w.used = nullptr;
        w.gkey = nullptr;
        w.gent = nullptr;
        w.gpool = w.g_off = w.g_n = w.g_own = w.g_sec = w.g_list = nullptr;
        w.gpool_cap = 0;
    }
    if (tr->dc.merge) {
        const int64_t S = s.R / tr->n_rows + 2;
        w.in_sec = a.take<int32_t>(s.P);
        w.st.par = a.take<float>(5 * s.T);
        w.st.cov = a.take<float>(15 * s.T);
        w.st.x = a.take<float>(s.T);
        w.st.alpha = a.take<float>(s.T);
        w.st.chi2 = a.take<float>(s.T);
        w.st.ndf = a.take<int32_t>(s.T);
        w.st.nhits = a.take<int32_t>(s.T);
        w.st.first = a.take<int32_t>(s.T);
        w.st.sector = a.take<int32_t>(s.T);
        w.st.event = a.take<int32_t>(s.T);
        w.st.hits = a.take<int32_t>(s.P);
        w.st.mcap = s.T;
        w.st.hcap = s.P;
        w.rf_ok = a.take<int32_t>(s.T);
        w.rf_sin = a.take<int32_t>(s.T);
        w.rf_sout = a.take<int32_t>(s.T);
        w.rf_P = a.take<float>(5 * s.T);
        w.rf_C = a.take<float>(15 * s.T);
        w.rf_oP = a.take<float>(5 * s.T);
        w.rf_oC = a.take<float>(15 * s.T);
        w.rf_xin = a.take<float>(s.T);
        w.rf_xout = a.take<float>(s.T);
        w.rf_rin = a.take<float>(s.T);
        w.rf_rout = a.take<float>(s.T);
        w.rf_chi2 = a.take<float>(s.T);
        w.mg_sec_cnt = a.take<int32_t>(S);
        w.mg_sec_first = a.take<int32_t>(S);
        w.mg_sec_cur = a.take<int32_t>(S);
        w.mg_by_sec = a.take<int32_t>(s.T);
        w.mg_best = a.take<int32_t>(s.T);
        w.mg_next = a.take<int32_t>(s.T);
        w.mg_prev = a.take<int32_t>(s.T);
        w.mg_head = a.take<int32_t>(s.T);
        w.mg_cnt = a.take<int32_t>(s.T);
        w.mg_idx = a.take<int32_t>(s.T);
        w.mg_first = a.take<int32_t>(s.T);
        w.mg_bkey = a.take<unsigned long long>(s.T);
        w.mg_nseg = a.take<int32_t>(s.T);
        w.mg_headof = a.take<int32_t>(s.T);
    }
    w.bits = a.take<uint32_t>(s.W);
    w.word_off = a.take<int32_t>(s.W);
    w.rank_trk = a.take<int32_t>(s.T);
    w.rank_first = a.take<int32_t>(s.T);
    w.scan_tmp = a.take<int32_t>((s.W > 2 * s.T ? s.W : 2 * s.T) / 4096 + 64);
    w.counters = a.take<int32_t>(kCountWords);
    w.err = w.counters + CNT_COUNT;
    w.ncap = s.P;
    w.pcap = s.P;
    w.ccap = s.C;
    w.tcap = s.T;
    w.tlim = s.T;
    w.rcap = s.R;
    w.wcap = s.W;
    return a.used;
}

static void destroy_result(tpc_result *r);

static int reserve(tpc_tracker *tr, int64_t n, int64_t events)
{
    if (n <= tr->cap_n && events <= tr->cap_units) return TPC_OK;
    int64_t nn = n > tr->cap_n ? n : tr->cap_n;
    int64_t ee = events > tr->cap_units ? events : tr->cap_units;
    if (nn < 1024) nn = 1024;
    if (ee < 1) ee = 1;
    WsSizes s = ws_sizes(tr, nn, ee);
    Alloc probe;              // dry run on a null base to get the size
    Workspace keep = tr->w;
    size_t need = carve(tr, s, probe);
    tr->w = keep;
    if (tr->budget && need + tr->bytes_results + tr->bytes_ring > tr->budget) return TPC_ERR_BUDGET;
    if (tr->ws_base) {
        TPC_CUDA(cudaDeviceSynchronize());
        cudaFree(tr->ws_base);
        tr->ws_base = nullptr;
        tr->bytes_ws = 0;
    }
    TPC_CUDA(cudaMalloc(&tr->ws_base, need));
    Alloc a;
    a.base = tr->ws_base;
    a.bytes = need;
    carve(tr, s, a);
    tr->bytes_ws = need;
    tr->cap_n = nn;
    tr->cap_units = ee;
    return TPC_OK;
}

// Pinned host staging of the per-unit metadata for calls of up to R row units: every buffer of
// the ring, so that no call allocates pinned memory later.
static int reserve_staging(tpc_tracker *tr, int64_t R)
{
    for (auto &sg : tr->staging) {
        if (sg.cap >= R) continue;
        if (sg.pending) {
            TPC_CUDA(cudaEventSynchronize(sg.consumed));
            sg.pending = false;
        }
        if (sg.meta) cudaFreeHost(sg.meta);
        if (sg.dims) cudaFreeHost(sg.dims);
        sg.meta = nullptr;
        sg.dims = nullptr;
        sg.cap = 0;
        const int64_t cap = R < 1 ? 1 : R;
        TPC_CUDA(cudaMallocHost((void **)&sg.meta, cap * sizeof(int4)));
        TPC_CUDA(cudaMallocHost((void **)&sg.dims, cap * sizeof(int2)));
        sg.cap = cap;
    }
    return TPC_OK;
}

extern "C" int tpc_tracker_reserve(tpc_tracker *tr, int64_t max_clusters, int max_events)
{
    if (!tr || max_clusters < 0 || max_events < 1) return TPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(tr->mu);
    const int s = reserve(tr, max_clusters, max_events);
    if (s != TPC_OK) return s;
    return reserve_staging(tr, (int64_t)max_events * tr->n_sectors * tr->n_rows);
}

static size_t result_bytes(int64_t tcap, int64_t ncap)
{
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add(tcap * 5 * 4);
    add(tcap * 15 * 4);
    for (int i = 0; i < 3; i++) add(tcap * 4);
    for (int i = 0; i < 5; i++) add(tcap * 4);
    add((ncap > 0 ? ncap : 1) * 4);
    return b;
}

static void carve_result(tpc_result *r, int64_t tcap, int64_t ncap)
{
    Alloc a;
    a.base = r->dev;
    r->out.par = a.take<float>(tcap * 5);
    r->out.cov = a.take<float>(tcap * 15);
    r->out.x = a.take<float>(tcap);
    r->out.alpha = a.take<float>(tcap);
    r->out.chi2 = a.take<float>(tcap);
    r->out.ndf = a.take<int32_t>(tcap);
    r->out.nhits = a.take<int32_t>(tcap);
    r->out.first = a.take<int32_t>(tcap);
    r->out.sector = a.take<int32_t>(tcap);
    r->out.event = a.take<int32_t>(tcap);
    r->out.hits = a.take<int32_t>(ncap > 0 ? ncap : 1);
    r->out.mcap = tcap;
    r->out.hcap = ncap;
}

// Result capacities of a call of n clusters: tracks <= tracklets <= n / min_chain (chains of
// one-to-one links are disjoint) and the tracklet pool; hits <= n.
static void result_caps(const tpc_tracker *tr, int64_t n, int64_t *tcap, int64_t *hcap)
{
    const int64_t tbound = n / (tr->params.min_chain > 0 ? tr->params.min_chain : 1) + 64;
    *tcap = tr->w.tcap < tbound ? tr->w.tcap : tbound;
    *hcap = n;
}

// (Re)size a ring result's device buffers for tcap tracks and hcap hits.  The result is free: its
// last call has finished (released after tpc_result_sync_counts' wait) and its reusable event
// is waited for before the old buffers go.
static int ring_size(tpc_tracker *tr, tpc_result *r, int64_t tcap, int64_t hcap)
{
    const size_t bytes = result_bytes(tcap, hcap);
    const size_t old = r->dev ? r->bytes : 0;
    if (tr->budget && tr->bytes_ws + tr->bytes_results + tr->bytes_ring - old + bytes > tr->budget)
        return TPC_ERR_BUDGET;
    if (r->dev) {
        if (r->reuse_pending) TPC_CUDA(cudaEventSynchronize(r->reusable));
        r->reuse_pending = false;
        cudaFree(r->dev);
        r->dev = nullptr;
        tr->bytes_ring -= old;
        r->bytes = 0;
    }
    TPC_CUDA(cudaMalloc(&r->dev, bytes));
    r->bytes = bytes;
    r->cap_t = tcap;
    r->cap_h = hcap;
    tr->bytes_ring += bytes;
    return TPC_OK;
}

// A new ring result with its pinned counters and events, buffers sized for the reserved workspace.
static int ring_add(tpc_tracker *tr)
{
    tpc_result *r = new (std::nothrow) tpc_result();
    if (!r) return TPC_ERR_CUDA;
    r->ring = true;
    r->tr = tr;
    int64_t tcap, hcap;
    result_caps(tr, tr->cap_n, &tcap, &hcap);
    int s = TPC_OK;
    if (cudaMallocHost((void **)&r->h_counts, kCountWords * sizeof(int32_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->reusable, cudaEventDisableTiming) != cudaSuccess)
        s = TPC_ERR_CUDA;
    for (auto &e : r->stage_ev)
        if (s == TPC_OK && cudaEventCreate(&e) != cudaSuccess) s = TPC_ERR_CUDA;
    if (s == TPC_OK) s = ring_size(tr, r, tcap, hcap);
    if (s != TPC_OK) {
        destroy_result(r);
        return s;
    }
    tr->ring_free.push_back(r);
    tr->ring_count++;
    return TPC_OK;
}

// Free a ring result that no call uses any more.
static void ring_drop(tpc_tracker *tr, tpc_result *r)
{
    if (r->reuse_pending) cudaEventSynchronize(r->reusable);
    if (r->dev) cudaFree(r->dev);
    r->dev = nullptr;
    tr->bytes_ring -= r->bytes;
    r->bytes = 0;
    tr->ring_count--;
    destroy_result(r);
}

extern "C" int tpc_tracker_reserve_results(tpc_tracker *tr, int depth)
{
    if (!tr || depth < 0 || depth > 4096) return TPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(tr->mu);
    if (tr->destroyed) return TPC_ERR_STATE;
    if (depth > 0 && tr->cap_n < 0) return TPC_ERR_STATE;     // sized from tpc_tracker_reserve's workspace
    tr->ring_depth = depth;
    while (tr->ring_count > depth && !tr->ring_free.empty()) {
        tpc_result *r = tr->ring_free.back();
        tr->ring_free.pop_back();
        ring_drop(tr, r);
    }
    while (tr->ring_count < depth) {
        const int s = ring_add(tr);
        if (s != TPC_OK) return s;
    }
    return TPC_OK;
}

// A result handed back unused (the call failed before its work was enqueued).
static void give_back(tpc_tracker *tr, tpc_result *r, cudaStream_t st)
{
    if (r->ring) {
        tr->ring_free.push_back(r);
        return;
    }
    if (r->dev) {
        cudaFreeAsync(r->dev, st);
        tr->bytes_results -= r->bytes;
    }
    r->dev = nullptr;
    r->bytes = 0;
    tr->free_results.push_back(r);
}

static int run(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row, const int32_t *counts,
               int n_events, int64_t n_total, cudaStream_t st, tpc_result **out)
{
    const int nr = tr->n_rows, ns = tr->n_sectors;
    const int64_t R = (int64_t)n_events * ns * nr;
    // host validation of counts
    int64_t sum = 0;
    for (int64_t u = 0; u < R; u++) {
        if (counts[u] < 0) return TPC_ERR_INVALID_ARG;
        sum += counts[u];
    }
    if (sum != n_total || n_total > INT32_MAX / 2) return TPC_ERR_INVALID_ARG;
    if ((int64_t)n_events * ns >= (1 << 15)) return TPC_ERR_INVALID_ARG;   // sector index packs into 15 bits
    if (n_total > 0 && (!y || !z || !row)) return TPC_ERR_INVALID_ARG;
    int s = reserve(tr, n_total, n_events);
    if (s != TPC_OK) return s;
    int64_t tcap, hcap;
    result_caps(tr, n_total, &tcap, &hcap);
    tpc_result *res = nullptr;
    if (tr->ring_depth > 0) {
        // preallocated result: the call allocates nothing; all ring results held -> not admitted
        if (tr->ring_free.empty()) return TPC_ERR_BUDGET;
        res = tr->ring_free.back();
        tr->ring_free.pop_back();
        if (res->cap_t < tcap || res->cap_h < hcap) {
            // the workspace grew since the ring was sized: this buffer grows with it (synchronous)
            int64_t rt, rh;
            result_caps(tr, tr->cap_n, &rt, &rh);
            s = ring_size(tr, res, rt > tcap ? rt : tcap, rh > hcap ? rh : hcap);
            if (s != TPC_OK) {
                tr->ring_free.push_back(res);
                return s;
            }
        }
        if (res->reuse_pending) {
            s = cuda_fail(cudaStreamWaitEvent(st, res->reusable, 0));
            if (s != TPC_OK) {
                tr->ring_free.push_back(res);
                return s;
            }
            res->reuse_pending = false;
        }
        res->synced = false;
        res->status = TPC_OK;
        res->n_tracks = res->n_hits = res->n_clusters = 0;
        res->launches = 0;
        res->timed = false;
        res->stream = st;
        carve_result(res, res->cap_t, res->cap_h);
    } else {
        // result object: reuse a released one (its pinned count buffer and events) when possible
        if (!tr->free_results.empty()) {
            res = tr->free_results.back();
            tr->free_results.pop_back();
            cudaEvent_t keep_done = res->done;
            int32_t *keep_counts = res->h_counts;
            cudaEvent_t keep_ev[10];
            memcpy(keep_ev, res->stage_ev, sizeof keep_ev);
            *res = tpc_result();
            res->done = keep_done;
            res->h_counts = keep_counts;
            memcpy(res->stage_ev, keep_ev, sizeof keep_ev);
        } else {
            res = new (std::nothrow) tpc_result();
            if (!res) return TPC_ERR_CUDA;
        }
        res->tr = tr;
        res->stream = st;
        res->bytes = result_bytes(tcap, hcap);
        if (tr->budget && tr->bytes_ws + tr->bytes_ring + tr->bytes_results + res->bytes > tr->budget) {
            tr->free_results.push_back(res);
            return TPC_ERR_BUDGET;
        }
        if (cudaMallocAsync(&res->dev, res->bytes, st) != cudaSuccess ||
            (!res->h_counts && cudaMallocHost((void **)&res->h_counts, kCountWords * sizeof(int32_t)) != cudaSuccess) ||
            (!res->done && cudaEventCreateWithFlags(&res->done, cudaEventDisableTiming) != cudaSuccess)) {
            if (res->dev) cudaFreeAsync(res->dev, st);
            res->dev = nullptr;
            destroy_result(res);
            return TPC_ERR_CUDA;
        }
        tr->bytes_results += res->bytes;
        carve_result(res, tcap, hcap);
    }
    // from here on a failure hands the result back
    struct Guard {
        tpc_tracker *tr;
        tpc_result *r;
        cudaStream_t st;
        bool armed = true;
        ~Guard()
        {
            if (armed) give_back(tr, r, st);
        }
    } guard{tr, res, st};
    // per row unit metadata
    tr->meta.resize(R);
    tr->dims.resize(R);
    int64_t in_off = 0, s_off = 0, c_off = 0;
    int smem_need = 0, max_row = 0;
    const float occ = tr->tuning.bin_occupancy;
    for (int64_t u = 0; u < R; u++) {
        const int n = counts[u];
        const int r = (int)(u % nr);
        int ncell = (int)std::ceil((double)n / occ);
        if (ncell < 1) ncell = 1;
        if (ncell > kCellMax) ncell = kCellMax;
        const double wy = 2.0 * tr->row_x[r] * tr->tan_half;
        const double wz = (ns == 36 ? 1.0 : 2.0) * tr->z_max;
        int ny = (int)std::lround(std::sqrt(ncell * wy / wz));
        if (ny < 1) ny = 1;
        if (ny > ncell) ny = ncell;
        int nz = ncell / ny;
        if (nz < 1) nz = 1;
        tr->meta[u] = make_int4((int)in_off, n, (int)s_off, (int)c_off);
        tr->dims[u] = make_int2(ny, nz);
        if (n > max_row) max_row = n;
        in_off += n;
        s_off += (n + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
        c_off += (ny * nz + 1 + kCellAlign - 1) / kCellAlign * kCellAlign;
    }
    for (int64_t u = 0; u < R; u++) {
        const int r = (int)(u % nr);
        if (r == 0 || r == nr - 1) continue;
        const int4 a = tr->meta[u + 1], b = tr->meta[u - 1];
        const int2 da = tr->dims[u + 1], db = tr->dims[u - 1];
        auto rb = [](int n, int nc) {
            auto r16 = [](int x) { return (x + 15) & ~15; };
            return r16(n * 8) + r16(n * 4) + r16((nc + 1) * 4);
        };
        const int bytes = rb(a.y, da.x * da.y) + rb(b.y, db.x * db.y);
        if (bytes > smem_need) smem_need = bytes;
    }
    if (s_off + 64 > tr->w.pcap || c_off + 64 > tr->w.ccap) return TPC_ERR_CAPACITY;   // cannot happen with ws_sizes' bounds
    int smem = smem_need < neighbours_smem_limit() ? smem_need : neighbours_smem_limit();

    Staging &sg = tr->staging[tr->next_staging];
    tr->next_staging = (tr->next_staging + 1) % kStaging;
    if (sg.pending) {
        TPC_CUDA(cudaEventSynchronize(sg.consumed));
        sg.pending = false;
    }
    if (sg.cap < R) {
        if (sg.meta) cudaFreeHost(sg.meta);
        if (sg.dims) cudaFreeHost(sg.dims);
        sg.meta = nullptr;
        sg.dims = nullptr;
        int64_t cap = R < 1 ? 1 : R;
        TPC_CUDA(cudaMallocHost((void **)&sg.meta, cap * sizeof(int4)));
        TPC_CUDA(cudaMallocHost((void **)&sg.dims, cap * sizeof(int2)));
        sg.cap = cap;
    }
    memcpy(sg.meta, tr->meta.data(), R * sizeof(int4));
    memcpy(sg.dims, tr->dims.data(), R * sizeof(int2));

    if (tr->ws_used) TPC_CUDA(cudaStreamWaitEvent(st, tr->ws_done, 0));
    const bool timed = tr->timing;
    if (timed) {
        for (auto &e : res->stage_ev)
            if (!e) TPC_CUDA(cudaEventCreate(&e));
        TPC_CUDA(cudaEventRecord(res->stage_ev[0], st));
    }
    res->timed = timed;
    res->n_clusters = n_total;
    Workspace wk = tr->w;
    if (tr->tuning.tracklet_capacity > 0 && tr->tuning.tracklet_capacity < wk.tcap) wk.tlim = tr->tuning.tracklet_capacity;
    const Workspace &w = wk;

    LaunchCfg lc;
    lc.num_sms = tr->num_sms;
    lc.neighbours_block = tr->tuning.neighbours_block;
    lc.construct_block = tr->tuning.construct_block;
    lc.construct_ctas_per_sm = tr->tuning.construct_ctas_per_sm;
    lc.construct_mode = tr->tuning.construct_mode;
    lc.stage_rows = tr->tuning.stage_rows;
    lc.neighbours_smem_max = smem;
    lc.seed_kernel = tr->tuning.seed_kernel;
    lc.n_clusters = n_total;
    lc.n_slots = s_off;
    lc.order_group = tr->tuning.order_group;
    lc.max_row_clusters = max_row;

    // The call's copies, clears and launches go to the caller's stream, or (graph mode) are
    // captured on the tracker's own stream into a graph that updates the cached executable graph
    // in place and is launched on the caller's stream as one unit.
    const bool graph = tr->tuning.use_graph != 0;
    cudaStream_t ls = st;
    if (graph) {
        if (!tr->cap_stream) TPC_CUDA(cudaStreamCreateWithFlags(&tr->cap_stream, cudaStreamNonBlocking));
        ls = tr->cap_stream;
        TPC_CUDA(cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal));
    }
    cudaError_t ce = cudaSuccess;
    auto chk = [&](cudaError_t e) {
        if (ce == cudaSuccess && e != cudaSuccess) ce = e;
    };
    auto mark = [&](int i) {
        if (timed)
            chk(graph ? cudaEventRecordWithFlags(res->stage_ev[i], ls, cudaEventRecordExternal)
                      : cudaEventRecord(res->stage_ev[i], ls));
    };
    if (R > 0) {
        chk(cudaMemcpyAsync(w.meta, sg.meta, R * sizeof(int4), cudaMemcpyHostToDevice, ls));
        chk(cudaMemcpyAsync(w.dims, sg.dims, R * sizeof(int2), cudaMemcpyHostToDevice, ls));
    }
    if (!graph) chk(cudaEventRecord(sg.consumed, st));
    chk(cudaMemsetAsync(w.counters, 0, kCountWords * sizeof(int32_t), ls));
    chk(cudaMemsetAsync(w.bits, 0, ((n_total + 31) / 32 + 2) * sizeof(uint32_t), ls));
    chk(cudaMemsetAsync(w.ckey, 0, s_off * sizeof(unsigned long long), ls));

    int launches = 0;
    NvtxRange nvtx_call(graph ? "tpc: capture call" : "tpc: launch call");
    mark(1);
    launches += launch_ingest(tr->dc, w, y, z, row, R, ls);
    mark(2);
    launches += launch_neighbours(tr->dc, w, R, smem, lc, ls);
    mark(3);
    launches += launch_evolve(tr->dc, w, R, ls);
    mark(4);
    launches += lc.construct_mode == 1 ? launch_construct_sweep(tr->dc, w, (int)(R / nr), lc, ls)
                                       : launch_construct(tr->dc, w, lc, ls);
    mark(5);
    launches += launch_select(tr->dc, w, n_total, lc, ls);
    mark(6);
    if (tr->dc.global) launches += launch_global(tr->dc, w, s_off, lc, ls);
    mark(8);
    launches += launch_output(tr->dc, w, tr->dc.merge ? w.st : res->out, n_total, lc, ls);
    mark(7);
    if (tr->dc.merge) launches += launch_merge(tr->dc, w, res->out, y, z, row, R, lc, ls);
    mark(9);
    chk(cudaGetLastError());
    if (graph) {
        cudaGraph_t g = nullptr;
        chk(cudaStreamEndCapture(ls, &g));
        if (ce == cudaSuccess && tr->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(tr->gexec, g, &info) != cudaSuccess) {
                cudaGetLastError();              // a different topology: instantiate anew
                cudaGraphExecDestroy(tr->gexec);
                tr->gexec = nullptr;
            }
        }
        if (ce == cudaSuccess && !tr->gexec) {
            chk(cudaGraphInstantiate(&tr->gexec, g, 0));
            tr->graph_builds++;
        }
        if (ce == cudaSuccess) chk(cudaGraphLaunch(tr->gexec, st));
        if (g) cudaGraphDestroy(g);
        if (ce == cudaSuccess) chk(cudaEventRecord(sg.consumed, st));
    }
    sg.pending = true;
    TPC_CUDA(ce);
    res->launches = launches;
    res->graph_builds = tr->graph_builds;
    TPC_CUDA(cudaMemcpyAsync(res->h_counts, w.counters, kCountWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TPC_CUDA(cudaEventRecord(res->done, st));
    TPC_CUDA(cudaEventRecord(tr->ws_done, st));
    tr->ws_used = true;
    guard.armed = false;
    tr->live_results++;
    tr->last_units = R;
    tr->last_slots = s_off;
    tr->last_n = n_total;
    *out = res;
    return TPC_OK;
}

extern "C" int tpc_track_batch(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                               const int32_t *counts, int n_events, int64_t n_total, void *stream,
                               tpc_result **out)
{
    NvtxRange nvtx("tpc_track_batch");
    if (!tr || !out || !counts || n_events < 1 || n_total < 0) return TPC_ERR_INVALID_ARG;
    *out = nullptr;
    std::lock_guard<std::mutex> g(tr->mu);
    if (tr->destroyed) return TPC_ERR_STATE;
    return run(tr, y, z, row, counts, n_events, n_total, (cudaStream_t)stream, out);
}

extern "C" int tpc_track_event(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                               const int32_t *counts, int64_t n, void *stream, tpc_result **out)
{
    return tpc_track_batch(tr, y, z, row, counts, 1, n, stream, out);
}

extern "C" int tpc_track_event_host(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                                    const int32_t *counts, int64_t n, void *stream, tpc_result **out)
{
    return tpc_track_batch_host(tr, y, z, row, counts, 1, n, stream, out);
}

extern "C" int tpc_track_batch_host(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                                    const int32_t *counts, int n_events, int64_t n, void *stream,
                                    tpc_result **out)
{
    NvtxRange nvtx("tpc_track_batch_host");
    if (!tr || !out || !counts || n < 0 || n_events < 1) return TPC_ERR_INVALID_ARG;
    if (n > 0 && (!y || !z || !row)) return TPC_ERR_INVALID_ARG;
    *out = nullptr;
    std::lock_guard<std::mutex> g(tr->mu);
    if (tr->destroyed) return TPC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (n > tr->in_cap) {
        // sized for the reserved workspace at least, so that calls up to that size never grow it again
        const int64_t cap = n > tr->cap_n ? n : tr->cap_n;
        if (tr->in_base) {
            TPC_CUDA(cudaDeviceSynchronize());
            cudaFree(tr->in_base);
            tr->bytes_ws -= (size_t)tr->in_cap * 12;
            tr->in_base = nullptr;
            tr->in_cap = 0;
        }
        size_t need = (size_t)cap * 12 + 1024;
        if (tr->budget && tr->bytes_ws + tr->bytes_ring + tr->bytes_results + need > tr->budget) {
            if (cap == n) return TPC_ERR_BUDGET;
            need = (size_t)n * 12 + 1024;            // the reserved size does not fit: this call's size
            if (tr->bytes_ws + tr->bytes_ring + tr->bytes_results + need > tr->budget) return TPC_ERR_BUDGET;
        }
        TPC_CUDA(cudaMalloc(&tr->in_base, need));
        tr->in_cap = (int64_t)((need - 1024) / 12);
        tr->bytes_ws += (size_t)tr->in_cap * 12;
    }
    float *dy = (float *)tr->in_base;
    float *dz = dy + tr->in_cap;
    uint8_t *dr = (uint8_t *)(dz + tr->in_cap);
    if (tr->ws_used) TPC_CUDA(cudaStreamWaitEvent(st, tr->ws_done, 0));
    if (n > 0) {
        TPC_CUDA(cudaMemcpyAsync(dy, y, n * sizeof(float), cudaMemcpyHostToDevice, st));
        TPC_CUDA(cudaMemcpyAsync(dz, z, n * sizeof(float), cudaMemcpyHostToDevice, st));
        TPC_CUDA(cudaMemcpyAsync(dr, row, n, cudaMemcpyHostToDevice, st));
    }
    return run(tr, dy, dz, dr, counts, n_events, n, st, out);
}

extern "C" int tpc_result_sync_counts(tpc_result *r, int64_t *n_tracks, int64_t *n_hits)
{
    if (!r) return TPC_ERR_INVALID_ARG;
    if (!r->synced) {
        TPC_CUDA(cudaEventSynchronize(r->done));
        r->synced = true;
        const int32_t *err = r->h_counts + CNT_COUNT;
        r->status = err[ERR_STATUS];
        r->n_tracks = r->h_counts[CNT_TRACKS];
        r->n_hits = r->h_counts[CNT_HITS];
        if (r->status != TPC_OK) {
            std::lock_guard<std::mutex> g(r->tr->mu);
            memcpy(r->tr->last_err, err, sizeof(r->tr->last_err));
        }
    }
    if (n_tracks) *n_tracks = r->n_tracks;
    if (n_hits) *n_hits = r->n_hits;
    return r->status;
}

extern "C" int tpc_result_ready(tpc_result *r)
{
    if (!r) return -TPC_ERR_INVALID_ARG;
    if (r->synced) return 1;
    cudaError_t e = cudaEventQuery(r->done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return -TPC_ERR_CUDA;
}

extern "C" int tpc_result_get(tpc_result *r, tpc_track_view *v)
{
    if (!r || !v) return TPC_ERR_INVALID_ARG;
    if (!r->synced) return TPC_ERR_STATE;
    v->n_tracks = r->n_tracks;
    v->n_hits = r->n_hits;
    v->par = r->out.par;
    v->cov = r->out.cov;
    v->x_ref = r->out.x;
    v->alpha = r->out.alpha;
    v->chi2 = r->out.chi2;
    v->ndf = r->out.ndf;
    v->nhits = r->out.nhits;
    v->first = r->out.first;
    v->sector = r->out.sector;
    v->event = r->out.event;
    v->hits = r->out.hits;
    return TPC_OK;
}

extern "C" int tpc_result_copy_to_host(tpc_result *r, float *par, float *cov, float *x_ref, float *alpha,
                                       float *chi2, int32_t *ndf, int32_t *nhits, int32_t *first, int32_t *sector,
                                       int32_t *event, int32_t *hits)
{
    if (!r) return TPC_ERR_INVALID_ARG;
    int s = tpc_result_sync_counts(r, nullptr, nullptr);
    if (s != TPC_OK) return s;
    const int64_t M = r->n_tracks, H = r->n_hits;
    cudaStream_t st;
    {
        std::lock_guard<std::mutex> g(r->tr->mu);
        if (!r->tr->copy_stream) TPC_CUDA(cudaStreamCreateWithFlags(&r->tr->copy_stream, cudaStreamNonBlocking));
        st = r->tr->copy_stream;
    }
    TPC_CUDA(cudaStreamWaitEvent(st, r->done, 0));     // complete already (synced above): orders the copies
    struct Item {
        void *dst;
        const void *src;
        size_t bytes;
    } items[] = {
        {par, r->out.par, (size_t)M * 5 * 4}, {cov, r->out.cov, (size_t)M * 15 * 4}, {x_ref, r->out.x, (size_t)M * 4},
        {alpha, r->out.alpha, (size_t)M * 4}, {chi2, r->out.chi2, (size_t)M * 4},    {ndf, r->out.ndf, (size_t)M * 4},
        {nhits, r->out.nhits, (size_t)M * 4}, {first, r->out.first, (size_t)M * 4},  {sector, r->out.sector, (size_t)M * 4},
        {event, r->out.event, (size_t)M * 4}, {hits, r->out.hits, (size_t)H * 4},
    };
    for (auto &it : items)
        if (it.dst && it.bytes) TPC_CUDA(cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost, st));
    TPC_CUDA(cudaStreamSynchronize(st));
    return TPC_OK;
}

static void free_tracker(tpc_tracker *tr);

extern "C" void tpc_result_release(tpc_result *r)
{
    if (!r) return;
    tpc_tracker *tr = r->tr;
    bool last = false;
    if (r->ring) {
        // back to the ring: the next call that takes these buffers waits (on the device) for
        // everything enqueued on this result's stream so far
        if (r->done) cudaEventSynchronize(r->done);
        std::lock_guard<std::mutex> g(tr->mu);
        if (tr->destroyed || tr->ring_count > tr->ring_depth) {
            ring_drop(tr, r);
        } else {
            r->reuse_pending = cudaEventRecord(r->reusable, r->stream) == cudaSuccess;
            if (!r->reuse_pending) cudaStreamSynchronize(r->stream);
            tr->ring_free.push_back(r);
        }
        tr->live_results--;
        last = tr->destroyed && tr->live_results == 0;
    } else {
        if (r->dev) cudaFreeAsync(r->dev, r->stream);
        r->dev = nullptr;
        if (r->done) cudaEventSynchronize(r->done);
        std::lock_guard<std::mutex> g(tr->mu);
        tr->bytes_results -= r->bytes;
        r->bytes = 0;
        tr->free_results.push_back(r);      // pinned counts and events are kept for the next call
        tr->live_results--;
        last = tr->destroyed && tr->live_results == 0;
    }
    if (last) free_tracker(tr);             // the tracker was destroyed while this result was alive
}

static void destroy_result(tpc_result *r)
{
    if (r->dev && r->ring) cudaFree(r->dev);
    if (r->reusable) cudaEventDestroy(r->reusable);
    if (r->done) cudaEventDestroy(r->done);
    if (r->h_counts) cudaFreeHost(r->h_counts);
    for (auto &e : r->stage_ev)
        if (e) cudaEventDestroy(e);
    delete r;
}

static void free_tracker(tpc_tracker *tr)
{
    for (tpc_result *r : tr->free_results) destroy_result(r);
    tr->free_results.clear();
    if (tr->copy_stream) cudaStreamDestroy(tr->copy_stream);
    delete tr;
}

extern "C" void tpc_tracker_destroy(tpc_tracker *tr)
{
    if (!tr) return;
    cudaDeviceSynchronize();
    bool now = false;
    {
        std::lock_guard<std::mutex> g(tr->mu);
        if (tr->destroyed) return;
        tr->destroyed = true;
        if (tr->ws_base) cudaFree(tr->ws_base);
        if (tr->in_base) cudaFree(tr->in_base);
        while (!tr->ring_free.empty()) {     // ring results the caller still holds go at their release
            tpc_result *r = tr->ring_free.back();
            tr->ring_free.pop_back();
            ring_drop(tr, r);
        }
        tr->ws_base = tr->in_base = nullptr;
        for (auto &st : tr->staging) {
            if (st.meta) cudaFreeHost(st.meta);
            if (st.dims) cudaFreeHost(st.dims);
            if (st.consumed) cudaEventDestroy(st.consumed);
            st.meta = nullptr;
            st.dims = nullptr;
            st.consumed = nullptr;
        }
        if (tr->ws_done) cudaEventDestroy(tr->ws_done);
        tr->ws_done = nullptr;
        if (tr->gexec) cudaGraphExecDestroy(tr->gexec);
        if (tr->cap_stream) cudaStreamDestroy(tr->cap_stream);
        tr->gexec = nullptr;
        tr->cap_stream = nullptr;
        now = tr->live_results == 0;
    }
    // results still held by the caller keep the (device-free) tracker object alive until released
    if (now) free_tracker(tr);
}

extern "C" int tpc_last_error_detail(tpc_tracker *tr, int *event, int *sector, int *stage)
{
    if (!tr) return TPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(tr->mu);
    if (event) *event = tr->last_err[ERR_EVENT];
    if (sector) *sector = tr->last_err[ERR_SECTOR];
    if (stage) *stage = tr->last_err[ERR_STAGE];
    return tr->last_err[ERR_STATUS];
}

extern "C" int tpc_tracker_inject(tpc_tracker *tr, int what)
{
    if (!tr || what < 0 || what > 1) return TPC_ERR_INVALID_ARG;
    tr->dc.inject = what;
    return TPC_OK;
}

extern "C" int tpc_tracker_set_timing(tpc_tracker *tr, int enable)
{
    if (!tr) return TPC_ERR_INVALID_ARG;
    tr->timing = enable != 0;
    return TPC_OK;
}

extern "C" int tpc_result_stats(tpc_result *r, tpc_call_stats *st)
{
    if (!r || !st) return TPC_ERR_INVALID_ARG;
    TPC_CUDA(cudaEventSynchronize(r->done));
    memset(st, 0, sizeof *st);
    if (r->timed) {
        // events: 0 start, 1..6 after set-up .. selection, 8 after global tracking, 7 after output
        for (int i = 0; i < 6; i++) TPC_CUDA(cudaEventElapsedTime(&st->ms[i], r->stage_ev[i], r->stage_ev[i + 1]));
        TPC_CUDA(cudaEventElapsedTime(&st->ms[TPC_STAGE_GLOBAL], r->stage_ev[6], r->stage_ev[8]));
        TPC_CUDA(cudaEventElapsedTime(&st->ms[TPC_STAGE_OUTPUT], r->stage_ev[8], r->stage_ev[7]));
        TPC_CUDA(cudaEventElapsedTime(&st->ms[TPC_STAGE_MERGE], r->stage_ev[7], r->stage_ev[9]));
    }
    st->kernel_launches = r->launches;
    st->clusters = r->n_clusters;
    st->tracklets = r->h_counts[CNT_STARTS];
    st->row_visits = r->h_counts[CNT_VISITS];
    st->candidates = r->h_counts[CNT_CANDS];
    st->tracks = r->h_counts[CNT_TRACKS];
    st->hits = r->h_counts[CNT_HITS];
    st->global_found = r->h_counts[CNT_GPOOL];
    st->graph_builds = r->graph_builds;
    st->sector_tracks = r->tr->dc.merge ? r->h_counts[CNT_STRACKS] : r->h_counts[CNT_TRACKS];
    st->tracklet_hits = r->h_counts[CNT_TLHITS];
    return TPC_OK;
}

extern "C" int tpc_tracker_debug_view(tpc_tracker *tr, tpc_debug_view *v)
{
    if (!tr || !v) return TPC_ERR_INVALID_ARG;
    if (!tr->ws_used) return TPC_ERR_STATE;
    TPC_CUDA(cudaDeviceSynchronize());
    int32_t cnt[CNT_COUNT];
    TPC_CUDA(cudaMemcpy(cnt, tr->w.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    const Workspace &w = tr->w;
    v->n_units = tr->last_units;
    v->n_slots = tr->last_slots;
    v->n_tracklets = cnt[CNT_STARTS] < w.tcap ? cnt[CNT_STARTS] : w.tcap;
    if (tr->tuning.tracklet_capacity > 0 && v->n_tracklets > tr->tuning.tracklet_capacity)
        v->n_tracklets = tr->tuning.tracklet_capacity;
    v->tracklet_capacity = w.tcap;
    v->unit_meta = (const int32_t *)w.meta;
    v->unit_cells = (const int32_t *)w.dims;
    v->unit_grid = (const float *)w.grid;
    v->cell_start = w.cell;
    v->yz = (const float *)w.yz;
    v->orig = w.orig;
    v->up_raw = w.up_raw;
    v->dn_raw = w.dn_raw;
    v->up = w.up;
    v->dn = w.dn;
    v->starts = (const int32_t *)w.starts;
    v->tl_nhits = w.tl_n;
    v->tl_hits = w.tl_hits;
    v->tl_par = w.tl_par;
    v->tl_cov = w.tl_cov;
    v->tl_x = w.tl_x;
    v->tl_chi2 = w.tl_chi2;
    v->tl_w = w.tl_w;
    v->tl_nowned = w.tl_nowned;
    v->cluster_key = (const uint64_t *)w.ckey;
    return TPC_OK;
}
