// Serving loop with continuous batching (the paper's HLT requirement: more than 200 central events
// per second, abstract; its CPU/GPU pipeline, Section 2, is the prior art this replaces).
//
// A server owns `lanes` trackers, each with its own stream, device input buffers and workspace
// reserved for `lane_clusters` clusters and `max_batch` events.  Callers submit events from any
// thread; one server thread forms batches from the queue whenever a lane is free (up to
// max_batch events that fit the lane), copies their clusters straight from the callers' buffers
// to the lane, tracks them with one tpc_track_batch call, copies the result back asynchronously
// and splits it per event.  Lanes run concurrently on the device, so events that arrive while
// others are being tracked start as soon as a lane frees up.  An event larger than a lane is
// refused at submission; a batch that fails on the device is retried event by event.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "../../include/tpcca.h"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    int64_t id = 0;
    const float *y = nullptr, *z = nullptr;
    const uint8_t *row = nullptr;
    std::vector<int32_t> counts;
    int64_t n = 0;
    int64_t t_submit = 0, t_launch = 0, t_done = 0;
    int status = TPC_OK;
    int batch = 0;
    std::vector<float> par, cov, x, alpha, chi2;
    std::vector<int32_t> ndf, nhits, first, sector, hits;
};

struct HostOut {                       // pinned copy of one batch result
    float *par = nullptr, *cov = nullptr, *x = nullptr, *alpha = nullptr, *chi2 = nullptr;
    int32_t *ndf = nullptr, *nhits = nullptr, *first = nullptr, *sector = nullptr, *event = nullptr, *hits = nullptr;
    int64_t mcap = 0, hcap = 0;
};

struct Lane {
    tpc_tracker *tr = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t copied = nullptr;
    float *dy = nullptr, *dz = nullptr;
    uint8_t *drow = nullptr;
    std::vector<Req *> batch;
    std::vector<int64_t> offs;
    std::vector<int32_t> counts;
    tpc_result *res = nullptr;
    int state = 0;                     // 0 idle, 1 tracking, 2 copying back
    int64_t M = 0, H = 0;
    HostOut out;
};

void free_out(HostOut &o)
{
    void *p[] = {o.par, o.cov, o.x, o.alpha, o.chi2, o.ndf, o.nhits, o.first, o.sector, o.event, o.hits};
    for (void *q : p)
        if (q) cudaFreeHost(q);
    o = HostOut();
}

// Larger pinned buffers for a batch result.  The old ones are kept until the server is destroyed:
// freeing page-locked memory waits for the whole device, which would stall the other lanes.
bool grow_out(HostOut &o, int64_t M, int64_t H, std::vector<HostOut> &retired)
{
    if (M <= o.mcap && H <= o.hcap) return true;
    int64_t m = std::max(M, 2 * o.mcap), h = std::max(H, 2 * o.hcap);
    m = std::max<int64_t>(m, 4096);
    h = std::max<int64_t>(h, 1 << 20);
    if (o.mcap) retired.push_back(o);
    o = HostOut();
    bool ok = cudaMallocHost((void **)&o.par, m * 5 * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.cov, m * 15 * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.x, m * 4) == cudaSuccess && cudaMallocHost((void **)&o.alpha, m * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.chi2, m * 4) == cudaSuccess && cudaMallocHost((void **)&o.ndf, m * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.nhits, m * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.first, m * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.sector, m * 4) == cudaSuccess &&
              cudaMallocHost((void **)&o.event, m * 4) == cudaSuccess && cudaMallocHost((void **)&o.hits, h * 4) == cudaSuccess;
    if (!ok) {
        free_out(o);
        return false;
    }
    o.mcap = m;
    o.hcap = h;
    return true;
}

}  // namespace

struct tpc_server {
    int device = 0;
    int max_batch = 1;
    int n_units = 0;                   // counts per event: sectors x rows
    int64_t lane_clusters = 0;
    std::vector<Lane> lanes;
    std::mutex mu;                     // guards pending, reqs, done_ids
    std::condition_variable cv;
    std::deque<Req *> pending;
    std::deque<Req *> retry;           // events of a failed batch, tracked one by one (server thread only)
    std::unordered_map<int64_t, Req *> reqs;
    std::vector<int64_t> done_ids;
    int64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::thread th;
    std::vector<HostOut> retired;      // outgrown pinned result buffers (server thread only)
    // Released requests, kept with the capacity of their result vectors (guarded by mu), so that a
    // steady stream of events allocates no host memory per event once the largest results have
    // been seen (large vectors would otherwise be mapped and unmapped for every event).
    std::vector<Req *> spare;
};

constexpr size_t kSpareMax = 64;       // requests kept for reuse; beyond that they are freed

namespace {

void finish(tpc_server *s, Req *r)
{
    std::lock_guard<std::mutex> g(s->mu);
    r->t_done = now_ns();
    s->done_ids.push_back(r->id);
}

// Split a copied batch result per event (tracks are sorted by event).
void split(Lane &L)
{
    const HostOut &o = L.out;
    int64_t t0 = 0;
    for (size_t e = 0; e < L.batch.size(); e++) {
        Req *r = L.batch[e];
        int64_t t1 = t0;
        while (t1 < L.M && o.event[t1] == (int32_t)e) t1++;
        const int64_t M = t1 - t0;
        const int64_t h0 = M ? o.first[t0] : 0;
        const int64_t h1 = M ? o.first[t1 - 1] + o.nhits[t1 - 1] : 0;
        r->par.assign(o.par + t0 * 5, o.par + t1 * 5);
        r->cov.assign(o.cov + t0 * 15, o.cov + t1 * 15);
        r->x.assign(o.x + t0, o.x + t1);
        r->alpha.assign(o.alpha + t0, o.alpha + t1);
        r->chi2.assign(o.chi2 + t0, o.chi2 + t1);
        r->ndf.assign(o.ndf + t0, o.ndf + t1);
        r->nhits.assign(o.nhits + t0, o.nhits + t1);
        r->sector.assign(o.sector + t0, o.sector + t1);
        r->first.resize(M);
        for (int64_t i = 0; i < M; i++) r->first[i] = (int32_t)(o.first[t0 + i] - h0);
        r->hits.resize(h1 - h0);
        const int32_t off = (int32_t)L.offs[e];
        for (int64_t i = 0; i < h1 - h0; i++) r->hits[i] = o.hits[h0 + i] - off;
        r->status = TPC_OK;
        r->batch = (int)L.batch.size();
        t0 = t1;
    }
}

bool launch(tpc_server *s, Lane &L, std::vector<Req *> &batch)
{
    nvtxRangePushA("tpc_server: launch batch");
    L.batch = batch;
    L.offs.clear();
    L.counts.clear();
    int64_t off = 0;
    const int64_t t = now_ns();
    for (Req *r : batch) {
        if (r->n > 0) {
            cudaMemcpyAsync(L.dy + off, r->y, r->n * sizeof(float), cudaMemcpyHostToDevice, L.st);
            cudaMemcpyAsync(L.dz + off, r->z, r->n * sizeof(float), cudaMemcpyHostToDevice, L.st);
            cudaMemcpyAsync(L.drow + off, r->row, r->n, cudaMemcpyHostToDevice, L.st);
        }
        L.offs.push_back(off);
        L.counts.insert(L.counts.end(), r->counts.begin(), r->counts.end());
        off += r->n;
        r->t_launch = t;
    }
    const int st = tpc_track_batch(L.tr, L.dy, L.dz, L.drow, L.counts.data(), (int)batch.size(), off, L.st, &L.res);
    nvtxRangePop();
    if (st != TPC_OK) {
        for (Req *r : batch) {
            r->status = st;
            finish(s, r);
        }
        L.batch.clear();
        L.res = nullptr;
        return false;
    }
    L.state = 1;
    return true;
}

void loop(tpc_server *s)
{
    cudaSetDevice(s->device);
    while (true) {
        bool moved = false;
        for (Lane &L : s->lanes) {
            if (L.state == 1) {
                const int rd = tpc_result_ready(L.res);
                if (rd == 0) continue;
                int64_t M = 0, H = 0;
                const int st = rd < 0 ? TPC_ERR_CUDA : tpc_result_sync_counts(L.res, &M, &H);
                tpc_track_view v;
                if (st == TPC_OK && tpc_result_get(L.res, &v) == TPC_OK && grow_out(L.out, M, H, s->retired)) {
                    L.M = M;
                    L.H = H;
                    const HostOut &o = L.out;
                    struct { void *d; const void *s; size_t b; } cp[] = {
                        {o.par, v.par, (size_t)M * 20}, {o.cov, v.cov, (size_t)M * 60}, {o.x, v.x_ref, (size_t)M * 4},
                        {o.alpha, v.alpha, (size_t)M * 4}, {o.chi2, v.chi2, (size_t)M * 4}, {o.ndf, v.ndf, (size_t)M * 4},
                        {o.nhits, v.nhits, (size_t)M * 4}, {o.first, v.first, (size_t)M * 4},
                        {o.sector, v.sector, (size_t)M * 4}, {o.event, v.event, (size_t)M * 4}, {o.hits, v.hits, (size_t)H * 4}};
                    for (auto &c : cp)
                        if (c.b) cudaMemcpyAsync(c.d, c.s, c.b, cudaMemcpyDeviceToHost, L.st);
                    cudaEventRecord(L.copied, L.st);
                    L.state = 2;
                } else {                           // the batch failed: its events go again one by one
                    tpc_result_release(L.res);
                    L.res = nullptr;
                    if (L.batch.size() > 1) {
                        for (Req *r : L.batch) s->retry.push_back(r);
                    } else {
                        for (Req *r : L.batch) {
                            r->status = st == TPC_OK ? TPC_ERR_CUDA : st;
                            finish(s, r);
                        }
                    }
                    L.batch.clear();
                    L.state = 0;
                }
                moved = true;
            } else if (L.state == 2 && cudaEventQuery(L.copied) == cudaSuccess) {
                nvtxRangePushA("tpc_server: split result");
                split(L);
                nvtxRangePop();
                tpc_result_release(L.res);
                L.res = nullptr;
                for (Req *r : L.batch) finish(s, r);
                L.batch.clear();
                L.state = 0;
                moved = true;
            }
        }
        for (Lane &L : s->lanes) {
            if (L.state != 0) continue;
            std::vector<Req *> batch;
            if (!s->retry.empty()) {
                batch.push_back(s->retry.front());
                s->retry.pop_front();
            } else {
                std::lock_guard<std::mutex> g(s->mu);
                int64_t tot = 0;
                while (!s->pending.empty() && (int)batch.size() < s->max_batch &&
                       tot + s->pending.front()->n <= s->lane_clusters) {
                    tot += s->pending.front()->n;
                    batch.push_back(s->pending.front());
                    s->pending.pop_front();
                }
            }
            if (batch.empty()) break;
            launch(s, L, batch);
            moved = true;
        }
        bool busy = !s->retry.empty();
        for (Lane &L : s->lanes) busy = busy || L.state != 0;
        if (s->stop.load() && !busy) {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->pending.empty()) break;
        }
        if (!moved) {                              // lanes running: poll again soon; idle: wait for a submit
            std::unique_lock<std::mutex> g(s->mu);
            s->cv.wait_for(g, std::chrono::microseconds(busy ? 10 : 200));
        }
    }
}

}  // namespace

extern "C" int64_t tpc_server_now_ns(void) { return now_ns(); }

extern "C" int tpc_server_create(const tpc_geometry *g, float bz, const tpc_params *params,
                                 const tpc_server_config *cfg, tpc_server **out)
{
    if (!g || !cfg || !out || cfg->lanes < 1 || cfg->max_batch < 1 || cfg->lane_clusters < 1)
        return TPC_ERR_INVALID_ARG;
    *out = nullptr;
    tpc_server *s = new (std::nothrow) tpc_server();
    if (!s) return TPC_ERR_CUDA;
    cudaGetDevice(&s->device);
    s->max_batch = cfg->max_batch;
    s->n_units = g->n_sectors * g->n_rows;
    s->lane_clusters = cfg->lane_clusters;
    s->lanes.resize(cfg->lanes);
    const size_t per_lane = cfg->hbm_budget ? cfg->hbm_budget / cfg->lanes : 0;
    int st = TPC_OK;
    for (Lane &L : s->lanes) {
        const size_t in_bytes = (size_t)cfg->lane_clusters * 9;
        if (per_lane && in_bytes >= per_lane) {
            st = TPC_ERR_BUDGET;
            break;
        }
        st = tpc_tracker_create(g, bz, params, per_lane ? per_lane - in_bytes : 0, &L.tr);
        if (st == TPC_OK) st = tpc_tracker_reserve(L.tr, cfg->lane_clusters, cfg->max_batch);
        if (st == TPC_OK) st = tpc_tracker_reserve_results(L.tr, 1);     // a lane holds one result at a time
        if (st != TPC_OK) break;
        if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.copied, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&L.dy, (size_t)cfg->lane_clusters * 4) != cudaSuccess ||
            cudaMalloc(&L.dz, (size_t)cfg->lane_clusters * 4) != cudaSuccess ||
            cudaMalloc(&L.drow, (size_t)cfg->lane_clusters) != cudaSuccess) {
            st = TPC_ERR_CUDA;
            break;
        }
    }
    if (st != TPC_OK) {
        tpc_server_destroy(s);
        return st;
    }
    s->th = std::thread(loop, s);
    *out = s;
    return TPC_OK;
}

extern "C" int tpc_server_submit(tpc_server *s, const float *y, const float *z, const uint8_t *row,
                                 const int32_t *counts, int64_t n, int64_t *id)
{
    if (!s || !counts || !id || n < 0 || (n > 0 && (!y || !z || !row))) return TPC_ERR_INVALID_ARG;
    if (n > s->lane_clusters) return TPC_ERR_BUDGET;
    int64_t sum = 0;
    for (int u = 0; u < s->n_units; u++) {
        if (counts[u] < 0) return TPC_ERR_INVALID_ARG;
        sum += counts[u];
    }
    if (sum != n) return TPC_ERR_INVALID_ARG;
    Req *r = nullptr;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (!s->spare.empty()) {
            r = s->spare.back();
            s->spare.pop_back();
        }
    }
    if (!r) r = new (std::nothrow) Req();
    if (!r) return TPC_ERR_CUDA;
    r->y = y;
    r->z = z;
    r->row = row;
    r->n = n;
    r->counts.assign(counts, counts + s->n_units);
    r->t_launch = r->t_done = 0;
    r->status = TPC_OK;
    r->batch = 0;
    for (auto *v : {&r->par, &r->cov, &r->x, &r->alpha, &r->chi2}) v->clear();      // capacity kept
    for (auto *v : {&r->ndf, &r->nhits, &r->first, &r->sector, &r->hits}) v->clear();
    r->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> g(s->mu);
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->pending.push_back(r);
    }
    s->cv.notify_one();
    *id = r->id;
    return TPC_OK;
}

extern "C" int tpc_server_poll(tpc_server *s, int64_t *ids, int max_ids, int *n_done)
{
    if (!s || !n_done || max_ids < 0 || (max_ids > 0 && !ids)) return TPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    const int n = std::min<int>(max_ids, (int)s->done_ids.size());
    for (int i = 0; i < n; i++) ids[i] = s->done_ids[i];
    s->done_ids.erase(s->done_ids.begin(), s->done_ids.begin() + n);
    *n_done = n;
    return TPC_OK;
}

extern "C" int tpc_server_get(tpc_server *s, int64_t id, tpc_server_result *o)
{
    if (!s || !o) return TPC_ERR_INVALID_ARG;
    Req *r;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return TPC_ERR_INVALID_ARG;
        r = it->second;
        if (r->t_done == 0) return TPC_ERR_STATE;
    }
    o->status = r->status;
    o->n_tracks = (int64_t)r->nhits.size();
    o->n_hits = (int64_t)r->hits.size();
    o->par = r->par.data();
    o->cov = r->cov.data();
    o->x_ref = r->x.data();
    o->alpha = r->alpha.data();
    o->chi2 = r->chi2.data();
    o->ndf = r->ndf.data();
    o->nhits = r->nhits.data();
    o->first = r->first.data();
    o->sector = r->sector.data();
    o->hits = r->hits.data();
    o->t_submit_ns = r->t_submit;
    o->t_launch_ns = r->t_launch;
    o->t_done_ns = r->t_done;
    o->batch_size = r->batch;
    return TPC_OK;
}

extern "C" int tpc_server_release(tpc_server *s, int64_t id)
{
    if (!s) return TPC_ERR_INVALID_ARG;
    Req *r;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return TPC_ERR_INVALID_ARG;
        r = it->second;
        if (r->t_done == 0) return TPC_ERR_STATE;
        s->reqs.erase(it);
        if (s->spare.size() < kSpareMax) {
            s->spare.push_back(r);
            r = nullptr;
        }
    }
    delete r;
    return TPC_OK;
}

extern "C" void tpc_server_destroy(tpc_server *s)
{
    if (!s) return;
    if (s->th.joinable()) {
        s->stop.store(true);
        s->cv.notify_one();
        s->th.join();                              // the queue is drained first
    }
    for (Lane &L : s->lanes) {
        if (L.res) tpc_result_release(L.res);
        if (L.tr) tpc_tracker_destroy(L.tr);
        if (L.dy) cudaFree(L.dy);
        if (L.dz) cudaFree(L.dz);
        if (L.drow) cudaFree(L.drow);
        if (L.copied) cudaEventDestroy(L.copied);
        if (L.st) cudaStreamDestroy(L.st);
        free_out(L.out);
    }
    for (HostOut &o : s->retired) free_out(o);
    for (auto &kv : s->reqs) delete kv.second;
    for (Req *r : s->spare) delete r;
    delete s;
}
