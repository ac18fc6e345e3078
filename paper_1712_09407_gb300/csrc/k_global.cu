// Global tracking (Section 5): every track is prolonged from both of its ends into the
// neighbouring sector, and the clusters found there are merged into the track.
//
// An end counts as lying at a sector edge if its one-row extrapolation in its own sector
// leaves the row's width.  Its state is then rotated into the neighbour sector on that side
// (same z half), and the rows beyond it are searched in the same direction with the
// construction's window, gate and stop rules, among the clusters that belong to no accepted
// track.  Clusters found by several prolongations go to the track of the higher weight (then the
// lower input index of its start cluster, then the inward prolongation), with one 64-bit
// atomicMax per cluster as in the selection.  A track's inward prolongation, if it fitted any
// cluster, gives the reported state.
//
// The prolongations of a call are few and mostly end at the edge test, so one thread takes one
// (track, end) pair.  A prolongation claims every cluster it finds at once and appends
// {slot, prolongation, position} to an unordered pool (warp-aggregated atomics); a scan of the
// per-prolongation counts then gives each prolongation its range, and one pass over the pool
// puts every entry in place and counts the clusters each prolongation owns.  The track's output
// assembles the owned clusters inner to outer.
#include "kf.cuh"
#include "../../include/tpcca.h"

namespace tpc {

constexpr int kGlobalBlock = 128;

// Row whose radius is x (x is one of the row radii, which strictly increase).
__device__ __forceinline__ int row_of_x(const DevConst &c, float x)
{
    int lo = 0, hi = c.nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c.row_x[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_state(const float *P, const float *V, int tcap, int t, KF &s)
{
    s.p0 = P[0 * tcap + t]; s.p1 = P[1 * tcap + t]; s.p2 = P[2 * tcap + t]; s.p3 = P[3 * tcap + t];
    s.p4 = P[4 * tcap + t];
    s.c00 = V[0 * tcap + t]; s.c10 = V[1 * tcap + t]; s.c11 = V[2 * tcap + t]; s.c20 = V[3 * tcap + t];
    s.c21 = V[4 * tcap + t]; s.c22 = V[5 * tcap + t]; s.c30 = V[6 * tcap + t]; s.c31 = V[7 * tcap + t];
    s.c32 = V[8 * tcap + t]; s.c33 = V[9 * tcap + t]; s.c40 = V[10 * tcap + t]; s.c41 = V[11 * tcap + t];
    s.c42 = V[12 * tcap + t]; s.c43 = V[13 * tcap + t]; s.c44 = V[14 * tcap + t];
}

__device__ __forceinline__ void store_state(float *P, float *V, int tcap, int t, const KF &s)
{
    P[0 * tcap + t] = s.p0; P[1 * tcap + t] = s.p1; P[2 * tcap + t] = s.p2; P[3 * tcap + t] = s.p3;
    P[4 * tcap + t] = s.p4;
    V[0 * tcap + t] = s.c00; V[1 * tcap + t] = s.c10; V[2 * tcap + t] = s.c11; V[3 * tcap + t] = s.c20;
    V[4 * tcap + t] = s.c21; V[5 * tcap + t] = s.c22; V[6 * tcap + t] = s.c30; V[7 * tcap + t] = s.c31;
    V[8 * tcap + t] = s.c32; V[9 * tcap + t] = s.c33; V[10 * tcap + t] = s.c40; V[11 * tcap + t] = s.c41;
    V[12 * tcap + t] = s.c42; V[13 * tcap + t] = s.c43; V[14 * tcap + t] = s.c44;
}

// The end state of prolongation (t, d) with its x and row.
__device__ __forceinline__ void end_state(const DevConst &c, const Workspace &w, int t, int d, KF &s, float &x,
                                          int &r)
{
    const int tcap = (int)w.tcap;
    if (d == 0) {          // inner end: the reported state, at the innermost fitted cluster
        load_state(w.tl_par, w.tl_cov, tcap, t, s);
        x = w.tl_x[t];
    } else {               // outer end: the outward pass's state at its last cluster
        load_state(w.tl_opar, w.tl_ocov, tcap, t, s);
        x = w.tl_ox[t];
    }
    r = row_of_x(c, x);
}

// Append one entry to the unordered pool; the lanes of a warp that append in the same step share
// one atomic.  Returns false (and records a capacity error) when the pool is full.
__device__ __forceinline__ bool pool_append(const DevConst &c, const Workspace &w, int slot, int p, int j, int sec)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&w.counters[CNT_GPOOL], __popc(act));
    base = __shfl_sync(act, base, leader) + __popc(act & lanemask_lt());
    if ((int64_t)base >= w.gpool_cap) {
        set_error(w.err, TPC_ERR_CAPACITY, sec * c.nr, c, TPC_STAGE_GLOBAL);
        return false;
    }
    w.gent[base] = make_int4(slot, p, j, 0);
    return true;
}

// Whether prolongation (end at x_end, row r_end, sector `sec`) leaves its sector at the next row in
// direction dir and can be taken into the neighbour's frame (the first steps of prolong, which
// repeats them).
__device__ __forceinline__ bool crosses_edge(const DevConst &c, int sec, const KF &end, float x_end, int r_end,
                                             int dir)
{
    const int rn = r_end + dir;
    if (rn < 0 || rn >= c.nr) return false;
    KF pr = end;
    if (!propagate(pr, c.row_x[rn] - x_end, c)) return false;
    if (!(fabsf(pr.p0) > c.row_x[rn] * c.th)) return false;
    const bool plus = pr.p0 > 0.0f;
    KF st = end;
    float xs;
    return rotate_state(st, x_end, c.c20, plus ? c.s20 : -c.s20, c, xs);
}

// One prolongation p = 2 t + d from `end` (at x_end, row r_end, sector `sec` of the call) in
// direction dir.  Claims and records the clusters it finds; returns their number.
__device__ int prolong(const DevConst &c, const Workspace &w, int p, int sec, const KF &end, float x_end, int r_end,
                       int dir, unsigned long long key, float &chi2_out, KF &fin, float &x_fin, int &s2_out)
{
    chi2_out = 0.0f;
    const int rn = r_end + dir;
    if (rn < 0 || rn >= c.nr) return 0;
    KF pr = end;
    if (!propagate(pr, c.row_x[rn] - x_end, c)) return 0;
    if (!(fabsf(pr.p0) > c.row_x[rn] * c.th)) return 0;      // still inside its own sector
    const int ev = sec / c.ns, s = sec % c.ns;
    const int side = s / 18, az = s % 18;
    const bool plus = pr.p0 > 0.0f;
    const int s2 = side * 18 + (plus ? (az + 1) % 18 : (az + 17) % 18);
    KF st = end;
    float xs;
    if (!rotate_state(st, x_end, c.c20, plus ? c.s20 : -c.s20, c, xs)) return 0;
    int r;
    if (dir < 0) {
        r = c.nr - 1;
        while (r >= 0 && !(c.row_x[r] < xs)) r--;
    } else {
        r = 0;
        while (r < c.nr && !(c.row_x[r] > xs)) r++;
    }
    const int gsec = ev * c.ns + s2;
    int n = 0, miss = 0, cands = 0;
    float chi2sum = 0.0f;
    for (; r >= 0 && r < c.nr; r += dir) {
        // the row's search record first, so that its latency overlaps the transport
        const int4 rg = __ldg(&w.rgi[gsec * c.nr + r]);
        const float4 gr = __ldg(&w.grid[gsec * c.nr + r]);
        const float xr = c.row_x[r];
        KF q = st;
        if (!propagate(q, xr - xs, c)) break;
        if (fabsf(q.p0) > __fmaf_rn(xr, c.th, c.margin)) break;
        const Gain g = residual_cov_inv(q, c);
        float chi2 = 0.0f;
        float2 m;
        const int bl = search_cells_mlp<4, true>(c, w.yz + rg.x, w.orig + rg.x, w.cell + rg.y, gr, rg.z, rg.w, q, g,
                                                 chi2, cands, w.used + rg.x, &m);
        if (bl >= 0 && chi2 <= c.chi2max) {
            const int b = rg.x + bl;
            chi2sum = chi2sum + chi2;
            kf_update(q, g, m.x, m.y);
            st = q;
            xs = xr;
            atomicMax(&w.gkey[b], key);
            pool_append(c, w, b, p, n, sec);
            n++;
            miss = 0;
        } else if (++miss >= c.max_miss) {
            break;
        }
    }
    chi2_out = chi2sum;
    fin = st;
    x_fin = xs;
    s2_out = s2;
    return n;
}

// Clusters owned by accepted tracks are closed to the prolongations.
__global__ void __launch_bounds__(256) k_global_used(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) w.counters[CNT_GLIST] = 2 * T;     // prolongations of the call
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < T; t += nwarps) {
        if (w.tl_inner[t] < 0) continue;
        const unsigned long long key = w.tl_key[t];
        const int n = w.tl_n[t];
        const int32_t *h = w.tl_hits + (int64_t)t * c.nr;
        for (int i = lane; i < n; i += 32)
            if (w.ckey[h[i]] == key) w.used[h[i]] = 1;
    }
}

// Edge test of every prolongation of every accepted track; the ones that will search are listed
// (warp-aggregated), so that the search kernel starts all of them at once.
__global__ void __launch_bounds__(kGlobalBlock) k_global_edge(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    const int lane = threadIdx.x & 31;
    for (int p0 = blockIdx.x * blockDim.x; p0 < 2 * T; p0 += gridDim.x * blockDim.x) {
        const int p = p0 + threadIdx.x;
        bool go = false;
        if (p < 2 * T) {
            const int t = p >> 1, d = p & 1;
            if (w.tl_inner[t] >= 0) {
                KF end;
                float xe;
                int re;
                end_state(c, w, t, d, end, xe, re);
                go = crosses_edge(c, w.starts[t].w >> 16, end, xe, re, d == 0 ? -1 : 1);
            }
            w.g_n[p] = 0;
            w.g_chi[p] = 0.0f;
            w.g_own[p] = 0;
        }
        const unsigned mask = __ballot_sync(kFull, go);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(&w.counters[CNT_GEDGE], __popc(mask));
        base = __shfl_sync(kFull, base, 0);
        if (go) w.g_list[base + __popc(mask & lanemask_lt())] = p;
    }
}

// The listed prolongations: clusters claimed and pooled, count, chi2, final inward state.
__global__ void __launch_bounds__(kGlobalBlock, 4) k_global_find(const DevConst c, const Workspace w)
{
    const int L = w.counters[CNT_GEDGE];
    const int tcap = (int)w.tcap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        const int p = w.g_list[i];
        const int t = p >> 1, d = p & 1;
        KF end, fin;
        float xe, xf, chi;
        int re, s2;
        end_state(c, w, t, d, end, xe, re);
        const int sec = w.starts[t].w >> 16;
        const int n = prolong(c, w, p, sec, end, xe, re, d == 0 ? -1 : 1, prolong_key(w, t, d), chi, fin, xf, s2);
        if (d == 0 && n > 0) {
            store_state(w.g_par, w.g_cov, tcap, t, fin);
            w.g_x[t] = xf;
            w.g_sec[t] = s2;
        }
        w.g_n[p] = n;
        w.g_chi[p] = chi;
    }
}

// Pool entries into place (g_off: exclusive scan of g_n) and owned counts.
__global__ void __launch_bounds__(256) k_global_place(const Workspace w)
{
    const int64_t L = w.counters[CNT_GPOOL] < w.gpool_cap ? w.counters[CNT_GPOOL] : w.gpool_cap;
    for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        const int4 e = w.gent[i];
        const int64_t at = (int64_t)w.g_off[e.y] + e.z;
        if (at < w.gpool_cap) w.gpool[at] = e.x;          // beyond only after a pool overflow (error set)
        if (w.gkey[e.x] == prolong_key(w, e.y >> 1, e.y & 1)) atomicAdd(&w.g_own[e.y], 1);
    }
}

int launch_global(const DevConst &c, const Workspace &w, int64_t n_slots, const LaunchCfg &lc, cudaStream_t s)
{
    cudaMemsetAsync(w.used, 0, (size_t)n_slots, s);
    cudaMemsetAsync(w.gkey, 0, (size_t)n_slots * sizeof(unsigned long long), s);
    const int grid = lc.num_sms * 8;
    k_global_used<<<grid, 256, 0, s>>>(c, w);
    k_global_edge<<<lc.num_sms * 16, kGlobalBlock, 0, s>>>(c, w);
    k_global_find<<<lc.num_sms * 4, kGlobalBlock, 0, s>>>(c, w);    // 78 k threads: every listed one starts at once
    const int scans = launch_scan_i32(w.g_n, w.g_off, 2 * w.tcap, w.counters + CNT_GLIST, w.scan_tmp, nullptr, s);
    k_global_place<<<grid, 256, 0, s>>>(w);
    return 4 + scans;
}

}  // namespace tpc
