// A5 tracklet construction (Section 1, "Tracklet construction"): a Kalman filter seeded from
// each chain of one-to-one links, extended outwards row by row with a chi2-gated cluster
// search, then refitted inwards from the outermost cluster with a fresh covariance.
//
// Persistent kernel: every lane owns one tracklet at a time, keeps its 5-parameter state and
// 15-element covariance in registers, and takes the next tracklet from a device work queue
// as soon as its current one ends.  The loop body is one row visit, so lanes of a warp stay
// converged while their tracklets have very different lengths.
//
// Floating-point expressions follow the same operation order as the CPU oracle's float mode
// (the library is compiled without FMA contraction), so both evaluate identical roundings.
#include <type_traits>

#include "kf.cuh"
#include "../../include/tpcca.h"

namespace tpc {

// ---------------------------------------------------------------------------------------------
// Longest-expected-first order of the tracklets (counting sort on a small key), so that the
// work queue hands out the long tracklets first and ends on short ones.  A chain of 4 or more
// clusters usually belongs to a real track, which runs outwards from its start row to the last
// row and back to row 0: about 2 * n_rows - start row visits.  Shorter chains are mostly noise
// triplets that stop after a few rows.  In a call with many events the tracklets are first
// grouped by the slot of their start cluster (groups of gslots consecutive slots, about one
// central-like event by default): the queue finishes one group's tracklets before the next
// group's, so the rows the resident lanes search stay in L2.  The order only changes which lane builds
// which tracklet when; every tracklet's result is the same.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int work_key(const DevConst &c, int packed)
{
    const int len = (packed >> 8) & 0xff, r0 = packed & 0xff;
    return len >= 4 ? 2 * c.nr - r0 + 1 : 0;       // 0 .. 2 nr + 1 < order_kb(nr)
}

// Buckets per group: the work keys 0 .. 2 nr + 1, rounded up to a multiple of 32.
__host__ __device__ __forceinline__ int order_kb(int nr) { return (2 * nr + 2 + 31) / 32 * 32; }

// Bucket of a tracklet: ascending group, then descending work key.
__device__ __forceinline__ int work_bucket(const DevConst &c, int4 sd, int gslots)
{
    const int kb = order_kb(c.nr);
    return (sd.x / gslots) * kb + (kb - 1 - work_key(c, sd.w));
}

__global__ void __launch_bounds__(256) k_order_hist(const DevConst c, const Workspace w, int gslots, int nb)
{
    extern __shared__ int h[];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int T = n_tracklets(w);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        atomicAdd(&h[work_bucket(c, w.starts[t], gslots)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (h[i]) atomicAdd(&w.buckets[i], h[i]);
}

// Exclusive scan of the nb buckets (one CTA, a contiguous run of buckets per thread); the
// cursors (at kOrderCursors) start at the offsets.
__global__ void __launch_bounds__(1024) k_order_scan(const Workspace w, int nb)
{
    __shared__ int sh[32];
    const int per = (nb + 1023) / 1024, i0 = threadIdx.x * per;
    const int i1 = i0 + per < nb ? i0 + per : nb;
    int sum = 0;
    for (int i = i0; i < i1; i++) sum += w.buckets[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int inc = warp_incl_scan(sum);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int x = sh[lane];
        sh[lane] = warp_incl_scan(x) - x;
    }
    __syncthreads();
    int run = sh[warp] + inc - sum;
    for (int i = i0; i < i1; i++) {
        const int v = w.buckets[i];
        w.buckets[kOrderCursors + i] = run;
        run += v;
    }
}

// Scatter in tiles of the block size: the tile's buckets are counted in shared memory, each
// bucket reserves its range with one global atomic per tile, and every tracklet takes its rank
// within the tile's range (an atomic on shared memory).  The order inside a bucket is free, so
// no ordering between tiles is needed.
__global__ void __launch_bounds__(256) k_order_scatter(const DevConst c, const Workspace w, int gslots, int nb)
{
    extern __shared__ int sm[];
    int *cnt = sm, *base = sm + nb;
    const int T = n_tracklets(w);
    for (int t0 = blockIdx.x * blockDim.x; t0 < T; t0 += gridDim.x * blockDim.x) {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const int t = t0 + threadIdx.x;
        const int key = t < T ? work_bucket(c, w.starts[t], gslots) : 0;
        const int rank = t < T ? atomicAdd(&cnt[key], 1) : 0;
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (cnt[i]) base[i] = atomicAdd(&w.buckets[kOrderCursors + i], cnt[i]);
        __syncthreads();
        if (t < T) {
            const int pos = base[key] + rank;
            if (TPC_IDX(pos, T, w.err, c, 4)) w.order[pos] = t;
        }
        __syncthreads();
    }
}

// Seed of every tracklet, written at its work-queue position: the walk along the chain and the
// three-point circle run here, one thread per tracklet with the latency of the chain's dependent
// loads hidden by occupancy, so that a constructor lane starting a tracklet reads one 32 B record
// instead of stalling its whole warp on the walk.
__global__ void __launch_bounds__(256) k_seed(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < T; q += gridDim.x * blockDim.x) {
        const int t = w.order[q];
        if (!TPC_IDX(t, T, w.err, c, 4)) continue;
        const int4 sd = w.starts[t];
        KF st{};
        const bool ok = seed_tracklet(c, w, sd, st);
        w.tl_n[t] = 0;
        w.tl_key[t] = 0ull;
        w.seeds[2 * q] = make_float4(st.p0, st.p1, st.p2, st.p3);
        w.seeds[2 * q + 1] = make_float4(st.p4, __int_as_float(ok ? t : -1 - t), __int_as_float(sd.w),
                                         __int_as_float(w.orig[sd.x]));
    }
}

constexpr int kSearchBatch = 4;   // candidates whose loads a row search issues together

// Where a lane keeps its filter state between row visits (the state at its last fitted cluster):
// in registers, or in the CTA's shared memory (21 floats per thread, see StateShared), which frees
// about 20 registers for more resident warps.  The prediction of a visit is always in registers.
constexpr bool kStateInShared = true;
constexpr int kConstructCtasPerSm = kStateInShared ? 6 : 5;

struct StateRegs {
    KF s;
    __device__ __forceinline__ KF get() const { return s; }
    __device__ __forceinline__ void put(const KF &x) { s = x; }
};

__device__ __forceinline__ void bind_state(StateRegs &, float *) {}

// One thread's 20 floats at a stride of kStateStride floats per thread: with an odd stride the 32
// lanes of a warp fall in 32 different banks, and each field sits at a constant offset from the
// thread's base.  The array is the launch's dynamic shared memory, sized to the block.
constexpr int kStateStride = 21;

struct StateShared {
    float *v;
    __device__ __forceinline__ KF get() const
    {
        KF s;
        s.p0 = v[0]; s.p1 = v[1]; s.p2 = v[2]; s.p3 = v[3]; s.p4 = v[4];
        s.c00 = v[5]; s.c10 = v[6]; s.c11 = v[7]; s.c20 = v[8]; s.c21 = v[9];
        s.c22 = v[10]; s.c30 = v[11]; s.c31 = v[12]; s.c32 = v[13]; s.c33 = v[14];
        s.c40 = v[15]; s.c41 = v[16]; s.c42 = v[17]; s.c43 = v[18]; s.c44 = v[19];
        return s;
    }
    __device__ __forceinline__ void put(const KF &s)
    {
        v[0] = s.p0; v[1] = s.p1; v[2] = s.p2; v[3] = s.p3; v[4] = s.p4;
        v[5] = s.c00; v[6] = s.c10; v[7] = s.c11; v[8] = s.c20; v[9] = s.c21;
        v[10] = s.c22; v[11] = s.c30; v[12] = s.c31; v[13] = s.c32; v[14] = s.c33;
        v[15] = s.c40; v[16] = s.c41; v[17] = s.c42; v[18] = s.c43; v[19] = s.c44;
    }
};

__device__ __forceinline__ void bind_state(StateShared &s, float *base) { s.v = base + threadIdx.x * kStateStride; }

// Row search and Kalman update of one lane's row visit: the best cluster within the chi2 gate
// updates the state (and, on the inward pass, is recorded as a hit), otherwise the row is a miss.
// Returns true when the pass stops (max_miss misses in a row).
template <class State>
__device__ __forceinline__ bool search_and_update(const DevConst &c, const Workspace &w, int4 rg, float4 gr, float xr,
                                                  KF &pr, State &st, float &xs, int phase, int t, int r, int &rlast,
                                                  int &miss, int &n, float &chi2sum, int &visits, int &cands)
{
    visits++;
    const Gain g = residual_cov_inv(pr, c);
    float chi2 = 0.0f;
    const int bl = search_cells_mlp<kSearchBatch>(c, w.yz + rg.x, w.orig + rg.x, w.cell + rg.y, gr, rg.z, rg.w, pr, g,
                                                  chi2, cands);
    const int b = bl < 0 ? -1 : rg.x + bl;
    if (b >= 0 && chi2 <= c.chi2max) {
        const float2 q = __ldg(w.yz + b);
        if (phase == 2) {
            chi2sum = chi2sum + chi2;
            if (TPC_IDX(n, c.nr, w.err, c, 4)) w.tl_hits[(int64_t)t * c.nr + n] = b;
            n++;
        } else {
            rlast = r;
        }
        kf_update(pr, g, q.x, q.y);
        st.put(pr);
        xs = xr;
        miss = 0;
        return false;
    }
    return ++miss >= c.max_miss;
}

// After a row visit: the next row of the pass, or the pass's end.  The outward pass turns into
// the inward pass from its last cluster with a fresh covariance (no cluster: no tracklet); the
// inward pass writes the tracklet, its state at the innermost fitted cluster.
template <bool GLOBAL, class State>
__device__ __forceinline__ void next_row(const DevConst &c, const Workspace &w, bool stop, int &phase, int t, int &r,
                                         int rlast, int &miss, int &n, float &chi2sum, State &sth, float xs, int orig0)
{
    if (!stop) {
        r += (phase == 1) ? 1 : -1;
        if (r < 0 || r >= c.nr) stop = true;
    }
    if (stop) {
        if (phase == 1) {
            if (rlast < 0) {
                phase = 0;
            } else {
                KF st = sth.get();
                if (GLOBAL) write_outer(w, t, st, xs);   // outer end for global tracking
                set_seed_cov(st, c);
                sth.put(st);
                r = rlast;
                miss = 0;
                n = 0;
                chi2sum = 0.0f;
                phase = 2;
            }
        } else {
            write_tracklet(c, w, t, sth.get(), xs, n, chi2sum, orig0);
            phase = 0;
        }
    }
}

// Register budget: the bounds of 128 threads and kConstructCtasPerSm CTAs per SM give 80
// registers with the state in shared memory, no spills (3 % faster than the state in registers at
// 96 registers and 5 CTAs; 7 or 8 CTAs of 128 spill and are slower).  The same budget admits the
// default launch, 11 CTAs of 64 threads per SM; 88 registers were slower with two calls on the
// device at once (no room left for the other call's kernels), and 72 spill.
// GLOBAL: also store the outward pass's final state (the outer end for global tracking); a
// separate instance so that the plain tracker keeps its register allocation.
// PRESEED selects between two shapes of the same loop (same rows, same arithmetic, same results):
// - false (few tracklets per lane, one event per call): a lane walks its tracklet's chain for the
//   seed when it takes the tracklet and leaves the loop on its own when the queue is empty.  The
//   time is set by the last long tracklets, so no lane waits for another.
// - true (several tracklets per lane): the seed is read from k_seed's record; the warp meets
//   once per row visit after the transport, so that lanes that took a tracklet or skipped the
//   transport search together instead of in separate passes of the visit.  Throughput-bound, so
//   fewer issued instructions win over waiting.
template <bool GLOBAL, bool PRESEED>
__global__ void __launch_bounds__(128, kConstructCtasPerSm)
k_construct(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    int phase = 0;            // 0: needs a tracklet, 1: outward pass, 2: inward pass
    int t = 0, sec = 0, r = 0, rlast = -1, miss = 0, n = 0, orig0 = 0;
    float xs = 0.0f, chi2sum = 0.0f;
    extern __shared__ float construct_state[];   // blockDim.x * kStateStride floats with the state in shared memory
    typename std::conditional<kStateInShared, StateShared, StateRegs>::type st;
    bind_state(st, construct_state);
    int visits = 0, cands = 0;
    if (!PRESEED) {
        while (true) {
            if (phase == 0) {
                const int q = atomicAdd(&w.counters[CNT_QUEUE], 1);
                if (q >= T) break;
                t = w.order[q];
                const int4 sd = w.starts[t];
                sec = sd.w >> 16;
                const int r0 = sd.w & 0xff;
                orig0 = w.orig[sd.x];
                w.tl_n[t] = 0;
                w.tl_key[t] = 0ull;
                KF s0;
                if (!seed_tracklet(c, w, sd, s0)) continue;
                st.put(s0);
                phase = 1;
                r = r0;
                xs = c.row_x[r0];
                rlast = -1;
                miss = 0;
            }
            // one row visit; the row's search record is loaded first so that its latency overlaps
            // the transport arithmetic
            const int unit = sec * c.nr + r;
            const int4 rg = __ldg(&w.rgi[unit]);
            const float4 gr = __ldg(&w.grid[unit]);
            const float xr = c.row_x[r];
            KF pr = st.get();
            bool stop = false;
            if (xr != xs && !propagate(pr, xr - xs, c)) {
                stop = true;
            } else if (fabsf(pr.p0) > __fmaf_rn(xr, c.th, c.margin)) {
                stop = true;
            } else {
                stop = search_and_update(c, w, rg, gr, xr, pr, st, xs, phase, t, r, rlast, miss, n, chi2sum,
                                                visits, cands);
            }
            next_row<GLOBAL>(c, w, stop, phase, t, r, rlast, miss, n, chi2sum, st, xs, orig0);
        }
        __syncwarp();
    } else {
        bool drained = false;     // this lane found the queue empty; the warp leaves when all have
        while (true) {
            if (phase == 0 && !drained) {
                const int q = atomicAdd(&w.counters[CNT_QUEUE], 1);
                if (q >= T) {
                    drained = true;
                } else {
                    const float4 sa = w.seeds[2 * q], sb = w.seeds[2 * q + 1];
                    t = __float_as_int(sb.y);
                    if (t >= 0) {                            // t < 0: unusable seed, the tracklet stays empty
                        const int packed = __float_as_int(sb.z);
                        sec = packed >> 16;
                        r = packed & 0xff;
                        orig0 = __float_as_int(sb.w);
                        KF s0;
                        s0.p0 = sa.x;
                        s0.p1 = sa.y;
                        s0.p2 = sa.z;
                        s0.p3 = sa.w;
                        s0.p4 = sb.x;
                        set_seed_cov(s0, c);
                        st.put(s0);
                        xs = c.row_x[r];
                        rlast = -1;
                        miss = 0;
                        phase = 1;
                    }
                }
            }
            if (__all_sync(kFull, phase == 0 && drained)) break;
            // transport to the row (lanes with a tracklet only), then the searching lanes meet
            KF pr = st.get();
            int4 rg = make_int4(0, 0, 0, 0);
            float4 gr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float xr = 0.0f;
            bool stop = phase == 0;
            if (!stop) {
                const int unit = sec * c.nr + r;
                rg = __ldg(&w.rgi[unit]);
                gr = __ldg(&w.grid[unit]);
                xr = c.row_x[r];
                if (xr != xs && !propagate(pr, xr - xs, c)) stop = true;
                else if (fabsf(pr.p0) > __fmaf_rn(xr, c.th, c.margin)) stop = true;
            }
            const unsigned searching = __ballot_sync(kFull, !stop);
            if (phase == 0) continue;
            if (!stop) {
                __syncwarp(searching);
                stop = search_and_update(c, w, rg, gr, xr, pr, st, xs, phase, t, r, rlast, miss, n, chi2sum,
                                               visits, cands);
            }
            next_row<GLOBAL>(c, w, stop, phase, t, r, rlast, miss, n, chi2sum, st, xs, orig0);
        }
    }
    // visit statistics, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        visits += __shfl_xor_sync(kFull, visits, o);
        cands += __shfl_xor_sync(kFull, cands, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&w.counters[CNT_VISITS], visits);
        atomicAdd(&w.counters[CNT_CANDS], cands);
    }
}

int launch_construct(const DevConst &c, const Workspace &w, const LaunchCfg &lc, cudaStream_t s)
{
    int per_sm = lc.construct_ctas_per_sm;
    const size_t state_bytes = kStateInShared ? (size_t)lc.construct_block * kStateStride * sizeof(float) : 0;
    if (per_sm <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.global ? k_construct<true, false> : k_construct<false, false>,
                                                      lc.construct_block, state_bytes);
        per_sm = occ > 0 ? occ : 1;
    }
    // seed kernel (and the pre-seeded constructor): always by default (seed_kernel 1); with
    // seed_kernel -1 when the call has more than 40 clusters per lane of 5 CTAs per SM (about one
    // start hit per 20 clusters in central-like events, so two tracklets per such lane), the rule
    // of an earlier constructor that the measurements no longer support (one central-like event:
    // 1.29 against 1.37 ms for its construction stage with the seed launch)
    const int64_t lanes = (int64_t)lc.num_sms * 5 * lc.construct_block;
    const bool preseed = lc.seed_kernel > 0 || (lc.seed_kernel < 0 && lc.n_clusters / 20 > 2 * lanes);
    // groups of order_group slots, as many as the histogram's kOrderCursors buckets hold
    const int kb = order_kb(c.nr), max_groups = kOrderCursors / kb;
    int64_t gs = lc.order_group > 0 ? lc.order_group : lc.n_slots + 1;
    if ((lc.n_slots + gs - 1) / gs > max_groups) gs = (lc.n_slots + max_groups - 1) / max_groups;
    if (gs < 1) gs = 1;
    const int ng = (int)((lc.n_slots + gs - 1) / gs) > 0 ? (int)((lc.n_slots + gs - 1) / gs) : 1;
    const int nb = ng * kb;
    cudaMemsetAsync(w.buckets, 0, nb * sizeof(int32_t), s);
    const int og = lc.num_sms * 2;
    k_order_hist<<<og, 256, nb * sizeof(int), s>>>(c, w, (int)gs, nb);
    k_order_scan<<<1, 1024, 0, s>>>(w, nb);
    k_order_scatter<<<og, 256, 2 * nb * sizeof(int), s>>>(c, w, (int)gs, nb);
    if (preseed) k_seed<<<lc.num_sms * 8, 256, 0, s>>>(c, w);
    const unsigned grid = lc.num_sms * per_sm;
    if (c.global) {
        if (preseed) k_construct<true, true><<<grid, lc.construct_block, state_bytes, s>>>(c, w);
        else k_construct<true, false><<<grid, lc.construct_block, state_bytes, s>>>(c, w);
    } else {
        if (preseed) k_construct<false, true><<<grid, lc.construct_block, state_bytes, s>>>(c, w);
        else k_construct<false, false><<<grid, lc.construct_block, state_bytes, s>>>(c, w);
    }
    return preseed ? 5 : 4;
}

}  // namespace tpc
