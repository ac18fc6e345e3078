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
#include "kf.cuh"
#include "../../include/tpcca.h"

namespace tpc {

// ---------------------------------------------------------------------------------------------
// Longest-expected-first order of the tracklets (counting sort on a small key), so that the
// work queue hands out the long tracklets first and ends on short ones.  A chain of 4 or more
// clusters usually belongs to a real track, which runs outwards from its start row to the last
// row and back to row 0: about 2 * n_rows - start row visits.  Shorter chains are mostly noise
// triplets that stop after a few rows.  The order only changes which lane builds which
// tracklet when; every tracklet's result is the same.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int work_key(const DevConst &c, int packed)
{
    const int len = (packed >> 8) & 0xff, r0 = packed & 0xff;
    return len >= 4 ? 2 * c.nr - r0 + 1 : 0;       // 0 .. 2 nr + 1 < kOrderBuckets
}

__global__ void __launch_bounds__(256) k_order_hist(const DevConst c, const Workspace w)
{
    __shared__ int h[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int T = n_tracklets(w);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        atomicAdd(&h[work_key(c, w.starts[t].w)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&w.buckets[i], h[i]);
}

// Exclusive scan of the buckets in descending key order; the cursors start at the offsets.
__global__ void __launch_bounds__(kOrderBuckets) k_order_scan(const Workspace w)
{
    __shared__ int sh[kOrderBuckets / 32 + 1];
    const int i = threadIdx.x;                      // bucket kOrderBuckets - 1 - i
    const int v = w.buckets[kOrderBuckets - 1 - i];
    const int lane = i & 31, warp = i >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = kOrderBuckets / 32;
        const int x = lane < nw ? sh[lane] : 0;
        const int xi = warp_incl_scan(x);
        if (lane < nw) sh[lane] = xi - x;
    }
    __syncthreads();
    w.buckets[kOrderBuckets + kOrderBuckets - 1 - i] = sh[warp] + inc - v;
}

// Scatter in tiles of the block size: the tile's keys are counted in shared memory, each key
// reserves its range of the bucket with one global atomic per tile, and every tracklet takes
// its rank within the tile's range (an atomic on shared memory).  The order inside a bucket is
// free, so no ordering between tiles is needed.
__global__ void __launch_bounds__(256) k_order_scatter(const DevConst c, const Workspace w)
{
    __shared__ int cnt[kOrderBuckets];
    __shared__ int base[kOrderBuckets];
    const int T = n_tracklets(w);
    for (int t0 = blockIdx.x * blockDim.x; t0 < T; t0 += gridDim.x * blockDim.x) {
        for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const int t = t0 + threadIdx.x;
        const int key = t < T ? work_key(c, w.starts[t].w) : 0;
        const int rank = t < T ? atomicAdd(&cnt[key], 1) : 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
            if (cnt[i]) base[i] = atomicAdd(&w.buckets[kOrderBuckets + i], cnt[i]);
        __syncthreads();
        if (t < T) {
            const int pos = base[key] + rank;
            if (TPC_IDX(pos, T, w.err, c, 4)) w.order[pos] = t;
        }
        __syncthreads();
    }
}

// 128 threads and 6 resident CTAs per SM: 80 registers without spills (measured fastest).
// GLOBAL: also store the outward pass's final state (the outer end for global tracking); a
// separate instance so that the plain tracker keeps its register allocation.
template <bool GLOBAL>
__global__ void __launch_bounds__(128, 6)
k_construct(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    int phase = 0;            // 0: needs a tracklet, 1: outward pass, 2: inward pass
    int t = 0, sec = 0, r = 0, rlast = -1, miss = 0, n = 0, orig0 = 0;
    float xs = 0.0f, chi2sum = 0.0f;
    KF st;
    int visits = 0, cands = 0;
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
            if (!seed_tracklet(c, w, sd, st)) continue;
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
        KF pr = st;
        bool stop = false;
        if (xr != xs && !propagate(pr, xr - xs, c)) {
            stop = true;
        } else if (fabsf(pr.p0) > __fmaf_rn(xr, c.th, c.margin)) {
            stop = true;
        } else {
            visits++;
            const Gain g = residual_cov_inv(pr, c);
            float chi2 = 0.0f;
            float2 q_unused;      // reloaded below instead: keeping it live costs spills at 80 registers
            const int bl = search_cells(c, w.yz + rg.x, w.orig + rg.x, w.cell + rg.y, gr, rg.z, rg.w, pr, g, chi2,
                                        q_unused, cands);
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
                st = pr;
                xs = xr;
                miss = 0;
            } else if (++miss >= c.max_miss) {
                stop = true;
            }
        }
        if (!stop) {
            r += (phase == 1) ? 1 : -1;
            if (r < 0 || r >= c.nr) stop = true;
        }
        if (stop) {
            if (phase == 1) {
                if (rlast < 0) {
                    phase = 0;
                } else {
                    if (GLOBAL) write_outer(w, t, st, xs);   // outer end for global tracking
                    set_seed_cov(st, c);
                    r = rlast;
                    miss = 0;
                    n = 0;
                    chi2sum = 0.0f;
                    phase = 2;
                }
            } else {
                // the state sits at the innermost fitted cluster
                write_tracklet(c, w, t, st, xs, n, chi2sum, orig0);
                phase = 0;
            }
        }
    }
    // visit statistics, one atomic per warp
    __syncwarp();
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
    if (per_sm <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.global ? k_construct<true> : k_construct<false>,
                                                      lc.construct_block, 0);
        per_sm = occ > 0 ? occ : 1;
    }
    cudaMemsetAsync(w.buckets, 0, kOrderBuckets * sizeof(int32_t), s);
    const int og = lc.num_sms * 2;
    k_order_hist<<<og, 256, 0, s>>>(c, w);
    k_order_scan<<<1, kOrderBuckets, 0, s>>>(w);
    k_order_scatter<<<og, 256, 0, s>>>(c, w);
    if (c.global)
        k_construct<true><<<lc.num_sms * per_sm, lc.construct_block, 0, s>>>(c, w);
    else
        k_construct<false><<<lc.num_sms * per_sm, lc.construct_block, 0, s>>>(c, w);
    return 4;
}

}  // namespace tpc
