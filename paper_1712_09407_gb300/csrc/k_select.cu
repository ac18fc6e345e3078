// A6 tracklet selection (Section 1 "Tracklet selection"; cluster weights, Section 3.1; minimum of
// 30 clusters, Section 5) and A7 output in canonical order (track sorting, Section 3.2).
//
// Selection: every tracklet claims its clusters with a 64-bit key (weight, then the lower input
// index of the start cluster) through atomicMax, so the maximal-weight tracklet owns each
// cluster whatever order the tracklets were built in.  A tracklet keeps the clusters it owns and
// becomes a track if it owns enough of them and passes the momentum cut.
//
// Output order: the innermost owned cluster of each track is unique, and input indices are
// grouped by (event, sector, row), so sorting tracks by that input index is the canonical
// (event, sector, row, index) order.  It is done without a sort: set one bit per track in a
// bitmap over input indices, scan the words' popcounts, and the rank of a track is the number of
// set bits before its own.
#include "common.cuh"
#include "../../include/tpcca.h"

namespace tpc {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------------------------------------
// exclusive scan of int32 values (mode 0) or of popcounts of uint32 words (mode 1)
// ---------------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ int scan_load(const void *in, int64_t i)
{
    if (MODE == 0) return ((const int32_t *)in)[i];
    return __popc(((const uint32_t *)in)[i]);
}

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? sh[lane] : 0;
        int si = warp_incl_scan(s);
        if (lane < nw) sh[lane] = si - s;
        if (lane == nw - 1) sh[32] = si;
    }
    __syncthreads();
    const int r = sh[warp] + inc - v;
    total = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int64_t scan_len(int64_t n, const int32_t *n_dev)
{
    if (n_dev) {
        int64_t d = *n_dev;
        return d < n ? d : n;
    }
    return n;
}

template <int MODE>
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const void *in, int64_t n, const int32_t *n_dev, int32_t *partials)
{
    __shared__ int sh[33];
    const int64_t len = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= len) {
        if (threadIdx.x == 0) partials[blockIdx.x] = 0;
        return;
    }
    int v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < len) v += scan_load<MODE>(in, i);
    }
    int total;
    block_excl_scan(v, sh, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_partials(int32_t *partials, int nb, int32_t *total_out)
{
    __shared__ int sh[33];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? partials[b] : 0;
        int tot;
        const int ex = block_excl_scan(v, sh, tot);
        if (b < nb) partials[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <int MODE>
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const void *in, int32_t *out, int64_t n, const int32_t *n_dev, const int32_t *partials)
{
    __shared__ int sh[33];
    const int64_t len = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= len) return;
    // each thread scans kScanItems consecutive values
    int vals[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        vals[k] = i < len ? scan_load<MODE>(in, i) : 0;
        sum += vals[k];
    }
    int tot;
    int ex = block_excl_scan(sum, sh, tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < len) out[i] = ex;
        ex += vals[k];
    }
}

// Exclusive scan of n values (or *n_dev of them when n_dev is given); writes the total to
// *total_out.  partials needs ceil(n / kScanTile) ints; at most kScanThreads * 64 tiles.
template <int MODE>
static void scan(const void *in, int32_t *out, int64_t n, const int32_t *n_dev, int32_t *partials,
                 int32_t *total_out, cudaStream_t s)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) nb = 1;
    k_scan_reduce<MODE><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, partials);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, (int)nb, total_out);
    k_scan_apply<MODE><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, n_dev, partials);
}

int launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, const int32_t *n_dev, int32_t *partials,
                    int32_t *total_out, cudaStream_t s)
{
    scan<0>(in, out, n, n_dev, partials, total_out, s);
    return 3;
}

// ---------------------------------------------------------------------------------------------
// A6
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_claim(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < T; t += nwarps) {
        const unsigned long long key = w.tl_key[t];
        if (key == 0ull) continue;
        const int n = w.tl_n[t];
        const int32_t *h = w.tl_hits + (int64_t)t * c.nr;
        for (int i = lane; i < n; i += 32) atomicMax(&w.ckey[h[i]], key);   // result unused: no wait
    }
}

__global__ void __launch_bounds__(256) k_count(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int nsum = 0;       // clusters of the claiming tracklets (statistics), one atomic per warp
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < T; t += nwarps) {
        const unsigned long long key = w.tl_key[t];
        const int n = key ? w.tl_n[t] : 0;
        nsum += n;
        const int32_t *h = w.tl_hits + (int64_t)t * c.nr;
        int owned = 0, inner_i = -1;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const bool own = i < n && w.ckey[h[i]] == key;
            const unsigned mask = __ballot_sync(kFull, own);
            if (lane == 0) w.tl_own[(int64_t)t * ((c.nr + 31) >> 5) + (i0 >> 5)] = mask;   // for the output
            owned += __popc(mask);
            if (mask) inner_i = i0 + 31 - __clz(mask);   // hits run outer to inner
        }
        const float q = w.tl_par[4 * w.tcap + t];
        const bool accept = key != 0ull && owned >= c.min_clusters && fabsf(q) <= c.qptmax;
        if (lane == 0) {
            w.tl_nowned[t] = owned;
            int inner = -1;
            if (accept) {
                inner = w.orig[h[inner_i]];
                atomicOr(&w.bits[inner >> 5], 1u << (inner & 31));
            }
            w.tl_inner[t] = inner;
        }
    }
    if (lane == 0 && nsum) atomicAdd(&w.counters[CNT_TLHITS], nsum);
}

int launch_select(const DevConst &c, const Workspace &w, int64_t n_input, const LaunchCfg &lc, cudaStream_t s)
{
    (void)n_input;
    const int grid = lc.num_sms * 8;
    k_claim<<<grid, 256, 0, s>>>(c, w);
    k_count<<<grid, 256, 0, s>>>(c, w);
    return 2;
}

// ---------------------------------------------------------------------------------------------
// A7
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rank(const DevConst c, const Workspace w)
{
    const int T = n_tracklets(w);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int o = w.tl_inner[t];
        if (o < 0) continue;
        const uint32_t word = w.bits[o >> 5];
        const int rank = w.word_off[o >> 5] + __popc(word & ((1u << (o & 31)) - 1u));
        w.rank_trk[rank] = t;
        w.rank_first[rank] = w.tl_nowned[t] + (c.global ? w.g_own[2 * t] + w.g_own[2 * t + 1] : 0);
    }
}

// Clusters of prolongation p that it owns (claim key equal to its own), written from pos on in
// search order (reverse = false) or reversed; returns the position after them.
__device__ __forceinline__ int write_prolongation(const Workspace &w, const OutBuffers &o, int p, int pos,
                                                  bool reverse)
{
    const int n = w.g_n[p];
    if (n == 0) return pos;
    const int lane = threadIdx.x & 31;
    const int32_t *h = w.gpool + w.g_off[p];
    const unsigned long long key = prolong_key(w, p >> 1, p & 1);
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = reverse ? n - 1 - (i0 + lane) : i0 + lane;
        const bool own = i >= 0 && i < n && w.gkey[h[i]] == key;
        const unsigned mask = __ballot_sync(kFull, own);
        if (own && TPC_IDX(pos + __popc(mask & lanemask_lt()), o.hcap, w.err, c, 6))
            o.hits[pos + __popc(mask & lanemask_lt())] = w.orig[h[i]];
        pos += __popc(mask);
    }
    return pos;
}

__global__ void __launch_bounds__(256) k_write(const DevConst c, const Workspace w, const OutBuffers o)
{
    const int M = w.counters[CNT_TRACKS];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int tcap = (int)w.tcap;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += nwarps) {
        if (!TPC_IDX(m, o.mcap, w.err, c, 6)) continue;
        const int t = w.rank_trk[m];
        const int first = w.rank_first[m];
        const int n = w.tl_n[t];
        const int32_t *h = w.tl_hits + (int64_t)t * c.nr;
        // with global tracking, an inward prolongation that fitted clusters gives the state
        const bool inward = c.global && w.g_n[2 * t] > 0;
        const float *P = inward ? w.g_par : w.tl_par;
        const float *V = inward ? w.g_cov : w.tl_cov;
        if (lane < 5) o.par[(int64_t)m * 5 + lane] = P[lane * tcap + t];
        if (lane < 15) o.cov[(int64_t)m * 15 + lane] = V[lane * tcap + t];
        if (lane == 0) {
            const int sec = w.starts[t].w >> 16;
            const int sector = inward ? w.g_sec[t] : sec % c.ns;
            float chi2 = w.tl_chi2[t];
            int ndf = 2 * n - 5, nhits = w.tl_nowned[t];
            if (c.global) {
                chi2 = chi2 + w.g_chi[2 * t];
                chi2 = chi2 + w.g_chi[2 * t + 1];
                ndf += 2 * (w.g_n[2 * t] + w.g_n[2 * t + 1]);
                nhits += w.g_own[2 * t] + w.g_own[2 * t + 1];
            }
            o.x[m] = inward ? w.g_x[t] : w.tl_x[t];
            o.alpha[m] = c.sec_alpha[sector];
            o.chi2[m] = chi2;
            o.ndf[m] = ndf;
            o.nhits[m] = nhits;
            o.first[m] = first;
            o.sector[m] = sector;
            o.event[m] = sec / c.ns;
        }
        int pos = first;
        // inward prolongation's clusters, inner to outer (found outer to inner); skipped when the call
        // failed (a full prolongation pool leaves holes in it)
        const bool gok = c.global && w.err[ERR_STATUS] == 0;
        if (gok) pos = write_prolongation(w, o, 2 * t, pos, true);
        // owned clusters, inner to outer (the tracklet stores them outer to inner), from the
        // ownership bits of the count
        const uint32_t *om = w.tl_own + (int64_t)t * ((c.nr + 31) >> 5);
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = n - 1 - (i0 + lane);
            const bool own = i >= 0 && ((om[i >> 5] >> (i & 31)) & 1u);
            const unsigned mask = __ballot_sync(kFull, own);
            if (own && TPC_IDX(pos + __popc(mask & lanemask_lt()), o.hcap, w.err, c, 6))
            o.hits[pos + __popc(mask & lanemask_lt())] = w.orig[h[i]];
            pos += __popc(mask);
        }
        // outward prolongation's clusters, in search order (inner to outer)
        if (gok) write_prolongation(w, o, 2 * t + 1, pos, false);
    }
}

int launch_output(const DevConst &c, const Workspace &w, const OutBuffers &o, int64_t n_input,
                   const LaunchCfg &lc, cudaStream_t s)
{
    const int64_t words = (n_input + 31) / 32 + 1;
    scan<1>(w.bits, w.word_off, words, nullptr, w.scan_tmp, w.counters + CNT_TRACKS, s);
    const int grid = lc.num_sms * 8;
    k_rank<<<grid, 256, 0, s>>>(c, w);
    scan<0>(w.rank_first, w.rank_first, w.tcap, w.counters + CNT_TRACKS, w.scan_tmp, w.counters + CNT_HITS, s);
    k_write<<<grid, 256, 0, s>>>(c, w, o);
    return 8;
}

}  // namespace tpc
