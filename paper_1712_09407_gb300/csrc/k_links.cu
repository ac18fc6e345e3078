// A1 cluster ingest and per-row grids, A2 neighbours finder, A3 evolution and A4 start hits.
//
// Section 1 of the paper ("Neighbors finder", "Evolution step", tracklets from chains
// of one-to-one links) and the initialisation step of Section 2.
#include <cfloat>
#include <cstdio>

#include "common.cuh"
#include "../../include/tpcca.h"

namespace tpc {

// ============================================================================================
// A1: per (event, sector, row) unit: y/z extent, grid, counting sort into padded slots.
// One warp per row unit; the sort is stable in input order.  The first pass over the row's
// clusters also copies their (y, z) into the warp's shared memory (rows of up to kIngestStage
// clusters), so that the histogram and scatter passes read them there instead of from L2
// (3-event call 0.186 -> 0.160 ms; 768 against 1024 staged clusters leaves room for 5 CTAs per
// SM instead of 4 and was the faster of the two).
// ============================================================================================
constexpr int kIngestWarps = 4;
constexpr int kIngestStage = 768;
constexpr int kIngestWarpInts = kCellMax + 2 * kIngestStage;   // histogram, then the staged (y, z)

__global__ void __launch_bounds__(kIngestWarps * 32)
k_ingest(const DevConst c, const Workspace w, const float *__restrict__ yin, const float *__restrict__ zin,
         const uint8_t *__restrict__ rin, int64_t R)
{
    extern __shared__ int sh_hist[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *hist = sh_hist + warp * kIngestWarpInts;
    float2 *syz = (float2 *)(hist + kCellMax);
    for (int64_t u = (int64_t)blockIdx.x * kIngestWarps + warp; u < R; u += (int64_t)gridDim.x * kIngestWarps) {
        const int4 m = w.meta[u];
        const int2 d = w.dims[u];
        const int in_off = m.x, n = m.y, s_off = m.z, cell_off = m.w;
        const int ny = d.x, nz = d.y, nc = ny * nz;
        const int r = (int)(u % c.nr);
        float ymin = FLT_MAX, ymax = -FLT_MAX, zmin = FLT_MAX, zmax = -FLT_MAX;
        int bad = 0;
        const bool staged = n <= kIngestStage;
#pragma unroll 4
        for (int i = lane; i < n; i += 32) {
            float y = __ldg(yin + in_off + i), z = __ldg(zin + in_off + i);
            if (staged) syz[i] = make_float2(y, z);
            ymin = fminf(ymin, y);
            ymax = fmaxf(ymax, y);
            zmin = fminf(zmin, z);
            zmax = fmaxf(zmax, z);
            bad |= (__ldg(rin + in_off + i) != r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ymin = fminf(ymin, __shfl_xor_sync(kFull, ymin, o));
            ymax = fmaxf(ymax, __shfl_xor_sync(kFull, ymax, o));
            zmin = fminf(zmin, __shfl_xor_sync(kFull, zmin, o));
            zmax = fmaxf(zmax, __shfl_xor_sync(kFull, zmax, o));
        }
        if (__any_sync(kFull, bad) && lane == 0) set_error(w.err, TPC_ERR_INVALID_ARG, (int)u, c, TPC_STAGE_INGEST);
        float idy = 1.0f, idz = 1.0f;
        if (n == 0) {
            ymin = zmin = 0.0f;
        } else {
            if (ymax > ymin) idy = (float)ny / (ymax - ymin);
            if (zmax > zmin) idz = (float)nz / (zmax - zmin);
        }
        if (lane == 0) {
            w.grid[u] = make_float4(ymin, zmin, idy, idz);
            if (w.rgi) w.rgi[u] = make_int4(s_off, cell_off, ny, nz);
        }
        for (int j = lane; j < nc; j += 32) hist[j] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const float2 q = staged ? syz[i] : make_float2(__ldg(yin + in_off + i), __ldg(zin + in_off + i));
            int cc = cell1(q.y, zmin, idz, nz) * ny + cell1(q.x, ymin, idy, ny);
            atomicAdd(&hist[cc], 1);
        }
        __syncwarp();
        int carry = 0;
        for (int j0 = 0; j0 < nc; j0 += 32) {
            int j = j0 + lane;
            int v = (j < nc) ? hist[j] : 0;
            int inc = warp_incl_scan(v);
            if (j < nc) {
                hist[j] = carry + inc - v;
                w.cell[cell_off + j] = carry + inc - v;
            }
            carry += __shfl_sync(kFull, inc, 31);
        }
        if (lane == 0) w.cell[cell_off + nc] = n;
        __syncwarp();
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const bool v = i < n;
            float y = 0.0f, z = 0.0f;
            int cc = -1 - lane;                       // distinct sentinel for idle lanes
            if (v) {
                const float2 q = staged ? syz[i] : make_float2(__ldg(yin + in_off + i), __ldg(zin + in_off + i));
                y = q.x;
                z = q.y;
                cc = cell1(z, zmin, idz, nz) * ny + cell1(y, ymin, idy, ny);
            }
            const unsigned peers = __match_any_sync(kFull, cc);
            const int rank = __popc(peers & lanemask_lt());
            const int base = v ? hist[cc] : 0;
            __syncwarp();
            if (v && rank == 0) hist[cc] = base + __popc(peers);
            __syncwarp();
            if (v && TPC_IDX(s_off + base + rank, w.pcap, w.err, c, 1)) {
                w.yz[s_off + base + rank] = make_float2(y, z);
                w.orig[s_off + base + rank] = in_off + i;
            }
        }
        __syncwarp();
    }
}

int launch_ingest(const DevConst &c, const Workspace &w, const float *y, const float *z, const uint8_t *row,
                   int64_t R, cudaStream_t s)
{
    if (R == 0) return 0;
    int64_t blocks = (R + kIngestWarps - 1) / kIngestWarps;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    k_ingest<<<(unsigned)blocks, kIngestWarps * 32, kIngestWarps * kIngestWarpInts * sizeof(int), s>>>(c, w, y, z, row, R);
    return 1;
}

// ============================================================================================
// A2: neighbours finder.  One CTA per row unit k; rows k-1 and k+1 (slots, input indices and
// cell starts) are staged into shared memory with bulk async copies completing on an mbarrier.
// Each thread takes clusters of row k and scans every (u, d) pair inside the windows.
// ============================================================================================
struct RowView {
    const float2 *yz;
    const int32_t *orig;
    const int32_t *cell;
    float ymin, zmin, idy, idz;
    int ny, nz, n, s_off;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait on an mbarrier phase for at most kWaitNs of device time; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__host__ __device__ __forceinline__ int round16(int bytes) { return (bytes + 15) & ~15; }

// Bytes of one staged row: yz (8 B/slot), orig (4 B/slot), cell starts (4 B/cell + 1).
__host__ __device__ __forceinline__ int staged_row_bytes(int n, int nc)
{
    return round16(n * 8) + round16(n * 4) + round16((nc + 1) * 4);
}

__device__ __noinline__ void search_pairs_full(const DevConst &c, const RowView &U, const RowView &D, float yc,
                                             float zc, float wyu, float wzu, float wyd, float wzd, float w,
                                             float gate, int &out_u, int &out_d)
{
    const int iy0u = cell1(yc - wyu - kBinSlack, U.ymin, U.idy, U.ny);
    const int iy1u = cell1(yc + wyu + kBinSlack, U.ymin, U.idy, U.ny);
    const int iz0u = cell1(zc - wzu - kBinSlack, U.zmin, U.idz, U.nz);
    const int iz1u = cell1(zc + wzu + kBinSlack, U.zmin, U.idz, U.nz);
    const int iy0d = cell1(yc - wyd - kBinSlack, D.ymin, D.idy, D.ny);
    const int iy1d = cell1(yc + wyd + kBinSlack, D.ymin, D.idy, D.ny);
    const int iz0d = cell1(zc - wzd - kBinSlack, D.zmin, D.idz, D.nz);
    const int iz1d = cell1(zc + wzd + kBinSlack, D.zmin, D.idz, D.nz);
    int bu = -1, bd = -1, bou = 0, bod = 0;
    float best = 0.0f;
    for (int izu = iz0u; izu <= iz1u; izu++) {
        const int au = U.cell[izu * U.ny + iy0u], eu = U.cell[izu * U.ny + iy1u + 1];
        for (int ju = au; ju < eu; ju++) {
            const float2 pu = U.yz[ju];
            if (!(fabsf(pu.x - yc) <= wyu && fabsf(pu.y - zc) <= wzu)) continue;
            const int ou = U.orig[ju];
            for (int izd = iz0d; izd <= iz1d; izd++) {
                const int ad = D.cell[izd * D.ny + iy0d], ed = D.cell[izd * D.ny + iy1d + 1];
                for (int jd = ad; jd < ed; jd++) {
                    const float2 pd = D.yz[jd];
                    if (!(fabsf(pd.x - yc) <= wyd && fabsf(pd.y - zc) <= wzd)) continue;
                    // residual of c from the chord d -> u, evaluated at x_k (same order as the oracle)
                    const float dy = __fmaf_rn(-(pu.x - pd.x), w, yc - pd.x);
                    const float dz = __fmaf_rn(-(pu.y - pd.y), w, zc - pd.y);
                    const float sc = __fmaf_rn(dz * dz, c.isz2, (dy * dy) * c.isy2);
                    if (bu >= 0 && sc > best) continue;
                    const int od = D.orig[jd];
                    if (bu < 0 || sc < best || ou < bou || (ou == bou && od < bod)) {
                        best = sc;
                        bu = ju;
                        bd = jd;
                        bou = ou;
                        bod = od;
                    }
                }
            }
        }
    }
    if (bu >= 0 && best <= gate) {
        out_u = U.s_off + bu;
        out_d = D.s_off + bd;
    } else {
        out_u = -1;
        out_d = -1;
    }
}

constexpr int kDList = 12;   // row k-1 candidates kept per cluster before falling back to re-scanning

// Best (u, d) pair for cluster (yc, zc): the row k-1 candidates inside the window are listed once,
// then every row k+1 candidate inside its window is paired with each of them.  More than kDList
// row k-1 candidates (very dense rows) use search_pairs_full, which gives the same answer.  Both
// rows' candidates are visited cell row by cell row, slots ascending, in flat loops that move on
// to the next non-empty cell row within a candidate's iteration (a warp runs as many iterations as
// its busiest lane has candidates).
__device__ __forceinline__ void search_pairs(const DevConst &c, const RowView &U, const RowView &D, float yc,
                                             float zc, float wyu, float wzu, float wyd, float wzd, float w,
                                             float gate, int &out_u, int &out_d)
{
    const int iy0d = cell1(yc - wyd - kBinSlack, D.ymin, D.idy, D.ny);
    const int iy1d = cell1(yc + wyd + kBinSlack, D.ymin, D.idy, D.ny);
    const int iz0d = cell1(zc - wzd - kBinSlack, D.zmin, D.idz, D.nz);
    const int iz1d = cell1(zc + wzd + kBinSlack, D.zmin, D.idz, D.nz);
    float dly[kDList], dlz[kDList];
    int dlj[kDList];
    int nd = 0;
    bool over = false;
    {
        int izd = iz0d - 1, jd = 0, ed = 0;
        while (jd >= ed && izd < iz1d) {
            ++izd;
            jd = D.cell[izd * D.ny + iy0d];
            ed = D.cell[izd * D.ny + iy1d + 1];
        }
        while (jd < ed) {
            const int k = jd++;
            const float2 pd = D.yz[k];
            while (jd >= ed && izd < iz1d) {
                ++izd;
                jd = D.cell[izd * D.ny + iy0d];
                ed = D.cell[izd * D.ny + iy1d + 1];
            }
            if (!(fabsf(pd.x - yc) <= wyd && fabsf(pd.y - zc) <= wzd)) continue;
            if (nd < kDList) {
                dly[nd] = pd.x;
                dlz[nd] = pd.y;
                dlj[nd] = k;
                nd++;
            } else {
                over = true;
            }
        }
    }
    if (over) {
        search_pairs_full(c, U, D, yc, zc, wyu, wzu, wyd, wzd, w, gate, out_u, out_d);
        return;
    }
    out_u = -1;
    out_d = -1;
    if (nd == 0) return;
    const int iy0u = cell1(yc - wyu - kBinSlack, U.ymin, U.idy, U.ny);
    const int iy1u = cell1(yc + wyu + kBinSlack, U.ymin, U.idy, U.ny);
    const int iz0u = cell1(zc - wzu - kBinSlack, U.zmin, U.idz, U.nz);
    const int iz1u = cell1(zc + wzu + kBinSlack, U.zmin, U.idz, U.nz);
    int bu = -1, bd = -1, bou = 0, bod = 0;
    float best = 0.0f;
    int izu = iz0u - 1, jn = 0, eu = 0;
    while (jn >= eu && izu < iz1u) {
        ++izu;
        jn = U.cell[izu * U.ny + iy0u];
        eu = U.cell[izu * U.ny + iy1u + 1];
    }
    while (jn < eu) {
        const int ju = jn++;
        {   // one row k+1 candidate
            const float2 pu = U.yz[ju];
            while (jn >= eu && izu < iz1u) {
                ++izu;
                jn = U.cell[izu * U.ny + iy0u];
                eu = U.cell[izu * U.ny + iy1u + 1];
            }
            if (!(fabsf(pu.x - yc) <= wyu && fabsf(pu.y - zc) <= wzu)) continue;
            const int ou = U.orig[ju];
            for (int k = 0; k < nd; k++) {
                // residual of c from the chord d -> u, evaluated at x_k (same order as the oracle)
                const float dy = __fmaf_rn(-(pu.x - dly[k]), w, yc - dly[k]);
                const float dz = __fmaf_rn(-(pu.y - dlz[k]), w, zc - dlz[k]);
                const float sc = __fmaf_rn(dz * dz, c.isz2, (dy * dy) * c.isy2);
                if (bu >= 0 && sc > best) continue;
                const int od = D.orig[dlj[k]];
                if (bu < 0 || sc < best || ou < bou || (ou == bou && od < bod)) {
                    best = sc;
                    bu = ju;
                    bd = dlj[k];
                    bou = ou;
                    bod = od;
                }
            }
        }
    }
    if (bu >= 0 && best <= gate) {
        out_u = U.s_off + bu;
        out_d = D.s_off + bd;
    }
}

// ============================================================================================
// A2, warp-cooperative search (stage_rows = 2).  A warp takes 32 clusters of row k, one per
// lane, and every lane finds the slot ranges of its windows in rows k-1 and k+1 (up to four cell
// rows each) and publishes them in a per-warp table in shared memory.  The candidates of all 32
// windows are then spread over the lanes: item i of the warp's flattened list goes to lane i mod
// 32, which finds its owner cluster by a binary search over the table's prefix offsets, tests
// the owner's window and, if the candidate is inside, appends it to a per-warp list (ballot
// compaction, in owner order).  The pairs are spread over the owners' row k+1 candidates: a lane
// takes one u, scores it against each of its owner's row k-1 candidates, keeps the best and
// offers it to the owner's running minimum with one 64-bit shared-memory atomicMin on (score,
// input index of u, input index of d; the indices relative to their rows, 16 bits each).  The
// lane whose offer is the minimum writes the pair's slots.  The best pair is the lexicographic
// minimum of the same key as in search_pairs, whatever the order, so the links are identical.
// Rows k-1 and k+1 are the CTA's shared-memory copies (or global memory when they do not fit).
// A window of more than four cell rows, or more in-window candidates than the lists hold, marks
// the warp's 32 clusters for k_neighbours_redo.  Rows of 65536 or more clusters use the
// per-thread form (the host checks).
// ============================================================================================
constexpr int kNbCap = 64;       // in-window candidates of one row kept per warp and 32 clusters
constexpr int kNbRedo = -2;      // link mark of a cluster left to k_neighbours_redo

// Slot ranges of one row inside the window: up to four cell rows along z, relative to the row.
struct CellRanges {
    int a0, a1, a2, a3;          // first slot of each cell row's range
    int p1, p2, p3, n;           // prefix counts: items [0, p1) in range 0, [p1, p2) in 1, ...
    bool over;                   // the window spans more than four cell rows
};

struct NbShared {
    int4 d[kNbCap], u[kNbCap];   // {slot within the row << 5 | owner lane, input index, y bits, z bits}
    int4 ra_d[32], rp_d[32];     // per lane: row k-1 ranges {a0..a3}, {p1, p2, p3, offset in the warp}
    int4 ra_u[32], rp_u[32];     // the same for row k+1
    float2 yz[32];               // per lane: the cluster
    int cnt_d[32], cnt_u[32];    // in-window candidates per owner
    int first_d[32];             // first row k-1 candidate of each owner in d
    unsigned long long best[32]; // per owner: (score bits << 32) | (u index << 16) | d index; ~0: none
    int b_su[32], b_sd[32];      // the best pair's slots within their rows
};

__device__ __forceinline__ CellRanges cell_ranges(const RowView &X, float yc, float zc, float wy, float wz)
{
    CellRanges r;
    const int iy0 = cell1(yc - wy - kBinSlack, X.ymin, X.idy, X.ny);
    const int iy1 = cell1(yc + wy + kBinSlack, X.ymin, X.idy, X.ny);
    const int iz0 = cell1(zc - wz - kBinSlack, X.zmin, X.idz, X.nz);
    const int iz1 = cell1(zc + wz + kBinSlack, X.zmin, X.idz, X.nz);
    const int32_t *c0 = X.cell + iz0 * X.ny;
    r.a0 = c0[iy0];
    const int e0 = c0[iy1 + 1];
    int e1 = 0, e2 = 0, e3 = 0;
    r.a1 = r.a2 = r.a3 = 0;
    if (iz1 > iz0) {
        r.a1 = c0[X.ny + iy0];
        e1 = c0[X.ny + iy1 + 1];
    }
    if (iz1 > iz0 + 1) {
        r.a2 = c0[2 * X.ny + iy0];
        e2 = c0[2 * X.ny + iy1 + 1];
    }
    if (iz1 > iz0 + 2) {
        r.a3 = c0[3 * X.ny + iy0];
        e3 = c0[3 * X.ny + iy1 + 1];
    }
    r.over = iz1 > iz0 + 3;
    r.p1 = e0 - r.a0;
    r.p2 = r.p1 + (e1 - r.a1);
    r.p3 = r.p2 + (e2 - r.a2);
    r.n = r.p3 + (e3 - r.a3);
    return r;
}

// Lane holding item i of a warp-flattened list: the last lane whose exclusive offset (rp[l].w)
// is <= i.
__device__ __forceinline__ int owner_of(const int4 *rp, int i)
{
    int lo = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1)
        if (rp[lo + s].w <= i) lo += s;              // lo + s <= 31
    return lo;
}

// Publishes the lane's ranges of row X and its offset in the warp's flattened list; returns
// the list's length.
__device__ __forceinline__ int publish(const CellRanges &cr, int4 *ra, int4 *rp, int lane)
{
    const int inc = warp_incl_scan(cr.n);
    ra[lane] = make_int4(cr.a0, cr.a1, cr.a2, cr.a3);
    rp[lane] = make_int4(cr.p1, cr.p2, cr.p3, inc - cr.n);
    return __shfl_sync(kFull, inc, 31);
}

// The in-window candidates of row X for the warp's 32 clusters, appended to list in owner order
// with their count per owner.  False (for the whole warp) if they do not fit.
__device__ __forceinline__ bool gather_row(const RowView &X, int tot, const int4 *ra, const int4 *rp,
                                           const float2 *yz, float wy, float wz, int4 *list, int *cnt, int lane)
{
    int used = 0;
    for (int base = 0; base < tot; base += 32) {
        const int i = base + lane;
        bool pass = false;
        int4 ent = make_int4(0, 0, 0, 0);
        int o = 0;
        if (i < tot) {
            o = owner_of(rp, i);
            const int4 a = ra[o], p = rp[o];
            const float2 co = yz[o];
            const int r = i - p.w;
            const int slot = r < p.x ? a.x + r : (r < p.y ? a.y + (r - p.x) : (r < p.z ? a.z + (r - p.y) : a.w + (r - p.z)));
            const float2 q = X.yz[slot];
            pass = fabsf(q.x - co.x) <= wy && fabsf(q.y - co.y) <= wz;
            if (pass) ent = make_int4((slot << 5) | o, X.orig[slot], __float_as_int(q.x), __float_as_int(q.y));
        }
        const unsigned m = __ballot_sync(kFull, pass);
        if (used + __popc(m) > kNbCap) return false;
        if (pass) {
            list[used + __popc(m & lanemask_lt())] = ent;
            atomicAdd(&cnt[o], 1);
        }
        used += __popc(m);
    }
    return true;
}

// Links of the warp's 32 clusters (lane: cluster at (yc, zc), v: the lane has one): slots of the
// best (u, d) pair within the gate, -1 for none, kNbRedo if the warp overflowed.  in_u, in_d:
// input offsets of rows k+1 and k-1.
__device__ __forceinline__ void coop_pairs(const DevConst &c, const RowView &U, const RowView &D, int in_u, int in_d,
                                           NbShared &S, int lane, bool v, float yc, float zc, float wyu, float wzu,
                                           float wyd, float wzd, float wgt, float gate, int &out_u, int &out_d)
{
    CellRanges cd{}, cu{};
    if (v) {
        cd = cell_ranges(D, yc, zc, wyd, wzd);
        cu = cell_ranges(U, yc, zc, wyu, wzu);
    }
    out_u = out_d = -1;
    if (__any_sync(kFull, cd.over || cu.over)) {
        out_u = out_d = kNbRedo;
        return;
    }
    S.yz[lane] = make_float2(yc, zc);
    S.cnt_d[lane] = 0;
    S.cnt_u[lane] = 0;
    S.best[lane] = ~0ull;
    const int tot_d = publish(cd, S.ra_d, S.rp_d, lane);
    const int tot_u = publish(cu, S.ra_u, S.rp_u, lane);
    __syncwarp();
    if (!gather_row(D, tot_d, S.ra_d, S.rp_d, S.yz, wyd, wzd, S.d, S.cnt_d, lane) ||
        !gather_row(U, tot_u, S.ra_u, S.rp_u, S.yz, wyu, wzu, S.u, S.cnt_u, lane)) {
        out_u = out_d = kNbRedo;
        __syncwarp();
        return;
    }
    __syncwarp();
    const int nd = S.cnt_d[lane];
    S.first_d[lane] = warp_incl_scan(nd) - nd;
    int n_u = S.cnt_u[lane];
    n_u = __shfl_sync(kFull, warp_incl_scan(n_u), 31);   // row k+1 candidates of the warp
    __syncwarp();
    for (int j = lane; j < n_u; j += 32) {
        const int4 eu = S.u[j];
        const int o = eu.x & 31;
        const int nd_o = S.cnt_d[o], f = S.first_d[o];
        const float puy = __int_as_float(eu.z), puz = __int_as_float(eu.w);
        const float2 co = S.yz[o];
        unsigned long long k = ~0ull;
        for (int q = f; q < f + nd_o; q++) {
            const int4 ed = S.d[q];
            const float pdy = __int_as_float(ed.z), pdz = __int_as_float(ed.w);
            // residual of c from the chord d -> u, evaluated at x_k (same order as the oracle)
            const float dy = __fmaf_rn(-(puy - pdy), wgt, co.x - pdy);
            const float dz = __fmaf_rn(-(puz - pdz), wgt, co.y - pdz);
            const float sc = __fmaf_rn(dz * dz, c.isz2, (dy * dy) * c.isy2);
            const unsigned long long kk = ((unsigned long long)__float_as_uint(sc) << 32) |
                                          ((unsigned long long)(eu.y - in_u) << 16) | (unsigned)(ed.y - in_d);
            if (kk < k) k = kk;
        }
        if (nd_o > 0) atomicMin(&S.best[o], k);
    }
    __syncwarp();
    // the u that won each owner's minimum (each u appears once per owner) writes the pair's slots
    for (int j = lane; j < n_u; j += 32) {
        const int4 eu = S.u[j];
        const int oo = eu.x & 31;
        const int nd_o = S.cnt_d[oo], f = S.first_d[oo];
        if (nd_o == 0) continue;
        const unsigned long long b = S.best[oo];
        if ((unsigned)((b >> 16) & 0xffff) != (unsigned)(eu.y - in_u)) continue;   // another u won
        const unsigned dl = (unsigned)(b & 0xffff);
        for (int q = f; q < f + nd_o; q++)
            if ((unsigned)(S.d[q].y - in_d) == dl) {
                S.b_su[oo] = eu.x >> 5;
                S.b_sd[oo] = S.d[q].x >> 5;
            }
    }
    __syncwarp();
    const unsigned long long b = S.best[lane];
    if (v && b != ~0ull && __uint_as_float((uint32_t)(b >> 32)) <= gate) {
        out_u = U.s_off + S.b_su[lane];
        out_d = D.s_off + S.b_sd[lane];
    }
    __syncwarp();                // the lists are reused by the next 32 clusters
}

// COOP = false: one thread per cluster (search_pairs); COOP = true: the warp-cooperative search.
// 5 CTAs per SM for the per-thread form (48 registers): more CTAs overlap one another's row
// staging (measured 6 % faster than 4).
template <bool COOP>
__global__ void __launch_bounds__(256, COOP ? 3 : 5)
k_neighbours(const DevConst c, const Workspace w, int64_t R, int smem_bytes, int stage)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t bar_idle;   // test hook: a barrier no copy and no thread completes
    __shared__ int abort_flag;
    __shared__ NbShared shm[COOP ? 8 : 1];       // the cooperative search's lists, one per warp
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&bar, 1);
        mbar_init(&bar_idle, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    for (int64_t u = blockIdx.x; u < R; u += gridDim.x) {
        const int r = (int)(u % c.nr);
        const int4 mk = w.meta[u];
        const int n = mk.y;
        if (n == 0) continue;
        const bool edge = (r == 0 || r == c.nr - 1);
        int4 mu = make_int4(0, 0, 0, 0), md = make_int4(0, 0, 0, 0);
        if (!edge) {
            mu = w.meta[u + 1];
            md = w.meta[u - 1];
        }
        if (edge || mu.y == 0 || md.y == 0) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                w.up_raw[mk.z + i] = -1;
                w.dn_raw[mk.z + i] = -1;
            }
            continue;
        }
        const int2 du = w.dims[u + 1], dd = w.dims[u - 1];
        const float4 gu = w.grid[u + 1], gd = w.grid[u - 1];
        RowView U{w.yz + mu.z, w.orig + mu.z, w.cell + mu.w, gu.x, gu.y, gu.z, gu.w, du.x, du.y, mu.y, mu.z};
        RowView D{w.yz + md.z, w.orig + md.z, w.cell + md.w, gd.x, gd.y, gd.z, gd.w, dd.x, dd.y, md.y, md.z};
        const int bytes_u = staged_row_bytes(mu.y, du.x * du.y);
        const int bytes_d = staged_row_bytes(md.y, dd.x * dd.y);
        const bool staged = stage && (bytes_u + bytes_d <= smem_bytes);
        if (staged) {
            unsigned char *p = sm;
            float2 *syz_u = (float2 *)p;
            p += round16(mu.y * 8);
            int32_t *sor_u = (int32_t *)p;
            p += round16(mu.y * 4);
            int32_t *sce_u = (int32_t *)p;
            p += round16((du.x * du.y + 1) * 4);
            float2 *syz_d = (float2 *)p;
            p += round16(md.y * 8);
            int32_t *sor_d = (int32_t *)p;
            p += round16(md.y * 4);
            int32_t *sce_d = (int32_t *)p;
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar, (unsigned)(bytes_u + bytes_d));
                bulk_g2s(syz_u, U.yz, round16(mu.y * 8), &bar);
                bulk_g2s(sor_u, U.orig, round16(mu.y * 4), &bar);
                bulk_g2s(sce_u, U.cell, round16((du.x * du.y + 1) * 4), &bar);
                bulk_g2s(syz_d, D.yz, round16(md.y * 8), &bar);
                bulk_g2s(sor_d, D.orig, round16(md.y * 4), &bar);
                bulk_g2s(sce_d, D.cell, round16((dd.x * dd.y + 1) * 4), &bar);
            }
            // one thread does the bounded wait and the CTA agrees on the outcome before anyone
            // leaves; then every thread passes the completed phase (acquire ordering)
            if (threadIdx.x == 0) {
                bool ok = mbar_wait_bounded(&bar, parity);
                if (!ok) {
                    // the copies did not complete in time and may still be landing: one more bounded
                    // wait for them before the CTA gives up its shared memory
                    mbar_wait_bounded(&bar, parity);
                } else if (c.inject == 1 && u == c.nr / 2) {
                    // test hook (sector 0's middle row): every copy of this CTA has landed; the wait
                    // on a barrier that nothing completes expires after the time limit, with no
                    // asynchronous copy outstanding, and the call reports TPC_ERR_TIMEOUT
                    ok = mbar_wait_bounded(&bar_idle, 0);
                }
                abort_flag = !ok;
                if (!ok) set_error(w.err, TPC_ERR_TIMEOUT, (int)u, c, TPC_STAGE_NEIGHBOURS);
            }
            __syncthreads();
            if (abort_flag) {
                // the staging gave up: this CTA writes "no link" for all its remaining clusters
                // (so later stages only ever follow valid slots) and stages nothing more
                for (int64_t v = u; v < R; v += gridDim.x) {
                    const int4 mv = w.meta[v];
                    for (int i = threadIdx.x; i < mv.y; i += blockDim.x) {
                        w.up_raw[mv.z + i] = -1;
                        w.dn_raw[mv.z + i] = -1;
                    }
                }
                return;
            }
            mbar_wait_bounded(&bar, parity);
            parity ^= 1u;
            U.yz = syz_u;
            U.orig = sor_u;
            U.cell = sce_u;
            D.yz = syz_d;
            D.orig = sor_d;
            D.cell = sce_d;
        }
        const float xk = c.row_x[r], xu = c.row_x[r + 1], xd = c.row_x[r - 1];
        const float dxu = xu - xk, dxd = xk - xd;
        const float wyu = c.ty * dxu, wzu = c.tz * dxu;
        const float wyd = c.ty * dxd, wzd = c.tz * dxd;
        const float wgt = dxd / (xu - xd);
        const float om = 1.0f - wgt;
        const float gate = c.gate9 * __fmaf_rn(wgt, wgt, __fmaf_rn(om, om, 1.0f));
        if (COOP) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int c0 = warp * 32; c0 < n; c0 += blockDim.x) {
                const int ci = c0 + lane;
                const bool v = ci < n;
                float2 pc = make_float2(0.0f, 0.0f);
                if (v) pc = w.yz[mk.z + ci];
                int ou, od;
                coop_pairs(c, U, D, mu.x, md.x, shm[warp], lane, v, pc.x, pc.y, wyu, wzu, wyd, wzd, wgt, gate, ou, od);
                if (v) {
                    w.up_raw[mk.z + ci] = ou;
                    w.dn_raw[mk.z + ci] = od;
                }
            }
        } else {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const float2 pc = w.yz[mk.z + i];
                int ou, od;
                search_pairs(c, U, D, pc.x, pc.y, wyu, wzu, wyd, wzd, wgt, gate, ou, od);
                w.up_raw[mk.z + i] = ou;
                w.dn_raw[mk.z + i] = od;
            }
        }
        __syncthreads();
    }
}

// The clusters that the cooperative search left to the per-thread search (windows of more than
// four cell rows, or more in-window candidates than its lists hold): search_pairs, one thread each.
__global__ void __launch_bounds__(256) k_neighbours_redo(const DevConst c, const Workspace w, int64_t R)
{
    for (int64_t u = blockIdx.x; u < R; u += gridDim.x) {
        const int4 mk = w.meta[u];
        for (int i = threadIdx.x; i < mk.y; i += blockDim.x) {
            if (w.up_raw[mk.z + i] != kNbRedo) continue;
            const int r = (int)(u % c.nr);
            const int4 mu = w.meta[u + 1], md = w.meta[u - 1];      // marked clusters have both rows
            const int2 du = w.dims[u + 1], dd = w.dims[u - 1];
            const float4 gu = w.grid[u + 1], gd = w.grid[u - 1];
            const RowView U{w.yz + mu.z, w.orig + mu.z, w.cell + mu.w, gu.x, gu.y, gu.z, gu.w, du.x, du.y, mu.y, mu.z};
            const RowView D{w.yz + md.z, w.orig + md.z, w.cell + md.w, gd.x, gd.y, gd.z, gd.w, dd.x, dd.y, md.y, md.z};
            const float xk = c.row_x[r], xu = c.row_x[r + 1], xd = c.row_x[r - 1];
            const float dxu = xu - xk, dxd = xk - xd;
            const float wgt = dxd / (xu - xd);
            const float om = 1.0f - wgt;
            const float gate = c.gate9 * __fmaf_rn(wgt, wgt, __fmaf_rn(om, om, 1.0f));
            const float2 pc = w.yz[mk.z + i];
            int ou, od;
            search_pairs(c, U, D, pc.x, pc.y, c.ty * dxu, c.tz * dxu, c.ty * dxd, c.tz * dxd, wgt, gate, ou, od);
            w.up_raw[mk.z + i] = ou;
            w.dn_raw[mk.z + i] = od;
        }
    }
}

int neighbours_smem_limit() { return 96 * 1024; }

int launch_neighbours(const DevConst &c, const Workspace &w, int64_t R, int smem_bytes, const LaunchCfg &lc,
                       cudaStream_t s)
{
    if (R == 0) return 0;
    // stage_rows: 0 per-thread search from global memory, 1 the same with rows k +- 1 staged,
    // 2 cooperative search on staged rows
    const int mode = (lc.stage_rows == 2 && lc.max_row_clusters >= 65536) ? 1 : lc.stage_rows;
    const int smem = mode ? smem_bytes : 0;
    int64_t grid = R;
    if (mode == 2) {
        if (grid > (int64_t)lc.num_sms * 24) grid = (int64_t)lc.num_sms * 24;
        if (smem > 48 * 1024 - (int)sizeof(NbShared) * 8)
            cudaFuncSetAttribute(k_neighbours<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_neighbours<true><<<(unsigned)grid, 256, smem, s>>>(c, w, R, smem, 1);
        k_neighbours_redo<<<(unsigned)grid, 256, 0, s>>>(c, w, R);
        return 2;
    }
    if (grid > (int64_t)lc.num_sms * 64) grid = (int64_t)lc.num_sms * 64;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_neighbours<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_neighbours<false><<<(unsigned)grid, lc.neighbours_block, smem, s>>>(c, w, R, smem, mode);
    return 1;
}

// ============================================================================================
// A3 evolution + A4 start hits.  A link survives only if it is reciprocal.  A start hit has a
// kept up link, no kept down link and a chain of >= min_chain clusters; its record holds the
// chain's first cluster and its length counted up to max(min_chain, 4).
// ============================================================================================
// One CTA per row unit, kEvolvePer clusters per thread in one pass (1024 per pass): the loads of
// all its clusters' links are issued together, then those of their partners, so that a pass waits
// for two round trips; the start candidates (kept up link, no kept down link) are gathered in
// shared memory and their chains are walked together afterwards, the next link's up index loaded
// with the current link's test, so that the walk waits for need - 1 more round trips per pass
// (need = max(min_chain, 4)) instead of each warp walking its chains in turn.
constexpr int kEvolveThreads = 256;
constexpr int kEvolvePer = 4;

__global__ void __launch_bounds__(kEvolveThreads) k_evolve(const DevConst c, const Workspace w, int64_t R)
{
    __shared__ int2 cand[kEvolveThreads * kEvolvePer];   // (candidate cluster, its kept up link)
    __shared__ int ncand;
    const int lane = threadIdx.x & 31;
    const int need = c.min_chain > 4 ? c.min_chain : 4;
    for (int64_t u = blockIdx.x; u < R; u += gridDim.x) {
        const int4 m = w.meta[u];
        const int n = m.y;
        const int r = (int)(u % c.nr);
        const int sec = (int)(u / c.nr);
        for (int i0 = 0; i0 < n; i0 += kEvolveThreads * kEvolvePer) {
            if (threadIdx.x == 0) ncand = 0;
            __syncthreads();
            int cl[kEvolvePer], u1[kEvolvePer], d1[kEvolvePer], bu[kEvolvePer], bd[kEvolvePer];
#pragma unroll
            for (int k = 0; k < kEvolvePer; k++) {
                const int i = i0 + k * kEvolveThreads + threadIdx.x;
                cl[k] = i < n ? m.z + i : -1;
                u1[k] = cl[k] >= 0 ? w.up_raw[cl[k]] : -1;
                d1[k] = cl[k] >= 0 ? w.dn_raw[cl[k]] : -1;
            }
#pragma unroll
            for (int k = 0; k < kEvolvePer; k++) {
                bu[k] = u1[k] >= 0 ? w.dn_raw[u1[k]] : -1;      // down link of the up partner
                bd[k] = d1[k] >= 0 ? w.up_raw[d1[k]] : -1;      // up link of the down partner
            }
#pragma unroll
            for (int k = 0; k < kEvolvePer; k++) {
                if (cl[k] < 0) continue;
                const int upk = (u1[k] >= 0 && bu[k] == cl[k]) ? u1[k] : -1;
                const int dnk = (d1[k] >= 0 && bd[k] == cl[k]) ? d1[k] : -1;
                w.up[cl[k]] = upk;
                w.dn[cl[k]] = dnk;
                if (upk >= 0 && dnk < 0) cand[atomicAdd(&ncand, 1)] = make_int2(cl[k], upk);
            }
            __syncthreads();
            // chain length of each candidate, counted only as far as the start test and the work
            // order need (min_chain, and >= 4 for the constructor's ordering key); the candidate and
            // its up link are the chain's first two clusters
            const int nc = ncand;
            for (int j0 = 0; j0 < nc; j0 += kEvolveThreads) {
                const int j = j0 + threadIdx.x;
                int first = -1, clen = 0;
                bool is_start = false;
                if (j < nc) {
                    const int2 e = cand[j];
                    int t = e.y, len = 2;
                    int nx = len < need ? w.up_raw[t] : -1;
                    while (len < need && nx >= 0) {
                        const int back = w.dn_raw[nx];
                        const int nn = len + 1 < need ? w.up_raw[nx] : -1;
                        if (back != t) break;
                        t = nx;
                        len++;
                        nx = nn;
                    }
                    if (len >= c.min_chain) {
                        is_start = true;
                        clen = len;
                        first = e.x;
                    }
                }
                const unsigned mask = __ballot_sync(kFull, is_start);
                int base = 0;
                if (lane == 0 && mask) base = atomicAdd(&w.counters[CNT_STARTS], __popc(mask));
                base = __shfl_sync(kFull, base, 0);
                if (is_start) {
                    const int slot = base + __popc(mask & lanemask_lt());
                    if (slot < w.tlim) {
                        w.starts[slot] = make_int4(first, -1, -1, (sec << 16) | (clen << 8) | r);
                    } else {
                        set_error(w.err, TPC_ERR_CAPACITY, (int)u, c, TPC_STAGE_EVOLUTION);
                    }
                }
            }
            __syncthreads();      // cand and ncand are reused by the next pass
        }
    }
}

int launch_evolve(const DevConst &c, const Workspace &w, int64_t R, cudaStream_t s)
{
    if (R == 0) return 0;
    int64_t grid = R < 65535 * 4 ? R : 65535 * 4;
    k_evolve<<<(unsigned)grid, kEvolveThreads, 0, s>>>(c, w, R);
    return 1;
}

}  // namespace tpc
