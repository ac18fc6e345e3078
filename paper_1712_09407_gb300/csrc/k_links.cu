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
// One warp per row unit; the sort is stable in input order.
// ============================================================================================
constexpr int kIngestWarps = 4;

__global__ void __launch_bounds__(kIngestWarps * 32)
k_ingest(const DevConst c, const Workspace w, const float *__restrict__ yin, const float *__restrict__ zin,
         const uint8_t *__restrict__ rin, int64_t R)
{
    extern __shared__ int sh_hist[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *hist = sh_hist + warp * kCellMax;
    for (int64_t u = (int64_t)blockIdx.x * kIngestWarps + warp; u < R; u += (int64_t)gridDim.x * kIngestWarps) {
        const int4 m = w.meta[u];
        const int2 d = w.dims[u];
        const int in_off = m.x, n = m.y, s_off = m.z, cell_off = m.w;
        const int ny = d.x, nz = d.y, nc = ny * nz;
        const int r = (int)(u % c.nr);
        float ymin = FLT_MAX, ymax = -FLT_MAX, zmin = FLT_MAX, zmax = -FLT_MAX;
        int bad = 0;
        for (int i = lane; i < n; i += 32) {
            float y = __ldg(yin + in_off + i), z = __ldg(zin + in_off + i);
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
            float y = __ldg(yin + in_off + i), z = __ldg(zin + in_off + i);
            int cc = cell1(z, zmin, idz, nz) * ny + cell1(y, ymin, idy, ny);
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
                y = __ldg(yin + in_off + i);
                z = __ldg(zin + in_off + i);
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
    k_ingest<<<(unsigned)blocks, kIngestWarps * 32, kIngestWarps * kCellMax * sizeof(int), s>>>(c, w, y, z, row, R);
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

// 5 CTAs per SM (48 registers): more CTAs overlap one another's row staging (measured 6 % faster than 4)
__global__ void __launch_bounds__(256, 5)
k_neighbours(const DevConst c, const Workspace w, int64_t R, int smem_bytes, int stage)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t bar_idle;   // test hook: a barrier no copy and no thread completes
    __shared__ int abort_flag;
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
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float2 pc = w.yz[mk.z + i];
            int ou, od;
            search_pairs(c, U, D, pc.x, pc.y, wyu, wzu, wyd, wzd, wgt, gate, ou, od);
            w.up_raw[mk.z + i] = ou;
            w.dn_raw[mk.z + i] = od;
        }
        __syncthreads();
    }
}

int neighbours_smem_limit() { return 96 * 1024; }

int launch_neighbours(const DevConst &c, const Workspace &w, int64_t R, int smem_bytes, const LaunchCfg &lc,
                       cudaStream_t s)
{
    if (R == 0) return 0;
    int block = lc.neighbours_block;
    int64_t grid = R;
    if (grid > (int64_t)lc.num_sms * 64) grid = (int64_t)lc.num_sms * 64;
    int smem = lc.stage_rows ? smem_bytes : 0;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_neighbours, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_neighbours<<<(unsigned)grid, block, smem, s>>>(c, w, R, smem, lc.stage_rows);
    return 1;
}

// ============================================================================================
// A3 evolution + A4 start hits.  A link survives only if it is reciprocal.  A start hit has a
// kept up link, no kept down link and a chain of >= min_chain clusters; its record holds the
// chain's first cluster and its length counted up to max(min_chain, 4).
// ============================================================================================
__global__ void __launch_bounds__(256) k_evolve(const DevConst c, const Workspace w, int64_t R)
{
    const int lane = threadIdx.x & 31;
    for (int64_t u = blockIdx.x; u < R; u += gridDim.x) {
        const int4 m = w.meta[u];
        const int n = m.y;
        const int r = (int)(u % c.nr);
        const int sec = (int)(u / c.nr);
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            const bool v = i < n;
            int first = -1, clen = 0;
            bool is_start = false;
            if (v) {
                const int cl = m.z + i;
                const int u1 = w.up_raw[cl], d1 = w.dn_raw[cl];
                const int upk = (u1 >= 0 && w.dn_raw[u1] == cl) ? u1 : -1;
                const int dnk = (d1 >= 0 && w.up_raw[d1] == cl) ? d1 : -1;
                w.up[cl] = upk;
                w.dn[cl] = dnk;
                if (upk >= 0 && dnk < 0) {
                    // chain length, counted only as far as the start test and the work order need
                    // (min_chain, and >= 4 for the constructor's ordering key); the constructor walks
                    // the whole chain for its seed
                    const int need = c.min_chain > 4 ? c.min_chain : 4;
                    int len = 1, t = cl;
                    while (len < need) {
                        const int nx = w.up_raw[t];
                        if (nx < 0 || w.dn_raw[nx] != t) break;
                        t = nx;
                        len++;
                    }
                    if (len >= c.min_chain) {
                        is_start = true;
                        clen = len;
                        first = cl;
                    }
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
    }
}

int launch_evolve(const DevConst &c, const Workspace &w, int64_t R, cudaStream_t s)
{
    if (R == 0) return 0;
    int64_t grid = R < 65535 * 4 ? R : 65535 * 4;
    k_evolve<<<(unsigned)grid, 128, 0, s>>>(c, w, R);
    return 1;
}

}  // namespace tpc
