// A5 tracklet construction, sector-sweep variant.
//
// The tracklets of one sector are split into chunks; a CTA takes a chunk and walks the sector's
// pad rows in lockstep: outwards from the chunk's lowest start row to the last row, then inwards
// from the highest outermost cluster to row 0.  At each step the row is staged into shared memory
// with bulk async copies (double-buffered, the next row is in flight while the current one is
// searched), the tracklets that visit this row are compacted onto the CTA's threads, and each
// visit runs the same arithmetic as the work-queue constructor (kf.cuh).  Each tracklet therefore
// visits exactly the rows, in exactly the order, and with exactly the operations of the other
// constructor; only the schedule differs.  Tracklet states live in shared memory between steps.
#include "kf.cuh"
#include "../../include/tpcca.h"

namespace tpc {

constexpr int kSwThreads = 256;
constexpr int kSwChunk = 640;                  // tracklets per chunk at most
constexpr int kSwRowBytes = 16 * 1024;         // one staging buffer

enum { SW_PENDING = 0, SW_UP = 1, SW_WAIT = 2, SW_DOWN = 3, SW_DONE = 4 };

struct SwState {                               // shared memory, structure of arrays
    float p[5][kSwChunk];
    float cv[15][kSwChunk];
    float xs[kSwChunk];
    float chi[kSwChunk];
    int phase[kSwChunk];
    int r0[kSwChunk];
    int rlast[kSwChunk];
    int miss[kSwChunk];
    int n[kSwChunk];
    int t[kSwChunk];
    int orig0[kSwChunk];
    int list[kSwChunk];
    int nlist[2], left[2];                     // per step parity: step r uses [r & 1]
    int lo, hi, abort;
};

__device__ __forceinline__ uint32_t sw_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool sw_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sw_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait on an mbarrier phase for at most kWaitNs of device time; false if it gave up.
__device__ __forceinline__ bool sw_wait(uint64_t *bar, unsigned parity)
{
    if (sw_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!sw_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void sw_bulk(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sw_smem(dst)),
                 "l"(src), "r"(bytes), "r"(sw_smem(bar))
                 : "memory");
}

__host__ __device__ __forceinline__ int sw_r16(int b) { return (b + 15) & ~15; }

// Bytes of the staged copy of one row unit (slots, input indices, cell starts), 0 if it does not
// fit a staging buffer (the row is then read from global memory).
__device__ __forceinline__ int sw_row_bytes(int n, int nc)
{
    const int b = sw_r16(n * 8) + sw_r16(n * 4) + sw_r16((nc + 1) * 4);
    return (n > 0 && b <= kSwRowBytes) ? b : 0;
}

// Issue the staging copies of unit u into buf (one thread).  Returns the bytes in flight.
__device__ __forceinline__ int sw_stage(const Workspace &w, int u, unsigned char *buf, uint64_t *bar)
{
    const int n = w.meta[u].y;
    const int4 rg = w.rgi[u];
    const int nc = rg.z * rg.w;
    const int bytes = sw_row_bytes(n, nc);
    if (!bytes) return 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sw_smem(bar)), "r"((unsigned)bytes)
                 : "memory");
    sw_bulk(buf, w.yz + rg.x, sw_r16(n * 8), bar);
    sw_bulk(buf + sw_r16(n * 8), w.orig + rg.x, sw_r16(n * 4), bar);
    sw_bulk(buf + sw_r16(n * 8) + sw_r16(n * 4), w.cell + rg.y, sw_r16((nc + 1) * 4), bar);
    return bytes;
}

__device__ __forceinline__ void sw_load(const SwState &S, int i, KF &k)
{
    k.p0 = S.p[0][i]; k.p1 = S.p[1][i]; k.p2 = S.p[2][i]; k.p3 = S.p[3][i]; k.p4 = S.p[4][i];
    k.c00 = S.cv[0][i]; k.c10 = S.cv[1][i]; k.c11 = S.cv[2][i]; k.c20 = S.cv[3][i]; k.c21 = S.cv[4][i];
    k.c22 = S.cv[5][i]; k.c30 = S.cv[6][i]; k.c31 = S.cv[7][i]; k.c32 = S.cv[8][i]; k.c33 = S.cv[9][i];
    k.c40 = S.cv[10][i]; k.c41 = S.cv[11][i]; k.c42 = S.cv[12][i]; k.c43 = S.cv[13][i]; k.c44 = S.cv[14][i];
}

__device__ __forceinline__ void sw_store(SwState &S, int i, const KF &k)
{
    S.p[0][i] = k.p0; S.p[1][i] = k.p1; S.p[2][i] = k.p2; S.p[3][i] = k.p3; S.p[4][i] = k.p4;
    S.cv[0][i] = k.c00; S.cv[1][i] = k.c10; S.cv[2][i] = k.c11; S.cv[3][i] = k.c20; S.cv[4][i] = k.c21;
    S.cv[5][i] = k.c22; S.cv[6][i] = k.c30; S.cv[7][i] = k.c31; S.cv[8][i] = k.c32; S.cv[9][i] = k.c33;
    S.cv[10][i] = k.c40; S.cv[11][i] = k.c41; S.cv[12][i] = k.c42; S.cv[13][i] = k.c43; S.cv[14][i] = k.c44;
}

// ---------------------------------------------------------------------------------------------
// planning: tracklets grouped by sector, cut into chunks sized so the chunks fill the GPU once
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sw_hist(const Workspace w)
{
    const int T = n_tracklets(w);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        atomicAdd(&w.sw_sec[w.starts[t].w >> 16], 1);
}

__global__ void __launch_bounds__(1024) k_sw_plan(const Workspace w, int n_sec, int slots)
{
    __shared__ int sh[33];
    __shared__ int carry_t, carry_c;
    const int T = n_tracklets(w);
    // per-sector rounding adds up to n_sec chunks: size them for slots - n_sec (at least half the slots)
    int eff = slots - n_sec;
    if (eff < slots / 2) eff = slots / 2;
    if (eff < 1) eff = 1;
    int ch = (T + eff - 1) / eff;
    ch = (ch + 31) & ~31;
    ch = ch < 32 ? 32 : (ch > kSwChunk ? kSwChunk : ch);
    if (threadIdx.x == 0) {
        carry_t = 0;
        carry_c = 0;
    }
    __syncthreads();
    for (int s0 = 0; s0 < n_sec; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const int cnt = s < n_sec ? w.sw_sec[s] : 0;
        const int nch = (cnt + ch - 1) / ch;
        // two block scans: tracklet offsets and chunk offsets
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int a = warp_incl_scan(cnt), b = warp_incl_scan(nch);
        if (lane == 31) sh[warp] = a;
        __syncthreads();
        if (warp == 0) {
            const int x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
            const int xi = warp_incl_scan(x);
            sh[lane] = xi - x;
        }
        __syncthreads();
        const int toff = carry_t + sh[warp] + a - cnt;
        __syncthreads();
        if (lane == 31) sh[warp] = b;
        __syncthreads();
        if (warp == 0) {
            const int x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
            const int xi = warp_incl_scan(x);
            sh[lane] = xi - x;
        }
        __syncthreads();
        const int coff = carry_c + sh[warp] + b - nch;
        if (s < n_sec) {
            w.sw_sec[n_sec + s] = toff;            // scatter cursor
            for (int k = 0; k < nch; k++) {
                const int beg = k * ch;
                w.sw_chunks[coff + k] = make_int4(s, toff + beg, cnt - beg < ch ? cnt - beg : ch, 0);
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            carry_t = toff + cnt;
            carry_c = coff + nch;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) w.counters[CNT_SW_CHUNKS] = carry_c;
}

__global__ void __launch_bounds__(256) k_sw_scatter(const Workspace w, int n_sec)
{
    const int T = n_tracklets(w);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&w.sw_sec[n_sec + (w.starts[t].w >> 16)], 1);
        if (TPC_IDX(pos, T, w.err, c, 4)) w.order[pos] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSwThreads, 2) k_construct_sweep(const DevConst c, const Workspace w)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    SwState &S = *reinterpret_cast<SwState *>(sm_raw);
    unsigned char *rowbuf[2] = {sm_raw + sw_r16(sizeof(SwState)), sm_raw + sw_r16(sizeof(SwState)) + kSwRowBytes};
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int chunk_id;
    __shared__ int staged[2];
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sw_smem(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sw_smem(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    unsigned par[2] = {0u, 0u};
    int visits = 0, cands = 0;
    const int nchunks = w.counters[CNT_SW_CHUNKS];
    __syncthreads();
    while (true) {
        if (tid == 0) chunk_id = atomicAdd(&w.counters[CNT_QUEUE], 1);
        __syncthreads();
        const int ci = chunk_id;
        if (ci >= nchunks) break;
        const int4 ck = w.sw_chunks[ci];
        const int sec = ck.x, beg = ck.y, cnt = ck.z;
        if (tid == 0) {
            S.lo = c.nr;
            S.hi = -1;
            S.abort = 0;
        }
        __syncthreads();
        // seeds
        for (int i = tid; i < cnt; i += blockDim.x) {
            const int t = w.order[beg + i];
            const int4 sd = w.starts[t];
            KF st;
            S.t[i] = t;
            S.orig0[i] = w.orig[sd.x];
            w.tl_n[t] = 0;
            w.tl_key[t] = 0ull;
            if (seed_tracklet(c, w, sd, st)) {
                const int r0 = sd.w & 0xff;
                sw_store(S, i, st);
                S.phase[i] = SW_PENDING;
                S.r0[i] = r0;
                S.xs[i] = c.row_x[r0];
                S.rlast[i] = -1;
                S.miss[i] = 0;
                S.n[i] = 0;
                S.chi[i] = 0.0f;
                atomicMin(&S.lo, r0);
            } else {
                S.phase[i] = SW_DONE;
            }
        }
        __syncthreads();
        for (int dir = 0; dir < 2; dir++) {
            const int up = dir == 0;
            const int rbeg = up ? S.lo : S.hi;
            const int rend = up ? c.nr : -1;
            const int step = up ? 1 : -1;
            // first row of the sweep
            if (tid == 0) {
                S.nlist[0] = S.nlist[1] = 0;
                S.left[0] = S.left[1] = 0;
                if (rbeg != rend && rbeg >= 0 && rbeg < c.nr)
                    staged[rbeg & 1] = sw_stage(w, sec * c.nr + rbeg, rowbuf[rbeg & 1], &bar[rbeg & 1]);
            }
            __syncthreads();
            for (int r = rbeg; r != rend && r >= 0 && r < c.nr; r += step) {
                const int b = r & 1;
                // prefetch the next row into the other buffer (its last reader finished at the
                // barrier that ended the previous step)
                const int rn = r + step;
                const int sp = r & 1;                  // this step's list counters
                if (tid == 0 && rn >= 0 && rn < c.nr)
                    staged[rn & 1] = sw_stage(w, sec * c.nr + rn, rowbuf[rn & 1], &bar[rn & 1]);
                // tracklets that visit row r: activation at their first row, then every row until they stop
                for (int i = tid; i < cnt; i += blockDim.x) {
                    int ph = S.phase[i];
                    if (up && ph == SW_PENDING && S.r0[i] == r) ph = S.phase[i] = SW_UP;
                    if (!up && ph == SW_WAIT && S.rlast[i] == r) {
                        ph = S.phase[i] = SW_DOWN;
                        S.n[i] = 0;
                        S.chi[i] = 0.0f;
                        S.miss[i] = 0;
                    }
                    const bool act = ph == (up ? SW_UP : SW_DOWN);
                    const bool wait = (up && ph == SW_PENDING) || (!up && ph == SW_WAIT);
                    // one shared atomic per warp for the list slots and the waiting count
                    const unsigned am = __ballot_sync(__activemask(), act);
                    const unsigned wm = __ballot_sync(__activemask(), wait);
                    const int lane = tid & 31;
                    const int leader = __ffs(__activemask()) - 1;
                    int base = 0;
                    if (lane == leader) {
                        if (am) base = atomicAdd(&S.nlist[sp], __popc(am));
                        if (wm) atomicAdd(&S.left[sp], __popc(wm));
                    }
                    base = __shfl_sync(__activemask(), base, leader);
                    if (act) S.list[base + __popc(am & lanemask_lt())] = i;
                }
                __syncthreads();
                const int nact = S.nlist[sp];
                const int left = S.left[sp];
                // the other parity's counters were last read before this step's barrier: clear them
                if (tid == 0) {
                    S.nlist[sp ^ 1] = 0;
                    S.left[sp ^ 1] = 0;
                }
                const int bytes = staged[b];
                if (bytes) {
                    // one thread does the bounded wait; the CTA agrees on the outcome before anyone
                    // leaves, then every thread passes the (completed) phase for acquire ordering
                    if (tid == 0) {
                        const bool ok = sw_wait(&bar[b], par[b]);
                        S.abort = !ok;
                        if (!ok) {
                            set_error(w.err, TPC_ERR_TIMEOUT, sec * c.nr + r, c, TPC_STAGE_CONSTRUCTION);
                            sw_wait(&bar[b], par[b]);   // let the copies land before leaving
                        }
                    }
                    __syncthreads();
                    if (S.abort) return;
                    sw_wait(&bar[b], par[b]);
                    par[b] ^= 1u;
                }
                const int u = sec * c.nr + r;
                const int4 rg = __ldg(&w.rgi[u]);
                const float4 gr = __ldg(&w.grid[u]);
                const int n = w.meta[u].y;
                const float2 *yz = bytes ? (const float2 *)rowbuf[b] : w.yz + rg.x;
                const int32_t *og = bytes ? (const int32_t *)(rowbuf[b] + sw_r16(n * 8)) : w.orig + rg.x;
                const int32_t *ce = bytes ? (const int32_t *)(rowbuf[b] + sw_r16(n * 8) + sw_r16(n * 4)) : w.cell + rg.y;
                const float xr = c.row_x[r];
                for (int j = tid; j < nact; j += blockDim.x) {
                    const int i = S.list[j];
                    KF st;
                    sw_load(S, i, st);
                    const float xs = S.xs[i];
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
                        float2 q;
                        const int bl = n > 0 ? search_cells(c, yz, og, ce, gr, rg.z, rg.w, pr, g, chi2, q, cands) : -1;
                        if (bl >= 0 && chi2 <= c.chi2max) {
                            if (!up) {
                                S.chi[i] = S.chi[i] + chi2;
                                if (TPC_IDX(S.n[i], c.nr, w.err, c, 4))
                                    w.tl_hits[(int64_t)S.t[i] * c.nr + S.n[i]] = rg.x + bl;
                                S.n[i] = S.n[i] + 1;
                            } else {
                                S.rlast[i] = r;
                            }
                            kf_update(pr, g, q.x, q.y);
                            sw_store(S, i, pr);
                            S.xs[i] = xr;
                            S.miss[i] = 0;
                        } else if (++S.miss[i] >= c.max_miss) {
                            stop = true;
                        }
                    }
                    if (stop) {
                        if (up) {
                            if (S.rlast[i] < 0) {
                                S.phase[i] = SW_DONE;
                            } else {
                                KF rs;
                                sw_load(S, i, rs);
                                if (c.global) write_outer(w, S.t[i], rs, S.xs[i]);
                                set_seed_cov(rs, c);
                                sw_store(S, i, rs);
                                S.phase[i] = SW_WAIT;
                                atomicMax(&S.hi, S.rlast[i]);
                            }
                        } else {
                            KF fs;
                            sw_load(S, i, fs);
                            write_tracklet(c, w, S.t[i], fs, S.xs[i], S.n[i], S.chi[i], S.orig0[i]);
                            S.phase[i] = SW_DONE;
                        }
                    }
                }
                __syncthreads();
                if (nact == 0 && left == 0) {
                    // nothing left in this direction: drain the prefetch still in flight, then stop
                    if (rn >= 0 && rn < c.nr && staged[rn & 1]) {
                        if (tid == 0) sw_wait(&bar[rn & 1], par[rn & 1]);
                        par[rn & 1] ^= 1u;
                    }
                    __syncthreads();
                    break;
                }
            }
            __syncthreads();
            // passes still running at the end of the sweep stop there
            for (int i = tid; i < cnt; i += blockDim.x) {
                if (up && S.phase[i] == SW_UP) {
                    if (S.rlast[i] < 0) {
                        S.phase[i] = SW_DONE;
                    } else {
                        KF rs;
                        sw_load(S, i, rs);
                        if (c.global) write_outer(w, S.t[i], rs, S.xs[i]);
                        set_seed_cov(rs, c);
                        sw_store(S, i, rs);
                        S.phase[i] = SW_WAIT;
                        atomicMax(&S.hi, S.rlast[i]);
                    }
                }
                if (!up && S.phase[i] == SW_DOWN) {
                    KF fs;
                    sw_load(S, i, fs);
                    write_tracklet(c, w, S.t[i], fs, S.xs[i], S.n[i], S.chi[i], S.orig0[i]);
                    S.phase[i] = SW_DONE;
                }
            }
            __syncthreads();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        visits += __shfl_xor_sync(kFull, visits, o);
        cands += __shfl_xor_sync(kFull, cands, o);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&w.counters[CNT_VISITS], visits);
        atomicAdd(&w.counters[CNT_CANDS], cands);
    }
}

size_t sweep_smem_bytes() { return sw_r16(sizeof(SwState)) + 2 * kSwRowBytes; }

int launch_construct_sweep(const DevConst &c, const Workspace &w, int n_sec, const LaunchCfg &lc, cudaStream_t s)
{
    const int per_sm = 2;
    const size_t smem = sweep_smem_bytes();
    cudaFuncSetAttribute(k_construct_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaMemsetAsync(w.sw_sec, 0, (size_t)n_sec * sizeof(int32_t), s);
    const int g = lc.num_sms * 2;
    k_sw_hist<<<g, 256, 0, s>>>(w);
    k_sw_plan<<<1, 1024, 0, s>>>(w, n_sec, lc.num_sms * per_sm);
    k_sw_scatter<<<g, 256, 0, s>>>(w, n_sec);
    k_construct_sweep<<<lc.num_sms * per_sm, kSwThreads, smem, s>>>(c, w);
    return 4;
}

}  // namespace tpc
