// Track merger with refit (Section 1: the sector tracks are merged by the track merger;
// Section 3.3: the merger refits every track from its cluster list, so equal cluster lists give
// bitwise equal results whatever rounding the sector tracker saw).
//
// 1. Every sector track is refitted from its clusters alone: seed from the circle through its
//    first, middle and last cluster (taken into the first cluster's frame), outward Kalman pass
//    with the seed covariance, inward pass with the covariance reset; the state changes frame
//    where the next cluster lies in a sector of another azimuth.  One thread per track; the next
//    cluster's data are loaded one step ahead.
// 2. A track's outer end is compared with the inner ends of the tracks of three sectors: the
//    same azimuth in the other z half and the two azimuth neighbours.  Gates: radial gap in
//    (0, gap], q/pT within n sigma, then the 5-parameter chi2 (Cholesky) of the outer state taken
//    into the other frame and transported to the other track's innermost cluster.  Each outer end
//    keeps its best partner; each inner end's best partner is a 64-bit atomicMin of
//    (chi2 bits, track).  Mutual best pairs merge; radii increase along a chain, so chains have no
//    cycles (the walks are bounded all the same).
// 3. One merged track per chain head, in the sector tracks' (canonical) order, with the chain's
//    clusters in order, refitted over all of them.
#include "kf.cuh"
#include "../../include/tpcca.h"

namespace tpc {

constexpr int kMergeBlock = 128;
constexpr int kMaxChain = 64;          // bound on a chain walk

struct MgIn {                          // the call's input clusters
    const float *y, *z;
    const uint8_t *row;
};

struct MgFit {
    KF in, out;                        // states at the innermost and outermost cluster
    float x_in, x_out, chi2, r_in, r_out;
    int s_in, s_out;                   // frame sectors (index within the call)
};

__device__ __forceinline__ int rot_steps(int from, int to) { return ((to % 18) - (from % 18) + 18) % 18; }

// Change of frame of the state to sector s_new (same azimuth: none).
__device__ __forceinline__ bool to_frame(const DevConst &c, KF &st, float &xs, int &sc, int s_new)
{
    const int d = rot_steps(sc, s_new);
    sc = s_new;
    if (d == 0) return true;
    float xn;
    if (!rotate_state(st, xs, c.crot[d], c.srot[d], c, xn)) return false;
    xs = xn;
    return true;
}

// One Kalman pass over h[0..n-1] in direction dir (every cluster used, no search).
__device__ __forceinline__ bool refit_pass(const DevConst &c, const MgIn &in, const int32_t *sec, const int32_t *h,
                                           int n, int dir, KF &st, float &xs, int &sc, float &chi2sum, bool sum)
{
    int i = dir > 0 ? 0 : n - 1;
    int cc = h[i];
    float yv = in.y[cc], zv = in.z[cc];
    int rv = in.row[cc], sv = sec[cc];
    for (int k = 0; k < n; k++) {
        // next cluster's data, loaded while this one is fitted
        const int in_next = i + dir;
        float yn = 0.0f, zn = 0.0f;
        int rn = 0, sn = 0;
        if (k + 1 < n) {
            const int cn = h[in_next];
            yn = in.y[cn];
            zn = in.z[cn];
            rn = in.row[cn];
            sn = sec[cn];
        }
        if (!to_frame(c, st, xs, sc, sv)) return false;
        const float xr = c.row_x[rv];
        if (xr != xs && !propagate(st, xr - xs, c)) return false;
        const Gain g = residual_cov_inv(st, c);
        if (sum) chi2sum = chi2sum + chi2_of(g, yv - st.p0, zv - st.p1);
        kf_update(st, g, yv, zv);
        xs = xr;
        i = in_next;
        yv = yn;
        zv = zn;
        rv = rn;
        sv = sn;
    }
    return true;
}

__device__ bool mg_refit(const DevConst &c, const MgIn &in, const int32_t *sec, const int32_t *h, int n, MgFit &o)
{
    if (n < 3) return false;
    const int s0 = sec[h[0]];
    float x3[3], y3[3], z3[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int cc = h[i == 0 ? 0 : (i == 1 ? (n - 1) / 2 : n - 1)];
        const int d = rot_steps(sec[cc], s0);
        const float x = c.row_x[in.row[cc]], yv = in.y[cc];
        const float cd = c.crot[d], sd = c.srot[d];
        x3[i] = d == 0 ? x : __fmaf_rn(x, cd, yv * sd);
        y3[i] = d == 0 ? yv : __fmaf_rn(yv, cd, -(x * sd));
        z3[i] = in.z[cc];
    }
    KF st;
    if (!seed3(x3, y3, z3, c, st)) return false;
    set_seed_cov(st, c);
    float xs = c.row_x[in.row[h[0]]];
    int sc = s0;
    float dummy = 0.0f;
    if (!refit_pass(c, in, sec, h, n, 1, st, xs, sc, dummy, false)) return false;
    o.out = st;
    o.x_out = xs;
    o.s_out = sc;
    set_seed_cov(st, c);
    float chi2 = 0.0f;
    if (!refit_pass(c, in, sec, h, n, -1, st, xs, sc, chi2, true)) return false;
    o.in = st;
    o.x_in = xs;
    o.s_in = sc;
    o.chi2 = chi2;
    const int ci = h[0], co = h[n - 1];
    const float xi = c.row_x[in.row[ci]], xo = c.row_x[in.row[co]];
    const float yi = in.y[ci], yo = in.y[co];
    o.r_in = sqrtf(__fmaf_rn(xi, xi, yi * yi));
    o.r_out = sqrtf(__fmaf_rn(xo, xo, yo * yo));
    return true;
}

// chi2 = d^T A^-1 d for a symmetric 5x5 A given as a lower triangle (row-major): Cholesky factor,
// forward substitution, squared norm; false if A is not positive definite.
__device__ __forceinline__ bool chi2_5(const float A[15], const float d[5], float &chi2)
{
    float L[15], u[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
#pragma unroll
        for (int j = 0; j <= i; j++) {
            float t = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int m = 0; m < j; m++) t = __fmaf_rn(-L[i * (i + 1) / 2 + m], L[j * (j + 1) / 2 + m], t);
            if (i == j) {
                if (!(t > 0.0f)) return false;
                L[i * (i + 1) / 2 + i] = sqrtf(t);
            } else {
                L[i * (i + 1) / 2 + j] = t / L[j * (j + 1) / 2 + j];
            }
        }
    }
    float q = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        float t = d[i];
#pragma unroll
        for (int m = 0; m < i; m++) t = __fmaf_rn(-L[i * (i + 1) / 2 + m], u[m], t);
        u[i] = t / L[i * (i + 1) / 2 + i];
        q = __fmaf_rn(u[i], u[i], q);
    }
    chi2 = q;
    return true;
}

__device__ __forceinline__ void kf_to15(const KF &s, float a[15])
{
    a[0] = s.c00; a[1] = s.c10; a[2] = s.c11; a[3] = s.c20; a[4] = s.c21; a[5] = s.c22; a[6] = s.c30;
    a[7] = s.c31; a[8] = s.c32; a[9] = s.c33; a[10] = s.c40; a[11] = s.c41; a[12] = s.c42; a[13] = s.c43;
    a[14] = s.c44;
}

__device__ __forceinline__ void kf_store(float *P, float *V, int64_t stride, int t, const KF &s)
{
    float a[15];
    kf_to15(s, a);
    P[0 * stride + t] = s.p0; P[1 * stride + t] = s.p1; P[2 * stride + t] = s.p2; P[3 * stride + t] = s.p3;
    P[4 * stride + t] = s.p4;
#pragma unroll
    for (int i = 0; i < 15; i++) V[i * stride + t] = a[i];
}

__device__ __forceinline__ void kf_load(const float *P, const float *V, int64_t stride, int t, KF &s)
{
    s.p0 = P[0 * stride + t]; s.p1 = P[1 * stride + t]; s.p2 = P[2 * stride + t]; s.p3 = P[3 * stride + t];
    s.p4 = P[4 * stride + t];
    s.c00 = V[0 * stride + t]; s.c10 = V[1 * stride + t]; s.c11 = V[2 * stride + t]; s.c20 = V[3 * stride + t];
    s.c21 = V[4 * stride + t]; s.c22 = V[5 * stride + t]; s.c30 = V[6 * stride + t]; s.c31 = V[7 * stride + t];
    s.c32 = V[8 * stride + t]; s.c33 = V[9 * stride + t]; s.c40 = V[10 * stride + t]; s.c41 = V[11 * stride + t];
    s.c42 = V[12 * stride + t]; s.c43 = V[13 * stride + t]; s.c44 = V[14 * stride + t];
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------

// Sector (index within the call) of every input cluster; the sector-track counts are kept.
__global__ void __launch_bounds__(256) k_mg_prep(const DevConst c, const Workspace w, int64_t R)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.counters[CNT_STRACKS] = w.counters[CNT_TRACKS];
        w.counters[CNT_SHITS] = w.counters[CNT_HITS];
    }
    for (int64_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < R; u += nwarps) {
        const int4 m = w.meta[u];
        const int s = (int)(u / c.nr);
        for (int i = lane; i < m.y; i += 32)
            if (TPC_IDX(m.x + i, w.pcap, w.err, c, 8)) w.in_sec[m.x + i] = s;
    }
}

// Refit of every sector track; tracks counted per inner sector.
__global__ void __launch_bounds__(kMergeBlock) k_mg_refit(const DevConst c, const Workspace w, const MgIn in)
{
    const int M = w.counters[CNT_TRACKS];
    const int64_t T = w.tcap;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        MgFit f;
        const bool ok = mg_refit(c, in, w.in_sec, w.st.hits + w.st.first[m], w.st.nhits[m], f);
        w.rf_ok[m] = ok ? 1 : 0;
        if (!ok) continue;
        kf_store(w.rf_P, w.rf_C, T, m, f.in);
        kf_store(w.rf_oP, w.rf_oC, T, m, f.out);
        w.rf_xin[m] = f.x_in;
        w.rf_xout[m] = f.x_out;
        w.rf_rin[m] = f.r_in;
        w.rf_rout[m] = f.r_out;
        w.rf_chi2[m] = f.chi2;
        w.rf_sin[m] = f.s_in;
        w.rf_sout[m] = f.s_out;
        atomicAdd(&w.mg_sec_cnt[f.s_in], 1);
    }
}

__global__ void __launch_bounds__(kMergeBlock) k_mg_scatter(const Workspace w)
{
    const int M = w.counters[CNT_TRACKS];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x)
        if (w.rf_ok[m]) {
            const int at = atomicAdd(&w.mg_sec_cur[w.rf_sin[m]], 1);
            if (TPC_IDX(at, w.tcap, w.err, c, 8)) w.mg_by_sec[at] = m;
        }
}

// chi2 of outer end `ar` (track a, already in b's frame at x = xa) with track b's inner end;
// false if the transport fails, the sum is not positive definite or the gate is not passed.
__device__ __forceinline__ bool match_pair(const DevConst &c, const Workspace &w, const KF &ar, float xa, int b,
                                           float &chi2)
{
    const int64_t T = w.tcap;
    const float xb = w.rf_xin[b];
    KF pr = ar;
    if (xa != xb && !propagate(pr, xb - xa, c)) return false;
    KF bs;
    kf_load(w.rf_P, w.rf_C, T, b, bs);
    float A[15], Bc[15], d[5];
    kf_to15(pr, A);
    kf_to15(bs, Bc);
#pragma unroll
    for (int i = 0; i < 15; i++) A[i] = A[i] + Bc[i];
    d[0] = bs.p0 - pr.p0;
    d[1] = bs.p1 - pr.p1;
    d[2] = bs.p2 - pr.p2;
    d[3] = bs.p3 - pr.p3;
    d[4] = bs.p4 - pr.p4;
    return chi2_5(A, d, chi2) && chi2 <= c.mchi2;
}

// Best partner of every outer end; best partner of every inner end by atomicMin.  One warp per
// outer end: the lanes sweep the candidate sectors' lists 32 tracks at a time (coalesced index
// loads) through the cheap gates (radial gap, q/pT); the survivors go to a per-warp queue in
// shared memory, and whenever it holds 32 of them the whole warp runs the transport and the
// chi2, so the expensive part executes with all lanes busy.  The warp's best is the minimum of
// (chi2 bits, track) over its lanes; chi2 >= 0, so the bits order like the values and equal chi2
// go to the lower track, whatever order the candidates were evaluated in.
constexpr int kMatchWarps = kMergeBlock / 32;

__global__ void __launch_bounds__(kMergeBlock) k_mg_match(const DevConst c, const Workspace w)
{
    __shared__ int queue[kMatchWarps][64];
    const int M = w.counters[CNT_TRACKS];
    const int64_t T = w.tcap;
    const int lane = threadIdx.x & 31;
    int *qu = queue[threadIdx.x >> 5];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < M; a += nwarps) {
        unsigned long long best = ~0ull;
        if (w.rf_ok[a]) {
            const int sa = w.rf_sout[a];
            const int ev = sa / 36, side = (sa % 36) / 18, az = sa % 18;
            const float r_out = w.rf_rout[a];
            const float aq = w.rf_oP[4 * T + a], ac44 = w.rf_oC[14 * T + a];   // unchanged by the rotation
            for (int q = 0; q < 3; q++) {
                const int sb = ev * 36 + (q == 0 ? (1 - side) * 18 + az
                                                 : side * 18 + (q == 1 ? (az + 1) % 18 : (az + 17) % 18));
                const int b0 = w.mg_sec_first[sb], b1 = w.mg_sec_first[sb + 1];
                if (b0 == b1) continue;
                KF ar;
                kf_load(w.rf_oP, w.rf_oC, T, a, ar);
                float xa = w.rf_xout[a];
                int sc = sa;
                if (!to_frame(c, ar, xa, sc, sb)) continue;       // the same for every lane
                int count = 0;                                      // warp-uniform queue length
                for (int i0 = b0; i0 < b1; i0 += 32) {
                    const int ib = i0 + lane;
                    const int b = ib < b1 ? w.mg_by_sec[ib] : a;
                    bool pass = b != a;
                    if (pass) {
                        const float gap = w.rf_rin[b] - r_out;
                        pass = gap > 0.0f && gap <= c.mgap;
                    }
                    if (pass) {
                        const float dq = w.rf_P[4 * T + b] - aq;
                        pass = dq * dq <= c.mq2 * (ac44 + w.rf_C[14 * T + b]);
                    }
                    const unsigned mask = __ballot_sync(kFull, pass);
                    if (pass) qu[count + __popc(mask & lanemask_lt())] = b;
                    count += __popc(mask);
                    __syncwarp();
                    if (count >= 32) {
                        const int bb = qu[count - 32 + lane];
                        float chi2;
                        if (match_pair(c, w, ar, xa, bb, chi2)) {
                            const unsigned long long key = ((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)bb;
                            if (key < best) best = key;
                            atomicMin(&w.mg_bkey[bb], ((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)a);
                        }
                        count -= 32;
                        __syncwarp();
                    }
                }
                if (lane < count) {
                    const int bb = qu[lane];
                    float chi2;
                    if (match_pair(c, w, ar, xa, bb, chi2)) {
                        const unsigned long long key = ((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)bb;
                        if (key < best) best = key;
                        atomicMin(&w.mg_bkey[bb], ((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)a);
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(kFull, best, o);
            if (other < best) best = other;
        }
        if (lane == 0) w.mg_best[a] = best == ~0ull ? -1 : (int)(best & 0xffffffffull);
    }
}

__global__ void __launch_bounds__(256) k_mg_link(const Workspace w)
{
    const int M = w.counters[CNT_TRACKS];
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < M; a += gridDim.x * blockDim.x) {
        const int b = w.mg_best[a];
        const int nx = (b >= 0 && (int)(w.mg_bkey[b] & 0xffffffffull) == a) ? b : -1;
        w.mg_next[a] = nx;
        if (nx >= 0) w.mg_prev[nx] = a;
    }
}

// Chain heads and their cluster counts.
__global__ void __launch_bounds__(256) k_mg_heads(const Workspace w)
{
    const int M = w.counters[CNT_TRACKS];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const bool head = w.mg_prev[m] < 0;
        int n = 0;
        if (head) {
            int t = m;
            for (int k = 0; k < kMaxChain && t >= 0; k++, t = w.mg_next[t]) n += w.st.nhits[t];
        }
        w.mg_head[m] = head ? 1 : 0;
        w.mg_cnt[m] = n;
    }
}

// Merged tracks: cluster lists and bookkeeping (one warp per chain head).
__global__ void __launch_bounds__(256) k_mg_write(const Workspace w, const OutBuffers o)
{
    const int M = w.counters[CNT_STRACKS];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += nwarps) {
        if (w.mg_prev[m] >= 0) continue;
        const int j = w.mg_idx[m];
        const int f = w.mg_first[m];
        if (!TPC_IDX(j, o.mcap, w.err, c, 8)) continue;
        int pos = f, nseg = 0, t = m;
        for (int k = 0; k < kMaxChain && t >= 0; k++, t = w.mg_next[t]) {
            const int n = w.st.nhits[t], s0 = w.st.first[t];
            for (int i = lane; i < n; i += 32)
                if (TPC_IDX(pos + i, o.hcap, w.err, c, 8)) o.hits[pos + i] = w.st.hits[s0 + i];
            pos += n;
            nseg++;
        }
        if (lane == 0) {
            o.first[j] = f;
            o.nhits[j] = pos - f;
            o.event[j] = w.st.event[m];
            w.mg_nseg[j] = nseg;
            w.mg_headof[j] = m;
        }
    }
}

// Parameters of the merged tracks: refit over the chain's clusters (a lone track keeps its refit;
// a failed refit keeps the sector tracker's parameters).
__global__ void __launch_bounds__(kMergeBlock) k_mg_fit(const DevConst c, const Workspace w, const MgIn in,
                                                        const OutBuffers o)
{
    const int Mm = w.counters[CNT_TRACKS];
    const int64_t T = w.tcap;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Mm; j += gridDim.x * blockDim.x) {
        const int m = w.mg_headof[j];
        const int n = o.nhits[j];
        MgFit f;
        bool ok;
        if (w.mg_nseg[j] > 1) {
            ok = mg_refit(c, in, w.in_sec, o.hits + o.first[j], n, f);
        } else {
            ok = w.rf_ok[m] != 0;
            if (ok) {
                kf_load(w.rf_P, w.rf_C, T, m, f.in);
                f.x_in = w.rf_xin[m];
                f.chi2 = w.rf_chi2[m];
                f.s_in = w.rf_sin[m];
            }
        }
        if (ok) {
            float a[15];
            kf_to15(f.in, a);
            o.par[(int64_t)j * 5 + 0] = f.in.p0;
            o.par[(int64_t)j * 5 + 1] = f.in.p1;
            o.par[(int64_t)j * 5 + 2] = f.in.p2;
            o.par[(int64_t)j * 5 + 3] = f.in.p3;
            o.par[(int64_t)j * 5 + 4] = f.in.p4;
#pragma unroll
            for (int i = 0; i < 15; i++) o.cov[(int64_t)j * 15 + i] = a[i];
            const int sector = f.s_in % c.ns;
            o.x[j] = f.x_in;
            o.chi2[j] = f.chi2;
            o.ndf[j] = 2 * n - 5;
            o.sector[j] = sector;
            o.alpha[j] = c.sec_alpha[sector];
        } else {
#pragma unroll
            for (int i = 0; i < 5; i++) o.par[(int64_t)j * 5 + i] = w.st.par[(int64_t)m * 5 + i];
#pragma unroll
            for (int i = 0; i < 15; i++) o.cov[(int64_t)j * 15 + i] = w.st.cov[(int64_t)m * 15 + i];
            o.x[j] = w.st.x[m];
            o.chi2[j] = w.st.chi2[m];
            o.ndf[j] = w.st.ndf[m];
            o.sector[j] = w.st.sector[m];
            o.alpha[j] = w.st.alpha[m];
        }
    }
}

int launch_merge(const DevConst &c, const Workspace &w, const OutBuffers &o, const float *y, const float *z,
                 const uint8_t *row, int64_t R, const LaunchCfg &lc, cudaStream_t s)
{
    const int64_t S = R / c.nr;                     // sectors of the call
    const MgIn in{y, z, row};
    const int grid = lc.num_sms * 8;
    int launches = 0;
    cudaMemsetAsync(w.mg_sec_cnt, 0, (size_t)(S + 1) * sizeof(int32_t), s);
    cudaMemsetAsync(w.mg_prev, 0xff, (size_t)w.tcap * sizeof(int32_t), s);
    cudaMemsetAsync(w.mg_bkey, 0xff, (size_t)w.tcap * sizeof(unsigned long long), s);
    k_mg_prep<<<grid, 256, 0, s>>>(c, w, R);
    k_mg_refit<<<lc.num_sms * 16, kMergeBlock, 0, s>>>(c, w, in);
    launches += 2;
    launches += launch_scan_i32(w.mg_sec_cnt, w.mg_sec_first, S + 1, nullptr, w.scan_tmp, nullptr, s);
    cudaMemcpyAsync(w.mg_sec_cur, w.mg_sec_first, (size_t)(S + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    k_mg_scatter<<<grid, kMergeBlock, 0, s>>>(w);
    k_mg_match<<<lc.num_sms * 16, kMergeBlock, 0, s>>>(c, w);       // one warp per track
    k_mg_link<<<grid, 256, 0, s>>>(w);
    k_mg_heads<<<grid, 256, 0, s>>>(w);
    launches += 4;
    // merged count and index of every head; cluster offsets; both scanned over the sector tracks
    launches += launch_scan_i32(w.mg_head, w.mg_idx, w.tcap, w.counters + CNT_STRACKS, w.scan_tmp,
                                w.counters + CNT_TRACKS, s);
    launches += launch_scan_i32(w.mg_cnt, w.mg_first, w.tcap, w.counters + CNT_STRACKS, w.scan_tmp,
                                w.counters + CNT_HITS, s);
    k_mg_write<<<grid, 256, 0, s>>>(w, o);
    k_mg_fit<<<lc.num_sms * 16, kMergeBlock, 0, s>>>(c, w, in, o);
    launches += 2;
    return launches;
}

}  // namespace tpc
