// Kalman-filter pieces of the tracklet construction (Section 1, "Tracklet construction"), shared
// by the two constructor kernels.  Expressions follow the same operation order as the CPU
// oracle's float mode, with the same fused multiply-adds written out (the library is otherwise
// compiled without FMA contraction), so both evaluate identical roundings.
#pragma once
#include "common.cuh"

namespace tpc {

struct KF {
    float p0, p1, p2, p3, p4;
    // lower triangle of the covariance, row-major
    float c00, c10, c11, c20, c21, c22, c30, c31, c32, c33, c40, c41, c42, c43, c44;
};

// asin(u)/u with a fixed series, so that every float implementation of the tracker rounds the
// same way (cluster ownership is decided by comparing weights): Maclaurin series of arcsin,
// asin(u)/u = sum_n (2n)! / (4^n (n!)^2 (2n+1)) u^(2n), twelve terms by Horner's rule for
// |u| <= 0.5, larger |u| reduced with asin(u) = 2 asin(u / sqrt(2 (1 + sqrt(1 - u^2)))).
__device__ __forceinline__ float asin_ratio(float u)
{
    float v = u, m = 1.0f;
    for (int k = 0; k < 3 && fabsf(v) > 0.5f; k++) {
        v = v / sqrtf(2.0f * (1.0f + sqrtf(1.0f - v * v)));
        m = m * 2.0f;
    }
    const float t = v * v;
    float s = 0.007312526f;
    s = __fmaf_rn(s, t, 0.00839033537f);
    s = __fmaf_rn(s, t, 0.00976160914f);
    s = __fmaf_rn(s, t, 0.0115518011f);
    s = __fmaf_rn(s, t, 0.0139648439f);
    s = __fmaf_rn(s, t, 0.0173527636f);
    s = __fmaf_rn(s, t, 0.0223721582f);
    s = __fmaf_rn(s, t, 0.030381944f);
    s = __fmaf_rn(s, t, 0.0446428582f);
    s = __fmaf_rn(s, t, 0.075000003f);
    s = __fmaf_rn(s, t, 0.166666672f);
    s = __fmaf_rn(s, t, 1.0f);
    if (m == 1.0f) return s;
    return ((m * v) * s) / u;
}

// Exact helix transport by dx with covariance C <- F C F^T (F: Jacobian of the transport).
// Fused multiply-adds are written out (__fmaf_rn) in the same places as in the oracle.
__device__ __forceinline__ bool propagate(KF &s, float dx, const DevConst &c)
{
    const float cur = c.kB * s.p4;
    const float s0 = s.p2;
    const float s1 = __fmaf_rn(cur, dx, s0);
    if (!(fabsf(s1) < c.smax)) return false;
    const float c0 = sqrtf(__fmaf_rn(-s0, s0, 1.0f));
    const float c1 = sqrtf(__fmaf_rn(-s1, s1, 1.0f));
    const float A = s0 + s1;
    const float B = c0 + c1;
    const float iB = 1.0f / B;
    const float tq = A * iB;
    const float dy = dx * tq;
    float L = sqrtf(__fmaf_rn(dx, dx, dy * dy));
    if (dx < 0.0f) L = -L;
    const float u = (cur * L) * 0.5f;
    const float ratio = asin_ratio(u);
    const float dS = L * ratio;
    const float tl = s.p3;
    const float iBB = iB * iB;       // one reciprocal of (c0 + c1) for the slope and both denominators
    const float s1c1 = s1 / c1;
    const float F02 = dx * __fmaf_rn(A, s0 / c0 + s1c1, 2.0f * B) * iBB;
    const float F04 = dx * (c.kB * dx) * __fmaf_rn(A, s1c1, B) * iBB;
    const float F24 = c.kB * dx;
    const float g = (L != 0.0f) ? dy / (L * sqrtf(__fmaf_rn(-u, u, 1.0f))) : 0.0f;
    const float F12 = tl * (g * F02);
    const float F13 = dS;
    const float F14 = tl * __fmaf_rn(g, F04, (((cur * L) * (L * L)) * 0.0833333358f) * c.kB);   // 1/12 rounded to float

    s.p0 = s.p0 + dy;
    s.p1 = __fmaf_rn(tl, dS, s.p1);
    s.p2 = s1;

    // FC = F C, row by row (k ascending, zero terms dropped, unit terms exact)
    const float C00 = s.c00, C01 = s.c10, C02 = s.c20, C03 = s.c30, C04 = s.c40;
    const float C11 = s.c11, C12 = s.c21, C13 = s.c31, C14 = s.c41;
    const float C22 = s.c22, C23 = s.c32, C24 = s.c42;
    const float C33 = s.c33, C34 = s.c43, C44 = s.c44;
    const float FC00 = __fmaf_rn(F04, C04, __fmaf_rn(F02, C02, C00));
    const float FC02 = __fmaf_rn(F04, C24, __fmaf_rn(F02, C22, C02));
    const float FC04 = __fmaf_rn(F04, C44, __fmaf_rn(F02, C24, C04));
    const float FC10 = __fmaf_rn(F14, C04, __fmaf_rn(F13, C03, __fmaf_rn(F12, C02, C01)));
    const float FC11 = __fmaf_rn(F14, C14, __fmaf_rn(F13, C13, __fmaf_rn(F12, C12, C11)));
    const float FC12 = __fmaf_rn(F14, C24, __fmaf_rn(F13, C23, __fmaf_rn(F12, C22, C12)));
    const float FC13 = __fmaf_rn(F14, C34, __fmaf_rn(F13, C33, __fmaf_rn(F12, C23, C13)));
    const float FC14 = __fmaf_rn(F14, C44, __fmaf_rn(F13, C34, __fmaf_rn(F12, C24, C14)));
    const float FC20 = __fmaf_rn(F24, C04, C02);
    const float FC21 = __fmaf_rn(F24, C14, C12);
    const float FC22 = __fmaf_rn(F24, C24, C22);
    const float FC23 = __fmaf_rn(F24, C34, C23);
    const float FC24 = __fmaf_rn(F24, C44, C24);
    // N = FC F^T, lower triangle (k ascending)
    s.c00 = __fmaf_rn(FC04, F04, __fmaf_rn(FC02, F02, FC00));
    s.c10 = __fmaf_rn(FC14, F04, __fmaf_rn(FC12, F02, FC10));
    s.c11 = __fmaf_rn(FC14, F14, __fmaf_rn(FC13, F13, __fmaf_rn(FC12, F12, FC11)));
    s.c20 = __fmaf_rn(FC24, F04, __fmaf_rn(FC22, F02, FC20));
    s.c21 = __fmaf_rn(FC24, F14, __fmaf_rn(FC23, F13, __fmaf_rn(FC22, F12, FC21)));
    s.c22 = __fmaf_rn(FC24, F24, FC22);
    s.c30 = __fmaf_rn(C34, F04, __fmaf_rn(C23, F02, C03));
    s.c31 = __fmaf_rn(C34, F14, __fmaf_rn(C33, F13, __fmaf_rn(C23, F12, C13)));
    s.c32 = __fmaf_rn(C34, F24, C23);
    // s.c33 unchanged
    s.c40 = __fmaf_rn(C44, F04, __fmaf_rn(C24, F02, C04));
    s.c41 = __fmaf_rn(C44, F14, __fmaf_rn(C34, F13, __fmaf_rn(C24, F12, C14)));
    s.c42 = __fmaf_rn(C44, F24, C24);
    // s.c43, s.c44 unchanged
    return true;
}

struct Gain {
    float s00, s01, s10, s11;   // inverse residual covariance
};

__device__ __forceinline__ Gain residual_cov_inv(const KF &s, const DevConst &c)
{
    const float S00 = s.c00 + c.sy2, S01 = s.c10, S10 = s.c10, S11 = s.c11 + c.sz2;
    const float det = __fmaf_rn(S00, S11, -S01 * S10);
    const float idet = 1.0f / det;
    Gain g;
    g.s00 = S11 * idet;
    g.s01 = -S01 * idet;
    g.s10 = -S10 * idet;
    g.s11 = S00 * idet;
    return g;
}

__device__ __forceinline__ float chi2_of(const Gain &g, float r0, float r1)
{
    const float t0 = __fmaf_rn(g.s01, r1, g.s00 * r0);
    const float t1 = __fmaf_rn(g.s11, r1, g.s10 * r0);
    return __fmaf_rn(r1, t1, r0 * t0);
}

__device__ __forceinline__ void kf_update(KF &s, const Gain &g, float my, float mz)
{
    const float r0 = my - s.p0, r1 = mz - s.p1;
    // K = C H^T S^-1
    const float K00 = __fmaf_rn(s.c10, g.s10, s.c00 * g.s00), K01 = __fmaf_rn(s.c10, g.s11, s.c00 * g.s01);
    const float K10 = __fmaf_rn(s.c11, g.s10, s.c10 * g.s00), K11 = __fmaf_rn(s.c11, g.s11, s.c10 * g.s01);
    const float K20 = __fmaf_rn(s.c21, g.s10, s.c20 * g.s00), K21 = __fmaf_rn(s.c21, g.s11, s.c20 * g.s01);
    const float K30 = __fmaf_rn(s.c31, g.s10, s.c30 * g.s00), K31 = __fmaf_rn(s.c31, g.s11, s.c30 * g.s01);
    const float K40 = __fmaf_rn(s.c41, g.s10, s.c40 * g.s00), K41 = __fmaf_rn(s.c41, g.s11, s.c40 * g.s01);
    s.p0 = __fmaf_rn(K01, r1, __fmaf_rn(K00, r0, s.p0));
    s.p1 = __fmaf_rn(K11, r1, __fmaf_rn(K10, r0, s.p1));
    s.p2 = __fmaf_rn(K21, r1, __fmaf_rn(K20, r0, s.p2));
    s.p3 = __fmaf_rn(K31, r1, __fmaf_rn(K30, r0, s.p3));
    s.p4 = __fmaf_rn(K41, r1, __fmaf_rn(K40, r0, s.p4));
    // C <- C - K H C (rows 0 and 1 of C are C(0, j) and C(1, j))
    const float A0 = s.c00, A1 = s.c10, A2 = s.c20, A3 = s.c30, A4 = s.c40;   // C(0, j)
    const float B0 = s.c10, B1 = s.c11, B2 = s.c21, B3 = s.c31, B4 = s.c41;   // C(1, j)
    s.c00 = __fmaf_rn(-K01, B0, __fmaf_rn(-K00, A0, s.c00));
    s.c10 = __fmaf_rn(-K11, B0, __fmaf_rn(-K10, A0, s.c10));
    s.c11 = __fmaf_rn(-K11, B1, __fmaf_rn(-K10, A1, s.c11));
    s.c20 = __fmaf_rn(-K21, B0, __fmaf_rn(-K20, A0, s.c20));
    s.c21 = __fmaf_rn(-K21, B1, __fmaf_rn(-K20, A1, s.c21));
    s.c22 = __fmaf_rn(-K21, B2, __fmaf_rn(-K20, A2, s.c22));
    s.c30 = __fmaf_rn(-K31, B0, __fmaf_rn(-K30, A0, s.c30));
    s.c31 = __fmaf_rn(-K31, B1, __fmaf_rn(-K30, A1, s.c31));
    s.c32 = __fmaf_rn(-K31, B2, __fmaf_rn(-K30, A2, s.c32));
    s.c33 = __fmaf_rn(-K31, B3, __fmaf_rn(-K30, A3, s.c33));
    s.c40 = __fmaf_rn(-K41, B0, __fmaf_rn(-K40, A0, s.c40));
    s.c41 = __fmaf_rn(-K41, B1, __fmaf_rn(-K40, A1, s.c41));
    s.c42 = __fmaf_rn(-K41, B2, __fmaf_rn(-K40, A2, s.c42));
    s.c43 = __fmaf_rn(-K41, B3, __fmaf_rn(-K40, A3, s.c43));
    s.c44 = __fmaf_rn(-K41, B4, __fmaf_rn(-K40, A4, s.c44));
}

__device__ __forceinline__ void set_seed_cov(KF &s, const DevConst &c)
{
    s.c00 = c.cov0[0];
    s.c10 = 0.0f;
    s.c11 = c.cov0[1];
    s.c20 = s.c21 = 0.0f;
    s.c22 = c.cov0[2];
    s.c30 = s.c31 = s.c32 = 0.0f;
    s.c33 = c.cov0[3];
    s.c40 = s.c41 = s.c42 = s.c43 = 0.0f;
    s.c44 = c.cov0[4];
}

// Circle through the (x, y) of three chain points; tan lambda from the z rise over the arc.
__device__ __forceinline__ bool seed3(const float x[3], const float y[3], const float z[3], const DevConst &c,
                                      KF &s)
{
    const float ax = x[1] - x[0], ay = y[1] - y[0];
    const float bx = x[2] - x[0], by = y[2] - y[0];
    const float cx = x[2] - x[1], cy = y[2] - y[1];
    const float la = sqrtf(ax * ax + ay * ay);
    const float lb = sqrtf(bx * bx + by * by);
    const float lc = sqrtf(cx * cx + cy * cy);
    const float cross = ax * by - ay * bx;
    const float den = (la * lb) * lc;
    if (!(den > 0.0f)) return false;
    const float C = (2.0f * cross) / den;
    const float sa = (C * lb) * 0.5f;
    if (!(fabsf(sa) < 1.0f)) return false;
    const float ca = sqrtf(1.0f - sa * sa);
    const float sinphi = (by / lb) * ca - (bx / lb) * sa;
    if (!(fabsf(sinphi) < c.smax)) return false;
    const float S02 = lb * asin_ratio(sa);
    s.p0 = y[0];
    s.p1 = z[0];
    s.p2 = sinphi;
    s.p3 = (z[2] - z[0]) / S02;
    s.p4 = (c.kB != 0.0f) ? C / c.kB : 0.0f;
    return true;
}

// Running minimum of a row search: the lowest chi2, ties to the lower input index.
struct BestCand {
    int best = -1, borig = -1;       // borig: input index of the best slot, loaded on the first tie
    float bc = 0.0f;
    float2 bq = make_float2(0.0f, 0.0f);

    __device__ __forceinline__ void offer(int k, float2 q, float x2, const int32_t *orig)
    {
        if (best < 0 || x2 < bc) {
            best = k;
            bc = x2;
            bq = q;
            borig = -1;
        } else if (x2 == bc) {
            if (borig < 0) borig = orig[best];
            const int o = orig[k];
            if (o < borig) {
                best = k;
                bq = q;
                borig = o;
            }
        }
    }
};

// Best cluster of one row for a predicted state: minimum chi2 inside the window, ties to the
// lower input index.  yz, orig, cell point at the row's slots and cell starts (global memory or a
// shared-memory copy); gr = {ymin, zmin, 1/dy, 1/dz}, ny, nz its grid.  Returns the slot index
// within the row, or -1; the best cluster's (y, z) in best_yz.  used (optional): clusters with a
// nonzero byte are skipped.
//
// Candidates are visited cell row by cell row (iz ascending, slots ascending) in one flat loop:
// an iteration tests one candidate and moves on to the next non-empty cell row within the same
// iteration, so a warp runs as many iterations as its busiest lane has candidates, instead of
// the sum over cell rows of the busiest lane in each (nested loops) or one more iteration per
// cell row (a loop whose iterations either move or test).
__device__ __forceinline__ int search_cells(const DevConst &c, const float2 *yz, const int32_t *orig,
                                            const int32_t *cell, const float4 gr, int ny, int nz, const KF &pr,
                                            const Gain &g, float &chi2_out, float2 &best_yz, int &ncand,
                                            const uint8_t *used = nullptr)
{
    const float wy = c.nsig * sqrtf(pr.c00 + c.sy2);
    const float wz = c.nsig * sqrtf(pr.c11 + c.sz2);
    const float y = pr.p0, z = pr.p1;
    const int iy0 = cell1(y - wy - kBinSlack, gr.x, gr.z, ny);
    const int iy1 = cell1(y + wy + kBinSlack, gr.x, gr.z, ny);
    const int iz0 = cell1(z - wz - kBinSlack, gr.y, gr.w, nz);
    const int iz1 = cell1(z + wz + kBinSlack, gr.y, gr.w, nz);
    BestCand b;
    int iz = iz0 - 1, j = 0, e = 0;
    while (j >= e && iz < iz1) {                    // first non-empty cell row
        ++iz;
        j = cell[iz * ny + iy0];
        e = cell[iz * ny + iy1 + 1];
        ncand += e - j;
    }
    while (j < e) {
        const int k = j++;
        const float2 q = yz[k];                     // issued together with the used[] load
        while (j >= e && iz < iz1) {                // next non-empty cell row, in the same iteration
            ++iz;
            j = cell[iz * ny + iy0];
            e = cell[iz * ny + iy1 + 1];
            ncand += e - j;
        }
        if (used && used[k]) continue;
        if (!(fabsf(q.x - y) <= wy && fabsf(q.y - z) <= wz)) continue;
        b.offer(k, q, chi2_of(g, q.x - y, q.y - z), orig);
    }
    chi2_out = b.bc;
    best_yz = b.bq;
    return b.best;
}

// The same row search for rows in global memory, arranged for memory-level parallelism: the slot
// ranges of the window's first three cell rows are loaded together, then the candidates are
// loaded CB at a time before any of them is tested, so that a visit waits for about two or three
// L2 round trips instead of one per candidate and per cell row.  Cell rows beyond the third
// (windows wider than three cells in z, rare) follow one at a time.  The best cluster is the
// lexicographic minimum of (chi2, input index) over the same candidates, whatever order they are
// offered in, so the result is identical to search_cells.  Statistics: ncand counts the clusters
// of every enumerated cell, as there.  USED: clusters with a nonzero byte in used are skipped and
// the best cluster's (y, z) is returned in best_yz (global tracking); otherwise best_yz is left.
template <int CB, bool USED = false>
__device__ __forceinline__ int search_cells_mlp(const DevConst &c, const float2 *__restrict__ yz,
                                                const int32_t *__restrict__ orig, const int32_t *__restrict__ cell,
                                                const float4 gr, int ny, int nz, const KF &pr, const Gain &g,
                                                float &chi2_out, int &ncand, const uint8_t *__restrict__ used = nullptr,
                                                float2 *best_yz = nullptr)
{
    const float wy = c.nsig * sqrtf(pr.c00 + c.sy2);
    const float wz = c.nsig * sqrtf(pr.c11 + c.sz2);
    const float y = pr.p0, z = pr.p1;
    const int iy0 = cell1(y - wy - kBinSlack, gr.x, gr.z, ny);
    const int iy1 = cell1(y + wy + kBinSlack, gr.x, gr.z, ny);
    const int iz0 = cell1(z - wz - kBinSlack, gr.y, gr.w, nz);
    const int iz1 = cell1(z + wz + kBinSlack, gr.y, gr.w, nz);
    const int32_t *c0 = cell + iz0 * ny;
    const int a0 = __ldg(c0 + iy0), e0 = __ldg(c0 + iy1 + 1);
    int a1 = 0, e1 = 0, a2 = 0, e2 = 0;
    if (iz1 > iz0) {
        a1 = __ldg(c0 + ny + iy0);
        e1 = __ldg(c0 + ny + iy1 + 1);
    }
    if (iz1 > iz0 + 1) {
        a2 = __ldg(c0 + 2 * ny + iy0);
        e2 = __ldg(c0 + 2 * ny + iy1 + 1);
    }
    const int n0 = e0 - a0, n01 = n0 + (e1 - a1), n = n01 + (e2 - a2);
    ncand += n;
    BestCand b;
    for (int i0 = 0; i0 < n; i0 += CB) {
        int sl[CB];
        float2 q[CB];
#pragma unroll
        for (int k = 0; k < CB; k++) {
            const int i = i0 + k;
            sl[k] = i < n0 ? a0 + i : (i < n01 ? a1 + (i - n0) : a2 + (i - n01));
        }
        uint8_t uk[CB];
#pragma unroll
        for (int k = 0; k < CB; k++) {
            q[k] = i0 + k < n ? __ldg(yz + sl[k]) : make_float2(0.0f, 0.0f);
            if (USED) uk[k] = i0 + k < n ? __ldg(used + sl[k]) : (uint8_t)1;
        }
#pragma unroll
        for (int k = 0; k < CB; k++) {
            if (i0 + k < n && (!USED || !uk[k]) && fabsf(q[k].x - y) <= wy && fabsf(q[k].y - z) <= wz)
                b.offer(sl[k], q[k], chi2_of(g, q[k].x - y, q[k].y - z), orig);
        }
    }
    for (int iz = iz0 + 3; iz <= iz1; iz++) {
        const int a = __ldg(cell + iz * ny + iy0), e = __ldg(cell + iz * ny + iy1 + 1);
        ncand += e - a;
        for (int k = a; k < e; k++) {
            if (USED && __ldg(used + k)) continue;
            const float2 q = __ldg(yz + k);
            if (fabsf(q.x - y) <= wy && fabsf(q.y - z) <= wz) b.offer(k, q, chi2_of(g, q.x - y, q.y - z), orig);
        }
    }
    chi2_out = b.bc;
    if (USED) *best_yz = b.bq;
    return b.best;
}

// Writes a finished tracklet: state at its innermost fitted cluster, chi2, weight and the 64-bit
// claim key used by the selection (Section 3.1: w = n (alpha - chi2/beta), chi2 read per degree
// of freedom; ties to the lower input index of the start cluster).
__device__ __forceinline__ void write_tracklet(const DevConst &c, const Workspace &w, int t, const KF &st, float xs,
                                               int n, float chi2sum, int orig0)
{
    const int tcap = (int)w.tcap;
    const int ndf = 2 * n - 5;
    w.tl_n[t] = n;
    w.tl_x[t] = xs;
    w.tl_chi2[t] = chi2sum;
    float *P = w.tl_par;
    P[0 * tcap + t] = st.p0;
    P[1 * tcap + t] = st.p1;
    P[2 * tcap + t] = st.p2;
    P[3 * tcap + t] = st.p3;
    P[4 * tcap + t] = st.p4;
    float *V = w.tl_cov;
    V[0 * tcap + t] = st.c00;
    V[1 * tcap + t] = st.c10;
    V[2 * tcap + t] = st.c11;
    V[3 * tcap + t] = st.c20;
    V[4 * tcap + t] = st.c21;
    V[5 * tcap + t] = st.c22;
    V[6 * tcap + t] = st.c30;
    V[7 * tcap + t] = st.c31;
    V[8 * tcap + t] = st.c32;
    V[9 * tcap + t] = st.c33;
    V[10 * tcap + t] = st.c40;
    V[11 * tcap + t] = st.c41;
    V[12 * tcap + t] = st.c42;
    V[13 * tcap + t] = st.c43;
    V[14 * tcap + t] = st.c44;
    if (ndf >= 1) {
        const float wt = (float)n * (c.alpha - (chi2sum / (float)ndf) / c.beta);
        w.tl_w[t] = wt;
        w.tl_key[t] = ((unsigned long long)ordered_bits(wt) << 32) | (unsigned)(~orig0);
    } else {
        w.tl_w[t] = -INFINITY;
    }
}

// State of the outward pass at its last cluster: the track's outer end for global tracking.
__device__ __forceinline__ void write_outer(const Workspace &w, int t, const KF &st, float xs)
{
    const int tcap = (int)w.tcap;
    float *P = w.tl_opar, *V = w.tl_ocov;
    P[0 * tcap + t] = st.p0; P[1 * tcap + t] = st.p1; P[2 * tcap + t] = st.p2; P[3 * tcap + t] = st.p3;
    P[4 * tcap + t] = st.p4;
    V[0 * tcap + t] = st.c00; V[1 * tcap + t] = st.c10; V[2 * tcap + t] = st.c11; V[3 * tcap + t] = st.c20;
    V[4 * tcap + t] = st.c21; V[5 * tcap + t] = st.c22; V[6 * tcap + t] = st.c30; V[7 * tcap + t] = st.c31;
    V[8 * tcap + t] = st.c32; V[9 * tcap + t] = st.c33; V[10 * tcap + t] = st.c40; V[11 * tcap + t] = st.c41;
    V[12 * tcap + t] = st.c42; V[13 * tcap + t] = st.c43; V[14 * tcap + t] = st.c44;
    w.tl_ox[t] = xs;
}

// Change of frame by an azimuth rotation (cos cd, sin sd), same operations as the oracle: the state at
// x is re-expressed at x' = x cd + y sd (y' = -x sd + y cd, phi' = phi - angle); the covariance is
// transported with the Jacobian of the map to fixed x'.  False if cos(phi') <= 0 or |sin phi'| >= smax.
__device__ __forceinline__ bool rotate_state(KF &s, float x, float cd, float sd, const DevConst &c, float &x_new)
{
    const float y = s.p0, sp = s.p2;
    const float cp = sqrtf(__fmaf_rn(-sp, sp, 1.0f));
    const float xn = __fmaf_rn(x, cd, y * sd);
    const float yn = __fmaf_rn(y, cd, -(x * sd));
    const float spn = __fmaf_rn(sp, cd, -(cp * sd));
    if (!(fabsf(spn) < c.smax)) return false;
    if (!(__fmaf_rn(cp, cd, sp * sd) > 0.0f)) return false;
    const float cpn = sqrtf(__fmaf_rn(-spn, spn, 1.0f));
    const float J00 = __fmaf_rn(-sd, spn / cpn, cd);
    const float J10 = -(sd * s.p3) / cpn;
    const float J20 = -(c.kB * s.p4) * sd;
    const float J22 = cpn / cp;
    s.p0 = yn;
    s.p2 = spn;
    // J C, rows (only rows 0, 1, 2 differ from C)
    const float C00 = s.c00, C01 = s.c10, C02 = s.c20, C03 = s.c30, C04 = s.c40;
    const float C11 = s.c11, C12 = s.c21, C13 = s.c31, C14 = s.c41;
    const float C22 = s.c22, C23 = s.c32, C24 = s.c42;
    const float JC00 = J00 * C00;    // only column 0 of row 0 enters the lower triangle
    const float JC10 = __fmaf_rn(1.0f, C01, J10 * C00), JC11 = __fmaf_rn(1.0f, C11, J10 * C01);
    const float JC12 = __fmaf_rn(1.0f, C12, J10 * C02), JC13 = __fmaf_rn(1.0f, C13, J10 * C03);
    const float JC14 = __fmaf_rn(1.0f, C14, J10 * C04);
    const float JC20 = __fmaf_rn(J22, C02, J20 * C00), JC21 = __fmaf_rn(J22, C12, J20 * C01);
    const float JC22 = __fmaf_rn(J22, C22, J20 * C02), JC23 = __fmaf_rn(J22, C23, J20 * C03);
    const float JC24 = __fmaf_rn(J22, C24, J20 * C04);
    // (J C) J^T, lower triangle; rows 3, 4 of J C are rows 3, 4 of C
    s.c00 = JC00 * J00;
    s.c10 = JC10 * J00;
    s.c11 = __fmaf_rn(JC11, 1.0f, JC10 * J10);
    s.c20 = JC20 * J00;
    s.c21 = __fmaf_rn(JC21, 1.0f, JC20 * J10);
    s.c22 = __fmaf_rn(JC22, J22, JC20 * J20);
    s.c30 = C03 * J00;
    s.c31 = __fmaf_rn(C13, 1.0f, C03 * J10);
    s.c32 = __fmaf_rn(C23, J22, C03 * J20);
    s.c40 = C04 * J00;
    s.c41 = __fmaf_rn(C14, 1.0f, C04 * J10);
    s.c42 = __fmaf_rn(C24, J22, C04 * J20);
    x_new = xn;
    return true;
}

// Seed of tracklet t from its chain of kept links (first, middle and last cluster).  Returns false
// if the circle or the direction is unusable.
__device__ __forceinline__ bool seed_tracklet(const DevConst &c, const Workspace &w, int4 sd, KF &st)
{
    const int r0 = sd.w & 0xff;
    // one pass over the chain: the middle cluster (index (len - 1) / 2) advances on every second
    // link, its load independent of the walk's own chain of loads
    int len = 1, last = sd.x, mid = sd.x;
    for (int nx = w.up[last]; nx >= 0 && len < c.nr; nx = w.up[nx]) {
        last = nx;
        len++;
        if (len & 1) mid = w.up[mid];
    }
    const float2 q0 = w.yz[sd.x], q1 = w.yz[mid], q2 = w.yz[last];
    const float x3[3] = {c.row_x[r0], c.row_x[r0 + (len - 1) / 2], c.row_x[r0 + len - 1]};
    const float y3[3] = {q0.x, q1.x, q2.x};
    const float z3[3] = {q0.y, q1.y, q2.y};
    if (!seed3(x3, y3, z3, c, st)) return false;
    set_seed_cov(st, c);
    return true;
}

}  // namespace tpc
