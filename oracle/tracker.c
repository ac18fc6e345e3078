/* CPU oracle of the TPC sector tracker: a plain, sequential restatement of the
 * algorithm of Section 1 with the cluster weight of Section 3.1, the track
 * sorting of Section 3.2 and the 30-cluster minimum of Section 5.
 *
 * Test infrastructure only.  This file is compiled twice: with ORC_F32 defined
 * (`real` = float, functions suffixed _f32) and without (`real` = double, _f64).
 * It must be built with floating-point contraction off (-ffp-contract=off) so
 * that every expression is evaluated exactly as written.
 *
 * Sectors are independent in the sector tracker (Section 1); like the paper's
 * CPU tracker (Section 4) the sectors are distributed over OpenMP threads.
 * Inside a sector everything is sequential, in the order the paper lists the
 * steps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle_internal.h"

#ifdef ORC_F32
typedef float real;
#define FMA fmaf
#define SQRT sqrtf
#define FABS fabsf
#define SFX(name) name##_f32
#else
typedef double real;
#define FMA fma
#define SQRT sqrt
#define FABS fabs
#define SFX(name) name##_f64
#endif

#ifdef ORC_F32
/* asin(u)/u in float.  The float mode evaluates arcsin with a fixed series so that two
 * float implementations of the tracker round identically (the weights of Section 3.1 decide
 * cluster ownership by comparison).  Maclaurin series of arcsin,
 *   asin(u)/u = sum_n (2n)! / (4^n (n!)^2 (2n+1)) u^(2n),
 * twelve terms evaluated by Horner's rule for |u| <= 0.5 (truncation below 4e-10), after
 * reducing larger |u| with the half-angle identity asin(u) = 2 asin(u / sqrt(2 (1 + sqrt(1 - u^2)))). */
static float asin_ratio(float u)
{
    float v = u, m = 1.0f;
    for (int k = 0; k < 3 && fabsf(v) > 0.5f; k++) {
        v = v / sqrtf(2.0f * (1.0f + sqrtf(1.0f - v * v)));
        m = m * 2.0f;
    }
    float t = v * v;
    float s = 0.007312526f;                 /* 88179/12058624 */
    s = fmaf(s, t, 0.00839033537f);         /* 46189/5505024 */
    s = fmaf(s, t, 0.00976160914f);         /* 12155/1245184 */
    s = fmaf(s, t, 0.0115518011f);          /* 6435/557056 */
    s = fmaf(s, t, 0.0139648439f);          /* 143/10240 */
    s = fmaf(s, t, 0.0173527636f);          /* 231/13312 */
    s = fmaf(s, t, 0.0223721582f);          /* 63/2816 */
    s = fmaf(s, t, 0.030381944f);           /* 35/1152 */
    s = fmaf(s, t, 0.0446428582f);          /* 5/112 */
    s = fmaf(s, t, 0.075000003f);           /* 3/40 */
    s = fmaf(s, t, 0.166666672f);           /* 1/6 */
    s = fmaf(s, t, 1.0f);
    if (m == 1.0f) return s;
    return ((m * v) * s) / u;
}
#else
static double asin_ratio(double u) { return (u != 0) ? asin(u) / u : 1.0; }
#endif

#define MAXB 4096            /* cap on grid cells per axis (the last cell absorbs the rest) */
/* Bin ranges are looked up for a window widened by this many cm, so that a
 * cluster which passes the exact window test can never fall in a cell outside
 * the enumerated range because of rounding. */
#define BIN_SLACK ((real)1e-3)

/* ----------------------------------------------------------------------------------------- */
/* constants of one run, in working precision                                                 */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
    int nr;
    real *X;                      /* row x */
    real th, margin, smax;
    real sy2, sz2, isy2, isz2;
    real ty, tz, gate9;
    real cov0[5];
    real nsig, chi2max;
    int max_miss, min_chain, min_clusters;
    real alpha, beta, qptmax;
    real kB;                      /* curvature per unit q/pT: -kappa * Bz */
    real bdy, bdz;
    int brute;
    int global;
    real c20, s20;                /* cos, sin of the 20 degree sector pitch */
    int ns;
    int merge;                    /* track merger with refit */
    real crot[18], srot[18];      /* cos, sin of d * 20 degrees (d = 0..17, read as -160..180) */
    real mchi2, mgap, mq2;        /* merger gates: chi2, radial gap, (q/pT sigmas)^2 */
} K;

static void make_consts(K *k, const orc_config *c)
{
    k->nr = c->n_rows;
    k->X = (real *)malloc(sizeof(real) * (size_t)c->n_rows);
    for (int i = 0; i < c->n_rows; i++) k->X[i] = (real)c->row_x[i];
    k->th = (real)c->tan_half;
    k->margin = (real)c->edge_margin;
    k->smax = (real)c->sin_max;
    real sy = (real)c->sigma_y, sz = (real)c->sigma_z;
    k->sy2 = sy * sy;
    k->sz2 = sz * sz;
    k->isy2 = (real)1 / k->sy2;
    k->isz2 = (real)1 / k->sz2;
    k->ty = (real)c->nb_ty;
    k->tz = (real)c->nb_tz;
    k->gate9 = (real)c->nb_gate;
    for (int i = 0; i < 5; i++) k->cov0[i] = (real)c->seed_cov[i];
    k->nsig = (real)c->win_nsigma;
    k->chi2max = (real)c->chi2_max;
    k->max_miss = c->max_miss;
    k->min_chain = c->min_chain;
    k->min_clusters = c->min_clusters;
    k->alpha = (real)c->alpha;
    k->beta = (real)c->beta;
    k->qptmax = (real)c->qpt_max;
    k->kB = (real)(-ORC_KAPPA * c->bz);
    k->bdy = (real)c->bin_dy;
    k->bdz = (real)c->bin_dz;
    k->brute = c->brute_force;
    k->global = c->global_tracking && c->n_sectors == 36;
    k->c20 = (real)cos(20.0 * 3.14159265358979323846 / 180.0);
    k->s20 = (real)sin(20.0 * 3.14159265358979323846 / 180.0);
    k->ns = c->n_sectors;
    k->merge = c->merge && c->n_sectors == 36;
    for (int d = 0; d < 18; d++) {
        int deg = d <= 9 ? 20 * d : 20 * (d - 18);          /* -160 .. 180 */
        double a = (double)(deg < 0 ? -deg : deg) * 3.14159265358979323846 / 180.0;
        k->crot[d] = (real)cos(a);
        k->srot[d] = deg < 0 ? -(real)sin(a) : (real)sin(a);
    }
    k->mchi2 = (real)c->merge_chi2;
    k->mgap = (real)c->merge_gap;
    k->mq2 = (real)(c->merge_qpt_nsigma * c->merge_qpt_nsigma);
}

/* ----------------------------------------------------------------------------------------- */
/* A1: per-row y/z grid and counting sort (initialisation, Section 2)                         */
/* ----------------------------------------------------------------------------------------- */

/* Cell index along one axis; monotone non-decreasing in v. */
static int cell1(real v, real vmin, real inv, int nb)
{
    real t = (v - vmin) * inv;
    if (!(t >= (real)0)) return 0;
    if (t >= (real)nb) return nb - 1;
    return (int)t;
}

typedef struct {
    int64_t off, n;               /* global index range of the row */
    real ymin, zmin, idy, idz;
    int ny, nz;
    int32_t *cstart;              /* [ny*nz+1] */
    int32_t *sorted;              /* [n] global indices in cell order */
} Row;

static void bin_row(Row *rw, const real *Y, const real *Zc, real dy, real dz)
{
    int64_t n = rw->n;
    real ymin = 0, ymax = 0, zmin = 0, zmax = 0;
    for (int64_t i = 0; i < n; i++) {
        real y = Y[rw->off + i], z = Zc[rw->off + i];
        if (i == 0 || y < ymin) ymin = y;
        if (i == 0 || y > ymax) ymax = y;
        if (i == 0 || z < zmin) zmin = z;
        if (i == 0 || z > zmax) zmax = z;
    }
    int ny = (int)ceil((double)((ymax - ymin) / dy));
    int nz = (int)ceil((double)((zmax - zmin) / dz));
    if (ny < 1) ny = 1;
    if (nz < 1) nz = 1;
    if (ny > MAXB) ny = MAXB;
    if (nz > MAXB) nz = MAXB;
    rw->ymin = ymin;
    rw->zmin = zmin;
    rw->idy = (real)1 / dy;
    rw->idz = (real)1 / dz;
    rw->ny = ny;
    rw->nz = nz;
    int nc = ny * nz;
    rw->cstart = (int32_t *)calloc((size_t)nc + 1, sizeof(int32_t));
    rw->sorted = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        int iy = cell1(Y[rw->off + i], ymin, rw->idy, ny);
        int iz = cell1(Zc[rw->off + i], zmin, rw->idz, nz);
        cell[i] = iz * ny + iy;
        rw->cstart[cell[i] + 1]++;
    }
    for (int c = 0; c < nc; c++) rw->cstart[c + 1] += rw->cstart[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
    memcpy(fill, rw->cstart, sizeof(int32_t) * (size_t)nc);
    for (int64_t i = 0; i < n; i++) rw->sorted[fill[cell[i]]++] = (int32_t)(rw->off + i);
    free(fill);
    free(cell);
}

/* Clusters of a row inside |y - yc| <= wy and |z - zc| <= wz (exact test), found
 * through the grid or, in brute-force mode, by scanning the whole row.  Returns
 * the count; *ncand receives the clusters looked at. */
static int row_window(const Row *rw, const real *Y, const real *Zc, int brute, real yc, real zc,
                      real wy, real wz, int32_t *out, int64_t *ncand, const uint8_t *used)
{
    int cnt = 0;
    if (rw->n == 0) return 0;
    if (brute) {
        for (int64_t i = 0; i < rw->n; i++) {
            int64_t g = rw->off + i;
            if (used && used[g]) continue;
            if (FABS(Y[g] - yc) <= wy && FABS(Zc[g] - zc) <= wz) out[cnt++] = (int32_t)g;
        }
        *ncand += rw->n;
        return cnt;
    }
    int iy0 = cell1(yc - wy - BIN_SLACK, rw->ymin, rw->idy, rw->ny);
    int iy1 = cell1(yc + wy + BIN_SLACK, rw->ymin, rw->idy, rw->ny);
    int iz0 = cell1(zc - wz - BIN_SLACK, rw->zmin, rw->idz, rw->nz);
    int iz1 = cell1(zc + wz + BIN_SLACK, rw->zmin, rw->idz, rw->nz);
    for (int iz = iz0; iz <= iz1; iz++) {
        int a = rw->cstart[iz * rw->ny + iy0], b = rw->cstart[iz * rw->ny + iy1 + 1];
        *ncand += b - a;
        for (int j = a; j < b; j++) {
            int32_t g = rw->sorted[j];
            if (used && used[g]) continue;
            if (FABS(Y[g] - yc) <= wy && FABS(Zc[g] - zc) <= wz) out[cnt++] = g;
        }
    }
    return cnt;
}

/* ----------------------------------------------------------------------------------------- */
/* Kalman filter pieces (tracklet construction, Section 1)                                    */
/* State p = (y, z, sin phi, tan lambda, q/pT) at a plane x; C is the full 5x5 covariance.    */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
    real p[5];
    real C[5][5];
} KS;

static void set_diag(KS *s, const real *d)
{
    memset(s->C, 0, sizeof s->C);
    for (int i = 0; i < 5; i++) s->C[i][i] = d[i];
}

/* Exact helix transport from x0 to x1 (curvature kB*q/pT, sin phi linear in x,
 * chord and arc length of the circle) and C <- F C F^T with F its Jacobian.
 * Returns 0 if |sin phi| at x1 reaches smax. */
static int propagate(KS *s, real x0, real x1, real kB, real smax)
{
    real dx = x1 - x0;
    real cur = kB * s->p[4];
    real s0 = s->p[2];
    real s1 = FMA(cur, dx, s0);
    if (!(FABS(s1) < smax)) return 0;
    real c0 = SQRT(FMA(-s0, s0, (real)1));
    real c1 = SQRT(FMA(-s1, s1, (real)1));
    real A = s0 + s1;
    real B = c0 + c1;
    real iB = (real)1 / B;
    real tq = A * iB;                         /* slope of the chord */
    real dy = dx * tq;
    real L = SQRT(FMA(dx, dx, dy * dy));      /* chord, signed like dx */
    if (dx < 0) L = -L;
    real u = (cur * L) * (real)0.5;           /* sin of half the turning angle */
    real ratio = asin_ratio(u);
    real dS = L * ratio;                      /* arc length = 2 asin(C L / 2) / C */
    real tl = s->p[3];

    real F[5][5];
    memset(F, 0, sizeof F);
    for (int i = 0; i < 5; i++) F[i][i] = 1;
    /* one reciprocal of (c0 + c1) serves the chord slope and both denominators (c0 + c1)^2 */
    real iBB = iB * iB;
    F[0][2] = dx * FMA(A, s0 / c0 + s1 / c1, (real)2 * B) * iBB;      /* d y1 / d sinphi0 */
    F[0][4] = dx * (kB * dx) * FMA(A, s1 / c1, B) * iBB;              /* d y1 / d q/pT */
    F[2][4] = kB * dx;                                               /* d sinphi1 / d q/pT */
    real g = (L != 0) ? dy / (L * SQRT(FMA(-u, u, (real)1))) : (real)0;   /* dS/dL * dL/ddy */
    F[1][2] = tl * (g * F[0][2]);                                    /* d z1 / d sinphi0 */
    F[1][3] = dS;                                                    /* d z1 / d tanl */
    F[1][4] = tl * FMA(g, F[0][4], (((cur * L) * (L * L)) * (real)(1.0 / 12.0)) * kB); /* d z1 / d q/pT */

    s->p[0] = s->p[0] + dy;
    s->p[1] = FMA(tl, dS, s->p[1]);           /* z += tan(lambda) * arc length */
    s->p[2] = s1;

    real FC[5][5], N[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            real a = 0;
            for (int k = 0; k < 5; k++) a = FMA(F[i][k], s->C[k][j], a);
            FC[i][j] = a;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            real a = 0;
            for (int k = 0; k < 5; k++) a = FMA(FC[i][k], F[j][k], a);
            N[i][j] = a;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) s->C[i][j] = s->C[j][i] = N[i][j];
    return 1;
}

/* Inverse of the 2x2 residual covariance S = H C H^T + R, H selecting (y, z). */
typedef struct {
    real Si[2][2];
} Gain;

static void residual_cov_inv(const KS *s, const K *k, Gain *g)
{
    real S00 = s->C[0][0] + k->sy2, S01 = s->C[0][1], S10 = s->C[1][0], S11 = s->C[1][1] + k->sz2;
    real det = FMA(S00, S11, -S01 * S10);
    real idet = (real)1 / det;
    g->Si[0][0] = S11 * idet;
    g->Si[0][1] = -S01 * idet;
    g->Si[1][0] = -S10 * idet;
    g->Si[1][1] = S00 * idet;
}

static real chi2_of(const Gain *g, real r0, real r1)
{
    real t0 = FMA(g->Si[0][1], r1, g->Si[0][0] * r0);
    real t1 = FMA(g->Si[1][1], r1, g->Si[1][0] * r0);
    return FMA(r1, t1, r0 * t0);
}

/* Kalman update with measurement (my, mz): K = C H^T S^-1, p += K r, C -= K H C. */
static void kf_update(KS *s, const Gain *g, real my, real mz)
{
    real r0 = my - s->p[0], r1 = mz - s->p[1];
    real Kg[5][2];
    for (int i = 0; i < 5; i++)
        for (int m = 0; m < 2; m++) {
            real a = 0;
            for (int j = 0; j < 2; j++) a = FMA(s->C[i][j], g->Si[j][m], a);
            Kg[i][m] = a;
        }
    for (int i = 0; i < 5; i++) s->p[i] = FMA(Kg[i][1], r1, FMA(Kg[i][0], r0, s->p[i]));
    real N[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            real a = s->C[i][j];
            for (int m = 0; m < 2; m++) a = FMA(-Kg[i][m], s->C[m][j], a);
            N[i][j] = a;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) s->C[i][j] = s->C[j][i] = N[i][j];
}

/* Seed: the circle through the (x, y) projections of three points gives y, sin phi
 * and the curvature at the first point; tan lambda is the z rise over the arc
 * length from the first to the last point. */
static int seed3(const real *x, const real *y, const real *z, real kB, real smax, real *p)
{
    real ax = x[1] - x[0], ay = y[1] - y[0];
    real bx = x[2] - x[0], by = y[2] - y[0];
    real cx = x[2] - x[1], cy = y[2] - y[1];
    real la = SQRT(ax * ax + ay * ay);
    real lb = SQRT(bx * bx + by * by);
    real lc = SQRT(cx * cx + cy * cy);
    real cross = ax * by - ay * bx;
    real den = (la * lb) * lc;
    if (!(den > 0)) return 0;
    real C = ((real)2 * cross) / den;         /* signed curvature, > 0 turning left */
    real sa = (C * lb) * (real)0.5;           /* sin of the angle between chord and tangent */
    if (!(FABS(sa) < (real)1)) return 0;
    real ca = SQRT((real)1 - sa * sa);
    real sinphi = (by / lb) * ca - (bx / lb) * sa;
    if (!(FABS(sinphi) < smax)) return 0;
    real S02 = lb * asin_ratio(sa);
    p[0] = y[0];
    p[1] = z[0];
    p[2] = sinphi;
    p[3] = (z[2] - z[0]) / S02;
    p[4] = (kB != 0) ? C / kB : (real)0;
    return 1;
}

/* ----------------------------------------------------------------------------------------- */
/* one sector                                                                                 */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
    Row *rows;
    int64_t off, n;
    int64_t nstarts;
    int32_t *starts;
    int64_t cnt[ORC_INFO_COUNT];
    /* output tracks of this sector */
    int64_t ntracks;
    int32_t *tracks;              /* tracklet ids in canonical order */
} Sector;

static int cmp_i64pair(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

/* A1 .. A4 for one sector. */
static void sector_links(Sector *S, const K *k, const real *Y, const real *Zc, const uint8_t *rowv,
                         orc_result *res, int32_t *buf_u, int32_t *buf_d)
{
    int nr = k->nr;
    for (int r = 0; r < nr; r++) bin_row(&S->rows[r], Y, Zc, k->bdy, k->bdz);

    /* A2 neighbours finder: for each cluster of row k the best pair (u in k+1, d in k-1)
     * that forms a straight line with it (Section 1, "Neighbors finder"). */
    for (int r = 1; r + 1 < nr; r++) {
        const Row *rc = &S->rows[r], *ru = &S->rows[r + 1], *rd = &S->rows[r - 1];
        if (rc->n == 0 || ru->n == 0 || rd->n == 0) continue;
        real xk = k->X[r], xu = k->X[r + 1], xd = k->X[r - 1];
        real dxu = xu - xk, dxd = xk - xd;
        real wyu = k->ty * dxu, wzu = k->tz * dxu;
        real wyd = k->ty * dxd, wzd = k->tz * dxd;
        real w = dxd / (xu - xd);             /* weight of u in the interpolation at x_k */
        real om = (real)1 - w;
        real gate = k->gate9 * FMA(w, w, FMA(om, om, (real)1));
        for (int64_t i = 0; i < rc->n; i++) {
            int64_t c = rc->off + i;
            real yc = Y[c], zc = Zc[c];
            int nu = row_window(ru, Y, Zc, k->brute, yc, zc, wyu, wzu, buf_u, &S->cnt[ORC_INFO_NB_CANDIDATES], NULL);
            int nd = row_window(rd, Y, Zc, k->brute, yc, zc, wyd, wzd, buf_d, &S->cnt[ORC_INFO_NB_CANDIDATES], NULL);
            int32_t bu = -1, bd = -1;
            real best = 0;
            for (int a = 0; a < nu; a++)
                for (int b = 0; b < nd; b++) {
                    int32_t u = buf_u[a], d = buf_d[b];
                    real dy = FMA(-(Y[u] - Y[d]), w, yc - Y[d]);
                    real dz = FMA(-(Zc[u] - Zc[d]), w, zc - Zc[d]);
                    real sc = FMA(dz * dz, k->isz2, (dy * dy) * k->isy2);
                    int better = (bu < 0) || (sc < best) || (sc == best && (u < bu || (u == bu && d < bd)));
                    if (better) {
                        best = sc;
                        bu = u;
                        bd = d;
                    }
                }
            if (bu >= 0 && best <= gate) {
                res->up_raw[c] = bu;
                res->dn_raw[c] = bd;
            }
        }
    }
    /* A3 evolution: keep only reciprocal links (Section 1, "Evolution step"). */
    for (int64_t c = S->off; c < S->off + S->n; c++) {
        int32_t u = res->up_raw[c], d = res->dn_raw[c];
        res->up[c] = (u >= 0 && res->dn_raw[u] == c) ? u : -1;
        res->dn[c] = (d >= 0 && res->up_raw[d] == c) ? d : -1;
    }
    /* A4 start hits: heads of chains of one-to-one links with >= min_chain clusters,
     * in (row, input index) order. */
    S->starts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->n > 0 ? S->n : 1));
    S->nstarts = 0;
    for (int64_t c = S->off; c < S->off + S->n; c++) {
        if (res->up[c] < 0 || res->dn[c] >= 0) continue;
        int len = 1;
        int32_t t = (int32_t)c;
        while (res->up[t] >= 0) {
            t = res->up[t];
            len++;
        }
        if (len >= k->min_chain) S->starts[S->nstarts++] = (int32_t)c;
    }
    (void)rowv;
}

/* Best cluster of row r for state s: minimum chi2, ties to the lower input index. */
static int32_t search_row(Sector *S, const K *k, const real *Y, const real *Zc, const KS *s, int r,
                          const Gain *g, real *chi2_out, int32_t *buf, const uint8_t *used)
{
    const Row *rw = &S->rows[r];
    real wy = k->nsig * SQRT(s->C[0][0] + k->sy2);
    real wz = k->nsig * SQRT(s->C[1][1] + k->sz2);
    int nc = row_window(rw, Y, Zc, k->brute, s->p[0], s->p[1], wy, wz, buf, &S->cnt[ORC_INFO_CANDIDATES], used);
    S->cnt[ORC_INFO_IN_WINDOW] += nc;
    S->cnt[ORC_INFO_VISITS]++;
    int32_t best = -1;
    real bc = 0;
    for (int i = 0; i < nc; i++) {
        int32_t c = buf[i];
        real x2 = chi2_of(g, Y[c] - s->p[0], Zc[c] - s->p[1]);
        if (best < 0 || x2 < bc || (x2 == bc && c < best)) {
            best = c;
            bc = x2;
        }
    }
    *chi2_out = bc;
    return best;
}

/* Section 3.1: the weight of a tracklet of n clusters whose fit collected chi2sum,
 * w = n * (alpha - chi2 / beta), the "normalized" chi2 of the whole track read as chi2 per
 * degree of freedom, ndf = 2 n - 5 (two measured coordinates per cluster, five fitted
 * parameters).  A tracklet with ndf < 1 has no weight and claims no cluster. */
static real tracklet_weight(int n, real chi2sum, real alpha, real beta)
{
    int ndf = 2 * n - 5;
    if (ndf < 1) return (real)-INFINITY;
    return (real)n * (alpha - (chi2sum / (real)ndf) / beta);
}

/* Section 3.1: every cluster goes to the tracklet of largest weight among those holding it;
 * of equal weights the earlier tracklet (lower index) keeps it.  Tracklets t0 .. t0 + T - 1,
 * hits[t * nr ..] their clusters, weights wv[t]; owner[c] is -1 for a cluster nobody claimed. */
static void claim_clusters(int64_t t0, int64_t T, const int32_t *nhits, const int32_t *hits, int nr,
                           const real *wv, int32_t *owner)
{
    for (int64_t i = 0; i < T; i++) {
        int64_t t = t0 + i;
        if (wv[t] == (real)-INFINITY) continue;
        const int32_t *h = hits + (size_t)t * (size_t)nr;
        for (int j = 0; j < nhits[t]; j++) {
            int32_t c = h[j];
            int32_t o = owner[c];
            if (o < 0 || wv[t] > wv[o]) owner[c] = (int32_t)t;
        }
    }
}

/* A5 tracklet construction for the tracklet starting at cluster c0 (Section 1,
 * "Tracklet construction"): seed from the chain, fit outwards while searching each
 * row, then refit inwards from the outermost cluster with a fresh covariance. */
static void construct(Sector *S, const K *k, const real *Y, const real *Zc, const uint8_t *rowv,
                      orc_result *res, int64_t t, int32_t c0, int32_t *buf, int32_t *chain)
{
    int nr = k->nr;
    int L = 0;
    for (int32_t c = c0; c >= 0; c = res->up[c]) chain[L++] = c;
    int m = (L - 1) / 2;
    int32_t c3[3] = {chain[0], chain[m], chain[L - 1]};
    real x3[3], y3[3], z3[3];
    for (int i = 0; i < 3; i++) {
        x3[i] = k->X[rowv[c3[i]]];
        y3[i] = Y[c3[i]];
        z3[i] = Zc[c3[i]];
    }
    int32_t *hits = res->tl_hits + (size_t)t * (size_t)nr;
    res->tl_nhits[t] = 0;
    res->tl_ndf[t] = -5;
    res->tl_nup[t] = 0;
    res->tl_w[t] = -INFINITY;
    KS st;
    if (!seed3(x3, y3, z3, k->kB, k->smax, st.p)) return;
    set_diag(&st, k->cov0);
    Gain g;
    real chi2;

    /* Outward pass.  `st` is the state at the last fitted cluster (at x = xs); the
     * prediction for row r is that state transported along the helix to x_r. */
    int r0 = rowv[c0];
    real xs = k->X[r0];
    int rlast = -1, miss = 0, nup = 0;
    KS pr;
    for (int r = r0; r < nr; r++) {
        real xr = k->X[r];
        pr = st;
        if (xr != xs && !propagate(&pr, xs, xr, k->kB, k->smax)) break;
        if (FABS(pr.p[0]) > FMA(xr, k->th, k->margin)) break;
        residual_cov_inv(&pr, k, &g);
        int32_t b = search_row(S, k, Y, Zc, &pr, r, &g, &chi2, buf, NULL);
        if (b >= 0 && chi2 <= k->chi2max) {
            kf_update(&pr, &g, Y[b], Zc[b]);
            S->cnt[ORC_INFO_UPDATES]++;
            st = pr;
            xs = xr;
            nup++;
            rlast = r;
            miss = 0;
        } else if (++miss >= k->max_miss) {
            break;
        }
    }
    res->tl_nup[t] = nup;
    if (rlast < 0) return;

    /* the outward pass's state at its last cluster is the track's outer end (global tracking) */
    {
        int q = 0;
        for (int i = 0; i < 5; i++) res->tl_opar[t * 5 + i] = (double)st.p[i];
        for (int i = 0; i < 5; i++)
            for (int j = 0; j <= i; j++) res->tl_ocov[t * 15 + q++] = (double)st.C[i][j];
        res->tl_ox[t] = (double)xs;
        res->tl_orow[t] = rlast;
    }
    /* Inward pass from the outermost cluster, covariance reset to the seed's; its
     * clusters are the tracklet's, its last state is reported. */
    set_diag(&st, k->cov0);
    miss = 0;
    int n = 0;
    real chi2sum = 0;
    for (int r = rlast; r >= 0; r--) {
        real xr = k->X[r];
        pr = st;
        if (xr != xs && !propagate(&pr, xs, xr, k->kB, k->smax)) break;
        if (FABS(pr.p[0]) > FMA(xr, k->th, k->margin)) break;
        residual_cov_inv(&pr, k, &g);
        int32_t b = search_row(S, k, Y, Zc, &pr, r, &g, &chi2, buf, NULL);
        if (b >= 0 && chi2 <= k->chi2max) {
            chi2sum = chi2sum + chi2;
            kf_update(&pr, &g, Y[b], Zc[b]);
            S->cnt[ORC_INFO_UPDATES]++;
            st = pr;
            xs = xr;
            hits[n++] = b;
            miss = 0;
        } else if (++miss >= k->max_miss) {
            break;
        }
    }
    KS inner = st;
    real xin = xs;
    int ndf = 2 * n - 5;
    res->tl_nhits[t] = n;
    res->tl_ndf[t] = ndf;
    for (int i = 0; i < 5; i++) res->tl_par[t * 5 + i] = (double)inner.p[i];
    int q = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) res->tl_cov[t * 15 + q++] = (double)inner.C[i][j];
    res->tl_x[t] = (double)xin;
    res->tl_chi2[t] = (double)chi2sum;
    res->tl_w[t] = (double)tracklet_weight(n, chi2sum, k->alpha, k->beta);
}

/* A6 selection and A7 output order for one sector. */
static void sector_select(Sector *S, const K *k, orc_result *res, int64_t t0, const real *wv)
{
    int nr = k->nr;
    int64_t T = S->nstarts;
    claim_clusters(t0, T, res->tl_nhits, res->tl_hits, nr, wv, res->owner);
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(T > 0 ? T : 1));
    int64_t na = 0;
    for (int64_t i = 0; i < T; i++) {
        int64_t t = t0 + i;
        if (res->tl_ndf[t] < 1) continue;
        const int32_t *h = res->tl_hits + (size_t)t * (size_t)nr;
        int own = 0;
        int32_t inner = -1;
        for (int j = 0; j < res->tl_nhits[t]; j++)
            if (res->owner[h[j]] == (int32_t)t) {
                own++;
                inner = h[j];               /* hits are stored outer to inner */
            }
        res->tl_nowned[t] = own;
        real q = (real)res->tl_par[t * 5 + 4];
        int acc = own >= k->min_clusters && FABS(q) <= k->qptmax;
        res->tl_accept[t] = (uint8_t)acc;
        if (acc) {
            keys[2 * na] = inner;           /* Section 3.2: sort by the innermost cluster */
            keys[2 * na + 1] = t;
            na++;
        }
    }
    qsort(keys, (size_t)na, 2 * sizeof(int64_t), cmp_i64pair);
    S->ntracks = na;
    S->tracks = (int32_t *)malloc(sizeof(int32_t) * (size_t)(na > 0 ? na : 1));
    for (int64_t i = 0; i < na; i++) S->tracks[i] = (int32_t)keys[2 * i + 1];
    free(keys);
}

/* Change of frame by an azimuth rotation (cos cd, sin sd): the state at x in the old frame is
 * re-expressed at x' = x cd + y sd in the new frame (y' = -x sd + y cd, phi' = phi - angle), with
 * the covariance transported by the Jacobian of the map to fixed x' (a change of y moves the
 * point along x', which is taken back along the track).  Returns 0 if the direction does not
 * point to increasing x' or |sin phi'| reaches smax. */
static int rotate(KS *s, real x, real cd, real sd, real kB, real smax, real *x_new)
{
    real y = s->p[0], sp = s->p[2];
    real cp = SQRT(FMA(-sp, sp, (real)1));
    real xn = FMA(x, cd, y * sd);
    real yn = FMA(y, cd, -(x * sd));
    real spn = FMA(sp, cd, -(cp * sd));
    if (!(FABS(spn) < smax)) return 0;
    if (!(FMA(cp, cd, sp * sd) > 0)) return 0;          /* cos(phi') > 0 */
    real cpn = SQRT(FMA(-spn, spn, (real)1));
    real J[5][5];
    memset(J, 0, sizeof J);
    for (int i = 0; i < 5; i++) J[i][i] = 1;
    J[0][0] = FMA(-sd, spn / cpn, cd);                 /* d y' / d y */
    J[1][0] = -(sd * s->p[3]) / cpn;                   /* d z' / d y */
    J[2][0] = -(kB * s->p[4]) * sd;                    /* d sinphi' / d y */
    J[2][2] = cpn / cp;                                /* d sinphi' / d sinphi */
    s->p[0] = yn;
    s->p[2] = spn;
    real JC[5][5], N[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            real a = 0;
            for (int k = 0; k < 5; k++) a = FMA(J[i][k], s->C[k][j], a);
            JC[i][j] = a;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            real a = 0;
            for (int k = 0; k < 5; k++) a = FMA(JC[i][k], J[j][k], a);
            N[i][j] = a;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) s->C[i][j] = s->C[j][i] = N[i][j];
    *x_new = xn;
    return 1;
}

/* Global tracking (Section 5): prolong a sector track from one of its ends into the neighbouring
 * sector.  end: the state at x_end (row r_end) in sector s; dir = -1 inwards, +1 outwards.  The end
 * counts as lying at the sector edge if the one-row extrapolation in its own sector leaves the
 * row's width; then the state is rotated into the neighbour sector on that side (same z half) and
 * the rows beyond x' are searched in direction dir with the construction's window, gate and stop
 * rules, among the clusters of no accepted track (used[] == 0).  Returns the clusters found
 * (hits_out, in search order); *fin receives the state at the last of them, *xfin its x, *sfin the
 * neighbour sector. */
static int prolong(Sector *S, const K *k, const real *Y, const real *Zc, int s, const KS *end, real x_end,
                   int r_end, int dir, const uint8_t *used, int32_t *buf, int32_t *hits_out, real *chi2_out,
                   KS *fin, real *xfin, int *sfin)
{
    int nr = k->nr;
    *chi2_out = 0;
    int rn = r_end + dir;
    if (rn < 0 || rn >= nr) return 0;
    KS pr = *end;
    if (!propagate(&pr, x_end, k->X[rn], k->kB, k->smax)) return 0;
    if (!(FABS(pr.p[0]) > k->X[rn] * k->th)) return 0;  /* still inside its sector */
    int side = s / 18, az = s % 18;
    int plus = pr.p[0] > 0;
    int s2 = side * 18 + (plus ? (az + 1) % 18 : (az + 17) % 18);
    KS st = *end;
    real xs;
    if (!rotate(&st, x_end, k->c20, plus ? k->s20 : -k->s20, k->kB, k->smax, &xs)) return 0;
    int r = dir < 0 ? nr - 1 : 0;
    if (dir < 0)
        while (r >= 0 && !(k->X[r] < xs)) r--;
    else
        while (r < nr && !(k->X[r] > xs)) r++;
    int n = 0, miss = 0;
    real chi2sum = 0;
    Gain g;
    real chi2;
    for (; r >= 0 && r < nr; r += dir) {
        real xr = k->X[r];
        pr = st;
        if (!propagate(&pr, xs, xr, k->kB, k->smax)) break;
        if (FABS(pr.p[0]) > FMA(xr, k->th, k->margin)) break;
        residual_cov_inv(&pr, k, &g);
        int32_t b = search_row(&S[s2], k, Y, Zc, &pr, r, &g, &chi2, buf, used);
        if (b >= 0 && chi2 <= k->chi2max) {
            chi2sum = chi2sum + chi2;
            kf_update(&pr, &g, Y[b], Zc[b]);
            st = pr;
            xs = xr;
            hits_out[n++] = b;
            miss = 0;
        } else if (++miss >= k->max_miss) {
            break;
        }
    }
    *chi2_out = chi2sum;
    *fin = st;
    *xfin = xs;
    *sfin = s2;
    return n;
}

/* ----------------------------------------------------------------------------------------- */
/* Track merger with refit (Section 1: "the sector tracks are merged by the track merger";      */
/* Section 3.3: the merger refits every track from its cluster list alone, so equal cluster     */
/* lists give bitwise equal results whatever rounding the sector tracker saw)                   */
/* ----------------------------------------------------------------------------------------- */

#define ORC_MAX_CHAIN 64   /* bound on a chain walk (radii increase along a chain, so it never binds) */

/* Steps of 20 degrees that take frame `from` to frame `to` (0..17; same azimuth: 0). */
static int rot_steps(int from, int to) { return ((to % 18) - (from % 18) + 18) % 18; }

/* Frame change of the state for the cluster's sector; returns 0 if the rotation fails. */
static int to_frame(const K *k, KS *st, real *xs, int *sc, int s_new)
{
    int d = rot_steps(*sc, s_new);
    *sc = s_new;
    if (d == 0) return 1;                 /* same azimuth (also the other z half): same frame */
    real xn;
    if (!rotate(st, *xs, k->crot[d], k->srot[d], k->kB, k->smax, &xn)) return 0;
    *xs = xn;
    return 1;
}

/* One Kalman pass over the clusters h[i0], h[i0 + dir], ... (n of them) from the state st at
 * (xs, sector sc); every cluster is used (no search).  chi2 of the updates is summed. */
static int refit_pass(const K *k, const real *Y, const real *Zc, const uint8_t *rowv, const int32_t *secv,
                      const int32_t *h, int n, int dir, KS *st, real *xs, int *sc, real *chi2sum)
{
    Gain g;
    for (int i = 0; i < n; i++) {
        int c = h[dir > 0 ? i : n - 1 - i];
        if (!to_frame(k, st, xs, sc, secv[c])) return 0;
        real xr = k->X[rowv[c]];
        if (xr != *xs && !propagate(st, *xs, xr, k->kB, k->smax)) return 0;
        residual_cov_inv(st, k, &g);
        *chi2sum = *chi2sum + chi2_of(&g, Y[c] - st->p[0], Zc[c] - st->p[1]);
        kf_update(st, &g, Y[c], Zc[c]);
        *xs = xr;
    }
    return 1;
}

typedef struct {
    int ok;
    KS in, out;                   /* states at the innermost and outermost cluster */
    real x_in, x_out;
    int s_in, s_out;              /* frame sectors */
    real chi2;                    /* sum of the inward pass's update chi2 */
    real r_in, r_out;             /* transverse radius of the innermost and outermost cluster */
} Refit;

/* Refit of a cluster list h[0..n-1] (inner to outer): seed from the circle through the first,
 * middle and last clusters (taken into the first cluster's frame), outward pass with the seed
 * covariance, inward pass with the covariance reset to the seed's, exactly as the tracklet
 * construction does but on the given clusters; the inward pass's last state is the result. */
static void refit(const K *k, const real *Y, const real *Zc, const uint8_t *rowv, const int32_t *secv,
                  const int32_t *h, int n, Refit *o)
{
    memset(o, 0, sizeof *o);
    if (n < 3) return;
    int s0 = secv[h[0]];
    int idx[3] = {0, (n - 1) / 2, n - 1};
    real x3[3], y3[3], z3[3];
    for (int i = 0; i < 3; i++) {
        int c = h[idx[i]];
        int d = rot_steps(secv[c], s0);
        real x = k->X[rowv[c]], yv = Y[c];
        real cd = k->crot[d], sd = k->srot[d];
        x3[i] = d == 0 ? x : FMA(x, cd, yv * sd);
        y3[i] = d == 0 ? yv : FMA(yv, cd, -(x * sd));
        z3[i] = Zc[c];
    }
    KS st;
    if (!seed3(x3, y3, z3, k->kB, k->smax, st.p)) return;
    set_diag(&st, k->cov0);
    real xs = k->X[rowv[h[0]]];
    int sc = s0;
    real dummy = 0;
    if (!refit_pass(k, Y, Zc, rowv, secv, h, n, 1, &st, &xs, &sc, &dummy)) return;
    o->out = st;
    o->x_out = xs;
    o->s_out = sc;
    set_diag(&st, k->cov0);
    real chi2 = 0;
    if (!refit_pass(k, Y, Zc, rowv, secv, h, n, -1, &st, &xs, &sc, &chi2)) return;
    o->in = st;
    o->x_in = xs;
    o->s_in = sc;
    o->chi2 = chi2;
    int ci = h[0], co = h[n - 1];
    real xi = k->X[rowv[ci]], xo = k->X[rowv[co]];
    o->r_in = SQRT(FMA(xi, xi, Y[ci] * Y[ci]));
    o->r_out = SQRT(FMA(xo, xo, Y[co] * Y[co]));
    o->ok = 1;
}

/* chi2 = d^T A^-1 d for a symmetric 5x5 A (lower triangle used): Cholesky factor L (A = L L^T),
 * then u = L^-1 d by forward substitution and chi2 = |u|^2.  0 if A is not positive definite. */
static int chi2_5(const real A[5][5], const real d[5], real *chi2)
{
    real L[5][5], u[5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            real t = A[i][j];
            for (int m = 0; m < j; m++) t = FMA(-L[i][m], L[j][m], t);
            if (i == j) {
                if (!(t > 0)) return 0;
                L[i][i] = SQRT(t);
            } else {
                L[i][j] = t / L[j][j];
            }
        }
    real q = 0;
    for (int i = 0; i < 5; i++) {
        real t = d[i];
        for (int m = 0; m < i; m++) t = FMA(-L[i][m], u[m], t);
        u[i] = t / L[i][i];
        q = FMA(u[i], u[i], q);
    }
    *chi2 = q;
    return 1;
}

/* Compatibility of track a's outer end with track b's inner end (b continuing a outwards):
 * radial gap in (0, mgap], q/pT within the gate, then a's outer state taken into b's frame and
 * transported to b's innermost cluster, and chi2 of the 5-parameter difference with the summed
 * covariances.  `ar` is a's outer state already in b's frame at x = xa. */
static int match_chi2(const K *k, const Refit *a, const KS *ar, real xa, const Refit *b, real *chi2)
{
    real gap = b->r_in - a->r_out;
    if (!(gap > 0 && gap <= k->mgap)) return 0;
    real dq = b->in.p[4] - ar->p[4];
    if (!(dq * dq <= k->mq2 * (ar->C[4][4] + b->in.C[4][4]))) return 0;
    KS pr = *ar;
    if (xa != b->x_in && !propagate(&pr, xa, b->x_in, k->kB, k->smax)) return 0;
    real A[5][5], d[5];
    for (int i = 0; i < 5; i++) {
        d[i] = b->in.p[i] - pr.p[i];
        for (int j = 0; j <= i; j++) A[i][j] = pr.C[i][j] + b->in.C[i][j];
    }
    if (!chi2_5(A, d, chi2)) return 0;
    return *chi2 <= k->mchi2;
}

/* Merger over the event's sector tracks (res->trk_*); fills res->rf_* (refit of every sector
 * track), res->mg_next and the merged tracks res->mrg_*. */
static void merge_tracks(const K *k, const real *Y, const real *Zc, const uint8_t *rowv, const int32_t *secv,
                         orc_result *res, int nth)
{
    int64_t M = res->n_tracks;
    size_t mm = (size_t)(M > 0 ? M : 1);
    Refit *rf = (Refit *)calloc(mm, sizeof(Refit));
    (void)nth;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nth > 0 ? nth : omp_get_max_threads())
#endif
    for (int64_t m = 0; m < M; m++)
        refit(k, Y, Zc, rowv, secv, res->trk_hits + res->trk_first[m], res->trk_nhits[m], &rf[m]);
    /* tracks by the sector of their innermost cluster, in track order (counting sort) */
    int64_t sec_first[37];
    int32_t *by_sec = (int32_t *)malloc(mm * sizeof(int32_t));
    memset(sec_first, 0, sizeof sec_first);
    for (int64_t m = 0; m < M; m++) sec_first[secv[res->trk_hits[res->trk_first[m]]] + 1]++;
    for (int s = 0; s < 36; s++) sec_first[s + 1] += sec_first[s];
    {
        int64_t cur[36];
        for (int s = 0; s < 36; s++) cur[s] = sec_first[s];
        for (int64_t m = 0; m < M; m++) by_sec[cur[secv[res->trk_hits[res->trk_first[m]]]]++] = (int32_t)m;
    }
    /* best partner of every outer end; best partner of every inner end (ties: lower index) */
    int32_t *best = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *bbest = (int32_t *)malloc(mm * sizeof(int32_t));
    real *bchi = (real *)malloc(mm * sizeof(real));
    real *bbchi = (real *)malloc(mm * sizeof(real));
    for (int64_t m = 0; m < M; m++) {
        best[m] = bbest[m] = -1;
        bchi[m] = bbchi[m] = 0;
    }
    for (int64_t a = 0; a < M; a++) {
        if (!rf[a].ok) continue;
        int sa = rf[a].s_out, side = sa / 18, az = sa % 18;
        int cand[3] = {(1 - side) * 18 + az, side * 18 + (az + 1) % 18, side * 18 + (az + 17) % 18};
        for (int q = 0; q < 3; q++) {
            int sb = cand[q];
            KS ar = rf[a].out;
            real xa = rf[a].x_out;
            int sc = sa;
            if (!to_frame(k, &ar, &xa, &sc, sb)) continue;
            for (int64_t ib = sec_first[sb]; ib < sec_first[sb + 1]; ib++) {
                int64_t b = by_sec[ib];
                if (b == a || !rf[b].ok) continue;
                real chi2;
                if (!match_chi2(k, &rf[a], &ar, xa, &rf[b], &chi2)) continue;
                if (best[a] < 0 || chi2 < bchi[a] || (chi2 == bchi[a] && b < best[a])) {
                    best[a] = (int32_t)b;
                    bchi[a] = chi2;
                }
                if (bbest[b] < 0 || chi2 < bbchi[b] || (chi2 == bbchi[b] && a < bbest[b])) {
                    bbest[b] = (int32_t)a;
                    bbchi[b] = chi2;
                }
            }
        }
    }
    /* mutual best pairs are merged; radii increase along a chain, so chains have no cycles */
    int32_t *prev = (int32_t *)malloc(mm * sizeof(int32_t));
    for (int64_t m = 0; m < M; m++) prev[m] = -1;
    for (int64_t a = 0; a < M; a++) {
        int32_t b = best[a];
        res->mg_next[a] = (b >= 0 && bbest[b] == a) ? b : -1;
        if (res->mg_next[a] >= 0) prev[b] = (int32_t)a;
    }
    for (int64_t m = 0; m < M; m++) {
        for (int i = 0; i < 5; i++) res->rf_par[m * 5 + i] = (double)rf[m].in.p[i];
        int q = 0;
        for (int i = 0; i < 5; i++)
            for (int j = 0; j <= i; j++) res->rf_cov[m * 15 + q++] = (double)rf[m].in.C[i][j];
        res->rf_x[m] = (double)rf[m].x_in;
        res->rf_chi2[m] = (double)rf[m].chi2;
        res->rf_ok[m] = rf[m].ok;
    }
    /* merged tracks: one per chain head, in canonical order; clusters of the chain's tracks in
     * order, refitted over all of them */
    int64_t Mm = 0, Hm = 0;
    for (int64_t m = 0; m < M; m++)
        if (prev[m] < 0) {
            Mm++;
            int64_t t = m;
            for (int step = 0; step < ORC_MAX_CHAIN && t >= 0; step++, t = res->mg_next[t]) Hm += res->trk_nhits[t];
        }
    res->n_merged = Mm;
    res->n_merged_hits = Hm;
    size_t mmm = (size_t)(Mm > 0 ? Mm : 1);
    res->mrg_first = (int32_t *)malloc(mmm * sizeof(int32_t));
    res->mrg_nhits = (int32_t *)malloc(mmm * sizeof(int32_t));
    res->mrg_nseg = (int32_t *)malloc(mmm * sizeof(int32_t));
    res->mrg_head = (int32_t *)malloc(mmm * sizeof(int32_t));
    res->mrg_hits = (int32_t *)malloc((size_t)(Hm > 0 ? Hm : 1) * sizeof(int32_t));
    res->mrg_par = (double *)calloc(mmm * 5, sizeof(double));
    res->mrg_cov = (double *)calloc(mmm * 15, sizeof(double));
    res->mrg_x = (double *)calloc(mmm, sizeof(double));
    res->mrg_chi2 = (double *)calloc(mmm, sizeof(double));
    res->mrg_ndf = (int32_t *)calloc(mmm, sizeof(int32_t));
    res->mrg_sector = (int32_t *)calloc(mmm, sizeof(int32_t));
    res->mrg_ok = (int32_t *)calloc(mmm, sizeof(int32_t));
    int64_t j = 0, h = 0;
    for (int64_t m = 0; m < M; m++) {
        if (prev[m] >= 0) continue;
        res->mrg_head[j] = (int32_t)m;
        res->mrg_first[j] = (int32_t)h;
        int nseg = 0;
        int64_t t = m;
        for (int step = 0; step < ORC_MAX_CHAIN && t >= 0; step++, t = res->mg_next[t]) {
            for (int i = 0; i < res->trk_nhits[t]; i++) res->mrg_hits[h++] = res->trk_hits[res->trk_first[t] + i];
            nseg++;
        }
        res->mrg_nhits[j] = (int32_t)(h - res->mrg_first[j]);
        res->mrg_nseg[j] = nseg;
        j++;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nth > 0 ? nth : omp_get_max_threads())
#endif
    for (int64_t i = 0; i < Mm; i++) {
        int64_t m = res->mrg_head[i];
        Refit r;
        if (res->mrg_nseg[i] > 1)
            refit(k, Y, Zc, rowv, secv, res->mrg_hits + res->mrg_first[i], res->mrg_nhits[i], &r);
        else
            r = rf[m];
        if (r.ok) {
            for (int a = 0; a < 5; a++) res->mrg_par[i * 5 + a] = (double)r.in.p[a];
            int q = 0;
            for (int a = 0; a < 5; a++)
                for (int b = 0; b <= a; b++) res->mrg_cov[i * 15 + q++] = (double)r.in.C[a][b];
            res->mrg_x[i] = (double)r.x_in;
            res->mrg_chi2[i] = (double)r.chi2;
            res->mrg_ndf[i] = 2 * res->mrg_nhits[i] - 5;
            res->mrg_sector[i] = r.s_in;
        } else {                            /* refit failed: the sector tracker's parameters */
            for (int a = 0; a < 5; a++) res->mrg_par[i * 5 + a] = res->trk_par[m * 5 + a];
            for (int a = 0; a < 15; a++) res->mrg_cov[i * 15 + a] = res->trk_cov[m * 15 + a];
            res->mrg_x[i] = res->trk_x[m];
            res->mrg_chi2[i] = res->trk_chi2[m];
            res->mrg_ndf[i] = res->trk_ndf[m];
            res->mrg_sector[i] = res->trk_sector[m];
        }
        res->mrg_ok[i] = r.ok;
    }
    free(rf);
    free(by_sec);
    free(best);
    free(bbest);
    free(bchi);
    free(bbchi);
    free(prev);
}

orc_result *SFX(orc_track_event)(const orc_config *cfg, const double *y, const double *z,
                                 const uint8_t *row, const int32_t *counts, int64_t n)
{
    K k;
    make_consts(&k, cfg);
    int nr = k.nr, ns = cfg->n_sectors;
    orc_result *res = orc_result_alloc(n, nr);
    real *Y = (real *)malloc(sizeof(real) * (size_t)(n > 0 ? n : 1));
    real *Zc = (real *)malloc(sizeof(real) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        Y[i] = (real)y[i];
        Zc[i] = (real)z[i];
    }
    Sector *S = (Sector *)calloc((size_t)ns, sizeof(Sector));
    int64_t off = 0;
    int maxrow = 1;
    for (int s = 0; s < ns; s++) {
        S[s].rows = (Row *)calloc((size_t)nr, sizeof(Row));
        S[s].off = off;
        for (int r = 0; r < nr; r++) {
            int32_t cnt = counts[s * nr + r];
            S[s].rows[r].off = off;
            S[s].rows[r].n = cnt;
            off += cnt;
            if (cnt > maxrow) maxrow = cnt;
        }
        S[s].n = off - S[s].off;
    }
#ifdef _OPENMP
    int nth = cfg->n_threads > 0 ? cfg->n_threads : omp_get_max_threads();
#endif

#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
    {
        int32_t *bu = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxrow);
        int32_t *bd = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxrow);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int s = 0; s < ns; s++) sector_links(&S[s], &k, Y, Zc, row, res, bu, bd);
        free(bu);
        free(bd);
    }

    int64_t T = 0;
    for (int s = 0; s < ns; s++) T += S[s].nstarts;
    orc_result_alloc_tracklets(res, T);
    int64_t *t0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
    t0[0] = 0;
    for (int s = 0; s < ns; s++) {
        t0[s + 1] = t0[s] + S[s].nstarts;
        for (int64_t i = 0; i < S[s].nstarts; i++) res->starts[t0[s] + i] = S[s].starts[i];
    }
    real *wv = (real *)malloc(sizeof(real) * (size_t)(T > 0 ? T : 1));

#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
    {
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxrow);
        int32_t *chain = (int32_t *)malloc(sizeof(int32_t) * (size_t)nr);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int s = 0; s < ns; s++) {
            for (int64_t i = 0; i < S[s].nstarts; i++) {
                int64_t t = t0[s] + i;
                construct(&S[s], &k, Y, Zc, row, res, t, S[s].starts[i], buf, chain);
                wv[t] = (real)res->tl_w[t];
            }
            sector_select(&S[s], &k, res, t0[s], wv);
        }
        free(buf);
        free(chain);
    }

    /* tracks in canonical order (input indices are grouped by sector, so concatenating the
     * sectors' sorted lists is the canonical order) */
    int64_t M = 0;
    for (int s = 0; s < ns; s++) M += S[s].ntracks;
    int32_t *tk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    int32_t *tsec = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    {
        int64_t m = 0;
        for (int s = 0; s < ns; s++)
            for (int64_t i = 0; i < S[s].ntracks; i++) {
                tk[m] = S[s].tracks[i];
                tsec[m] = s;
                m++;
            }
    }

    /* Global tracking (Section 5): both ends of every track, then each contested cluster goes to
     * the prolongation of the track with the higher weight (ties: the earlier start cluster, then
     * the inward prolongation) */
    int32_t *gh = NULL, *gn = NULL, *gown = NULL, *gsec = NULL;
    real *gchi = NULL, *gx = NULL;
    KS *gfin = NULL;
    if (k.global && M > 0) {
        uint8_t *used = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
        for (int64_t m = 0; m < M; m++) {
            int32_t t = tk[m];
            const int32_t *hh = res->tl_hits + (size_t)t * (size_t)nr;
            for (int j = 0; j < res->tl_nhits[t]; j++)
                if (res->owner[hh[j]] == t) used[hh[j]] = 1;
        }
        gh = (int32_t *)malloc(sizeof(int32_t) * (size_t)M * 2 * (size_t)nr);
        gn = (int32_t *)calloc((size_t)M * 2, sizeof(int32_t));
        gown = (int32_t *)calloc((size_t)M * 2, sizeof(int32_t));
        gsec = (int32_t *)calloc((size_t)M * 2, sizeof(int32_t));
        gchi = (real *)calloc((size_t)M * 2, sizeof(real));
        gx = (real *)calloc((size_t)M * 2, sizeof(real));
        gfin = (KS *)calloc((size_t)M * 2, sizeof(KS));
#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
        {
            int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxrow);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t m = 0; m < M; m++) {
                int32_t t = tk[m];
                for (int d = 0; d < 2; d++) {
                    KS end;
                    real xe;
                    int re;
                    if (d == 0) {           /* inner end: the reported state */
                        for (int i = 0; i < 5; i++) end.p[i] = (real)res->tl_par[t * 5 + i];
                        int q = 0;
                        for (int i = 0; i < 5; i++)
                            for (int j = 0; j <= i; j++, q++) end.C[i][j] = end.C[j][i] = (real)res->tl_cov[t * 15 + q];
                        xe = (real)res->tl_x[t];
                        re = row[res->tl_hits[(size_t)t * (size_t)nr + res->tl_nhits[t] - 1]];
                    } else {                /* outer end: the outward pass's state */
                        for (int i = 0; i < 5; i++) end.p[i] = (real)res->tl_opar[t * 5 + i];
                        int q = 0;
                        for (int i = 0; i < 5; i++)
                            for (int j = 0; j <= i; j++, q++) end.C[i][j] = end.C[j][i] = (real)res->tl_ocov[t * 15 + q];
                        xe = (real)res->tl_ox[t];
                        re = res->tl_orow[t];
                    }
                    int64_t pi = m * 2 + d;
                    gn[pi] = prolong(S, &k, Y, Zc, tsec[m], &end, xe, re, d == 0 ? -1 : 1, used, buf,
                                     gh + (size_t)pi * (size_t)nr, &gchi[pi], &gfin[pi], &gx[pi], &gsec[pi]);
                }
            }
            free(buf);
        }
        /* claims: each contested cluster goes to one prolongation */
        int64_t *win = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; i++) win[i] = -1;
        for (int64_t pi = 0; pi < M * 2; pi++)
            for (int j = 0; j < gn[pi]; j++) {
                int32_t c = gh[(size_t)pi * (size_t)nr + j];
                int64_t o = win[c];
                int better = o < 0;
                if (!better) {
                    int32_t ta = tk[pi / 2], tb = tk[o / 2];
                    real wa = wv[ta], wb = wv[tb];
                    if (wa > wb) better = 1;
                    else if (wa == wb && res->starts[ta] < res->starts[tb]) better = 1;
                    else if (wa == wb && res->starts[ta] == res->starts[tb] && (pi & 1) < (o & 1)) better = 1;
                }
                if (better) win[c] = pi;
            }
        /* keep only the clusters each prolongation owns, in search order */
        for (int64_t pi = 0; pi < M * 2; pi++) {
            int q = 0;
            int32_t *hp = gh + (size_t)pi * (size_t)nr;
            for (int j = 0; j < gn[pi]; j++)
                if (win[hp[j]] == pi) hp[q++] = hp[j];
            gown[pi] = q;
        }
        free(win);
        free(used);
    }

    /* A7 output: hits from the innermost to the outermost cluster (inward prolongation, the
     * sector's own clusters, outward prolongation) */
    int64_t H = 0;
    for (int64_t m = 0; m < M; m++) {
        H += res->tl_nowned[tk[m]];
        if (gown) H += gown[m * 2] + gown[m * 2 + 1];
    }
    res->n_tracks = M;
    res->n_track_hits = H;
    res->trk_hits = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H > 0 ? H : 1));
    int64_t h = 0;
    for (int64_t m = 0; m < M; m++) {
        int32_t t = tk[m];
        res->trk_tracklet[m] = t;
        res->trk_first[m] = (int32_t)h;
        int ng = 0;
        if (gown)
            for (int j = gown[m * 2] - 1; j >= 0; j--) res->trk_hits[h++] = gh[(size_t)(m * 2) * (size_t)nr + j];
        const int32_t *hh = res->tl_hits + (size_t)t * (size_t)nr;
        for (int j = res->tl_nhits[t] - 1; j >= 0; j--)
            if (res->owner[hh[j]] == t) res->trk_hits[h++] = hh[j];
        if (gown)
            for (int j = 0; j < gown[m * 2 + 1]; j++) res->trk_hits[h++] = gh[(size_t)(m * 2 + 1) * (size_t)nr + j];
        if (gown) ng = gown[m * 2] + gown[m * 2 + 1];
        res->trk_nhits[m] = res->tl_nowned[t] + ng;
        res->trk_nglobal[m] = ng;
        /* parameters: the inward prolongation's last state if it fitted any cluster */
        int inward = gn && gn[m * 2] > 0;
        for (int i = 0; i < 5; i++) res->trk_par[m * 5 + i] = inward ? (double)gfin[m * 2].p[i] : res->tl_par[t * 5 + i];
        int q = 0;
        for (int i = 0; i < 5; i++)
            for (int j = 0; j <= i; j++, q++)
                res->trk_cov[m * 15 + q] = inward ? (double)gfin[m * 2].C[i][j] : res->tl_cov[t * 15 + q];
        res->trk_x[m] = inward ? (double)gx[m * 2] : res->tl_x[t];
        res->trk_sector[m] = inward ? gsec[m * 2] : tsec[m];
        real chi = (real)res->tl_chi2[t];
        int ndf = res->tl_ndf[t];
        if (gn) {
            chi = chi + gchi[m * 2];
            chi = chi + gchi[m * 2 + 1];
            ndf += 2 * (gn[m * 2] + gn[m * 2 + 1]);
        }
        res->trk_chi2[m] = (double)chi;
        res->trk_ndf[m] = ndf;
    }
    free(tk);
    free(tsec);
    free(gh);
    free(gn);
    free(gown);
    free(gsec);
    free(gchi);
    free(gx);
    free(gfin);
    for (int s = 0; s < ns; s++)
        for (int i = 0; i < ORC_INFO_COUNT; i++) res->counters[i] += S[s].cnt[i];

    /* track merger with refit */
    {
        size_t mm = (size_t)(M > 0 ? M : 1);
        res->rf_par = (double *)calloc(mm * 5, sizeof(double));
        res->rf_cov = (double *)calloc(mm * 15, sizeof(double));
        res->rf_x = (double *)calloc(mm, sizeof(double));
        res->rf_chi2 = (double *)calloc(mm, sizeof(double));
        res->rf_ok = (int32_t *)calloc(mm, sizeof(int32_t));
        res->mg_next = (int32_t *)malloc(mm * sizeof(int32_t));
        for (size_t i = 0; i < mm; i++) res->mg_next[i] = -1;
        if (k.merge) {
            int32_t *secv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            for (int s = 0; s < ns; s++)
                for (int64_t i = S[s].off; i < S[s].off + S[s].n; i++) secv[i] = s;
#ifdef _OPENMP
            merge_tracks(&k, Y, Zc, row, secv, res, nth);
#else
            merge_tracks(&k, Y, Zc, row, secv, res, 0);
#endif
            free(secv);
        }
    }

    for (int s = 0; s < ns; s++) {
        for (int r = 0; r < nr; r++) {
            free(S[s].rows[r].cstart);
            free(S[s].rows[r].sorted);
        }
        free(S[s].rows);
        free(S[s].starts);
        free(S[s].tracks);
    }
    free(S);
    free(t0);
    free(wv);
    free(Y);
    free(Zc);
    free(k.X);
    return res;
}

/* ----------------------------------------------------------------------------------------- */
/* pieces exposed for pins                                                                    */
/* ----------------------------------------------------------------------------------------- */
int SFX(orc_propagate)(double *state, double *cov15, double x0, double x1, double bz, double sin_max)
{
    KS s;
    for (int i = 0; i < 5; i++) s.p[i] = (real)state[i];
    int q = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            s.C[i][j] = s.C[j][i] = (real)cov15[q];
            q++;
        }
    int ok = propagate(&s, (real)x0, (real)x1, (real)(-ORC_KAPPA * bz), (real)sin_max);
    for (int i = 0; i < 5; i++) state[i] = (double)s.p[i];
    q = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) cov15[q++] = (double)s.C[i][j];
    return ok;
}

#ifndef ORC_F32
int orc_rotate_f64(double *state, double *cov15, double x, double cos_d, double sin_d, double bz, double sin_max,
                   double *x_new)
{
    KS s;
    for (int i = 0; i < 5; i++) s.p[i] = state[i];
    int q = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++, q++) s.C[i][j] = s.C[j][i] = cov15[q];
    double xn = 0;
    int ok = rotate(&s, x, cos_d, sin_d, -ORC_KAPPA * bz, sin_max, &xn);
    for (int i = 0; i < 5; i++) state[i] = s.p[i];
    q = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) cov15[q++] = s.C[i][j];
    *x_new = xn;
    return ok;
}

int orc_chi2_5_f64(const double *A15, const double *d5, double *chi2)
{
    double A[5][5], d[5];
    int q = 0;
    for (int i = 0; i < 5; i++) {
        d[i] = d5[i];
        for (int j = 0; j <= i; j++) A[i][j] = A[j][i] = A15[q++];
    }
    return chi2_5(A, d, chi2);
}

int orc_seed_f64(const double *x3, const double *y3, const double *z3, double bz, double sin_max,
                 double *state)
{
    return seed3(x3, y3, z3, -ORC_KAPPA * bz, sin_max, state);
}
#endif

#ifdef ORC_F32
float orc_asin_ratio_f32(float u) { return asin_ratio(u); }

void orc_bin_row_f32(const double *y, const double *z, int n, float ymin, float zmin, float inv_dy,
                     float inv_dz, int ny, int nz, int32_t *cell, int32_t *perm, int32_t *cell_start)
{
    int nc = ny * nz;
    for (int c = 0; c <= nc; c++) cell_start[c] = 0;
    for (int i = 0; i < n; i++) {
        int iy = cell1((float)y[i], ymin, inv_dy, ny);
        int iz = cell1((float)z[i], zmin, inv_dz, nz);
        cell[i] = iz * ny + iy;
        cell_start[cell[i] + 1]++;
    }
    for (int c = 0; c < nc; c++) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    for (int c = 0; c < nc; c++) fill[c] = cell_start[c];
    for (int i = 0; i < n; i++) perm[fill[cell[i]]++] = i;
    free(fill);
}
#endif

/* Section 3.1 as the tracker applies it, for pins: weights of T tracklets from their cluster
 * counts and fit chi2 (in working precision), then the owner of each of n_clusters clusters
 * (hits: [T * n_rows], the first nhits[t] entries of row t used). */
void SFX(orc_select)(int64_t T, const int32_t *nhits, const double *chi2, const int32_t *hits, int n_rows,
                     double alpha, double beta, int64_t n_clusters, double *w_out, int32_t *owner_out)
{
    real *wv = (real *)malloc(sizeof(real) * (size_t)(T > 0 ? T : 1));
    for (int64_t t = 0; t < T; t++) {
        wv[t] = tracklet_weight(nhits[t], (real)chi2[t], (real)alpha, (real)beta);
        w_out[t] = (double)wv[t];
    }
    for (int64_t c = 0; c < n_clusters; c++) owner_out[c] = -1;
    claim_clusters(0, T, nhits, hits, n_rows, wv, owner_out);
    free(wv);
}
