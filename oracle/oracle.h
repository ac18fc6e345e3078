/* CPU oracle of the TPC sector tracker (test infrastructure only).
 *
 * A plain, slow, sequential restatement of the sector tracker of
 * Rohr et al., "ALICE HLT TPC Tracking of Pb-Pb Events on GPUs" (2012):
 * neighbours finder, evolution, tracklets from chains of one-to-one links,
 * Kalman tracklet construction and tracklet selection (Section 1), the cluster
 * weight w = n (alpha - chi2/beta) (Section 3.1), track sorting (Section 3.2)
 * and the 30-cluster minimum (Section 5).  Every point the paper leaves open is
 * fixed by a parameter in orc_config; the readings are documented next to the
 * code that applies them.
 *
 * It is compiled twice from tracker.c: once with `real` = double (suffix _f64)
 * and once with `real` = float (suffix _f32).  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code with the CUDA library.
 */
#ifndef TPC_ORACLE_H
#define TPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    /* geometry (Section 1: 2 x 18 sectors, 159 pad rows) */
    int n_rows;
    const double *row_x;      /* [n_rows] cm */
    double tan_half;          /* tan(10 deg): sector half-opening */
    double bz;                /* tesla */
    int n_sectors;
    /* measurement model */
    double sigma_y, sigma_z;  /* cluster errors (cm) */
    /* neighbours finder window and gate */
    double nb_ty, nb_tz;      /* |dy| <= ty*dx, |dz| <= tz*dx */
    double nb_gate;           /* accept score <= nb_gate * (1 + wd^2 + wu^2) */
    /* start hits */
    int min_chain;            /* clusters in a chain */
    /* construction */
    double seed_cov[5];       /* diagonal of the seed covariance */
    double win_nsigma;        /* search window half-width in sigmas */
    double chi2_max;          /* 2-dof gate on a cluster */
    int max_miss;             /* consecutive rows without a cluster that end a pass */
    double edge_margin;       /* stop when |y| > x*tan_half + margin */
    double sin_max;           /* stop when |sin phi| >= sin_max */
    /* selection */
    double alpha, beta;       /* weight w = n * (alpha - (chi2/ndf)/beta) */
    int min_clusters;         /* Section 5: 30 */
    double qpt_max;           /* low-momentum cut |q/pT| <= qpt_max */
    /* the oracle's own search grid (results do not depend on it) */
    double bin_dy, bin_dz;
    int brute_force;          /* 1: every search scans whole rows instead of grid bins */
    int n_threads;            /* OpenMP threads over sectors (<=0: runtime default) */
    int global_tracking;      /* 1: prolong tracks across sector edges (Section 5) */
    /* track merger with refit (Sections 1 and 3.3) */
    int merge;                /* 1: refit every track from its clusters and merge across sector borders */
    double merge_chi2;        /* 5-parameter chi2 gate of a merge */
    double merge_gap;         /* largest radial gap (cm) between the merged ends */
    double merge_qpt_nsigma;  /* q/pT gate in combined sigmas */
} orc_config;

/* Result of one event.  Indices of clusters are input ("original") indices. */
typedef struct orc_result orc_result;

enum {
    ORC_INFO_N = 0,           /* clusters */
    ORC_INFO_N_STARTS,        /* tracklets (= start hits) */
    ORC_INFO_N_TRACKS,
    ORC_INFO_N_TRACK_HITS,
    ORC_INFO_N_ROWS,
    ORC_INFO_VISITS,          /* construction row visits (both passes) */
    ORC_INFO_CANDIDATES,      /* construction clusters inside grid bin ranges */
    ORC_INFO_IN_WINDOW,       /* construction clusters inside the search window */
    ORC_INFO_NB_CANDIDATES,   /* neighbours finder clusters inside bin ranges (both rows) */
    ORC_INFO_UPDATES,         /* construction Kalman updates (both passes) */
    ORC_INFO_N_MERGED,        /* tracks after the merger */
    ORC_INFO_N_MERGED_HITS,
    ORC_INFO_COUNT
};

enum {
    ORC_PTR_UP_RAW = 0, ORC_PTR_DN_RAW, ORC_PTR_UP, ORC_PTR_DN,           /* int32 [N] */
    ORC_PTR_STARTS,                                                      /* int32 [T] */
    ORC_PTR_TL_NHITS, ORC_PTR_TL_NDF, ORC_PTR_TL_NUP,                    /* int32 [T] */
    ORC_PTR_TL_HITS,                                                     /* int32 [T*n_rows], outer to inner */
    ORC_PTR_TL_PAR, ORC_PTR_TL_COV, ORC_PTR_TL_X, ORC_PTR_TL_CHI2, ORC_PTR_TL_W, /* double */
    ORC_PTR_OWNER,                                                       /* int32 [N] */
    ORC_PTR_TL_NOWNED,                                                   /* int32 [T] */
    ORC_PTR_TL_ACCEPT,                                                   /* uint8 [T] */
    ORC_PTR_TRK_TRACKLET, ORC_PTR_TRK_FIRST, ORC_PTR_TRK_NHITS,          /* int32 [M] */
    ORC_PTR_TRK_HITS,                                                    /* int32 [sum nhits], inner to outer */
    ORC_PTR_TRK_PAR, ORC_PTR_TRK_COV, ORC_PTR_TRK_X, ORC_PTR_TRK_CHI2,    /* double [M*5], [M*15], [M], [M] */
    ORC_PTR_TRK_NDF, ORC_PTR_TRK_SECTOR,                                 /* int32 [M]: frame sector of par */
    ORC_PTR_TRK_NGLOBAL,                                                 /* int32 [M]: clusters added by global tracking */
    ORC_PTR_RF_PAR, ORC_PTR_RF_COV, ORC_PTR_RF_X, ORC_PTR_RF_CHI2,        /* double [M*5], [M*15], [M], [M]: refits */
    ORC_PTR_RF_OK, ORC_PTR_MG_NEXT,                                      /* int32 [M] */
    ORC_PTR_MRG_FIRST, ORC_PTR_MRG_NHITS, ORC_PTR_MRG_NSEG, ORC_PTR_MRG_HEAD, /* int32 [Mm] */
    ORC_PTR_MRG_HITS,                                                    /* int32 [sum] */
    ORC_PTR_MRG_PAR, ORC_PTR_MRG_COV, ORC_PTR_MRG_X, ORC_PTR_MRG_CHI2,    /* double */
    ORC_PTR_MRG_NDF, ORC_PTR_MRG_SECTOR, ORC_PTR_MRG_OK,                 /* int32 [Mm] */
    ORC_PTR_COUNT
};

void orc_default_config(orc_config *cfg, const double *row_x, int n_rows, int n_sectors);

orc_result *orc_track_event_f64(const orc_config *cfg, const double *y, const double *z,
                                const uint8_t *row, const int32_t *counts, int64_t n);
orc_result *orc_track_event_f32(const orc_config *cfg, const double *y, const double *z,
                                const uint8_t *row, const int32_t *counts, int64_t n);
void orc_result_info(const orc_result *r, int64_t *info /* [ORC_INFO_COUNT] */);
void orc_result_ptrs(const orc_result *r, void **ptrs /* [ORC_PTR_COUNT] */);
void orc_result_free(orc_result *r);

/* Stage pieces exposed for pins. */
/* A1: grid cell of every cluster of one row and the counting-sort permutation
 * (stable in input order).  cell[i] for i < n; perm[j] = local index of the j-th
 * cluster in cell order; cell_start[0..ny*nz]. */
void orc_bin_row_f32(const double *y, const double *z, int n, float ymin, float zmin,
                     float inv_dy, float inv_dz, int ny, int nz,
                     int32_t *cell, int32_t *perm, int32_t *cell_start);
/* Helix propagation of a state (y, z, sinphi, tanl, q/pT) from x0 to x1;
 * returns 0 when |sin phi| reaches sin_max. */
int orc_propagate_f64(double *state, double *cov15, double x0, double x1, double bz, double sin_max);
int orc_propagate_f32(double *state, double *cov15, double x0, double x1, double bz, double sin_max);
/* asin(u)/u as the float mode evaluates it (series with half-angle reduction). */
float orc_asin_ratio_f32(float u);
/* Change of frame of a state at x by an azimuth rotation (cos, sin of the angle); returns 0
 * if the direction does not point to increasing x in the new frame.  *x_new receives x'. */
int orc_rotate_f64(double *state, double *cov15, double x, double cos_d, double sin_d, double bz, double sin_max,
                   double *x_new);
/* chi2 = d^T A^-1 d of the merger's match (A: 5x5 lower triangle, row-major); returns 0 if A is
 * not positive definite. */
int orc_chi2_5_f64(const double *A15, const double *d5, double *chi2);
/* Seed state from three (x, y, z) points (first, middle, last of a chain). */
int orc_seed_f64(const double *x3, const double *y3, const double *z3, double bz, double sin_max,
                 double *state);

/* Cluster weights and ownership of Section 3.1 on given tracklets, exactly as the tracker
 * applies them: w_out[t] = n (alpha - (chi2 / ndf) / beta) with ndf = 2 n - 5 (-inf when
 * ndf < 1), owner_out[c] = the tracklet of largest weight holding cluster c, the lower index of
 * equal weights, -1 if none.  hits: [T * n_rows], the first nhits[t] entries of row t used. */
void orc_select_f64(int64_t T, const int32_t *nhits, const double *chi2, const int32_t *hits, int n_rows,
                    double alpha, double beta, int64_t n_clusters, double *w_out, int32_t *owner_out);
void orc_select_f32(int64_t T, const int32_t *nhits, const double *chi2, const int32_t *hits, int n_rows,
                    double alpha, double beta, int64_t n_clusters, double *w_out, int32_t *owner_out);

#ifdef __cplusplus
}
#endif
#endif
