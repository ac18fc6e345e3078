/* Oracle-internal result layout, shared by the two precision builds of tracker.c
 * and by common.c.  Test infrastructure only. */
#ifndef TPC_ORACLE_INTERNAL_H
#define TPC_ORACLE_INTERNAL_H
#include "oracle.h"

#define ORC_KAPPA 2.99792458e-3   /* GeV / (T cm) */

struct orc_result {
    int64_t n, n_starts, n_tracks, n_track_hits;
    int n_rows;
    int64_t counters[ORC_INFO_COUNT];
    int32_t *up_raw, *dn_raw, *up, *dn;
    int32_t *starts;
    int32_t *tl_nhits, *tl_ndf, *tl_nup, *tl_hits;
    double *tl_par, *tl_cov, *tl_x, *tl_chi2, *tl_w;
    int32_t *owner, *tl_nowned;
    uint8_t *tl_accept;
    int32_t *trk_tracklet, *trk_first, *trk_nhits, *trk_hits;
    double *tl_opar, *tl_ocov, *tl_ox;   /* outward-pass state at its last cluster (global tracking) */
    int32_t *tl_orow;
    double *trk_par, *trk_cov, *trk_x, *trk_chi2;
    int32_t *trk_ndf, *trk_sector, *trk_nglobal;
    /* track merger: refit of every sector track, outward partner, merged tracks */
    double *rf_par, *rf_cov, *rf_x, *rf_chi2;
    int32_t *rf_ok, *mg_next;
    int64_t n_merged, n_merged_hits;
    int32_t *mrg_first, *mrg_nhits, *mrg_nseg, *mrg_head, *mrg_hits, *mrg_ndf, *mrg_sector, *mrg_ok;
    double *mrg_par, *mrg_cov, *mrg_x, *mrg_chi2;
};

orc_result *orc_result_alloc(int64_t n, int n_rows);
void orc_result_alloc_tracklets(orc_result *r, int64_t n_starts);

#endif
