/* Oracle configuration defaults and result bookkeeping (test infrastructure only). */
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"

/* Defaults.  Only alpha = 6 (Section 3.1) and 30 clusters (Section 5) come from
 * the paper; every other value is a reading of a point the paper leaves open. */
void orc_default_config(orc_config *c, const double *row_x, int n_rows, int n_sectors)
{
    memset(c, 0, sizeof *c);
    c->n_rows = n_rows;
    c->row_x = row_x;
    c->tan_half = 0.17632698070846498;   /* tan(10 deg) */
    c->bz = 0.5;
    c->n_sectors = n_sectors;
    c->sigma_y = 0.08;
    c->sigma_z = 0.1;
    c->nb_ty = 1.0;
    c->nb_tz = 2.0;
    c->nb_gate = 9.0;
    c->min_chain = 3;
    c->seed_cov[0] = 0.08 * 0.08;
    c->seed_cov[1] = 0.1 * 0.1;
    c->seed_cov[2] = 0.01;
    c->seed_cov[3] = 0.01;
    c->seed_cov[4] = 1.0;
    c->win_nsigma = 3.0;
    c->chi2_max = 16.0;
    c->max_miss = 10;
    c->edge_margin = 2.0;
    c->sin_max = 0.99;
    c->alpha = 6.0;
    c->beta = 1.0;
    c->min_clusters = 30;
    c->qpt_max = 20.0;
    c->bin_dy = 2.0;
    c->bin_dz = 4.0;
    c->brute_force = 0;
    c->n_threads = 0;
    c->global_tracking = 0;
    c->merge = 0;
    c->merge_chi2 = 25.0;
    c->merge_gap = 40.0;
    c->merge_qpt_nsigma = 5.0;
}

orc_result *orc_result_alloc(int64_t n, int n_rows)
{
    orc_result *r = (orc_result *)calloc(1, sizeof *r);
    size_t nn = (size_t)(n > 0 ? n : 1);
    r->n = n;
    r->n_rows = n_rows;
    r->up_raw = (int32_t *)malloc(nn * sizeof(int32_t));
    r->dn_raw = (int32_t *)malloc(nn * sizeof(int32_t));
    r->up = (int32_t *)malloc(nn * sizeof(int32_t));
    r->dn = (int32_t *)malloc(nn * sizeof(int32_t));
    r->owner = (int32_t *)malloc(nn * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) {
        r->up_raw[i] = r->dn_raw[i] = r->up[i] = r->dn[i] = r->owner[i] = -1;
    }
    return r;
}

void orc_result_alloc_tracklets(orc_result *r, int64_t t)
{
    size_t tt = (size_t)(t > 0 ? t : 1);
    r->n_starts = t;
    r->starts = (int32_t *)malloc(tt * sizeof(int32_t));
    r->tl_nhits = (int32_t *)calloc(tt, sizeof(int32_t));
    r->tl_ndf = (int32_t *)calloc(tt, sizeof(int32_t));
    r->tl_nup = (int32_t *)calloc(tt, sizeof(int32_t));
    r->tl_hits = (int32_t *)malloc(tt * (size_t)r->n_rows * sizeof(int32_t));
    for (size_t i = 0; i < tt * (size_t)r->n_rows; i++) r->tl_hits[i] = -1;
    r->tl_par = (double *)calloc(tt * 5, sizeof(double));
    r->tl_cov = (double *)calloc(tt * 15, sizeof(double));
    r->tl_x = (double *)calloc(tt, sizeof(double));
    r->tl_chi2 = (double *)calloc(tt, sizeof(double));
    r->tl_w = (double *)calloc(tt, sizeof(double));
    r->tl_nowned = (int32_t *)calloc(tt, sizeof(int32_t));
    r->tl_accept = (uint8_t *)calloc(tt, 1);
    r->trk_tracklet = (int32_t *)malloc(tt * sizeof(int32_t));
    r->trk_first = (int32_t *)malloc(tt * sizeof(int32_t));
    r->trk_nhits = (int32_t *)malloc(tt * sizeof(int32_t));
    r->tl_opar = (double *)calloc(tt * 5, sizeof(double));
    r->tl_ocov = (double *)calloc(tt * 15, sizeof(double));
    r->tl_ox = (double *)calloc(tt, sizeof(double));
    r->tl_orow = (int32_t *)calloc(tt, sizeof(int32_t));
    r->trk_par = (double *)calloc(tt * 5, sizeof(double));
    r->trk_cov = (double *)calloc(tt * 15, sizeof(double));
    r->trk_x = (double *)calloc(tt, sizeof(double));
    r->trk_chi2 = (double *)calloc(tt, sizeof(double));
    r->trk_ndf = (int32_t *)calloc(tt, sizeof(int32_t));
    r->trk_sector = (int32_t *)calloc(tt, sizeof(int32_t));
    r->trk_nglobal = (int32_t *)calloc(tt, sizeof(int32_t));
}

void orc_result_info(const orc_result *r, int64_t *info)
{
    for (int i = 0; i < ORC_INFO_COUNT; i++) info[i] = r->counters[i];
    info[ORC_INFO_N] = r->n;
    info[ORC_INFO_N_STARTS] = r->n_starts;
    info[ORC_INFO_N_TRACKS] = r->n_tracks;
    info[ORC_INFO_N_TRACK_HITS] = r->n_track_hits;
    info[ORC_INFO_N_ROWS] = r->n_rows;
    info[ORC_INFO_N_MERGED] = r->n_merged;
    info[ORC_INFO_N_MERGED_HITS] = r->n_merged_hits;
}

void orc_result_ptrs(const orc_result *r, void **p)
{
    p[ORC_PTR_UP_RAW] = r->up_raw;
    p[ORC_PTR_DN_RAW] = r->dn_raw;
    p[ORC_PTR_UP] = r->up;
    p[ORC_PTR_DN] = r->dn;
    p[ORC_PTR_STARTS] = r->starts;
    p[ORC_PTR_TL_NHITS] = r->tl_nhits;
    p[ORC_PTR_TL_NDF] = r->tl_ndf;
    p[ORC_PTR_TL_NUP] = r->tl_nup;
    p[ORC_PTR_TL_HITS] = r->tl_hits;
    p[ORC_PTR_TL_PAR] = r->tl_par;
    p[ORC_PTR_TL_COV] = r->tl_cov;
    p[ORC_PTR_TL_X] = r->tl_x;
    p[ORC_PTR_TL_CHI2] = r->tl_chi2;
    p[ORC_PTR_TL_W] = r->tl_w;
    p[ORC_PTR_OWNER] = r->owner;
    p[ORC_PTR_TL_NOWNED] = r->tl_nowned;
    p[ORC_PTR_TL_ACCEPT] = r->tl_accept;
    p[ORC_PTR_TRK_TRACKLET] = r->trk_tracklet;
    p[ORC_PTR_TRK_FIRST] = r->trk_first;
    p[ORC_PTR_TRK_NHITS] = r->trk_nhits;
    p[ORC_PTR_TRK_HITS] = r->trk_hits;
    p[ORC_PTR_TRK_PAR] = r->trk_par;
    p[ORC_PTR_TRK_COV] = r->trk_cov;
    p[ORC_PTR_TRK_X] = r->trk_x;
    p[ORC_PTR_TRK_CHI2] = r->trk_chi2;
    p[ORC_PTR_TRK_NDF] = r->trk_ndf;
    p[ORC_PTR_TRK_SECTOR] = r->trk_sector;
    p[ORC_PTR_TRK_NGLOBAL] = r->trk_nglobal;
    p[ORC_PTR_RF_PAR] = r->rf_par;
    p[ORC_PTR_RF_COV] = r->rf_cov;
    p[ORC_PTR_RF_X] = r->rf_x;
    p[ORC_PTR_RF_CHI2] = r->rf_chi2;
    p[ORC_PTR_RF_OK] = r->rf_ok;
    p[ORC_PTR_MG_NEXT] = r->mg_next;
    p[ORC_PTR_MRG_FIRST] = r->mrg_first;
    p[ORC_PTR_MRG_NHITS] = r->mrg_nhits;
    p[ORC_PTR_MRG_NSEG] = r->mrg_nseg;
    p[ORC_PTR_MRG_HEAD] = r->mrg_head;
    p[ORC_PTR_MRG_HITS] = r->mrg_hits;
    p[ORC_PTR_MRG_PAR] = r->mrg_par;
    p[ORC_PTR_MRG_COV] = r->mrg_cov;
    p[ORC_PTR_MRG_X] = r->mrg_x;
    p[ORC_PTR_MRG_CHI2] = r->mrg_chi2;
    p[ORC_PTR_MRG_NDF] = r->mrg_ndf;
    p[ORC_PTR_MRG_SECTOR] = r->mrg_sector;
    p[ORC_PTR_MRG_OK] = r->mrg_ok;
}

void orc_result_free(orc_result *r)
{
    if (!r) return;
    free(r->up_raw); free(r->dn_raw); free(r->up); free(r->dn); free(r->owner);
    free(r->starts); free(r->tl_nhits); free(r->tl_ndf); free(r->tl_nup); free(r->tl_hits);
    free(r->tl_par); free(r->tl_cov); free(r->tl_x); free(r->tl_chi2); free(r->tl_w);
    free(r->tl_nowned); free(r->tl_accept);
    free(r->trk_tracklet); free(r->trk_first); free(r->trk_nhits); free(r->trk_hits);
    free(r->tl_opar); free(r->tl_ocov); free(r->tl_ox); free(r->tl_orow);
    free(r->trk_par); free(r->trk_cov); free(r->trk_x); free(r->trk_chi2);
    free(r->trk_ndf); free(r->trk_sector); free(r->trk_nglobal);
    free(r->rf_par); free(r->rf_cov); free(r->rf_x); free(r->rf_chi2); free(r->rf_ok); free(r->mg_next);
    free(r->mrg_first); free(r->mrg_nhits); free(r->mrg_nseg); free(r->mrg_head); free(r->mrg_hits);
    free(r->mrg_par); free(r->mrg_cov); free(r->mrg_x); free(r->mrg_chi2); free(r->mrg_ndf);
    free(r->mrg_sector); free(r->mrg_ok);
    free(r);
}
