"""Pins of the cluster weight and ownership of Section 3.1, and of the fit chi2 the weight uses.

1. A hand-derived golden (tests/golden/weight_shared_clusters.json): five tracklets sharing
   clusters, the weights w = n (alpha - (chi2/ndf) / beta) worked out by hand for four (alpha,
   beta) pairs, and the owner of every cluster.  The shorter tracklet with the smaller chi2/ndf
   wins the shared clusters at alpha = 1, the longer one at alpha = 6 and in the longest-wins
   limit; equal weights go to the earlier tracklet; a tracklet with ndf < 1 claims nothing.
   It runs through orc_select, the same two functions the tracker's construction and selection
   call, in both precisions.
2. The golden fails on copies of the oracle with a planted mistake in the weight (raw chi2,
   beta applied twice, chi2 per cluster instead of per degree of freedom, ndf as the multiplier)
   or in the tie rule, so a wrong reading of the formula cannot pass.
3. The chi2 the weight uses, end to end: at zero field a straight track along the sector centre
   (y = 0) with z offsets is a linear Gaussian problem in (z, tan lambda), and the sum of the
   Kalman update chi2 of a pass equals the minimum of the regularised least-squares objective of
   that pass (prior state and covariance plus all its measurements).  The oracle's tracklet chi2,
   inner state and weight are checked against that closed form, computed here with numpy.
"""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1712_09407_gb300 import eventgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "weight_shared_clusters.json")
ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))


def _golden():
    g = json.load(open(GOLDEN))
    tracklets = [(list(range(t["first"], t["last"] + 1)), t["chi2"]) for t in g["tracklets"]]
    return g, tracklets


def _check_golden(library=None, precision=64):
    """Mismatches of the oracle (or a rebuilt copy) against the hand-derived golden."""
    g, tracklets = _golden()
    bad = []
    rtol = 1e-12 if precision == 64 else 1e-6
    for case in g["cases"]:
        w, owner = oracle.select(tracklets, case["alpha"], case["beta"], g["n_clusters"], precision=precision,
                                 library=library)
        for t, (got, want) in enumerate(zip(w, case["weights"])):
            want = -np.inf if want == "-inf" else float(want)
            if not (got == want or abs(got - want) <= rtol * abs(want)):
                bad.append(("weight", case["alpha"], case["beta"], t, got, want))
        expect = np.full(g["n_clusters"], -1)
        for lo, hi, t in case["owners"]:
            expect[lo:hi + 1] = t
        if not np.array_equal(owner, expect):
            bad.append(("owners", case["alpha"], case["beta"], np.nonzero(owner != expect)[0][:5].tolist()))
    return bad


@pytest.mark.parametrize("precision", [64, 32])
def test_weights_and_owners_match_hand_derivation(precision):
    assert _check_golden(precision=precision) == []


MUTANTS = {
    "raw chi2": ("(real)n * (alpha - (chi2sum / (real)ndf) / beta)", "(real)n * (alpha - chi2sum / beta)"),
    "beta twice": ("(real)n * (alpha - (chi2sum / (real)ndf) / beta)",
                   "(real)n * (alpha - ((chi2sum / (real)ndf) / beta) / beta)"),
    "chi2 per cluster": ("(real)n * (alpha - (chi2sum / (real)ndf) / beta)", "(real)n * (alpha - (chi2sum / (real)n) / beta)"),
    "ndf as multiplier": ("(real)n * (alpha - (chi2sum / (real)ndf) / beta)",
                          "(real)ndf * (alpha - (chi2sum / (real)ndf) / beta)"),
    "ties to the later": ("if (o < 0 || wv[t] > wv[o]) owner[c] = (int32_t)t;",
                          "if (o < 0 || wv[t] >= wv[o]) owner[c] = (int32_t)t;"),
}


def _build_mutant(tmp, name):
    old, new = MUTANTS[name]
    d = tmp / name.replace(" ", "_")
    d.mkdir()
    for f in ("common.c", "tracker.c", "oracle.h", "oracle_internal.h"):
        shutil.copy(os.path.join(ORACLE_DIR, f), d / f)
    src = (d / "tracker.c").read_text()
    assert src.count(old) == 1, "the planted line is no longer in the oracle: %s" % name
    (d / "tracker.c").write_text(src.replace(old, new))
    flags = ["-O2", "-fPIC", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-w"]
    objs = []
    for src_, extra, obj in [("common.c", [], "common.o"), ("tracker.c", [], "f64.o"), ("tracker.c", ["-DORC_F32"], "f32.o")]:
        subprocess.check_call(["gcc", *flags, *extra, "-c", str(d / src_), "-o", str(d / obj)])
        objs.append(str(d / obj))
    so = d / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-shared", "-fopenmp", *objs, "-o", str(so), "-lm"])
    L = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    for pre in ("f64", "f32"):
        f = getattr(L, "orc_select_" + pre)
        f.restype = None
        f.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64, P, P]
    return L


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_weight_mistakes_fail_the_golden(tmp_path, name):
    L = _build_mutant(tmp_path, name)
    assert _check_golden(library=L, precision=64) != [], name
    assert _check_golden(library=L, precision=32) != [], name


# ------------------------------------------------------------------------------------------------
# the fit chi2, end to end, against the least-squares minimum of a linear problem
# ------------------------------------------------------------------------------------------------
def _straight_track(seed=3, sigma=0.03, slope=0.3, z0=-20.0):
    geo = eventgen.Geometry(n_sectors=1, bz=0.0)
    x = np.asarray(geo.row_x, dtype=np.float64)
    rng = np.random.default_rng(seed)
    z = z0 + slope * x + rng.normal(0.0, sigma, x.shape[0])
    y = np.zeros_like(z)
    row = np.arange(x.shape[0], dtype=np.uint8)
    counts = np.ones(x.shape[0], dtype=np.int32)
    return geo, x, y, z, row, counts


def _ls_pass(x_ref, mu, P0, xs, ms, R):
    """Regularised least squares of theta = (z at x_ref, tan lambda) with prior (mu, P0) and
    measurements z_k = theta0 + theta1 (x_k - x_ref) of variance R: the minimiser and the minimum."""
    H = np.stack([np.ones_like(xs), xs - x_ref], axis=1)
    Pi = np.linalg.inv(P0)
    A = Pi + H.T @ H / R
    b = Pi @ mu + H.T @ ms / R
    th = np.linalg.solve(A, b)
    r = ms - H @ th
    J = float((th - mu) @ Pi @ (th - mu) + r @ r / R)
    return th, J


@pytest.mark.parametrize("precision", [64, 32])
def test_fit_chi2_equals_least_squares_minimum(precision):
    geo, x, y, z, row, counts = _straight_track()
    cfg = oracle.config_for(geo)
    assert cfg.bz == 0.0
    res = oracle.track_event(cfg, y, z, row, counts, precision=precision)
    # one chain of one-to-one links: rows 1 .. 157 (rows 0 and 158 get no links)
    assert res.starts.tolist() == [1], res.starts
    assert res.tl_nhits[0] == 159 and res.tl_nup[0] == 158
    R = cfg.sigma_z ** 2
    P0 = np.diag([cfg.seed_cov[1], cfg.seed_cov[3]])
    # seed from the chain's first, middle and last clusters (rows 1, 79, 157)
    mu = np.array([z[1], (z[157] - z[1]) / (x[157] - x[1])])
    # outward pass: rows 1 .. 158 from the seed at x_1; its state at x_158 starts the inward pass
    th, _ = _ls_pass(x[1], mu, P0, x[1:], z[1:], R)
    mu_in = np.array([th[0] + th[1] * (x[158] - x[1]), th[1]])
    # inward pass: covariance reset, rows 158 .. 0; its chi2 is the tracklet's
    th_in, chi2 = _ls_pass(x[158], mu_in, P0, x, z, R)
    tol = 1e-9 if precision == 64 else 2e-4
    assert abs(res.tl_chi2[0] - chi2) <= tol * chi2, (res.tl_chi2[0], chi2)
    assert abs(res.tl_par[0, 1] - (th_in[0] + th_in[1] * (x[0] - x[158]))) <= (1e-9 if precision == 64 else 1e-4)
    assert abs(res.tl_par[0, 3] - th_in[1]) <= (1e-12 if precision == 64 else 1e-6)
    assert res.tl_par[0, 0] == 0.0 and res.tl_par[0, 2] == 0.0      # y and sin phi stay exactly 0
    # the weight of Section 3.1 from n and this chi2, through the golden-pinned function
    w, owner = oracle.select([(list(range(159)), chi2)], cfg.alpha, cfg.beta, 159, precision=precision)
    assert abs(res.tl_w[0] - w[0]) <= tol * abs(w[0])
    assert res.owner.tolist() == [0] * 159
