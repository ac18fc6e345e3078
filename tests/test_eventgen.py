"""Pins of the synthetic event generator (the stand-in for the paper's Monte-Carlo, Section 3)."""
import math

import numpy as np
import pytest

from paper_1712_09407_gb300 import eventgen as eg


def _local_x_of_s(p, i, alpha, s):
    x, y, z, _ = eg.helix_point(p["vx"][i], p["vy"][i], p["vz"][i], p["phi"][i], p["curv"][i], p["tanl"][i], s)
    ca, sa = math.cos(alpha), math.sin(alpha)
    return x * ca + y * sa, -x * sa + y * ca, z


def test_crossings_match_numeric_march():
    """Closed-form circle/plane crossings against a fine march along the arc plus bisection."""
    geo = eg.Geometry()
    spec = eg.EventSpec(n_primaries=40, n_secondaries=10, pt_cut=0.07, efficiency=1.0, smear=False,
                        noise_frac=0.0)
    ev = eg.generate_event(spec, geo, seed=3, truth=True)
    p = ev.particles
    sec = ev.sector_of()
    rng = np.random.default_rng(0)
    idx = rng.choice(ev.n, size=min(200, ev.n), replace=False)
    worst = 0.0
    for c in idx:
        i = ev.label[c] // 2
        alpha = float(geo.alpha(sec[c]))
        s_true = ev.truth[c, 5]
        xk = geo.row_x[ev.row[c]]
        # march with 0.05 cm steps from s = 0 and bracket the crossing closest to s_true
        grid = np.arange(0.0, s_true + 1.0, 0.05)
        xs, _, _ = _local_x_of_s(p, i, alpha, grid)
        f = xs - xk
        sgn = np.nonzero(np.sign(f[:-1]) != np.sign(f[1:]))[0]
        assert sgn.size, "march found no crossing"
        j = sgn[np.argmin(np.abs(grid[sgn] - s_true))]
        lo, hi = grid[j], grid[j + 1]
        flo = f[j]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = _local_x_of_s(p, i, alpha, mid)[0] - xk
            if np.sign(fm) == np.sign(flo):
                lo, flo = mid, fm
            else:
                hi = mid
            if hi - lo < 1e-14:
                break
        s_m = 0.5 * (lo + hi)
        _, ym, zm = _local_x_of_s(p, i, alpha, s_m)
        worst = max(worst, abs(ym - ev.truth[c, 0]), abs(zm - ev.truth[c, 1]), abs(s_m - s_true))
    assert worst < 1e-10, worst


def test_truth_direction_is_derivative_of_position():
    """sin(phi) and tan(lambda) of the truth are the derivatives of the crossing point."""
    geo = eg.Geometry()
    spec = eg.EventSpec(n_primaries=20, pt_cut=0.08, efficiency=1.0, smear=False, noise_frac=0.0)
    ev = eg.generate_event(spec, geo, seed=11, truth=True)
    p = ev.particles
    sec = ev.sector_of()
    for c in range(0, ev.n, max(1, ev.n // 100)):
        i = ev.label[c] // 2
        leg = ev.label[c] % 2
        alpha = float(geo.alpha(sec[c]))
        s = ev.truth[c, 5]
        h = 1e-5
        x1, y1, z1 = _local_x_of_s(p, i, alpha, s + h)
        x0, y0, z0 = _local_x_of_s(p, i, alpha, s - h)
        dirn = 1.0 if leg == 0 else -1.0          # leg 1 is quoted time-reversed
        sinphi = dirn * (y1 - y0) / (2 * h)
        cosphi = dirn * (x1 - x0) / (2 * h)
        assert cosphi > 0
        assert abs(sinphi - ev.truth[c, 2]) < 1e-6
        assert abs(dirn * (z1 - z0) / (2 * h) - ev.truth[c, 3]) < 1e-6
        assert abs(dirn * p["q"][i] / p["pt"][i] - ev.truth[c, 4]) < 1e-12


def test_event_layout_and_determinism():
    ev = eg.config_event(1)
    ev2 = eg.config_event(1)
    assert np.array_equal(ev.y, ev2.y) and np.array_equal(ev.z, ev2.z)
    assert ev.counts.shape == (36 * 159,) and int(ev.counts.sum()) == ev.n
    rows = np.repeat(np.tile(np.arange(159), 36), ev.counts)
    assert np.array_equal(rows, ev.row.astype(np.int64))
    sec = ev.sector_of()
    # acceptance: |y| within the row half-width (plus smearing), z on the sector's side
    half = ev.geometry.row_x[ev.row] * ev.geometry.tan_half
    assert np.all(np.abs(ev.y) <= half + 1.0)
    assert np.all((ev.z[sec < 18] >= -1.0)) and np.all(ev.z[sec >= 18] <= 1.0)
    noise = (ev.label < 0).mean()
    assert 0.08 < noise / (1 - noise) < 0.12          # 10 % noise per true cluster
    other = eg.config_event(1, seed=2)
    assert not np.array_equal(other.y[:100], ev.y[:100])


def test_workload_sizes():
    ev0 = eg.config_event(0)
    assert ev0.geometry.n_sectors == 1 and ev0.counts.shape == (159,)
    ev3a, ev3b = eg.config_event(3, event=0), eg.config_event(3, event=1)
    assert ev3a.n != ev3b.n
