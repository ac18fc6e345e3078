"""Seeded synthetic TPC events: helix tracks, their pad-row crossings, smearing and noise.

This module stands in for the Monte-Carlo simulation the paper validates its
tracker on (Section 3) and for the ALICE Pb-Pb data it times it on (Section 4);
neither is available here.  It only *produces inputs*: it holds none of the
tracker's arithmetic (no links, no fit, no selection).  Both the CPU oracle and
the CUDA path consume what it produces.

Geometry (Section 1, Fig. "Geometry of a TPC sector"): two volumes of 18
trapezoidal sectors, 159 pad rows.  Sector ``s`` has its centre at azimuth
``alpha_s = 20 deg * (s mod 18) + 10 deg``; sectors 0-17 read z >= 0 and 18-35
read z < 0.  The local frame of a sector has x along the sector centre, y in
the r-phi direction (right-handed with z) and z global.  Row k is the plane
x = x_k; a crossing belongs to the sector if |y| <= x_k tan(10 deg).

Helix convention shared with the tracker's documented state: a particle of
charge q and transverse momentum pT in a field Bz turns with signed curvature
C = dphi/ds = -kappa * Bz * q / pT (kappa = 2.99792458e-3 GeV/(T cm)), so
positive charges in +Bz bend clockwise.  The trajectory is followed for one
turn at most and stops where it leaves the drift volume (r > 250 cm or
|z| > 250 cm).  Each plane is crossed at most once with cos(phi) > 0 (leg 0,
moving to increasing local x) and once with cos(phi) < 0 (leg 1, a returning
curler).  Truth for leg 1 is quoted for the time-reversed particle
(q -> -q, tan(lambda) -> -tan(lambda), sin(phi) -> -sin(phi)), which moves
to increasing x.

Random numbers: numpy's PCG64 seeded through ``SeedSequence([seed, event])``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KAPPA = 2.99792458e-3          # GeV / (T cm): pT = kappa * B * R
N_ROWS = 159
TAN_HALF_SECTOR = math.tan(math.radians(10.0))
Z_MAX = 250.0
R_OUTER = 250.0
R_SAMPLE_MIN = 80.0            # below the innermost pad row (85.2 cm)


def default_row_x() -> np.ndarray:
    """Pad-row x positions in cm: 63 rows at 0.75 cm pitch from 85.2 cm,
    64 at 1.0 cm from 135.1 cm and 32 at 1.5 cm from 199.4 cm."""
    a = 85.2 + 0.75 * np.arange(63)
    b = 135.1 + 1.0 * np.arange(64)
    c = 199.4 + 1.5 * np.arange(32)
    return np.concatenate([a, b, c]).astype(np.float64)


@dataclasses.dataclass(frozen=True)
class Geometry:
    row_x: np.ndarray = dataclasses.field(default_factory=default_row_x)
    tan_half: float = TAN_HALF_SECTOR
    z_max: float = Z_MAX
    n_sectors: int = 36            # 36 = 2 x 18 sectors; 1 = one phi sector spanning both z halves
    bz: float = 0.5                # tesla

    @property
    def z_split(self) -> bool:
        return self.n_sectors == 36

    @property
    def n_rows(self) -> int:
        return int(self.row_x.shape[0])

    def alpha(self, sector: np.ndarray | int):
        """Centre azimuth (radians) of a sector."""
        return np.radians(20.0 * (np.asarray(sector) % 18) + 10.0)


@dataclasses.dataclass(frozen=True)
class EventSpec:
    """One event's recipe.  ``phi_lo/phi_hi`` bound the primaries' azimuth."""
    n_primaries: int = 200
    n_secondaries: int = 0
    pt_cut: float = 0.1            # GeV
    pt_mean: float = 0.5           # exponential slope above the cut
    eta_max: float = 0.9
    sigma_vz: float = 5.0          # cm
    sec_r_max: float = 60.0        # secondaries: vertex radius uniform in [0, sec_r_max]
    phi_lo: float = 0.0
    phi_hi: float = 2.0 * math.pi
    efficiency: float = 0.95       # probability that a crossing yields a cluster
    sigma_y: float = 0.08          # cm
    sigma_z: float = 0.1           # cm
    noise_frac: float = 0.05       # noise clusters per true cluster, per sector
    smear: bool = True


@dataclasses.dataclass
class Event:
    geometry: Geometry
    spec: EventSpec
    seed: int
    event_id: int
    y: np.ndarray                  # float32 [N]  local y (cm)
    z: np.ndarray                  # float32 [N]  z (cm)
    row: np.ndarray                # uint8   [N]
    counts: np.ndarray             # int32 [n_sectors * 159], clusters grouped by sector then row
    label: np.ndarray              # int32 [N]  particle*2 + leg, -1 for noise
    particles: dict                # per-particle generator parameters
    truth: np.ndarray | None = None  # float64 [N, 7]: y, z, sinphi, tanlambda, q/pT (leg convention), s, x

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    def sector_of(self) -> np.ndarray:
        return np.repeat(np.arange(self.geometry.n_sectors, dtype=np.int32),
                         self.counts.reshape(self.geometry.n_sectors, -1).sum(1))


# --------------------------------------------------------------------------------------------
# helix pieces (global frame)
# --------------------------------------------------------------------------------------------

def _norm_turn(delta: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Turning angle theta with the sign of C and |theta| in [0, 2 pi) such that
    theta == delta (mod 2 pi)."""
    two_pi = 2.0 * math.pi
    pos = np.mod(delta, two_pi)
    neg = -np.mod(-delta, two_pi)
    return np.where(c > 0, pos, neg)


def exit_arc_length(x0, y0, z0, phi0, curv, tanl, z_max=Z_MAX, r_outer=R_OUTER):
    """Arc length at which a helix leaves the volume: the first of one full turn,
    |z| = z_max, or r = r_outer (vectorised over tracks)."""
    x0, y0, z0, phi0, curv, tanl = map(np.asarray, (x0, y0, z0, phi0, curv, tanl))
    straight = np.abs(curv) < 1e-12
    c = np.where(straight, 1e-12, curv)
    s_loop = np.where(straight, np.inf, 2.0 * math.pi / np.abs(c))
    with np.errstate(divide="ignore", invalid="ignore"):
        s_z = np.where(tanl > 0, (z_max - z0) / tanl, np.where(tanl < 0, (-z_max - z0) / tanl, np.inf))
    # circle: centre (xc, yc), position P(a) = centre + (sin a, -cos a) / C with a = phi0 + C s
    xc = x0 - np.sin(phi0) / c
    yc = y0 + np.cos(phi0) / c
    dc = np.hypot(xc, yc)
    kk = (r_outer ** 2 - dc ** 2 - 1.0 / c ** 2) * c / 2.0
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = kk / dc
    ok = np.abs(ratio) <= 1.0
    beta = np.arctan2(yc, xc)
    asr = np.arcsin(np.clip(ratio, -1.0, 1.0))
    s_r = np.full(x0.shape, np.inf)
    for a in (beta + asr, beta + math.pi - asr):
        th = _norm_turn(a - phi0, c)
        s = th / c
        s = np.where(ok & (s > 0), s, np.inf)
        s_r = np.minimum(s_r, s)
    # straight line: |P0 + s d| = r_outer
    b = x0 * np.cos(phi0) + y0 * np.sin(phi0)
    disc = b * b - (x0 * x0 + y0 * y0 - r_outer ** 2)
    s_r_straight = -b + np.sqrt(np.maximum(disc, 0.0))
    s_r = np.where(straight, s_r_straight, s_r)
    return np.minimum(np.minimum(s_loop, s_z), s_r)


def helix_point(x0, y0, z0, phi0, curv, tanl, s):
    """Global position and direction azimuth after arc length s (vectorised)."""
    straight = np.abs(curv) < 1e-12
    c = np.where(straight, 1.0, curv)
    a = phi0 + curv * s
    xh = x0 + (np.sin(a) - np.sin(phi0)) / c
    yh = y0 - (np.cos(a) - np.cos(phi0)) / c
    xs = x0 + np.cos(phi0) * s
    ys = y0 + np.sin(phi0) * s
    return (np.where(straight, xs, xh), np.where(straight, ys, yh), z0 + tanl * s,
            np.where(straight, phi0, a))


def plane_crossings(x0l, y0l, z0, phil0, curv, tanl, s_end, row_x):
    """Closed-form crossings of a helix with the planes x = row_x[k] of one local frame.

    Arguments are per (track, sector) pair, already rotated into the sector frame.
    Returns arrays of shape [P, K, 2] (last axis = leg) of: valid, y, z, s, sin(phi)
    of the direction of flight at the crossing.
    """
    x0l, y0l, z0, phil0, curv, tanl, s_end = (np.asarray(v, dtype=np.float64)[:, None, None]
                                               for v in (x0l, y0l, z0, phil0, curv, tanl, s_end))
    xk = np.asarray(row_x, dtype=np.float64)[None, :, None]
    straight = np.abs(curv) < 1e-12
    c = np.where(straight, 1.0, curv)
    xc = x0l - np.sin(phil0) / c
    yc = y0l + np.cos(phil0) / c
    S = c * (xk - xc)                                    # sin of the direction angle at the plane
    hit = np.abs(S) <= 1.0
    a0 = np.arcsin(np.clip(S, -1.0, 1.0))
    legs = np.concatenate([a0, math.pi - a0], axis=2)    # leg 0: cos >= 0, leg 1: cos <= 0
    th = _norm_turn(legs - phil0, c)
    s = th / c
    y = yc - np.cos(legs) / c
    sinp = np.sin(legs)
    # straight line: one crossing, leg fixed by the sign of cos(phi)
    cs = np.cos(phil0)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_st = (xk - x0l) / cs
    y_st = y0l + np.sin(phil0) * s_st
    leg_st = np.where(cs >= 0, 0, 1)
    s_st2 = np.concatenate([np.where(leg_st == 0, s_st, np.nan), np.where(leg_st == 1, s_st, np.nan)], axis=2)
    y_st2 = np.concatenate([y_st, y_st], axis=2)
    sin_st2 = np.broadcast_to(np.sin(phil0), s_st2.shape)
    s = np.where(straight, s_st2, s)
    y = np.where(straight, y_st2, y)
    sinp = np.where(straight, sin_st2, sinp)
    hit2 = np.where(straight, np.isfinite(s), np.concatenate([hit, hit], axis=2))
    valid = hit2 & (s > 0) & (s < s_end)
    z = z0 + tanl * s
    return valid, y, z, s, sinp


# --------------------------------------------------------------------------------------------
# event assembly
# --------------------------------------------------------------------------------------------

def _rng(seed: int, event: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(event)])))


def _draw_particles(spec: EventSpec, geo: Geometry, rng: np.random.Generator) -> dict:
    n1, n2 = spec.n_primaries, spec.n_secondaries
    n = n1 + n2
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    pt = spec.pt_cut + rng.exponential(spec.pt_mean, n)
    eta = rng.uniform(-spec.eta_max, spec.eta_max, n)
    phi = np.empty(n)
    phi[:n1] = rng.uniform(spec.phi_lo, spec.phi_hi, n1)
    phi[n1:] = rng.uniform(0.0, 2.0 * math.pi, n2)
    vx = np.zeros(n)
    vy = np.zeros(n)
    vz = rng.normal(0.0, spec.sigma_vz, n)
    if n2:
        r = rng.uniform(0.0, spec.sec_r_max, n2)
        ang = rng.uniform(0.0, 2.0 * math.pi, n2)
        vx[n1:] = r * np.cos(ang)
        vy[n1:] = r * np.sin(ang)
    curv = -KAPPA * geo.bz * q / pt
    tanl = np.sinh(eta)
    return dict(q=q, pt=pt, eta=eta, phi=phi, vx=vx, vy=vy, vz=vz, curv=curv, tanl=tanl,
                secondary=np.arange(n) >= n1)


def _candidate_pairs(p: dict, geo: Geometry, s_end: np.ndarray, n_samples: int = 256):
    """(track, sector) pairs that may hold crossings: sectors the sampled trajectory
    visits at r >= 80 cm, plus their azimuthal neighbours on the same side.  The exact
    solver decides; this only prunes."""
    n = p["q"].shape[0]
    if geo.n_sectors == 1:
        return np.arange(n), np.zeros(n, dtype=np.int64)
    frac = (np.arange(n_samples) + 0.5) / n_samples
    s = s_end[:, None] * frac[None, :]
    x, y, z, _ = helix_point(p["vx"][:, None], p["vy"][:, None], p["vz"][:, None], p["phi"][:, None],
                             p["curv"][:, None], p["tanl"][:, None], s)
    r = np.hypot(x, y)
    az = np.floor(np.mod(np.arctan2(y, x), 2 * math.pi) / math.radians(20.0)).astype(np.int64) % 18
    side = (z < 0).astype(np.int64)
    inside = r >= R_SAMPLE_MIN
    trk = np.broadcast_to(np.arange(n)[:, None], r.shape)[inside]
    key = trk * 36 + side[inside] * 18 + az[inside]
    key = np.unique(key)
    t = key // 36
    sec = key % 36
    side_k = sec // 18
    az_k = sec % 18
    keys = [key]
    for d in (-1, 1):
        keys.append(t * 36 + side_k * 18 + (az_k + d) % 18)
    key = np.unique(np.concatenate(keys))
    return key // 36, key % 36


def generate_event(spec: EventSpec, geo: Geometry | None = None, seed: int = 1, event: int = 0,
                   truth: bool = False, chunk: int = 4096) -> Event:
    geo = geo or Geometry()
    rng = _rng(seed, event)
    p = _draw_particles(spec, geo, rng)
    s_end = exit_arc_length(p["vx"], p["vy"], p["vz"], p["phi"], p["curv"], p["tanl"], geo.z_max)
    trk, sec = _candidate_pairs(p, geo, s_end)
    row_x = geo.row_x
    cols = {k: [] for k in ("trk", "sec", "row", "leg", "y", "z", "s", "sinp")}
    for lo in range(0, trk.shape[0], chunk):
        t = trk[lo:lo + chunk]
        sc = sec[lo:lo + chunk]
        al = geo.alpha(sc)
        ca, sa = np.cos(al), np.sin(al)
        x0l = p["vx"][t] * ca + p["vy"][t] * sa
        y0l = -p["vx"][t] * sa + p["vy"][t] * ca
        phil = p["phi"][t] - al
        valid, y, z, s, sinp = plane_crossings(x0l, y0l, p["vz"][t], phil, p["curv"][t], p["tanl"][t],
                                               s_end[t], row_x)
        xk = row_x[None, :, None]
        valid &= np.abs(y) <= xk * geo.tan_half
        valid &= np.abs(z) < geo.z_max
        if geo.z_split:
            side = (sc >= 18)[:, None, None]
            valid &= np.where(side, z < 0, z >= 0)
        ip, ik, il = np.nonzero(valid)
        cols["trk"].append(t[ip])
        cols["sec"].append(sc[ip])
        cols["row"].append(ik)
        cols["leg"].append(il)
        for name, arr in (("y", y), ("z", z), ("s", s), ("sinp", sinp)):
            cols[name].append(arr[ip, ik, il])
    c = {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in cols.items()}
    ntrue_all = c["y"].shape[0]
    keep = rng.random(ntrue_all) < spec.efficiency
    c = {k: v[keep] for k, v in c.items()}
    nt = c["y"].shape[0]
    if spec.smear:
        ys = c["y"] + rng.normal(0.0, spec.sigma_y, nt)
        zs = c["z"] + rng.normal(0.0, spec.sigma_z, nt)
    else:
        ys, zs = c["y"].copy(), c["z"].copy()
    trk_i = c["trk"].astype(np.int64)
    leg = c["leg"].astype(np.int64)
    label = (trk_i * 2 + leg).astype(np.int32)
    sector = c["sec"].astype(np.int64)
    row = c["row"].astype(np.int64)
    # noise: per sector, round(noise_frac * true clusters of that sector)
    ns = geo.n_sectors
    ntrue_sec = np.bincount(sector, minlength=ns)
    nnoise = np.rint(spec.noise_frac * ntrue_sec).astype(np.int64)
    nn = int(nnoise.sum())
    nsec = np.repeat(np.arange(ns), nnoise)
    nrow = rng.integers(0, geo.n_rows, nn)
    half = row_x[nrow] * geo.tan_half
    ny = rng.uniform(-1.0, 1.0, nn) * half
    if geo.z_split:
        nz = rng.uniform(0.0, geo.z_max, nn)
        nz = np.where(nsec >= 18, -nz, nz)
    else:
        nz = rng.uniform(-geo.z_max, geo.z_max, nn)
    all_sec = np.concatenate([sector, nsec])
    all_row = np.concatenate([row, nrow])
    all_y = np.concatenate([ys, ny])
    all_z = np.concatenate([zs, nz])
    all_label = np.concatenate([label, np.full(nn, -1, np.int32)])
    # group by (sector, row), random order inside a group
    shuffle = rng.permutation(all_y.shape[0])
    grp = (all_sec * geo.n_rows + all_row)[shuffle]
    order = shuffle[np.argsort(grp, kind="stable")]
    counts = np.bincount(all_sec * geo.n_rows + all_row, minlength=ns * geo.n_rows).astype(np.int32)
    tr = None
    if truth:
        tsin = np.where(leg == 0, c["sinp"], -c["sinp"])
        tq = p["q"][trk_i] / p["pt"][trk_i]
        ttl = p["tanl"][trk_i]
        flip = np.where(leg == 0, 1.0, -1.0)
        tr_true = np.stack([c["y"], c["z"], tsin, ttl * flip, tq * flip, c["s"], row_x[row]], axis=1)
        tr = np.full((all_y.shape[0], 7), np.nan)
        tr[:nt] = tr_true
        tr = tr[order]
    return Event(geometry=geo, spec=spec, seed=seed, event_id=event,
                 y=all_y[order].astype(np.float32), z=all_z[order].astype(np.float32),
                 row=all_row[order].astype(np.uint8), counts=counts, label=all_label[order],
                 particles=p, truth=tr)


# --------------------------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------------------------

def config_event(cfg: int, event: int = 0, seed: int = 1, truth: bool = False) -> Event:
    """The standard workloads.

    0: one phi sector (both z halves), 200 primaries within the sector, 5 % noise.
    1: 36 sectors, 4000 primaries over 2 pi, 10 % noise.
    2: central-like, 16000 primaries + 3000 secondaries (vertex radius U[0, 60] cm),
       pT cut 0.05 GeV, 20 % noise.
    3: one event of the batched workload: primaries log-uniform in [500, 16000],
       noise fraction uniform in [5 %, 20 %]; event ``event`` is seeded with (seed, event).
    """
    if cfg == 0:
        geo = Geometry(n_sectors=1)
        spec = EventSpec(n_primaries=200, phi_lo=0.0, phi_hi=math.radians(20.0), noise_frac=0.05)
    elif cfg == 1:
        geo = Geometry()
        spec = EventSpec(n_primaries=4000, noise_frac=0.10)
    elif cfg == 2:
        geo = Geometry()
        spec = EventSpec(n_primaries=16000, n_secondaries=3000, pt_cut=0.05, noise_frac=0.20)
    elif cfg == 3:
        geo = Geometry()
        r = _rng(seed, 1_000_000 + event)
        npri = int(round(math.exp(r.uniform(math.log(500.0), math.log(16000.0)))))
        spec = EventSpec(n_primaries=npri, noise_frac=float(r.uniform(0.05, 0.20)))
    else:
        raise ValueError("unknown workload %r" % cfg)
    return generate_event(spec, geo, seed=seed, event=event, truth=truth)
