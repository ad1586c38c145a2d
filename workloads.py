"""Seeded synthetic inputs for batched 2-D distance reporting.

This module only draws numbers: it holds none of the method's arithmetic (no keys, no
ranges, no distance tests), and both the CUDA path and the CPU oracle read what it returns.
Coordinates are int32 in [0, 2^30); radii are int32 >= 0.

Workloads (shapes of the paper's experiments, Sec. 3; the paper's real-world data sets are
not available, so synthetic stand-ins with their structure are used):

  uniform-1e5      n = 100,000 uniform in [0, 2^20)^2; m = 10,000 uniform queries in the same
                   box; one radius 8366, so that about 20 points fall in each disc
                   (density 1e5 / 2^40, pi * 8366^2 * 1e5 / 2^40 = 20.0).  Seed 1.
  mixed-1e7        n = 10^7: half uniform in [0, 2^30)^2, half from 1,000 isotropic Gaussian
                   clusters (sigma 2^18, centres uniform, cluster picked uniformly; rounded and
                   clamped); m = 10^6 queries at random data points; per-query radius set
                   from the generator's own density so that the expected count k* is
                   log-uniform in [1, 2000].  Seed 2.
  roads-3e7        n = 3 * 10^7 points at jittered spacing h along 200,000 random polylines of
                   10-50 segments with log-normal lengths (median 2^14, sigma_ln 1) and a
                   random-walk heading; m = 2 * 10^6 queries at data points; fixed radius
                   25 h (about 50 points along a road).  Seed 3.
  mixed-1e8        as mixed-1e7 with n = 10^8 and m = 10^7.  Seed 4.
  dynamic-5e7      base n = 5 * 10^7, all clustered; per round 500,000 deletes of live ids,
                   1,000,000 inserts from the same mixture, 1,000,000 queries at live points
                   with log-uniform k*.  Seed 5.

Every workload takes a ``scale`` that shrinks n and m (and the cluster count) so the same
shapes can be run at sizes the oracle finishes in seconds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SIDE = 1 << 30
DOMAIN_MAX = SIDE - 1


@dataclass
class Workload:
    name: str
    points: np.ndarray          # int32 [n, 2]
    queries: np.ndarray         # int32 [m, 2]
    delta: np.ndarray           # int32 [m]
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.points.shape[0])

    @property
    def m(self):
        return int(self.queries.shape[0])


def _streams(seed: int, k: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(k)]


def _clamp_round(a: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(a), 0, DOMAIN_MAX).astype(np.int32)


# --------------------------------------------------------------------------------------
# Point sets
# --------------------------------------------------------------------------------------

def uniform_points(rng, n: int, side: int = SIDE) -> np.ndarray:
    return rng.integers(0, side, size=(n, 2), dtype=np.int64).astype(np.int32)


@dataclass
class Mixture:
    """Half uniform background, half isotropic Gaussian clusters (configs mixed-* / dynamic)."""
    centres: np.ndarray        # float64 [C, 2]
    sigma: float
    n_uniform: int
    n_cluster: int

    def density(self, xy: np.ndarray, cluster_of: np.ndarray) -> np.ndarray:
        """Generator density (points per unit^2) at xy: background plus the own cluster's
        Gaussian (other clusters are at least ~2^25 away on average and contribute ~0);
        background-drawn points (cluster_of < 0) get the background only."""
        rho = np.full(xy.shape[0], self.n_uniform / float(SIDE) ** 2)
        sel = cluster_of >= 0
        if self.n_cluster and sel.any():
            c = self.centres[cluster_of[sel]]
            r2 = ((xy[sel].astype(np.float64) - c) ** 2).sum(axis=1)
            per = self.n_cluster / self.centres.shape[0]
            rho[sel] += per / (2 * math.pi * self.sigma ** 2) * np.exp(-r2 / (2 * self.sigma ** 2))
        return rho


def mixture_points(rng, n: int, frac_uniform: float, n_clusters: int, sigma: float,
                   centres: np.ndarray | None = None):
    n_u = int(round(n * frac_uniform))
    n_c = n - n_u
    if centres is None:
        centres = rng.uniform(0, SIDE, size=(n_clusters, 2))
    pts = np.empty((n, 2), np.int32)
    cluster_of = np.full(n, -1, np.int32)
    pts[:n_u] = uniform_points(rng, n_u)
    if n_c:
        which = rng.integers(0, centres.shape[0], size=n_c)
        off = rng.normal(0.0, sigma, size=(n_c, 2))
        pts[n_u:] = _clamp_round(centres[which] + off)
        cluster_of[n_u:] = which
    # shuffle so that ids do not encode the source
    perm = rng.permutation(n)
    return pts[perm], cluster_of[perm], Mixture(centres, sigma, n_u, n_c)


def road_points(rng, n: int, n_lines: int, seg_min=10, seg_max=50, median_len=2.0 ** 14,
                sigma_ln=1.0, turn_sigma=0.35):
    """Points at jittered spacing h along random polylines (roads-3e7).

    Each polyline starts uniformly in the domain, has U{seg_min..seg_max} segments with
    log-normal lengths, and a heading that performs a Gaussian random walk.  The n points are
    spread over the total arc length L at spacing h = L / n, each moved along the track by
    U(-h/4, h/4) and across it by U{-1, 0, 1}, then rounded and clamped."""
    nseg = rng.integers(seg_min, seg_max + 1, size=n_lines)
    total = int(nseg.sum())
    lengths = np.exp(rng.normal(math.log(median_len), sigma_ln, size=total))
    turns = rng.normal(0.0, turn_sigma, size=total)
    line_of_seg = np.repeat(np.arange(n_lines), nseg)
    first_seg = np.concatenate([[0], np.cumsum(nseg)[:-1]])
    h0 = rng.uniform(0, 2 * math.pi, size=n_lines)
    # heading: initial heading of the line plus the cumulative turns within the line
    cum_turn = np.cumsum(turns)
    cum_turn -= np.repeat(cum_turn[first_seg] - turns[first_seg], nseg)
    heading = h0[line_of_seg] + cum_turn
    dx = lengths * np.cos(heading)
    dy = lengths * np.sin(heading)
    starts = rng.uniform(0, SIDE, size=(n_lines, 2))
    # segment start points: line start plus cumulative displacement of earlier segments
    cx = np.cumsum(dx)
    cy = np.cumsum(dy)
    cx_prev = cx - dx
    cy_prev = cy - dy
    base_x = np.repeat(cx_prev[first_seg], nseg)
    base_y = np.repeat(cy_prev[first_seg], nseg)
    sx = starts[line_of_seg, 0] + (cx_prev - base_x)
    sy = starts[line_of_seg, 1] + (cy_prev - base_y)
    arc = np.concatenate([[0.0], np.cumsum(lengths)])
    L = float(arc[-1])
    h = L / n
    t = (np.arange(n, dtype=np.float64) + 0.5) * h + rng.uniform(-h / 4, h / 4, size=n)
    t = np.clip(t, 0.0, np.nextafter(L, 0.0))
    seg = np.searchsorted(arc, t, side="right") - 1
    seg = np.clip(seg, 0, total - 1)
    frac = t - arc[seg]
    ux, uy = np.cos(heading[seg]), np.sin(heading[seg])
    across = rng.integers(-1, 2, size=n).astype(np.float64)
    px = sx[seg] + frac * ux - across * uy
    py = sy[seg] + frac * uy + across * ux
    pts = np.stack([px, py], axis=1)
    return _clamp_round(pts), h


# --------------------------------------------------------------------------------------
# Queries and radii
# --------------------------------------------------------------------------------------

def density_matched_delta(rng, rho: np.ndarray, k_min=1.0, k_max=2000.0) -> np.ndarray:
    """Radius per query so that the expected count pi delta^2 rho equals a target k* drawn
    log-uniformly in [k_min, k_max]."""
    kstar = np.exp(rng.uniform(math.log(k_min), math.log(k_max), size=rho.shape[0]))
    d = np.sqrt(kstar / (math.pi * rho))
    return np.clip(np.rint(d), 1, 2 ** 31 - 1).astype(np.int32)


def normal_points(rng, n: int) -> np.ndarray:
    """The paper's Normal distribution (Sec. 3, "Data"): centre at half the domain side,
    standard deviation one eighth of it; rounded and clamped."""
    return _clamp_round(rng.normal(SIDE / 2, SIDE / 8, size=(n, 2)))


def skewed_points(rng, n: int) -> np.ndarray:
    """The paper's Skewed distribution (Sec. 3, "Data"): x uniform over the side, y geometric
    with success probability 5 / side (mean side / 5), clamped to the domain."""
    x = rng.integers(0, SIDE, size=n, dtype=np.int64)
    y = np.minimum(rng.geometric(5.0 / SIDE, size=n) - 1, SIDE - 1)
    return np.stack([x, y], axis=1).astype(np.int32)


def paper_points(rng, dist: str, n: int) -> np.ndarray:
    if dist == "uniform":
        return uniform_points(rng, n)
    if dist == "normal":
        return normal_points(rng, n)
    if dist == "skewed":
        return skewed_points(rng, n)
    raise ValueError(dist)


def queries_at_points(rng, pts: np.ndarray, m: int):
    idx = rng.integers(0, pts.shape[0], size=m)
    return pts[idx].copy(), idx


# --------------------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------------------

def uniform_1e5(scale: float = 1.0, seed: int = 1) -> Workload:
    n = max(1, int(round(100_000 * scale)))
    m = max(1, int(round(10_000 * scale)))
    rp, rq = _streams(seed, 2)
    side = 1 << 20
    pts = uniform_points(rp, n, side)
    qs = uniform_points(rq, m, side)
    delta = int(round(math.sqrt(20.0 * float(side) ** 2 / (math.pi * n))))
    return Workload("uniform-1e5", pts, qs, np.full(m, delta, np.int32),
                    {"seed": seed, "side": side, "delta": delta, "expected_k": 20.0})


def mixed(n_full: int, m_full: int, seed: int, name: str, scale: float = 1.0,
          n_clusters_full: int = 1000) -> Workload:
    n = max(2, int(round(n_full * scale)))
    m = max(1, int(round(m_full * scale)))
    C = max(1, int(round(n_clusters_full * min(1.0, scale ** 0.5))))
    rp, rq, rd = _streams(seed, 3)
    pts, cl, mix = mixture_points(rp, n, 0.5, C, 2.0 ** 18)
    qs, qi = queries_at_points(rq, pts, m)
    rho = mix.density(qs, cl[qi])
    delta = density_matched_delta(rd, rho)
    return Workload(name, pts, qs, delta,
                    {"seed": seed, "clusters": C, "sigma": 2 ** 18, "k_range": [1, 2000]})


def mixed_1e7(scale: float = 1.0, seed: int = 2) -> Workload:
    return mixed(10_000_000, 1_000_000, seed, "mixed-1e7", scale)


def mixed_1e8(scale: float = 1.0, seed: int = 4) -> Workload:
    return mixed(100_000_000, 10_000_000, seed, "mixed-1e8", scale)


def roads_3e7(scale: float = 1.0, seed: int = 3) -> Workload:
    n = max(2, int(round(30_000_000 * scale)))
    m = max(1, int(round(2_000_000 * scale)))
    lines = max(1, int(round(200_000 * scale)))
    rp, rq = _streams(seed, 2)
    pts, h = road_points(rp, n, lines)
    qs, _ = queries_at_points(rq, pts, m)
    delta = max(1, int(round(25.0 * h)))
    return Workload("roads-3e7", pts, qs, np.full(m, delta, np.int32),
                    {"seed": seed, "lines": lines, "spacing_h": h, "delta": delta,
                     "expected_k": 50})


@dataclass
class DynamicWorkload:
    name: str
    base: np.ndarray
    rounds: list            # list of dicts: inserts int32[k,2], delete_pos_seed, queries, delta
    meta: dict


def dynamic_5e7(scale: float = 1.0, seed: int = 5, rounds: int = 20) -> DynamicWorkload:
    """Base set and per-round update batches.  Deletes are given as ranks r in [0, live)
    into the ascending list of live ids at that round (ids themselves depend on the ids the
    structure hands out, which follow the fixed policy first_new_id = next_id)."""
    n = max(4, int(round(50_000_000 * scale)))
    k_ins = max(1, int(round(1_000_000 * scale)))
    k_del = max(1, int(round(500_000 * scale)))
    m = max(1, int(round(1_000_000 * scale)))
    C = max(1, int(round(1000 * min(1.0, scale ** 0.5))))
    rs = _streams(seed, 1 + 4 * rounds)
    base, cl, mix = mixture_points(rs[0], n, 0.0, C, 2.0 ** 18)
    rnds = []
    live = n
    for r in range(rounds):
        ri, rdl, rq, rd = rs[1 + 4 * r: 5 + 4 * r]
        ins, icl, _ = mixture_points(ri, k_ins, 0.0, C, 2.0 ** 18, centres=mix.centres)
        kd = min(k_del, live)
        del_rank = rdl.choice(live, size=kd, replace=False).astype(np.int64)
        live = live - kd + k_ins
        rnds.append({"inserts": ins, "insert_cluster": icl, "delete_rank": del_rank,
                     "query_rng": rq, "delta_rng": rd, "m": m})
    return DynamicWorkload("dynamic-5e7", base, rnds,
                           {"seed": seed, "clusters": C, "mixture": mix, "base_cluster": cl})


def dynamic_round_queries(wl: DynamicWorkload, r: int, live_xy: np.ndarray,
                          live_cluster: np.ndarray):
    """Queries of round r at live points with density-matched radii (drawn after the
    round's updates are applied, from the round's own streams)."""
    rd = wl.rounds[r]
    qs, qi = queries_at_points(rd["query_rng"], live_xy, rd["m"])
    rho = wl.meta["mixture"].density(qs, live_cluster[qi])
    return qs, density_matched_delta(rd["delta_rng"], rho)


def normal_uniform_queries(n: int, m: int, rel_side: float, seed: int = 6) -> Workload:
    """The paper's static synthetic setting (Sec. 3.1): Normal points, uniform query centres,
    and a disc whose diameter is rel_side times the domain side."""
    rp, rq = _streams(seed, 2)
    pts = normal_points(rp, n)
    qs = uniform_points(rq, m)
    delta = max(0, int(round(rel_side * SIDE / 2)))
    return Workload("normal-uniform", pts, qs, np.full(m, delta, np.int32),
                    {"seed": seed, "rel_side": rel_side, "delta": delta})


def paper_static(dist: str, n: int, m: int, rel_side: float, qdist: str = "uniform", seed: int = 7,
                 scale: float = 1.0) -> Workload:
    """The paper's static experiments (Sec. 3.1): points from its Uniform / Normal / Skewed
    distributions, query centres from one of them, and square windows whose side is rel_side
    times the domain side: the closed square of half-side delta = round(rel_side * side / 2)
    (side 2 delta + 1 grid points), queried with norm "square"."""
    n = max(2, int(round(n * scale)))
    m = max(1, int(round(m * scale)))
    rp, rq = _streams(seed, 2)
    pts = paper_points(rp, dist, n)
    qs = paper_points(rq, qdist, m)
    delta = int(round(rel_side * SIDE / 2))
    return Workload(f"paper-{dist}", pts, qs, np.full(m, delta, np.int32),
                    {"seed": seed, "dist": dist, "qdist": qdist, "rel_side": rel_side, "delta": delta,
                     "norm": "square"})


SIDE3 = 1 << 21   # 3-D domain side (63-bit keys)


def mixed3d(n: int = 10_000_000, m: int = 1_000_000, seed: int = 8, scale: float = 1.0,
            n_clusters: int = 1000, sigma: float = 2.0 ** 11) -> Workload:
    """3-D counterpart of the mixed workloads (the paper's d-dimensional remark, Sec. 2.1):
    half the points uniform in [0, 2^21)^3, half from 1,000 isotropic Gaussian clusters with
    sigma 2^11 (2^-10 of the side), queries at data points, and per-query radii from the
    generator's density so that the expected count (4/3) pi delta^3 rho is log-uniform in
    [1, 2000]."""
    n = max(2, int(round(n * scale)))
    m = max(1, int(round(m * scale)))
    C = max(1, int(round(n_clusters * min(1.0, scale ** 0.5))))
    rp, rq, rd = _streams(seed, 3)
    n_u = n // 2
    n_c = n - n_u
    centres = rp.uniform(0, SIDE3, size=(C, 3))
    pts = np.empty((n, 3), np.int64)
    cl = np.full(n, -1, np.int64)
    pts[:n_u] = rp.integers(0, SIDE3, size=(n_u, 3))
    which = rp.integers(0, C, size=n_c)
    pts[n_u:] = np.clip(np.rint(centres[which] + rp.normal(0.0, sigma, size=(n_c, 3))), 0, SIDE3 - 1)
    cl[n_u:] = which
    perm = rp.permutation(n)
    pts, cl = pts[perm].astype(np.int32), cl[perm]
    qi = rq.integers(0, n, size=m)
    qs = pts[qi].copy()
    rho = np.full(m, n_u / float(SIDE3) ** 3)
    sel = cl[qi] >= 0
    r2 = ((qs[sel].astype(np.float64) - centres[cl[qi][sel]]) ** 2).sum(axis=1)
    rho[sel] += (n_c / C) / ((2 * math.pi) ** 1.5 * sigma ** 3) * np.exp(-r2 / (2 * sigma ** 2))
    kstar = np.exp(rd.uniform(math.log(1.0), math.log(2000.0), size=m))
    delta = np.clip(np.rint(np.cbrt(kstar / (4.0 / 3.0 * math.pi * rho))), 1, SIDE3 - 1).astype(np.int32)
    return Workload("mixed3d-1e7", pts, qs, delta, {"seed": seed, "clusters": C, "sigma": sigma,
                                                    "k_range": [1, 2000], "dim": 3})


WORKLOADS = {
    "uniform-1e5": uniform_1e5,
    "mixed-1e7": mixed_1e7,
    "roads-3e7": roads_3e7,
    "mixed-1e8": mixed_1e8,
}


# --------------------------------------------------------------------------------------
# Small adversarial shapes for tests
# --------------------------------------------------------------------------------------

def tiny_dense(seed: int, n: int, m: int, side_bits: int, max_delta: int):
    """Points on a small grid (many duplicates), queries anywhere in the grid, radii in
    [0, max_delta]: exercises duplicates, ties and boundary cells."""
    rp, rq, rd = _streams(seed, 3)
    side = 1 << side_bits
    pts = uniform_points(rp, n, side)
    qs = uniform_points(rq, m, side)
    d = rd.integers(0, max_delta + 1, size=m).astype(np.int32)
    return pts, qs, d


def pythagorean_ring(cx: int, cy: int, scale: int):
    """Points at exactly distance 5*scale from (cx, cy) along (3,4)-type offsets, plus points
    one unit further out: a query of radius 5*scale must report exactly the first group."""
    offs = [(3, 4), (4, 3), (-3, 4), (-4, 3), (3, -4), (4, -3), (-3, -4), (-4, -3), (5, 0),
            (0, 5), (-5, 0), (0, -5)]
    on = [(cx + a * scale, cy + b * scale) for a, b in offs]
    out = [(cx + a * scale + (1 if a > 0 else -1 if a < 0 else 0),
            cy + b * scale + (1 if b > 0 else -1 if b < 0 else 0)) for a, b in offs]
    return np.array(on, np.int32), np.array(out, np.int32)
