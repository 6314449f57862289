"""Seeded synthetic inputs for the ensemble flood model.

This module only *generates inputs*: terrain, roughness, rainfall series,
ensemble priors, gauge locations, noisy observations and the random draws the
particle filter consumes.  It holds none of the scheme's arithmetic (no flux,
continuity, time step, likelihood or resampling), so both the CUDA path and
the FP64 oracle can consume the same arrays without sharing any method code.

The paper's Fuzhou DEM and land-use rasters (Section 4.1, Fig. 6) are not
available; the generator stands in for them with terrain of the same kind:
3 m cells, a gentle planar slope, smooth hills, 10 m building blocks and a
road network with lower roughness.  Every value is FP32 (the precision the GPU
path stores), so the oracle sees exactly the numbers the GPU sees.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MM_PER_H = 1.0 / 3.6e6  # one mm/h expressed in m/s


@dataclasses.dataclass
class Terrain:
    z: np.ndarray          # [ny, nx] float32, bed elevation (m), min(z) == 0
    n: np.ndarray          # [ny, nx] float32, Manning n per cell (s m^-1/3)
    building: np.ndarray   # [ny, nx] bool, building footprint mask
    road: np.ndarray       # [ny, nx] bool, road mask
    dx: float              # cell size (m)
    slope: float           # planar slope (descends toward column nx-1)


def make_terrain(ny: int, nx: int, seed: int, dx: float = 3.0, slope: float = 0.005,
                 n_bumps: int = 40, bump_amp=(0.0, 1.0), bump_sigma_m=(10.0, 40.0),
                 building_frac: float = 0.05, building_side=(4, 12),
                 building_height: float = 10.0, road_spacing=(20, 60),
                 road_width=(2, 3), n_road: float = 0.03, n_other: float = 0.05) -> Terrain:
    """Synthetic urban DEM: planar slope + Gaussian hills + buildings + roads.

    * planar slope of ``slope`` descending toward column ``nx-1`` (the lowest
      edge, where the free-outflow boundary sits);
    * ``n_bumps`` Gaussian hills, centre uniform over the domain, amplitude
      U[bump_amp], standard deviation U[bump_sigma_m] metres;
    * a road grid: rows and columns at random spacing U{road_spacing} cells,
      each U{road_width} cells wide, Manning n = ``n_road`` (``n_other``
      elsewhere);
    * axis-aligned building blocks with sides U{building_side} cells, raised
      ``building_height`` metres, placed off the roads until they cover at
      least ``building_frac`` of the area;
    * elevations referenced to min(z) = 0.
    """
    rng = np.random.default_rng(seed)
    cc = np.arange(nx, dtype=np.float64)
    z = np.broadcast_to(slope * dx * (nx - 1 - cc)[None, :], (ny, nx)).copy()

    ys = (np.arange(ny) + 0.5) * dx
    xs = (np.arange(nx) + 0.5) * dx
    for _ in range(n_bumps):
        cy = rng.uniform(0.0, ny * dx)
        cx = rng.uniform(0.0, nx * dx)
        amp = rng.uniform(*bump_amp)
        sig = rng.uniform(*bump_sigma_m)
        # evaluate only inside a +-6 sigma window (exp(-18) ~ 1.5e-8 outside)
        r0 = max(0, int((cy - 6 * sig) / dx)); r1 = min(ny, int((cy + 6 * sig) / dx) + 1)
        c0 = max(0, int((cx - 6 * sig) / dx)); c1 = min(nx, int((cx + 6 * sig) / dx) + 1)
        if r0 >= r1 or c0 >= c1:
            continue
        dy2 = (ys[r0:r1, None] - cy) ** 2
        dx2 = (xs[None, c0:c1] - cx) ** 2
        z[r0:r1, c0:c1] += amp * np.exp(-(dy2 + dx2) / (2.0 * sig * sig))

    road = np.zeros((ny, nx), dtype=bool)
    for axis, size in ((0, ny), (1, nx)):
        pos = int(rng.integers(road_spacing[0], road_spacing[1] + 1)) // 2
        while pos < size:
            w = int(rng.integers(road_width[0], road_width[1] + 1))
            if axis == 0:
                road[pos:pos + w, :] = True
            else:
                road[:, pos:pos + w] = True
            pos += w + int(rng.integers(road_spacing[0], road_spacing[1] + 1))

    building = np.zeros((ny, nx), dtype=bool)
    target = building_frac * ny * nx
    covered = 0
    tries = 0
    lo, hi = building_side
    while covered < target and tries < 200000 and ny >= lo and nx >= lo:
        tries += 1
        bh = int(rng.integers(lo, hi + 1)); bw = int(rng.integers(lo, hi + 1))
        bh = min(bh, ny); bw = min(bw, nx)
        r0 = int(rng.integers(0, ny - bh + 1)); c0 = int(rng.integers(0, nx - bw + 1))
        blk = (slice(r0, r0 + bh), slice(c0, c0 + bw))
        if road[blk].any():
            continue
        covered += int((~building[blk]).sum())
        building[blk] = True
    z[building] += building_height
    z -= z.min()

    n = np.where(road, n_road, n_other)
    return Terrain(z=z.astype(np.float32), n=n.astype(np.float32), building=building,
                   road=road, dx=float(dx), slope=float(slope))


def hyetograph_constant(rate_mm_h: float, duration_s: float, block_s: float = 300.0) -> np.ndarray:
    """Piecewise-constant rain blocks (m/s) for a uniform storm of given length."""
    n_blocks = int(math.ceil(duration_s / block_s))
    out = np.zeros(n_blocks, dtype=np.float64)
    for k in range(n_blocks):
        t0, t1 = k * block_s, min((k + 1) * block_s, duration_s)
        out[k] = rate_mm_h * MM_PER_H * (t1 - t0) / block_s
    return out.astype(np.float32)


def hyetograph_triangular(peak_mm_h: float = 60.0, t_peak_s: float = 1200.0,
                          duration_s: float = 3600.0, block_s: float = 300.0) -> np.ndarray:
    """Block means (m/s) of a triangular storm: 0 at t=0, peak at ``t_peak_s``,
    0 again at ``duration_s``.  Each block holds the exact mean of the
    triangle over the block (integrated piecewise-linearly)."""

    def rate(t):
        if t <= t_peak_s:
            return peak_mm_h * t / t_peak_s
        return peak_mm_h * max(0.0, duration_s - t) / (duration_s - t_peak_s)

    n_blocks = int(math.ceil(duration_s / block_s))
    out = np.zeros(n_blocks, dtype=np.float64)
    for k in range(n_blocks):
        t0, t1 = k * block_s, (k + 1) * block_s
        knots = sorted({t0, t1, *(x for x in (t_peak_s, duration_s) if t0 < x < t1)})
        area = sum(0.5 * (rate(a) + rate(b)) * (b - a) for a, b in zip(knots[:-1], knots[1:]))
        out[k] = area / block_s * MM_PER_H
    return out.astype(np.float32)


def ensemble_prior(seed: int, n_members: int, rain_sigma: float = 0.3,
                   manning_range=(0.6, 1.4)):
    """Monte Carlo draws of the uncertain inputs (the prior of Eq. 7):
    per-member rainfall multiplier ~ lognormal(0, rain_sigma) and per-member
    Manning scale ~ U[manning_range]."""
    rng = np.random.default_rng([seed, 0x5EED])
    rain_mult = rng.lognormal(0.0, rain_sigma, n_members)
    scale = rng.uniform(manning_range[0], manning_range[1], n_members)
    return rain_mult.astype(np.float32), scale.astype(np.float32)


def gauge_cells(terrain: Terrain, n_gauges: int, seed: int) -> np.ndarray:
    """Depth gauges at ponding spots: open cells whose down-slope (+column)
    neighbour is a building, one per stratum of a near-square grid of strata.
    Returns flat row-major cell indices (int32)."""
    b = terrain.building
    ny, nx = b.shape
    cand = np.zeros_like(b)
    cand[:, :-1] = (~b[:, :-1]) & b[:, 1:]
    rng = np.random.default_rng([seed, 0x6A06E])
    rows = int(math.floor(math.sqrt(n_gauges)))
    while n_gauges % rows:
        rows -= 1
    cols = n_gauges // rows
    out = []
    for i in range(rows):
        for j in range(cols):
            r0, r1 = i * ny // rows, (i + 1) * ny // rows
            c0, c1 = j * nx // cols, (j + 1) * nx // cols
            rr, cc = np.nonzero(cand[r0:r1, c0:c1])
            if len(rr) == 0:
                rr, cc = np.nonzero(~b[r0:r1, c0:c1])
            k = int(rng.integers(0, len(rr)))
            out.append((r0 + rr[k]) * nx + (c0 + cc[k]))
    return np.asarray(out, dtype=np.int32)


def observe(truth_depth: np.ndarray, seed: int, window: int, sigma_m: float = 0.05) -> np.ndarray:
    """Synthetic observation d = truth depth at the gauges + N(0, sigma^2)."""
    rng = np.random.default_rng([seed, 0x0B5, window])
    return (np.asarray(truth_depth, np.float64) + rng.normal(0.0, sigma_m, np.shape(truth_depth)))


def pf_draws(seed: int, window: int, n_members: int, beta_sigma: float = 0.05):
    """Random numbers one particle-filter update consumes: the systematic
    resampling offset u ~ U[0, 1) and the post-resampling rain perturbation
    beta ~ N(1, beta_sigma^2) per member (Section 4.4)."""
    rng = np.random.default_rng([seed, 0xF1, window])
    u = float(rng.random())
    beta = rng.normal(1.0, beta_sigma, n_members).astype(np.float32)
    return u, beta


@dataclasses.dataclass
class Scenario:
    """One member of an uneven batch: its own grid, DEM seed, rain and duration."""
    ny: int
    nx: int
    seed: int
    rain_mm_h: float
    duration_s: float


def uneven_batch(n: int = 64, side=(512, 2048), rain=(20.0, 100.0),
                 duration=(900.0, 3600.0), seed0: int = 100, master_seed: int = 2):
    """Scenarios of uneven size and length: square sides U{side}, DEM seeds
    seed0+k, rain U[rain] mm/h, duration U[duration] s."""
    rng = np.random.default_rng([master_seed, 0xBA7C4])
    out = []
    for k in range(n):
        s = int(rng.integers(side[0], side[1] + 1))
        out.append(Scenario(ny=s, nx=s, seed=seed0 + k,
                            rain_mm_h=float(rng.uniform(*rain)),
                            duration_s=float(rng.uniform(*duration))))
    return out


# ---- land cover (Section 4.1, Table 1) -------------------------------------
# classes: 0 green land, 1 water bodies, 2 hardened ground, 3 outside the domain
LAND_CLASSES = [
    # (Manning n of the deterministic model (Table 1), runoff coefficient,
    #  drainage applies, outside the domain)
    (0.15, 0.9, 0, 0),    # green land: 10 % of the rain infiltrates
    (0.020, 1.0, 0, 0),   # water bodies: no infiltration
    (0.017, 1.0, 1, 0),   # hardened ground: the pipe network drains I_drn
    (0.05, 0.0, 0, 1),    # outside the domain
]
N_RANGES = [(0.08, 0.22), (0.016, 0.030), (0.010, 0.022), (0.05, 0.05)]  # Table 1 ensemble
I_DRN_MM_H = 12.0


def irregular_domain(ny: int, nx: int, active_frac: float, seed: int) -> np.ndarray:
    """An irregular domain inside its bounding box (True = active), shaped
    like the paper's study area (Section 4.1: 4,002,457 active cells of 3 m
    in an 8.2 x 7.6 km box, 58 % of it): a blob whose radius varies smoothly
    with the angle (random harmonics 2-7), centred a little east of the box
    centre so that it reaches the eastern (outflow) edge, scaled so that
    ``active_frac`` of the box is active."""
    rng = np.random.default_rng([seed, 0xD0A1])
    k = np.arange(2, 8)
    amp = rng.uniform(0.03, 0.12, len(k)) / k ** 0.5
    phase = rng.uniform(0.0, 2.0 * np.pi, len(k))
    rr, cc = np.mgrid[0:ny, 0:nx]
    y = (rr - 0.5 * ny) / (0.5 * ny)
    x = (cc - 0.62 * nx) / (0.5 * nx)
    theta = np.arctan2(y, x)
    shape = 1.0 + np.sum(amp[:, None, None] * np.cos(k[:, None, None] * theta + phase[:, None, None]),
                         axis=0)
    rad = np.hypot(x, y) / shape
    lo, hi = 0.0, 3.0
    for _ in range(60):                       # bisection on the blob's scale
        mid = 0.5 * (lo + hi)
        if (rad < mid).mean() < active_frac:
            lo = mid
        else:
            hi = mid
    return rad < hi


def land_cover(terrain: Terrain, seed: int, n_ponds: int = 6, pond_side=(8, 30),
               corner_frac: float = 0.25, domain: np.ndarray | None = None) -> np.ndarray:
    """Class per cell (uint8): roads and buildings are hardened ground, a few
    rectangular ponds are water bodies, the rest green land; two quarter
    discs of radius ``corner_frac`` x min(ny, nx) at the western (upstream)
    corners lie outside the domain, so the domain is irregular and its
    outflow edge stays open -- or, given ``domain`` (True = active, e.g.
    ``irregular_domain``), every cell outside it."""
    rng = np.random.default_rng(seed)
    ny, nx = terrain.z.shape
    cls = np.zeros((ny, nx), np.uint8)
    cls[terrain.road | terrain.building] = 2
    for _ in range(n_ponds):
        h = int(rng.integers(pond_side[0], pond_side[1] + 1)); w = int(rng.integers(pond_side[0], pond_side[1] + 1))
        h = min(h, ny); w = min(w, nx)
        r0 = int(rng.integers(0, ny - h + 1)); c0 = int(rng.integers(0, nx - w + 1))
        blk = cls[r0:r0 + h, c0:c0 + w]
        blk[blk == 0] = 1
    if domain is not None:
        out = ~np.asarray(domain, bool)
    else:
        rad = corner_frac * min(ny, nx)
        rr, cc = np.mgrid[0:ny, 0:nx]
        out = ((rr ** 2 + cc ** 2) < rad ** 2) | (((ny - 1 - rr) ** 2 + cc ** 2) < rad ** 2)
    cls[out] = 3
    return cls


def land_prior(seed: int, n_members: int, drain_spread: float = 0.5):
    """Per-member land-cover parameters: Manning n of every class uniform
    over Table 1's ensemble range, and the drainage rate I_drn = 12 mm/h
    times U[1 - spread, 1 + spread] (m/s).  Returns ([M, 4], [M]) float32."""
    rng = np.random.default_rng(seed + 777)
    n = np.stack([rng.uniform(lo, hi, n_members) for lo, hi in N_RANGES], axis=1)
    d = I_DRN_MM_H * MM_PER_H * rng.uniform(1.0 - drain_spread, 1.0 + drain_spread, n_members)
    return n.astype(np.float32), d.astype(np.float32)
