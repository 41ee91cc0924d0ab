"""Seeded synthetic cartogram inputs: maps of polygonal regions with target values.

The paper's maps (US states, Indian states, Chinese provinces, London LSOAs) and
their data are not available, so the workloads here are seeded stand-ins with the
same structure: a few hundred to a few thousand contiguous regions that share
their boundaries, embedded in a rectangular box with an empty margin around them
(the paper embeds the map in a box 1.5x the map's extent, filled with the mean
density; see the section "Benchmarking the algorithm with data for the USA, India,
and China").

This module holds geometry and random numbers only, none of the method's
arithmetic; both the CUDA path and the CPU oracle consume what it produces.

Output layout (the one the C-ABI takes):
    values        float64[R]           target value of each region (> 0)
    ring_offsets  int64[n_rings + 1]   ring k owns vertices ring_offsets[k]:ring_offsets[k+1]
    ring_region   int32[n_rings]       region of each ring
    xy            float64[n_vert, 2]   vertices in grid units, box [0, Lx] x [0, Ly];
                                       rings are implicitly closed (last -> first),
                                       counter-clockwise for outer boundaries.
Shared boundaries between neighbouring regions are subdivided once, so both
neighbours carry bit-identical vertices along their common edge.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _MASK64


class Xoshiro256ss:
    """xoshiro256** generator (Blackman & Vigna, 2018) seeded through SplitMix64.

    Pure integer arithmetic, so the stream is identical on every host.
    """

    def __init__(self, seed: int):
        s = seed & _MASK64
        self.s = []
        for _ in range(4):
            s = (s + 0x9E3779B97F4A7C15) & _MASK64
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
            self.s.append(z ^ (z >> 31))

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & _MASK64, 7) * 9) & _MASK64
        t = (s[1] << 17) & _MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_open(self) -> float:
        """Uniform double in (0, 1)."""
        return ((self.next_u64() >> 11) + 0.5) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal deviate by the Box-Muller transform (one per call)."""
        u1 = self.uniform_open()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def lognormal(self, mu: float, sigma: float) -> float:
        return math.exp(mu + sigma * self.normal())

    def pareto(self, alpha: float, xm: float) -> float:
        """Pareto(alpha, x_m) by inversion: x_m * U^(-1/alpha), U in (0, 1)."""
        return xm * self.uniform_open() ** (-1.0 / alpha)


@dataclass
class RegionMap:
    Lx: int
    Ly: int
    values: np.ndarray
    ring_offsets: np.ndarray
    ring_region: np.ndarray
    xy: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_regions(self) -> int:
        return int(self.values.shape[0])

    @property
    def n_rings(self) -> int:
        return int(self.ring_region.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.xy.shape[0])


# ----------------------------------------------------------------------------
# seed point distributions
# ----------------------------------------------------------------------------

def seeds_uniform(rng: Xoshiro256ss, n: int, lo: float, hi: float) -> np.ndarray:
    return np.array([[lo + (hi - lo) * rng.uniform(), lo + (hi - lo) * rng.uniform()]
                     for _ in range(n)], dtype=np.float64)


def seeds_clustered(rng: Xoshiro256ss, n: int, lo: float, hi: float,
                    n_clusters: int, sigma: float) -> np.ndarray:
    """Gaussian clusters with uniformly placed centres; points outside [lo, hi]^2 are redrawn."""
    centres = [(lo + (hi - lo) * rng.uniform(), lo + (hi - lo) * rng.uniform())
               for _ in range(n_clusters)]
    pts = []
    while len(pts) < n:
        cx, cy = centres[len(pts) % n_clusters]
        x = cx + sigma * rng.normal()
        y = cy + sigma * rng.normal()
        if lo < x < hi and lo < y < hi:
            pts.append((x, y))
    return np.array(pts, dtype=np.float64)


def seeds_power_law(rng: Xoshiro256ss, n: int, cx: float, cy: float, radius: float) -> np.ndarray:
    """Radial power law: area density proportional to 1/r about (cx, cy), i.e. r = R*u."""
    pts = []
    for _ in range(n):
        r = radius * rng.uniform_open()
        a = 2.0 * math.pi * rng.uniform()
        pts.append((cx + r * math.cos(a), cy + r * math.sin(a)))
    return np.array(pts, dtype=np.float64)


# ----------------------------------------------------------------------------
# bounded Voronoi tessellation with canonical edge subdivision
# ----------------------------------------------------------------------------

def _signed_area(poly: np.ndarray) -> float:
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * float(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))


def voronoi_rings(seeds: np.ndarray, lo: float, hi: float, spacing: float):
    """Voronoi cells of `seeds` clipped to the square [lo, hi]^2, one ring per cell.

    Clipping uses mirror images of the seeds across the four sides, which makes the
    sides themselves cell boundaries. Every unique edge is split into
    ceil(length / spacing) equal pieces once, so neighbours share vertices exactly.
    Returns (ring_offsets, xy).
    """
    from scipy.spatial import Voronoi

    n = seeds.shape[0]
    mirrored = [seeds]
    for axis in (0, 1):
        for wall in (lo, hi):
            m = seeds.copy()
            m[:, axis] = 2.0 * wall - m[:, axis]
            mirrored.append(m)
    vor = Voronoi(np.concatenate(mirrored, axis=0))
    verts = vor.vertices.copy()
    # snap vertices that lie on the square's sides (they are exact in real arithmetic)
    tol = 1e-9 * max(1.0, hi - lo)
    for c in (0, 1):
        for wall in (lo, hi):
            sel = np.abs(verts[:, c] - wall) < tol
            verts[sel, c] = wall

    cells = []
    for s in range(n):
        reg = vor.regions[vor.point_region[s]]
        if len(reg) == 0 or -1 in reg:
            raise RuntimeError("unbounded Voronoi cell for an interior seed")
        ids = list(reg)
        if _signed_area(verts[ids]) < 0.0:
            ids = ids[::-1]
        cells.append(ids)

    # subdivide every unique edge once, from its lower to its higher vertex id
    interior = {}
    for ids in cells:
        k = len(ids)
        for a_i in range(k):
            a, b = ids[a_i], ids[(a_i + 1) % k]
            key = (a, b) if a < b else (b, a)
            if key in interior:
                continue
            p, q = verts[key[0]], verts[key[1]]
            length = float(np.hypot(*(q - p)))
            pieces = max(1, int(math.ceil(length / spacing - 1e-12)))
            f = np.arange(1, pieces, dtype=np.float64)[:, None] / pieces
            interior[key] = p[None, :] + f * (q - p)[None, :]

    offsets = [0]
    out = []
    for ids in cells:
        k = len(ids)
        count = 0
        for a_i in range(k):
            a, b = ids[a_i], ids[(a_i + 1) % k]
            pts = interior[(a, b) if a < b else (b, a)]
            out.append(verts[a][None, :])
            out.append(pts if a < b else pts[::-1])
            count += 1 + pts.shape[0]
        offsets.append(offsets[-1] + count)
    xy = np.ascontiguousarray(np.concatenate(out, axis=0))
    return np.array(offsets, dtype=np.int64), xy


def voronoi_map(Lx: int, Ly: int, seeds: np.ndarray, inset: float, spacing: float,
                values: np.ndarray, meta=None) -> RegionMap:
    assert Lx == Ly, "the square-inset Voronoi maps are generated on square boxes"
    offsets, xy = voronoi_rings(seeds, inset, Lx - inset, spacing)
    n = seeds.shape[0]
    return RegionMap(Lx, Ly, np.asarray(values, dtype=np.float64), offsets,
                     np.arange(n, dtype=np.int32), xy, dict(meta or {}))


def rectangle_ring(x0, y0, x1, y1, spacing):
    """Counter-clockwise rectangle, sides split into pieces no longer than `spacing`."""
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    pts = []
    for k in range(4):
        p = np.array(corners[k], dtype=np.float64)
        q = np.array(corners[(k + 1) % 4], dtype=np.float64)
        pieces = max(1, int(math.ceil(float(np.hypot(*(q - p))) / spacing - 1e-12)))
        for s in range(pieces):
            pts.append(p + (q - p) * (s / pieces))
    return np.array(pts, dtype=np.float64)


def blocks_map(Lx: int = 128, Ly: int = 64, nx: int = 4, ny: int = 2, seed: int = 5,
               spacing: float = 0.5) -> RegionMap:
    """An nx x ny arrangement of rectangular regions filling the inner half of an Lx x Ly box
    (a non-square grid), with seeded lognormal(0, 0.7) values; neighbouring rectangles carry
    bit-identical shared vertices."""
    x0, y0, w, h = Lx / 4.0, Ly / 4.0, Lx / 2.0 / nx, Ly / 2.0 / ny
    rings = [rectangle_ring(x0 + i * w, y0 + j * h, x0 + (i + 1) * w, y0 + (j + 1) * h, spacing)
             for j in range(ny) for i in range(nx)]
    offsets = np.cumsum([0] + [r.shape[0] for r in rings]).astype(np.int64)
    g = Xoshiro256ss(180207625 + seed)
    values = np.array([g.lognormal(0.0, 0.7) for _ in rings])
    return RegionMap(Lx, Ly, values, offsets, np.arange(len(rings), dtype=np.int32),
                     np.concatenate(rings, axis=0), meta={"name": "blocks", "Lx": Lx, "Ly": Ly})


def holes_map(L: int = 64, spacing: float = 0.5) -> RegionMap:
    """Four regions on an L x L grid with multi-ring structure: region 0 is a square with
    a square hole (a clockwise ring), region 2 fills the hole, region 1 is two islands
    (listed apart in the ring order), region 3 is a strip. Rings:
    [0 outer, 1 island, 0 hole, 2, 3, 1 island]."""
    f = L / 64.0

    def sq(x0, y0, x1, y1):
        return rectangle_ring(x0 * f, y0 * f, x1 * f, y1 * f, spacing)

    rings = [sq(8, 8, 40, 40), sq(44, 8, 56, 20), sq(16, 16, 28, 28)[::-1].copy(), sq(16, 16, 28, 28),
             sq(8, 44, 56, 56), sq(44, 26, 56, 40)]
    region = np.array([0, 1, 0, 2, 3, 1], dtype=np.int32)
    offsets = np.cumsum([0] + [r.shape[0] for r in rings]).astype(np.int64)
    return RegionMap(L, L, np.array([1.0, 4.0, 6.0, 2.0]), offsets, region, np.concatenate(rings, axis=0),
                     meta={"name": "holes", "L": L})


def strip_map(Lx: int, Ly: int, cuts, values, spacing: float = 0.5) -> RegionMap:
    """Vertical strips [cuts[k], cuts[k+1]] x [0, Ly] that tile the whole box.

    Their density depends on x alone, so the unique one-dimensional equalising map
    is known in closed form; used to pin the integrator.
    """
    cuts = list(cuts)
    assert cuts[0] == 0 and cuts[-1] == Lx
    rings = [rectangle_ring(cuts[k], 0.0, cuts[k + 1], float(Ly), spacing)
             for k in range(len(cuts) - 1)]
    offsets = np.cumsum([0] + [r.shape[0] for r in rings]).astype(np.int64)
    return RegionMap(Lx, Ly, np.asarray(values, dtype=np.float64), offsets,
                     np.arange(len(rings), dtype=np.int32), np.concatenate(rings, axis=0),
                     {"kind": "strips", "cuts": cuts})


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

SEED_BASE = 180207625

WORKLOADS = {
    # 64 x 64, 16 uniform Voronoi cells in the square inset 8 cells, 0.5-cell edges,
    # lognormal(0, 1) values, blur 1 cell, FP64 path
    "voronoi16_64": dict(L=64, n=16, inset=8.0, spacing=0.5, seeds="uniform",
                         values=("lognormal", 0.0, 1.0), blur=1.0, precision="fp64", seed_offset=1),
    # 512 x 512, 300 cells from 10 Gaussian clusters (sigma = 0.05 L), ~0.5-cell edges,
    # lognormal(0, 1.5) values, blur 2, mixed precision
    "clustered300_512": dict(L=512, n=300, inset=64.0, spacing=0.5, seeds="clustered",
                             values=("lognormal", 0.0, 1.5), blur=2.0, precision="mixed", seed_offset=2),
    # 1024 x 1024, 3000 cells from a 1/r radial seed density, 0.25-cell edges,
    # Pareto(1.2, 1) values, blur 2, mixed precision
    "powerlaw3000_1024": dict(L=1024, n=3000, inset=128.0, spacing=0.25, seeds="powerlaw",
                              values=("pareto", 1.2, 1.0), blur=2.0, precision="mixed", seed_offset=3),
}


def make_workload(name: str, L: int | None = None, n: int | None = None) -> RegionMap:
    """Build a named workload; `L` and `n` may shrink it (same recipe, same seed)."""
    w = dict(WORKLOADS[name])
    scale = 1.0
    if L is not None:
        scale = L / w["L"]
        w["L"] = L
        w["inset"] = w["inset"] * scale
    if n is not None:
        w["n"] = n
    rng = Xoshiro256ss(SEED_BASE + w["seed_offset"])
    Lb = w["L"]
    lo, hi = w["inset"], Lb - w["inset"]
    if w["seeds"] == "uniform":
        seeds = seeds_uniform(rng, w["n"], lo, hi)
    elif w["seeds"] == "clustered":
        seeds = seeds_clustered(rng, w["n"], lo, hi, 10, 0.05 * Lb)
    else:
        seeds = seeds_power_law(rng, w["n"], 0.5 * Lb, 0.5 * Lb, 0.5 * (hi - lo))
    kind, a, b = w["values"]
    if kind == "lognormal":
        vals = np.array([rng.lognormal(a, b) for _ in range(w["n"])])
    else:
        vals = np.array([rng.pareto(a, b) for _ in range(w["n"])])
    spacing = w["spacing"]
    m = voronoi_map(Lb, Lb, seeds, lo, spacing, vals,
                    meta={"name": name, "blur": w["blur"], "precision": w["precision"]})
    return m


# ----------------------------------------------------------------------------
# batched frames
# ----------------------------------------------------------------------------

# 64 cartograms (animation frames) with grid sizes drawn uniformly from {128, 256, 512,
# 1024}. One 300-region Voronoi geometry (uniform seeds in the unit square, scaled into
# each size's square inset L/8, 0.5-cell edges); its lognormal(0, 1) values drift from
# frame to frame by a multiplicative random walk, log-step N(0, 0.1^2). Blur 1 cell.
BATCH = dict(frames=64, sizes=(128, 256, 512, 1024), n=300, spacing=0.5, sigma=1.0, step=0.1, blur=1.0,
             seed_offset=4)


def make_batch(frames: int | None = None, sizes=None) -> list:
    """The batched workload: a list of RegionMaps, one per frame (same seed every call)."""
    w = dict(BATCH)
    if frames is not None:
        w["frames"] = frames
    if sizes is not None:
        w["sizes"] = tuple(sizes)
    rng = Xoshiro256ss(SEED_BASE + w["seed_offset"])
    unit = seeds_uniform(rng, w["n"], 0.0, 1.0)
    base = np.array([rng.lognormal(0.0, w["sigma"]) for _ in range(w["n"])])
    geometry = {}
    out = []
    # the C library's log and exp, element by element (numpy's vectorised versions round
    # differently on different hosts; these give the same bits on x86 and Arm)
    logv = np.array([math.log(x) for x in base])
    for f in range(w["frames"]):
        L = w["sizes"][int(rng.uniform() * len(w["sizes"]))]
        if f > 0:
            logv = logv + np.array([w["step"] * rng.normal() for _ in range(w["n"])])
        if L not in geometry:
            lo, hi = L / 8.0, L - L / 8.0
            geometry[L] = voronoi_map(L, L, lo + unit * (hi - lo), lo, w["spacing"], base)
        g = geometry[L]
        out.append(RegionMap(L, L, np.array([math.exp(x) for x in logv]), g.ring_offsets, g.ring_region, g.xy,
                             {"name": "batch_frame%d" % f, "blur": w["blur"], "precision": "mixed"}))
    return out

