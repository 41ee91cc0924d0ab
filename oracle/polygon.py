"""Polygon-level distortion measures (SI section 4), plain FP64 numpy / Python.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests may use this module; the
library's product path never does.

- Mean aspect ratio alpha: for each region, the bounding rectangle of minimum area over
  all orientations phi in [0, 90 deg); alpha_i = longer side / shorter side of that
  rectangle; alpha = mean over the regions. The minimum lies at an orientation parallel
  to an edge of the region's convex hull (rotating calipers), so the hull's edges are the
  candidates. The paper's argmin is ambiguous where two orientations give the same area
  (common: a cell cut by the axis-aligned sides of the inset square has two), and the
  ratio jumps there; orientations whose areas agree to 1e-9 relative are read as ties,
  which go to the smaller ratio (so that rounding cannot pick the side).
- Relative position error theta: with c_i the centroids of the regions on the input map
  and d_i on the cartogram, phi_ij = the angle between c_i - c_j and d_i - d_j (the
  paper's arccos of the normalised dot product, evaluated as atan2(|cross|, dot)), and
  theta = 2 / (p (p - 1) pi) * sum over pairs i < j of phi_ij (in [0, 1]); a pair whose
  centroids coincide on either map contributes 0.
A region's vertices are those of all its rings; its centroid is that of the signed sum
of its rings (holes subtract).

Parity status (tests/test_oracle_pins.py): region_centroids by a square with a hole in
closed form; relative_position_error by similarity maps (0 for translations and scalings,
beta / pi for a rotation by beta); convex_hull and min_area_rectangle by rectangles at
several angles and a regular hexagon in closed form, a brute-force scan over 20,000
orientations, and the tie rule on a tied cell (pinned).
"""
import math

import numpy as np


def region_centroids(n_regions, ring_offsets, ring_region, xy):
    """Area-weighted centroids of the regions, [n_regions][2], from the shoelace moments."""
    A = np.zeros(n_regions)
    M = np.zeros((n_regions, 2))
    for k in range(len(ring_region)):
        p = xy[ring_offsets[k]:ring_offsets[k + 1]]
        q = np.roll(p, -1, axis=0)
        cross = p[:, 0] * q[:, 1] - q[:, 0] * p[:, 1]
        r = int(ring_region[k])
        A[r] += 0.5 * cross.sum()
        M[r, 0] += ((p[:, 0] + q[:, 0]) * cross).sum() / 6.0
        M[r, 1] += ((p[:, 1] + q[:, 1]) * cross).sum() / 6.0
    return M / A[:, None]


def relative_position_error(c, d):
    """theta of SI section 4 for centroids c (input map) and d (cartogram)."""
    p = len(c)
    total = 0.0
    for i in range(p - 1):
        u = c[i] - c[i + 1:]
        w = d[i] - d[i + 1:]
        # the angle as atan2(|u x w|, u . w): the arccos of the normalised dot product,
        # without its loss of accuracy near 0 and pi; 0 where a vector vanishes
        cross = u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0]
        dot = u[:, 0] * w[:, 0] + u[:, 1] * w[:, 1]
        total += np.arctan2(np.abs(cross), dot).sum()
    return 2.0 * total / (p * (p - 1) * math.pi)


def convex_hull(points):
    """Andrew's monotone chain: the hull's vertices counter-clockwise, without collinear
    points."""
    pts = sorted(set(map(tuple, np.asarray(points, dtype=np.float64))))
    if len(pts) <= 2:
        return np.array(pts)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return np.array(lower[:-1] + upper[:-1])


TIE = 1e-9  # relative: rectangle areas this close are the same minimum


def min_area_rectangle(hull):
    """(area, aspect ratio) of the minimum-area bounding rectangle of a convex polygon
    (ties in area, to TIE relative, to the smaller ratio)."""
    cands = []
    h = len(hull)
    for e in range(h):
        u = hull[(e + 1) % h] - hull[e]
        u = u / math.hypot(u[0], u[1])
        a = hull @ u
        b = hull @ np.array([-u[1], u[0]])
        w, t = a.max() - a.min(), b.max() - b.min()
        cands.append((w * t, max(w, t) / min(w, t)))
    amin = min(c[0] for c in cands)
    return amin, min(r for a, r in cands if a <= amin * (1.0 + TIE))


def aspect_ratios(n_regions, ring_offsets, ring_region, xy):
    """alpha_i of every region."""
    out = np.zeros(n_regions)
    for r in range(n_regions):
        rings = np.nonzero(np.asarray(ring_region) == r)[0]
        pts = np.concatenate([xy[ring_offsets[k]:ring_offsets[k + 1]] for k in rings])
        out[r] = min_area_rectangle(convex_hull(pts))[1]
    return out


def mean_aspect_ratio(n_regions, ring_offsets, ring_region, xy):
    return float(aspect_ratios(n_regions, ring_offsets, ring_region, xy).mean())
