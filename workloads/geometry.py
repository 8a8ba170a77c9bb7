"""Seeded layered media and scatterer polygons for the synthetic workloads.

Every workload is synthetic: the paper (Sec. 5) measures on its own generated
geometries, not on a dataset.  The recipes below follow the paper's examples
(Sec. 5, Examples 1-3; the sine-star family r = a sin k(theta-theta0) + b of
Example 2) and the benchmark configurations C1-C5 (two- to four-layer media,
circles and ellipses placed at random).

A medium is described by
  * ``interfaces``: the interface heights y_j = -d_j, strictly decreasing,
  * ``k``: one real wavenumber per layer (L+1 values, top layer first),
  * ``eta``: one density ("reflection index") per layer.
A body is a closed counter-clockwise polygon, an ``(nv, 2)`` float64 array of
vertices.  Turning vertices into elements is left to the consumers.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Medium:
    interfaces: np.ndarray  # (L,) strictly decreasing interface heights
    k: np.ndarray  # (L+1,) wavenumbers, top layer first
    eta: np.ndarray  # (L+1,) densities

    def __post_init__(self):
        self.interfaces = np.asarray(self.interfaces, dtype=np.float64).reshape(-1)
        self.k = np.asarray(self.k, dtype=np.float64).reshape(-1)
        self.eta = np.asarray(self.eta, dtype=np.float64).reshape(-1)
        if self.k.size != self.interfaces.size + 1 or self.eta.size != self.k.size:
            raise ValueError("need L interfaces and L+1 wavenumbers/densities")
        if np.any(np.diff(self.interfaces) >= 0):
            raise ValueError("interfaces must be strictly decreasing")

    @property
    def n_layers(self) -> int:
        return int(self.k.size)


@dataclass
class Workload:
    name: str
    medium: Medium
    bodies: list  # list of (nv, 2) float64 arrays, CCW closed polygons
    angles_deg: np.ndarray = field(default_factory=lambda: np.array([45.0]))
    p: int = 20
    leaf_size: int = 64
    extra: dict = field(default_factory=dict)

    @property
    def n_elements(self) -> int:
        return int(sum(b.shape[0] for b in self.bodies))


# --------------------------------------------------------------------------
# shapes
# --------------------------------------------------------------------------

def circle(cx: float, cy: float, r: float, n: int) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def ellipse(cx: float, cy: float, a: float, b: float, rot: float, n: int) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(n) / n
    ex, ey = a * np.cos(t), b * np.sin(t)
    c, s = math.cos(rot), math.sin(rot)
    return np.stack([cx + c * ex - s * ey, cy + s * ex + c * ey], axis=1)


def sine_star(cx: float, cy: float, a: float, b: float, kk: int, theta0: float, n: int) -> np.ndarray:
    """Polar curve r(theta) = a sin(kk (theta - theta0)) + b about (cx, cy) (Sec. 5, Example 2)."""
    t = 2.0 * np.pi * np.arange(n) / n
    r = a * np.sin(kk * (t - theta0)) + b
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


L_SHAPE_VERTICES = np.array(
    [(0.75, 0.75), (-0.75, 0.75), (-0.75, -2.5), (2.25, -2.5), (2.25, -1.5), (0.75, -1.5)]
)


def l_shape(n: int) -> np.ndarray:
    """The L-shaped scatterer of Sec. 5, Example 1, split into n equal-length edges.

    The perimeter is 12.5 = 50 quarter units; n must be a multiple of 50 so that
    every side holds a whole number of elements.
    """
    if n % 50:
        raise ValueError("l_shape: n must be a multiple of 50")
    per_quarter = n // 50
    out = []
    v = L_SHAPE_VERTICES
    for i in range(len(v)):
        a, b = v[i], v[(i + 1) % len(v)]
        m = int(round(np.hypot(*(b - a)) / 0.25)) * per_quarter
        s = np.arange(m) / m
        out.append(a[None, :] + s[:, None] * (b - a)[None, :])
    return np.concatenate(out, axis=0)


# --------------------------------------------------------------------------
# random circle/ellipse fields (configs C2-C5)
# --------------------------------------------------------------------------

def _min_dist_to_interfaces(poly: np.ndarray, interfaces: np.ndarray) -> float:
    if interfaces.size == 0:
        return np.inf
    mid_y = 0.5 * (poly[:, 1] + np.roll(poly[:, 1], -1))
    ys = np.concatenate([poly[:, 1], mid_y])
    return float(np.min(np.abs(ys[:, None] - interfaces[None, :])))


def random_bodies(rng: np.random.Generator, n_bodies: int, region, interfaces, nodes: int,
                  rmin: float = 0.2, rmax: float = 0.6, gap: float = 0.05,
                  iface_tol: float = 1e-6, max_tries: int = 200000):
    """Place ``n_bodies`` circles/ellipses (half each) uniformly in ``region``.

    Bodies whose bounding circles come closer than ``gap``, or with a vertex or
    chord midpoint within ``iface_tol`` of an interface, are redrawn.
    """
    (x0, x1), (y0, y1) = region
    interfaces = np.asarray(interfaces, dtype=np.float64)
    centres, radii, polys = [], [], []
    tries = 0
    while len(polys) < n_bodies:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_bodies: could not place all bodies")
        cx, cy = rng.uniform(x0, x1), rng.uniform(y0, y1)
        if rng.uniform() < 0.5:
            r = rng.uniform(rmin, rmax)
            poly, rb = circle(cx, cy, r, nodes), r
        else:
            a, b = rng.uniform(rmin, rmax), rng.uniform(rmin, rmax)
            rot = rng.uniform(0.0, np.pi)
            poly, rb = ellipse(cx, cy, a, b, rot, nodes), max(a, b)
        if centres:
            c = np.asarray(centres)
            d = np.hypot(c[:, 0] - cx, c[:, 1] - cy)
            if np.any(d < np.asarray(radii) + rb + gap):
                continue
        if _min_dist_to_interfaces(poly, interfaces) < iface_tol:
            continue
        centres.append((cx, cy))
        radii.append(rb)
        polys.append(poly)
    return polys


def _crosses(poly: np.ndarray, interfaces: np.ndarray) -> bool:
    lo, hi = poly[:, 1].min(), poly[:, 1].max()
    return bool(np.any((interfaces > lo) & (interfaces < hi)))


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

def config_c1() -> Workload:
    """Two layers split at y=0, k=(2,4), eta=(1,2); one circle r=0.5 at (0,1), 256 nodes, 45 deg."""
    med = Medium(interfaces=[0.0], k=[2.0, 4.0], eta=[1.0, 2.0])
    return Workload("C1", med, [circle(0.0, 1.0, 0.5, 256)], np.array([45.0]), p=20, leaf_size=64)


def config_c2(n_bodies: int = 64, nodes: int = 1024, seed: int = 12452) -> Workload:
    """Three layers (interfaces y=0,-2), k=(4,6,8), eta=(1,2,3); 64 random bodies x 1024 nodes."""
    med = Medium(interfaces=[0.0, -2.0], k=[4.0, 6.0, 8.0], eta=[1.0, 2.0, 3.0])
    rng = np.random.default_rng(seed)
    while True:
        polys = random_bodies(rng, n_bodies, ((-10.0, 10.0), (-4.0, 2.0)), med.interfaces, nodes)
        if any(_crosses(p, med.interfaces) for p in polys):
            break
    return Workload("C2", med, polys, np.array([45.0]), p=20, leaf_size=64,
                    extra={"seed": seed})


def config_c3(n_bodies: int = 1024, nodes: int = 1024, seed: int = 12453) -> Workload:
    """Four layers (interfaces y=0,-6,-12), k=(6,10,8,12), eta=(1..4); region scaled x4."""
    med = Medium(interfaces=[0.0, -6.0, -12.0], k=[6.0, 10.0, 8.0, 12.0], eta=[1.0, 2.0, 3.0, 4.0])
    rng = np.random.default_rng(seed)
    while True:
        polys = random_bodies(rng, n_bodies, ((-40.0, 40.0), (-18.0, 6.0)), med.interfaces, nodes)
        if any(_crosses(p, med.interfaces) for p in polys):
            break
    return Workload("C3", med, polys, np.array([45.0]), p=20, leaf_size=64,
                    extra={"seed": seed})


def _round256(x: float) -> int:
    return max(256, int(round(x / 256.0)) * 256)


def config_c4(seed: int = 12454):
    """Sixteen uneven geometries (4k..128k points) with 32 incidence angles as a block RHS."""
    rng = np.random.default_rng(seed)
    out = []
    angles = (np.arange(32) + 0.5) * 180.0 / 32.0
    for i in range(16):
        nlay = 2 + (i % 3)
        interfaces = -2.0 * np.arange(nlay - 1)
        k = rng.uniform(2.0, 12.0, size=nlay)
        med = Medium(interfaces=interfaces, k=k, eta=np.arange(1, nlay + 1, dtype=float))
        n_target = _round256(4096.0 * 32.0 ** (i / 15.0))
        nb = max(1, n_target // 1024)
        nodes = n_target // nb
        side = 20.0 * math.sqrt(nb / 64.0)
        ylo = float(interfaces[-1]) - 2.0 if interfaces.size else -2.0
        region = ((-side / 2, side / 2), (ylo - side * 0.15, ylo + side * 0.15 + 4.0))
        polys = random_bodies(rng, nb, region, med.interfaces, nodes)
        out.append(Workload(f"C4_{i}", med, polys, angles.copy(), p=20, leaf_size=64))
    return out


def config_c5_request(rng: np.random.Generator, n_min: float = 2048.0, n_max: float = 262144.0,
                      max_bodies: int = 512) -> Workload:
    """One serving request: random layer stack and a random field of bodies."""
    nlay = int(rng.integers(2, 5))
    interfaces = -2.0 * np.arange(nlay - 1)
    k = rng.uniform(2.0, 12.0, size=nlay)
    med = Medium(interfaces=interfaces, k=k, eta=np.arange(1, nlay + 1, dtype=float))
    nb = int(rng.integers(1, max_bodies + 1))
    n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
    nodes = max(64, int(round(n / nb)))
    side = 20.0 * math.sqrt(nb / 64.0)
    region = ((-side / 2, side / 2), (-side * 0.25 - 1.0, side * 0.25 + 1.0))
    polys = random_bodies(rng, nb, region, med.interfaces, nodes)
    return Workload("C5_req", med, polys, np.array([float(rng.uniform(5.0, 175.0))]), p=20)


def config_c5_stream(n_requests: int = 24, seed: int = 12455, n_min: float = 2048.0, n_max: float = 32768.0,
                     max_bodies: int = 32) -> list:
    """A bounded stand-in for the serving stream: requests drawn like config_c5_request but
    with N in [n_min, n_max] and at most ``max_bodies`` bodies, so a run takes about a minute."""
    rng = np.random.default_rng(seed)
    return [config_c5_request(rng, n_min, n_max, max_bodies) for _ in range(n_requests)]


def example1(n: int = 12000) -> Workload:
    """Sec. 5, Example 1: L-shape across four of five layers, manufactured solution."""
    med = Medium(interfaces=[0.0, -1.0, -2.0, -3.0], k=[3.2, 2.5, 5.1, 8.6, 6.9],
                 eta=[1.0, 2.0, 3.0, 4.0, 5.0])
    return Workload("E1", med, [l_shape(n)], np.array([45.0]),
                    extra={"source": (0.0, 0.375)})


def example2(n: int = 12000) -> Workload:
    """Sec. 5, Example 2: two peanut scatterers in six layers."""
    med = Medium(interfaces=[0.0, -1.0, -2.0, -3.0, -4.0], k=[1.2, 2.3, 4.5, 6.1, 7.7, 10.0],
                 eta=[1.1, 2.3, 3.4, 4.6, 5.0, 6.6])
    half = n // 2
    bodies = [sine_star(0.0, -1.0, 0.5, 1.0, 2, np.pi / 4, half),
              sine_star(2.0, -3.0, 0.5, 1.0, 2, np.pi / 4, n - half)]
    # incident direction (-3 sqrt2/5, -3 sqrt2/5): 225 degrees below the x axis,
    # i.e. the angle convention u_inc = exp(i k0 (x cos th - y sin th)) with th = 135 deg.
    return Workload("E2", med, bodies, np.array([135.0]))


def example3(n: int = 12000) -> Workload:
    """Sec. 5, Example 3: five flower scatterers in six layers, normal incidence."""
    med = Medium(interfaces=[0.0, -1.0, -2.0, -3.0, -4.0], k=[2.0, 3.0, 6.0, 5.0, 8.0, 10.0],
                 eta=[1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    centres = [(-1.5, 0.0), (1.5, 0.0), (0.0, -2.0), (-1.5, -4.0), (1.5, 4.0)]
    per = n // 5
    bodies = [sine_star(cx, cy, 0.2, 0.7, 5, 0.0, per) for cx, cy in centres]
    return Workload("E3", med, bodies, np.array([90.0]))


def layered_small(n_bodies: int = 3, nodes: int = 200, seed: int = 7, n_layers: int = 3) -> Workload:
    """A small multi-layer case for parity tests (a few hundred to a few thousand points)."""
    interfaces = [0.0, -1.5, -3.0][: n_layers - 1]
    k = [4.0, 6.0, 8.0, 5.0][:n_layers]
    eta = [1.0, 2.0, 3.0, 4.0][:n_layers]
    med = Medium(interfaces=interfaces, k=k, eta=eta)
    rng = np.random.default_rng(seed)
    lo = (interfaces[-1] - 1.2) if interfaces else -1.5
    while True:
        polys = random_bodies(rng, n_bodies, ((-2.0, 2.0), (lo, 1.2)), med.interfaces, nodes,
                              rmin=0.25, rmax=0.7, iface_tol=1e-3)
        if not interfaces or any(_crosses(p, med.interfaces) for p in polys):
            break
    return Workload(f"small_{n_layers}L", med, polys, np.array([45.0]), p=20, leaf_size=32)


def layered_wide(n_bodies: int = 5, nodes: int = 80, seed: int = 21) -> Workload:
    """Few small bodies spread over the C2 region (same medium): coarse tree levels are
    many wavelengths wide and their cells straddle interfaces, at a size the oracle
    can still evaluate densely."""
    med = Medium(interfaces=[0.0, -2.0], k=[4.0, 6.0, 8.0], eta=[1.0, 2.0, 3.0])
    rng = np.random.default_rng(seed)
    while True:
        polys = random_bodies(rng, n_bodies, ((-10.0, 10.0), (-4.0, 2.0)), med.interfaces, nodes,
                              rmin=0.2, rmax=0.6, iface_tol=1e-3)
        if any(_crosses(p, med.interfaces) for p in polys):
            break
    return Workload("wide_c2_medium", med, polys, np.array([45.0]), p=20, leaf_size=8)


def layered_wide_c3(n_bodies: int = 10, nodes: int = 48, seed: int = 53) -> Workload:
    """Few small bodies spread over the region of the million-point four-layer workload
    (interfaces y = 0, -6, -12; k = 6, 10, 8, 12; region [-40, 40] x [-18, 6]): its
    wide-band levels (orders up to 75) and straddling cells at a size the oracle can
    still evaluate densely."""
    med = Medium(interfaces=[0.0, -6.0, -12.0], k=[6.0, 10.0, 8.0, 12.0], eta=[1.0, 2.0, 3.0, 4.0])
    rng = np.random.default_rng(seed)
    while True:
        polys = random_bodies(rng, n_bodies, ((-40.0, 40.0), (-18.0, 6.0)), med.interfaces, nodes,
                              rmin=0.2, rmax=0.6, iface_tol=1e-3)
        if sum(_crosses(p, med.interfaces) for p in polys) >= 2:
            break
    return Workload("wide_c3_medium", med, polys, np.array([45.0]), p=20, leaf_size=8)

