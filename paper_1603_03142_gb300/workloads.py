"""Seeded synthetic inputs: nest geometries and surface densities.

This module feeds both the CUDA path and the CPU oracle.  It holds none of
the force method's arithmetic: it only builds nest descriptors (integer patch
offsets) and samples surface densities at cell centres.  All random numbers
come from ``numpy.random.Generator(PCG64(seed))``.

Geometry convention (Sec. 2.1, one patch per level): every level has ``n`` x
``n`` cells; level l has cell size h0/2^l; level l's lower-left corner is
level (l-1)'s corner plus ``off[l]`` cells of level l-1.  Arrays are row-major
``[j][i]`` (y row, x column).

The workloads mirror the paper's test problems (Sec. 3: generalized Maclaurin
disks sigma_{D_n}) and the benchmark configurations:
  config1: 64^2, one level, D_1 (Maclaurin) disk a = 0.8, FP64.
  config2: 3 levels of 256^2, nest centred at (0.3, 0), D_1 a = 0.9 plus a
           Gaussian clump (peak 5, width 0.02) at the nest centre, x(1 +- 1%).
  config3: 4096^2, one level, lognormal(0, 0.5) per cell, tapered to 0 beyond
           r = 0.95.
  config4: batches of concentric nests, N in {128..1024}, 1-4 levels.
  config5: Poisson request stream (serving).

Forests (several patches per level, Sec. 2.1 Omega^l_k; Examples 3-4 of
Sec. 3) are ``Forest`` objects: patch p has ``n`` x ``n`` cells of size
h0/2^level[p] and its lower-left corner at (x0, y0) + org[p] cells of its
level; patches are listed coarsest first.  A forest's ``levels`` attribute is
its number of patches, so every per-level list (densities, forces) is a
per-patch list.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

MAX_LEVELS = 8


@dataclass
class Nest:
    """One-patch-per-level nest descriptor (mirrors ``sgf_nest_desc``)."""
    n: int
    levels: int = 1
    x0: float = -1.0
    y0: float = -1.0
    h0: float = 0.0  # 0 -> 2/n (level 0 spans [-1, 1]^2)
    off: List[Tuple[int, int]] = field(default_factory=list)

    def __post_init__(self):
        if self.h0 == 0.0:
            self.h0 = 2.0 / self.n
        off = [tuple(int(v) for v in o) for o in self.off]
        off = (off + [(0, 0)] * self.levels)[:self.levels] if off else [(0, 0)] * self.levels
        off[0] = (0, 0)  # level 0 has no parent
        self.off = off

    def h(self, l: int) -> float:
        return self.h0 / (1 << l)

    def origin(self, l: int) -> Tuple[float, float]:
        x, y = self.x0, self.y0
        for k in range(1, l + 1):
            x += self.off[k][0] * self.h(k - 1)
            y += self.off[k][1] * self.h(k - 1)
        return x, y

    def centres(self, l: int):
        """(X, Y) cell-centre coordinates of level l, each (n, n), row-major [j][i]."""
        X0, Y0 = self.origin(l)
        h = self.h(l)
        c = (np.arange(self.n) + 0.5) * h
        Y, X = np.meshgrid(Y0 + c, X0 + c, indexing="ij")
        return X, Y

    def covered_mask(self, l: int) -> np.ndarray:
        """True where level l's cell lies under the level l+1 patch."""
        m = np.zeros((self.n, self.n), dtype=bool)
        if l + 1 < self.levels:
            ox, oy = self.off[l + 1]
            m[oy:oy + self.n // 2, ox:ox + self.n // 2] = True
        return m

    def key(self):
        return (self.n, self.levels, tuple(self.off))


@dataclass
class Forest:
    """Several n x n patches per level (mirrors ``sgf_forest_desc``)."""
    n: int
    level: List[int]
    org: List[Tuple[int, int]]
    x0: float = -1.0
    y0: float = -1.0
    h0: float = 0.0  # 0 -> 2/n

    def __post_init__(self):
        if self.h0 == 0.0:
            self.h0 = 2.0 / self.n
        self.level = [int(v) for v in self.level]
        self.org = [tuple(int(v) for v in o) for o in self.org]
        if len(self.level) != len(self.org):
            raise ValueError("one level and one corner per patch")

    @property
    def patches(self) -> int:
        return len(self.level)

    @property
    def levels(self) -> int:  # per-patch lists stand where nests have per-level ones
        return len(self.level)

    def h(self, p: int) -> float:
        return self.h0 / (1 << self.level[p])

    def origin(self, p: int) -> Tuple[float, float]:
        return self.x0 + self.org[p][0] * self.h(p), self.y0 + self.org[p][1] * self.h(p)

    def centres(self, p: int):
        X0, Y0 = self.origin(p)
        c = (np.arange(self.n) + 0.5) * self.h(p)
        Y, X = np.meshgrid(Y0 + c, X0 + c, indexing="ij")
        return X, Y

    def covered_mask(self, p: int) -> np.ndarray:
        """True where patch p's cell lies under a patch of the next finer level."""
        n, half = self.n, self.n // 2
        m = np.zeros((n, n), dtype=bool)
        for q in range(self.patches):
            if self.level[q] != self.level[p] + 1:
                continue
            cx = self.org[q][0] // 2 - self.org[p][0]
            cy = self.org[q][1] // 2 - self.org[p][1]
            m[max(cy, 0):max(min(cy + half, n), 0), max(cx, 0):max(min(cx + half, n), 0)] = True
        return m

    def key(self):
        return (self.n, tuple(self.level), tuple(self.org))

    @staticmethod
    def from_nest(nest: "Nest") -> "Forest":
        """The one-patch-per-level nest as a forest (same cells, same order)."""
        org, cx, cy = [], 0, 0
        for l in range(nest.levels):
            if l > 0:
                cx, cy = 2 * (cx + nest.off[l][0]), 2 * (cy + nest.off[l][1])
            org.append((cx, cy))
        return Forest(n=nest.n, level=list(range(nest.levels)), org=org, x0=nest.x0, y0=nest.y0, h0=nest.h0)


def example3_forest(n: int) -> Forest:
    """Sec. 3, Example 3 exactly on Omega = [-1, 1]^2: level 0 of 2n cells across
    [-1, 1] (cell 1/n) as six n x n tiles, columns x in [-1, 0] and [0, 1], rows
    y in [-1.5, -0.5], [-0.5, 0.5], [0.5, 1.5]; level 1 the paper's two patches
    [-0.75, -0.25] x [-0.25, 0.25] and [0.25, 0.75] x [-0.25, 0.25] (n cells of
    1/(2n)).  The tile seams lie where the two disks have no mass, and cells
    outside Omega carry none, so forces inside Omega are those of one level-0
    patch over Omega; the paper's N is 2n."""
    org0 = [(0, 0), (n, 0), (0, n), (n, n), (0, 2 * n), (n, 2 * n)]
    org1 = [(n // 2, 5 * n // 2), (5 * n // 2, 5 * n // 2)]
    return Forest(n=n, level=[0] * 6 + [1, 1], org=org0 + org1, x0=-1.0, y0=-1.5, h0=1.0 / n)


def two_patch_forest(n: int) -> Forest:
    """One level-0 patch [-1, 1]^2 (cell 2/n) and one level-1 patch over each disk of
    Examples 3-4, [-1, 0] x [-0.5, 0.5] and [0, 1] x [-0.5, 0.5], sharing an edge."""
    return Forest(n=n, level=[0, 1, 1], org=[(0, 0), (0, n // 2), (n, n // 2)])


def example4_forest(n: int) -> Forest:
    """Two disks, three levels (Sec. 3, Example 4): level 0 [-1, 1]^2 (cell 2/n);
    level 1 as in two_patch_forest (the paper's 0.8-wide level-1 patches are not a
    whole number of level-0 cells); level 2 exactly the paper's
    [-0.75, -0.25] x [-0.25, 0.25] and [0.25, 0.75] x [-0.25, 0.25]."""
    return Forest(n=n, level=[0, 1, 1, 2, 2],
                  org=[(0, 0), (0, n // 2), (n, n // 2), (n // 2, 3 * n // 2), (5 * n // 2, 3 * n // 2)])


def two_disk_density(forest, order: int = 5, alpha: float = math.sqrt(2.0) / 4.0) -> List[np.ndarray]:
    """Examples 3-4: sigma_{D_order} disks of radius alpha centred at (-1/2, 0) and (1/2, 0)."""
    return dn_density(forest, order, alpha, centres=((-0.5, 0.0), (0.5, 0.0)))


def centred_nest(n: int, levels: int, centre=(0.0, 0.0), x0: float = -1.0, y0: float = -1.0,
                 h0: float = 0.0) -> Nest:
    """Nest whose refined patches are centred as closely as the lattice allows on
    ``centre``: level l's corner is round((c - halfwidth_l - corner_{l-1}) / h_{l-1})
    parent cells from its parent's corner, clamped so the child stays inside."""
    g = Nest(n=n, levels=1, x0=x0, y0=y0, h0=h0)
    off = [(0, 0)]
    X, Y = g.x0, g.y0
    for l in range(1, levels):
        hp = g.h0 / (1 << (l - 1))
        half_w = 0.5 * n * g.h0 / (1 << l)
        ox = int(round((centre[0] - half_w - X) / hp))
        oy = int(round((centre[1] - half_w - Y) / hp))
        ox = min(max(ox, 0), n // 2)
        oy = min(max(oy, 0), n // 2)
        off.append((ox, oy))
        X += ox * hp
        Y += oy * hp
    return Nest(n=n, levels=levels, x0=g.x0, y0=g.y0, h0=g.h0, off=off)


# --------------------------------------------------------------- densities

def dn_density(nest: Nest, order: int, alpha: float, sigma0: float = 1.0,
               centres: Sequence[Tuple[float, float]] = ((0.0, 0.0),)) -> List[np.ndarray]:
    """sigma_{D_n}(r; alpha) = sigma0 (1 - r^2/alpha^2)^(order - 1/2) for r < alpha
    (Sec. 3), summed over the given disk centres, sampled at cell centres."""
    out = []
    for l in range(nest.levels):
        X, Y = nest.centres(l)
        s = np.zeros_like(X)
        for cx, cy in centres:
            r2 = ((X - cx) ** 2 + (Y - cy) ** 2) / alpha ** 2
            inside = r2 < 1.0
            s[inside] += sigma0 * (1.0 - r2[inside]) ** (order - 0.5)
        out.append(s)
    return out


def gaussian_clumps(nest: Nest, clumps) -> List[np.ndarray]:
    """sum_k peak_k exp(-|x - c_k|^2 / (2 w_k^2)) at cell centres; clumps = [(cx, cy, peak, w)]."""
    out = []
    for l in range(nest.levels):
        X, Y = nest.centres(l)
        s = np.zeros_like(X)
        for cx, cy, peak, w in clumps:
            s += peak * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * w * w))
        out.append(s)
    return out


def config1(n: int = 64):
    """Uniform level, D_1 (Maclaurin) disk a = 0.8, sigma0 = 1."""
    nest = Nest(n=n, levels=1)
    return nest, dn_density(nest, 1, 0.8)


def config2(n: int = 256, levels: int = 3, seed: int = 0):
    """3-level nest centred at (0.3, 0); Maclaurin a = 0.9 + Gaussian clump
    (peak 5, width 0.02) at the nest centre, times (1 + U(-0.01, 0.01))."""
    nest = centred_nest(n, levels, centre=(0.3, 0.0))
    rng = np.random.Generator(np.random.PCG64(seed))
    base = dn_density(nest, 1, 0.9)
    clump = gaussian_clumps(nest, [(0.3, 0.0, 5.0, 0.02)])
    out = []
    for l in range(levels):
        noise = 1.0 + rng.uniform(-0.01, 0.01, size=(n, n))
        out.append((base[l] + clump[l]) * noise)
    return nest, out


def lognormal_taper(nest: Nest, seed: int = 0, mu: float = 0.0, s: float = 0.5):
    """sigma = exp(mu + s Z) per cell, Z ~ N(0,1), times the taper
    w(r) = 1 (r <= 0.9), cos^2(pi (r - 0.9)/0.1) (0.9 < r < 0.95), 0 beyond."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for l in range(nest.levels):
        X, Y = nest.centres(l)
        r = np.hypot(X, Y)
        w = np.where(r <= 0.9, 1.0, np.where(r < 0.95, np.cos(np.pi * (r - 0.9) / 0.1) ** 2, 0.0))
        z = rng.standard_normal(size=X.shape)
        out.append(np.exp(mu + s * z) * w)
    return out


def config3(n: int = 4096, seed: int = 0):
    nest = Nest(n=n, levels=1)
    return nest, lognormal_taper(nest, seed)


def random_nest_problem(rng: np.random.Generator, n: int, levels: int):
    """Concentric nest at the origin; Maclaurin disk of radius U(0.5, 0.95) plus
    K ~ U{0..3} Gaussian clumps (centre uniform in the disk of radius 0.7a,
    peak U(1, 5), width U(0.01, 0.05))."""
    nest = centred_nest(n, levels, centre=(0.0, 0.0))
    a = rng.uniform(0.5, 0.95)
    k = int(rng.integers(0, 4))
    clumps = []
    for _ in range(k):
        rr = 0.7 * a * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2.0 * math.pi)
        clumps.append((rr * math.cos(th), rr * math.sin(th), rng.uniform(1.0, 5.0), rng.uniform(0.01, 0.05)))
    base = dn_density(nest, 1, a)
    cl = gaussian_clumps(nest, clumps) if clumps else [np.zeros((n, n)) for _ in range(levels)]
    return nest, [base[l] + cl[l] for l in range(levels)]


def config4(count: int = 256, seed: int = 0, sizes=(128, 256, 512, 1024), max_levels: int = 4):
    """Batch of independent concentric nests of uneven N and level count."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        L = int(rng.integers(1, max_levels + 1))
        probs.append(random_nest_problem(rng, n, L))
    return probs


def config5_arrivals(rate: float = 200.0, duration: float = 60.0, seed: int = 0,
                     sizes=(256, 512, 1024, 2048), levels=(2, 5)):
    """Poisson arrivals: list of (t_arrival, n, levels, precision, problem_seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(rng.choice(sizes))
        L = int(rng.integers(levels[0], levels[1] + 1))
        prec = "fp32" if rng.uniform() < 0.5 else "bf16x"
        reqs.append((t, n, L, prec, int(rng.integers(0, 2 ** 31 - 1))))
    return reqs
