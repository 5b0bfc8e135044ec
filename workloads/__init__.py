"""Seeded synthetic inputs for the pressurized phase-field fracture solver.

This module only *generates inputs*: tensor-product mesh coordinates, the
initial phase field that marks the crack, material / loading parameters and
random test vectors.  It holds none of the finite-element, Newton or Krylov
arithmetic of the method, so both the CUDA path and the CPU oracle may import
it without sharing any of the method's code.

The workloads follow the Sneddon tests of the paper (Section 4): a pressurized
straight crack (2d) or penny-shaped crack (3d) of half length / radius ``l0``
centred at the origin of the box ``(-K, K)^d``, with E = 1, nu = 0.2, G_c = 1,
p = 1e-3 and eps tied to the mesh size.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "uniform_axis", "graded_axis", "crack_phi", "Workload", "config",
    "CONFIG_NAMES", "batched_instances", "served_requests", "random_state",
    "scaled_workload", "cyclic_loading", "CYCLIC_PRESSURES", "plateau_axis",
    "domain_study",
]


# ---------------------------------------------------------------- meshes ----

def uniform_axis(n_cells: int, lo: float, hi: float) -> np.ndarray:
    """n_cells + 1 equally spaced node coordinates on [lo, hi]."""
    return np.linspace(lo, hi, n_cells + 1, dtype=np.float64)


def _solve_ratio(m: int, h_min: float, half: float) -> float:
    """Ratio r with h_min * (1 + r + ... + r^(m-1)) = half (bisection)."""
    if abs(h_min * m - half) <= 1e-14 * half:
        return 1.0
    if h_min * m > half:
        raise ValueError("h_min too large for a graded axis")

    def total(r):
        return h_min * m if r == 1.0 else h_min * (r ** m - 1.0) / (r - 1.0)

    lo, hi = 1.0, 2.0
    while total(hi) < half:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < half:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def graded_axis(n_cells: int, half_width: float, h_min: float) -> np.ndarray:
    """Symmetric geometric grading of [-half_width, half_width].

    ``n_cells`` must be even; the n/2 cells on each side of 0 grow by a ratio r
    from ``h_min`` next to 0, where r is solved so the cells exactly fill the
    half width.  Node 0 sits at x = 0 (the crack plane / line).
    """
    if n_cells % 2:
        raise ValueError("graded axes need an even number of cells")
    m = n_cells // 2
    r = _solve_ratio(m, h_min, half_width)
    h = h_min * r ** np.arange(m, dtype=np.float64)
    pos = np.concatenate([[0.0], np.cumsum(h)])
    pos[-1] = half_width
    return np.concatenate([-pos[::-1], pos[1:]])


def crack_phi(coords: Sequence[np.ndarray], l0: float) -> np.ndarray:
    """Initial phase field marking the crack: 0 on every node of a cut cell, 1 elsewhere.

    2d: cell [x0,x1]x[y0,y1] is cut iff x0 < l0, x1 > -l0 and y0 <= 0 <= y1
    (a straight crack of half length l0 on y = 0).
    3d: cell is cut iff z0 <= 0 <= z1 and its xy-rectangle meets the open disc
    x^2 + y^2 < l0^2 (a penny-shaped crack of radius l0 in z = 0).
    Nodes are numbered lexicographically, x fastest.
    """
    d = len(coords)
    nn = [len(c) for c in coords]
    phi = np.ones(nn[::-1], dtype=np.float64)  # index [k][j][i]
    x = coords[0]
    y = coords[1]
    if d == 2:
        cx = (x[:-1] < l0) & (x[1:] > -l0)
        cy = (y[:-1] <= 0.0) & (y[1:] >= 0.0)
        cut = cy[:, None] & cx[None, :]          # [j][i]
        for dj in (0, 1):
            for di in (0, 1):
                sub = phi[dj:dj + cut.shape[0], di:di + cut.shape[1]]
                sub[cut] = 0.0
    elif d == 3:
        z = coords[2]
        px = np.clip(0.0, x[:-1], x[1:])          # closest point of each cell interval to 0
        py = np.clip(0.0, y[:-1], y[1:])
        disc = (py[:, None] ** 2 + px[None, :] ** 2) < l0 * l0   # [j][i]
        cz = (z[:-1] <= 0.0) & (z[1:] >= 0.0)
        cut = cz[:, None, None] & disc[None, :, :]                # [k][j][i]
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    sub = phi[dk:dk + cut.shape[0], dj:dj + cut.shape[1], di:di + cut.shape[2]]
                    sub[cut] = 0.0
    else:
        raise ValueError("dim must be 2 or 3")
    return phi.reshape(-1).copy()


# ------------------------------------------------------------- workloads ----

@dataclass
class Workload:
    """One synthetic Sneddon problem: mesh, material, crack and load schedule."""
    name: str
    dim: int
    coords: List[np.ndarray]
    E: float = 1.0
    nu: float = 0.2
    Gc: float = 1.0
    kappa: float = 1e-10
    eps: float = 0.0625
    l0: float = 0.25
    pressures: List[float] = field(default_factory=lambda: [1e-3])
    precision: str = "fp64"   # "fp64" or "mixed"

    @property
    def n_cells(self) -> List[int]:
        return [len(c) - 1 for c in self.coords]

    @property
    def n_nodes(self) -> int:
        return int(np.prod([len(c) for c in self.coords]))

    @property
    def n_dofs(self) -> int:
        return (self.dim + 1) * self.n_nodes

    def phi0(self) -> np.ndarray:
        return crack_phi(self.coords, self.l0)

    def h_min(self) -> float:
        return float(min(np.min(np.diff(c)) for c in self.coords))


CONFIG_NAMES = ("sneddon2d_128", "sneddon2d_graded_1024", "penny3d_graded_128",
                "batched2d_256", "served_mixed")


def config(i: int) -> Workload:
    """The five standard workloads (index 0..2 are single problems)."""
    if i == 0:
        # [-2,2]^2, uniform 128x128, h = 1/32, eps = 2h, one loading step
        ax = uniform_axis(128, -2.0, 2.0)
        return Workload("sneddon2d_128", 2, [ax, ax.copy()], eps=2.0 / 32.0)
    if i == 1:
        # [-10,10]^2, 1024x1024 graded from h_min = 2e-4, eps = 2 h_min,
        # five loading steps p = 2e-4 * n
        ax = graded_axis(1024, 10.0, 2e-4)
        return Workload("sneddon2d_graded_1024", 2, [ax, ax.copy()], eps=4e-4,
                        pressures=[2e-4 * n for n in range(1, 6)], precision="mixed")
    if i == 2:
        # [-2,2]^3, 128^3 graded from h_min = 4e-3, penny radius 0.25
        ax = graded_axis(128, 2.0, 4e-3)
        return Workload("penny3d_graded_128", 3, [ax, ax.copy(), ax.copy()], eps=8e-3,
                        precision="mixed")
    raise ValueError("configs 3 and 4 are instance sets: use batched_instances / served_requests")


def scaled_workload(w: Workload, n_cells: int, graded: Optional[bool] = None) -> Workload:
    """Same geometry / material recipe as ``w`` at another resolution.

    Uniform workloads keep eps = 2h; graded ones keep the grading recipe with
    h_min scaled by the resolution ratio (so eps = 2 h_min stays tied to h).
    """
    half = float(w.coords[0][-1])
    n0 = w.n_cells[0]
    hmin0 = w.h_min()
    is_graded = graded if graded is not None else (np.ptp(np.diff(w.coords[0])) > 1e-12 * half)
    if is_graded:
        hmin = hmin0 * n0 / n_cells
        ax = graded_axis(n_cells, half, hmin)
        eps = w.eps * hmin / hmin0
    else:
        ax = uniform_axis(n_cells, -half, half)
        eps = w.eps * n0 / n_cells
    return replace(w, name=f"{w.name}@{n_cells}", coords=[ax.copy() for _ in range(w.dim)], eps=eps)


def plateau_axis(half_width: float, h: float, plateau: float, ratio: float = 1.05) -> np.ndarray:
    """Uniform cells of size h on [-plateau, plateau] (rounded to whole cells),
    then cells growing geometrically from h to the edges of [-half_width,
    half_width], with the smallest cell count whose ratio does not exceed
    ``ratio`` (the ratio is then solved so the cells fill the half width)."""
    n_plat = int(round(2.0 * plateau / h))
    a = n_plat * h / 2.0
    rest = half_width - a
    m = int(math.ceil(math.log(1.0 + rest * (ratio - 1.0) / h) / math.log(ratio)))
    r = _solve_ratio(m, h, rest)
    right = a + np.concatenate([[0.0], np.cumsum(h * r ** np.arange(m, dtype=np.float64))])
    right[-1] = half_width
    return np.concatenate([-right[::-1][:-1], np.linspace(-a, a, n_plat + 1), right[1:]])


def domain_study(K: float, h: float, l0: float = 1.0, ratio: float = 1.05) -> Workload:
    """One mesh of the finite-domain study of Section 4.2 (2d Sneddon, l0 = 1).

    The box (-K, K)^2 with cells of size h on the crack and around it in x
    (uniform on |x| <= 1.25 l0) and next to the crack line in y, growing
    geometrically (ratio <= 1.05) toward the edges; eps = 2h, E = 1, nu = 0.2,
    G_c = 1, p = 1e-3, kappa = 1e-10.  The paper refines adaptively; this is
    the tensor-product stand-in with the same finest cell size on the crack.
    """
    x = plateau_axis(K, h, 1.25 * l0, ratio)
    m = int(math.ceil(math.log(1.0 + K * (ratio - 1.0) / h) / math.log(ratio)))
    y = graded_axis(2 * m, K, h)
    return Workload(f"domain2d_K{K:g}_h{h:g}", 2, [x, y], eps=2.0 * h, l0=l0, pressures=[1e-3])


# load, unload, reload: the first three steps approach the critical pressure, the
# next two unload, the last two reload past the earlier maximum
CYCLIC_PRESSURES = (4e-3, 8e-3, 1.1e-2, 6e-3, 2e-3, 8e-3, 1.2e-2)


def cyclic_loading(n_cells: int = 64) -> Workload:
    """A crack that grows under a load / unload / reload pressure cycle.

    Geometry of the 2d Sneddon test (uniform on [-2,2]^2, l0 = 0.25, eps = 2h,
    E = 1, nu = 0.2, kappa = 1e-10) with G_c lowered to 1e-4, so that the
    sharp-crack critical pressure sqrt(E G_c / ((1 - nu^2) pi l0)) ~ 1.15e-2
    lies inside the schedule CYCLIC_PRESSURES.  While the pressure rises the
    phase field drops ahead of both tips and the crack lengthens; while it
    falls the phase field would heal, and the irreversibility constraint
    phi <= phi_old holds it on the whole damaged zone (Formulation 1).
    Pressure control past the critical pressure makes the growth unstable, so
    the schedule stays near it.
    """
    ax = uniform_axis(n_cells, -2.0, 2.0)
    return Workload(f"cyclic2d_{n_cells}", 2, [ax, ax.copy()], Gc=1e-4, eps=2.0 * 4.0 / n_cells,
                    pressures=list(CYCLIC_PRESSURES))


def adaptive_sneddon2d(n0: int = 32, cycles: int = 6):
    """Adaptive 2d Sneddon sequence (Section 3 refinement strategy, Section 4.4 study).

    Config 0's geometry and material ([-2,2]^2, l0 = 0.25, p = 1e-3) starting
    from a uniform n0^2 mesh.  Cycle k solves one loading step with
    eps_k = 2 h_k, h_k = h_0 / 2^k, and the next mesh keeps the crack region
    at h <= h_{k+1} (h_band = eps_{k+1} / 2) besides the gradient-jump marking
    (theta = 0.3, crack region = slabs with min phi < 0.5).  Returns the cycle-0
    workload and a list of (h_k, eps_k) for k = 0 .. cycles - 1.
    """
    ax = uniform_axis(n0, -2.0, 2.0)
    h0 = 4.0 / n0
    w = Workload(f"adaptive_sneddon2d_{n0}", 2, [ax, ax.copy()], eps=2.0 * h0)
    return w, [(h0 / 2 ** k, 2.0 * h0 / 2 ** k) for k in range(cycles)]


ADAPT_THETA = 0.3
ADAPT_PHI_BAND = 0.5


def batched_instances(count: int = 256, seed: int = 1806) -> List[Workload]:
    """Independent 2d Sneddon instances of mixed size (seeded, numpy PCG64).

    n = 2 * round(16 * 16^U) cells per axis (even, 32..512), uniform on [-2,2]^2,
    p ~ U[1e-4, 1e-2], l0 ~ U[0.1, 0.5], nu ~ U[0.15, 0.35], eps = c h with
    c ~ U[2, 4], E = G_c = 1, kappa = 1e-10, one loading step.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        U, p, l0, nu, c = rng.random(5)
        n = int(2 * round(16.0 * 16.0 ** U))
        n = max(32, min(512, n))
        ax = uniform_axis(n, -2.0, 2.0)
        h = 4.0 / n
        out.append(Workload(f"inst{k:03d}_n{n}", 2, [ax, ax.copy()],
                            nu=0.15 + 0.2 * nu, eps=(2.0 + 2.0 * c) * h,
                            l0=0.1 + 0.4 * l0, pressures=[1e-4 + (1e-2 - 1e-4) * p],
                            precision="mixed"))
    return out


def served_requests(count: int, seed: int = 1807, steps: int = 10):
    """Mixed 2d / 3d requests for the serving stream (seeded, numpy PCG64).

    70 % 2d (n log-uniform in 64..1024, graded with h_min = 1/4 of the uniform
    spacing), 30 % 3d (n log-uniform in 32..128, graded likewise), parameters as
    for the batched instances, a linear pressure ramp of ``steps`` steps.
    Returns a list of (Workload, arrival_fraction) where the fraction is a
    unit-rate exponential inter-arrival draw, to be divided by the rate.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        u_dim, u_n, p, l0, nu, c, gap = rng.random(7)
        if u_dim < 0.7:
            d, lo_n, hi_n = 2, 64, 1024
        else:
            d, lo_n, hi_n = 3, 32, 128
        n = int(round(lo_n * (hi_n / lo_n) ** u_n / 2.0)) * 2
        hmin = 0.25 * 4.0 / n
        ax = graded_axis(n, 2.0, hmin)
        pmax = 1e-4 + (1e-2 - 1e-4) * p
        w = Workload(f"req{k:04d}_{d}d_n{n}", d, [ax.copy() for _ in range(d)],
                     nu=0.15 + 0.2 * nu, eps=(2.0 + 2.0 * c) * hmin, l0=0.1 + 0.4 * l0,
                     pressures=[pmax * (s + 1) / steps for s in range(steps)],
                     precision="mixed")
        out.append((w, float(-math.log(1.0 - gap))))
    return out


def random_state(w: Workload, seed: int, u_scale: float = 1e-3):
    """Seeded random smooth-ish state (u, phi, phi_old, phi_tilde) for operator tests.

    u is random in [-u_scale, u_scale] with zeros on the outer boundary nodes;
    phi, phi_old and phi_tilde are random in [0, 1] with phi <= phi_old.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = w.n_nodes
    u = u_scale * (2.0 * rng.random((n, w.dim)) - 1.0)
    nn = [len(c) for c in w.coords]
    idx = np.indices(nn[::-1]).reshape(w.dim, -1)[::-1]   # idx[a] = axis-a index, x fastest
    bnd = np.zeros(n, dtype=bool)
    for a in range(w.dim):
        bnd |= (idx[a] == 0) | (idx[a] == nn[a] - 1)
    u[bnd] = 0.0
    phi_old = rng.random(n)
    phi = phi_old * rng.random(n)
    phi_tilde = rng.random(n)
    return u, phi, phi_old, phi_tilde
