"""Crack functionals and Sneddon's closed forms (oracle; test infrastructure only).

Section 4: TCV_h = int_Omega u . grad phi dx; the crack opening along a line
crossing the crack is the same integrand integrated along that line (the full
opening, i.e. twice Sneddon's one-sided u_n).  Closed forms from Section 4:
TCV_2d = 2 pi p l0^2 (1-nu^2)/E, TCV_3d = 16 p l0^3 (1-nu^2)/(3E),
u_n = c p l0 (1-nu^2)/E sqrt(1 - (rho/l0)^2), c = 2 (2d) or 4/pi (3d).
"""
from __future__ import annotations

import math

import numpy as np

from .fe import GAUSS_1D, WEIGHT_1D, Mesh, cell_geometry


def tcv(mesh: Mesh, u: np.ndarray, phi: np.ndarray) -> float:
    """TCV_h = int u . grad phi over all cells with the 2^d Gauss rule (exact for Q1 x Q1')."""
    N, dN, JxW = cell_geometry(mesh)
    cn = mesh.cell_nodes()
    uq = np.einsum("qa,cam->cqm", N, u[cn])
    gp = np.einsum("cqal,ca->cql", dN, phi[cn])
    return float(np.sum(JxW * np.einsum("cqm,cqm->cq", uq, gp)))


def _columns(coords_a: np.ndarray, x: float):
    """Cells of one axis whose closed interval contains x, with averaging weights.

    A point strictly inside a cell uses that cell; a point on a mesh line is the
    average of the two adjacent cells (or the single one at the domain edge).
    """
    n = len(coords_a) - 1
    if x < coords_a[0] or x > coords_a[-1]:
        raise ValueError("COD point outside the domain")
    hits = [i for i in range(max(0, np.searchsorted(coords_a, x) - 2), min(n, np.searchsorted(coords_a, x) + 2))
            if coords_a[i] <= x <= coords_a[i + 1]]
    return [(i, 1.0 / len(hits)) for i in hits]


def cod(mesh: Mesh, u: np.ndarray, phi: np.ndarray, pts) -> np.ndarray:
    """COD_h at each point: int u . grad phi along the line through the point normal to the crack.

    2d: pts are x values, the line is x = const (integrated over y).
    3d: pts are (x, y) pairs, the line is parallel to z.
    Two Gauss points per crossed cell integrate the (quadratic) integrand exactly.
    """
    d = mesh.d
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, d - 1)
    out = np.zeros(len(pts))
    X = mesh.coords
    for k, pt in enumerate(pts):
        cols = [_columns(X[a], pt[a]) for a in range(d - 1)]
        total = 0.0
        combos = [([], 1.0)]
        for a in range(d - 1):
            combos = [(c + [i], w * wi) for (c, w) in combos for (i, wi) in cols[a]]
        for idx, wt in combos:
            hxy = [X[a][idx[a] + 1] - X[a][idx[a]] for a in range(d - 1)]
            xi = [(pt[a] - X[a][idx[a]]) / hxy[a] for a in range(d - 1)]
            zl = X[d - 1]
            for j in range(len(zl) - 1):
                hz = zl[j + 1] - zl[j]
                for g, wg in zip(GAUSS_1D, WEIGHT_1D):
                    loc = xi + [g]
                    h = hxy + [hz]
                    val = 0.0
                    uq = np.zeros(d)
                    gph = np.zeros(d)
                    for a in range(2 ** d):
                        off = [(a >> l) & 1 for l in range(d)]
                        f = [loc[l] if off[l] else 1.0 - loc[l] for l in range(d)]
                        Na = float(np.prod(f))
                        node = 0
                        stride = 1
                        base = idx + [j]
                        for l in range(d):
                            node += (base[l] + off[l]) * stride
                            stride *= mesh.nn[l]
                        uq += Na * u[node]
                        for l in range(d):
                            dfl = (1.0 if off[l] else -1.0) / h[l]
                            gph[l] += dfl * float(np.prod([f[m] for m in range(d) if m != l])) * phi[node]
                    val = float(uq @ gph)
                    total += wt * wg * hz * val
        out[k] = total
    return out


def sneddon_tcv(dim: int, p: float, l0: float, E: float, nu: float) -> float:
    """Total crack volume of Sneddon's pressurized crack (Section 4)."""
    if dim == 2:
        return 2.0 * math.pi * p * l0 ** 2 * (1.0 - nu ** 2) / E
    return 16.0 * p * l0 ** 3 * (1.0 - nu ** 2) / (3.0 * E)


def sneddon_cod(dim: int, p: float, l0: float, E: float, nu: float, rho) -> np.ndarray:
    """Full opening 2 u_n(rho) with Sneddon's one-sided u_n of Section 4 (0 outside the crack)."""
    c = 2.0 if dim == 2 else 4.0 / math.pi
    rho = np.asarray(rho, dtype=np.float64)
    inside = np.clip(1.0 - (rho / l0) ** 2, 0.0, None)
    return 2.0 * c * p * l0 * (1.0 - nu ** 2) / E * np.sqrt(inside)


def cod_points(l0: float, count: int = 64) -> np.ndarray:
    """Sample abscissae x_j = l0 (-1 + (2j+1)/count) across the crack."""
    j = np.arange(count)
    return l0 * (-1.0 + (2.0 * j + 1.0) / count)
