"""Q1 finite elements on tensor-product meshes (oracle; test infrastructure only).

Section 3: the discrete spaces V_h x W_h consist of bilinear (2d) / trilinear
(3d) Q1^c functions on quadrilaterals / hexahedra.  The paper does not state
the quadrature; the oracle uses the tensor 2^d-point Gauss rule, which
integrates the Q1 stiffness, mass and TCV integrands on rectangular cells
exactly.

Numbering: nodes lexicographic with x fastest, node = i + (nx+1)(j + (ny+1)k);
cells likewise, cell = i + nx(j + ny k); local node a of a cell has offsets
(a & 1, (a >> 1) & 1, (a >> 2) & 1) along x, y, z.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache
from typing import List, Sequence

import numpy as np

GAUSS_1D = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
WEIGHT_1D = np.array([0.5, 0.5])


@lru_cache(maxsize=None)
def reference_element(d: int):
    """Shape values N[q, a], reference gradients dN[q, a, l] and weights w[q] on [0,1]^d.

    Quadrature point q has 1d Gauss indices (q & 1, (q >> 1) & 1, ...), the same
    ordering convention as local nodes.
    """
    nq = na = 2 ** d
    N = np.zeros((nq, na))
    dN = np.zeros((nq, na, d))
    w = np.zeros(nq)
    for q in range(nq):
        qi = [(q >> l) & 1 for l in range(d)]
        xi = [GAUSS_1D[qi[l]] for l in range(d)]
        w[q] = np.prod([WEIGHT_1D[qi[l]] for l in range(d)])
        for a in range(na):
            ai = [(a >> l) & 1 for l in range(d)]
            f = [xi[l] if ai[l] else 1.0 - xi[l] for l in range(d)]
            df = [1.0 if ai[l] else -1.0 for l in range(d)]
            N[q, a] = np.prod(f)
            for l in range(d):
                dN[q, a, l] = df[l] * np.prod([f[k] for k in range(d) if k != l])
    return N, dN, w


class Mesh:
    """Tensor-product mesh given by per-axis node coordinates (strictly increasing)."""

    def __init__(self, coords: Sequence[np.ndarray]):
        self.coords: List[np.ndarray] = [np.asarray(c, dtype=np.float64) for c in coords]
        self.d = len(self.coords)
        if self.d not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        for c in self.coords:
            if len(c) < 2 or np.any(np.diff(c) <= 0):
                raise ValueError("axis coordinates must be strictly increasing")
        self.nn = [len(c) for c in self.coords]
        self.nc = [n - 1 for n in self.nn]
        self.n_nodes = int(np.prod(self.nn))
        self.n_cells = int(np.prod(self.nc))

    # node (i, j, k) -> global id
    def node_id(self, *ijk) -> np.ndarray:
        gid = np.zeros_like(np.asarray(ijk[0]))
        stride = 1
        for a in range(self.d):
            gid = gid + np.asarray(ijk[a]) * stride
            stride *= self.nn[a]
        return gid

    def node_index(self) -> np.ndarray:
        """(d, n_nodes) axis indices of every node."""
        return np.indices(self.nn[::-1]).reshape(self.d, -1)[::-1].copy()

    def cell_index(self, cells=None) -> np.ndarray:
        """(d, n) axis indices of the given cells (all cells by default)."""
        ci = np.indices(self.nc[::-1]).reshape(self.d, -1)[::-1]
        return ci if cells is None else ci[:, cells]

    def cell_nodes(self, cells=None) -> np.ndarray:
        """(n, 2^d) global node ids of each cell's local nodes."""
        ci = self.cell_index(cells)
        out = np.zeros((ci.shape[1], 2 ** self.d), dtype=np.int64)
        for a in range(2 ** self.d):
            off = [(a >> l) & 1 for l in range(self.d)]
            out[:, a] = self.node_id(*[ci[l] + off[l] for l in range(self.d)])
        return out

    def cell_h(self, cells=None) -> np.ndarray:
        """(n, d) cell edge lengths."""
        ci = self.cell_index(cells)
        return np.stack([np.diff(self.coords[l])[ci[l]] for l in range(self.d)], axis=1)

    def cell_origin(self, cells=None) -> np.ndarray:
        ci = self.cell_index(cells)
        return np.stack([self.coords[l][ci[l]] for l in range(self.d)], axis=1)

    def node_xyz(self) -> np.ndarray:
        idx = self.node_index()
        return np.stack([self.coords[l][idx[l]] for l in range(self.d)], axis=1)

    def boundary_nodes(self) -> np.ndarray:
        idx = self.node_index()
        b = np.zeros(self.n_nodes, dtype=bool)
        for l in range(self.d):
            b |= (idx[l] == 0) | (idx[l] == self.nn[l] - 1)
        return b

    def cells_around(self, nodes) -> np.ndarray:
        """Sorted ids of all cells that contain any of the given nodes."""
        idx = self.node_index()[:, np.asarray(nodes)]
        out = []
        for off in itertools.product((0, 1), repeat=self.d):
            ci = [idx[l] - off[l] for l in range(self.d)]
            ok = np.ones(idx.shape[1], dtype=bool)
            for l in range(self.d):
                ok &= (ci[l] >= 0) & (ci[l] < self.nc[l])
            cid = np.zeros(int(ok.sum()), dtype=np.int64)
            stride = 1
            for l in range(self.d):
                cid += ci[l][ok] * stride
                stride *= self.nc[l]
            out.append(cid)
        return np.unique(np.concatenate(out))


def cell_geometry(mesh: Mesh, cells=None):
    """Physical gradients dN[c, q, a, l], shape values N[q, a] and JxW[c, q].

    Cells are axis-aligned boxes, so the map from [0,1]^d is diagonal:
    d/dx_l = (1/h_l) d/dxi_l and det J = prod h_l.
    """
    N, dNr, w = reference_element(mesh.d)
    h = mesh.cell_h(cells)
    dN = dNr[None, :, :, :] / h[:, None, None, :]
    JxW = w[None, :] * np.prod(h, axis=1)[:, None]
    return N, dN, JxW


def lame(E: float, nu: float):
    """Lame coefficients (mu_s, lambda_s) from Young's modulus and Poisson's ratio.

    Section 2: sigma = 2 mu_s e(u) + lambda_s tr e(u) I.  In 2d the same
    formulas give plane strain, the setting of Sneddon's (1 - nu^2)/E.
    """
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam
