"""Adaptive refinement of tensor-product meshes (oracle; test infrastructure only).

Section 3, refinement strategy: cells of the crack region are refined until
eps = 2h holds there, and a gradient-jump estimator for the displacements
drives the rest of the refinement (needed for the convergence of Section 4.4).
The paper refines octree meshes with hanging nodes and does not print its
estimator or marking rule.  These functions state the readings used here:

* Indicator (Kelly-type gradient jump; Kelly, Gago, Zienkiewicz & Babuska
  1983): for every cell K,
      eta_K^2 = (h_K / 24) * sum over the interior faces F of K of
                integral_F |[du/dn]|^2 ds,
  with h_K the diameter of K and [du/dn] the jump of the normal derivative of
  every displacement component across F.  Faces on the domain boundary
  (homogeneous Dirichlet) contribute nothing.
* Slabs: the mesh stays a tensor product, so refinement acts on axis
  intervals.  Slab i of axis a is the set of cells whose a-index is i; its
  indicator is S_a[i] = sum of eta_K^2 over the slab, and its crack measure
  is the smallest nodal phi on the slab's cells.
* Marking: interval i of axis a is split when S_a[i] >= theta * max_i S_a[i]
  (with S_a[i] > 0), or when the slab reaches the crack region
  (min phi < phi_band) and the interval is longer than h_band (eps = 2h:
  h_band = eps / 2).
* Splitting: a marked interval [x_i, x_{i+1}] gains the node 0.5 (x_i + x_{i+1}).
* Transfer: nodal fields move to the new mesh by Q1 interpolation (the finite
  element function itself, evaluated at the new nodes).

The face integrals use the 2^(d-1)-point Gauss rule on the face, exact for the
squared jump of a Q1 gradient (degree 2 in each face coordinate).

Parity unpinned against the paper for the readings themselves (the paper prints
neither the estimator nor the marking rule); the functions are pinned to these
definitions by closed forms and brute force in tests/test_oracle_adapt.py.
"""
from __future__ import annotations

import itertools
from typing import List, Sequence, Tuple

import numpy as np

from .fe import GAUSS_1D, WEIGHT_1D, Mesh


def _shape_gradients(d: int, xi: np.ndarray) -> np.ndarray:
    """Reference gradients dN[p, a, l] of the 2^d Q1 shape functions at points xi[p, l] in [0,1]^d."""
    n = xi.shape[0]
    out = np.zeros((n, 2 ** d, d))
    for a in range(2 ** d):
        off = [(a >> l) & 1 for l in range(d)]
        f = np.stack([xi[:, l] if off[l] else 1.0 - xi[:, l] for l in range(d)], axis=1)
        for l in range(d):
            g = np.full(n, 1.0 if off[l] else -1.0)
            for k in range(d):
                if k != l:
                    g = g * f[:, k]
            out[:, a, l] = g
    return out


def cell_indicators(mesh: Mesh, u: np.ndarray) -> np.ndarray:
    """eta_K^2 for every cell (Kelly-type gradient jump of the displacements, Section 3)."""
    d = mesh.d
    U = np.asarray(u, dtype=np.float64).reshape(mesh.n_nodes, d)
    eta2 = np.zeros(mesh.n_cells)
    ci = mesh.cell_index()
    h = mesh.cell_h()
    diam = np.sqrt(np.sum(h * h, axis=1))
    cn = mesh.cell_nodes()
    stride = np.cumprod([1] + mesh.nc[:-1])
    for a in range(d):
        # faces between cell K (a-index i) and K' (a-index i + 1)
        left = np.nonzero(ci[a] < mesh.nc[a] - 1)[0]
        right = left + stride[a]
        others = [l for l in range(d) if l != a]
        # Gauss points on the face, in each cell's reference coordinates
        pts_l, pts_r, wts = [], [], []
        for q in itertools.product(range(2), repeat=d - 1):
            xl = np.zeros(d)
            xr = np.zeros(d)
            xl[a], xr[a] = 1.0, 0.0
            w = 1.0
            for k, l in enumerate(others):
                xl[l] = xr[l] = GAUSS_1D[q[k]]
                w *= WEIGHT_1D[q[k]]
            pts_l.append(xl)
            pts_r.append(xr)
            wts.append(w)
        gl = _shape_gradients(d, np.array(pts_l))[:, :, a]     # [q, node] d/dxi_a
        gr = _shape_gradients(d, np.array(pts_r))[:, :, a]
        # physical normal derivative of each component at each face point
        dl = np.einsum("qn,fnm->fqm", gl, U[cn[left]]) / h[left, a][:, None, None]
        dr = np.einsum("qn,fnm->fqm", gr, U[cn[right]]) / h[right, a][:, None, None]
        area = np.ones(len(left))
        for l in others:
            area = area * h[left, l]
        jump2 = np.einsum("q,fq->f", np.array(wts), np.sum((dr - dl) ** 2, axis=2)) * area
        np.add.at(eta2, left, diam[left] / 24.0 * jump2)
        np.add.at(eta2, right, diam[right] / 24.0 * jump2)
    return eta2


def slab_indicators(mesh: Mesh, eta2: np.ndarray) -> List[np.ndarray]:
    """S_a[i] = sum of eta_K^2 over the cells of slab i of axis a."""
    ci = mesh.cell_index()
    return [np.bincount(ci[a], weights=eta2, minlength=mesh.nc[a]) for a in range(mesh.d)]


def slab_min_phi(mesh: Mesh, phi: np.ndarray) -> List[np.ndarray]:
    """Smallest nodal phi on the cells of slab i of axis a (its nodes have a-index i or i + 1)."""
    idx = mesh.node_index()
    out = []
    for a in range(mesh.d):
        per_line = np.full(mesh.nn[a], np.inf)
        np.minimum.at(per_line, idx[a], phi)
        out.append(np.minimum(per_line[:-1], per_line[1:]))
    return out


def mark_intervals(coords: Sequence[np.ndarray], S: Sequence[np.ndarray], minphi: Sequence[np.ndarray],
                   theta: float, h_band: float, phi_band: float) -> List[np.ndarray]:
    """Boolean mask of the intervals of each axis to split (the marking reading above)."""
    marks = []
    for a, x in enumerate(coords):
        h = np.diff(np.asarray(x, dtype=np.float64))
        s = np.asarray(S[a])
        smax = float(np.max(s)) if s.size else 0.0
        by_eta = (s > 0.0) & (s >= theta * smax) if smax > 0.0 else np.zeros(len(h), dtype=bool)
        by_band = (np.asarray(minphi[a]) < phi_band) & (h > h_band)
        marks.append(by_eta | by_band)
    return marks


def split_intervals(coords: Sequence[np.ndarray], marks: Sequence[np.ndarray]) -> List[np.ndarray]:
    """New axis coordinates: each marked interval gains its midpoint (when it lies strictly inside)."""
    out = []
    for x, m in zip(coords, marks):
        x = np.asarray(x, dtype=np.float64)
        mid = 0.5 * (x[:-1] + x[1:])
        keep = np.asarray(m, dtype=bool) & (mid > x[:-1]) & (mid < x[1:])
        out.append(np.sort(np.concatenate([x, mid[keep]])))
    return out


def refine(mesh: Mesh, u: np.ndarray, phi: np.ndarray, theta: float, h_band: float,
           phi_band: float) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """One refinement pass: indicators, slab sums, marking, splitting.  Returns (new coords, marks)."""
    eta2 = cell_indicators(mesh, u)
    marks = mark_intervals(mesh.coords, slab_indicators(mesh, eta2), slab_min_phi(mesh, phi),
                           theta, h_band, phi_band)
    return split_intervals(mesh.coords, marks), marks


def transfer(mesh: Mesh, field: np.ndarray, coords_new: Sequence[np.ndarray]) -> np.ndarray:
    """Q1 interpolation of a nodal field (n_nodes,) or (n_nodes, m) onto the nodes of a new mesh.

    New nodes must lie inside the old mesh's box.  Each new coordinate finds the
    old interval that holds it (the last one whose left end is <= it) and its
    local coordinate t; the value is the sum over the 2^d corners of the old
    cell of prod(t or 1 - t) times the corner value.
    """
    f = np.asarray(field, dtype=np.float64)
    vec = f.ndim == 2
    F = f.reshape(mesh.n_nodes, -1)
    d = mesh.d
    cell, t = [], []
    for a in range(d):
        x = mesh.coords[a]
        xn = np.asarray(coords_new[a], dtype=np.float64)
        if xn[0] < x[0] or xn[-1] > x[-1]:
            raise ValueError("new mesh leaves the old mesh's box")
        i = np.clip(np.searchsorted(x, xn, side="right") - 1, 0, len(x) - 2)
        cell.append(i)
        t.append((xn - x[i]) / (x[i + 1] - x[i]))
    new_mesh = Mesh(coords_new)
    idx = new_mesh.node_index()
    out = np.zeros((new_mesh.n_nodes, F.shape[1]))
    for corner in range(2 ** d):
        off = [(corner >> l) & 1 for l in range(d)]
        w = np.ones(new_mesh.n_nodes)
        src = [cell[a][idx[a]] + off[a] for a in range(d)]
        for a in range(d):
            ta = t[a][idx[a]]
            w = w * (ta if off[a] else 1.0 - ta)
        out += w[:, None] * F[mesh.node_id(*src)]
    return out if vec else out[:, 0]
