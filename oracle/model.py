"""Formulation 1 of the paper, discretized with Q1 elements (oracle; test infrastructure only).

Everything here is FP64 numpy/scipy, vectorized over cells but otherwise the
plain definition: interpolate nodal fields to the 2^d Gauss points of each
cell, evaluate the integrands of Eq. (E22ATW) / (E33ATW) and of the Jacobian
blocks of Section 3.1, integrate, and scatter-add into global vectors /
sparse matrices.

Conventions (readings of the paper where it is silent or inconsistent):

* ``gradient`` returns r(U), the left-hand sides of Eq. (E22ATW) and
  (E33ATW) tested with each basis function (r = grad E).  The Newton
  right-hand side is F = -r (commented algorithm of Section 3, step 3).
* Coefficients at quadrature points use the interpolated nodal phi, phi~,
  which are then squared (phi^2 is not interpolated).
* The elastic degradation uses phi~ ((1-kappa) phi~^2 + kappa); the pressure
  term of Eq. (E22ATW) uses phi^2 as printed.
* The symbol alpha in M_phi_u and M_phi_phi is never defined in the paper;
  consistency with the derivative of 2(phi p div u, psi) in Eq. (E33ATW)
  requires -2(alpha - 1) = 2, i.e. the coefficient 2p.
* The extra "+ (sigma(chi_j), e(chi_i))" printed in M_uu is not the
  derivative of Eq. (E22ATW) and is omitted; M_u_phi = 0 as the paper states
  (the pressure coupling is dropped from the Jacobian, not from the residual).
  ``full_jacobian=True`` adds M_u_phi = 2 (phi p chi_j, div chi_i^u).

Global DoF order (Section 3.1, basis psi_i): all displacement DoFs first,
node-major with interleaved components (dof = node*d + m), then the phase
field (dof = d*n_nodes + node).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .fe import Mesh, cell_geometry, lame


@dataclass
class Params:
    """Material and loading of Formulation 1 (Section 2) and Section 4."""
    E: float = 1.0
    nu: float = 0.2
    Gc: float = 1.0
    kappa: float = 1e-10
    eps: float = 0.0625
    p: float = 1e-3

    @property
    def mu_lam(self):
        return lame(self.E, self.nu)


def _scatter(n: int, idx: np.ndarray, vals: np.ndarray) -> np.ndarray:
    return np.bincount(idx.reshape(-1), weights=vals.reshape(-1), minlength=n)


def qp_fields(mesh: Mesh, prm: Params, u, phi, phit, cells=None):
    """Quadrature-point values of the state on the given cells.

    Returns a dict with N, dN, JxW, cell nodes cn and, per (cell, q):
    grad_u[m, l] = du_m/dx_l, strain e, div u, stress sigma, sigma:e,
    phi, phi~, grad phi and the degradation g = (1-kappa) phi~^2 + kappa.
    """
    d = mesh.d
    mu, lam = prm.mu_lam
    N, dN, JxW = cell_geometry(mesh, cells)
    cn = mesh.cell_nodes(cells)
    ue = u[cn]                                          # (C, a, m)
    G = np.einsum("cqal,cam->cqml", dN, ue)             # du_m / dx_l
    e = 0.5 * (G + np.swapaxes(G, 2, 3))
    div = np.trace(G, axis1=2, axis2=3)
    I = np.eye(d)
    sig = 2.0 * mu * e + lam * div[:, :, None, None] * I
    sige = np.einsum("cqml,cqml->cq", sig, e)
    ph = np.einsum("qa,ca->cq", N, phi[cn])
    pht = np.einsum("qa,ca->cq", N, phit[cn])
    gph = np.einsum("cqal,ca->cql", dN, phi[cn])
    g = (1.0 - prm.kappa) * pht ** 2 + prm.kappa
    return dict(N=N, dN=dN, JxW=JxW, cn=cn, G=G, e=e, div=div, sig=sig, sige=sige,
                phi=ph, phit=pht, gphi=gph, g=g)


def gradient(mesh: Mesh, prm: Params, u, phi, phit, cells=None):
    """r(U): Eq. (E22ATW) tested with chi_i^u and Eq. (E33ATW) with chi_i^phi.

    r_u[i, m] = (g(phi~) sigma(u), e(chi_i e_m)) + (phi^2 p, div(chi_i e_m))
    r_phi[i]  = (1-kappa)(phi sigma(u):e(u), chi_i) + 2(phi p div u, chi_i)
                - G_c/eps (1 - phi, chi_i) + G_c eps (grad phi, grad chi_i)
    (Section 2, Formulation 1, with psi - phi -> chi_i.)
    Only the given cells contribute (all cells by default).
    """
    d, n = mesh.d, mesh.n_nodes
    f = qp_fields(mesh, prm, u, phi, phit, cells)
    dN, JxW, N, cn = f["dN"], f["JxW"], f["N"], f["cn"]
    # displacement rows
    t = f["g"][:, :, None, None] * f["sig"]                       # (C,q,m,l)
    ru_e = np.einsum("cq,cqml,cqal->cam", JxW, t, dN)
    ru_e += np.einsum("cq,cq,cqam->cam", JxW, f["phi"] ** 2 * prm.p, dN)
    r_u = np.stack([_scatter(n, cn, ru_e[:, :, m]) for m in range(d)], axis=1)
    # phase-field rows
    k = prm.kappa
    coef = ((1.0 - k) * f["phi"] * f["sige"] + 2.0 * f["phi"] * prm.p * f["div"]
            - prm.Gc / prm.eps * (1.0 - f["phi"]))
    rp_e = np.einsum("cq,cq,qa->ca", JxW, coef, N)
    rp_e += prm.Gc * prm.eps * np.einsum("cq,cql,cqal->ca", JxW, f["gphi"], dN)
    r_phi = _scatter(n, cn, rp_e)
    return r_u, r_phi


def energy(mesh: Mesh, prm: Params, u, phi, degr_field):
    """E(u, phi) = int 1/2 g sigma(u):e(u) + phi^2 p div u + G_c/2 ((1-phi)^2/eps + eps |grad phi|^2).

    ``degr_field`` is the nodal field whose interpolant enters g = (1-kappa)(.)^2
    + kappa.  With degr_field = phi~ its u-gradient is r_u; with
    degr_field = phi its phi-gradient is r_phi (Formulation 1 is the
    Euler-Lagrange system of this energy, Section 2).
    """
    f = qp_fields(mesh, prm, u, phi, degr_field)
    dens = (0.5 * f["g"] * f["sige"] + f["phi"] ** 2 * prm.p * f["div"]
            + 0.5 * prm.Gc * ((1.0 - f["phi"]) ** 2 / prm.eps
                              + prm.eps * np.sum(f["gphi"] ** 2, axis=2)))
    return float(np.sum(f["JxW"] * dens))


def jacobian_blocks(mesh: Mesh, prm: Params, u, phi, phit, cells=None, full_jacobian=False):
    """Sparse blocks (M_uu, M_phi_u, M_phi_phi[, M_u_phi]) of Section 3.1.

    (M_uu)_ij     = (g(phi~) sigma(chi_j^u), e(chi_i^u))
    (M_phi_u)_ij  = 2(1-kappa)(phi sigma(chi_j^u):e(u), chi_i^phi) + 2p(phi div chi_j^u, chi_i^phi)
    (M_phi_phi)_ij = (1-kappa)(sigma(u):e(u) chi_j, chi_i) + 2p(div u chi_j, chi_i)
                     + G_c(1/eps (chi_j, chi_i) + eps (grad chi_j, grad chi_i))
    (M_u_phi)_ij  = 2p(phi chi_j^phi, div chi_i^u)   [only with full_jacobian]
    Rows/cols are unreduced (no Dirichlet or active-set elimination).
    """
    d, n = mesh.d, mesh.n_nodes
    mu, lam = prm.mu_lam
    k = prm.kappa
    f = qp_fields(mesh, prm, u, phi, phit, cells)
    dN, JxW, N, cn = f["dN"], f["JxW"], f["N"], f["cn"]
    C, na = cn.shape
    I = np.eye(d)
    wg = JxW * f["g"]
    gradgrad = np.einsum("cqal,cqbl->cqab", dN, dN)
    # M_uu: g [ mu (delta_mn gradNa.gradNb + d_n Na d_m Nb) + lam d_m Na d_n Nb ]
    Kuu = (mu * np.einsum("cq,cqab,mn->cambn", wg, gradgrad, I)
           + mu * np.einsum("cq,cqan,cqbm->cambn", wg, dN, dN)
           + lam * np.einsum("cq,cqam,cqbn->cambn", wg, dN, dN))
    rows = (cn[:, :, None, None, None] * d + np.arange(d)[None, None, :, None, None])
    cols = (cn[:, None, None, :, None] * d + np.arange(d)[None, None, None, None, :])
    rows, cols = np.broadcast_to(rows, Kuu.shape), np.broadcast_to(cols, Kuu.shape)
    Muu = sp.csr_matrix((Kuu.ravel(), (rows.ravel(), cols.ravel())), shape=(d * n, d * n))
    # M_phi_u: N_a [ 2(1-kappa) phi sigma(u)[n,l] d_l Nb + 2 p phi d_n Nb ]
    sdn = np.einsum("cqnl,cqbl->cqbn", f["sig"], dN)              # sigma(u):e(N_b e_n)
    Kpu = np.einsum("cq,qa,cqbn->cabn", JxW * 2.0 * (1.0 - k) * f["phi"], N, sdn)
    Kpu += np.einsum("cq,qa,cqbn->cabn", JxW * 2.0 * prm.p * f["phi"], N, dN)
    rows = np.broadcast_to(cn[:, :, None, None], Kpu.shape)
    cols = np.broadcast_to(cn[:, None, :, None] * d + np.arange(d)[None, None, None, :], Kpu.shape)
    Mpu = sp.csr_matrix((Kpu.ravel(), (rows.ravel(), cols.ravel())), shape=(n, d * n))
    # M_phi_phi
    c0 = (1.0 - k) * f["sige"] + 2.0 * prm.p * f["div"] + prm.Gc / prm.eps
    Kpp = np.einsum("cq,qa,qb->cab", JxW * c0, N, N)
    Kpp += prm.Gc * prm.eps * np.einsum("cq,cqab->cab", JxW, gradgrad)
    rows = np.broadcast_to(cn[:, :, None], Kpp.shape)
    cols = np.broadcast_to(cn[:, None, :], Kpp.shape)
    Mpp = sp.csr_matrix((Kpp.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n))
    if not full_jacobian:
        return Muu, Mpu, Mpp
    Kup = np.einsum("cq,qb,cqam->camb", JxW * 2.0 * prm.p * f["phi"], N, dN)
    rows = np.broadcast_to(cn[:, :, None, None] * d + np.arange(d)[None, None, :, None], Kup.shape)
    cols = np.broadcast_to(cn[:, None, None, :], Kup.shape)
    Mup = sp.csr_matrix((Kup.ravel(), (rows.ravel(), cols.ravel())), shape=(d * n, n))
    return Muu, Mpu, Mpp, Mup


def jacobian(mesh: Mesh, prm: Params, u, phi, phit, cells=None, full_jacobian=False):
    """Full (unreduced) Jacobian G = [[M_uu, M_u_phi], [M_phi_u, M_phi_phi]] as CSR."""
    blocks = jacobian_blocks(mesh, prm, u, phi, phit, cells, full_jacobian)
    Muu, Mpu, Mpp = blocks[:3]
    Mup = blocks[3] if full_jacobian else None
    return sp.bmat([[Muu, Mup], [Mpu, Mpp]], format="csr")


def phase_field_matrices(mesh: Mesh, cells=None):
    """Consistent mass (chi_j, chi_i) and stiffness (grad chi_j, grad chi_i) of the Q1 space."""
    n = mesh.n_nodes
    N, dN, JxW = cell_geometry(mesh, cells)
    cn = mesh.cell_nodes(cells)
    Me = np.einsum("cq,qa,qb->cab", JxW, N, N)
    Ke = np.einsum("cq,cqal,cqbl->cab", JxW, dN, dN)
    rows = np.broadcast_to(cn[:, :, None], Me.shape).ravel()
    cols = np.broadcast_to(cn[:, None, :], Me.shape).ravel()
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    return M, K


def lumped_mass(mesh: Mesh) -> np.ndarray:
    """m_i = sum_j (chi_j, chi_i) = (1, chi_i): the diagonal "B" of the active-set rule."""
    N, dN, JxW = cell_geometry(mesh)
    cn = mesh.cell_nodes()
    return _scatter(mesh.n_nodes, cn, np.einsum("cq,qa->ca", JxW, N))


def scaling(mesh: Mesh, prm: Params, phit) -> np.ndarray:
    """Fixed Jacobi scaling S used for reduced-residual norms within one loading step.

    S_u = diag(M_uu(phi~)) (depends only on phi~, fixed during a loading step),
    S_phi = diag(G_c (M/eps + eps K)); Dirichlet displacement DoFs get 1.
    """
    d, n = mesh.d, mesh.n_nodes
    z = np.zeros((n, d))
    Muu, _, _ = jacobian_blocks(mesh, prm, z, np.ones(n), phit)
    M, K = phase_field_matrices(mesh)
    s = np.concatenate([Muu.diagonal(), prm.Gc * (M.diagonal() / prm.eps + prm.eps * K.diagonal())])
    bnd = mesh.boundary_nodes()
    s[: d * n].reshape(n, d)[bnd] = 1.0
    return s
