"""Pins of the oracle's residual and Jacobian (Formulation 1, Section 3.1 blocks).

* The energy is checked in closed form on constant fields.
* Formulation 1 is the Euler-Lagrange system of that energy (with phi~ in the
  elastic degradation of the displacement equation): the residual must equal
  central finite differences of the energy.  This ties the factors and signs
  of Eq. (E22ATW) and Eq. (E33ATW) to each other.
* The Jacobian blocks must equal central finite differences of the residual
  (M_u_phi is the one block the paper drops; it must equal the FD block when
  full_jacobian is requested).
"""
import numpy as np
import pytest

from oracle import fe, model
import workloads as W


def _small_mesh(dim, seed=0):
    rng = np.random.default_rng(seed)
    coords = [np.cumsum(np.r_[0.0, rng.uniform(0.3, 1.0, 3 if dim == 3 else 4)]) for _ in range(dim)]
    return fe.Mesh(coords), rng


def _random_state(mesh, rng, u_scale=0.05):
    n, d = mesh.n_nodes, mesh.d
    u = u_scale * rng.standard_normal((n, d))
    phi = rng.uniform(0.2, 1.0, n)
    phit = rng.uniform(0.0, 1.0, n)
    return u, phi, phit


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_constant_fields_closed_form(dim):
    mesh, rng = _small_mesh(dim)
    n = mesh.n_nodes
    vol = np.prod([c[-1] - c[0] for c in mesh.coords])
    prm = model.Params(E=1.7, nu=0.3, Gc=1.3, kappa=1e-3, eps=0.2, p=0.05)
    Bm = rng.standard_normal((dim, dim)) * 0.1
    u = mesh.node_xyz() @ Bm.T
    c_phi = 0.6
    phi = np.full(n, c_phi)
    mu, lam = prm.mu_lam
    e = 0.5 * (Bm + Bm.T)
    sige = 2 * mu * np.sum(e * e) + lam * np.trace(e) ** 2
    g = (1 - prm.kappa) * c_phi ** 2 + prm.kappa
    expect = vol * (0.5 * g * sige + c_phi ** 2 * prm.p * np.trace(Bm)
                    + 0.5 * prm.Gc * (1 - c_phi) ** 2 / prm.eps)
    assert model.energy(mesh, prm, u, phi, phi) == pytest.approx(expect, rel=1e-13)
    # gradient part of the crack energy: phi = x -> G_c eps / 2 * vol
    phi_x = mesh.node_xyz()[:, 0]
    e_x = model.energy(mesh, model.Params(Gc=2.0, eps=0.3, p=0.0), np.zeros((n, dim)), phi_x, phi_x)
    ref = 0.5 * 2.0 * (1.0 / 0.3) * float(np.sum(
        model.phase_field_matrices(mesh)[0] @ (1 - phi_x) * (1 - phi_x)))
    assert e_x == pytest.approx(ref + 0.5 * 2.0 * 0.3 * vol, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_residual_is_energy_gradient(dim):
    mesh, rng = _small_mesh(dim, 3)
    n = mesh.n_nodes
    prm = model.Params(E=1.0, nu=0.2, Gc=1.0, kappa=1e-2, eps=0.25, p=0.3)
    u, phi, phit = _random_state(mesh, rng)
    h = 1e-6
    # phase-field rows: degradation of the energy evaluated with phi itself
    r_u, r_phi = model.gradient(mesh, prm, u, phi, phi)
    for i in rng.choice(n, 6, replace=False):
        dp = np.zeros(n); dp[i] = h
        fd = (model.energy(mesh, prm, u, phi + dp, phi + dp)
              - model.energy(mesh, prm, u, phi - dp, phi - dp)) / (2 * h)
        assert r_phi[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # displacement rows: degradation with phi~ (fixed), the residual uses phi~
    r_u, _ = model.gradient(mesh, prm, u, phi, phit)
    for i in rng.choice(n, 6, replace=False):
        for m in range(dim):
            du = np.zeros((n, dim)); du[i, m] = h
            fd = (model.energy(mesh, prm, u + du, phi, phit)
                  - model.energy(mesh, prm, u - du, phi, phit)) / (2 * h)
            assert r_u[i, m] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_blocks_match_finite_differences(dim):
    mesh, rng = _small_mesh(dim, 5)
    n, d = mesh.n_nodes, dim
    prm = model.Params(E=1.0, nu=0.2, Gc=1.0, kappa=1e-2, eps=0.25, p=0.3)
    u, phi, phit = _random_state(mesh, rng)
    Muu, Mpu, Mpp, Mup = model.jacobian_blocks(mesh, prm, u, phi, phit, full_jacobian=True)
    J = model.jacobian(mesh, prm, u, phi, phit)
    Jfull = model.jacobian(mesh, prm, u, phi, phit, full_jacobian=True)
    h = 1e-6

    def R(uu, pp):
        a, b = model.gradient(mesh, prm, uu, pp, phit)
        return np.concatenate([a.ravel(), b])

    cols = list(rng.choice(d * n, 5, replace=False)) + list(d * n + rng.choice(n, 5, replace=False))
    for c in cols:
        e = np.zeros(d * n + n); e[c] = h
        up, pp = u + e[:d * n].reshape(n, d), phi + e[d * n:]
        um, pm = u - e[:d * n].reshape(n, d), phi - e[d * n:]
        fd = (R(up, pp) - R(um, pm)) / (2 * h)
        col_full = Jfull[:, c].toarray().ravel()
        assert np.allclose(col_full, fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)))
        col = J[:, c].toarray().ravel()
        if c >= d * n:   # the paper's Jacobian drops exactly the M_u_phi block
            assert np.all(col[:d * n] == 0.0)
            assert np.allclose(col[d * n:], fd[d * n:], rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)))
        else:
            assert np.array_equal(col, col_full)
    # M_uu is symmetric and positive definite once the boundary is clamped
    K = Muu.toarray()
    assert np.allclose(K, K.T, rtol=0, atol=1e-14 * np.abs(K).max())
    free = ~np.repeat(mesh.boundary_nodes(), d)
    np.linalg.cholesky(K[np.ix_(free, free)])


def test_pressure_pushes_crack_faces_apart():
    """With u = 0 the displacement residual is the pressure load -(phi^2 p, div w):
    F_u = -r_u points away from the crack band (sign of Eq. E22ATW)."""
    w = W.scaled_workload(W.config(0), 32)
    mesh = fe.Mesh(w.coords)
    n = mesh.n_nodes
    prm = model.Params(eps=w.eps, p=1e-3)
    phi = w.phi0()
    r_u, _ = model.gradient(mesh, prm, np.zeros((n, 2)), phi, phi)
    F = -r_u
    xyz = mesh.node_xyz()
    near = (np.abs(xyz[:, 0]) < 0.2) & (np.abs(xyz[:, 1]) > 0.05) & (np.abs(xyz[:, 1]) < 0.3)
    assert np.all(np.sign(F[near & (F[:, 1] != 0), 1]) == np.sign(xyz[near & (F[:, 1] != 0), 1]))
    assert np.count_nonzero(F[near, 1]) > 4
