"""Pins of the oracle's Newton / primal-dual active-set loop (Section 3 algorithm).

* The block forward substitution equals a dense LU solve of the reduced system.
* The converged point satisfies the KKT conditions of the discrete VI
  (Formulation 1 with phi <= phi_old), independent of how it was reached.
* A different algorithm -- staggered minimization with a projected
  Gauss-Seidel solve of the bound-constrained phase-field QP -- reaches the
  same point on a small mesh.
* Path-only options (full Jacobian with M_u_phi, another c) reach the same point.
* The Sneddon configuration is symmetric: u_x odd in x, u_y odd in y, phi even.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fe, model, pdas
import workloads as W


def _setup(n_cells, **kw):
    w = W.scaled_workload(W.config(0), n_cells)
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
    for k, v in kw.items():
        setattr(prm, k, v)
    return w, mesh, prm


def test_block_substitution_equals_dense_solve():
    for dim, n in ((2, 4), (2, 8), (3, 4)):
        ax = W.uniform_axis(n, -1.0, 1.0)
        mesh = fe.Mesh([ax] * dim)
        rng = np.random.default_rng(n + dim)
        nn = mesh.n_nodes
        prm = model.Params(eps=0.5, p=0.1, kappa=1e-6)
        u = 0.01 * rng.standard_normal((nn, dim))
        phi = rng.uniform(0.3, 1.0, nn)
        J = model.jacobian(mesh, prm, u, phi, rng.random(nn))
        free = np.ones(J.shape[0], dtype=bool)
        free[: dim * nn] = ~np.repeat(mesh.boundary_nodes(), dim)
        free[dim * nn:][rng.random(nn) < 0.3] = False
        rhs = rng.standard_normal(J.shape[0])
        x = pdas._solve_reduced(J, rhs, free, dim * nn, False)
        idx = np.flatnonzero(free)
        dense = np.linalg.solve(J.toarray()[np.ix_(idx, idx)], rhs[idx])
        assert np.allclose(x[idx], dense, rtol=1e-12, atol=1e-13 * np.max(np.abs(dense)))
        assert np.all(x[~free] == 0.0)


@pytest.fixture(scope="module")
def solved32():
    w, mesh, prm = _setup(32)
    st = pdas.State.initial(mesh, prm, w.phi0())
    rep = pdas.loading_step(st, w.pressures[0])
    return w, mesh, prm, st, rep


def test_kkt_conditions_at_converged_point(solved32):
    w, mesh, prm, st, rep = solved32
    assert rep.converged and rep.locked == 0
    d, n = mesh.d, mesh.n_nodes
    # phi~ of the first loading step is the initial phase field, kept as phi_prev afterwards
    r_u, r_phi = model.gradient(mesh, prm, st.u, st.phi, st.phi_prev)
    S = model.scaling(mesh, prm, st.phi_prev)
    m = model.lumped_mass(mesh)
    free_u = ~np.repeat(mesh.boundary_nodes(), d)
    ref = rep.rho0
    assert np.max(np.abs(r_u.ravel()[free_u] / S[: d * n][free_u])) <= 1e-10 * ref
    A = st.active
    assert np.all(st.phi <= st.phi_prev + 1e-15)              # phi <= phi_old
    assert np.all(st.phi[A] == st.phi_prev[A])                # active: constraint holds exactly
    lam = -r_phi / m
    assert np.all(lam[A] > 0)                                 # multiplier >= 0 on the active set
    assert np.max(np.abs(r_phi[~A] / S[d * n:][~A])) <= 1e-10 * ref   # stationarity on the rest
    assert np.all(st.phi_prev[~A] - st.phi[~A] >= 0)


def _staggered_reference(mesh, prm, phi0, sweeps=20000, outer=60):
    """Alternating minimization: exact u-solve, then the bound-constrained phi QP
    by projected Gauss-Seidel; phi~ = phi0 (first loading step)."""
    d, n = mesh.d, mesh.n_nodes
    free_u = np.flatnonzero(~np.repeat(mesh.boundary_nodes(), d))
    u = np.zeros((n, d))
    phi = phi0.copy()
    for _ in range(outer):
        Muu, _, _ = model.jacobian_blocks(mesh, prm, u, phi, phi0)
        r0, _ = model.gradient(mesh, prm, np.zeros((n, d)), phi, phi0)   # r_u is affine in u
        x = np.zeros(d * n)
        x[free_u] = spla.spsolve(Muu[free_u][:, free_u].tocsc(), -r0.ravel()[free_u])
        u_new = x.reshape(n, d)
        _, _, H = model.jacobian_blocks(mesh, prm, u_new, phi, phi0)     # phi-Hessian at fixed u
        H = H.tocsr()
        _, rphi = model.gradient(mesh, prm, u_new, phi, phi0)
        b = H @ phi - rphi                                               # r_phi = H phi - b
        p = phi.copy()
        diag = H.diagonal()
        for _s in range(sweeps):
            old = p.copy()
            for i in range(n):
                row = slice(H.indptr[i], H.indptr[i + 1])
                ri = H.data[row] @ p[H.indices[row]] - b[i]
                p[i] = min(phi0[i], p[i] - ri / diag[i])
            if np.max(np.abs(p - old)) < 1e-16:
                break
        change = max(np.max(np.abs(u_new - u)) / max(np.max(np.abs(u_new)), 1e-300),
                     np.max(np.abs(p - phi)))
        u, phi = u_new, p
        if change < 1e-14:
            break
    return u, phi


def test_staggered_projected_gauss_seidel_reaches_same_point():
    w, mesh, prm = _setup(8)
    phi0 = w.phi0()
    st = pdas.State.initial(mesh, prm, phi0)
    rep = pdas.loading_step(st, prm.p)
    assert rep.converged
    u_ref, phi_ref = _staggered_reference(mesh, prm, phi0)
    assert np.linalg.norm(st.u - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    assert np.linalg.norm(st.phi - phi_ref) <= 1e-9 * np.linalg.norm(phi_ref)


def test_path_options_reach_same_point(solved32):
    w, mesh, prm, st, rep = solved32
    for opts in (pdas.Options(full_jacobian=True), pdas.Options(c=0.02)):
        st2 = pdas.State.initial(mesh, prm, w.phi0())
        rep2 = pdas.loading_step(st2, w.pressures[0], opts)
        assert rep2.converged
        assert np.linalg.norm(st2.u - st.u) <= 1e-9 * np.linalg.norm(st.u)
        assert np.linalg.norm(st2.phi - st.phi) <= 1e-9 * np.linalg.norm(st.phi)
        assert np.array_equal(st2.active, st.active)


def test_sneddon_symmetry(solved32):
    w, mesh, prm, st, rep = solved32
    nx, ny = mesh.nn
    u = st.u.reshape(ny, nx, 2)
    phi = st.phi.reshape(ny, nx)
    s = np.max(np.abs(u))
    assert np.max(np.abs(u[:, ::-1, 0] + u[:, :, 0])) <= 1e-10 * s     # u_x odd in x
    assert np.max(np.abs(u[::-1, :, 1] + u[:, :, 1])) <= 1e-10 * s     # u_y odd in y
    assert np.max(np.abs(u[::-1, :, 0] - u[:, :, 0])) <= 1e-10 * s     # u_x even in y
    assert np.max(np.abs(phi[::-1, :] - phi)) <= 1e-12
    assert np.max(np.abs(phi[:, ::-1] - phi)) <= 1e-12
    # the crack opens: u_y > 0 just above the crack centre
    ic, jc = nx // 2, ny // 2
    assert u[jc + 2, ic, 1] > 0 and u[jc - 2, ic, 1] < 0


def test_two_loading_steps_irreversible_and_extrapolated():
    w, mesh, prm = _setup(32)
    phi0 = w.phi0()
    st = pdas.State.initial(mesh, prm, phi0)
    r1 = pdas.loading_step(st, 5e-4)
    phi1 = st.phi.copy()
    np.testing.assert_array_equal(st.phi_old, phi1)
    np.testing.assert_array_equal(st.phi_prev, phi0)
    # the initial crack field is not a computed time level: no extrapolation yet
    np.testing.assert_array_equal(st.phi_tilde(), phi1)
    r2 = pdas.loading_step(st, 1e-3)
    phi2 = st.phi.copy()
    np.testing.assert_array_equal(st.phi_tilde(), np.clip(2 * phi2 - phi1, 0.0, 1.0))
    r3 = pdas.loading_step(st, 1.5e-3)
    assert r1.converged and r2.converged and r3.converged
    assert np.all(phi2 <= phi1 + 1e-15) and np.all(st.phi <= phi2 + 1e-15)   # phi <= phi_old
    # the opening grows with the pressure and stays bounded (no kappa-only region is loaded)
    assert np.max(np.abs(st.u)) < 10 * 1.5e-3
