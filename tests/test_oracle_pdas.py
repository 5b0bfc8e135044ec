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


# ---------------------------------------------------------------- cycle rule --
def _cyclic_case(n_cells, p):
    w = W.cyclic_loading(n_cells)
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p)
    return w, mesh, prm


def test_cycle_lock_replays_the_unlocked_iteration():
    """Section 3: indices whose active-set membership alternates are locked active.

    Reading: an index is locked once its raw membership (indicator > tau) has
    changed ``cycle_lock`` times within the loading step.  Until the first
    lock the locked run must repeat the unlocked run exactly; the lock must
    fire at the first iteration where the toggle counts -- counted here by
    hand from the unlocked run's raw sets -- reach the limit, on exactly those
    indices; a locked index never unlocks and stays in A_k; and the converged
    point satisfies the complementarity conditions on every index the rule
    did not lock.  The case (low G_c, pressure near critical) alternates."""
    L = 2
    w, mesh, prm = _cyclic_case(24, 5e-3)
    st_free = pdas.State.initial(mesh, prm, w.phi0())
    rep_free = pdas.loading_step(st_free, prm.p, pdas.Options(cycle_lock=10 ** 9, trace=True))
    st = pdas.State.initial(mesh, prm, w.phi0())
    rep = pdas.loading_step(st, prm.p, pdas.Options(cycle_lock=L, trace=True))
    raws = [t[0] for t in rep_free.trace]
    counts = np.zeros(mesh.n_nodes, dtype=np.int64)
    t_star = None
    for k in range(1, len(raws)):
        counts += raws[k] != raws[k - 1]
        if np.any(counts >= L):
            t_star = k
            break
    assert t_star is not None, "the case must alternate"
    for k in range(t_star + 1):
        assert np.array_equal(rep.trace[k][0], raws[k])
    for k in range(t_star):
        assert not rep.trace[k][1].any()
    assert np.array_equal(rep.trace[t_star][1], counts >= L)
    for k in range(t_star, len(rep.trace)):
        raw, lk, A = rep.trace[k]
        assert np.array_equal(A, raw | lk)
        if k > t_star:
            assert np.all(lk[rep.trace[k - 1][1]])          # locks persist
    locked = rep.trace[-1][1]
    assert rep.converged and rep.locked == int(locked.sum()) > 0
    # complementarity at the converged point
    d, n = mesh.d, mesh.n_nodes
    phit = st.phi_prev                                       # first step: phi~ = phi_old
    r_u, r_phi = model.gradient(mesh, prm, st.u, st.phi, phit)
    S = model.scaling(mesh, prm, phit)
    m = model.lumped_mass(mesh)
    A = st.active
    free_u = ~np.repeat(mesh.boundary_nodes(), d)
    assert np.max(np.abs(r_u.ravel()[free_u] / S[: d * n][free_u])) <= 1e-10 * rep.rho0
    assert np.all(A[locked]) and np.all(st.phi[A] == st.phi_prev[A])
    lam = -r_phi / m
    tau = pdas.active_threshold(prm, pdas.Options())
    assert np.all(lam[A & ~locked] > tau)                    # multiplier positive where not locked
    assert np.max(np.abs(r_phi[~A] / S[d * n:][~A])) <= 1e-10 * rep.rho0


def test_phi_tilde_is_exact_on_linear_histories():
    """Formulation 1: phi~ is the linear extrapolation in time of the two
    previous levels.  A history that is linear in time, phi(t) = a + b t with
    phi_prev = phi(0), phi_old = phi(1), must give phi(2) wherever that value
    lies in [0, 1]; only outside [0, 1] may the clamp act, and then it returns
    the nearer bound.  A constant history extrapolates to itself, and before
    two computed time levels exist (steps 1, 2) phi~ = phi_old."""
    rng = np.random.default_rng(7)
    n = 4000
    a = rng.uniform(0.3, 0.7, n)
    b = rng.uniform(-0.3, 0.3, n)
    b[:50] = 0.0
    st = pdas.State(mesh=None, prm=None, u=None, phi=a + b, phi_old=a + b, phi_prev=a,
                    steps_done=2)
    pred = a + 2.0 * b
    got = st.phi_tilde()
    inside = (pred >= 0.0) & (pred <= 1.0)
    assert inside.sum() > n // 2 and (~inside).sum() > 100
    np.testing.assert_allclose(got[inside], pred[inside], rtol=0, atol=4e-16)
    assert np.all(got[pred < 0.0] == 0.0) and np.all(got[pred > 1.0] == 1.0)
    np.testing.assert_allclose(got[:50], a[:50], rtol=0, atol=4e-16)
    for done in (0, 1):
        st.steps_done = done
        assert np.array_equal(st.phi_tilde(), st.phi_old)


@pytest.mark.parametrize("which", ["sneddon64", "cyclic24"])
def test_irreversibility_slack_is_bounded_by_tau_over_c(which):
    """phi <= phi_old (Formulation 1) holds up to tau / c on the inactive set.

    The active-set rule with threshold tau > 0 leaves a node free while
    lambda_i + c (phi_i - phi_old,i) <= tau, and at a converged point the free
    rows are stationary (lambda_i ~ 0), so a free node can exceed phi_old by
    up to (tau - lambda_i) / c ~ tau / c = 1e-9 (c = 0.1 G_c/eps, tau = 1e-10
    G_c/eps); active nodes meet the constraint exactly.  Checked over every
    step of a load / unload / reload cycle and on the Sneddon step, where the
    slack is attained in part (far-field nodes with phi_old = 1)."""
    if which == "sneddon64":
        w = W.scaled_workload(W.config(0), 64)
    else:
        w = W.cyclic_loading(24)
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    o = pdas.Options()
    tau, c = pdas.active_threshold(prm, o), pdas.active_constant(prm, o)
    worst = -np.inf
    for p in w.pressures:
        rep = pdas.loading_step(st, p, o)
        assert rep.converged
        free = ~st.active
        lam = st.indicator - c * (st.phi - st.phi_prev)
        assert np.max(np.abs(lam[free])) <= 1e-3 * tau
        exc = st.phi - st.phi_prev
        assert np.all(exc[st.active] == 0.0)
        assert np.max(exc[free]) <= (tau + np.max(np.abs(lam[free]))) / c
        worst = max(worst, float(np.max(exc[free])))
    if which == "sneddon64":
        assert worst > 0.1 * tau / c       # the slack is real, not vacuous
