"""Pins of the oracle's refinement strategy (oracle/adapt.py; Section 3).

The indicator is pinned by closed forms: fields whose Q1 interpolant has a
continuous gradient give zero, and fields with a known kink give the
hand-integrated jump on the cells beside it (with the cell diameter, the 1/24
factor and the face area written out).  Slab sums and minima are checked by
brute-force loops, marking by hand-made cases, and the transfer by exactness
on multilinear functions and the old nodes.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import adapt, fe


def _mesh(d, seed=0, n=(5, 4, 3)):
    rng = np.random.default_rng(seed)
    coords = [np.cumsum(np.concatenate([[-1.0], rng.uniform(0.2, 1.0, n[a])])) for a in range(d)]
    return fe.Mesh(coords)


@pytest.mark.parametrize("d", [2, 3])
def test_indicator_vanishes_for_continuous_gradients(d):
    # affine and multilinear fields are Q1 on every cell with a continuous gradient
    m = _mesh(d, 1)
    X = m.node_xyz()
    rng = np.random.default_rng(2)
    A = rng.normal(size=(d, d))
    u_aff = X @ A.T + rng.normal(size=d)
    assert np.max(np.abs(adapt.cell_indicators(m, u_aff))) < 1e-26
    u_bil = np.zeros((m.n_nodes, d))
    u_bil[:, 0] = X[:, 0] * X[:, 1]
    u_bil[:, d - 1] = np.prod(X, axis=1)
    assert np.max(np.abs(adapt.cell_indicators(m, u_bil))) < 1e-24


def test_indicator_of_a_kink_2d():
    # u_0 = |x - x_k|: the x-derivative jumps by 2 across the mesh line x = x_k
    m = _mesh(2, 3)
    k = 2
    xk = m.coords[0][k]
    X = m.node_xyz()
    u = np.zeros((m.n_nodes, 2))
    u[:, 0] = np.abs(X[:, 0] - xk)
    eta2 = adapt.cell_indicators(m, u)
    ci = m.cell_index()
    h = m.cell_h()
    expect = np.zeros(m.n_cells)
    beside = (ci[0] == k - 1) | (ci[0] == k)
    diam = np.sqrt(h[:, 0] ** 2 + h[:, 1] ** 2)
    expect[beside] = diam[beside] / 24.0 * 4.0 * h[beside, 1]
    np.testing.assert_allclose(eta2, expect, rtol=1e-13, atol=1e-30)


def test_indicator_of_a_jump_varying_along_the_face_2d():
    # u_1 = |x - x_k| * y: the jump 2y varies linearly along each face; its
    # squared integral over [y0, y1] is 4 (y1^3 - y0^3) / 3
    m = _mesh(2, 4)
    k = 3
    xk = m.coords[0][k]
    X = m.node_xyz()
    u = np.zeros((m.n_nodes, 2))
    u[:, 1] = np.abs(X[:, 0] - xk) * X[:, 1]
    eta2 = adapt.cell_indicators(m, u)
    ci = m.cell_index()
    h = m.cell_h()
    y = m.coords[1]
    expect = np.zeros(m.n_cells)
    for c in range(m.n_cells):
        if ci[0, c] in (k - 1, k):
            j = ci[1, c]
            face = 4.0 * (y[j + 1] ** 3 - y[j] ** 3) / 3.0
            expect[c] = math.hypot(h[c, 0], h[c, 1]) / 24.0 * face
    np.testing.assert_allclose(eta2, expect, rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("d", [2, 3])
def test_indicator_of_a_quadratic_on_a_graded_axis(d):
    # u_last = x_last^2: on cell j the interpolant's derivative is x_j + x_{j+1};
    # across the face at x_{j+1} it jumps by x_{j+2} - x_j (both neighbours'
    # spacings, so a swapped or dropped h shows up)
    m = _mesh(d, 5)
    a = d - 1
    X = m.node_xyz()
    u = np.zeros((m.n_nodes, d))
    u[:, a] = X[:, a] ** 2
    eta2 = adapt.cell_indicators(m, u)
    x = m.coords[a]
    ci = m.cell_index()
    h = m.cell_h()
    expect = np.zeros(m.n_cells)
    for c in range(m.n_cells):
        j = ci[a, c]
        area = np.prod([h[c, l] for l in range(d) if l != a])
        s = 0.0
        if j > 0:
            s += (x[j + 1] - x[j - 1]) ** 2 * area
        if j < m.nc[a] - 1:
            s += (x[j + 2] - x[j]) ** 2 * area
        expect[c] = np.sqrt(np.sum(h[c] ** 2)) / 24.0 * s
    np.testing.assert_allclose(eta2, expect, rtol=1e-12)


def test_indicator_of_a_kink_3d_face_axes():
    # u_2 = |z - z_k|: jump 2 on the faces z = z_k, area h_x h_y
    m = _mesh(3, 6)
    k = 1
    zk = m.coords[2][k]
    X = m.node_xyz()
    u = np.zeros((m.n_nodes, 3))
    u[:, 2] = np.abs(X[:, 2] - zk)
    eta2 = adapt.cell_indicators(m, u)
    ci = m.cell_index()
    h = m.cell_h()
    beside = (ci[2] == k - 1) | (ci[2] == k)
    expect = np.where(beside, np.sqrt(np.sum(h ** 2, axis=1)) / 24.0 * 4.0 * h[:, 0] * h[:, 1], 0.0)
    np.testing.assert_allclose(eta2, expect, rtol=1e-13, atol=1e-30)


@pytest.mark.parametrize("d", [2, 3])
def test_slab_sums_and_minima_by_brute_force(d):
    m = _mesh(d, 7)
    rng = np.random.default_rng(8)
    eta2 = rng.uniform(size=m.n_cells)
    phi = rng.uniform(size=m.n_nodes)
    S = adapt.slab_indicators(m, eta2)
    P = adapt.slab_min_phi(m, phi)
    ci = m.cell_index()
    cn = m.cell_nodes()
    for a in range(d):
        for i in range(m.nc[a]):
            cells = [c for c in range(m.n_cells) if ci[a, c] == i]
            assert S[a][i] == pytest.approx(sum(eta2[c] for c in cells), rel=1e-14)
            assert P[a][i] == min(phi[cn[c]].min() for c in cells)


def test_marking_rules():
    x = np.array([0.0, 1.0, 1.5, 3.0, 3.125])
    S = [np.array([0.0, 0.2, 1.0, 0.05])]
    minphi = [np.array([1.0, 1.0, 1.0, 0.0])]
    # estimator only: S >= 0.2 * max, positive
    m = adapt.mark_intervals([x], S, [np.ones(4)], 0.2, 0.0, 0.5)
    assert m[0].tolist() == [False, True, True, False]
    # band only (theta > 1 disables the estimator): slab 3 is in the crack
    # region, but its length 0.125 is not above h_band = 0.125
    m = adapt.mark_intervals([x], S, minphi, 2.0, 0.125, 0.5)
    assert m[0].tolist() == [False, False, False, False]
    m = adapt.mark_intervals([x], S, minphi, 2.0, 0.0625, 0.5)
    assert m[0].tolist() == [False, False, False, True]
    # all-zero indicator marks nothing even with theta = 0
    m = adapt.mark_intervals([x], [np.zeros(4)], [np.ones(4)], 0.0, 0.0, 0.5)
    assert not m[0].any()
    new = adapt.split_intervals([x], [np.array([False, True, False, True])])
    np.testing.assert_array_equal(new[0], [0.0, 1.0, 1.25, 1.5, 3.0, 3.0625, 3.125])


def test_band_rule_reaches_eps_over_two():
    # repeated passes on a crack field end with every crack-region interval <= h_band
    ax = np.linspace(-1.0, 1.0, 9)
    coords = [ax, ax.copy()]
    phi_fn = lambda X: np.minimum(1.0, np.abs(X[:, 1]) / 0.1)  # noqa: E731
    h_band = 0.02
    for _ in range(8):
        m = fe.Mesh(coords)
        phi = phi_fn(m.node_xyz())
        marks = adapt.mark_intervals(coords, [np.zeros(n) for n in m.nc], adapt.slab_min_phi(m, phi),
                                     2.0, h_band, 0.5)
        if not any(mk.any() for mk in marks):
            break
        coords = adapt.split_intervals(coords, marks)
    m = fe.Mesh(coords)
    P = adapt.slab_min_phi(m, phi_fn(m.node_xyz()))
    for a in range(2):
        h = np.diff(coords[a])
        assert np.all(h[P[a] < 0.5] <= h_band)
    # refinement is nested: the old nodes are kept
    assert set(ax).issubset(set(coords[1]))


@pytest.mark.parametrize("d", [2, 3])
def test_transfer_is_exact_on_multilinear_fields(d):
    m = _mesh(d, 9)
    rng = np.random.default_rng(10)
    c = rng.normal(size=2 ** d)

    def f(X):
        out = np.zeros(len(X))
        for k, corner in enumerate(itertools.product((0, 1), repeat=d)):
            term = np.full(len(X), c[k])
            for l in range(d):
                if corner[l]:
                    term = term * X[:, l]
            out += term
        return out

    new = [np.sort(np.concatenate([x, rng.uniform(x[0], x[-1], 4)])) for x in m.coords]
    got = adapt.transfer(m, f(m.node_xyz()), new)
    np.testing.assert_allclose(got, f(fe.Mesh(new).node_xyz()), rtol=1e-12, atol=1e-12)
    # vector fields component by component; old nodes keep their values exactly
    F = rng.normal(size=(m.n_nodes, d))
    G = adapt.transfer(m, F, new)
    nm = fe.Mesh(new)
    pos = [np.searchsorted(new[a], m.coords[a]) for a in range(d)]
    old_in_new = nm.node_id(*[pos[a][m.node_index()[a]] for a in range(d)])
    np.testing.assert_array_equal(G[old_in_new], F)


def test_transfer_keeps_bounds_and_irreversibility():
    m = _mesh(2, 11)
    rng = np.random.default_rng(12)
    phi_old = rng.uniform(size=m.n_nodes)
    phi = phi_old * rng.uniform(size=m.n_nodes)
    new = adapt.split_intervals(m.coords, [np.ones(n, dtype=bool) for n in m.nc])
    po = adapt.transfer(m, phi_old, new)
    p = adapt.transfer(m, phi, new)
    assert np.all(p <= po + 1e-15) and np.all(p >= 0) and np.all(po <= 1)
    with pytest.raises(ValueError):
        adapt.transfer(m, phi, [np.append(new[0], new[0][-1] + 1.0), new[1]])


def test_adaptive_sequence_tracks_global_refinement():
    """Section 4.4 on the oracle alone: the adaptive Sneddon sequence (eps = 2 h_k,
    crack region refined to h_k, gradient-jump marking) gives TCV and COD(0)
    within 0.5 % of the uniform mesh with the same finest h, at a fraction of
    its unknowns."""
    import workloads as W
    from oracle import functionals as fn, model, pdas
    w, sched = W.adaptive_sneddon2d(32, 3)
    coords = w.coords
    for k, (hk, eps) in enumerate(sched):
        prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=eps, p=w.pressures[0])
        mesh = fe.Mesh(coords)
        st = pdas.State.initial(mesh, prm, W.crack_phi(coords, w.l0))
        assert all(r.converged for r in pdas.solve_loading_steps(st, w.pressures))
        tcv, cod0 = fn.tcv(mesh, st.u, st.phi), fn.cod(mesh, st.u, st.phi, [0.0])[0]
        if k > 0:
            n = int(round(4.0 / hk))
            ax = W.uniform_axis(n, -2.0, 2.0)
            um = fe.Mesh([ax, ax.copy()])
            su = pdas.State.initial(um, prm, W.crack_phi([ax, ax], w.l0))
            pdas.solve_loading_steps(su, w.pressures)
            tcv_u, cod_u = fn.tcv(um, su.u, su.phi), fn.cod(um, su.u, su.phi, [0.0])[0]
            assert abs(tcv - tcv_u) <= 5e-3 * tcv_u and abs(cod0 - cod_u) <= 5e-3 * cod_u
            assert mesh.n_nodes < (0.4 if k == 1 else 0.2) * um.n_nodes
            # the crack region is resolved to h_k
            P = adapt.slab_min_phi(mesh, st.phi)
            for a in range(2):
                assert np.all(np.diff(coords[a])[P[a] < W.ADAPT_PHI_BAND] <= hk * (1 + 1e-12))
        coords, _ = adapt.refine(mesh, st.u, st.phi, W.ADAPT_THETA, hk / 2.0, W.ADAPT_PHI_BAND)
