"""Pins of the oracle's Q1 discretization against exact integration and FE invariants.

Each check computes the expected value by a route that does not use the
oracle's quadrature or its einsum contractions: symbolic integration of the
textbook Voigt form B^T D B (which uses E and nu directly, so it also pins the
Lame conversion), rigid-body and patch-test invariants, and closed-form
integrals of the Q1 mass and stiffness.
"""
import numpy as np
import pytest
import sympy as sy

from oracle import fe, model
import workloads as W


def _voigt_D(d, E, nu):
    c = E / ((1 + nu) * (1 - 2 * nu))
    if d == 2:   # plane strain
        return c * sy.Matrix([[1 - nu, nu, 0], [nu, 1 - nu, 0], [0, 0, (1 - 2 * nu) / 2]])
    D = sy.zeros(6, 6)
    for i in range(3):
        for j in range(3):
            D[i, j] = c * (1 - nu if i == j else nu)
        D[3 + i, 3 + i] = c * (1 - 2 * nu) / 2
    return D


def _symbolic_element_stiffness(h, E, nu):
    d = len(h)
    X = sy.symbols("x0:%d" % d)
    H = [sy.Rational(str(v)) for v in h]
    Es, nus = sy.Rational(str(E)), sy.Rational(str(nu))
    shapes = []
    for a in range(2 ** d):
        f = 1
        for l in range(d):
            f *= (X[l] / H[l]) if (a >> l) & 1 else (1 - X[l] / H[l])
        shapes.append(sy.expand(f))
    nd = d * 2 ** d
    # Voigt strain rows: normal strains, then engineering shears
    pairs = [(0, 1)] if d == 2 else [(1, 2), (0, 2), (0, 1)]
    nv = d + len(pairs)
    B = sy.zeros(nv, nd)
    for a, N in enumerate(shapes):
        for m in range(d):
            B[m, a * d + m] = sy.diff(N, X[m])
        for r, (i, j) in enumerate(pairs):
            B[d + r, a * d + i] = sy.diff(N, X[j])
            B[d + r, a * d + j] = sy.diff(N, X[i])
    D = _voigt_D(d, Es, nus)
    integrand = (B.T * D * B).applyfunc(sy.expand)
    K = np.zeros((nd, nd))
    for i in range(nd):
        for j in range(i, nd):
            v = integrand[i, j]
            for l in range(d):
                v = sy.integrate(v, (X[l], 0, H[l]))
            K[i, j] = K[j, i] = float(v)
    return K


@pytest.mark.parametrize("h", [(0.5, 0.25), (1.0, 1.0), (0.3, 0.2, 0.1)])
def test_element_stiffness_matches_exact_voigt_integral(h):
    E, nu = 1.0, 0.2
    d = len(h)
    mesh = fe.Mesh([np.array([0.0, hl]) for hl in h])
    n = mesh.n_nodes
    prm = model.Params(E=E, nu=nu, kappa=0.0)
    Muu, _, _ = model.jacobian_blocks(mesh, prm, np.zeros((n, d)), np.ones(n), np.ones(n))
    K_exact = _symbolic_element_stiffness(h, E, nu)
    K = Muu.toarray()
    assert np.max(np.abs(K - K_exact)) <= 1e-13 * np.max(np.abs(K_exact))


def test_lame_plane_strain_constants():
    mu, lam = fe.lame(1.0, 0.2)
    assert mu == pytest.approx(1.0 / 2.4, rel=1e-15)
    assert lam == pytest.approx(0.2 / (1.2 * 0.6), rel=1e-15)
    # P-wave modulus of plane strain: E (1-nu) / ((1+nu)(1-2nu))
    assert lam + 2 * mu == pytest.approx(0.8 / (1.2 * 0.6), rel=1e-15)


def _rigid_modes(xyz):
    n, d = xyz.shape
    modes = []
    for m in range(d):
        v = np.zeros((n, d)); v[:, m] = 1.0; modes.append(v)
    rots = [(0, 1)] if d == 2 else [(0, 1), (1, 2), (0, 2)]
    for i, j in rots:
        v = np.zeros((n, d)); v[:, i] = -xyz[:, j]; v[:, j] = xyz[:, i]; modes.append(v)
    return modes


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_body_modes_in_kernel_of_unconstrained_Muu(dim):
    rng = np.random.default_rng(0)
    coords = [np.cumsum(np.r_[0.0, rng.uniform(0.2, 1.0, 4)]) - 1.0 for _ in range(dim)]
    mesh = fe.Mesh(coords)
    n = mesh.n_nodes
    prm = model.Params()
    phit = rng.random(n)
    Muu, _, _ = model.jacobian_blocks(mesh, prm, np.zeros((n, dim)), np.ones(n), phit)
    modes = _rigid_modes(mesh.node_xyz())
    assert len(modes) == (3 if dim == 2 else 6)
    scale = abs(Muu).max()
    for v in modes:
        r = Muu @ v.ravel()
        assert np.max(np.abs(r)) <= 1e-13 * scale * np.max(np.abs(v))
    # and nothing else: a random field is not annihilated
    assert np.linalg.norm(Muu @ rng.standard_normal(dim * n)) > 1e-3 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_uniform_strain(dim):
    """A linear displacement on a graded mesh: interior rows vanish and the
    energy 1/2 u^T M_uu u equals 1/2 g |Omega| sigma(B):e(B) (Voigt, E and nu)."""
    rng = np.random.default_rng(1)
    ax = W.graded_axis(6, 1.0, 0.1)
    mesh = fe.Mesh([ax] * dim)
    n = mesh.n_nodes
    E, nu = 1.3, 0.27
    prm = model.Params(E=E, nu=nu, kappa=1e-10)
    phit = np.full(n, 0.7)
    g = (1 - 1e-10) * 0.49 + 1e-10
    Muu, _, _ = model.jacobian_blocks(mesh, prm, np.zeros((n, dim)), np.ones(n), phit)
    Bm = rng.standard_normal((dim, dim))
    u = mesh.node_xyz() @ Bm.T + rng.standard_normal(dim)
    r = (Muu @ u.ravel()).reshape(n, dim)
    interior = ~mesh.boundary_nodes()
    assert np.max(np.abs(r[interior])) <= 1e-12 * np.max(np.abs(r))
    eps = 0.5 * (Bm + Bm.T)
    if dim == 2:
        ev = np.array([eps[0, 0], eps[1, 1], 2 * eps[0, 1]])
    else:
        ev = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
    D = np.array(_voigt_D(dim, E, nu).evalf(), dtype=float)
    vol = 2.0 ** dim
    expect = 0.5 * g * vol * ev @ D @ ev
    assert 0.5 * u.ravel() @ Muu @ u.ravel() == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_phase_field_mass_and_laplace(dim):
    ax = W.graded_axis(8, 1.5, 0.1)
    mesh = fe.Mesh([ax] * dim)
    M, K = model.phase_field_matrices(mesh)
    one = np.ones(mesh.n_nodes)
    vol = 3.0 ** dim
    assert one @ M @ one == pytest.approx(vol, rel=1e-14)
    assert np.max(np.abs(K @ one)) < 1e-13 * abs(K).max()
    x = mesh.node_xyz()[:, 0]
    assert x @ K @ x == pytest.approx(vol, rel=1e-13)              # int |grad x|^2
    # int x^2 over the box is exact for the Q1 interpolant of x (x linear)
    assert x @ M @ x == pytest.approx(vol / 3.0 * 1.5 ** 2, rel=1e-13)
    m = model.lumped_mass(mesh)
    assert m.sum() == pytest.approx(vol, rel=1e-14)
    assert np.allclose(m, M @ one, rtol=1e-14, atol=0)


def test_lumped_mass_interior_node_uniform():
    ax = W.uniform_axis(8, -2.0, 2.0)
    mesh = fe.Mesh([ax, ax])
    m = model.lumped_mass(mesh)
    h = 0.5
    idx = mesh.node_id(np.array([3]), np.array([4]))[0]
    assert m[idx] == pytest.approx(h * h, rel=1e-15)
    assert m[0] == pytest.approx(h * h / 4, rel=1e-15)


def test_table1_dof_counts():
    from conftest import read_golden
    for ref, dofs in read_golden("table1_dofs.txt"):
        n = 2 ** (int(ref) + 3)
        w = W.Workload("t", 2, [W.uniform_axis(n, -1, 1)] * 2)
        assert w.n_dofs == int(dofs)
    assert W.config(0).n_dofs == 49923       # 128^2 cells = refinement 4 of Table 1
    assert W.config(1).n_dofs == 3151875     # 1024^2 cells = refinement 7
