"""Pins of the TCV / COD functionals and of Sneddon's closed forms (Section 4).

* The printed closed-form values (tests/golden/sneddon_values.txt).
* Integrating the full opening 2 u_n over the crack gives back TCV, in 2d and
  3d (consistency of the two closed forms of Section 4).
* TCV and COD of fields with a known integral (divergence theorem, Fubini).
* The oracle's converged Sneddon solutions converge toward the closed form as
  h and eps = 2h go to zero, to within the finite-domain gap of Section 4.2.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from conftest import read_golden
from oracle import fe, functionals as fn, model, pdas
import workloads as W


def _golden():
    return {r[0]: [float(v) for v in r[1:]] for r in read_golden("sneddon_values.txt")}


def test_closed_forms_match_printed_values():
    g = _golden()
    l0, E, p, nu = g["l0"][0], g["E"][0], g["p"][0], g["nu"][0]
    assert fn.sneddon_tcv(2, p, l0, E, nu) == pytest.approx(g["tcv2d"][0], rel=5e-5)
    assert fn.sneddon_tcv(3, p, l0, E, nu) == pytest.approx(g["tcv3d"][0], rel=5e-5)


def test_opening_integrates_to_tcv():
    p, l0, E, nu = 1e-3, 0.7, 1.3, 0.25
    v2, _ = integrate.quad(lambda x: fn.sneddon_cod(2, p, l0, E, nu, abs(x)), -l0, l0, epsabs=0, epsrel=1e-12)
    assert v2 == pytest.approx(fn.sneddon_tcv(2, p, l0, E, nu), rel=1e-9)
    v3, _ = integrate.quad(lambda r: 2 * math.pi * r * fn.sneddon_cod(3, p, l0, E, nu, r), 0, l0,
                           epsabs=0, epsrel=1e-12)
    assert v3 == pytest.approx(fn.sneddon_tcv(3, p, l0, E, nu), rel=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_tcv_of_constant_displacement_is_boundary_flux(dim):
    """u = c constant: int c . grad phi = sum_l c_l (int over the faces x_l = max of phi - x_l = min)."""
    rng = np.random.default_rng(2)
    coords = [np.sort(np.r_[-1.0, rng.uniform(-1, 1, 4), 1.0]) for _ in range(dim)]
    mesh = fe.Mesh(coords)
    phi = rng.random(mesh.n_nodes)
    c = rng.standard_normal(dim)
    u = np.tile(c, (mesh.n_nodes, 1))
    shape = mesh.nn[::-1]
    P = phi.reshape(shape)           # [k][j][i] (3d) or [j][i]
    expect = 0.0
    for l in range(dim):
        ax = dim - 1 - l             # array axis of coordinate l
        hi = np.take(P, -1, axis=ax)
        lo = np.take(P, 0, axis=ax)
        face = hi - lo               # a Q1 function on the face: integrate with the trapezoid rule
        others = [mesh.coords[m] for m in range(dim) if m != l]
        val = face
        for m in range(len(others)):     # integrate over the remaining coordinates (x fastest = last axis)
            val = np.trapezoid(val, others[m], axis=-1)
        expect += c[l] * val
    assert fn.tcv(mesh, u, phi) == pytest.approx(expect, rel=1e-12)


def test_cod_integrates_to_tcv_fubini():
    """Integrating COD(x) over x (2 Gauss points per cell column, exact) gives TCV."""
    rng = np.random.default_rng(4)
    coords = [np.sort(np.r_[-1.0, rng.uniform(-1, 1, 5), 1.0]) for _ in range(2)]
    mesh = fe.Mesh(coords)
    u = rng.standard_normal((mesh.n_nodes, 2))
    phi = rng.random(mesh.n_nodes)
    X = coords[0]
    pts, wts = [], []
    for i in range(len(X) - 1):
        for g, wg in zip(fe.GAUSS_1D, fe.WEIGHT_1D):
            pts.append(X[i] + g * (X[i + 1] - X[i]))
            wts.append(wg * (X[i + 1] - X[i]))
    total = float(np.dot(fn.cod(mesh, u, phi, pts), wts))
    assert total == pytest.approx(fn.tcv(mesh, u, phi), rel=1e-12)


def test_cod_on_mesh_line_is_average_of_neighbours():
    rng = np.random.default_rng(5)
    ax = W.uniform_axis(6, -1, 1)
    mesh = fe.Mesh([ax, ax])
    u = rng.standard_normal((mesh.n_nodes, 2))
    phi = rng.random(mesh.n_nodes)
    x0 = ax[3]
    on = fn.cod(mesh, u, phi, [x0])[0]
    left = fn.cod(mesh, u, phi, [x0 - 1e-9])[0]
    right = fn.cod(mesh, u, phi, [x0 + 1e-9])[0]
    assert on == pytest.approx(0.5 * (left + right), rel=1e-6)


def test_sneddon_2d_convergence_toward_closed_form():
    """TCV and the centre opening approach Sneddon as h, eps = 2h -> 0 (Section 4.1, 4.2).

    The box is (-2,2)^2 with l0 = 0.25, i.e. K/l0 = 8; Section 4.2 reports a
    finite-domain TCV deficit of 1.5 % at K/l0 = 10 and 5.6 % at K/l0 = 5.
    """
    w0 = W.config(0)
    snd_t = fn.sneddon_tcv(2, 1e-3, w0.l0, w0.E, w0.nu)
    snd_c = fn.sneddon_cod(2, 1e-3, w0.l0, w0.E, w0.nu, [0.0])[0]
    errs_t, errs_c = [], []
    for n in (32, 64, 128):
        w = W.scaled_workload(w0, n)
        mesh = fe.Mesh(w.coords)
        prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=1e-3)
        st = pdas.State.initial(mesh, prm, w.phi0())
        assert pdas.loading_step(st, 1e-3).converged
        errs_t.append(fn.tcv(mesh, st.u, st.phi) / snd_t - 1.0)
        errs_c.append(fn.cod(mesh, st.u, st.phi, [w0.l0 / 64])[0] / snd_c - 1.0)
    # TCV error shrinks by at least 3x per halving of h (and eps) and ends within 5 %
    assert abs(errs_t[1]) < abs(errs_t[0]) / 3 and abs(errs_t[2]) < abs(errs_t[1]) / 3
    assert abs(errs_t[2]) < 0.05
    # the opening at the centre approaches from below, monotonically
    assert errs_c[0] < errs_c[1] < errs_c[2] < 0.0
    assert errs_c[2] > -0.15


def test_penny_3d_tcv_reasonable():
    """3d penny crack on a coarse graded mesh: positive TCV of the closed form's order."""
    w = W.scaled_workload(W.config(2), 16)
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=1e-3)
    st = pdas.State.initial(mesh, prm, w.phi0())
    rep = pdas.loading_step(st, 1e-3)
    assert rep.converged
    T = fn.tcv(mesh, st.u, st.phi)
    snd = fn.sneddon_tcv(3, 1e-3, w.l0, w.E, w.nu)
    assert 0.2 * snd < T < 5 * snd
