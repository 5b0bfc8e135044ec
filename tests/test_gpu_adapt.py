"""GPU parity of the refinement strategy (Section 3) through the C ABI.

* Indicator eta_K^2 per cell against the oracle, element by element (1e-12).
* One refinement pass: the refined axes equal the oracle's bit for bit (the
  marking is decided on slab sums that agree to rounding; the test checks that
  no slab sits within 1e-9 of the threshold, where the two could differ).
* Transfer: bit-identical to the oracle (both round every product and sum of
  the corner formula on its own).
* The adaptive Sneddon sequence: every cycle's mesh equals the oracle's, and
  its solution matches the oracle's to the Newton parity bar.
* Section 4.4's point (adaptivity reaches the accuracy of global refinement
  with far fewer unknowns): at the same finest h the adaptive TCV and COD(0)
  stay within 1 % of the uniform mesh's with under a tenth of its DoFs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adapt, fe, functionals as fn, model, pdas

pytestmark = pytest.mark.gpu

from test_gpu_parity import _assert_solution_parity  # noqa: E402  (same Newton parity bar)

torch = pytest.importorskip("torch")
pff = pytest.importorskip("paper_1806_09924_gb300")


def _graded(rng, n, lo=-1.0, hi=1.0):
    w = rng.uniform(0.3, 1.0, n)
    return lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(w) / np.sum(w)])


def _case(dim, shape, seed):
    rng = np.random.default_rng(seed)
    coords = [_graded(rng, n) for n in shape[:dim]]
    coords = [np.concatenate([c[:-1], [1.0]]) for c in coords]
    w = W.Workload("adapt_case", dim, coords, eps=0.3)
    u, phi, phi_old, _ = W.random_state(w, seed, u_scale=0.05)
    P = pff.Problem(coords)
    P.set_material(w.E, w.nu, w.Gc, w.kappa, w.eps)
    P.set_state(u, phi, phi_old, phi_old, steps_done=1)
    return P, fe.Mesh(coords), u, phi, phi_old


CASES = [(2, (37, 23), 31), (2, (1, 1), 32), (2, (2, 5), 33), (3, (9, 7, 5), 34), (3, (1, 2, 3), 35)]


@pytest.mark.parametrize("dim,shape,seed", CASES)
def test_indicator_parity(dim, shape, seed):
    P, mesh, u, _, _ = _case(dim, shape, seed)
    eta2 = torch.zeros(mesh.n_cells, dtype=torch.float64, device="cuda")
    P.cell_indicators_dev(eta2)
    torch.cuda.synchronize()
    got = eta2.cpu().numpy()
    ref = adapt.cell_indicators(mesh, u)
    scale = max(float(np.max(np.abs(ref))), 1e-300)
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-14 * scale)
    if np.any(u != 0):   # (meshes one cell thick in an axis have only boundary nodes, u = 0)
        assert np.max(ref) > 0


@pytest.mark.parametrize("dim,shape,seed", CASES)
@pytest.mark.parametrize("theta,h_band,phi_band", [(0.3, 0.05, 0.5), (0.0, 0.0, -1.0), (2.0, 0.02, 0.9)])
def test_refine_axes_parity(dim, shape, seed, theta, h_band, phi_band):
    P, mesh, u, phi, _ = _case(dim, shape, seed)
    eta2 = adapt.cell_indicators(mesh, u)
    S = adapt.slab_indicators(mesh, eta2)
    for s in S:
        smax = float(np.max(s))
        if smax > 0 and 0 < theta <= 1:
            assert np.min(np.abs(s - theta * smax)) > 1e-9 * smax, "slab at the threshold"
    ref, _ = adapt.refine(mesh, u, phi, theta, h_band, phi_band)
    got = P.refine_axes(theta, h_band, phi_band)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("dim,shape,seed", CASES)
def test_transfer_is_bit_identical(dim, shape, seed):
    P, mesh, u, phi, phi_old = _case(dim, shape, seed)
    rng = np.random.default_rng(seed + 100)
    nested = adapt.split_intervals(mesh.coords, [rng.random(n) < 0.5 for n in mesh.nc])
    general = [np.unique(np.concatenate([[c[0]], rng.uniform(c[0], c[-1], 2 * len(c)), [c[-1]]]))
               for c in mesh.coords]
    for new in (nested, general):
        Q = pff.Problem(new)
        Q.set_material(1.0, 0.2, 1.0, 1e-10, 0.3)
        P.transfer_state(Q, pff.PFF_FIELD_ALL)
        qu, qphi, _ = Q.get_solution()
        np.testing.assert_array_equal(qu, adapt.transfer(mesh, u.reshape(-1, dim), new))
        np.testing.assert_array_equal(qphi, adapt.transfer(mesh, phi, new))
        Q.close()
    # only the selected fields move; a mesh outside the box is refused
    Q = pff.Problem(nested)
    Q.set_material(1.0, 0.2, 1.0, 1e-10, 0.3)
    Q.set_crack(0.25)
    _, phi_before, _ = Q.get_solution()
    P.transfer_state(Q, pff.PFF_FIELD_U)
    qu, qphi, _ = Q.get_solution()
    np.testing.assert_array_equal(qphi, phi_before)
    np.testing.assert_array_equal(qu, adapt.transfer(mesh, u.reshape(-1, dim), nested))
    wide = [np.concatenate([c, [c[-1] + 1.0]]) for c in mesh.coords]
    R = pff.Problem(wide)
    with pytest.raises(pff.PffError):
        P.transfer_state(R, pff.PFF_FIELD_U)
    with pytest.raises(pff.PffError):
        P.transfer_state(P, pff.PFF_FIELD_U)


def _gpu_cycle(coords, eps, l0, p, prev, opts):
    Q = pff.Problem(coords)
    Q.set_material(1.0, 0.2, 1.0, 1e-10, eps)
    Q.set_crack(l0)
    if prev is not None:
        prev.transfer_state(Q, pff.PFF_FIELD_U)
    Q.solve_loading_steps([p], opts)
    return Q


def test_adaptive_sneddon_sequence_matches_oracle():
    w, sched = W.adaptive_sneddon2d(32, 4)
    opts = pff.options(precision=pff.PFF_PREC_FP64)
    coords, prev, o_prev = w.coords, None, None
    for k, (hk, eps) in enumerate(sched):
        mesh = fe.Mesh(coords)
        Q = _gpu_cycle(coords, eps, w.l0, w.pressures[0], prev, opts)
        prm = model.Params(E=1.0, nu=0.2, Gc=1.0, kappa=1e-10, eps=eps, p=w.pressures[0])
        st = pdas.State.initial(mesh, prm, W.crack_phi(coords, w.l0))
        if o_prev is not None:
            st.u = adapt.transfer(o_prev[0], o_prev[1], coords)
        pdas.solve_loading_steps(st, w.pressures)
        u, phi, act = Q.get_solution()
        _assert_solution_parity(mesh, st, u, phi, act, f"adaptive k={k} cells={mesh.nc}")
        tcv, cod = Q.eval_tcv_cod([0.0])
        assert abs(tcv - fn.tcv(mesh, st.u, st.phi)) <= 1e-6 * abs(tcv)
        # next mesh: both sides refine their own solution
        h_next = hk / 2.0
        ref, _ = adapt.refine(mesh, st.u, st.phi, W.ADAPT_THETA, h_next, W.ADAPT_PHI_BAND)
        got = Q.refine_axes(W.ADAPT_THETA, h_next, W.ADAPT_PHI_BAND)
        for g, r in zip(got, ref):
            np.testing.assert_array_equal(g, r)
        if prev is not None:
            prev.close()
        prev, o_prev, coords = Q, (mesh, st.u), got
    prev.close()


def test_adaptive_reaches_uniform_accuracy_with_fewer_dofs():
    w, sched = W.adaptive_sneddon2d(32, 6)
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    coords, prev = w.coords, None
    for k, (hk, eps) in enumerate(sched):
        Q = _gpu_cycle(coords, eps, w.l0, w.pressures[0], None, opts)
        tcv, cod = Q.eval_tcv_cod([0.0])
        n_uni = int(round(4.0 / hk))
        ax = W.uniform_axis(n_uni, -2.0, 2.0)
        U = _gpu_cycle([ax, ax.copy()], eps, w.l0, w.pressures[0], None, opts)
        tcv_u, cod_u = U.eval_tcv_cod([0.0])
        ratio = Q.n_dofs / U.n_dofs
        print(f"ADAPT-VS-UNIFORM k={k} h={hk:.5f} dofs {Q.n_dofs} vs {U.n_dofs} "
              f"tcv {tcv:.6e} vs {tcv_u:.6e} cod0 {cod[0]:.6e} vs {cod_u[0]:.6e}")
        if k >= 3:
            assert ratio < 0.1
            assert abs(tcv - tcv_u) <= 0.01 * tcv_u
            assert abs(cod[0] - cod_u[0]) <= 0.01 * cod_u[0]
        U.close()
        got = Q.refine_axes(W.ADAPT_THETA, hk / 2.0, W.ADAPT_PHI_BAND)
        if prev is not None:
            prev.close()
        prev, coords = Q, got
    prev.close()


def test_cyclic_loading_with_refinement_matches_oracle():
    """Crack growth under the load / unload / reload cycle (32^2 start, eps
    fixed) with a refinement pass after every loading step: u, phi, phi_old
    and phi_prev move to the refined mesh on both sides (the GPU by
    pff_transfer_state, the oracle by its own interpolation), the step count
    carries the phi~ extrapolation across, and every step's mesh, solution,
    active set and cycle-lock count match.

    The refinement takes the cells below eps/4, where the phase-field block's
    Laplacian dominates its mass term; the default phase-field preconditioner
    then switches from smoothing to the full hierarchy.  With smoothing only,
    the last step (1.2e-2, past the critical pressure, where the crack runs)
    stalled FGMRES at its 600-iteration cap; with the hierarchy it takes 34
    Newton iterations, as in the oracle."""
    w = W.cyclic_loading(32)
    theta = 0.5
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    P = pff.problem_from_workload(w)
    o = pff.options(precision=pff.PFF_PREC_FP64)
    locked = 0
    for k, p in enumerate(w.pressures):
        orep = pdas.loading_step(st, p)
        rep = P.solve_loading_steps([p], o)[0]
        assert orep.converged and rep["converged"] == 1, (k, rep)
        assert rep["locked"] == orep.locked
        locked += orep.locked
        u, phi, act = P.get_solution()
        _assert_solution_parity(mesh, st, u, phi, act.astype(bool), f"cyclic_adaptive_step{k} cells={mesh.nc}")
        ref, _ = adapt.refine(mesh, st.u, st.phi, theta, w.eps / 2.0, W.ADAPT_PHI_BAND)
        got = P.refine_axes(theta, w.eps / 2.0, W.ADAPT_PHI_BAND)
        for g, r in zip(got, ref):
            np.testing.assert_array_equal(g, r)
        nm = fe.Mesh(ref)
        st = pdas.State(nm, prm, adapt.transfer(mesh, st.u, ref), adapt.transfer(mesh, st.phi, ref),
                        adapt.transfer(mesh, st.phi_old, ref), adapt.transfer(mesh, st.phi_prev, ref),
                        st.steps_done)
        Q = pff.Problem(got)
        Q.set_material(w.E, w.nu, w.Gc, w.kappa, w.eps)
        P.transfer_state(Q, pff.PFF_FIELD_ALL)
        P.close()
        P, mesh = Q, nm
    assert mesh.n_cells > 32 * 32 and locked > 0
    P.close()
