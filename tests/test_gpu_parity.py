"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (FP64 path): residual and reduced-Jacobian apply relative L2 <= 1e-12;
functionals and lumped quantities 1e-12; converged u, phi relative L2 <= 1e-8
with identical active sets away from round-off ties; TCV / COD <= 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fe, functionals as fn, model, pdas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pff = pytest.importorskip("paper_1806_09924_gb300")

RTOL_OP = 1e-12
RTOL_SOL = 1e-8
RTOL_FUNC = 1e-6


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_coords(rng, n, lo=-1.0, hi=1.0):
    x = np.sort(rng.uniform(lo, hi, n - 1))
    c = np.concatenate([[lo], x, [hi]])
    if np.min(np.diff(c)) < 1e-3 * (hi - lo) / n:
        return np.linspace(lo, hi, n + 1)
    return c


def make_case(dim, shape, seed, p=3e-2):
    rng = np.random.default_rng(seed)
    coords = [random_coords(rng, n) for n in shape[:dim]]
    mesh = fe.Mesh(coords)
    n = mesh.n_nodes
    w = W.Workload("case", dim, coords, E=1.3, nu=0.27, Gc=0.9, kappa=1e-6, eps=0.3)
    u, phi, phi_old, _ = W.random_state(w, seed, u_scale=0.05)
    phi_prev = rng.random(n)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p)
    phit = np.clip(2 * phi_old - phi_prev, 0.0, 1.0)
    P = pff.Problem(coords)
    P.set_material(w.E, w.nu, w.Gc, w.kappa, w.eps)
    # two completed loading steps: phi~ is the clamped linear extrapolation
    P.set_state(u, phi, phi_old, phi_prev, steps_done=2)
    P.set_pressure(p)
    return P, mesh, prm, (u, phi, phi_old, phi_prev, phit)


CASES = [(2, (37, 23), 11), (2, (8, 5), 12), (2, (1, 1), 13), (3, (9, 7, 5), 14), (3, (2, 3, 2), 15)]


@pytest.mark.parametrize("dim,shape,seed", CASES)
def test_residual_parity(dim, shape, seed):
    P, mesh, prm, (u, phi, phi_old, phi_prev, phit) = make_case(dim, shape, seed)
    F = torch.empty(P.n_dofs, dtype=torch.float64, device="cuda")
    P.residual_dev(F)
    torch.cuda.synchronize()
    r_u, r_phi = model.gradient(mesh, prm, u, phi, phit)
    F_ref = -np.concatenate([r_u.ravel(), r_phi])
    assert rel(F.cpu().numpy(), F_ref) <= RTOL_OP
    P.close()


def oracle_reduced_apply(mesh, prm, state, active, x):
    u, phi, _, _, phit = state
    d, n = mesh.d, mesh.n_nodes
    J = model.jacobian(mesh, prm, u, phi, phit)
    fixed = np.concatenate([np.repeat(mesh.boundary_nodes(), d), active.astype(bool)])
    xm = np.where(fixed, 0.0, x)
    y = J @ xm
    y[fixed] = x[fixed]
    return y


@pytest.mark.parametrize("dim,shape,seed", CASES)
def test_active_set_and_jacobian_apply_parity(dim, shape, seed):
    P, mesh, prm, state = make_case(dim, shape, seed)
    u, phi, phi_old, phi_prev, phit = state
    n = mesh.n_nodes
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    ind = torch.empty(n, dtype=torch.float64, device="cuda")
    P.active_set_dev(1.0, act, ind)
    r_u, r_phi = model.gradient(mesh, prm, u, phi, phit)
    # c is given in units of G_c / eps
    ind_ref = pdas.active_indicator(-r_phi, model.lumped_mass(mesh), phi, phi_old, prm.Gc / prm.eps)
    assert rel(ind.cpu().numpy(), ind_ref) <= RTOL_OP
    a = act.cpu().numpy().astype(bool)
    clear = np.abs(ind_ref) > 1e-12 * np.max(np.abs(ind_ref))
    assert np.array_equal(a[clear], (ind_ref > 0)[clear])
    P.assemble()
    rng = np.random.default_rng(seed + 100)
    x = rng.standard_normal(P.n_dofs)
    y_ref = oracle_reduced_apply(mesh, prm, state, a, x)
    xd = torch.tensor(x, device="cuda")
    for variant in (pff.PFF_APPLY_ASSEMBLED, pff.PFF_APPLY_MATFREE):
        y = torch.empty_like(xd)
        P.apply_jacobian_dev(variant, xd, y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), y_ref) <= RTOL_OP, variant
    P.close()


@pytest.mark.parametrize("dim,shape,seed", [(2, (37, 23), 21), (3, (9, 7, 5), 22)])
def test_tcv_cod_parity(dim, shape, seed):
    P, mesh, prm, (u, phi, *_rest) = make_case(dim, shape, seed)
    rng = np.random.default_rng(seed)
    if dim == 2:
        pts = np.concatenate([rng.uniform(-1, 1, 6), [mesh.coords[0][3], -1.0, 1.0]])
    else:
        pts = np.concatenate([rng.uniform(-1, 1, (4, 2)),
                              [[mesh.coords[0][2], mesh.coords[1][4]], [0.1, mesh.coords[1][1]]]]).ravel()
    tcv, cod = P.eval_tcv_cod(pts)
    assert rel(tcv, fn.tcv(mesh, u, phi)) <= RTOL_OP
    assert rel(cod, fn.cod(mesh, u, phi, pts)) <= 1e-12
    P.close()


def _oracle_solution(w, pressures, opts=None):
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    reps = pdas.solve_loading_steps(st, pressures, opts or pdas.Options())
    return mesh, st, reps


def _gpu_solution(w, pressures, **kw):
    P = pff.problem_from_workload(w)
    reps = P.solve_loading_steps(pressures, pff.options(**kw))
    u, phi, act = P.get_solution()
    return P, u, phi, act.astype(bool), reps


TIE_BAND = 1e-7   # in units of G_c / eps


def rel_inf(a, b, mask=None):
    """max |a - b| / max |b| (over the masked entries)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    nb = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (nb if nb > 0 else 1.0)) if b.size else 0.0


def _assert_solution_parity(mesh, st, u, phi, act, label=""):
    """u, phi within RTOL_SOL, in relative L2 and element by element (max norm),
    over the whole mesh and separately over the crack band (nodes where phi or
    phi_old is below 1/2: the kappa-degenerate rows); active sets identical
    wherever the oracle's indicator exceeds TIE_BAND G_c/eps.

    The band: the Newton stop leaves the converged state within ~1e-10 of the
    discrete solution and the GPU's linear solves stop at 1e-8, so the two
    converged phase fields differ by ~1e-10..1e-9 per node; the indicator
    (F_phi/m + c (phi - phi_old), slope ~ G_c/eps per unit of phi) then
    differs by ~1e-9 G_c/eps, and a node within that distance of the
    threshold may land on either side.  TIE_BAND keeps a 100x margin.
    Mismatches inside it are counted and printed (pytest -rP shows them)."""
    d = mesh.d
    u_ref = st.u.reshape(-1, d)
    u = np.asarray(u).reshape(-1, d)
    band = (np.minimum(st.phi, st.phi_prev) < 0.5)
    assert rel(u, u_ref) <= RTOL_SOL
    assert rel(phi, st.phi) <= RTOL_SOL
    assert rel_inf(u, u_ref) <= RTOL_SOL, rel_inf(u, u_ref)
    assert rel_inf(phi, st.phi) <= RTOL_SOL, rel_inf(phi, st.phi)
    assert band.any()
    assert rel_inf(u, u_ref, band) <= RTOL_SOL, rel_inf(u, u_ref, band)
    assert rel_inf(phi, st.phi, band) <= RTOL_SOL or np.max(np.abs(phi[band] - st.phi[band])) <= 1e-12
    ind = st.indicator
    scale = st.prm.Gc / st.prm.eps
    clear = np.abs(ind) > TIE_BAND * scale
    mism = np.count_nonzero(act[clear] != st.active[clear])
    assert mism == 0, f"{mism} active-set mismatches away from ties"
    total = int(np.count_nonzero(act != st.active))
    near = np.abs(ind) <= 1e-9 * scale
    print(f"PARITY {label} n={mesh.n_nodes} rel_l2_u={rel(u, u_ref):.2e} rel_inf_u={rel_inf(u, u_ref):.2e} "
          f"rel_inf_u_band={rel_inf(u, u_ref, band):.2e} rel_inf_phi={rel_inf(phi, st.phi):.2e} "
          f"active_mismatch_total={total} outside_1e-9_band={int(np.count_nonzero((act != st.active) & ~near))} "
          f"inside_1e-9_band_nodes={int(near.sum())}")
    return total


@pytest.mark.parametrize("n_cells,precision", [(32, 0), (64, 0), (64, 1)])
def test_newton_solution_parity_2d(n_cells, precision):
    w = W.scaled_workload(W.config(0), n_cells)
    mesh, st, oreps = _oracle_solution(w, w.pressures)
    P, u, phi, act, reps = _gpu_solution(w, w.pressures, precision=precision)
    assert reps[0]["converged"] == 1 and oreps[0].converged
    _assert_solution_parity(mesh, st, u, phi, act, f"sneddon{n_cells}_p{precision}")
    pts = fn.cod_points(w.l0, 64)
    tcv, cod = P.eval_tcv_cod(pts)
    assert rel(tcv, fn.tcv(mesh, st.u, st.phi)) <= RTOL_FUNC
    assert rel(cod, fn.cod(mesh, st.u, st.phi, pts)) <= RTOL_FUNC
    P.close()


def test_newton_solution_parity_sneddon_128():
    """The 128x128 Sneddon configuration (Table 1 refinement 4 size), FP64 and mixed."""
    w = W.config(0)
    mesh, st, oreps = _oracle_solution(w, w.pressures)
    pts = fn.cod_points(w.l0, 64)
    tcv_ref = fn.tcv(mesh, st.u, st.phi)
    cod_ref = fn.cod(mesh, st.u, st.phi, pts)
    for precision in (0, 1):
        P, u, phi, act, reps = _gpu_solution(w, w.pressures, precision=precision)
        assert reps[0]["converged"] == 1
        _assert_solution_parity(mesh, st, u, phi, act, f"sneddon128_p{precision}")
        tcv, cod = P.eval_tcv_cod(pts)
        assert rel(tcv, tcv_ref) <= RTOL_FUNC
        assert rel(cod, cod_ref) <= RTOL_FUNC
        P.close()


def test_three_loading_steps_parity():
    """Three steps: the third uses the clamped linear extrapolation phi~."""
    w = W.scaled_workload(W.config(0), 48)
    pressures = [5e-4, 1e-3, 1.5e-3]
    mesh, st, oreps = _oracle_solution(w, pressures)
    P, u, phi, act, reps = _gpu_solution(w, pressures)
    assert all(r["converged"] == 1 for r in reps)
    _assert_solution_parity(mesh, st, u, phi, act, "three_steps48")
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graded_ramp_parity(precision):
    """The graded-mesh recipe of the 1024^2 workload at 64^2 cells, three ramp steps."""
    w = W.scaled_workload(W.config(1), 64)
    pressures = w.pressures[:3]
    mesh, st, oreps = _oracle_solution(w, pressures)
    P, u, phi, act, reps = _gpu_solution(w, pressures, precision=precision)
    assert all(r["converged"] == 1 for r in reps) and all(r.converged for r in oreps)
    _assert_solution_parity(mesh, st, u, phi, act, f"graded64_3steps_p{precision}")
    pts = fn.cod_points(w.l0, 16)
    tcv, cod = P.eval_tcv_cod(pts)
    assert rel(tcv, fn.tcv(mesh, st.u, st.phi)) <= RTOL_FUNC
    assert rel(cod, fn.cod(mesh, st.u, st.phi, pts)) <= RTOL_FUNC
    P.close()


def test_hierarchy_reuse_across_loading_steps():
    """A displacement hierarchy carried over between loading steps (phi~ barely
    moves in the ramp) changes the preconditioner, not the converged solution."""
    w = W.scaled_workload(W.config(1), 96)
    out = {}
    for reuse in (0, 1):
        P = pff.problem_from_workload(w)
        reps = P.solve_loading_steps(w.pressures, pff.options(precision=1, amg_reuse=reuse))
        assert all(r["converged"] == 1 for r in reps)
        u, phi, act = P.get_solution()
        out[reuse] = (u, phi, act, [r["amg_builds_u"] for r in reps])
        P.close()
    assert out[0][3] == [1] * len(w.pressures)
    assert out[1][3][0] == 1 and sum(out[1][3]) < len(w.pressures)
    assert rel(out[1][0], out[0][0]) <= 1e-9
    assert rel(out[1][1], out[0][1]) <= 1e-9


@pytest.mark.parametrize("n_cells", [12, 24])
def test_newton_solution_parity_3d(n_cells):
    """The penny-shaped crack recipe (graded, mixed precision) at 12^3 and 24^3
    cells; the cycle rule locks indices here on both sides (the oracle locks
    620 at 24^3), so the locked sets must agree too."""
    w = W.scaled_workload(W.config(2), n_cells)
    mesh, st, oreps = _oracle_solution(w, [1e-3])
    P, u, phi, act, reps = _gpu_solution(w, [1e-3], precision=1)
    assert reps[0]["converged"] == 1
    assert reps[0]["locked"] == oreps[0].locked
    _assert_solution_parity(mesh, st, u, phi, act, f"penny{n_cells}")
    tcv, _ = P.eval_tcv_cod([])
    assert rel(tcv, fn.tcv(mesh, st.u, st.phi)) <= RTOL_FUNC
    P.close()


def test_newton_solution_parity_3d_32_stored_oracle():
    """The penny recipe at 32^3 (143,748 DoFs) against the oracle solution
    stored by tests/golden/make_oracle_fixtures.py (the oracle run takes
    minutes); the fixture must come from the current oracle sources."""
    import sys
    import os
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_oracle_fixtures as mf
    z = np.load(mf.fixture_path("penny3d_32"))
    w, pressures = mf.penny3d_32_workload()
    stale = "stale fixture: run python tests/golden/make_oracle_fixtures.py penny3d_32"
    assert str(z["source_sha256"]) == mf.source_hash(), stale
    assert str(z["input_sha256"]) == mf.input_hash(w, pressures), stale
    assert int(z["n_dofs"]) == w.n_dofs
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=1e-3)
    st = pdas.State(mesh, prm, z["u"], z["phi"], z["phi"].copy(), phi_prev=w.phi0(), steps_done=1,
                    active=z["active"].astype(bool), indicator=z["indicator"])
    P, u, phi, act, reps = _gpu_solution(w, [1e-3], precision=1)
    assert reps[0]["converged"] == 1
    assert reps[0]["locked"] == int(z["locked"][0])
    _assert_solution_parity(mesh, st, u, phi, act, "penny32")
    tcv, _ = P.eval_tcv_cod([])
    assert rel(tcv, float(z["tcv"])) <= RTOL_FUNC
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graded_ramp_parity_full_schedule(precision):
    """All five loading steps of the graded 1024^2 recipe at 128^2 cells:
    steps 3-5 run on the extrapolated phi~ (Formulation 1)."""
    w = W.scaled_workload(W.config(1), 128)
    mesh, st, oreps = _oracle_solution(w, w.pressures)
    P, u, phi, act, reps = _gpu_solution(w, w.pressures, precision=precision)
    assert all(r["converged"] == 1 for r in reps) and all(r.converged for r in oreps)
    _assert_solution_parity(mesh, st, u, phi, act, f"graded128_5steps_p{precision}")
    pts = fn.cod_points(w.l0, 64)
    tcv, cod = P.eval_tcv_cod(pts)
    assert rel(tcv, fn.tcv(mesh, st.u, st.phi)) <= RTOL_FUNC
    assert rel(cod, fn.cod(mesh, st.u, st.phi, pts)) <= RTOL_FUNC
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_cyclic_loading_parity(precision):
    """A crack that grows and is then unloaded and reloaded (load / unload /
    reload pressure cycle near the critical pressure, G_c = 1e-4, 64^2): the
    damaged zone ahead of the tips grows while the pressure rises, and the
    irreversibility constraint binds on it while the pressure falls
    (Formulation 1, phi <= phi_old).  Every step is compared, not only the
    last: solutions, active sets and the cycle-lock counts."""
    w = W.cyclic_loading(64)
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    P = pff.problem_from_workload(w)
    o = pff.options(precision=precision)
    grew = False
    for k, p in enumerate(w.pressures):
        orep = pdas.loading_step(st, p)
        rep = P.solve_loading_steps([p], o)[0]
        assert orep.converged and rep["converged"] == 1, (k, rep)
        assert rep["locked"] == orep.locked
        u, phi, act = P.get_solution()
        _assert_solution_parity(mesh, st, u, phi, act.astype(bool), f"cyclic64_step{k}_p{precision}")
        grew |= np.count_nonzero(st.phi < 0.5) > np.count_nonzero(w.phi0() < 0.5)
    assert grew
    P.close()


def test_cycle_lock_parity():
    """Indices that alternate are locked identically on both sides (cycle rule
    of Section 3 with a lock after 2 membership changes; 24^2 cyclic recipe,
    first loading step, where the oracle locks 16 indices)."""
    w = W.cyclic_loading(24)
    p = 5e-3
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p)
    st = pdas.State.initial(mesh, prm, w.phi0())
    orep = pdas.loading_step(st, p, pdas.Options(cycle_lock=2))
    assert orep.locked > 0
    P = pff.problem_from_workload(w)
    rep = P.solve_loading_steps([p], pff.options(cycle_lock=2))[0]
    assert rep["converged"] == 1 and rep["locked"] == orep.locked
    u, phi, act = P.get_solution()
    _assert_solution_parity(mesh, st, u, phi, act.astype(bool), "cycle_lock24")
    P.close()


def test_preconditioner_is_a_convergent_linear_map():
    rng = np.random.default_rng(31)
    coords = [W.graded_axis(40, 1.0, 0.01), W.graded_axis(34, 1.0, 0.02)]
    mesh = fe.Mesh(coords)
    n, d = mesh.n_nodes, 2
    phi_old = 1.0 - 0.1 * rng.random(n)
    u = 1e-3 * rng.standard_normal((n, d))
    u[mesh.boundary_nodes()] = 0.0
    P = pff.Problem(coords)
    P.set_material(1.0, 0.2, 1.0, 1e-10, 0.2)
    P.set_state(u, phi_old * 0.99, phi_old, phi_old, steps_done=1)
    P.set_pressure(1e-3)
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.active_set_dev(1.0, act, None)
    P.assemble()
    P.precond_setup(pff.options())
    N = P.n_dofs
    r1 = torch.tensor(rng.standard_normal(N), device="cuda")
    r2 = torch.tensor(rng.standard_normal(N), device="cuda")
    z1, z2, z3 = (torch.empty_like(r1) for _ in range(3))
    P.precond_apply_dev(r1, z1)
    P.precond_apply_dev(r2, z2)
    P.precond_apply_dev(2.0 * r1 - 3.0 * r2, z3)
    torch.cuda.synchronize()
    assert rel(z3.cpu().numpy(), (2.0 * z1 - 3.0 * z2).cpu().numpy()) <= 1e-12
    # the stationary iteration x <- x + V(b - A x) contracts on each diagonal block
    a = act.cpu().numpy().astype(bool)
    fixed = np.concatenate([np.repeat(mesh.boundary_nodes(), d), a])
    for blk, is_u in ((slice(0, d * n), True), (slice(d * n, N), False)):
        b = np.zeros(N)
        b[blk] = rng.standard_normal(b[blk].shape)
        b[fixed] = 0.0
        bd = torch.tensor(b, device="cuda")
        x = torch.zeros_like(bd)
        Ax = torch.empty_like(bd)
        z = torch.empty_like(bd)
        norms = []
        for _ in range(6):
            P.apply_jacobian_dev(pff.PFF_APPLY_ASSEMBLED, x, Ax)
            res = bd - Ax
            if is_u:
                res[d * n:] = 0.0
            norms.append(float(torch.linalg.norm(res[blk])))
            P.precond_apply_dev(res, z)
            x = x + z
        assert norms[-1] < 0.05 * norms[0], norms
    P.close()


@pytest.mark.parametrize("dim,shape,seed", [(2, (48, 40), 51), (3, (14, 12, 10), 52)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_sparse_kernel_variants_agree(dim, shape, seed, precision):
    """Every lane-group width of the vector block-sparse kernels and the SELL-32
    layout (SpMV, residual, Chebyshev step on the coarse levels and transfers)
    give the V-cycle of the row-per-thread reference kernels, up to the
    summation order."""
    P, mesh, prm, state = make_case(dim, shape, seed, p=1e-3)
    act = torch.empty(mesh.n_nodes, dtype=torch.uint8, device="cuda")
    P.active_set_dev(1.0, act, None)
    P.assemble()
    prec = pff.PFF_PREC_FP64 if precision == "fp64" else pff.PFF_PREC_MIXED
    rng = np.random.default_rng(seed)
    r = torch.tensor(rng.standard_normal(P.n_dofs), device="cuda")
    out = {}
    for g in (-1, 0, 1, 2, 4, 8, 16, 32, 64):
        # a small coarse level gives several block-sparse levels on these meshes
        P.precond_setup(pff.options(precision=prec, spmv_group=g, amg_coarse_max=24))
        z = torch.empty_like(r)
        P.precond_apply_dev(r, z)
        torch.cuda.synchronize()
        out[g] = z.cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-5
    for g in (0, 1, 2, 4, 8, 16, 32, 64):
        assert rel(out[g], out[-1]) <= tol, (g, rel(out[g], out[-1]))
    with pytest.raises(RuntimeError):
        P.precond_setup(pff.options(spmv_group=3))
    P.close()


@pytest.mark.parametrize("dim,shape,seed", [(2, (36, 22), 71), (3, (8, 6, 4), 72)])
def test_mixed_vcycle_matches_fp64_vcycle(dim, shape, seed):
    """The FP32 V-cycle and the FP64 V-cycle on the same hierarchy agree to FP32
    accuracy.  The FP32 level-0 kernels read only the symmetric half of each
    stencil (the other half transposed from the neighbours, 2d u in the
    node-major layout); the FP64 ones read the full stencil, so a wrong slot or
    a missing transpose shows here.  Node counts that are not multiples of 4
    exercise the ragged tail."""
    P, mesh, prm, state = make_case(dim, shape, seed, p=1e-3)
    assert mesh.n_nodes % 4 != 0
    act = torch.empty(mesh.n_nodes, dtype=torch.uint8, device="cuda")
    P.active_set_dev(1.0, act, None)
    P.assemble()
    r = torch.tensor(np.random.default_rng(seed).standard_normal(P.n_dofs), device="cuda")
    out = []
    for prec in (0, 1):
        P.precond_setup(pff.options(precision=prec, amg_coarse_max=24))
        z = torch.empty_like(r)
        P.precond_apply_dev(r, z)
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
    assert rel(out[1], out[0]) <= 1e-4, rel(out[1], out[0])
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_concurrent_block_vcycles_equal_sequential(precision):
    """The two diagonal blocks' V-cycles on two streams give the sequential result bit for bit."""
    P, mesh, prm, state = make_case(2, (40, 36), 61, p=1e-3)
    act = torch.empty(mesh.n_nodes, dtype=torch.uint8, device="cuda")
    P.active_set_dev(1.0, act, None)
    P.assemble()
    r = torch.tensor(np.random.default_rng(5).standard_normal(P.n_dofs), device="cuda")
    out = []
    for ov in (0, 1):
        P.precond_setup(pff.options(precision=precision, precond_overlap=ov, spmv_group=8))
        z = torch.empty_like(r)
        P.precond_apply_dev(r, z)
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    P.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_solve_matches_direct_solve(precision):
    """FGMRES to 1e-12 against a sparse direct solve of the reduced system; in
    mixed precision the preconditioner runs in FP32 and the Gram-Schmidt
    coefficients come from FP32 views, the Arnoldi update stays FP64."""
    P, mesh, prm, state = make_case(2, (30, 26), 41, p=1e-3)
    act = torch.empty(mesh.n_nodes, dtype=torch.uint8, device="cuda")
    P.active_set_dev(1.0, act, None)
    P.assemble()
    prec = pff.PFF_PREC_FP64 if precision == "fp64" else pff.PFF_PREC_MIXED
    opts = pff.options(tol_linear=1e-12, precision=prec, krylov_restart=20)
    P.precond_setup(opts)
    a = act.cpu().numpy().astype(bool)
    d, n = 2, mesh.n_nodes
    fixed = np.concatenate([np.repeat(mesh.boundary_nodes(), d), a])
    rng = np.random.default_rng(3)
    b = rng.standard_normal(P.n_dofs)
    b[fixed] = 0.0
    x = torch.zeros(P.n_dofs, dtype=torch.float64, device="cuda")
    its = P.linear_solve_dev(torch.tensor(b, device="cuda"), x, opts)
    u, phi, _, _, phit = state
    J = model.jacobian(mesh, prm, u, phi, phit)
    free = np.flatnonzero(~fixed)
    import scipy.sparse.linalg as spla
    xr = np.zeros(P.n_dofs)
    xr[free] = spla.spsolve(J[free][:, free].tocsc(), b[free])
    assert its > 0
    assert rel(x.cpu().numpy(), xr) <= 1e-8
    P.close()


def test_krylov_iterations_nearly_independent_of_h():
    """Table 1: GMRES iterations per Newton step of the block-AMG preconditioned
    system stay nearly constant under uniform refinement (the paper: 14-19 up to
    25-37 from 49,923 to 3,151,875 DoFs).  Uniform Sneddon meshes 128^2..512^2."""
    per_newton = []
    for cells in (128, 256, 512):
        w = W.scaled_workload(W.config(0), cells)
        P = pff.problem_from_workload(w)
        r = P.solve_loading_steps(w.pressures, pff.options(precision=1))[0]
        assert r["converged"] == 1
        per_newton.append(r["krylov_its"] / r["newton_its"])
        P.close()
    assert max(per_newton) <= 60, per_newton
    assert max(per_newton) <= 1.5 * min(per_newton), per_newton


def test_block_triangular_preconditioner_reaches_the_same_solution():
    """PFF_PC_AMG_TRI (the phase-field V-cycle sees r_phi - M_phi_u z_u) changes
    the path of FGMRES, not the converged Newton solution."""
    w = W.scaled_workload(W.config(1), 64)
    out = []
    for pc in (pff.PFF_PC_AMG, pff.PFF_PC_AMG_TRI):
        P = pff.problem_from_workload(w)
        reps = P.solve_loading_steps(w.pressures[:3], pff.options(precision=1, precond=pc))
        assert all(r["converged"] == 1 for r in reps)
        out.append(P.get_solution())
        P.close()
    assert rel(out[1][0], out[0][0]) <= 1e-9 and rel(out[1][1], out[0][1]) <= 1e-9



@pytest.mark.parametrize("dim", [2, 3])
def test_coarse_space_with_or_without_rotations_reaches_the_same_solution(dim):
    """The near-null space of the displacement hierarchy (rigid-body modes, or
    translations only) shapes the FGMRES path, not the converged Newton solution."""
    w = W.scaled_workload(W.config(1), 64) if dim == 2 else W.scaled_workload(W.config(2), 12)
    pressures = w.pressures[:2]
    out = []
    for rot in (0, 1):
        P = pff.problem_from_workload(w)
        reps = P.solve_loading_steps(pressures, pff.options(precision=1, amg_rotations=rot))
        assert all(r["converged"] == 1 for r in reps)
        out.append(P.get_solution())
        P.close()
    assert rel(out[1][0], out[0][0]) <= 1e-9 and rel(out[1][1], out[0][1]) <= 1e-9


_TILE_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import paper_1806_09924_gb300 as pff, workloads as W
w = W.scaled_workload(W.config(2), 10)
P = pff.problem_from_workload(w)
P.solve_loading_steps(w.pressures, pff.options(precision=1))
u, phi, act = P.get_solution()
np.savez({out!r}, u=u, phi=phi, act=act)
"""


def test_element_tiles_do_not_change_results(tmp_path):
    """The element kernels (residual, assembly, assembled apply) give bit-identical
    results whatever tile the autotuner picks: one 3d solve with each tile forced
    (PFF_ELEM_TILE, read once per process, so each runs in a child process).
    The two children share a tuning record, so that the other timed choices
    (sparse-kernel variants, which sum in different orders, and the apply
    variant) are the same in both: on matrices this small their timings are
    within noise and may fall either way in two processes."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    rec = str(tmp_path / "tune.txt")
    for tile in (64, 256):
        out = str(tmp_path / f"tile{tile}.npz")
        env = dict(os.environ, PFF_ELEM_TILE=str(tile), PFF_TUNE_CACHE=rec)
        subprocess.run([sys.executable, "-c", _TILE_CHILD.format(root=root, out=out)], env=env,
                       check=True, timeout=600)
        res.append(np.load(out))
    for k in ("u", "phi", "act"):
        assert np.array_equal(res[0][k], res[1][k]), k


def test_stencil_variants_do_not_change_results(tmp_path):
    """The 3d displacement smoother and residual have three kernel variants
    (node per thread; component rows with 4 or 3 resident blocks per SM) that
    accumulate in the same order: one 3d mixed-precision solve with each forced
    (PFF_STENCIL_VARIANT, read once per process) gives bit-identical results.
    The children share a tuning record, as in the element-tile test."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = str(tmp_path / "tune.txt")
    res = []
    for v in (0, 1, 2):
        out = str(tmp_path / f"variant{v}.npz")
        env = dict(os.environ, PFF_STENCIL_VARIANT=str(v), PFF_TUNE_CACHE=rec)
        subprocess.run([sys.executable, "-c", _TILE_CHILD.format(root=root, out=out)], env=env,
                       check=True, timeout=600)
        res.append(np.load(out))
    for r in res[1:]:
        for k in ("u", "phi", "act"):
            assert np.array_equal(res[0][k], r[k]), k


def test_tuning_record_replays_the_same_choices(tmp_path):
    """PFF_TUNE_CACHE: a first process records every autotuner choice (sparse
    formats, element tiles, apply variant); a second process with the same file
    reuses them without timing and reaches a bit-identical solution."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = str(tmp_path / "tune.txt")
    res = []
    for k in range(2):
        out = str(tmp_path / f"run{k}.npz")
        env = dict(os.environ, PFF_TUNE_CACHE=rec)
        env.pop("PFF_ELEM_TILE", None)
        subprocess.run([sys.executable, "-c", _TILE_CHILD.format(root=root, out=out)], env=env,
                       check=True, timeout=600)
        res.append(np.load(out))
        if k == 0:
            text = open(rec).read()
            assert "spmv:" in text and "tile:" in text and "apply:" in text, text
    for k in ("u", "phi", "act"):
        assert np.array_equal(res[0][k], res[1][k]), k
