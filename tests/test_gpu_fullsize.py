"""Parity at the benchmark sizes (1024^2 graded 2d, 128^3 graded 3d).

The oracle cannot assemble these meshes, but one row of the residual or of the
Jacobian involves only the 2^d cells around its node.  The oracle therefore
evaluates sampled rows on the 3^d-node patch cut out of the full mesh, and the
GPU rows of the full problem (computed in the launch configuration the bench
uses) must match them.  After a full-size Newton solve the complementarity
conditions of the Section 3 algorithm are checked directly (they hold at any
size).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fe, model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pff = pytest.importorskip("paper_1806_09924_gb300")

RTOL_OP = 1e-12


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def sample_nodes(w, rng, k):
    """Interior nodes: random ones plus the nodes around the crack tips."""
    nn = [len(c) for c in w.coords]
    picks = []
    for _ in range(k):
        picks.append([int(rng.integers(1, m - 1)) for m in nn])
    # around the tip x = l0 on the crack plane (y = 0, z = 0)
    mids = [int(np.argmin(np.abs(c))) for c in w.coords]
    tip = int(np.argmin(np.abs(w.coords[0] - w.l0)))
    for dx in (-2, -1, 0, 1, 2):
        for dy in (-1, 0, 1):
            p = list(mids)
            p[0] = tip + dx
            p[1] = mids[1] + dy
            picks.append(p)
    return picks


def patch(w, idx):
    """Patch mesh of the 2^d cells around node idx, the global ids of its nodes
    (x fastest) and the local id of the centre node."""
    d = w.dim
    nn = [len(c) for c in w.coords]
    coords = [w.coords[a][idx[a] - 1: idx[a] + 2] for a in range(d)]
    offs = np.indices([3] * d).reshape(d, -1)[::-1]       # offs[a] = axis-a offset, x fastest
    gid = np.zeros(offs.shape[1], dtype=np.int64)
    stride = 1
    for a in range(d):
        gid += (idx[a] - 1 + offs[a]) * stride
        stride *= nn[a]
    centre = 1 + 3 + (9 if d == 3 else 0)
    return fe.Mesh(coords), gid, centre


def global_boundary(w, gid):
    nn = [len(c) for c in w.coords]
    rem = gid.copy()
    on = np.zeros(len(gid), dtype=bool)
    for a in range(w.dim):
        i = rem % nn[a]
        rem //= nn[a]
        on |= (i == 0) | (i == nn[a] - 1)
    return on


@pytest.mark.parametrize("config", [1, 2])
def test_sampled_rows_at_full_size(config):
    w = W.config(config)
    d = w.dim
    u, phi, phi_old, _ = W.random_state(w, 7 + config, u_scale=1e-3)
    rng = np.random.default_rng(config)
    phi_prev = np.minimum(1.0, phi_old + 0.1 * rng.random(w.n_nodes))
    phit = np.clip(2 * phi_old - phi_prev, 0.0, 1.0)
    p = w.pressures[-1]
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p)
    P = pff.problem_from_workload(w, crack=False)
    P.set_state(u, phi, phi_old, phi_prev, steps_done=2)
    P.set_pressure(p)
    n, N = w.n_nodes, w.n_dofs
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    P.residual_dev(F)
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.active_set_dev(0.1, act, None)   # c in units of G_c / eps
    P.assemble()
    x = torch.tensor(rng.standard_normal(N), device="cuda")
    y = torch.empty_like(x)
    P.apply_jacobian_dev(pff.PFF_APPLY_ASSEMBLED, x, y)
    torch.cuda.synchronize()
    F, y, x, act = F.cpu().numpy(), y.cpu().numpy(), x.cpu().numpy(), act.cpu().numpy().astype(bool)
    P.close()
    got_F, ref_F, got_y, ref_y = [], [], [], []
    for idx in sample_nodes(w, rng, 150):
        mesh, gid, c = patch(w, idx)
        r_u, r_phi = model.gradient(mesh, prm, u[gid], phi[gid], phit[gid])
        g = gid[c]
        got_F += list(F[g * d: g * d + d]) + [F[d * n + g]]
        ref_F += list(-r_u[c]) + [-r_phi[c]]
        # reduced Jacobian rows: Dirichlet displacement and active phase-field
        # columns eliminated (identity rows where the row itself is eliminated)
        J = model.jacobian(mesh, prm, u[gid], phi[gid], phit[gid]).tocsr()
        npch = len(gid)
        col_g = np.concatenate([(gid[:, None] * d + np.arange(d)).ravel(), d * n + gid])
        fixed = np.concatenate([np.repeat(global_boundary(w, gid), d), act[gid]])
        xm = np.where(fixed, 0.0, x[col_g])
        rows = [c * d + a for a in range(d)] + [d * npch + c]
        for r in rows:
            got_y.append(y[col_g[r]])
            ref_y.append(x[col_g[r]] if fixed[r] else J[r].dot(xm)[0])
    assert rel(got_F, ref_F) <= RTOL_OP
    assert rel(got_y, ref_y) <= RTOL_OP


def lumped_mass(w):
    """m_i = integral of the Q1 basis function of node i: the product of the
    half-widths of the two cells on each side, per axis."""
    per_axis = []
    for c in w.coords:
        h = np.diff(c)
        m = np.zeros(len(c))
        m[:-1] += 0.5 * h
        m[1:] += 0.5 * h
        per_axis.append(m)
    out = per_axis[0]
    for a in range(1, w.dim):
        out = np.multiply.outer(per_axis[a], out).ravel()
    return out


@pytest.mark.parametrize("config", [1, 2])
def test_complementarity_after_full_size_solve(config):
    """The last loading step of the bench's workload (mixed precision), solved by
    single Newton / active-set iterations: irreversibility, phi = phi_old on the
    active set, a non-negative multiplier there and a vanishing one elsewhere."""
    w = W.config(config)
    d, n = w.dim, w.n_nodes
    P = pff.problem_from_workload(w)
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    reps = P.solve_loading_steps(w.pressures[:-1], opts)
    assert all(r["converged"] == 1 for r in reps)
    _, phi_old, _ = P.get_solution()
    P.set_pressure(w.pressures[-1])
    F0 = torch.empty(w.n_dofs, dtype=torch.float64, device="cuda")
    P.residual_dev(F0)
    for k in range(51):
        rep = P.newton_step(opts)
        if rep["converged"]:
            break
    assert rep["converged"] == 1
    u, phi, act = P.get_solution()
    F = torch.empty(w.n_dofs, dtype=torch.float64, device="cuda")
    P.residual_dev(F)
    F, F0 = F.cpu().numpy(), F0.cpu().numpy()
    P.close()
    act = act.astype(bool)
    scale = w.Gc / w.eps
    lam = F[d * n:] / lumped_mass(w)
    # phi = phi_old on the active set (nodes that joined it as ties in the last
    # iteration may still differ by the tie band); inactive nodes may sit above
    # phi_old by the threshold band of the rule (tau / c)
    assert np.max(np.abs(phi[act] - phi_old[act])) <= 1e-8
    assert np.max(phi - phi_old) <= 1e-8
    # dual feasibility on the active set, except where the cycle rule locked an
    # index active (the rule keeps such a node active whatever its multiplier)
    assert np.count_nonzero(lam[act] < -1e-8 * scale) <= rep["locked"]
    assert np.max(np.abs(lam[~act])) <= 1e-6 * scale
    # displacement rows: equilibrium on the free rows, relative to the step's load
    nn = [len(c) for c in w.coords]
    on = np.zeros(n, dtype=bool)
    rem = np.arange(n)
    for a in range(d):
        i = rem % nn[a]
        rem //= nn[a]
        on |= (i == 0) | (i == nn[a] - 1)
    free_u = ~np.repeat(on, d)
    assert np.max(np.abs(F[: d * n][free_u])) <= 1e-7 * np.max(np.abs(F0[: d * n][free_u]))
