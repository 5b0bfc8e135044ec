"""Batch executor and request server (many independent problems on one GPU).

A problem's result must not depend on what else runs: solved in a batch or in
a mix of concurrent requests it equals the one-at-a-time solve (same kernels,
same autotuned variants, deterministic reductions), and one instance is
checked against the oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from oracle import fe, model, pdas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pff = pytest.importorskip("paper_1806_09924_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def small_instances(k, max_n=96):
    out = [w for w in W.batched_instances() if len(w.coords[0]) - 1 <= max_n]
    return out[:k]


def small_requests():
    """Served-style requests at small sizes: graded 2d and one 3d, three steps each."""
    reqs = []
    for n, d in ((40, 2), (64, 2), (48, 2), (12, 3), (80, 2)):
        ax = W.graded_axis(n, 2.0, 0.25 * 4.0 / n)
        hmin = float(np.min(np.diff(ax)))
        reqs.append(W.Workload(f"small_{d}d_{n}", d, [ax.copy() for _ in range(d)], nu=0.25,
                               eps=2.5 * hmin, l0=0.3, pressures=[1e-3, 2e-3, 3e-3],
                               precision="mixed"))
    return reqs


def test_batch_solve_matches_one_at_a_time_and_oracle():
    inst = small_instances(6)
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    alone = []
    for w in inst:
        P = pff.problem_from_workload(w)
        reps = P.solve_loading_steps(w.pressures, opts)
        assert all(r["converged"] == 1 for r in reps)
        alone.append(P.get_solution())
        P.close()
    probs = [pff.problem_from_workload(w) for w in inst]
    reports, status = pff.batch_solve(probs, [w.pressures for w in inst], opts, workers=3)
    assert status == [0] * len(inst)
    for w, P, reps, (u0, phi0, a0) in zip(inst, probs, reports, alone):
        assert reps[0]["converged"] == 1
        u, phi, act = P.get_solution()
        assert rel(u, u0) <= 1e-12 and rel(phi, phi0) <= 1e-12, w.name
        assert np.array_equal(act, a0), w.name
    # the smallest instance against the oracle
    i = int(np.argmin([len(w.coords[0]) for w in inst]))
    w = inst[i]
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    rep = pdas.loading_step(st, w.pressures[0])
    assert rep.converged
    u, phi, _ = probs[i].get_solution()
    assert rel(u, st.u) <= 1e-8 and rel(phi, st.phi) <= 1e-8
    for P in probs:
        P.close()


def test_iteration_graph_gives_the_direct_launch_result():
    """On a non-default stream a small problem runs each FGMRES iteration's
    preconditioner and Jacobian apply as one CUDA graph: the same kernels in the
    same order, so the solution is bit-identical to ordinary launches."""
    w = W.scaled_workload(W.config(1), 96)
    stream = torch.cuda.Stream()
    out = []
    for g in (0, 1):
        P = pff.problem_from_workload(w)
        P.set_stream(stream)
        reps = P.solve_loading_steps(w.pressures[:3], pff.options(precision=1, iter_graph=g))
        assert all(r["converged"] == 1 for r in reps)
        out.append((P.get_solution(), [r["krylov_its"] for r in reps]))
        P.close()
    (u0, phi0, a0), k0 = out[0]
    (u1, phi1, a1), k1 = out[1]
    assert k0 == k1
    assert np.array_equal(u0, u1) and np.array_equal(phi0, phi1) and np.array_equal(a0, a1)


def test_server_result_is_the_same_alone_and_in_the_mix():
    reqs = small_requests()
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    budget = 64 << 30
    cod_x = [0.0, 0.1]
    alone = {}
    S = pff.Server(budget, 1, opts)
    for w in reqs:
        rid = S.submit(w, cod_x=cod_x, keep_solution=True)
        res = S.wait(rid, timeout=300)
        assert res["status"] == 0 and res["converged_steps"] == len(w.pressures)
        alone[w.name] = (S.solution(rid), res["tcv"], S.cod(rid))
        S.release(rid)
    S.close()
    S = pff.Server(budget, 4, opts)
    ids = [S.submit(w, cod_x=cod_x, keep_solution=True) for w in reqs]
    for w, rid in zip(reqs, ids):
        res = S.wait(rid, timeout=300)
        assert res["status"] == 0 and res["converged_steps"] == len(w.pressures)
        (u, phi, act) = S.solution(rid)
        (u0, phi0, a0), tcv0, cod0 = alone[w.name]
        assert rel(u, u0) <= 1e-12 and rel(phi, phi0) <= 1e-12, w.name
        assert np.array_equal(act, a0), w.name
        assert rel(res["tcv"], tcv0) <= 1e-12 and rel(S.cod(rid), cod0) <= 1e-12
        # the served COD lines are those of pff_eval_tcv_cod on the returned solution:
        # along y at each abscissa (2d), along z through y = 0 (3d)
        Q = pff.Problem(w.coords)
        Q.set_material(w.E, w.nu, w.Gc, w.kappa, w.eps)
        Q.set_state(u, phi, phi, phi, 1)
        pts = np.array(cod_x) if w.dim == 2 else np.stack([cod_x, np.zeros(len(cod_x))], 1).ravel()
        tcv_q, cod_q = Q.eval_tcv_cod(pts)
        Q.close()
        assert rel(S.cod(rid), cod_q) <= 1e-12 and rel(res["tcv"], tcv_q) <= 1e-12
        S.release(rid)
    st = S.stats()
    assert st["finished"] == len(reqs) and st["max_running"] >= 2, st
    S.close()


def test_server_admission_respects_the_memory_budget():
    reqs = small_requests()
    est = [pff.request_bytes(w.dim, [len(c) - 1 for c in w.coords]) for w in reqs]
    budget = int(1.5 * max(est))
    S = pff.Server(budget, 4)
    ids = [S.submit(w) for w in reqs]
    res = [S.wait(rid, timeout=300) for rid in ids]
    assert all(r["status"] == 0 for r in res)
    st = S.stats()
    assert st["peak_reserved_bytes"] <= budget, st
    # FIFO: admissions in submission order
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)
    # a request larger than the whole budget still runs, alone
    S.close()
    S = pff.Server(min(est) // 2, 2)
    ids = [S.submit(w) for w in reqs[:3]]
    res = [S.wait(rid, timeout=300) for rid in ids]
    assert all(r["status"] == 0 for r in res)
    assert S.stats()["max_running"] == 1
    for a, b in zip(res, res[1:]):
        assert b["t_admit"] >= a["t_finish"]
    S.close()


_MEASURE = r"""
import sys, json
sys.path.insert(0, {root!r})
import numpy as np
import paper_1806_09924_gb300 as pff
import workloads as W
d, n = {dim}, {n}
ax = W.graded_axis(n, 2.0, 0.25 * 4.0 / n)
w = W.Workload("m", d, [ax.copy() for _ in range(d)], nu=0.2, eps=2.5 * float(np.min(np.diff(ax))),
               l0=0.3, pressures=[1e-3, 2e-3], precision="mixed")
S = pff.Server(1 << 40, 1, pff.options(precision=1))
res = S.wait(S.submit(w), timeout=600)
S.close()
print(json.dumps({{"status": res["status"], "used": pff.memory_usage()[1], "est": res["bytes"]}}))
"""


@pytest.mark.parametrize("dim,n", [(2, 256), (2, 1024), (3, 24)])
def test_request_estimate_covers_device_memory(dim, n):
    """The admission estimate bounds the peak device memory the library holds
    while one request runs (a fresh process, so nothing else is counted)."""
    import json
    out = subprocess.run([sys.executable, "-c", _MEASURE.format(root=ROOT, dim=dim, n=n)],
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["status"] == 0
    assert 0 < r["used"] <= r["est"], r
