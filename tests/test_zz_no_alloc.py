"""The allocation-free TCV / COD entry point agrees with the allocating one.

Some callers cannot let a library allocate device memory while they evaluate
the crack functionals: an application whose device memory is all handed out
by its own pool allocator, or that reserved the whole GPU up front, would see
an unplanned cudaMalloc fail.  pff_eval_tcv_cod_noalloc serves them from a
fixed scratch array inside the library.  It must return what pff_eval_tcv_cod
returns, also on a second call with fewer points (the scratch keeps the
previous call's contents), and it must refuse more points than its scratch
holds.
"""
import numpy as np
import pytest

import workloads as W
from oracle import functionals as fn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pff = pytest.importorskip("paper_1806_09924_gb300")

RTOL = 1e-12   # the tolerance the operator-level parity tests use


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_matches_allocating_entry_point_on_two_calls(dim):
    w = W.scaled_workload(W.config(0), 32) if dim == 2 else W.scaled_workload(W.config(2), 10)
    P = pff.problem_from_workload(w)
    P.solve_loading_steps(w.pressures[:1], pff.options(precision=pff.PFF_PREC_MIXED))
    if dim == 2:
        pts = np.concatenate([fn.cod_points(w.l0, 64), [w.coords[0][10]]])   # one on a mesh line
        second = pts[:7]
    else:
        xs = fn.cod_points(w.l0, 8)
        pts = np.stack([xs, np.zeros_like(xs)], axis=1).ravel()             # y = 0 is a mesh plane
        second = pts[:6]
    for call_pts in (pts, second):
        t_ref, c_ref = P.eval_tcv_cod(call_pts)
        t_na, c_na = P.eval_tcv_cod_noalloc(call_pts)
        assert _rel(t_na, t_ref) <= RTOL
        assert c_na.shape == c_ref.shape
        assert _rel(c_na, c_ref) <= RTOL
    P.close()


def test_noalloc_rejects_more_points_than_its_scratch():
    w = W.scaled_workload(W.config(0), 16)
    P = pff.problem_from_workload(w)
    too_many = np.zeros(pff.PFF_NOALLOC_MAX_POINTS + 1)
    with pytest.raises(pff.PffError) as e:
        P.eval_tcv_cod_noalloc(too_many)
    assert e.value.code == pff.PFF_ERR_CAPACITY
    # a call at the limit still works
    t, c = P.eval_tcv_cod_noalloc(np.zeros(pff.PFF_NOALLOC_MAX_POINTS))
    assert c.shape == (pff.PFF_NOALLOC_MAX_POINTS,)
    P.close()
