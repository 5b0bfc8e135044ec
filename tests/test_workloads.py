"""The seeded input generators hold the recipes the benchmarks and tests are
quoted on: mesh grading, the standard problems, the batched and served
instance sets, and the initial crack field (CPU only).

The expected values are the recipe's own statements (sizes, ratios, ranges,
DoF totals), closed forms (node counts of the cut cells) and invariants
(symmetry, reproducibility), not re-evaluations of the generator code.
"""
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("n,half,hmin", [(1024, 10.0, 2e-4), (128, 2.0, 4e-3), (40, 2.0, 0.025)])
def test_graded_axis_fills_the_box_geometrically(n, half, hmin):
    ax = W.graded_axis(n, half, hmin)
    assert len(ax) == n + 1
    assert ax[0] == -half and ax[-1] == half and ax[n // 2] == 0.0
    np.testing.assert_allclose(ax, -ax[::-1], rtol=0, atol=1e-15 * half)
    h = np.diff(ax)
    assert np.all(h > 0)
    right = h[n // 2:]
    assert right[0] == pytest.approx(hmin, rel=1e-12)
    ratios = right[1:-1] / right[:-2]
    assert np.ptp(ratios) < 1e-9 * ratios[0]   # one ratio throughout (the last cell absorbs rounding)
    assert right.sum() == pytest.approx(half, rel=1e-13)


def test_graded_axis_rejects_odd_or_too_coarse():
    with pytest.raises(ValueError):
        W.graded_axis(7, 1.0, 0.01)
    with pytest.raises(ValueError):
        W.graded_axis(8, 1.0, 0.5)          # 4 cells of 0.5 overfill the half width


def test_standard_problems():
    w0, w1, w2 = W.config(0), W.config(1), W.config(2)
    # uniform Sneddon, Table 1 refinement 4: [-2,2]^2, h = 1/32, eps = 2h
    assert w0.n_cells == [128, 128] and w0.h_min() == pytest.approx(1 / 32)
    assert w0.eps == pytest.approx(2 * w0.h_min()) and w0.pressures == [1e-3]
    # graded bench workload: 1024^2 on [-10,10]^2 from h_min = 2e-4, eps = 2 h_min,
    # ratio solved to fill the box, five loading steps p = 2e-4 n
    h1 = np.diff(w1.coords[0])
    assert w1.n_cells == [1024, 1024] and w1.n_dofs == 3_151_875
    assert w1.h_min() == pytest.approx(2e-4) and w1.eps == pytest.approx(2 * w1.h_min())
    assert h1[513] / h1[512] == pytest.approx(1.0126853, abs=1e-7)
    np.testing.assert_allclose(w1.pressures, [2e-4 * k for k in range(1, 6)], rtol=1e-15)
    assert w1.coords[0][0] == -10.0 and w1.precision == "mixed"
    # penny 3d: 128^3 on [-2,2]^3 from h_min = 4e-3, ratio 1.0532, radius 0.25
    h2 = np.diff(w2.coords[2])
    assert w2.n_cells == [128, 128, 128] and w2.n_dofs == 8_586_756
    assert h2[65] / h2[64] == pytest.approx(1.0532, abs=1e-4)
    assert w2.eps == pytest.approx(2 * w2.h_min()) and w2.l0 == 0.25


def test_scaled_workloads_keep_the_recipe():
    w = W.scaled_workload(W.config(1), 256)
    assert w.n_cells == [256, 256]
    assert w.h_min() == pytest.approx(2e-4 * 1024 / 256, rel=1e-12)
    assert w.eps == pytest.approx(2 * w.h_min(), rel=1e-12)
    assert w.coords[0][-1] == 10.0 and w.pressures == W.config(1).pressures
    u = W.scaled_workload(W.config(0), 64)
    assert u.h_min() == pytest.approx(4 / 64) and u.eps == pytest.approx(2 * 4 / 64)


def test_batched_instances():
    inst = W.batched_instances()
    assert len(inst) == 256
    assert sum(w.n_dofs for w in inst) == 29_182_488
    again = W.batched_instances()
    assert [w.name for w in again] == [w.name for w in inst]
    assert all(np.array_equal(a.coords[0], b.coords[0]) and a.pressures == b.pressures
               for a, b in zip(inst, again))
    other = W.batched_instances(seed=7)
    assert [w.name for w in other] != [w.name for w in inst]
    for w in inst:
        n = w.n_cells[0]
        assert w.dim == 2 and w.n_cells == [n, n] and n % 2 == 0 and 32 <= n <= 512
        h = 4.0 / n
        assert w.coords[0][0] == -2.0 and w.h_min() == pytest.approx(h)
        assert 1e-4 <= w.pressures[0] <= 1e-2 and len(w.pressures) == 1
        assert 0.1 <= w.l0 <= 0.5 and 0.15 <= w.nu <= 0.35
        assert 2 * h <= w.eps <= 4 * h * (1 + 1e-12)
        assert w.E == 1.0 and w.Gc == 1.0 and w.kappa == 1e-10
    sizes = [w.n_cells[0] for w in inst]
    assert min(sizes) < 48 and max(sizes) > 400      # log-uniform spread over the range


def test_served_requests():
    reqs = W.served_requests(200)
    dims = [w.dim for w, _ in reqs]
    assert 0.6 < dims.count(2) / len(dims) < 0.8     # 70 % 2d
    for w, gap in reqs:
        n = w.n_cells[0]
        assert n % 2 == 0 and w.n_cells == [n] * w.dim
        assert (64 <= n <= 1024) if w.dim == 2 else (32 <= n <= 128)
        assert w.h_min() == pytest.approx(0.25 * 4.0 / n, rel=1e-12)
        assert 2.0 - 1e-12 <= w.eps / w.h_min() <= 4.0 + 1e-12
        p = np.array(w.pressures)
        assert len(p) == 10
        np.testing.assert_allclose(p, p[-1] * np.arange(1, 11) / 10, rtol=1e-14)
        assert gap > 0
    first12 = W.served_requests(12)
    assert [w.dim for w, _ in first12].count(2) == 9    # the served bench's mix


def test_crack_field_2d():
    w = W.config(0)
    phi = w.phi0().reshape(129, 129)            # [j][i], x fastest
    assert set(np.unique(phi)) <= {0.0, 1.0}
    zj, zi = np.nonzero(phi == 0.0)
    x, y = w.coords[0], w.coords[1]
    # cells cut by the open segment |x| < 0.25 on y = 0 (a mesh line): the 16 cells
    # spanning [-0.25, 0.25] in x and the two rows on either side of y = 0, so the
    # nodes of x in [-0.25, 0.25] (17) times y in {-h, 0, h} (3)
    assert len(zi) == 17 * 3
    assert x[zi].min() == -0.25 and x[zi].max() == 0.25
    assert np.allclose(sorted(set(y[zj])), [-1 / 32, 0.0, 1 / 32])
    np.testing.assert_array_equal(phi, phi[::-1, :])
    np.testing.assert_array_equal(phi, phi[:, ::-1])


def test_crack_field_3d_penny():
    w = W.scaled_workload(W.config(2), 32)
    n = 33
    phi = w.phi0().reshape(n, n, n)             # [k][j][i]
    k0 = n // 2
    assert np.all(phi[: k0 - 1] == 1.0) and np.all(phi[k0 + 2:] == 1.0)   # only z in {-h, 0, h}
    np.testing.assert_array_equal(phi, phi[::-1])
    np.testing.assert_array_equal(phi, np.transpose(phi, (0, 2, 1)))      # x <-> y
    np.testing.assert_array_equal(phi, phi[:, ::-1, ::-1])
    x = w.coords[0]
    zk, zj, zi = np.nonzero(phi == 0.0)
    # every zero node lies within one cell of the disc of radius l0
    hmax = np.max(np.diff(x))
    r = np.hypot(x[zi], x[zj])
    assert r.max() < w.l0 + 2 * hmax and r.min() == 0.0


def test_plateau_axis_and_domain_study_recipe():
    """Section 4.2 stand-in meshes: uniform cells of size h on the crack region,
    geometric growth (ratio <= 1.05) to the box edges, eps = 2h, a node at 0."""
    for K, h in ((5.0, 0.01), (40.0, 0.00125)):
        x = W.plateau_axis(K, h, 1.25)
        dx = np.diff(x)
        assert x[0] == -K and x[-1] == K and np.all(dx > 0)
        assert np.any(np.abs(x) < 1e-12)
        plat = np.abs(x[:-1] + x[1:]) / 2 < 1.25
        np.testing.assert_allclose(dx[plat], h, rtol=1e-9)
        grow = dx[len(dx) // 2:][~plat[len(dx) // 2:]]
        assert np.all(grow[1:] / grow[:-1] <= 1.05 + 1e-12) and np.all(np.diff(grow) > 0)
        np.testing.assert_allclose(dx, dx[::-1], rtol=1e-9)
        w = W.domain_study(K, h)
        assert w.eps == 2 * h and w.l0 == 1.0 and w.pressures == [1e-3]
        assert w.h_min() == pytest.approx(h, rel=1e-9)
        # the crack |x| < 1 on y = 0 marks the nodes of its cut cells
        phi0 = w.phi0()
        assert phi0.min() == 0.0 and 0 < np.count_nonzero(phi0 == 0) < w.n_nodes // 10


def test_cyclic_loading_recipe():
    w = W.cyclic_loading(64)
    assert w.Gc == 1e-4 and w.n_cells == [64, 64] and w.eps == pytest.approx(2 * 4.0 / 64)
    p = w.pressures
    assert p == list(W.CYCLIC_PRESSURES)
    assert p[0] < p[1] < p[2] and p[2] > p[3] > p[4] and p[4] < p[5] < p[6] and p[6] > p[2]
    # the critical pressure of the sharp crack lies inside the schedule
    pc = math.sqrt(w.E * w.Gc / ((1 - w.nu ** 2) * math.pi * w.l0))
    assert min(p) < pc < max(p)
