"""Write stored oracle solutions for GPU parity tests whose oracle run is too slow to repeat.

Only the CPU oracle (``oracle/``) and the seeded input generators
(``workloads/``) are called here; nothing comes from the CUDA path.  Each
fixture records the sha256 of the oracle sources and of the inputs it was
made from, so a test can tell when either changed and the fixture is stale.

    python tests/golden/make_oracle_fixtures.py            # every fixture
    python tests/golden/make_oracle_fixtures.py penny3d_32

Fixtures:
  penny3d_32  -- the penny-shaped crack recipe (graded, Section 4.3 geometry
                 scaled to 32^3 cells, 143,748 DoFs), one loading step at
                 p = 1e-3: u, phi, the final active set and indicator, TCV.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SOURCES = ("oracle/__init__.py", "oracle/fe.py", "oracle/model.py", "oracle/pdas.py",
           "oracle/functionals.py")


def source_hash() -> str:
    """sha256 of the oracle's sources."""
    h = hashlib.sha256()
    for rel in SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode())
            h.update(f.read())
    return h.hexdigest()


def input_hash(w, pressures) -> str:
    """sha256 of a workload's inputs: mesh coordinates, material, crack field, loads."""
    h = hashlib.sha256()
    for c in w.coords:
        h.update(np.ascontiguousarray(c, dtype=np.float64).tobytes())
    h.update(np.array([w.E, w.nu, w.Gc, w.kappa, w.eps, w.l0, *pressures], dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(w.phi0(), dtype=np.float64).tobytes())
    return h.hexdigest()


def penny3d_32_workload():
    import workloads as W
    return W.scaled_workload(W.config(2), 32), [1e-3]


def fixture_path(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.npz")


def _penny3d_32():
    from oracle import fe, functionals as fn, model, pdas
    w, pressures = penny3d_32_workload()
    mesh = fe.Mesh(w.coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=pressures[0])
    st = pdas.State.initial(mesh, prm, w.phi0())
    reps = pdas.solve_loading_steps(st, pressures)
    assert all(r.converged for r in reps)
    return dict(name=w.name, n_dofs=w.n_dofs, pressures=np.array(pressures),
                input_sha256=input_hash(w, pressures), u=st.u, phi=st.phi,
                active=st.active.astype(np.uint8), indicator=st.indicator,
                tcv=fn.tcv(mesh, st.u, st.phi), locked=np.array([r.locked for r in reps]),
                newton_its=np.array([r.newton_its for r in reps]))


FIXTURES = {"penny3d_32": _penny3d_32}


def main(names):
    for name in names or FIXTURES:
        t = time.time()
        data = FIXTURES[name]()
        np.savez_compressed(fixture_path(name), source_sha256=source_hash(), **data)
        print(f"{name}: {time.time() - t:.1f} s -> {fixture_path(name)}")


if __name__ == "__main__":
    main(sys.argv[1:])
