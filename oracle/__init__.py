"""CPU oracle for the pressurized phase-field fracture hot path (FP64, plain numpy/scipy).

TEST INFRASTRUCTURE ONLY.  This package is the independent, slow, obviously
correct reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  It shares no code with the CUDA path: the only
module both sides import is ``workloads`` (seeded input generators without any
of the method's arithmetic).

Contents (each function cites the passage of the paper it follows):

* ``fe``          -- tensor-product Q1 mesh, reference element, 2^d Gauss rule.
* ``model``       -- residual of Formulation 1 (Eq. E22ATW / E33ATW), its
                     Jacobian blocks M_uu, M_phi_u, M_phi_phi (Section 3.1),
                     the energy whose gradient the residual is, lumped mass.
* ``pdas``        -- the combined semi-smooth Newton / primal-dual active set
                     loop (Section 3, commented algorithm) with exact block
                     solves, line search and cycle locking.
* ``functionals`` -- TCV and COD (Section 4) and Sneddon's closed forms.
* ``adapt``       -- refinement strategy of Section 3 on tensor-product meshes:
                     gradient-jump indicator, slab marking, Q1 transfer.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: exact symbolic integration, rigid-body and patch invariants, finite
differences of the energy and of the residual, brute-force dense and staggered
solves, KKT conditions, Table 1 DoF counts and Sneddon's closed forms.
"""
from . import fe, model, pdas, functionals, adapt  # noqa: F401
