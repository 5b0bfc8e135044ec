"""CPU checks of the C ABI: the library builds, loads, exports every entry point
declared in include/pff.h, and its structs have the layout the binding assumes.
No compute call is made (there may be no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pff.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G
    B = G._build_module()
    if not os.path.exists(B.LIB):
        B.build()
    import paper_1806_09924_gb300 as pff
    return pff.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pff_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    import paper_1806_09924_gb300 as pff
    assert set(declared_functions()) == set(pff._SIGS)


def test_struct_layout_matches_header(tmp_path):
    """Every field of the binding's structs sits at the header's offset."""
    import paper_1806_09924_gb300 as pff
    structs = {"pff_options": pff.PffOptions, "pff_step_report": pff.PffStepReport,
               "pff_request": pff.PffRequest, "pff_request_result": pff.PffRequestResult,
               "pff_server_stats": pff.PffServerStats}
    lines = []
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "sz.c"
    src.write_text('#include "pff.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                   + "".join(lines) + "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        cname, field, value = line.split()
        cls = structs[cname]
        if field == "size":
            assert int(value) == ctypes.sizeof(cls), cname
        else:
            assert int(value) == getattr(cls, field).offset, (cname, field)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_defaults_and_argument_errors_without_gpu(lib):
    import paper_1806_09924_gb300 as pff
    o = pff.options()
    assert o.tol_linear == 1e-8 and o.c == 0.1 and o.amg_theta == 0.02 and o.precision == pff.PFF_PREC_FP64
    assert o.tol_active == 1e-10 and o.tol_change == 1e-9 and o.atol_newton == 1e-14
    assert o.krylov_restart == 40 and o.max_newton == 50
    assert o.spmv_group == 0 and o.amg_reuse == 1 and o.amg_reuse_tol == 0.05
    assert o.precond_overlap == 1 and o.iter_graph == 1 and o.cheb_degree_coarse == -1
    assert o.amg_rotations == -1
    assert o.cheb_degree == 4 and o.cheb_degree_phi == 4 and o.amg_levels_phi == -1
    assert o.amg_coarse_max == 1000
    assert o.forcing_max == 0.0
    assert o.amg_rebuild_phi == 1e-3 and o.amg_age_phi == 8
    h = ctypes.c_void_p()
    nc = (ctypes.c_int32 * 3)(4, 4, 4)
    # invalid dimension is rejected before any device work
    rc = lib.pff_create_mesh(5, nc, None, ctypes.byref(h))
    assert rc == pff.PFF_ERR_INVALID_ARG
    assert b"dim" in lib.pff_last_error()
    assert lib.pff_set_pressure(None, 1e-3) == pff.PFF_ERR_INVALID_ARG
    assert lib.pff_newton_step(None, None, None) == pff.PFF_ERR_INVALID_ARG


def test_degenerate_meshes_are_rejected_without_gpu(lib):
    """Zero cells, missing axes and coordinates that are not finite and strictly
    increasing are argument errors, found before any device work."""
    import numpy as np
    import paper_1806_09924_gb300 as pff
    h = ctypes.c_void_p()

    def create(dim, axes):
        nc = (ctypes.c_int32 * 3)(*[len(a) - 1 if a is not None else 1 for a in axes], *([1] * (3 - dim)))
        keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in axes]
        ptrs = (ctypes.POINTER(ctypes.c_double) * dim)(
            *[k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if k is not None else None for k in keep])
        rc = lib.pff_create_mesh(dim, nc, ptrs, ctypes.byref(h))
        return rc, lib.pff_last_error()

    good = np.linspace(-1.0, 1.0, 5)
    cases = {
        "zero cells": (2, [np.array([0.0]), good], b"n_cells"),
        "missing axis": (2, [good, None], b"NULL"),
        "repeated coordinate": (2, [good, np.array([0.0, 0.5, 0.5, 1.0])], b"strictly increasing"),
        "decreasing": (3, [good, good, good[::-1].copy()], b"strictly increasing"),
        "nan": (2, [good, np.array([0.0, np.nan, 1.0])], b"finite"),
        "inf at the end": (2, [np.array([0.0, 1.0, np.inf]), good], b"finite"),
    }
    for name, (dim, axes, why) in cases.items():
        rc, msg = create(dim, axes)
        assert rc == pff.PFF_ERR_INVALID_ARG, name
        assert why in msg, (name, msg)


def test_option_ranges_without_gpu(lib):
    """pff_check_options accepts the defaults and rejects each out-of-range field
    with its reason; a server is not created with invalid options."""
    import paper_1806_09924_gb300 as pff
    pff.check_options(pff.options())
    assert lib.pff_check_options(None) == pff.PFF_OK
    bad = [dict(precision=7), dict(krylov_restart=0), dict(cheb_degree=0), dict(max_newton=-1),
           dict(tol_change=-1.0), dict(amg_reuse_tol=-0.1), dict(forcing_max=1.0), dict(precond=9),
           dict(spmv_group=3), dict(amg_rebuild_phi=-1e-3), dict(amg_age_phi=0),
           dict(amg_levels_phi=-2), dict(cheb_degree_phi=-1), dict(amg_rotations=2),
           dict(amg_rotations=-2), dict(cheb_degree_coarse=-2)]
    for kw in bad:
        with pytest.raises(pff.PffError) as e:
            pff.check_options(pff.options(**kw))
        assert e.value.code == pff.PFF_ERR_INVALID_ARG, kw
    h = ctypes.c_void_p()
    o = pff.options(amg_age_phi=0)
    assert lib.pff_server_create(1 << 30, 1, ctypes.byref(o), ctypes.byref(h)) == pff.PFF_ERR_INVALID_ARG
    assert b"amg_age_phi" in lib.pff_last_error()


def test_server_host_logic_without_gpu(lib):
    """Argument checks, the admission estimate and the request queue need no GPU
    (workers that cannot get a stream leave the queue untouched)."""
    import paper_1806_09924_gb300 as pff
    b2 = pff.request_bytes(2, [64, 64])
    assert 0 < b2 < pff.request_bytes(2, [128, 128]) < pff.request_bytes(2, [256, 256])
    # per DoF a 3d problem needs more (27-point stencils)
    assert (pff.request_bytes(3, [96, 96, 96]) / (4 * 97 ** 3)
            > pff.request_bytes(2, [1024, 1024]) / (3 * 1025 ** 2))
    assert lib.pff_request_bytes(4, (ctypes.c_int32 * 3)(2, 2, 2)) == -1
    h = ctypes.c_void_p()
    assert lib.pff_server_create(0, 1, None, ctypes.byref(h)) == pff.PFF_ERR_INVALID_ARG
    assert lib.pff_server_create(1 << 30, 0, None, ctypes.byref(h)) == pff.PFF_ERR_INVALID_ARG
    if torch_gpu():
        return
    S = pff.Server(1 << 30, 2)
    bad = pff.PffRequest()
    bad.dim = 5
    rid = ctypes.c_int64()
    assert lib.pff_server_submit(S._h, ctypes.byref(bad), ctypes.byref(rid)) == pff.PFF_ERR_INVALID_ARG
    import workloads as W
    w = W.config(0)
    r = S.submit(w)
    res = S.result(r)
    assert res["done"] == 0 and res["n_dofs"] == w.n_dofs and res["bytes"] == pff.request_bytes(2, [128, 128])
    with pytest.raises(pff.PffError):
        S.wait(r, timeout=0.05)
    with pytest.raises(pff.PffError):
        S.release(r)          # not finished
    st = S.stats()
    assert st["queued"] == 1 and st["running"] == 0 and st["finished"] == 0
    S.close()                 # drops the queued request


def torch_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
