"""The C ABI library loads without a GPU, exports every symbol declared in
include/blp.h, and its region-major layout is a bijection (host-side checks)."""
import ctypes
import os
import re

import pytest

from paper_2108_13468_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "blp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(blp_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, f"{name} has no ctypes signature"


def test_host_only_calls():
    lib = _native.load()
    assert lib.blp_strerror(0) == b"ok"
    assert b"coefficients" in lib.blp_strerror(2)
    p = _native.Params()
    lib.blp_params_default(ctypes.byref(p))
    assert p.restart == 30 and p.corner_reduction == 1e3 and p.sigma == 2.0
    import numpy as np
    x = np.zeros(129)
    tau = lib.blp_mesh(128, 1e-4, 2.0, 1.0, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert abs(tau - 2e-4 * np.log(128)) < 1e-18 and x[64] == tau and x[-1] == 1.0
    assert lib.blp_mesh(127, 1e-4, 2.0, 1.0, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) < 0
    h = ctypes.c_void_p()
    assert lib.blp_setup(None, None, None, None, ctypes.byref(h)) == _native.BLP_ERR_ARG


def test_library_mesh_matches_oracle_mesh():
    import numpy as np
    import oracle
    for N, eps in ((64, 1e-3), (1024, 1e-8), (96, 0.3)):
        x = np.zeros(N + 1)
        _native.load().blp_mesh(N, eps, 2.0, 1.0, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        np.testing.assert_array_equal(x, oracle.mesh(N, eps)[0])
        g = np.zeros(N + 1)
        _native.load().blp_mesh_graded(N, eps, 2.0, 1.0, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        np.testing.assert_array_equal(g, oracle.mesh(N, eps, graded=True)[0])
        pm = np.zeros(N + 1)   # eq. (tau parabolic), sigma = 5/2
        tau = _native.load().blp_mesh_parabolic(N, eps, 2.5, pm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        xo, tauo = oracle.mesh(N, eps, 2.5, 1.0, parabolic=True)
        assert tau == tauo
        np.testing.assert_array_equal(pm, xo)
    assert _native.load().blp_mesh_parabolic(63, 1e-4, 2.5, pm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) < 0
    for N, NL, eps in ((16, 4, 1e-3), (64, 48, 1e-6), (100, 30, 1e-2), (128, 64, 1e-8)):
        qm = np.zeros(N + 1)
        tau = _native.load().blp_mesh_q(N, NL, eps, 2.0, 1.0, qm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        xo, tauo = oracle.mesh(N, eps, layer_intervals=NL)
        assert tau == tauo
        np.testing.assert_array_equal(qm, xo)
    qm = np.zeros(17)
    assert _native.load().blp_mesh_q(16, 15, 1e-3, 2.0, 1.0, qm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) < 0


@pytest.mark.parametrize("N", [8, 10, 34, 64, 66, 96, 130])
def test_region_layout_is_a_bijection(N):
    lib = _native.load()
    npad = lib.blp_layout_npad(N)
    seen = {}
    for j in range(1, N):
        for i in range(1, N):
            p = lib.blp_layout_addr(N, i, j)
            assert 0 <= p < npad
            assert p not in seen
            seen[p] = (i, j)
    assert len(seen) == (N - 1) ** 2
    ii, jj = ctypes.c_int(), ctypes.c_int()
    valid = 0
    for p in range(npad):
        v = lib.blp_layout_node(N, p, ctypes.byref(ii), ctypes.byref(jj))
        if v == 1:
            valid += 1
            assert seen[p] == (ii.value, jj.value)
        else:
            assert p not in seen
    assert valid == (N - 1) ** 2
    assert npad % 32 == 0


def test_host_side_argument_checks_of_the_newer_entry_points():
    """Refusals that happen on the host, before any device work (no GPU here):
    null handles and arguments, invalid tuning values, invalid meshes, 1D
    problems with bad sizes or non-device arrays, and empty batches."""
    lib = _native.load()
    t = _native.Tuning(16, 8, 1, -1.0)
    assert lib.blp_get_tuning(None, ctypes.byref(t)) == _native.BLP_ERR_ARG
    assert lib.blp_set_tuning(None, ctypes.byref(t)) == _native.BLP_ERR_ARG
    assert lib.blp_autotune(None, _native.BLP_MIXED, 3, None) == _native.BLP_ERR_ARG
    x = (ctypes.c_double * 65)()
    assert lib.blp_mesh_graded(63, 1e-4, 2.0, 1.0, x) < 0 and lib.blp_mesh_graded(64, 0.0, 2.0, 1.0, x) < 0
    assert lib.blp_solve_batched_tuned(None, 0, 4) == _native.BLP_OK
    assert lib.blp_solve_batched_tuned(None, 3, 4) == _native.BLP_ERR_ARG
    assert lib.blp_solve_1d_batched(None, 0, None) == _native.BLP_OK
    assert lib.blp_solve_1d_batched(None, 1, None) == _native.BLP_ERR_ARG
    host = (ctypes.c_double * 63)()
    ptr = ctypes.cast(host, ctypes.c_void_p)
    probs = (_native.Problem1D * 3)()
    for k, (N, maxit) in enumerate([(64, 8), (63, 8), (64, _native.BLP_1D_MAXIT + 1)]):
        probs[k].N, probs[k].eps, probs[k].c_low, probs[k].sigma = N, 1e-4, 1.0, 2.0
        probs[k].c = probs[k].r = probs[k].f = probs[k].u = ptr     # host memory: refused
        probs[k].stop, probs[k].maxit = 1e-3, maxit
    assert lib.blp_solve_1d_batched(probs, 3, None) == _native.BLP_ERR_ARG
    assert [probs[k].status for k in range(3)] == [_native.BLP_ERR_ARG] * 3
    assert all(probs[k].iters == 0 and probs[k].resid == -1.0 for k in range(3))


STRUCTS = [("blp_params", _native.Params), ("blp_info", _native.Info), ("blp_batch_item", _native.BatchItem),
           ("blp_tuning", _native.Tuning), ("blp_1d_problem", _native.Problem1D)]


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs agree with the C compiler's layout
    of include/blp.h: size and every field's offset."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "blp.h"', "int main(void) {"]
    for cname, py in STRUCTS:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        struct, field, value = line.split()
        got[(struct, field)] = int(value)
    for cname, py in STRUCTS:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
