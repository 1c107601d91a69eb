"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, and rejects invalid meshes and arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from _util import ROOT, ensure_lib
from paper_1710_08679_gb300 import fe
from paper_1710_08679_gb300 import meshgen as mg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ensure_lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fe.EXPORTED)


def test_version_and_defaults():
    lib = ensure_lib()
    assert b"sm_103a" in lib.fe_version()
    o = fe.SolveOpts()
    ctypes.memset(ctypes.byref(o), 0xFF, ctypes.sizeof(o))     # every field must be written by the default
    lib.fe_solve_opts_default(ctypes.byref(o))
    assert o.solver == fe.FE_SOLVER_FCG_MIXED and o.tol == 1e-8 and o.n_inner == 30 and o.eps_inner == 0.1
    assert o.n_inner1 == 300 and o.eps_inner1 == 0.05 and o.n_inner2 == 3000 and o.eps_inner2 == 0.025
    assert o.coarse_op == 0 and not o.cg_coef and o.cg_coef_len == 0 and o.inner_kernel == 1


def _create(m, **over):
    lib = ensure_lib()
    arrs = dict(coords=np.ascontiguousarray(m.coords, np.float64), conn=np.ascontiguousarray(m.conn, np.int32),
                young=np.ascontiguousarray(m.young, np.float64), poisson=np.ascontiguousarray(m.poisson, np.float64),
                free=np.ascontiguousarray(m.free, np.uint8))
    arrs.update(over)
    h = ctypes.c_void_p()
    st = lib.fe_mesh_create(arrs["coords"].shape[0], arrs["coords"].ctypes.data, arrs["conn"].shape[0],
                            arrs["conn"].ctypes.data, arrs["young"].ctypes.data, arrs["poisson"].ctypes.data,
                            arrs["free"].ctypes.data, 0, None, ctypes.byref(h))
    return st, lib.fe_last_error().decode(), h


@pytest.mark.parametrize("case", ["node_range", "repeat_node", "inverted", "not_midpoint", "nan_coord",
                                  "bad_young", "bad_poisson", "bad_mask"])
def test_invalid_mesh_rejected_on_host(case):
    m = mg.plain_box(n=2)
    over = {}
    if case == "node_range":
        c = m.conn.copy(); c[5, 2] = m.n_nodes; over["conn"] = c
    elif case == "repeat_node":
        c = m.conn.copy(); c[5, 2] = c[5, 1]; over["conn"] = c
    elif case == "inverted":
        c = m.conn.copy(); c[7, [1, 2]] = c[7, [2, 1]]; c[7, 4:] = c[7, [6, 5, 4, 7, 9, 8]]; over["conn"] = c
    elif case == "not_midpoint":
        x = m.coords.copy(); x[m.conn[3, 5]] += 10.0; over["coords"] = x
    elif case == "nan_coord":
        x = m.coords.copy(); x[11, 1] = np.nan; over["coords"] = x
    elif case == "bad_young":
        y = m.young.copy(); y[2] = -1.0; over["young"] = y
    elif case == "bad_poisson":
        p = m.poisson.copy(); p[2] = 0.5; over["poisson"] = p
    elif case == "bad_mask":
        f = m.free.copy(); f[3, 1] = 2; over["free"] = f
    st, msg, h = _create(m, **over)
    assert st == fe.FE_EINVAL, (st, msg)
    assert msg
    assert not h.value


def test_null_arguments_rejected():
    lib = ensure_lib()
    assert lib.fe_ebe_apply(None, 1, 0, None, None, None) == fe.FE_EINVAL
    assert b"NULL" in lib.fe_last_error()
    assert lib.fe_pcg_solve(None, 1, None, None, None, None, None) == fe.FE_EINVAL
    assert lib.fe_adjoint_grad(None, 1, None, None, None, None) == fe.FE_EINVAL
    assert lib.fe_wait_selftest(None, 0, 1000, None) == fe.FE_EINVAL
    lib.fe_mesh_destroy(None)
