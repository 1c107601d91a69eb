"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never loads it, and it
never loads the product library: the two share no code. What it computes and the
passages it follows are documented in ``fe_oracle.c``; this module is argument
marshalling (numpy <-> C) plus thin library-primitive steps (scipy's sparse direct
solve) used by the pins.

Functions whose parity with the paper is checked by the pin tests:
  element_stiffness, assemble, spmv, sampled_product, block_jacobi, pcg,
  fcg_mixed, adjoint_grad.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile fe_oracle.c with gcc (no FMA contraction, so results do not depend on
    the host architecture's fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = configure(ctypes.CDLL(_LIB))
    return _lib


def configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    if True:
        lib.oracle_tet10_stiffness.argtypes = [_f64p, ctypes.c_double, ctypes.c_double, _f64p]
        lib.oracle_pattern.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i64p, _i32p]
        lib.oracle_pattern.restype = ctypes.c_int64
        lib.oracle_assemble.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p, _f64p, _f64p,
                                        _i64p, _i32p, _f64p]
        lib.oracle_apply_bc.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _u8p]
        lib.oracle_spmv.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int, _f64p, _f64p]
        lib.oracle_spmv.restype = None
        lib.oracle_sampled_product.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p, _f64p, _f64p,
                                               _u8p, ctypes.c_int, _f64p, ctypes.c_int64, _i64p, _f64p]
        lib.oracle_block_jacobi.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p]
        lib.oracle_pcg.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int, _f64p, _f64p,
                                   ctypes.c_double, ctypes.c_int, _i32p, _f64p]
        lib.oracle_fcg_mixed.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int, _f64p,
                                         _f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, _i32p, _i32p, _f64p]
        lib.oracle_adjoint_grad.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p, _f64p, _f64p, _u8p,
                                            ctypes.c_int, _f64p, _f64p, _f64p]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        lib.oracle_pattern_n.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _i32p, _i64p, _i32p]
        lib.oracle_pattern_n.restype = ctypes.c_int64
        lib.oracle_tet4_stiffness.argtypes = [_f64p, ctypes.c_double, ctypes.c_double, _f64p]
        lib.oracle_assemble4.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p, _f64p, _f64p, _i64p, _i32p,
                                         _f64p]
        lib.oracle_prolong.argtypes = [ctypes.c_int64, ctypes.c_int, _i32p, _f64p, _f64p]
        lib.oracle_prolong.restype = None
        lib.oracle_restrict.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _i32p, _f64p, _f64p]
        lib.oracle_restrict.restype = None
        lib.oracle_fcg_mg.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int, _f64p, _f64p,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      _u8p, ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _u8p, _i32p, ctypes.c_int,
                                      ctypes.c_double, _i32p, _i32p, _i32p, _f64p]
        lib.oracle_aggregate.argtypes = [ctypes.c_int64, _i64p, _i32p, _i32p]
        lib.oracle_aggregate.restype = ctypes.c_int64
        lib.oracle_galerkin_agg.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _u8p, _i32p, ctypes.c_int64,
                                            _i64p, _i32p, _f64p, _u8p]
        lib.oracle_galerkin_agg.restype = ctypes.c_int64
        lib.oracle_fcg_ml.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int, _f64p, _f64p,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      _u8p, ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _u8p, _i32p, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _i32p,
                                      ctypes.c_int, ctypes.c_double, _i32p, _i32p, _i32p, _i32p, _f64p]
    return lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (timing of the CPU baseline)."""
    _load().oracle_set_num_threads(int(n))


def element_stiffness(xe: np.ndarray, E: float, nu: float) -> np.ndarray:
    """30x30 stiffness of one TET10 (nodes xe [10, 3], VTK order)."""
    lib = _load()
    xe = _c(xe, np.float64).reshape(30)
    Ke = np.zeros(900)
    rc = lib.oracle_tet10_stiffness(_p(xe, _f64p), float(E), float(nu), _p(Ke, _f64p))
    if rc != 0:
        raise ValueError("non-positive element Jacobian")
    return Ke.reshape(30, 30)


@dataclass
class Assembled:
    """Node-block CSR matrix: block b of row n couples nodes n and col[b]."""
    n_nodes: int
    rowptr: np.ndarray  # int64 [N+1]
    col: np.ndarray     # int32 [nnzb]
    vals: np.ndarray    # float64 [nnzb, 3, 3]

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.vals, self.col.astype(np.int64), self.rowptr),
                             shape=(3 * self.n_nodes, 3 * self.n_nodes)).tocsr()

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def _mesh_arrays(mesh):
    return (_c(mesh.coords, np.float64), _c(mesh.conn, np.int32), _c(mesh.young, np.float64),
            _c(mesh.poisson, np.float64), _c(mesh.free, np.uint8))


def assemble(mesh, apply_bc: bool = True, young=None) -> Assembled:
    """K (or K_bc = P K P + (I - P) when apply_bc) of a mesh-like object with
    attributes coords, conn, young, poisson, free."""
    lib = _load()
    coords, conn, E, nu, free = _mesh_arrays(mesh)
    if young is not None:
        E = _c(young, np.float64)
    N, Ne = coords.shape[0], conn.shape[0]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    nnzb = lib.oracle_pattern(N, Ne, _p(conn, _i32p), _p(rowptr, _i64p), None)
    if nnzb < 0:
        raise ValueError("bad connectivity")
    col = np.zeros(nnzb, dtype=np.int32)
    lib.oracle_pattern(N, Ne, _p(conn, _i32p), _p(rowptr, _i64p), _p(col, _i32p))
    vals = np.zeros((nnzb, 3, 3))
    rc = lib.oracle_assemble(N, _p(coords, _f64p), Ne, _p(conn, _i32p), _p(E, _f64p), _p(nu, _f64p),
                             _p(rowptr, _i64p), _p(col, _i32p), _p(vals, _f64p))
    if rc != 0:
        raise ValueError("assembly failed (%d)" % rc)
    if apply_bc:
        lib.oracle_apply_bc(N, _p(rowptr, _i64p), _p(col, _i32p), _p(vals, _f64p), _p(free, _u8p))
    return Assembled(N, rowptr, col, vals)


def spmv(K: Assembled, x: np.ndarray) -> np.ndarray:
    """y [N, R, 3] = K x for x [N, R, 3]."""
    lib = _load()
    x = _c(x, np.float64)
    R = x.shape[1]
    y = np.empty_like(x)
    lib.oracle_spmv(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p), R,
                    _p(x, _f64p), _p(y, _f64p))
    return y


def sampled_product(mesh, x: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Rows `nodes` of K_bc x, element by element, without full assembly: [S, R, 3]."""
    lib = _load()
    coords, conn, E, nu, free = _mesh_arrays(mesh)
    x = _c(x, np.float64)
    nodes = _c(nodes, np.int64)
    R = x.shape[1]
    ys = np.zeros((nodes.shape[0], R, 3))
    rc = lib.oracle_sampled_product(coords.shape[0], _p(coords, _f64p), conn.shape[0], _p(conn, _i32p),
                                    _p(E, _f64p), _p(nu, _f64p), _p(free, _u8p), R, _p(x, _f64p),
                                    nodes.shape[0], _p(nodes, _i64p), _p(ys, _f64p))
    if rc != 0:
        raise ValueError("sampled product failed (%d)" % rc)
    return ys


def block_jacobi(K: Assembled) -> np.ndarray:
    """Inverse 3x3 diagonal blocks [N, 3, 3]."""
    lib = _load()
    Minv = np.zeros((K.n_nodes, 3, 3))
    rc = lib.oracle_block_jacobi(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p),
                                 _p(Minv, _f64p))
    if rc != 0:
        raise ValueError("singular diagonal block (%d)" % rc)
    return Minv


def pcg(K: Assembled, f: np.ndarray, u0=None, tol: float = 1e-8, maxit: int = 100000, Minv=None):
    """PCG with 3x3 block Jacobi for every case: returns (u, iters, true relres)."""
    lib = _load()
    f = _c(f, np.float64)
    R = f.shape[1]
    u = np.zeros_like(f) if u0 is None else _c(u0, np.float64).copy()
    Minv = block_jacobi(K) if Minv is None else _c(Minv, np.float64)
    iters = np.zeros(R, dtype=np.int32)
    rel = np.zeros(R)
    lib.oracle_pcg(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p), _p(Minv, _f64p), R,
                   _p(f, _f64p), _p(u, _f64p), float(tol), int(maxit), _p(iters, _i32p), _p(rel, _f64p))
    return u, iters, rel


def fcg_mixed(K: Assembled, f: np.ndarray, u0=None, tol: float = 1e-8, max_outer: int = 10000,
              n_inner: int = 30, eps_inner: float = 0.1, literal_beta: bool = False, Minv=None):
    """Flexible CG (FP64) with FP32 inner block-Jacobi PCG: (u, outer, inner_total, relres)."""
    lib = _load()
    f = _c(f, np.float64)
    R = f.shape[1]
    u = np.zeros_like(f) if u0 is None else _c(u0, np.float64).copy()
    Minv = block_jacobi(K) if Minv is None else _c(Minv, np.float64)
    outer = np.zeros(R, dtype=np.int32)
    inner = np.zeros(R, dtype=np.int32)
    rel = np.zeros(R)
    lib.oracle_fcg_mixed(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p), _p(Minv, _f64p),
                         R, _p(f, _f64p), _p(u, _f64p), float(tol), int(max_outer), int(n_inner),
                         float(eps_inner), int(bool(literal_beta)), _p(outer, _i32p), _p(inner, _i32p),
                         _p(rel, _f64p))
    return u, outer, inner, rel


def adjoint_grad(mesh, u: np.ndarray, lam: np.ndarray, young=None) -> np.ndarray:
    """g[e] = -sum_r (P lam_r)_e^T K_e (P u_r)_e  (derivative w.r.t. log E_e)."""
    lib = _load()
    coords, conn, E, nu, free = _mesh_arrays(mesh)
    if young is not None:
        E = _c(young, np.float64)
    u = _c(u, np.float64)
    lam = _c(lam, np.float64)
    R = u.shape[1]
    g = np.zeros(conn.shape[0])
    rc = lib.oracle_adjoint_grad(coords.shape[0], _p(coords, _f64p), conn.shape[0], _p(conn, _i32p), _p(E, _f64p),
                                 _p(nu, _f64p), _p(free, _u8p), R, _p(u, _f64p), _p(lam, _f64p), _p(g, _f64p))
    if rc != 0:
        raise ValueError("adjoint gradient failed (%d)" % rc)
    return g


def direct_solve(K: Assembled, f: np.ndarray) -> np.ndarray:
    """Sparse direct solve of K u = f per case (scipy's SuperLU), u [N, R, 3]."""
    import scipy.sparse.linalg as spla
    A = K.to_scipy().tocsc()
    lu = spla.splu(A)
    N, R, _ = f.shape
    # rows of A are ordered (node, component); move R to the last axis
    rhs = np.ascontiguousarray(np.moveaxis(f, 1, 2)).reshape(3 * N, R)
    sol = lu.solve(rhs)
    return np.ascontiguousarray(np.moveaxis(sol.reshape(N, 3, R), 2, 1))


# ---------------------------------------------------------------------------
# first-order (TET4) coarse level: the same mesh without edge nodes
# ---------------------------------------------------------------------------

_EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))


@dataclass
class Coarse:
    """TET4 mesh made of the corner nodes of a TET10 mesh.
    coords [N4, 3], conn [E, 4], free [N4, 3], young/poisson [E], vertex [N4] (TET10
    id of each TET4 node), ends [N10, 2] (TET4 nodes whose mean gives each TET10 node)."""
    coords: np.ndarray
    conn: np.ndarray
    young: np.ndarray
    poisson: np.ndarray
    free: np.ndarray
    vertex: np.ndarray
    ends: np.ndarray


def coarse_mesh(mesh) -> Coarse:
    conn = np.asarray(mesh.conn, dtype=np.int64)
    vert = np.unique(conn[:, :4])
    new = -np.ones(np.asarray(mesh.coords).shape[0], dtype=np.int64)
    new[vert] = np.arange(vert.size)
    ends = np.zeros((new.size, 2), dtype=np.int32)
    ends[vert, 0] = new[vert]
    ends[vert, 1] = new[vert]
    for q, (a, b) in enumerate(_EDGES):
        ends[conn[:, 4 + q], 0] = new[conn[:, a]]
        ends[conn[:, 4 + q], 1] = new[conn[:, b]]
    return Coarse(coords=np.asarray(mesh.coords)[vert], conn=new[conn[:, :4]].astype(np.int32),
                  young=np.asarray(mesh.young), poisson=np.asarray(mesh.poisson), free=np.asarray(mesh.free)[vert],
                  vertex=vert, ends=ends)


def tet4_stiffness(xe: np.ndarray, E: float, nu: float) -> np.ndarray:
    lib = _load()
    xe = _c(xe, np.float64).reshape(12)
    Ke = np.zeros(144)
    if lib.oracle_tet4_stiffness(_p(xe, _f64p), float(E), float(nu), _p(Ke, _f64p)) != 0:
        raise ValueError("non-positive element Jacobian")
    return Ke.reshape(12, 12)


def assemble4(coarse: Coarse, apply_bc: bool = True, young=None) -> Assembled:
    lib = _load()
    coords, conn = _c(coarse.coords, np.float64), _c(coarse.conn, np.int32)
    E = _c(coarse.young if young is None else young, np.float64)
    nu = _c(coarse.poisson, np.float64)
    N, Ne = coords.shape[0], conn.shape[0]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    nnzb = lib.oracle_pattern_n(N, Ne, 4, _p(conn, _i32p), _p(rowptr, _i64p), None)
    if nnzb < 0:
        raise ValueError("bad connectivity")
    col = np.zeros(nnzb, dtype=np.int32)
    lib.oracle_pattern_n(N, Ne, 4, _p(conn, _i32p), _p(rowptr, _i64p), _p(col, _i32p))
    vals = np.zeros((nnzb, 3, 3))
    if lib.oracle_assemble4(N, _p(coords, _f64p), Ne, _p(conn, _i32p), _p(E, _f64p), _p(nu, _f64p),
                            _p(rowptr, _i64p), _p(col, _i32p), _p(vals, _f64p)) != 0:
        raise ValueError("assembly failed")
    if apply_bc:
        free = _c(coarse.free, np.uint8)
        lib.oracle_apply_bc(N, _p(rowptr, _i64p), _p(col, _i32p), _p(vals, _f64p), _p(free, _u8p))
    return Assembled(N, rowptr, col, vals)


def prolong(coarse: Coarse, u4: np.ndarray) -> np.ndarray:
    """u10 = P1 u4 ([N4, R, 3] -> [N10, R, 3])."""
    lib = _load()
    u4 = _c(u4, np.float64)
    R = u4.shape[1]
    N10 = coarse.ends.shape[0]
    out = np.zeros((N10, R, 3))
    ends = _c(coarse.ends, np.int32)
    lib.oracle_prolong(N10, R, _p(ends, _i32p), _p(u4, _f64p), _p(out, _f64p))
    return out


def restrict(coarse: Coarse, r10: np.ndarray) -> np.ndarray:
    """r4 = P1^T r10 ([N10, R, 3] -> [N4, R, 3])."""
    lib = _load()
    r10 = _c(r10, np.float64)
    R = r10.shape[1]
    N10, N4 = coarse.ends.shape[0], coarse.coords.shape[0]
    out = np.zeros((N4, R, 3))
    ends = _c(coarse.ends, np.int32)
    lib.oracle_restrict(N10, N4, R, _p(ends, _i32p), _p(r10, _f64p), _p(out, _f64p))
    return out


def fcg_mg(K: Assembled, f: np.ndarray, coarse: Coarse = None, K1: Assembled = None, free=None, u0=None,
           tol: float = 1e-8,
           max_outer: int = 10000, n_inner: int = 30, eps_inner: float = 0.1, n_inner1: int = 300,
           eps_inner1: float = 0.05, literal_beta: bool = False):
    """Flexible CG with the FP32 inner loop at level 0 and, with `coarse`, the TET4
    level 1 before it: (u, outer, inner0_total, inner1_total, relres)."""
    lib = _load()
    f = _c(f, np.float64)
    R = f.shape[1]
    u = np.zeros_like(f) if u0 is None else _c(u0, np.float64).copy()
    Minv = block_jacobi(K)
    outer = np.zeros(R, dtype=np.int32)
    inner = np.zeros(R, dtype=np.int32)
    inner1 = np.zeros(R, dtype=np.int32)
    rel = np.zeros(R)
    if coarse is not None:
        if K1 is None:
            K1 = assemble4(coarse)
        Minv1 = block_jacobi(K1)
        ends = _c(coarse.ends, np.int32)
        free4 = _c(coarse.free, np.uint8)
        if free is None:
            raise ValueError("the free mask of the fine mesh is needed with a coarse level")
        free10 = _c(free, np.uint8)
        args1 = (_p(free10, _u8p), K1.n_nodes, _p(K1.rowptr, _i64p), _p(K1.col, _i32p), _p(K1.vals, _f64p),
                 _p(Minv1, _f64p), _p(free4, _u8p), _p(ends, _i32p), int(n_inner1), float(eps_inner1))
    else:
        args1 = (None, 0, None, None, None, None, None, None, 0, 0.0)
    rc = lib.oracle_fcg_mg(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p), _p(Minv, _f64p), R,
                           _p(f, _f64p), _p(u, _f64p), float(tol), int(max_outer), int(n_inner), float(eps_inner),
                           int(bool(literal_beta)), *args1, _p(outer, _i32p), _p(inner, _i32p), _p(inner1, _i32p),
                           _p(rel, _f64p))
    if rc != 0:
        raise RuntimeError("fcg_mg failed (%d)" % rc)
    return u, outer, inner, inner1, rel


# ---------------------------------------------------------------------------
# level 2: aggregation coarsening of the TET4 level
# ---------------------------------------------------------------------------

def aggregate(K1: Assembled) -> np.ndarray:
    """Plain aggregation of K1's node graph (two passes in node order, see
    oracle_aggregate): int32 aggregate id per coarse node."""
    lib = _load()
    agg = np.empty(K1.n_nodes, dtype=np.int32)
    n = lib.oracle_aggregate(K1.n_nodes, _p(K1.rowptr, _i64p), _p(K1.col, _i32p), _p(agg, _i32p))
    if n < 0:
        raise RuntimeError("aggregation failed (%d)" % n)
    return agg


def galerkin_agg(K1: Assembled, free4: np.ndarray, agg: np.ndarray):
    """A2 = P2^T K1_bc P2 on the free aggregate DOFs, identity on the others:
    (Assembled A2, free2 [NA, 3])."""
    lib = _load()
    NA = int(agg.max()) + 1
    free4 = _c(free4, np.uint8)
    agg = _c(agg, np.int32)
    cap = int(K1.rowptr[-1])
    rowptr2 = np.zeros(NA + 1, dtype=np.int64)
    col2 = np.zeros(cap, dtype=np.int32)
    vals2 = np.zeros((cap, 3, 3))
    free2 = np.zeros((NA, 3), dtype=np.uint8)
    nnz = lib.oracle_galerkin_agg(K1.n_nodes, _p(K1.rowptr, _i64p), _p(K1.col, _i32p), _p(K1.vals, _f64p),
                                  _p(free4, _u8p), _p(agg, _i32p), NA, _p(rowptr2, _i64p), _p(col2, _i32p),
                                  _p(vals2, _f64p), _p(free2, _u8p))
    if nnz < 0:
        raise RuntimeError("galerkin_agg failed (%d)" % nnz)
    return Assembled(n_nodes=NA, rowptr=rowptr2, col=col2[:nnz].copy(), vals=vals2[:nnz].copy()), free2


def fcg_ml(K: Assembled, f: np.ndarray, coarse: Coarse, free, K1: Assembled = None, levels: int = 3, u0=None,
           tol: float = 1e-8, max_outer: int = 10000, n_inner: int = 30, eps_inner: float = 0.1,
           n_inner1: int = 300, eps_inner1: float = 0.05, n_inner2: int = 3000, eps_inner2: float = 0.025,
           literal_beta: bool = False):
    """Algorithm 1 with inner loops at levels 2 (aggregation of the TET4 level), 1
    (TET4) and 0: (u, outer, inner0_total, inner1_total, inner2_total, relres)."""
    lib = _load()
    f = _c(f, np.float64)
    R = f.shape[1]
    u = np.zeros_like(f) if u0 is None else _c(u0, np.float64).copy()
    Minv = block_jacobi(K)
    if K1 is None:
        K1 = assemble4(coarse)
    Minv1 = block_jacobi(K1)
    ends = _c(coarse.ends, np.int32)
    free4 = _c(coarse.free, np.uint8)
    free10 = _c(free, np.uint8)
    counts = [np.zeros(R, dtype=np.int32) for _ in range(4)]
    rel = np.zeros(R)
    if levels >= 3:
        agg = aggregate(K1)
        A2, _ = galerkin_agg(K1, free4, agg)
        Minv2 = block_jacobi(A2)
        args2 = (A2.n_nodes, _p(A2.rowptr, _i64p), _p(A2.col, _i32p), _p(A2.vals, _f64p), _p(Minv2, _f64p),
                 _p(agg, _i32p), int(n_inner2), float(eps_inner2))
    else:
        args2 = (0, None, None, None, None, None, 0, 0.0)
    rc = lib.oracle_fcg_ml(K.n_nodes, _p(K.rowptr, _i64p), _p(K.col, _i32p), _p(K.vals, _f64p), _p(Minv, _f64p), R,
                           _p(f, _f64p), _p(u, _f64p), float(tol), int(max_outer), int(n_inner), float(eps_inner),
                           int(bool(literal_beta)), _p(free10, _u8p), K1.n_nodes, _p(K1.rowptr, _i64p),
                           _p(K1.col, _i32p), _p(K1.vals, _f64p), _p(Minv1, _f64p), _p(free4, _u8p), _p(ends, _i32p),
                           int(n_inner1), float(eps_inner1), *args2, *[_p(c, _i32p) for c in counts], _p(rel, _f64p))
    if rc != 0:
        raise RuntimeError("fcg_ml failed (%d)" % rc)
    return (u, *counts, rel)
