"""Thin Python binding of libfe (argument marshalling only).

Every step of the computation runs in libfe's CUDA kernels; this module checks
shapes and dtypes, passes raw pointers and the current CUDA stream, and turns
fe_status codes into exceptions. There is no CPU fallback: if libfe.so is
missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_ENOCONV, FE_EBREAKDOWN, FE_ETIMEOUT = range(7)
FE_F64, FE_F32 = 0, 1
FE_SOLVER_PCG64, FE_SOLVER_FCG_MIXED, FE_SOLVER_FCG_MG, FE_SOLVER_FCG_AMG = 0, 1, 2, 3
SOLVERS = {"pcg64": FE_SOLVER_PCG64, "fcg_mixed": FE_SOLVER_FCG_MIXED, "fcg_mg": FE_SOLVER_FCG_MG,
           "fcg_amg": FE_SOLVER_FCG_AMG}
COARSE_OPS = {"auto": 0, "assembled": 1, "ebe": 2}
INNER_KERNELS = {"persistent": 0, "steps": 1}
EBE_DIRECT, EBE_TILED = 0, 1

STATUS_NAMES = {0: "FE_OK", 1: "FE_EINVAL", 2: "FE_ENOMEM", 3: "FE_ECUDA", 4: "FE_ENOCONV",
                5: "FE_EBREAKDOWN", 6: "FE_ETIMEOUT"}

# every symbol include/fe.h declares
EXPORTED = ["fe_last_error", "fe_version", "fe_solve_opts_default", "fe_mesh_create", "fe_mesh_destroy",
            "fe_mesh_info", "fe_mesh_set_log_young", "fe_ebe_apply", "fe_ebe_set_variant",
            "fe_ebe_get_variant", "fe_ebe_tune", "fe_pcg_solve", "fe_solve_many", "fe_block_jacobi",
            "fe_block_jacobi_noalloc", "fe_adjoint_grad", "fe_coarse_info", "fe_ebe4_apply", "fe_coarse_restrict",
            "fe_coarse_prolong", "fe_coarse_block_jacobi", "fe_coarse_apply", "fe_level2_info", "fe_level2_apply",
            "fe_level2_restrict", "fe_level2_prolong", "fe_level2_block_jacobi", "fe_coarse_matrix_info",
            "fe_ebe_apply_host", "fe_mesh_device_status", "fe_obs_create", "fe_obs_destroy", "fe_obs_apply",
            "fe_obs_adjoint", "fe_combine_cases", "fe_case_dots", "fe_wait_selftest"]


class FeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("tol", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("n_inner", ctypes.c_int32), ("eps_inner", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("literal_beta", ctypes.c_int32), ("check_every", ctypes.c_int32), ("verbose", ctypes.c_int32),
                ("n_inner1", ctypes.c_int32), ("eps_inner1", ctypes.c_double), ("coarse_op", ctypes.c_int32),
                ("n_inner2", ctypes.c_int32), ("eps_inner2", ctypes.c_double),
                ("cg_coef", ctypes.c_void_p), ("cg_coef_len", ctypes.c_int32), ("inner_kernel", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32), ("relres", ctypes.c_double),
                ("status", ctypes.c_int32), ("inner1_iters", ctypes.c_int32), ("inner2_iters", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def load(path: Optional[str] = None):
    """Load libfe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libfe.so not found at {path}; build it with paper_1710_08679_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.fe_last_error.restype = ctypes.c_char_p
    lib.fe_version.restype = ctypes.c_char_p
    lib.fe_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.fe_solve_opts_default.restype = None
    lib.fe_mesh_create.argtypes = [_i64, _vp, _i64, _vp, _vp, _vp, _vp, _i32, _vp, ctypes.POINTER(_vp)]
    lib.fe_mesh_destroy.argtypes = [_vp]
    lib.fe_mesh_destroy.restype = None
    lib.fe_mesh_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    lib.fe_mesh_set_log_young.argtypes = [_vp, _vp, _vp]
    lib.fe_ebe_apply.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    lib.fe_ebe_set_variant.argtypes = [_vp, _i32, _i32, _i32, _i32, _vp]
    lib.fe_ebe_get_variant.argtypes = [_vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
    lib.fe_ebe_tune.argtypes = [_vp, _i32, _i32, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
    lib.fe_pcg_solve.argtypes = [_vp, _i32, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _vp]
    lib.fe_adjoint_grad.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp]
    lib.fe_solve_many.argtypes = [_vp, _i32, _vp, _vp, _i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats),
                                  ctypes.POINTER(_i32), _vp]
    lib.fe_block_jacobi.argtypes = [_vp, _vp, _vp]
    lib.fe_block_jacobi_noalloc.argtypes = [_vp, _vp, _vp]
    lib.fe_coarse_info.argtypes = [_vp, ctypes.POINTER(_i64), _vp, _vp]
    lib.fe_ebe4_apply.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    lib.fe_coarse_restrict.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    lib.fe_coarse_prolong.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    lib.fe_coarse_block_jacobi.argtypes = [_vp, _vp, _vp]
    lib.fe_coarse_apply.argtypes = [_vp, _i32, _vp, _vp, _vp]
    lib.fe_level2_info.argtypes = [_vp, ctypes.POINTER(_i64), _vp, _vp]
    for name in ("fe_level2_apply", "fe_level2_restrict", "fe_level2_prolong"):
        getattr(lib, name).argtypes = [_vp, _i32, _vp, _vp, _vp]
    lib.fe_level2_block_jacobi.argtypes = [_vp, _vp, _vp]
    lib.fe_coarse_matrix_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp]
    lib.fe_ebe_apply_host.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    lib.fe_mesh_device_status.argtypes = [_vp, _vp]
    lib.fe_wait_selftest.argtypes = [_vp, _i32, _i64, _vp]
    lib.fe_obs_create.argtypes = [_vp, _i64, _i32, _vp, _vp, ctypes.POINTER(_vp)]
    lib.fe_obs_destroy.argtypes = [_vp]
    lib.fe_obs_destroy.restype = None
    lib.fe_obs_apply.argtypes = [_vp, _i32, _vp, _vp, _vp]
    lib.fe_obs_adjoint.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp]
    lib.fe_combine_cases.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp]
    lib.fe_case_dots.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp]
    for name in ("fe_mesh_create", "fe_mesh_info", "fe_mesh_set_log_young", "fe_ebe_apply", "fe_ebe_set_variant",
                 "fe_ebe_get_variant", "fe_ebe_tune", "fe_pcg_solve", "fe_solve_many", "fe_block_jacobi",
                 "fe_block_jacobi_noalloc", "fe_adjoint_grad", "fe_coarse_info", "fe_ebe4_apply",
                 "fe_coarse_restrict", "fe_coarse_prolong", "fe_coarse_block_jacobi", "fe_coarse_apply",
                 "fe_level2_info", "fe_level2_apply", "fe_level2_restrict", "fe_level2_prolong",
                 "fe_level2_block_jacobi", "fe_coarse_matrix_info", "fe_ebe_apply_host", "fe_mesh_device_status",
                 "fe_obs_create", "fe_obs_apply", "fe_obs_adjoint", "fe_combine_cases", "fe_case_dots",
                 "fe_wait_selftest"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != FE_OK:
        msg = load().fe_last_error().decode(errors="replace")
        raise FeError(status, f"{what}: {msg}")


def version() -> str:
    return load().fe_version().decode()


def _torch():
    import torch
    return torch


def _stream_ptr(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_ptr(t, dtype, shape=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Device-resident TET10 mesh (libfe handle)."""

    def __init__(self, coords, conn, young, poisson, free, device: int = 0):
        lib = load()
        self._coords = np.ascontiguousarray(coords, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        young = np.ascontiguousarray(young, dtype=np.float64)
        poisson = np.ascontiguousarray(poisson, dtype=np.float64)
        free = np.ascontiguousarray(free, dtype=np.uint8)
        N, E = self._coords.shape[0], conn.shape[0]
        if self._coords.shape != (N, 3) or conn.shape != (E, 10) or young.shape != (E,) or \
                poisson.shape != (E,) or free.shape != (N, 3):
            raise ValueError("mesh arrays have inconsistent shapes")
        self.device = int(device)
        torch = _torch()
        h = ctypes.c_void_p()
        st = lib.fe_mesh_create(N, self._coords.ctypes.data, E, conn.ctypes.data, young.ctypes.data,
                                poisson.ctypes.data, free.ctypes.data, self.device,
                                _stream_ptr(torch.device("cuda", self.device)), ctypes.byref(h))
        _check(st, "fe_mesh_create")
        self._h = h
        self.log_young = None   # the moduli given at creation
        self.n_nodes, self.n_elem = N, E
        self.free = torch.from_numpy(free.astype(np.float64)).to(f"cuda:{self.device}")

    @classmethod
    def from_mesh(cls, m, device: int = 0) -> "Mesh":
        return cls(m.coords, m.conn, m.young, m.poisson, m.free, device)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().fe_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    def _stream(self):
        return _stream_ptr(_torch().device("cuda", self.device))

    # ---- operator -------------------------------------------------------
    def ebe(self, x, out=None):
        """y = K_bc x for x [N, R, 3] (float64 or float32 CUDA tensor)."""
        torch = _torch()
        if x.dim() != 3 or x.shape[0] != self.n_nodes or x.shape[2] != 3:
            raise ValueError("x must be [N, R, 3]")
        R = int(x.shape[1])
        dt = {torch.float64: FE_F64, torch.float32: FE_F32}.get(x.dtype)
        if dt is None:
            raise TypeError("x must be float64 or float32")
        xp = _dev_ptr(x, x.dtype, name="x")
        y = torch.empty_like(x) if out is None else out
        yp = _dev_ptr(y, x.dtype, x.shape, name="out")
        _check(load().fe_ebe_apply(self._h, R, dt, xp, yp, self._stream()), "fe_ebe_apply")
        return y

    def ebe_host(self, x, out=None):
        """y = K_bc x for host tensors x [N, R, 3] (float64 or float32; pinned memory
        lets consecutive calls overlap copies and products). Asynchronous on the
        current stream: synchronise it before reading the result or changing x."""
        torch = _torch()
        if not isinstance(x, torch.Tensor) or x.is_cuda or not x.is_contiguous():
            raise TypeError("x must be a contiguous CPU tensor")
        if x.dim() != 3 or x.shape[0] != self.n_nodes or x.shape[2] != 3:
            raise ValueError("x must be [N, R, 3]")
        dt = {torch.float64: FE_F64, torch.float32: FE_F32}.get(x.dtype)
        if dt is None:
            raise TypeError("x must be float64 or float32")
        y = torch.empty_like(x) if out is None else out
        if y.is_cuda or not y.is_contiguous() or y.shape != x.shape or y.dtype != x.dtype:
            raise ValueError("out must be a contiguous CPU tensor like x")
        _check(load().fe_ebe_apply_host(self._h, int(x.shape[1]), dt, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), self._stream()), "fe_ebe_apply_host")
        return y

    def set_variant(self, R: int, dtype, variant: int, tile_elems: int = 48):
        dt = FE_F32 if dtype in ("f32", np.float32) or str(dtype).endswith("float32") else FE_F64
        _check(load().fe_ebe_set_variant(self._h, int(R), dt, int(variant), int(tile_elems), self._stream()),
               "fe_ebe_set_variant")

    def get_variant(self, R: int, dtype):
        dt = FE_F32 if dtype in ("f32", np.float32) or str(dtype).endswith("float32") else FE_F64
        v, t = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fe_ebe_get_variant(self._h, int(R), dt, ctypes.byref(v), ctypes.byref(t)),
               "fe_ebe_get_variant")
        return v.value, t.value

    def tune(self, R: int, dtype):
        """Time the EBE variants for (R, dtype) on this mesh and keep the fastest."""
        dt = FE_F32 if dtype in ("f32", np.float32) or str(dtype).endswith("float32") else FE_F64
        v, t = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fe_ebe_tune(self._h, int(R), dt, self._stream(), ctypes.byref(v), ctypes.byref(t)),
               "fe_ebe_tune")
        return v.value, t.value

    def device_status(self):
        """Synchronise the current stream and raise FeError(FE_ETIMEOUT) if a kernel on
        this mesh gave up a bounded device-side wait since the last check."""
        _check(load().fe_mesh_device_status(self._h, self._stream()), "fe_mesh_device_status")

    def wait_selftest(self, which: str = "mbarrier", cycles: int = 1 << 21):
        """Runs a bounded device-side wait that nothing ends ("mbarrier": the wait of the
        warp-specialised EBE kernel; "grid": the inner-loop kernel's grid barrier); it
        gives up after `cycles` SM cycles and the next device_status() raises FE_ETIMEOUT."""
        _check(load().fe_wait_selftest(self._h, {"mbarrier": 0, "grid": 1}[which], int(cycles), self._stream()),
               "fe_wait_selftest")

    def set_log_young(self, logE):
        torch = _torch()
        p = _dev_ptr(logE, torch.float64, (self.n_elem,), name="logE")
        _check(load().fe_mesh_set_log_young(self._h, p, self._stream()), "fe_mesh_set_log_young")
        self.log_young = logE.detach().clone()   # the moduli the mesh holds now

    # ---- solvers --------------------------------------------------------
    def solve(self, f, u0=None, solver: str = "fcg_mixed", tol: float = 1e-8, max_outer: int = 20000,
              n_inner: int = 30, eps_inner: float = 0.1, use_graph: bool = True, literal_beta: bool = False,
              check_every: int = 1, n_inner1: int = 300, eps_inner1: float = 0.05, coarse_op: str = "auto",
              n_inner2: int = 3000, eps_inner2: float = 0.025, raise_on_fail: bool = True, cg_coef=None,
              inner_kernel: str = "steps"):
        """Solve K_bc u = f for f [N, R, 3] float64; returns (u, stats list, status).
        cg_coef (solver "pcg64" only): a C-contiguous float64 numpy array [k, R, 2] that
        receives (alpha, beta) of the first k CG iterations of every case.
        inner_kernel: "steps" (one launch per vector pass and scalar step, the default) or
        "persistent" (one cooperative kernel per inner loop on the assembled levels 1 and 2)."""
        torch = _torch()
        R = int(f.shape[1])
        fp = _dev_ptr(f, torch.float64, (self.n_nodes, R, 3), name="f")
        u = torch.zeros_like(f) if u0 is None else u0.clone()
        up = _dev_ptr(u, torch.float64, (self.n_nodes, R, 3), name="u")
        o = SolveOpts()
        load().fe_solve_opts_default(ctypes.byref(o))
        o.solver = SOLVERS[solver]
        o.tol, o.max_outer, o.n_inner, o.eps_inner = float(tol), int(max_outer), int(n_inner), float(eps_inner)
        o.use_graph, o.literal_beta, o.check_every = int(bool(use_graph)), int(bool(literal_beta)), int(check_every)
        o.n_inner1, o.eps_inner1 = int(n_inner1), float(eps_inner1)
        o.coarse_op = COARSE_OPS[coarse_op]
        o.n_inner2, o.eps_inner2 = int(n_inner2), float(eps_inner2)
        o.inner_kernel = INNER_KERNELS[inner_kernel]
        if cg_coef is not None:
            if not (isinstance(cg_coef, np.ndarray) and cg_coef.dtype == np.float64 and cg_coef.ndim == 3 and
                    cg_coef.shape[1:] == (R, 2) and cg_coef.flags["C_CONTIGUOUS"]):
                raise ValueError("cg_coef must be a C-contiguous float64 array [k, R, 2]")
            o.cg_coef, o.cg_coef_len = cg_coef.ctypes.data, int(cg_coef.shape[0])
        stats = (SolveStats * R)()
        st = load().fe_pcg_solve(self._h, R, fp, up, ctypes.byref(o), stats, self._stream())
        out = [dict(outer=s.outer_iters, inner=s.inner_iters, inner1=s.inner1_iters, inner2=s.inner2_iters,
                    relres=s.relres, status=s.status) for s in stats]
        if st not in (FE_OK, FE_ENOCONV, FE_EBREAKDOWN) or (raise_on_fail and st != FE_OK):
            _check(st, "fe_pcg_solve")
        return u, out, st

    def solve_many(self, f_cases, R_slots: int = 0, solver: str = "fcg_mixed", tol: float = 1e-8,
                   max_outer: int = 20000, n_inner: int = 30, eps_inner: float = 0.1, use_graph: bool = True,
                   n_inner1: int = 300, eps_inner1: float = 0.05, coarse_op: str = "auto",
                   n_inner2: int = 3000, eps_inner2: float = 0.025, raise_on_fail: bool = True,
                   inner_kernel: str = "steps"):
        """Solve for f_cases [n_cases, N, 3] (float64, case-major) with at most R_slots
        in flight (0 = from free memory); returns (u [n_cases, N, 3], stats, status, R_used)."""
        torch = _torch()
        n = int(f_cases.shape[0])
        fp = _dev_ptr(f_cases, torch.float64, (n, self.n_nodes, 3), name="f_cases")
        u = torch.empty_like(f_cases)
        o = SolveOpts()
        load().fe_solve_opts_default(ctypes.byref(o))
        o.solver = SOLVERS[solver]
        o.tol, o.max_outer, o.n_inner, o.eps_inner = float(tol), int(max_outer), int(n_inner), float(eps_inner)
        o.use_graph = int(bool(use_graph))
        o.n_inner1, o.eps_inner1 = int(n_inner1), float(eps_inner1)
        o.coarse_op = COARSE_OPS[coarse_op]
        o.n_inner2, o.eps_inner2 = int(n_inner2), float(eps_inner2)
        o.inner_kernel = INNER_KERNELS[inner_kernel]
        stats = (SolveStats * n)()
        r_used = _i32()
        st = load().fe_solve_many(self._h, n, fp, ctypes.c_void_p(u.data_ptr()), int(R_slots), ctypes.byref(o),
                                  stats, ctypes.byref(r_used), self._stream())
        out = [dict(outer=s.outer_iters, inner=s.inner_iters, inner1=s.inner1_iters, inner2=s.inner2_iters,
                    relres=s.relres, status=s.status) for s in stats]
        if st not in (FE_OK, FE_ENOCONV, FE_EBREAKDOWN) or (raise_on_fail and st != FE_OK):
            _check(st, "fe_solve_many")
        return u, out, st, r_used.value

    def block_jacobi(self):
        """Inverse 3x3 diagonal blocks of K_bc, float64 [N, 3, 3]."""
        torch = _torch()
        out = torch.empty((self.n_nodes, 3, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(load().fe_block_jacobi(self._h, ctypes.c_void_p(out.data_ptr()), self._stream()), "fe_block_jacobi")
        return out

    # ---- TET4 coarse level (level 1) -------------------------------------
    def coarse_info(self):
        """(N4, vertex): coarse node count and the TET10 node id of each coarse node."""
        n4 = _i64()
        _check(load().fe_coarse_info(self._h, ctypes.byref(n4), None, self._stream()), "fe_coarse_info")
        vertex = np.empty(n4.value, dtype=np.int32)
        _check(load().fe_coarse_info(self._h, ctypes.byref(n4), vertex.ctypes.data, self._stream()),
               "fe_coarse_info")
        self.n_nodes4 = int(n4.value)
        return self.n_nodes4, vertex

    def _n4(self) -> int:
        if getattr(self, "n_nodes4", None) is None:
            self.coarse_info()
        return self.n_nodes4

    def _coarse_vec(self, fn: str, x, n_in: int, n_out: int):
        torch = _torch()
        if x.dim() != 3 or x.shape[0] != n_in or x.shape[2] != 3:
            raise ValueError(f"input must be [{n_in}, R, 3]")
        R = int(x.shape[1])
        dt = {torch.float64: FE_F64, torch.float32: FE_F32}.get(x.dtype)
        if dt is None:
            raise TypeError("input must be float64 or float32")
        y = torch.empty((n_out, R, 3), dtype=x.dtype, device=x.device)
        _check(getattr(load(), fn)(self._h, R, dt, _dev_ptr(x, x.dtype, name="input"),
                                   ctypes.c_void_p(y.data_ptr()), self._stream()), fn)
        return y

    def ebe4(self, x4):
        """y4 = K1_bc x4 on the TET4 coarse mesh, x4 [N4, R, 3]."""
        n4 = self._n4()
        return self._coarse_vec("fe_ebe4_apply", x4, n4, n4)

    def coarse_apply(self, x4):
        """y4 = K1_bc x4 with the assembled coarse matrix (FP32), x4 [N4, R, 3]."""
        torch = _torch()
        n4 = self._n4()
        if x4.dim() != 3 or x4.shape[0] != n4 or x4.shape[2] != 3:
            raise ValueError(f"x4 must be [{n4}, R, 3]")
        xp = _dev_ptr(x4, torch.float32, name="x4")
        y = torch.empty_like(x4)
        _check(load().fe_coarse_apply(self._h, int(x4.shape[1]), xp, ctypes.c_void_p(y.data_ptr()), self._stream()),
               "fe_coarse_apply")
        return y

    def coarse_restrict(self, r10):
        """r4 = P (P1^T r10): [N, R, 3] -> [N4, R, 3]."""
        return self._coarse_vec("fe_coarse_restrict", r10, self.n_nodes, self._n4())

    def coarse_prolong(self, u4):
        """u10 = P (P1 u4): [N4, R, 3] -> [N, R, 3]."""
        return self._coarse_vec("fe_coarse_prolong", u4, self._n4(), self.n_nodes)

    def coarse_block_jacobi(self):
        """Inverse 3x3 diagonal blocks of K1_bc, float64 [N4, 3, 3]."""
        torch = _torch()
        out = torch.empty((self._n4(), 3, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(load().fe_coarse_block_jacobi(self._h, ctypes.c_void_p(out.data_ptr()), self._stream()),
               "fe_coarse_block_jacobi")
        return out

    # ---- level 2 (aggregation of the TET4 level) --------------------------
    def level2_info(self):
        """(NA, agg): aggregate count and the aggregate of each coarse node."""
        na = _i64()
        _check(load().fe_level2_info(self._h, ctypes.byref(na), None, self._stream()), "fe_level2_info")
        agg = np.empty(self._n4(), dtype=np.int32)
        _check(load().fe_level2_info(self._h, ctypes.byref(na), agg.ctypes.data, self._stream()), "fe_level2_info")
        self.n_agg = int(na.value)
        return self.n_agg, agg

    def _na(self) -> int:
        if getattr(self, "n_agg", None) is None:
            self.level2_info()
        return self.n_agg

    def _level2_vec(self, fn: str, x, n_in: int, n_out: int):
        torch = _torch()
        if x.dim() != 3 or x.shape[0] != n_in or x.shape[2] != 3:
            raise ValueError(f"input must be [{n_in}, R, 3]")
        xp = _dev_ptr(x, torch.float32, name="input")
        y = torch.empty((n_out, int(x.shape[1]), 3), dtype=torch.float32, device=x.device)
        _check(getattr(load(), fn)(self._h, int(x.shape[1]), xp, ctypes.c_void_p(y.data_ptr()), self._stream()), fn)
        return y

    def coarse_matrix_info(self):
        """(blocks of K1_bc, blocks of A2), building the assembled coarse matrices if needed."""
        a, b = _i64(), _i64()
        _check(load().fe_coarse_matrix_info(self._h, ctypes.byref(a), ctypes.byref(b), self._stream()),
               "fe_coarse_matrix_info")
        return int(a.value), int(b.value)

    def level2_apply(self, x2):
        """y2 = A2 x2 (FP32), x2 [NA, R, 3]."""
        return self._level2_vec("fe_level2_apply", x2, self._na(), self._na())

    def level2_restrict(self, r4):
        """r2 = P2^T r4: [N4, R, 3] -> [NA, R, 3] (FP32)."""
        return self._level2_vec("fe_level2_restrict", r4, self._n4(), self._na())

    def level2_prolong(self, u2):
        """u4 = P2 u2: [NA, R, 3] -> [N4, R, 3] (FP32)."""
        return self._level2_vec("fe_level2_prolong", u2, self._na(), self._n4())

    def level2_block_jacobi(self):
        """Inverse 3x3 diagonal blocks of A2, float64 [NA, 3, 3]."""
        torch = _torch()
        out = torch.empty((self._na(), 3, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(load().fe_level2_block_jacobi(self._h, ctypes.c_void_p(out.data_ptr()), self._stream()),
               "fe_level2_block_jacobi")
        return out

    def adjoint_grad(self, u, lam):
        """g_e = -sum_r (P lam_r)_e^T K_e (P u_r)_e, float64 [E]."""
        torch = _torch()
        R = int(u.shape[1])
        up = _dev_ptr(u, torch.float64, (self.n_nodes, R, 3), name="u")
        lp = _dev_ptr(lam, torch.float64, (self.n_nodes, R, 3), name="lambda")
        g = torch.empty(self.n_elem, dtype=torch.float64, device=u.device)
        _check(load().fe_adjoint_grad(self._h, R, up, lp, ctypes.c_void_p(g.data_ptr()), self._stream()),
               "fe_adjoint_grad")
        return g

    def combine_cases(self, G, a):
        """u [N, 3] = sum_r a[r] G[:, r, :] (fe_combine_cases), G float64 [N, R, 3], a float64 [R]."""
        torch = _torch()
        R = int(G.shape[1])
        gp = _dev_ptr(G, torch.float64, (self.n_nodes, R, 3), name="G")
        ap = _dev_ptr(a, torch.float64, (R,), name="a")
        u = torch.empty((self.n_nodes, 3), dtype=torch.float64, device=G.device)
        _check(load().fe_combine_cases(self._h, R, gp, ap, ctypes.c_void_p(u.data_ptr()), self._stream()),
               "fe_combine_cases")
        return u

    def case_dots(self, f, lam):
        """out[r] = (P f_r) . lam (fe_case_dots), f float64 [N, R, 3], lam float64 [N, 3]."""
        torch = _torch()
        R = int(f.shape[1])
        fp = _dev_ptr(f, torch.float64, (self.n_nodes, R, 3), name="f")
        lp = _dev_ptr(lam, torch.float64, (self.n_nodes, 3), name="lam")
        out = torch.empty(R, dtype=torch.float64, device=f.device)
        _check(load().fe_case_dots(self._h, R, fp, lp, ctypes.c_void_p(out.data_ptr()), self._stream()),
               "fe_case_dots")
        return out


class Observation:
    """Observation operator of libfe (fe_obs_*): u_obs[p] = sum_j w[p, j] u[node[p, j]]."""

    def __init__(self, mesh: Mesh, node, weight):
        node = np.ascontiguousarray(node, dtype=np.int32)
        weight = np.ascontiguousarray(weight, dtype=np.float64)
        if node.ndim != 2 or weight.shape != node.shape:
            raise ValueError("node and weight must be [n_obs, n_per] arrays of one shape")
        self.mesh = mesh
        self.n_obs, self.n_per = int(node.shape[0]), int(node.shape[1])
        h = ctypes.c_void_p()
        _check(load().fe_obs_create(mesh._h, self.n_obs, self.n_per, node.ctypes.data, weight.ctypes.data,
                                    ctypes.byref(h)), "fe_obs_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().fe_obs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, u):
        """u [N, 3] or [N, R, 3] -> [n_obs, 3] or [n_obs, R, 3]."""
        torch = _torch()
        v = u if u.dim() == 3 else u.reshape(u.shape[0], 1, 3)
        R = int(v.shape[1])
        up = _dev_ptr(v.contiguous(), torch.float64, (self.mesh.n_nodes, R, 3), name="u")
        out = torch.empty((self.n_obs, R, 3), dtype=torch.float64, device=u.device)
        _check(load().fe_obs_apply(self._h, R, up, ctypes.c_void_p(out.data_ptr()), self.mesh._stream()),
               "fe_obs_apply")
        return out if u.dim() == 3 else out[:, 0, :]

    def adjoint(self, g):
        """P Obs^T g: g [n_obs, 3] or [n_obs, R, 3] -> [N, 3] or [N, R, 3], zero on constrained DOFs."""
        torch = _torch()
        v = g if g.dim() == 3 else g.reshape(g.shape[0], 1, 3)
        R = int(v.shape[1])
        v = v.contiguous()
        gp = _dev_ptr(v, torch.float64, (self.n_obs, R, 3), name="g")
        out = torch.empty((self.mesh.n_nodes, R, 3), dtype=torch.float64, device=g.device)
        _check(load().fe_obs_adjoint(self.mesh._h, self._h, R, gp, ctypes.c_void_p(out.data_ptr()),
                                     self.mesh._stream()), "fe_obs_adjoint")
        return out if g.dim() == 3 else out[:, 0, :]
