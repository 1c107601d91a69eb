"""Many load cases with a checkpoint on disk: finished cases survive an interruption.

Sec. 5 of the paper computes Green's functions of many unit slips, one solve per
slip. `solve_many_resumable` feeds the cases to the library's many-case driver
(`fe_solve_many`, which streams them through R slots of one batched solve) a chunk
at a time and stores every finished case in a directory:

    manifest.json        mesh and solver-option fingerprint of the run
    case_00017.npy       u of case 17, float64 [N, 3]
    case_00017.json      its statistics and the SHA-256 of its right-hand side

Each file is written to a temporary name first and then renamed, so a case is
either stored completely or not at all. When the run starts again with the same
directory, mesh and options, a stored case is kept if its right-hand side has the
same hash; only the others are solved. A directory written for another mesh or
other options raises instead of mixing results. Cases that did not converge are
stored with their status and solved again on the next run.
"""
from __future__ import annotations

import hashlib
import inspect
import json
import os
from typing import Callable, Optional

import numpy as np

# solver options that change the stored solutions (tolerance, loop settings)
_OPTION_KEYS = ("solver", "tol", "max_outer", "n_inner", "eps_inner", "n_inner1", "eps_inner1", "n_inner2",
                "eps_inner2", "coarse_op")


def _digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _write_atomic(path: str, write: Callable[[str], None]) -> None:
    tmp = path + ".tmp"
    write(tmp)
    os.replace(tmp, path)


def _save_npy(path: str, a: np.ndarray) -> None:
    def w(tmp):
        with open(tmp, "wb") as fh:
            np.save(fh, a)
    _write_atomic(path, w)


def _save_json(path: str, obj) -> None:
    def w(tmp):
        with open(tmp, "w") as fh:
            json.dump(obj, fh, sort_keys=True)
    _write_atomic(path, w)


def mesh_fingerprint(mesh, key: str = "") -> str:
    """Identifies the mesh a store belongs to: its sizes, node coordinates, the
    log-moduli set since creation (if any) and a caller's key (for what the
    coordinates do not show, e.g. the materials given at creation)."""
    h = hashlib.sha256()
    h.update(np.array([mesh.n_nodes, mesh.n_elem], dtype=np.int64).tobytes())
    coords = getattr(mesh, "_coords", None)
    if coords is not None:
        h.update(np.ascontiguousarray(coords).tobytes())
    logE = getattr(mesh, "log_young", None)
    if logE is not None:
        h.update(np.ascontiguousarray(logE.detach().cpu().numpy()).tobytes())
    h.update(key.encode())
    return h.hexdigest()


class CaseStore:
    """The directory of one resumable run (see the module docstring)."""

    def __init__(self, path: str, manifest: dict):
        self.path = path
        os.makedirs(path, exist_ok=True)
        mp = os.path.join(path, "manifest.json")
        if os.path.exists(mp):
            with open(mp) as fh:
                old = json.load(fh)
            if old != manifest:
                raise ValueError("case store %s was written for another mesh or other solver options" % path)
        else:
            _save_json(mp, manifest)

    def _base(self, c: int) -> str:
        return os.path.join(self.path, "case_%05d" % c)

    def done(self, c: int, f_digest: str) -> bool:
        """True if case c is stored, converged, for this right-hand side."""
        b = self._base(c)
        if not (os.path.exists(b + ".json") and os.path.exists(b + ".npy")):
            return False
        with open(b + ".json") as fh:
            meta = json.load(fh)
        return meta.get("f_sha256") == f_digest and meta.get("status") == 0

    def put(self, c: int, u: np.ndarray, stats: dict, f_digest: str) -> None:
        b = self._base(c)
        _save_npy(b + ".npy", u)                       # the solution first, its record last:
        _save_json(b + ".json", dict(stats, f_sha256=f_digest, case=c))   # a record means a whole file

    def get(self, c: int):
        """(u, statistics) of case c; u is memory-mapped from its file."""
        b = self._base(c)
        with open(b + ".json") as fh:
            meta = json.load(fh)
        return np.load(b + ".npy", mmap_mode="r"), meta


def solve_many_resumable(mesh, f_cases, store_dir: str, chunk: int = 0, R_slots: int = 0,
                         on_chunk: Optional[Callable[[list], None]] = None, key: str = "", **opts):
    """Solves K_bc u_c = f_c for every case c of f_cases [n, N, 3] (float64, on the
    mesh's device) through `mesh.solve_many`, `chunk` cases per call (0: four times
    the slot count the first call used, at least 8), storing each finished case in
    `store_dir`. Cases already stored there for the same right-hand side are not
    solved again. `on_chunk(cases)` runs after each chunk is stored (for progress,
    or to stop the run); `key` joins the mesh fingerprint (mesh_fingerprint). Returns
    (u, stats, solved): u a list of n float64 [N, 3] arrays memory-mapped from the
    store (so that hundreds of cases of a large mesh need no host memory of their
    own), the statistics of every case, and the cases solved by this call. Right-hand
    sides are hashed one case at a time."""
    import torch

    n = int(f_cases.shape[0])
    if n == 0:
        return [], [], []
    opts.setdefault("raise_on_fail", False)
    defaults = {k: v.default for k, v in inspect.signature(mesh.solve_many).parameters.items()
                if v.default is not inspect.Parameter.empty}
    eff = {**defaults, **opts}
    manifest = {"mesh": mesh_fingerprint(mesh, key), "n_nodes": int(mesh.n_nodes),
                "options": {k: eff[k] for k in _OPTION_KEYS if k in eff}}
    store = CaseStore(store_dir, manifest)
    digests = [_digest(f_cases[c].detach().cpu().numpy()) for c in range(n)]
    pending = [c for c in range(n) if not store.done(c, digests[c])]
    solved = []   # cases solved by this call
    while pending:
        size = chunk if chunk > 0 else 8
        part = pending[:size]
        idx = torch.as_tensor(part, device=f_cases.device)
        u, stats, _, r_used = mesh.solve_many(f_cases.index_select(0, idx).contiguous(), R_slots=R_slots, **opts)
        if chunk <= 0:
            chunk = max(8, 4 * int(r_used))
        u_host = u.cpu().numpy()
        for k, c in enumerate(part):
            store.put(c, u_host[k], stats[k], digests[c])
        solved.extend(part)
        pending = pending[len(part):]
        if on_chunk is not None:
            on_chunk(part)
    us, metas = [], []
    for c in range(n):
        u_c, meta = store.get(c)
        us.append(u_c)
        metas.append(meta)
    return us, metas, solved
