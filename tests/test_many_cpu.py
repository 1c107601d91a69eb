"""Bookkeeping of the resumable many-case driver (paper_1710_08679_gb300.many) on
the CPU: a stand-in mesh whose solve_many returns u = 2 f lets every path of the
store be checked without a GPU (interruption and resume, changed right-hand
sides, changed options, cases that did not converge, half-written files)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1710_08679_gb300 import many


class FakeMesh:
    def __init__(self, n_nodes=5, fail=()):
        self.n_nodes, self.n_elem = n_nodes, 2
        self._coords = np.arange(3 * n_nodes, dtype=np.float64).reshape(n_nodes, 3)
        self.log_young = None
        self.calls = []
        self.fail = set(fail)      # rows of f whose first entry marks a case that does not converge

    def solve_many(self, f_cases, R_slots=0, solver="fcg_mixed", tol=1e-8, max_outer=20000, n_inner=30,
                   eps_inner=0.1, raise_on_fail=True):
        self.calls.append(int(f_cases.shape[0]))
        stats = [dict(outer=3, inner=40, inner1=0, inner2=0, relres=1e-9,
                      status=5 if float(f[0, 0]) in self.fail else 0) for f in f_cases]
        return 2.0 * f_cases, stats, 0, 2


def cases(n, N=5, seed=0):
    return torch.from_numpy(np.random.default_rng(seed).standard_normal((n, N, 3)))


def test_full_run_then_nothing_left(tmp_path):
    m, f = FakeMesh(), cases(7)
    u, st, solved = many.solve_many_resumable(m, f, str(tmp_path), chunk=3)
    assert solved == list(range(7)) and m.calls == [3, 3, 1]
    assert np.array_equal(np.stack(u), 2.0 * f.numpy()) and all(s["status"] == 0 for s in st)
    u2, _, solved2 = many.solve_many_resumable(m, f, str(tmp_path), chunk=3)
    assert solved2 == [] and m.calls == [3, 3, 1] and np.array_equal(np.stack(u2), np.stack(u))


def test_interrupted_run_resumes_with_pending_cases_only(tmp_path):
    m, f = FakeMesh(), cases(8)

    def stop(part):
        raise KeyboardInterrupt

    with pytest.raises(KeyboardInterrupt):
        many.solve_many_resumable(m, f, str(tmp_path), chunk=3, on_chunk=stop)
    assert sorted(p for p in os.listdir(tmp_path) if p.endswith(".json")) == \
        ["case_00000.json", "case_00001.json", "case_00002.json", "manifest.json"]
    u, _, solved = many.solve_many_resumable(m, f, str(tmp_path), chunk=3)
    assert solved == [3, 4, 5, 6, 7] and m.calls == [3, 3, 2]
    assert np.array_equal(np.stack(u), 2.0 * f.numpy())


def test_changed_right_hand_side_is_solved_again(tmp_path):
    m, f = FakeMesh(), cases(4)
    many.solve_many_resumable(m, f, str(tmp_path))
    g = f.clone()
    g[2] += 1.0
    u, _, solved = many.solve_many_resumable(m, g, str(tmp_path))
    assert solved == [2] and np.array_equal(np.stack(u), 2.0 * g.numpy())


def test_other_options_or_mesh_are_refused(tmp_path):
    m, f = FakeMesh(), cases(2)
    many.solve_many_resumable(m, f, str(tmp_path), tol=1e-8)
    with pytest.raises(ValueError):
        many.solve_many_resumable(m, f, str(tmp_path), tol=1e-10)
    with pytest.raises(ValueError):
        many.solve_many_resumable(FakeMesh(n_nodes=5), f, str(tmp_path), key="other materials")
    m2 = FakeMesh()
    m2._coords = m2._coords + 1.0
    with pytest.raises(ValueError):
        many.solve_many_resumable(m2, f, str(tmp_path))


def test_unconverged_case_is_kept_with_its_status_and_retried(tmp_path):
    f = cases(3)
    m = FakeMesh(fail={float(f[1, 0, 0])})
    _, st, solved = many.solve_many_resumable(m, f, str(tmp_path))
    assert solved == [0, 1, 2] and [s["status"] for s in st] == [0, 5, 0]
    m.fail.clear()
    _, st2, solved2 = many.solve_many_resumable(m, f, str(tmp_path))
    assert solved2 == [1] and [s["status"] for s in st2] == [0, 0, 0]


def test_half_written_case_counts_as_pending(tmp_path):
    m, f = FakeMesh(), cases(3)
    many.solve_many_resumable(m, f, str(tmp_path))
    os.remove(os.path.join(tmp_path, "case_00001.json"))          # solution written, record not
    with open(os.path.join(tmp_path, "case_00002.json.tmp"), "w") as fh:
        fh.write("{")                                              # a rename that never happened
    _, _, solved = many.solve_many_resumable(m, f, str(tmp_path))
    assert solved == [1]
    meta = json.load(open(os.path.join(tmp_path, "case_00001.json")))
    assert meta["case"] == 1 and meta["status"] == 0 and len(meta["f_sha256"]) == 64
