"""Benchmark: EBE product throughput (GDOF x cases / s) on the 70x70x35-hexahedra
layered crust block (1,029,000 TET10 elements, 4,234,653 DOF), FP32, R = 16, plus
the batched mixed-precision solve against the plain one-case FP64 PCG on the same
mesh (case-solves / s at relative residual 1e-8).

One timed step = one fe_ebe_apply of R = 16 load cases (the product of Eq. 3 that
dominates the inner loop). Inputs stay resident in HBM; x and y (271 MB each) are
larger than L2, so no L2 flush is needed between steps. Multi-GPU (torchrun):
every rank holds the mesh and its own cases (case sharding, weak scaling, no
data-path collective); rank 0 prints the line, value = all ranks' work / max time.

--impl reference times the CPU oracle (assembled CSR product) on a bounded slab
of the same workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EBE GDOF·cases/s and case-solves/s at 1e-8 residual; batched-mixed vs plain FP64"
SHAPE = (70, 70, 35)
# inner-loop settings tuned on GB300 (level 0: 0.01 / 100 steps, level 1: 0.01 / 500);
# the paper's table (0.1 / 30, 0.05 / 300) is the library default
GB300_LOOPS = dict(eps_inner=0.01, n_inner=100, eps_inner1=0.01, n_inner1=500)
R_MAIN = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true", help="skip the solve comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the R / precision sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--shape", default=None, help="override mesh shape, e.g. 20x20x10 (testing only)")
    ap.add_argument("--profile", action="store_true",
                    help="EBE timing only, kernel fixed by --variant/--tile (no tuning, e2e, sweep, solve, CPU)")
    ap.add_argument("--variant", default="direct", choices=["direct", "tiled", "gather", "df", "x2", "colour", "ws", "dflean", "ws2"],
                    help="kernel for --profile (df: float-float FP64 kernel, --dtype f64 only)")
    ap.add_argument("--tile", type=int, default=48, help="elements per tile for --variant tiled")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"], help="precision for --profile")
    ap.add_argument("--workload", default="ebe", choices=["ebe", "many", "two_layer", "coarse", "solve", "adjoint", "cpu_solves", "inner_steps"],
                    help="ebe: the EBE line on the 70x70x35 crust block (default); many: 96 unit-slip cases on "
                         "the 120x120x60 block through fe_solve_many vs the plain FP64 PCG one case at a time; "
                         "cpu_solves: the oracle's plain PCG timed on the host cores on the solve meshes")
    ap.add_argument("--cpu-solves-small", action="store_true", help="cpu_solves on 24x24x12 meshes (testing only)")
    ap.add_argument("--many-cases", type=int, default=96, help="cases of --workload many")
    ap.add_argument("--fd-directions", type=int, default=10, help="random directions of the FD noise check "
                    "of --workload adjoint")
    ap.add_argument("--many-plain", type=int, default=1, help="cases timed with the plain FP64 PCG")
    ap.add_argument("--solver", choices=["pcg64", "fcg_mixed", "fcg_mg", "fcg_amg"], default="fcg_mg",
                    help="solver of --workload solve")
    ap.add_argument("--many-solver", choices=["fcg_mixed", "fcg_mg", "fcg_amg"], default="fcg_mixed",
                    help="many-case solver: inner loop at level 0 only, with the TET4 level 1 first, or with "
                         "levels 2 and 1 first")
    ap.add_argument("--many-loops", choices=["paper", "gb300"], default="paper",
                    help="inner-loop settings of --workload many: the paper's table (0.1/30, 0.05/300) or the "
                         "GB300-tuned 0.01/100, 0.01/500")
    return ap.parse_args()


def aggregate(units_per_rank: float, elapsed_ms: float, dist=None, device=None):
    """Whole-job throughput of a case-sharded run: every rank did `units_per_rank`
    units; the job took as long as the slowest rank. Returns (units/s over all
    ranks, max elapsed ms). With `dist` (torch.distributed, initialised) the max
    is taken over ranks; this is the only collective and it is not on the data path."""
    import torch
    world = dist.get_world_size() if dist is not None else 1
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return units_per_rank * world / (tmax * 1e-3), tmax


def shard_cases(n_cases: int, world: int, rank: int) -> range:
    """The contiguous block of case indices rank `rank` of `world` solves: sizes differ
    by at most one, earlier ranks take the larger blocks, every case goes to exactly
    one rank. Cases are independent right-hand sides, so the ranks exchange nothing
    while they solve."""
    if world < 1 or not 0 <= rank < world or n_cases < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n_cases, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def aggregate_sharded(units_this_rank: float, elapsed_ms: float, dist=None, device=None):
    """Whole-job throughput when ranks did different numbers of units: (sum of the
    units over ranks / slowest rank's time, max elapsed ms, total units). Two
    all-reduces after the timed region, none inside it."""
    import torch
    u = torch.tensor([float(units_this_rank)], dtype=torch.float64, device=device)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    if dist is not None and dist.get_world_size() > 1:
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total, tmax = float(u.item()), float(t.item())
    return total / (tmax * 1e-3), tmax, total


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(shape):
    from paper_1710_08679_gb300 import meshgen as mg
    m, iface = mg.crust_block(shape=shape, h=1000.0, jitter=0.15, seed=1)
    return m, iface


def ebe_flops_per_element(R: int) -> float:
    """Algorithmic flops of the lean element product (multiply-add = 2):
    774 per case and element plus 100 per element for geometry and Lame constants
    (counted from the element arithmetic)."""
    return 774.0 * R + 100.0


def ebe_bytes(N: int, E: int, R: int, s: int) -> float:
    """Algorithmic bytes per product: connectivity (40 B) and material (2s) per
    element, coordinates (3s) per node, x read once and y written once."""
    return E * (40.0 + 2 * s) + N * (3 * s + 2 * 3 * R * s)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock = 80.5


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded slab of the same mesh)
# ---------------------------------------------------------------------------
def oracle_slab(m, n_layers: int):
    """Elements of the bottom `n_layers` hexahedron layers (hexahedra are stored
    k-major, 6 tetrahedra each) with their nodes renumbered."""
    nx, ny, _ = m.shape
    ne = nx * ny * 6 * n_layers
    conn = m.conn[:ne]
    used = np.unique(conn)
    remap = -np.ones(m.n_nodes, dtype=np.int64)
    remap[used] = np.arange(used.size)
    from paper_1710_08679_gb300 import meshgen as mg
    return mg.Mesh(coords=m.coords[used], conn=remap[conn].astype(np.int32), young=m.young[:ne],
                   poisson=m.poisson[:ne], free=m.free[used], shape=(nx, ny, n_layers), h=m.h, lengths=m.lengths)


def cpu_baseline(m, R: int, reps: int = 3, n_layers: int = 4):
    import oracle
    sub = oracle_slab(m, n_layers)
    t0 = time.perf_counter()
    K = oracle.assemble(sub)
    t_asm = time.perf_counter() - t0
    from paper_1710_08679_gb300 import meshgen as mg
    x = mg.random_vectors(sub.n_nodes, R, seed=100 + R)
    oracle.spmv(K, x)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.spmv(K, x)
    t = (time.perf_counter() - t0) / reps
    return {"value": 3 * sub.n_nodes * R / t / 1e9, "unit": "GDOF·cases/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": (f"assembled CSR product y = K_bc x of the bottom {n_layers} of 35 hexahedron layers "
                       f"({sub.n_elem} elements, {3 * sub.n_nodes} DOF), R = {R}, FP64, mean of {reps}; "
                       f"assembly {t_asm:.1f} s not included")}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    m, _ = make_workload(shape)
    import oracle
    sub = oracle_slab(m, 4)
    K = oracle.assemble(sub)
    from paper_1710_08679_gb300 import meshgen as mg
    x = mg.random_vectors(sub.n_nodes, R_MAIN, seed=100 + R_MAIN)
    for _ in range(args.warmup):
        oracle.spmv(K, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(K, x)
    t = time.perf_counter() - t0
    val = 3 * sub.n_nodes * R_MAIN * args.steps / t / 1e9
    out = {"metric": METRIC, "value": val, "unit": "GDOF·cases/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "crust_%dx%dx%d_tet10_R%d_fp32_ebe" % (shape + (R_MAIN,)), "R": R_MAIN,
                      "mesh_elements": m.n_elem, "mesh_dof": 3 * m.n_nodes,
                      "parallelism": "oracle on the host cores (rate of a bounded sample, per DOF x case)"},
           "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": val,
                            "sample": f"assembled CSR product of the bottom 4 of {shape[2]} hexahedron layers "
                                      f"({sub.n_elem} elements, {3 * sub.n_nodes} DOF), R = {R_MAIN}, FP64; "
                                      f"assembly not timed"},
           "e2e": {"value": val, "unit": "GDOF·cases/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_ebe(M, x, y, steps, warmup, torch):
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        M.ebe(x, out=y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.nvtx.range_push("timed")
    ev[0].record(s)
    for k in range(steps):
        M.ebe(x, out=y)
        ev[k + 1].record(s)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[-1]), per


def slip_rhs(m, iface, R, M_ext, torch, fe, profile="uniform"):
    """Split-node forces of R unit-slip patches, computed on the GPU with the EBE
    product of each patch's hanging-wall elements: f = -P sum K_e s_e."""
    from paper_1710_08679_gb300 import meshgen as mg
    cases = mg.patch_grid_cases(m, iface, profile=profile)[:R]
    f = torch.zeros((m.n_nodes, R, 3), dtype=torch.float64, device="cuda")
    free = torch.from_numpy(m.free.astype(np.float64)).cuda()
    for r, c in enumerate(cases):
        sub = mg.Mesh(coords=m.coords, conn=m.conn[c.elems], young=m.young[c.elems], poisson=m.poisson[c.elems],
                      free=np.ones_like(m.free), shape=m.shape, h=m.h, lengths=m.lengths)
        Ms = fe.Mesh.from_mesh(sub)
        y = Ms.ebe(torch.from_numpy(np.ascontiguousarray(c.slip[:, None, :])).cuda())
        f[:, r, :] = -y[:, 0, :] * free
        Ms.close()
    return f


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg

    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    m, iface = make_workload(shape)
    N, E = m.n_nodes, m.n_elem
    M = fe.Mesh.from_mesh(m, device=torch.cuda.current_device())
    R = R_MAIN
    if args.profile:
        M.set_variant(R, args.dtype, {"direct": 0, "tiled": 1, "gather": 2, "df": 3, "x2": 4, "colour": 5, "ws": 6,
                                    "dflean": 7, "ws2": 8}[args.variant], args.tile)
        tt = torch.float32 if args.dtype == "f32" else torch.float64
        x = torch.from_numpy(mg.random_vectors(N, R, seed=100 + R)).to("cuda", tt)
        y = torch.empty_like(x)
        ms, per = time_ebe(M, x, y, args.steps, args.warmup, torch)
        print(json.dumps({"profile": True, "variant": args.variant, "tile": args.tile, "dtype": args.dtype, "R": R,
                          "ms_per_product": ms / args.steps, "per_step_ms": per}), flush=True)
        return
    v32, us32 = M.tune(R, "f32")
    kind_name = {0: "direct", 1: "tiled", 2: "pipelined gather", 3: "gather-df",
                 4: "pipelined gather, two cases per thread in paired FP32", 5: "colour by colour",
                 6: "warp-specialised", 7: "gather-df-lean", 8: "warp-specialised, two blocks per SM"}[v32 // 65536]
    kernel_desc = kind_name + ("" if v32 // 65536 in (0, 5) else " %d elements/tile" % (v32 % 65536))
    first_pass = "prep pass (element geometry, y = 0)" if v32 // 65536 in (2, 4) else "zero pass"
    # zero or prep pass + the kernel; the colour kernel launches once per colour
    launches_per_product = 1 + (v32 % 65536 if v32 // 65536 == 5 else 1)
    x = torch.from_numpy(mg.random_vectors(N, R, seed=100 + R + rank).astype(np.float32)).cuda()
    y = torch.empty_like(x)

    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[torch.cuda.current_device()]))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    total_ms, per = time_ebe(M, x, y, args.steps, args.warmup, torch)
    clocks = sampler.stop()
    rate, total_ms = aggregate(3.0 * N * R * args.steps, total_ms, dist if world > 1 else None, "cuda")
    value = rate / 1e9
    ms_step = total_ms / args.steps
    ebe_ms = float(np.mean(per))

    # e2e: through fe_ebe_apply_host, every step copies its x from pinned host memory
    # and its y back (consecutive calls overlap copy-in, product and copy-out)
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(3):
        M.ebe_host(xh, out=yh)
    torch.cuda.synchronize()
    e_steps = max(5, args.steps // 5)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(e_steps):
        M.ebe_host(xh, out=yh)
    t1.record()
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / e_steps
    e2e = {"value": 3.0 * N * R * world / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF·cases/s",
           "h2d_bytes_per_step": int(x.numel() * 4), "d2h_bytes_per_step": int(y.numel() * 4),
           "api": "fe_ebe_apply_host (pinned host x and y, copies overlapped across calls)"}

    hbm, peak_src = load_peaks()
    flops = E * ebe_flops_per_element(R)
    achieved_tf = flops / (ebe_ms * 1e-3) / 1e12
    bytes_alg = ebe_bytes(N, E, R, 4)
    achieved_gbs = bytes_alg / (ebe_ms * 1e-3) / 1e9
    traffic = None
    ncu = None
    tp = os.path.join(ROOT, "profiles", "ebe_traffic.json")
    if os.path.exists(tp):
        # the committed capture counts only while the kernel's sources are the ones it measured
        try:
            import hashlib
            tj = json.load(open(tp))
            same_src = bool(tj.get("source_sha256")) and all(
                hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                for f, h in tj.get("source_sha256", {}).items())
            applies = (same_src and tj.get("variant") == kernel_desc and tj.get("shape") == list(shape)
                       and tj.get("R") == R)
            if applies:
                traffic = tj.get("traffic_bytes_per_launch")
            ncu = {"kernel": tj.get("kernel"), "counters": tj.get("kernels"), "command": tj.get("command"),
                   "applies_to_this_run": applies,
                   "note": "one ncu capture of the committed kernel (DRAM bytes and duration of one launch, "
                           "cold caches); used for roofline.traffic only while its source hash and "
                           "configuration match this run"}
        except Exception:
            traffic, ncu = None, None
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP32_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "fe_ebe_apply (%s + %s EBE kernel)" % (first_pass, kernel_desc),
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                        "peak_source": peak_src, "algorithmic_bytes": bytes_alg}}

    out = {"metric": METRIC, "value": value, "unit": "GDOF·cases/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "crust_%dx%dx%d_tet10_R%d_fp32_ebe" % (shape + (R,)), "mesh_elements": E,
                      "mesh_dof": 3 * N, "R": R, "kernel_variant": kernel_desc,
                      "l2": "inputs larger than L2 (x and y %d MB each), no flush" % (x.numel() * 4 // 2 ** 20),
                      "parallelism": "case-sharded replicas x%d" % world},
           "e2e": e2e, "gpu_launches": launches_per_product * args.steps, "roofline": roofline, "clocks": clocks,
           "ncu": ncu}

    if not args.no_sweep:
        sweep = {}
        for dt in ("f32", "f64"):
            for RR in (1, 4, 8, 16, 32):
                M.tune(RR, dt)
                tt = torch.float32 if dt == "f32" else torch.float64
                xx = torch.from_numpy(mg.random_vectors(N, RR, seed=100 + RR)).to("cuda", tt)
                yy = torch.empty_like(xx)
                ms, _ = time_ebe(M, xx, yy, 5 if dt == "f64" else 10, 2, torch)
                n = 5 if dt == "f64" else 10
                kv, kt = M.get_variant(RR, dt)
                sweep[f"{dt}_R{RR}"] = {"GDOF_cases_per_s": 3.0 * N * RR / (ms / n * 1e-3) / 1e9,
                                        "ms": ms / n, "variant": {0: "direct", 1: "tiled", 2: "gather", 3: "gather-df", 4: "gather-x2", 5: "colour", 6: "ws",
                                                    7: "gather-df-lean", 8: "ws2"}[kv],
                                        "tile": kt}
                del xx, yy
        out["ebe_sweep"] = sweep

    if not args.no_solve:
        out["solve"] = run_solves(m, iface, M, torch, fe, world)

    if rank == 0 and not args.no_cpu and world == 1:
        try:
            out["cpu_baseline"] = cpu_baseline(m, R)
            out["cpu_baseline"]["solve"] = cpu_solve_baseline(torch, fe)
        except Exception as exc:  # report, never fail the line
            out["cpu_baseline"] = {"error": str(exc)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def timed_solve(M, f, torch, reps=3, **kw):
    """One untimed solve (workspace, block Jacobi, coarse levels and kernel choices
    are set up on first use and then kept), then `reps` timed solves of the same
    batch; wall time to all cases converged (including the per-call graph capture)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, stats, st = M.solve(f, raise_on_fail=False, **kw)
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, stats, st = M.solve(f, raise_on_fail=False, **kw)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    return u, stats, st, {"first_call_seconds": first, "seconds_median": float(np.median(times)),
                          "seconds_min": float(np.min(times)), "seconds_max": float(np.max(times)), "repeats": reps}


def lanczos_condition(coef):
    """Extreme eigenvalues of M^-1 K from the CG coefficients of one case (the Lanczos
    tridiagonal: T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_k,k+1 = sqrt(beta_k)/alpha_k)."""
    from scipy.linalg import eigh_tridiagonal
    al, be = coef[:, 0], coef[:, 1]
    k = int(np.count_nonzero(al))
    al, be = al[:k], be[:k]
    d = 1.0 / al
    d[1:] += be[:-1] / al[:-1]
    e = np.sqrt(be[:-1]) / al[:-1]
    ev = eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[0]), float(ev[-1]), k


def block_condition(M, free):
    """Condition number of the block-Jacobi matrix M (the 3x3 diagonal blocks of K
    over each node's free components), from the inverse blocks the library builds."""
    B = M.block_jacobi().cpu().numpy()
    lo, hi = np.inf, 0.0
    for pat in np.unique(free, axis=0):
        idx = np.flatnonzero(pat)
        if idx.size == 0:
            continue
        sel = np.all(free == pat, axis=1)
        ev = 1.0 / np.linalg.eigvalsh(B[sel][:, idx][:, :, idx])
        lo, hi = min(lo, float(ev.min())), max(hi, float(ev.max()))
    return hi / lo


def run_solves(m, iface, M, torch, fe, world, profile="uniform",
               workload="crust_70x70x35_tet10 16 unit-slip patches (4x4 grid, 2x2 km)"):
    """Batched mixed FCG (R = 16 unit-slip patches) vs plain FP64 PCG, one case
    at a time, on the same mesh; both to true relative residual 1e-8. Every solver:
    one untimed solve, then three timed ones (median, min, max). The displacement
    error is bounded by kappa_est * relres, kappa_est = kappa(M) kappa(M^-1 K) with
    kappa(M^-1 K) from the Lanczos tridiagonal of the plain PCG's coefficients."""
    R = 16
    f = slip_rhs(m, iface, R, M, torch, fe, profile)
    M.tune(R, "f64")
    M.tune(1, "f64")
    M.tune(R, "f32")
    out = {"workload": workload, "timing": "one untimed solve, then the median of 3 timed solves (min/max given)"}
    # set-up of the coarse levels, once per mesh (reported, not in the solve times)
    t0 = time.perf_counter()
    M.coarse_block_jacobi()
    n4 = M.coarse_info()[0]
    M.coarse_apply(torch.zeros((n4, R, 3), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    coarse_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    M.level2_info()
    torch.cuda.synchronize()
    l2_setup = time.perf_counter() - t0
    # plain FP64 PCG, one case at a time (three cases), recording the CG coefficients of the first
    coef = np.zeros((4000, 1, 2))
    plain = []
    for r in range(3):
        fr = f[:, r:r + 1, :].contiguous()
        ur, sr, _, tm = timed_solve(M, fr, torch, reps=1, solver="pcg64", tol=1e-8,
                                    **({"cg_coef": coef} if r == 0 else {}))
        plain.append((ur, sr[0], tm))
    lmin, lmax, kc = lanczos_condition(coef[:, 0, :])
    kappa_pk = lmax / lmin
    kappa_m = block_condition(M, m.free)
    kappa = kappa_pk * kappa_m
    plain_s = [p[2]["seconds_median"] for p in plain]
    plain_rate = 1.0 / float(np.mean(plain_s))
    out["plain_pcg64_one_case"] = {
        "case_solves_per_s": plain_rate * world, "seconds_per_case": plain_s,
        "first_call_seconds": plain[0][2]["first_call_seconds"], "iters": [p[1]["outer"] for p in plain],
        "relres": [p[1]["relres"] for p in plain]}
    out["condition_estimate"] = {"kappa_MinvK_lanczos": kappa_pk, "lanczos_steps": kc, "lambda_min": lmin,
                                 "lambda_max": lmax, "kappa_M_blocks": kappa_m, "kappa_est": kappa,
                                 "note": "||u - u*|| / ||u*|| <= kappa_est * relres (kappa(K) <= kappa(M) kappa(M^-1 K))"}
    runs = [("mixed_fcg", dict(solver="fcg_mixed")),
            ("mixed_fcg_two_level", dict(solver="fcg_mg")),
            ("mixed_fcg_three_level", dict(solver="fcg_amg")),
            ("mixed_fcg_two_level_gb300_loops", dict(solver="fcg_mg", **GB300_LOOPS))]
    u_ref = None
    for name, kw in runs:
        u, stats, st, tm = timed_solve(M, f, torch, reps=3, tol=1e-8, **kw)
        relmax = max(s["relres"] for s in stats)
        entry = {"case_solves_per_s": R / tm["seconds_median"] * world, **tm,
                 "case_solves_per_s_min_max": [R / tm["seconds_max"] * world, R / tm["seconds_min"] * world],
                 "all_converged": all(s["relres"] <= 1e-8 for s in stats), "status": int(st),
                 "outer": [s["outer"] for s in stats], "inner0": [s["inner"] for s in stats],
                 "inner1": [s["inner1"] for s in stats], "inner2": [s["inner2"] for s in stats],
                 "relres_max": relmax, "displacement_error_bound": kappa * relmax,
                 "speedup_vs_plain": (R / tm["seconds_median"]) / plain_rate}
        if kw.get("n_inner") is not None or name.endswith("gb300_loops"):
            entry["loops"] = GB300_LOOPS
        if u_ref is None:
            u_ref = u
        else:
            entry["rel_diff_vs_one_level"] = float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref))
        # the plain solves of the first three cases against this batch
        entry["rel_diff_vs_plain"] = [float(torch.linalg.norm(p[0][:, 0] - u[:, r]) / torch.linalg.norm(p[0][:, 0]))
                                      for r, p in enumerate(plain)]
        out[name] = entry
    out["mixed_fcg_two_level"]["coarse_setup_seconds"] = coarse_setup
    out["mixed_fcg_three_level"]["level2_setup_seconds"] = l2_setup
    for name, _ in runs:
        out["speedup" + name[len("mixed_fcg"):]] = out[name]["speedup_vs_plain"]
    return out


def cpu_solve_baseline(torch, fe):
    """Solve leg of the CPU baseline on the plain box (8^3 hexahedra, 3,072 TET10,
    14,739 DOF, one double couple): the oracle's block-Jacobi PCG to 1e-8 timed
    with one thread and with every host core (assembly timed apart), and, as the
    displacement error of the GPU solvers, their solutions against the oracle's
    sparse direct solution of the same system."""
    import oracle
    from paper_1710_08679_gb300 import meshgen as mg
    m = mg.plain_box()
    f = mg.plain_box_rhs(m)
    cores = os.cpu_count()
    t0 = time.perf_counter()
    K = oracle.assemble(m)
    t_asm = time.perf_counter() - t0
    out = {"kind": "oracle", "unit": "case-solves/s", "assembly_seconds": t_asm,
           "sample": "plain box 8^3 hexahedra (3,072 TET10, 14,739 DOF), one double couple, FP64 block-Jacobi "
                     "PCG to 1e-8; assembly not in the rate"}
    for n in (1, cores):
        oracle.set_num_threads(n)
        t0 = time.perf_counter()
        u_cg, it, rel = oracle.pcg(K, f, tol=1e-8)
        dt = time.perf_counter() - t0
        out["threads_%d" % n] = {"cores": oracle.num_threads(), "seconds": dt, "case_solves_per_s": 1.0 / dt,
                                 "iters": int(it[0]), "relres": float(rel[0])}
    oracle.set_num_threads(cores)
    out["value"], out["cores"] = out["threads_%d" % cores]["case_solves_per_s"], cores
    ud = oracle.direct_solve(K, f)
    out["oracle_pcg_error_vs_direct"] = float(np.linalg.norm(u_cg - ud) / np.linalg.norm(ud))
    M = fe.Mesh.from_mesh(m)
    gpu = {}
    for name in ("pcg64", "fcg_mixed", "fcg_mg"):
        u, stats, st = M.solve(torch.from_numpy(f).cuda(), solver=name, tol=1e-8, raise_on_fail=False)
        gpu[name] = {"relres": stats[0]["relres"], "outer": stats[0]["outer"],
                     "displacement_error_vs_oracle_direct": float(np.linalg.norm(u.cpu().numpy() - ud) /
                                                                  np.linalg.norm(ud))}
    M.close()
    out["gpu_displacement_error"] = gpu
    return out


def run_cpu_solves(args):
    """The oracle's plain FP64 PCG on the bench meshes, timed on the host cores: the
    plain box solved in full (cpu_solve_baseline), the 70x70x35 crust block with its
    first two slip cases and the 120x120x60 block with its first case. On the two
    large meshes the oracle runs a bounded number of iterations and the full solve
    is projected from its seconds per iteration times the iteration count the GPU's
    plain FP64 PCG needs for the same right-hand side (measured here); assembly
    and block-Jacobi set-up are timed apart."""
    import torch
    import oracle
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg
    cores = os.cpu_count()
    out = {"metric": "oracle case-solves/s (plain FP64 block-Jacobi PCG to 1e-8) on the host cores",
           "impl": "oracle", "host_cores": cores, "plain_box": cpu_solve_baseline(torch, fe)}
    for key, shape, n_cases, maker, iters in (
            ("crust_70x70x35_2_cases", (70, 70, 35), 2, "patch", (20, 5)),
            ("crust_120x120x60_1_case", (120, 120, 60), 1, "many", (6, 2))):
        if args.cpu_solves_small:
            shape = (24, 24, 12)
        if maker == "patch":
            m, iface = make_workload(shape)
            M = fe.Mesh.from_mesh(m)
            f = slip_rhs(m, iface, n_cases, M, torch, fe)
        else:
            m, iface = mg.crust_block(shape=shape, h=1000.0, jitter=0.10, seed=3, n_layers=6)
            M = fe.Mesh.from_mesh(m)
            sc = mg.many_cases(m, iface, n_patches=1, seed=3)[0]
            sub = mg.Mesh(coords=m.coords, conn=m.conn[sc.elems], young=m.young[sc.elems],
                          poisson=m.poisson[sc.elems], free=np.ones_like(m.free), shape=m.shape, h=m.h,
                          lengths=m.lengths)
            Ms = fe.Mesh.from_mesh(sub)
            free = torch.from_numpy(m.free.astype(np.float64)).cuda()
            f = (-Ms.ebe(torch.from_numpy(np.ascontiguousarray(sc.slip[:, None, :])).cuda()) *
                 free[:, None, :]).contiguous()
            Ms.close()
        gpu_iters = []
        for r in range(n_cases):
            _, st_r, _ = M.solve(f[:, r:r + 1, :].contiguous(), solver="pcg64", tol=1e-8, raise_on_fail=False)
            gpu_iters.append(int(st_r[0]["outer"]))
        M.close()
        fh = f.cpu().numpy()
        del f
        torch.cuda.empty_cache()
        oracle.set_num_threads(cores)
        t0 = time.perf_counter()
        K = oracle.assemble(m)
        t_asm = time.perf_counter() - t0
        t0 = time.perf_counter()
        Minv = oracle.block_jacobi(K)
        t_bj = time.perf_counter() - t0
        entry = {"mesh_elements": m.n_elem, "mesh_dof": 3 * m.n_nodes, "cases": n_cases,
                 "assembly_seconds": t_asm, "block_jacobi_seconds": t_bj, "gpu_pcg64_iters": gpu_iters}
        for n, k in ((cores, iters[0]), (1, iters[1])):
            oracle.set_num_threads(n)
            t0 = time.perf_counter()
            oracle.pcg(K, fh, tol=1e-30, maxit=k, Minv=Minv)
            per_it = (time.perf_counter() - t0) / k
            proj = per_it * max(gpu_iters)       # the batch runs until its slowest case converges
            entry["threads_%d" % n] = {"cores": oracle.num_threads(), "iterations_timed": k,
                                       "seconds_per_iteration": per_it, "projected_solve_seconds": proj,
                                       "projected_case_solves_per_s": n_cases / proj}
        oracle.set_num_threads(cores)
        out[key] = entry
        del K, Minv, fh
    out["value"] = out["crust_70x70x35_2_cases"]["threads_%d" % cores]["projected_case_solves_per_s"]
    out["unit"] = "case-solves/s"
    print(json.dumps(out), flush=True)


def run_many(args):
    """96 unit-slip cases (48 patches x strike/dip) on the 120x120x60-hexahedra,
    6-layer crust block (5,184,000 TET10, 21,083,403 DOF) through fe_solve_many
    (memory-aware slot count, converged slots refilled) against the plain FP64
    PCG one case at a time; both to true relative residual 1e-8. Under torchrun
    the cases are sharded over the ranks (shard_cases): every rank builds the
    mesh, solves its own block of cases with no exchange, and the job's time is
    the slowest rank's (strong scaling: the 96 cases are fixed)."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg
    shape = (120, 120, 60) if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    t0 = time.perf_counter()
    m, iface = mg.crust_block(shape=shape, h=1000.0, jitter=0.10, seed=3, n_layers=6)
    M = fe.Mesh.from_mesh(m, device=torch.cuda.current_device())
    cases_all = mg.many_cases(m, iface, n_patches=(args.many_cases + 1) // 2, seed=3)[:args.many_cases]
    mine = shard_cases(len(cases_all), world, rank)
    cases = [cases_all[c] for c in mine]
    F = torch.zeros((len(cases), m.n_nodes, 3), dtype=torch.float64, device="cuda")
    free = torch.from_numpy(m.free.astype(np.float64)).cuda()
    for c, sc in enumerate(cases):
        if len(sc.elems) == 0:
            continue
        sub = mg.Mesh(coords=m.coords, conn=m.conn[sc.elems], young=m.young[sc.elems], poisson=m.poisson[sc.elems],
                      free=np.ones_like(m.free), shape=m.shape, h=m.h, lengths=m.lengths)
        Ms = fe.Mesh.from_mesh(sub, device=torch.cuda.current_device())
        F[c] = -Ms.ebe(torch.from_numpy(np.ascontiguousarray(sc.slip[:, None, :])).cuda())[:, 0, :] * free
        Ms.close()
    # kernels for the slot count the memory-aware admission picks (32 here) are tuned
    # before the timed region; fe_solve_many would otherwise tune on first use
    for RR, dt in ((32, "f32"), (32, "f64"), (1, "f64")):
        M.tune(RR, dt)
    if args.many_solver in ("fcg_mg", "fcg_amg"):
        M.coarse_block_jacobi()
        M.coarse_matrix_info()          # assembled coarse matrices (and level 2) before the timed call
    setup_s = time.perf_counter() - t0
    loops = GB300_LOOPS if args.many_loops == "gb300" else {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, stats, st, R_used = M.solve_many(F, R_slots=0, solver=args.many_solver, tol=1e-8, raise_on_fail=False,
                                        **loops)
    torch.cuda.synchronize()
    t_many = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    rate, tmax_ms, total = aggregate_sharded(len(cases), 1e3 * t_many, dist if world > 1 else None, "cuda")
    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, {"stats": stats, "status": int(st), "slots": R_used, "seconds": t_many})
        stats = [s for g in gathered for s in g["stats"]]
        st = max(g["status"] for g in gathered)
        per_rank = [{"cases": len(g["stats"]), "seconds": g["seconds"], "slots": g["slots"]} for g in gathered]
    else:
        per_rank = [{"cases": len(cases), "seconds": t_many, "slots": R_used}]
    plain = []
    if rank == 0:
        for c in range(min(args.many_plain, len(cases))):
            fr = F[c].reshape(m.n_nodes, 1, 3).contiguous()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ur, sr, _ = M.solve(fr, solver="pcg64", tol=1e-8, raise_on_fail=False)
            torch.cuda.synchronize()
            plain.append({"seconds": time.perf_counter() - t1, "iters": sr[0]["outer"], "relres": sr[0]["relres"],
                          "rel_diff_vs_many": float(torch.linalg.norm(ur[:, 0] - u[c]) / torch.linalg.norm(ur[:, 0]))})
    plain_rate = 1.0 / float(np.mean([p["seconds"] for p in plain])) if plain else None
    if rank == 0:
        out = {"metric": "case-solves/s at 1e-8 residual, many-case admission vs plain FP64", "value": rate,
               "unit": "case-solves/s", "n_gpus": world, "higher_is_better": True,
               "scaling": "strong", "dtype": "f64+f32", "data": "synthetic",
               "config": {"workload": "crust_%dx%dx%d_tet10_%d_slip_cases" % (shape + (int(total),)),
                          "mesh_elements": m.n_elem, "mesh_dof": 3 * m.n_nodes, "slots": R_used,
                          "solver": args.many_solver, "inner_loops": args.many_loops, "setup_seconds": setup_s,
                          "parallelism": "cases sharded over %d rank(s), no exchange while solving" % world},
               "many": {"seconds": tmax_ms * 1e-3, "per_rank": per_rank, "status": int(st),
                        "all_converged": all(s["relres"] <= 1e-8 for s in stats),
                        "outer_min_max": [min(s["outer"] for s in stats), max(s["outer"] for s in stats)],
                        "inner0_total": sum(s["inner"] for s in stats), "inner1_total": sum(s["inner1"] for s in stats),
                        "inner2_total": sum(s["inner2"] for s in stats),
                        "relres_max": max(s["relres"] for s in stats)},
               "plain_pcg64_one_case": {"case_solves_per_s": plain_rate, "cases": plain,
                                        "note": "rank 0, one GPU"},
               "speedup": rate / plain_rate / world if plain_rate else None,
               "speedup_note": "job rate / (plain one-case rate x n_gpus): per-GPU speed-up over the plain solve"}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_inner_steps(args):
    """Time of one inner step (Algorithm 1(b)) per level on the 70x70x35 crust block
    with R = 16 slip cases: solves with the stop rule off (eps = 0), so every outer
    iteration runs exactly the given number of steps, and a fixed count of outer
    iterations (tol below reach); the step time is the difference between a run
    with n steps and one with none, divided by outer iterations x n. Level 1 is
    timed with the persistent inner-loop kernel and with per-step launches;
    level 0's step is compared with its FP32 EBE product."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import fe
    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    m, iface = make_workload(shape)
    M = fe.Mesh.from_mesh(m)
    R, n_outer = 16, 3
    f = slip_rhs(m, iface, R, M, torch, fe)
    M.tune(R, "f32")
    M.tune(R, "f64")

    def t_solve(**kw):
        _, _, _, tm = timed_solve(M, f, torch, reps=3, solver="fcg_mg", tol=1e-30, max_outer=n_outer, **kw)
        return tm["seconds_median"]

    out = {"metric": "inner-step time per level", "unit": "ms", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "crust_%dx%dx%d_tet10 16 unit-slip patches" % shape, "R": R,
                      "outer_iterations": n_outer, "timing": "median of 3 solves, difference of two step counts"}}
    base = dict(eps_inner=0.0, eps_inner1=0.0)
    for kind in ("persistent", "steps"):
        n1 = 200
        t0 = t_solve(n_inner=0, n_inner1=0, inner_kernel=kind, **base)
        t1 = t_solve(n_inner=0, n_inner1=n1, inner_kernel=kind, **base)
        out["level1_step_ms_" + kind] = 1e3 * (t1 - t0) / (n_outer * n1)
    n0 = 20
    t0 = t_solve(n_inner=0, n_inner1=0, **base)
    t1 = t_solve(n_inner=n0, n_inner1=0, **base)
    step0 = 1e3 * (t1 - t0) / (n_outer * n0)
    x = torch.randn((m.n_nodes, R, 3), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    ms, _ = time_ebe(M, x, y, 50, 5, torch)
    out["level0_step_ms"] = step0
    out["level0_ebe_ms"] = ms / 50
    out["level0_overhead_ms"] = step0 - ms / 50
    print(json.dumps(out), flush=True)


def run_two_layer(args):
    """The paper's two-layer Vp/Vs/rho model (soft top layer, nu = 0.467, 74x
    stiffness contrast) on the 70x70x35 block with 16 B-spline unit-slip patches:
    batched mixed FCG (level 0; levels 1 and 0) against the plain FP64 PCG one case
    at a time, all to true relative residual 1e-8."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg
    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    t0 = time.perf_counter()
    m, iface = mg.two_layer_block(shape=shape)
    M = fe.Mesh.from_mesh(m)
    M.tune(16, "f32")
    setup_s = time.perf_counter() - t0
    res = run_solves(m, iface, M, torch, fe, 1, profile="bspline",
                     workload="two_layer_%dx%dx%d_tet10 16 B-spline unit-slip patches (4x4 grid, 2x2 km)" % shape)
    out = {"metric": "case-solves/s at 1e-8 residual, batched mixed vs plain FP64",
           "value": res["mixed_fcg_two_level"]["case_solves_per_s"], "unit": "case-solves/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": res["workload"], "mesh_elements": m.n_elem, "mesh_dof": 3 * m.n_nodes,
                      "materials": "Vp/Vs/rho 1600/400/1850 (top 5 km), 5800/3000/2700", "setup_seconds": setup_s},
           "solve": res}
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Misfit and gradient of the adjoint workload: the 24^3-hexahedra box (82,944
    TET10, 352,947 DOF), 16 double-couple sources, 1,000 surface observations
    with 5 % noise. One evaluation = a batched forward solve of the 16 Green's
    functions, the adjoint solve and the element-sensitivity kernel, all to
    relative residual 1e-8 (mixed two-level solver); timed over --steps
    evaluations after --warmup, plus one central-difference check along a
    random direction with solves to 1e-13 by the one-level mixed solver (the
    adjoint right-hand side sits at the observation points, and FP64 cannot
    certify much below 1e-11 for it: the two-level solver stalls there, the
    one-level one gets through in a few hundred outer iterations)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import adjoint, fe
    from paper_1710_08679_gb300 import meshgen as mg
    m = mg.adjoint_box(n=24)
    M = fe.Mesh.from_mesh(m)
    sources = torch.from_numpy(mg.adjoint_sources(m)).cuda()
    obs_np = mg.surface_observations(m, 1000, (500.0, 7500.0), 2)
    obs = adjoint.Observation(M, obs_np.node, obs_np.weight)
    opts = dict(solver="fcg_mg", tol=1e-8)
    a = torch.ones(16, dtype=torch.float64, device="cuda")
    M.set_log_young(torch.from_numpy(mg.adjoint_true_logE(m)).cuda())
    G, _, _ = M.solve(sources, **opts)
    clean = obs.apply(M.combine_cases(G, a))
    rms = torch.sqrt(torch.mean(clean ** 2))
    d = clean + 0.05 * rms * torch.from_numpy(mg.noise(tuple(clean.shape), 2)).cuda()
    logE0 = torch.from_numpy(np.log(m.young)).cuda()
    for _ in range(max(args.warmup, 1)):
        adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, opts)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(steps):
        J0, g_logE, g_a = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, opts)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # one central difference along a random unit direction, solves at 1e-13
    fine = dict(solver="fcg_mixed", tol=1e-13)
    J0f, gf_logE, gf_a = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, fine)
    v = mg.unit_directions(1, m.n_elem + 16, seed=2)[0]
    ve, va = torch.from_numpy(v[:m.n_elem]).cuda(), torch.from_numpy(v[m.n_elem:]).cuda()
    h = 1e-6
    fd = (adjoint.misfit(M, logE0 + h * ve, a + h * va, sources, obs, d, fine) -
          adjoint.misfit(M, logE0 - h * ve, a - h * va, sources, obs, d, fine)) / (2 * h)
    an = float(gf_logE @ ve + gf_a @ va)
    # noise of J itself (solves to 1e-13; atomic summation order varies between runs)
    # and the central-difference error over further random directions
    Js = [adjoint.misfit(M, logE0, a, sources, obs, d, fine) for _ in range(5)]
    fd_err = []
    for v2 in mg.unit_directions(args.fd_directions, m.n_elem + 16, seed=5):
        ve2, va2 = torch.from_numpy(v2[:m.n_elem]).cuda(), torch.from_numpy(v2[m.n_elem:]).cuda()
        fd2 = (adjoint.misfit(M, logE0 + h * ve2, a + h * va2, sources, obs, d, fine) -
               adjoint.misfit(M, logE0 - h * ve2, a - h * va2, sources, obs, d, fine)) / (2 * h)
        fd_err.append(abs(float(gf_logE @ ve2 + gf_a @ va2) - fd2) / abs(J0f))
    noise = {"J_spread_over_5_evaluations_rel": (max(Js) - min(Js)) / abs(J0f),
             "fd_abs_error_rel_to_J": {"directions": len(fd_err), "max": max(fd_err) if fd_err else None,
                                       "median": float(np.median(fd_err)) if fd_err else None}}
    print(json.dumps({"metric": "adjoint gradient evaluations/s (forward + adjoint solves + sensitivity kernel)",
                      "value": 1.0 / dt, "unit": "gradients/s", "seconds_per_gradient": dt, "n_gpus": 1,
                      "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "adjoint box 24^3 hexahedra (82,944 TET10, 352,947 DOF), 16 sources, "
                                             "1,000 observations", "solver": "fcg_mg", "tol": 1e-8,
                                 "steps": steps},
                      "fd_check": {"directional_derivative": an, "central_difference": fd,
                                   "relative_difference": abs(an - fd) / max(abs(fd), 1e-300), "h": h,
                                   "solver": "fcg_mixed", "solve_tol": 1e-13}, "fd_noise": noise}), flush=True)


def run_one_solve(args):
    """One batched solve of the 16 slip patches on the 70x70x35 crust block with
    --solver, after all set-up (kernel tuning, coarse levels, one untimed solve),
    inside the NVTX range "timed_solve" (so a profiler can be limited to it)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg
    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    m, iface = make_workload(shape)
    M = fe.Mesh.from_mesh(m)
    R = R_MAIN
    f = slip_rhs(m, iface, R, M, torch, fe)
    M.tune(R, "f32")
    M.tune(R, "f64")
    M.tune(1, "f64")
    if args.solver in ("fcg_mg", "fcg_amg"):
        M.coarse_block_jacobi()
        M.coarse_matrix_info()
    M.solve(f, solver=args.solver, tol=1e-8, raise_on_fail=False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_solve")
    t0 = time.perf_counter()
    u, stats, st = M.solve(f, solver=args.solver, tol=1e-8, raise_on_fail=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": "crust_%dx%dx%d_tet10 16 unit-slip patches" % shape, "solver": args.solver,
                      "seconds": dt, "case_solves_per_s": R / dt, "status": int(st),
                      "outer": [s["outer"] for s in stats], "inner0": [s["inner"] for s in stats],
                      "inner1": [s["inner1"] for s in stats], "inner2": [s["inner2"] for s in stats],
                      "relres_max": max(s["relres"] for s in stats)}), flush=True)


def run_coarse(args):
    """The level-1 (TET4) and level-2 (aggregation) operators at R = 16, FP32, on
    the 70x70x35 crust block: assembled K1_bc product, TET4 element-by-element
    product, transfers, and the A2 product; CUDA events over --steps launches of
    each after --warmup. The assembled product's roofline: algorithmic bytes =
    blocks (36 B + 4 B column) + row pointers + x read once + y written once."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08679_gb300 import fe
    from paper_1710_08679_gb300 import meshgen as mg
    shape = SHAPE if not args.shape else tuple(int(v) for v in args.shape.split("x"))
    m, _ = mg.crust_block(shape=shape)
    M = fe.Mesh.from_mesh(m)
    R = R_MAIN
    n4 = M.coarse_info()[0]
    na = M.level2_info()[0]
    g = torch.Generator(device="cuda").manual_seed(5)
    x4 = torch.randn((n4, R, 3), generator=g, device="cuda", dtype=torch.float32)
    x10 = torch.randn((m.n_nodes, R, 3), generator=g, device="cuda", dtype=torch.float32)
    x2 = torch.randn((na, R, 3), generator=g, device="cuda", dtype=torch.float32)
    ops = {"assembled_K1": lambda: M.coarse_apply(x4), "tet4_ebe": lambda: M.ebe4(x4),
           "restrict_P1T": lambda: M.coarse_restrict(x10), "prolong_P1": lambda: M.coarse_prolong(x4),
           "A2": lambda: M.level2_apply(x2), "restrict_P2T": lambda: M.level2_restrict(x4),
           "prolong_P2": lambda: M.level2_prolong(x2)}
    res = {}
    for name, fn in ops.items():
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    nnzb, nnzb2 = M.coarse_matrix_info()
    bytes_k1 = nnzb * 40 + (n4 + 1) * 4 + 2 * n4 * R * 12
    gbs = bytes_k1 / (res["assembled_K1_ms"] * 1e-3) / 1e9
    hbm, hbm_src = load_peaks()
    out = {"metric": "coarse-level operator time (ms per product)", "unit": "ms", "n_gpus": 1,
           "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "crust_%dx%dx%d_tet10 coarse levels" % shape, "R": R, "coarse_nodes": n4,
                      "coarse_blocks": nnzb, "aggregates": na, "level2_blocks": nnzb2, "steps": args.steps,
                      "warmup": args.warmup},
           "times": res,
           "roofline_assembled_K1": {"bound": "hbm", "achieved": gbs, "peak": hbm, "peak_source": hbm_src,
                                     "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": bytes_k1}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "many":
        run_many(args)
    elif args.workload == "two_layer":
        run_two_layer(args)
    elif args.workload == "coarse":
        run_coarse(args)
    elif args.workload == "solve":
        run_one_solve(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "cpu_solves":
        run_cpu_solves(args)
    elif args.workload == "inner_steps":
        run_inner_steps(args)
    else:
        run_ours(args)



if __name__ == "__main__":
    main()
