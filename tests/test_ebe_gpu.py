"""GPU parity of the EBE product (fe_ebe_apply through the C ABI) against the
CPU oracle's assembled CSR product.

Bar: relative L2 error <= 1e-12 in FP64 and <= 2e-6 in FP32 (the FP32 input is
the FP32-rounded x, and the oracle evaluates that same x in FP64).
"""
import numpy as np
import pytest

from _util import ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

TOL64, TOL32 = 1e-12, 2e-6


def gpu_mesh(m):
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    return fe.Mesh.from_mesh(m)


def run(M, x, dtype, variant=None, tile=48):
    """Product through the C ABI; for the tiled kernel, the largest tile <= `tile`
    (halving) whose shared-memory footprint fits at this R and precision."""
    from paper_1710_08679_gb300 import fe
    t = torch.from_numpy(x).to("cuda", dtype=dtype)
    if variant is not None:
        while True:
            try:
                M.set_variant(x.shape[1], "f32" if dtype == torch.float32 else "f64", variant, tile)
                break
            except fe.FeError as exc:
                if variant == 0 or tile <= 1 or "does not fit" not in str(exc):
                    raise
                tile //= 2
    y = M.ebe(t)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


MESHES = {
    "box1": lambda: mg.plain_box(n=1, jitter=0.0),
    "box2": lambda: mg.plain_box(n=2, jitter=0.1, seed=4),
    "ragged": lambda: mg.crust_block(shape=(5, 3, 4), h=1000.0, jitter=0.15, seed=2)[0],
    "box8": lambda: mg.plain_box(),
}


@pytest.fixture(scope="module", params=list(MESHES))
def mesh_pair(request):
    m = MESHES[request.param]()
    return m, oracle.assemble(m), gpu_mesh(m)


@pytest.mark.gpu
@pytest.mark.parametrize("R", [1, 3, 4, 16, 32])
@pytest.mark.parametrize("variant", [0, 1, 2, 5])
def test_ebe_fp64_matches_oracle(mesh_pair, R, variant):
    m, K, M = mesh_pair
    x = mg.random_vectors(m.n_nodes, R, seed=100 + R)
    y_ref = oracle.spmv(K, x)
    y = run(M, x, torch.float64, variant, tile=48)
    assert rel_l2(y, y_ref) <= TOL64


@pytest.mark.gpu
@pytest.mark.parametrize("R", [1, 3, 4, 16, 32])
@pytest.mark.parametrize("variant", [0, 1, 2, 5])
def test_ebe_fp32_matches_oracle(mesh_pair, R, variant):
    m, K, M = mesh_pair
    x = mg.random_vectors(m.n_nodes, R, seed=200 + R).astype(np.float32).astype(np.float64)
    y_ref = oracle.spmv(K, x)
    y = run(M, x, torch.float32, variant, tile=24)
    assert rel_l2(y, y_ref) <= TOL32


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("tile", [1, 7, 24, 96, 384])
def test_tiled_tile_sizes_and_ragged_tail(tile, variant):
    m = MESHES["ragged"]()
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, 4, seed=9)
    y = run(M, x, torch.float64, variant, tile=tile)
    assert rel_l2(y, oracle.spmv(K, x)) <= TOL64
    kind, used = M.get_variant(4, "f64")
    assert kind == variant and 1 <= used <= tile      # the largest fitting tile <= the request
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = run(M, x32, torch.float32, variant, tile=tile)
    assert rel_l2(y32, oracle.spmv(K, x32)) <= TOL32


@pytest.mark.gpu
@pytest.mark.parametrize("R,dtype", [(16, "f32"), (4, "f32"), (32, "f32"), (4, "f64"), (16, "f64")])
def test_gather_many_tiles_per_cta(R, dtype):
    """Small tiles on a 24,000-element crust block: thousands of tiles, so every
    persistent CTA walks many tiles through the prefetch pipeline."""
    m, _ = mg.crust_block(shape=(20, 20, 10), h=1000.0, jitter=0.15, seed=5)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, R, seed=31)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    for tile in (4, 13):
        y = run(M, x, tdt, 2, tile=tile)
        assert rel_l2(y, oracle.spmv(K, x)) <= (TOL32 if dtype == "f32" else TOL64)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [3, 7])
@pytest.mark.parametrize("R", [2, 4, 16, 32])
def test_float_float_fp64_kernel_matches_oracle(mesh_pair, R, variant):
    """The FP64 product computed in float-float arithmetic on the FP32 pipe meets
    the FP64 bar (1e-12), in the one-block and the two-blocks-per-SM kernel."""
    m, K, M = mesh_pair
    x = mg.random_vectors(m.n_nodes, R, seed=300 + R)
    y = run(M, x, torch.float64, variant, tile=16)
    assert M.get_variant(R, "f64")[0] == variant
    assert rel_l2(y, oracle.spmv(K, x)) <= TOL64


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 16])
def test_float_float_kernels_agree(R):
    """The lean element routine performs the same operations in the same order as
    the one-block kernel's and the node sums add the slots in the same order, so
    the two float-float kernels agree far below the FP64 bar at the same tile size
    (not necessarily bitwise: the compiler may contract a product and a sum into
    one FMA differently in the two)."""
    m, _ = mg.crust_block(shape=(12, 10, 6), h=1000.0, jitter=0.15, seed=6)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, R, seed=61 + R)
    y3 = run(M, x, torch.float64, 3, tile=12)
    y7 = run(M, x, torch.float64, 7, tile=12)
    assert M.get_variant(R, "f64") == (7, 12)
    assert rel_l2(y7, y3) <= 1e-15


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 16])
def test_float_float_many_tiles_and_scales(R):
    """Many tiles per CTA, and inputs spanning 40 orders of magnitude."""
    m, _ = mg.crust_block(shape=(20, 20, 10), h=1000.0, jitter=0.15, seed=5)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    rng = np.random.default_rng(7)
    x = mg.random_vectors(m.n_nodes, R, seed=32) * 10.0 ** rng.uniform(-20, 20, size=(m.n_nodes, R, 1))
    y_ref = oracle.spmv(K, x)
    for variant in (3, 7):
        for tile in (4, 13):
            y = run(M, x, torch.float64, variant, tile=tile)
            for r in range(R):
                assert rel_l2(y[:, r], y_ref[:, r]) <= TOL64


@pytest.mark.gpu
@pytest.mark.parametrize("R,tile", [(32, 10), (16, 17), (8, 20), (2, 7)])
def test_float_float_tile_sizes_and_ragged_tail(R, tile):
    """Tiles with more element-case items than the CTA has threads (several
    passes, the last partly idle) and tile sizes that leave a ragged last tile:
    every output must land (FP64 bar, per case)."""
    m, _ = mg.crust_block(shape=(9, 7, 5), h=1000.0, jitter=0.15, seed=8)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, R, seed=41 + R)
    y_ref = oracle.spmv(K, x)
    for variant in (3, 7):
        y = run(M, x, torch.float64, variant, tile=tile)
        for r in range(R):
            assert rel_l2(y[:, r], y_ref[:, r]) <= TOL64


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 8, 16, 32])
def test_paired_fp32_kernel_matches_oracle(mesh_pair, R):
    """Two cases per thread (r and r + R/2) in paired FP32 arithmetic: every case
    on its own meets the FP32 bar, so the lanes are neither swapped nor mixed."""
    m, K, M = mesh_pair
    x = mg.random_vectors(m.n_nodes, R, seed=400 + R).astype(np.float32).astype(np.float64)
    y = run(M, x, torch.float32, 4, tile=24)
    assert M.get_variant(R, "f32")[0] == 4
    ref = oracle.spmv(K, x)
    for r in range(R):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 16, 32])
@pytest.mark.parametrize("tile", [1, 13, 48, 96])
def test_paired_fp32_tiles_and_ragged_tail(R, tile):
    """Paired kernel on a 24,000-element crust block: one-element tiles, a ragged
    last tile (24,000 = 13 x 1,846 + 2), and tiles with more element items than
    the CTA has threads (96 x R/2 > 384 for R >= 16)."""
    m, _ = mg.crust_block(shape=(20, 20, 10), h=1000.0, jitter=0.15, seed=5)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, R, seed=33).astype(np.float32).astype(np.float64)
    y = run(M, x, torch.float32, 4, tile=tile)
    kind, used = M.get_variant(R, "f32")
    assert kind == 4 and 1 <= used <= tile      # the largest fitting tile <= the request
    assert rel_l2(y, oracle.spmv(K, x)) <= TOL32


@pytest.mark.gpu
def test_paired_kernel_rejects_unsupported_requests():
    """FP64 or an R outside {4, 8, 16, 32}: fe_ebe_set_variant refuses, and the
    previous choice stays in force."""
    from paper_1710_08679_gb300 import fe
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    before = M.get_variant(16, "f64")
    for R, dt in ((16, "f64"), (3, "f32"), (1, "f32"), (64, "f32")):
        with pytest.raises(fe.FeError):
            M.set_variant(R, dt, 4, 24)
    assert M.get_variant(16, "f64") == before


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_colour_kernel_is_deterministic_and_matches_oracle(dtype):
    """Colour-by-colour products on a 24,000-element crust block: no atomics, so two
    calls give bitwise the same y, and y meets the oracle's bar (a colour holding
    two elements that share a node would lose updates and fail it)."""
    m, _ = mg.crust_block(shape=(20, 20, 10), h=1000.0, jitter=0.15, seed=5)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    R = 16
    tdt = torch.float32 if dtype == "f32" else torch.float64
    x = mg.random_vectors(m.n_nodes, R, seed=34)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    y1 = run(M, x, tdt, 5)
    y2 = run(M, x, tdt, 5)
    kind, n_colours = M.get_variant(R, dtype)
    # the elements sharing a node all need distinct colours
    max_incidence = int(np.bincount(m.conn.ravel()).max())
    assert kind == 5 and max_incidence <= n_colours <= 256
    assert np.array_equal(y1, y2)
    assert rel_l2(y1, oracle.spmv(K, x)) <= (TOL32 if dtype == "f32" else TOL64)


@pytest.mark.gpu
def test_batched_equals_separate_products():
    m = MESHES["box8"]()
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, 8, seed=5)
    yb = run(M, x, torch.float64)
    for r in (0, 3, 7):
        ys = run(M, np.ascontiguousarray(x[:, r:r + 1]), torch.float64)
        assert rel_l2(yb[:, r:r + 1], ys) <= 1e-14


@pytest.mark.gpu
def test_constrained_dofs_copy_input():
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, 2, seed=6)
    y = run(M, x, torch.float64)
    fixed = m.free == 0
    assert np.array_equal(y[:, 0][fixed], x[:, 0][fixed])
    assert np.array_equal(y[:, 1][fixed], x[:, 1][fixed])


@pytest.mark.gpu
def test_autotuner_picks_a_valid_kernel():
    m = MESHES["box8"]()
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    v, us = M.tune(16, "f32")
    assert v >= 0 and us > 0
    x = mg.random_vectors(m.n_nodes, 16, seed=7).astype(np.float32).astype(np.float64)
    y = run(M, x, torch.float32)
    assert rel_l2(y, oracle.spmv(K, x)) <= TOL32


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_crust_block_sampled_rows(dtype):
    """The 70x70x35-hexahedra crust block (1,029,000 elements, 4,234,653 DOF) at
    R = 16 in the kernel configuration the benchmark times (after tuning): rows
    sampled across the mesh against the oracle's element-by-element row sums."""
    m, _ = mg.crust_block()
    M = gpu_mesh(m)
    R = 16
    x = mg.random_vectors(m.n_nodes, R, seed=100 + R)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    M.tune(R, dtype)
    y = run(M, x, tdt)
    # the float-float (FP64) or paired-arithmetic (FP32) kernel too, whatever the tuner picked
    y2 = run(M, x, tdt, 3, tile=16) if dtype == "f64" else run(M, x, tdt, 4, tile=48)
    rng = np.random.default_rng(0)
    nodes = np.unique(np.concatenate([rng.integers(0, m.n_nodes, 3000), [0, m.n_nodes - 1]]))
    ys = oracle.sampled_product(m, x, nodes)
    assert rel_l2(y[nodes], ys) <= (TOL64 if dtype == "f64" else TOL32)
    assert rel_l2(y2[nodes], ys) <= (TOL64 if dtype == "f64" else TOL32)


@pytest.mark.gpu
@pytest.mark.slow
def test_full_size_crust_block_R32_paired_kernel():
    """R = 32 on the full crust block in the configuration the benchmark's sweep
    reports for it (paired-arithmetic kernel, 24-element tiles): sampled rows
    against the oracle's element-by-element row sums."""
    m, _ = mg.crust_block()
    M = gpu_mesh(m)
    R = 32
    x = mg.random_vectors(m.n_nodes, R, seed=100 + R).astype(np.float32).astype(np.float64)
    y = run(M, x, torch.float32, 4, tile=24)
    assert M.get_variant(R, "f32") == (4, 24)
    rng = np.random.default_rng(1)
    nodes = np.unique(np.concatenate([rng.integers(0, m.n_nodes, 2000), [0, m.n_nodes - 1]]))
    ys = oracle.sampled_product(m, x, nodes)
    assert rel_l2(y[nodes], ys) <= TOL32
    for r in (0, 15, 16, 31):   # both lanes of the pairs (r, r + 16)
        assert rel_l2(y[nodes, r], ys[:, r]) <= TOL32, r


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_products_pipeline_across_calls(dtype, pinned):
    """fe_ebe_apply_host: three calls in a row with different host inputs (the
    copies of consecutive calls overlap) each give the oracle's product."""
    m = MESHES["ragged"]()
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    xs = [torch.from_numpy(mg.random_vectors(m.n_nodes, 4, seed=80 + k)).to(tdt) for k in range(3)]
    if pinned:
        xs = [x.pin_memory() for x in xs]
    ys = [torch.empty_like(x).pin_memory() if pinned else torch.empty_like(x) for x in xs]
    for x, y in zip(xs, ys):
        M.ebe_host(x, out=y)
    torch.cuda.synchronize()
    for x, y in zip(xs, ys):
        ref = oracle.spmv(K, x.double().numpy())
        assert rel_l2(y.double().numpy(), ref) <= (TOL32 if dtype == "f32" else TOL64)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_largest_case_count_R64(dtype):
    """R = 64, the largest batch the ABI accepts (the tuned choice among the
    kernels compiled for it), against the oracle."""
    m = MESHES["ragged"]()
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = mg.random_vectors(m.n_nodes, 64, seed=64)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    M.tune(64, dtype)
    y = run(M, x, torch.float32 if dtype == "f32" else torch.float64)
    assert rel_l2(y, oracle.spmv(K, x)) <= (TOL32 if dtype == "f32" else TOL64)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 7])
def test_fully_constrained_mesh_is_identity(variant):
    """Every DOF fixed: K_bc = I, so every kernel must return x exactly (the
    paired kernel computes FP32 products only)."""
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = MESHES["box2"]()
    M = fe.Mesh(m.coords, m.conn, m.young, m.poisson, np.zeros_like(m.free))
    for dtype in ((torch.float32,) if variant == 4 else (torch.float64,) if variant in (3, 7)
                  else (torch.float64, torch.float32)):
        x = torch.from_numpy(mg.random_vectors(m.n_nodes, 4, seed=9)).to(dtype)
        y = run(M, x.numpy().astype(np.float64), dtype, variant, tile=8)
        assert np.array_equal(y, x.double().numpy())
