"""GPU parity of the warp-specialised FP32 EBE kernel (FE_EBE_WS) against the CPU
oracle's assembled CSR product, through the C ABI.

Bar: relative L2 error <= 2e-6 per case (the FP32 input is the FP32-rounded x,
evaluated by the oracle in FP64). Every case is checked on its own, so the two
cases a compute thread carries in the lanes of its paired instructions can be
neither swapped nor mixed.
"""
import numpy as np
import pytest

from _util import ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

TOL32 = 2e-6
WS, WS2 = 6, 8     # 512-thread blocks (one per SM) and 256-thread blocks (two per SM)


def gpu_mesh(m, free=None):
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    if free is None:
        return fe.Mesh.from_mesh(m)
    return fe.Mesh(m.coords, m.conn, m.young, m.poisson, free)


def ws_product(M, x, tile, variant=WS):
    M.set_variant(x.shape[1], "f32", variant, tile)
    assert M.get_variant(x.shape[1], "f32") == (variant, tile)
    y = M.ebe(torch.from_numpy(x).to("cuda", torch.float32))
    M.device_status()   # no bounded wait of the kernel gave up
    return y.double().cpu().numpy()


def fp32_vectors(n, R, seed):
    return mg.random_vectors(n, R, seed=seed).astype(np.float32).astype(np.float64)


MESHES = {
    "box1": lambda: mg.plain_box(n=1, jitter=0.0),
    "box2": lambda: mg.plain_box(n=2, jitter=0.1, seed=4),
    "ragged": lambda: mg.crust_block(shape=(5, 3, 4), h=1000.0, jitter=0.15, seed=2)[0],
    "box8": lambda: mg.plain_box(),
}

# tile shapes that fit shared memory on every mesh here: 448 element-case items
# per tile (7 compute warps) for R = 16 and 32, 256 for R = 4 and 8
TILE = {4: 64, 8: 32, 16: 28, 32: 14}


@pytest.fixture(scope="module", params=list(MESHES))
def mesh_pair(request):
    m = MESHES[request.param]()
    return m, oracle.assemble(m), gpu_mesh(m)


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 8, 16, 32])
def test_ws_kernel_matches_oracle_per_case(mesh_pair, R):
    m, K, M = mesh_pair
    x = fp32_vectors(m.n_nodes, R, 500 + R)
    y = ws_product(M, x, TILE[R])
    ref = oracle.spmv(K, x)
    for r in range(R):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.fixture(scope="module")
def crust20():
    m, _ = mg.crust_block(shape=(20, 20, 10), h=1000.0, jitter=0.15, seed=5)
    return m, oracle.assemble(m), gpu_mesh(m)


# (R, tile): one compute warp and fifteen staging warps (R = 16, tile 4; R = 4,
# tile 16), two to seven compute warps, and tiles that do not divide the 24,000
# elements (ragged last tile: 28 and 14 elements)
WS_SHAPES = [(16, 4), (4, 16), (16, 8), (32, 8), (8, 40), (16, 24), (4, 80), (8, 48), (16, 28), (32, 14),
             (4, 48), (32, 12)]


@pytest.mark.gpu
@pytest.mark.parametrize("R,tile", WS_SHAPES)
def test_ws_many_tiles_shapes_and_ragged_tail(crust20, R, tile):
    """24,000-element crust block: hundreds to thousands of tiles, so every CTA
    walks many tiles through both stages and all three packet slots."""
    m, K, M = crust20
    x = fp32_vectors(m.n_nodes, R, 600 + R + tile)
    y = ws_product(M, x, tile)
    ref = oracle.spmv(K, x)
    assert rel_l2(y, ref) <= TOL32
    for r in (0, 1, R // 2, R - 1):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.mark.gpu
def test_ws_repeated_products_agree():
    """Ten products in a row on the same input: the stages and barriers leave no
    state behind (each call equals the oracle to the same bar; atomics only change
    the summation order)."""
    m, _ = mg.crust_block(shape=(12, 10, 6), h=1000.0, jitter=0.15, seed=8)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = fp32_vectors(m.n_nodes, 16, 77)
    ref = oracle.spmv(K, x)
    M.set_variant(16, "f32", WS, 28)
    t = torch.from_numpy(x).to("cuda", torch.float32)
    ys = [M.ebe(t).double().cpu().numpy() for _ in range(10)]
    for y in ys:
        assert rel_l2(y, ref) <= TOL32
        assert rel_l2(y, ys[0]) <= 1e-6


@pytest.mark.gpu
def test_ws_constrained_dofs_copy_input():
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    x = fp32_vectors(m.n_nodes, 16, 6)
    y = ws_product(M, x, 28)
    fixed = m.free == 0
    for r in range(16):
        assert np.array_equal(y[:, r][fixed], x[:, r][fixed])


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 16, 32])
def test_ws_fully_constrained_mesh_is_identity(R):
    m = MESHES["box2"]()
    M = gpu_mesh(m, free=np.zeros_like(m.free))
    x = fp32_vectors(m.n_nodes, R, 9)
    y = ws_product(M, x, TILE[R])
    assert np.array_equal(y, x)


@pytest.mark.gpu
def test_ws_zero_input_gives_zero():
    m = MESHES["ragged"]()
    M = gpu_mesh(m)
    y = ws_product(M, np.zeros((m.n_nodes, 16, 3)), 28)
    assert not np.any(y)


@pytest.mark.gpu
def test_ws_rejects_unsupported_requests():
    """FP64, an R outside {4, 8, 16, 32}, or a tile whose element-case items do not
    fill whole compute warps (or need more than twelve): fe_ebe_set_variant refuses
    and the previous choice stays in force."""
    from paper_1710_08679_gb300 import fe
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    before32, before64 = M.get_variant(16, "f32"), M.get_variant(16, "f64")
    for R, dt, tile in ((16, "f64", 32), (3, "f32", 32), (1, "f32", 64), (64, "f32", 8), (16, "f32", 6),
                        (16, "f32", 52), (4, "f32", 8), (32, "f32", 25)):
        with pytest.raises(fe.FeError):
            M.set_variant(R, dt, WS, tile)
    assert M.get_variant(16, "f32") == before32 and M.get_variant(16, "f64") == before64


@pytest.mark.gpu
def test_ws_after_material_change():
    """The kernel reads (E, nu) from the mesh at every product: after
    fe_mesh_set_log_young the product follows the new materials."""
    m = MESHES["ragged"]()
    M = gpu_mesh(m)
    rng = np.random.default_rng(3)
    logE = np.log(m.young) + rng.uniform(-0.5, 0.5, m.n_elem)
    M.set_log_young(torch.from_numpy(logE).cuda())
    m2 = mg.Mesh(coords=m.coords, conn=m.conn, young=np.exp(logE), poisson=m.poisson, free=m.free,
                 shape=m.shape, h=m.h, lengths=m.lengths)
    K2 = oracle.assemble(m2)
    x = fp32_vectors(m.n_nodes, 16, 12)
    y = ws_product(M, x, 28)
    assert rel_l2(y, oracle.spmv(K2, x)) <= TOL32


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("R", [16, 32])
def test_ws_full_size_crust_block_sampled_rows(R):
    """The 70x70x35-hexahedra crust block (1,029,000 elements, 4,234,653 DOF) with
    the default tile shape: rows sampled across the mesh against the oracle's
    element-by-element row sums, every case on its own."""
    m, _ = mg.crust_block()
    M = gpu_mesh(m)
    x = fp32_vectors(m.n_nodes, R, 100 + R)
    y = ws_product(M, x, TILE[R])
    rng = np.random.default_rng(2)
    nodes = np.unique(np.concatenate([rng.integers(0, m.n_nodes, 3000), [0, m.n_nodes - 1]]))
    ys = oracle.sampled_product(m, x, nodes)
    assert rel_l2(y[nodes], ys) <= TOL32
    for r in range(R):
        assert rel_l2(y[nodes, r], ys[:, r]) <= TOL32, r


# FE_EBE_WS2 (256-thread blocks, two per SM): one to four compute warps, i.e.
# tile * R / 2 in {32, 64, 96, 128}, with two blocks' buffers in one SM's shared
# memory (on the crust blocks that leaves three compute warps at most for
# R = 16 and 32, and two for R = 4)
WS2_SHAPES = [(16, 4), (16, 8), (16, 12), (4, 16), (4, 32), (8, 24), (32, 2), (32, 4), (32, 6), (8, 16)]
TILE2 = {4: 32, 8: 16, 16: 12, 32: 6}


@pytest.mark.gpu
@pytest.mark.parametrize("R", [4, 8, 16, 32])
def test_ws2_kernel_matches_oracle_per_case(mesh_pair, R):
    m, K, M = mesh_pair
    x = fp32_vectors(m.n_nodes, R, 700 + R)
    y = ws_product(M, x, TILE2[R], WS2)
    ref = oracle.spmv(K, x)
    for r in range(R):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.mark.gpu
@pytest.mark.parametrize("R,tile", WS2_SHAPES)
def test_ws2_many_tiles_shapes_and_ragged_tail(crust20, R, tile):
    m, K, M = crust20
    x = fp32_vectors(m.n_nodes, R, 800 + R + tile)
    y = ws_product(M, x, tile, WS2)
    ref = oracle.spmv(K, x)
    assert rel_l2(y, ref) <= TOL32
    for r in (0, 1, R // 2, R - 1):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.mark.gpu
@pytest.mark.parametrize("R,tile", [(16, 12), (4, 32), (32, 4), (8, 16)])
def test_ws2_ragged_last_tile(R, tile):
    """1,890 elements, not a multiple of 12, 32, 4 or 16: the last tile is short."""
    m, _ = mg.crust_block(shape=(9, 7, 5), h=1000.0, jitter=0.15, seed=8)
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    x = fp32_vectors(m.n_nodes, R, 900 + R)
    y = ws_product(M, x, tile, WS2)
    ref = oracle.spmv(K, x)
    for r in range(R):
        assert rel_l2(y[:, r], ref[:, r]) <= TOL32, r


@pytest.mark.gpu
def test_ws2_constrained_repeated_and_identity():
    """Constrained DOFs copy the input, ten products in a row agree, and a fully
    constrained mesh is the identity, with two blocks per SM."""
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    x = fp32_vectors(m.n_nodes, 16, 6)
    ys = [ws_product(M, x, 12, WS2) for _ in range(10)]
    fixed = m.free == 0
    for r in range(16):
        assert np.array_equal(ys[0][:, r][fixed], x[:, r][fixed])
    for y in ys[1:]:
        assert rel_l2(y, ys[0]) <= 1e-6
    Mf = gpu_mesh(m, free=np.zeros_like(m.free))
    assert np.array_equal(ws_product(Mf, x, 12, WS2), x)


@pytest.mark.gpu
def test_ws2_rejects_more_than_four_compute_warps():
    from paper_1710_08679_gb300 import fe
    m = MESHES["box2"]()
    M = gpu_mesh(m)
    for R, tile in ((16, 20), (32, 10), (4, 80)):       # 5 compute warps: too many for 256 threads
        with pytest.raises(fe.FeError):
            M.set_variant(R, "f32", WS2, tile)
