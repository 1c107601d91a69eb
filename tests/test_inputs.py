"""Checks of the seeded input generators that need no GPU: the paper's two-layer
Vp/Vs/rho materials and the B-spline unit-slip profile (Sec. 5)."""
import math

import numpy as np

import _util  # noqa: F401  (puts the repository root on sys.path)
from paper_1710_08679_gb300 import meshgen as mg


def test_moduli_reproduce_the_tabulated_wave_speeds():
    for vp, vs, rho in mg.PAPER_LAYERS:
        E, nu = mg.elastic_from_velocities(vp, vs, rho)
        mu = E / (2.0 * (1.0 + nu))
        lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        assert math.isclose(math.sqrt(mu / rho), vs, rel_tol=1e-12)
        assert math.isclose(math.sqrt((lam + 2.0 * mu) / rho), vp, rel_tol=1e-12)
    # the soft top layer is nearly incompressible
    assert abs(mg.elastic_from_velocities(*mg.PAPER_LAYERS[0])[1] - 7.0 / 15.0) < 1e-12


def test_two_layer_split_follows_hexahedron_layers():
    m, _ = mg.two_layer_block(shape=(6, 4, 6), soft_thickness=2000.0)
    soft = mg.elastic_from_velocities(*mg.PAPER_LAYERS[0])
    is_soft = m.young == soft[0]
    assert is_soft.sum() * 3 == m.n_elem              # the top 2 of 6 hexahedron layers
    assert np.all(m.centroids()[is_soft, 2] > 4000.0)
    assert np.all(m.centroids()[~is_soft, 2] < 4000.0)


def test_cubic_bspline_is_a_partition_of_unity():
    t = np.linspace(-0.5, 0.5, 101)
    total = sum(mg.bspline3(t - k) for k in range(-3, 4))
    assert np.allclose(total, 1.0, atol=1e-14)
    assert mg.bspline3(np.array([0.0]))[0] == 2.0 / 3.0
    assert np.all(mg.bspline3(np.array([-2.0, 2.0, 2.5, -7.0])) == 0.0)


def test_bspline_slip_is_unit_at_the_centre_and_vanishes_at_the_edge():
    m, iface = mg.two_layer_block(shape=(12, 6, 6))
    on, hw = mg.interface_nodes(m, iface)
    pc = iface.plane_coords(m.coords)
    c = (float(np.median(pc[on, 0])), float(np.median(pc[on, 1])))
    uni = mg.slip_patch(m, iface, on, hw, c, 3000.0, "dip")
    bsp = mg.slip_patch(m, iface, on, hw, c, 3000.0, "dip", profile="bspline")
    amp_u = np.linalg.norm(uni.slip, axis=1)
    amp_b = np.linalg.norm(bsp.slip, axis=1)
    assert np.all(amp_b <= amp_u + 1e-15)             # inside the same patch, at most 1
    assert np.all(amp_b[amp_u == 0.0] == 0.0)
    assert amp_b.max() > 0.5
    # direction unchanged, only the amplitude tapers
    nz = amp_b > 0
    assert np.allclose(bsp.slip[nz] / amp_b[nz, None], iface.dip_vector()[None, :])
    assert set(bsp.elems.tolist()) <= set(uni.elems.tolist())
