"""The synthetic media reproduce the stiffness values the paper prints (Sec. 4.1 Model 1, Table 2)."""
import os

import numpy as np

import synthetic as sy

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _model1():
    return np.loadtxt(os.path.join(GOLD, "model1_vti_stiffness.txt")) * 1e9


def test_model1_is_vti_and_thomsen_roundtrip():
    C = _model1()
    # VTI symmetry relation c12 = c11 - 2 c66 holds in the printed matrix
    assert abs(C[0, 1] - (C[0, 0] - 2 * C[5, 5])) < 1e-6 * C[0, 0]
    rho = 2500.0
    vp0, vs0 = np.sqrt(C[2, 2] / rho), np.sqrt(C[3, 3] / rho)
    eps = (C[0, 0] - C[2, 2]) / (2 * C[2, 2])
    gam = (C[5, 5] - C[3, 3]) / (2 * C[3, 3])
    dlt = ((C[0, 2] + C[3, 3]) ** 2 - (C[2, 2] - C[3, 3]) ** 2) / (2 * C[2, 2] * (C[2, 2] - C[3, 3]))
    assert np.allclose(sy.thomsen_vti(vp0, vs0, rho, eps, dlt, gam), C, rtol=1e-12, atol=1e-3)
    # the paper's isotropic background is the vertical-velocity medium of the same VTI rock
    lam, mu = sy.iso_lame(vp0, vs0, rho)
    assert abs(lam + 2 * mu - 26.5e9) < 1.0 and abs(mu - 10.4e9) < 1.0


def test_table2_layers():
    rows = {}
    with open(os.path.join(GOLD, "table2_layers.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            rows[k] = [float(x) for x in v]
    for key, (c11, c33, c55, c66, c13) in rows.items():
        C = sy.media.vti_from_table(**sy.media.TABLE2[key]) / 1e9
        assert np.allclose([C[0, 0], C[2, 2], C[4, 4], C[5, 5], C[0, 2]], [c11, c33, c55, c66, c13])
        assert abs(C[0, 1] - (c11 - 2 * c66)) < 1e-12


def test_pack_roundtrip_and_bond_rotation_identity():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6))
    A = A + A.T
    assert np.array_equal(sy.unpack21(sy.pack21(A)), A)
    C = sy.thomsen_vti(3000, 1730, 2300, 0.15, 0.1, 0.12)
    assert np.allclose(sy.bond_rotate_y(C, 0.0), C)
    # rotating by 90 degrees about y swaps the x and z axes: c11 <-> c33
    R = sy.bond_rotate_y(C, np.pi / 2)
    assert np.isclose(R[0, 0], C[2, 2]) and np.isclose(R[2, 2], C[0, 0])


def test_workloads_shapes():
    wl = sy.get_workload("inclusion16_fp64")
    med = wl.medium()
    assert med.dC.shape == (21, 16, 16, 16) and med.drho.shape == (16, 16, 16)
    # contrast vanishes on boundary planes, inclusion on nodes 5..10
    assert np.all(med.dC[:, 0] == 0) and np.all(med.dC[:, :, :, -1] == 0)
    assert np.all(med.drho[5:11, 5:11, 5:11] > 0) and med.drho[4, 8, 8] == 0
    M, xs = wl.sources()
    assert np.allclose(xs[0], [75.0, 75.0, 75.0])
