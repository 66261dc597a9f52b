"""The seeded synthetic inputs follow the stated recipe (shapes, rotation and
shift ranges, masks, rotation sets), and the generator's geometry is the one
the method inverts: B's mask is M_A moved by (q_true, t)."""
import numpy as np
import pytest

from paper_2110_10156_gb300 import synth


def _angle_deg(q):
    return float(np.rad2deg(2.0 * np.arccos(min(1.0, abs(float(q[0]))))))


def _rotmat(q):
    """Hamilton matrix of a unit quaternion (w, x, y, z), acting on (x, y, z)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_uniform_quaternions():
    """Shoemake's method: unit, w >= 0, and each squared component has mean 1/4
    (the uniform measure on rotations is symmetric in the four components)."""
    q = synth.random_quaternions(np.random.default_rng(3), 40000)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)
    assert np.all(q[:, 0] >= 0)
    m = (q ** 2).mean(axis=0)
    assert np.all(np.abs(m - 0.25) < 0.01), m


def test_small_workload_recipe():
    p = synth.config_pair(0)
    assert p.A.shape == p.B.shape == (32, 32, 32)
    assert p.A.dtype == p.B.dtype == np.float32
    assert len(p.quats) == 8 and p.true_index == 0
    np.testing.assert_array_equal(p.quats[0], p.q_true)
    np.testing.assert_array_equal(p.quats[1], [1.0, 0.0, 0.0, 0.0])      # identity included
    assert p.MA.all() and p.MB.all()                                       # full masks
    assert max(abs(v) for v in p.t_zyx) <= 6
    assert _angle_deg(p.q_true) <= 45.0 + 1e-9
    # a second call gives the same arrays (seeded)
    p2 = synth.config_pair(0)
    np.testing.assert_array_equal(p.A, p2.A)
    np.testing.assert_array_equal(p.B, p2.B)


def _moved_mask_agreement(p, R, t_xyz):
    """Fraction of voxels y with M_B(y) = M_A(round(R^T (y - c) + c - t))
    among those whose source lies inside, and whether M_B is 0 wherever the
    source lies well outside."""
    nz, ny, nx = p.A.shape
    c = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2])
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3).astype(np.float64)
    src = (pts - c) @ R + c - t_xyz                  # rows: R^T (y - c) + c - t
    hi = np.array([nx, ny, nz]) - 1
    idx = np.rint(src).astype(int)
    inside = np.all((src >= 0) & (src <= hi), axis=1)     # the edge's half-voxel band is left out
    far = np.any((src < -1) | (src > hi + 1), axis=1)
    mb = p.MB.reshape(-1)
    ma = p.MA[idx[inside, 2], idx[inside, 1], idx[inside, 0]]
    return float((ma == mb[inside]).mean()), not mb[far].any()


def test_moved_mask_is_the_generator_geometry():
    """M_B(y) = M_A(R^T (y - c) + c - t) by nearest neighbour, with R the
    Hamilton matrix of q_true and t the reported shift: the convention under
    which the method recovers chi = t at q_true.  A transposed R or a flipped
    shift agrees far less, so the check tells the conventions apart."""
    p = synth.small_pair(5, (24, 22, 20), n_rot=2, masks="threshold", max_shift=3)
    R = _rotmat(p.q_true)
    t = np.array(p.t_zyx[::-1], dtype=np.float64)
    agree, empty_outside = _moved_mask_agreement(p, R, t)
    assert agree > 0.995 and empty_outside
    assert _moved_mask_agreement(p, R.T, t)[0] < 0.95
    assert _moved_mask_agreement(p, R, -t)[0] < 0.95


@pytest.mark.parametrize("config,dims,n_rot,shift,angle", [(1, (150, 150, 150), 1000, 20, 30.0)])
def test_paper_scale_workload_recipe(config, dims, n_rot, shift, angle):
    p = synth.config_pair(config)
    assert p.A.shape == dims and len(p.quats) == n_rot
    assert 0 <= p.true_index < n_rot
    np.testing.assert_array_equal(p.quats[p.true_index], p.q_true)
    assert np.allclose(np.linalg.norm(p.quats, axis=1), 1.0, atol=1e-12)
    assert max(abs(v) for v in p.t_zyx) <= shift
    assert _angle_deg(p.q_true) <= angle + 1e-9
    # thresholded foreground at 0.05 max(A); B's mask covers a similar volume
    np.testing.assert_array_equal(p.MA, (p.A > 0.05 * p.A.max()).astype(np.uint8))
    fa, fb = p.MA.mean(), p.MB.mean()
    assert 0.05 < fa < 0.5 and abs(fb - fa) < 0.02 * fa + 0.005
    # the remap makes B multimodal: not a monotone function of the moved A
    assert p.B.std() > 0
