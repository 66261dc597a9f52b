"""Pins for the search driver's reference: SplitMix64 against its published
reference outputs, Euler angles against scipy, the pyramid levels against
scipy's Gaussian filter definition."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import search_oracle as S


def test_splitmix64_matches_published_sequence():
    # first outputs for seed 1234567 from the reference C implementation
    # (Vigna, splitmix64.c)
    rng = S.SplitMix64(1234567)
    got = [rng.next() for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_in_unit_interval():
    rng = S.SplitMix64(7)
    u = np.array([rng.uniform() for _ in range(2000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.03


def test_euler_intrinsic_xyz_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(10):
        e = rng.uniform(-180, 180, 3)
        q = S.euler_to_quat(e)
        R = Rotation.from_euler("XYZ", e, degrees=True).as_matrix()    # intrinsic x, y', z''
        from oracle import cs_ngf_oracle as O
        np.testing.assert_allclose(O.quat_to_rotmat(q), R, atol=1e-12)


def test_level_volume_definition():
    rng = np.random.default_rng(2)
    V = rng.random((9, 10, 11))
    M = (rng.random((9, 10, 11)) > 0.5).astype(np.uint8)
    L, LM = S.level_volume(V, M, 1.5, 2)
    from scipy import ndimage
    ref = ndimage.gaussian_filter(V, 1.5, mode="nearest", truncate=4.0)[::2, ::2, ::2]
    np.testing.assert_allclose(L, ref, rtol=1e-12, atol=1e-14)
    assert L.shape == (5, 5, 6) and np.array_equal(LM, M[::2, ::2, ::2])
