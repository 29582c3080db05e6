"""The seeded input generators shared by oracle-side and CUDA-side tests."""
import math

import numpy as np

from paper_2107_03747_gb300 import inputs as I


def test_splitmix64_published_vector():
    """First outputs of SplitMix64 from state 0 (Steele, Lea, Flood 2014; Vigna's reference code)."""
    ref = [int(x, 16) for x in open(__file__.replace("test_inputs.py", "golden/splitmix64_seed0.txt")).read().split()
           if x.startswith("0x")]
    assert [int(x) for x in I.splitmix64(0, len(ref))] == ref


def test_gaussians_moments_and_determinism():
    g = I.gaussians(5, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    assert np.array_equal(g[:10], I.gaussians(5, 10))
    assert np.array_equal(I.gaussians(5, 10, offset=4), g[4:14])


def test_random_links_are_su3_and_match_amplitude():
    U = I.random_links((2, 2, 6, 6), 0, 0.3)
    assert U.shape == (6, 6, 2, 2, 4, 3, 3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # small amplitude: U ~ 1 + i amp omega T, so <|U - 1|_F^2> ~ amp^2 * 8 * 1/2
    d = np.mean(np.sum(np.abs(U - np.eye(3)) ** 2, axis=(-1, -2)))
    assert abs(d / (0.3 ** 2 * 4) - 1) < 0.1


def test_twist_eater_shape():
    U = I.twist_eater((4, 4, 12, 12))
    g1, g2 = I.twist_matrices()
    assert np.array_equal(U[3, 5, 2, 0, 0], g1) and np.array_equal(U[3, 5, 0, 2, 1], g2)
    assert np.array_equal(U[3, 5, 2, 1, 0], np.eye(3))


def test_batched_member_amplitude_range():
    amps = [I.batched_amplitude(s) for s in range(256)]
    assert min(amps) >= 0.2 and max(amps) < 0.6
