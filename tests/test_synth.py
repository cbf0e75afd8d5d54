"""Sanity of the seeded input generator (inputs only, no method arithmetic)."""
import numpy as np

from paper_1409_4256_gb300 import synth


def test_detector_support_and_mask():
    det = synth.make_detector(64, 64, 0.10)
    assert np.all(np.linalg.norm(det.q, axis=1) <= 64 / 2 - 1 + 1e-12)
    mask = synth.detector_mask(64, 0.10)
    assert abs(mask.mean() - 0.10) < 0.01
    # q_max is reached at the middle of a detector edge
    qa = synth.detector_q(64, 64)
    assert np.isclose(np.linalg.norm(qa, axis=1).max() > 31, True)


def test_intensity_closed_form():
    atoms = synth.make_atoms(5, 4.0)
    # at zero frequency every atom adds in phase: I(0) = n_atoms^2
    assert np.isclose(synth.intensity(np.zeros((1, 3)), atoms, 32)[0], 25.0)
    # Friedel symmetry I(p) = I(-p)
    p = np.random.default_rng(0).uniform(-10, 10, size=(20, 3))
    assert np.allclose(synth.intensity(p, atoms, 32), synth.intensity(-p, atoms, 32))


def test_rotations_haar():
    R = synth.random_rotations(500)
    assert np.allclose(np.einsum("kab,kcb->kac", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0)
    assert np.abs(R.mean(0)).max() < 0.1  # E[R] = 0 under Haar measure


def test_dataset_mean_and_seed():
    a = synth.make_dataset(32, 32, 50, 0.5)
    b = synth.make_dataset(32, 32, 50, 0.5)
    assert np.array_equal(a.K, b.K)
    assert abs(a.K.mean() - 0.5) < 0.05
    assert a.K.dtype == np.int32 and a.K.min() >= 0
