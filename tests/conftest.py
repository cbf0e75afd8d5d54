"""Shared fixtures. GPU tests are marked ``gpu``; everything else runs on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture(scope="session")
def small_problem(oracle):
    """A ragged small problem: 32^3 grid, 32x32 detector (812 used pixels),
    n=3 (1380 rotations), 300 frames at 0.5 photons/pixel."""
    from paper_1409_4256_gb300 import synth
    ds = synth.make_dataset(32, 32, 300, 0.5, radius=8.0)
    quat, w = oracle.quat_generate(3)
    grid = ds.model_start.astype(np.float32).astype(np.float64)  # what the GPU receives
    return dict(ds=ds, quat=quat, w=w, grid=grid, q=ds.q, K=ds.K, N=32,
                w_floor=1e-10 * float(grid.mean()))
