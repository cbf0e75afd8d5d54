"""The C-ABI library loads, exports every entry point include/emc.h declares,
and its host-only parts behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libemc():
    from paper_1409_4256_gb300 import build, emc
    build.build()
    return emc.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[\w\s\*]+?\b(emc_\w+)\s*\(", src, flags=re.M))
    return names


def test_exports_every_declared_symbol(libemc):
    names = _declared()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(libemc, n), n


def test_binding_covers_header():
    from paper_1409_4256_gb300 import emc
    assert _declared() == set(emc._SIGS)


def test_quat_count_and_generate_match_oracle(libemc, oracle):
    from paper_1409_4256_gb300 import emc
    for n in (1, 2, 3, 4, 5):
        assert emc.quat_count(n) == 10 * (5 * n ** 3 + n)
        qa, wa = emc.quat_generate(n)
        qb, wb = oracle.quat_generate(n)
        assert qa.shape == qb.shape
        assert np.abs(qa - qb).max() < 1e-12
        assert np.abs(wa / wb - 1).max() < 1e-12
    qa, wa = emc.quat_generate(3, uniform=True)
    assert np.allclose(wa, 1 / len(wa))


def test_library_counts_printed_in_paper(libemc):
    # the library's own sampling gives every count printed with Eq. 2.7
    # (tests/golden/eq2_7_rotation_counts.txt)
    from paper_1409_4256_gb300 import emc
    from test_oracle_rotations import printed_counts
    for d, m in printed_counts():
        assert emc.quat_count(d) == m
        assert emc.quat_generate(d)[0].shape[0] == m


def test_status_strings_and_config_checks(libemc):
    from paper_1409_4256_gb300 import emc
    assert emc.status_string(0) == "ok"
    assert "argument" in emc.status_string(-1)
    cfg = emc.Config(N=32, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10,
                     compress_mode=0, flags=0, rot_chunk=0)
    nb = ctypes.c_size_t()
    assert libemc.emc_workspace_size(ctypes.byref(cfg), ctypes.byref(nb)) == 0 and nb.value > 0
    bad = emc.Config(N=2, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10)
    assert libemc.emc_workspace_size(ctypes.byref(bad), ctypes.byref(nb)) == -1
    neg = emc.Config(N=32, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=-1.0)
    assert libemc.emc_workspace_size(ctypes.byref(neg), ctypes.byref(nb)) == -1
    tiny = emc.Config(N=32, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=1e-30)
    assert libemc.emc_workspace_size(ctypes.byref(tiny), ctypes.byref(nb)) == -4
    b = emc.BufferSizes()
    assert libemc.emc_buffer_sizes_for(ctypes.byref(cfg), 50, ctypes.byref(b)) == 0
    assert b.ld_pix == 128 and b.ld_data == 256 and b.rows == 128
    assert b.logw_bytes == 3 * 2 * 128 * 128
    assert libemc.emc_buffer_sizes_for(ctypes.byref(cfg), 51, ctypes.byref(b)) == -1


def test_gaussian_config_checks(libemc):
    # the Gaussian model needs the FP16 split, stored scores, sigma > 0 and no
    # candidate sets; the checks run before anything touches a device
    from paper_1409_4256_gb300 import emc
    nb = ctypes.c_size_t()

    def ws(**kw):
        base = dict(N=32, precision=3, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10,
                    compress_mode=0, flags=1, rot_chunk=0, n_cand=0, model=1, sigma=1.0)
        base.update(kw)
        return libemc.emc_workspace_size(ctypes.byref(emc.Config(**base)), ctypes.byref(nb))

    assert ws() == 0
    assert ws(precision=2) == -4 and ws(flags=0) == -4 and ws(n_cand=8) == -4
    assert ws(sigma=0.0) == -1 and ws(sigma=float("nan")) == -1 and ws(model=3) == -1
    assert ws(model=0, sigma=0.0) == 0  # sigma is not read for the Poisson model


def test_poisson_fluence_config_checks(libemc):
    # the Poisson-fluence model takes the BF16 split only (one rounded value of
    # log(W / B_j) per element would bias every rotation's score by a multiple
    # of N_k); its P buffer carries den[rows] after the planes
    from paper_1409_4256_gb300 import emc
    nb = ctypes.c_size_t()

    def cfg(**kw):
        base = dict(N=32, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10,
                    compress_mode=0, flags=0, rot_chunk=0, n_cand=0, model=2, sigma=0.0)
        base.update(kw)
        return emc.Config(**base)

    def ws(**kw):
        return libemc.emc_workspace_size(ctypes.byref(cfg(**kw)), ctypes.byref(nb))

    assert ws() == 0 and ws(flags=1) == 0 and ws(n_cand=8) == 0
    assert ws(precision=0) == -4 and ws(precision=1) == -4 and ws(precision=3) == -4
    # a tiny floor is no error on the host: log(W / B_j) is range-checked on the device
    assert ws(w_floor=1e-30) == 0
    b, b0 = emc.BufferSizes(), emc.BufferSizes()
    assert libemc.emc_buffer_sizes_for(ctypes.byref(cfg()), 50, ctypes.byref(b)) == 0
    assert libemc.emc_buffer_sizes_for(ctypes.byref(cfg(model=0)), 50, ctypes.byref(b0)) == 0
    assert b.prob_bytes == b0.prob_bytes + 4 * 128  # float den[128] after the planes
    assert b.logw_bytes == b0.logw_bytes


def test_sparse_k_config_checks(libemc):
    from paper_1409_4256_gb300 import emc
    nb = ctypes.c_size_t()

    def ws(**kw):
        base = dict(N=32, precision=0, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10,
                    compress_mode=0, flags=2, rot_chunk=0, n_cand=0, model=0, sigma=1.0)
        base.update(kw)
        return libemc.emc_workspace_size(ctypes.byref(emc.Config(**base)), ctypes.byref(nb))

    assert ws() == 0
    small = nb.value
    assert ws(flags=0) == 0 and nb.value < small  # the non-zero lists take workspace
    assert ws(n_pix=70000) == -4  # pixel indices must fit 16 bits
    assert ws(flags=16) == -1
    assert ws(model=1, precision=3, flags=3) == -4  # Poisson only


def test_wide_counts_reserve_duplicate_columns(libemc):
    # EMC_FLAG_WIDE_COUNTS: 64 more columns in the pixel stride for duplicates
    from paper_1409_4256_gb300 import emc
    b = emc.BufferSizes()
    for flags, want in ((0, 128), (4, 192)):
        cfg = emc.Config(N=32, precision=2, n_pix=100, n_rot=50, n_data=10, w_floor=1e-10,
                         compress_mode=0, flags=flags, rot_chunk=0, n_cand=0, model=0, sigma=1.0)
        assert libemc.emc_buffer_sizes_for(ctypes.byref(cfg), 50, ctypes.byref(b)) == 0
        assert b.ld_pix == want


def test_pruned_estep_workspace(libemc):
    # a split precision + a Poisson model: emc_iteration prunes pass 1 (and a
    # recomputed pass 2) and keeps a second, reordered copy of the frames;
    # EMC_FLAG_DENSE_ESTEP (or any other configuration) does without
    from paper_1409_4256_gb300 import emc
    nb = ctypes.c_size_t()

    def ws(**kw):
        base = dict(N=32, precision=2, n_pix=100, n_rot=500, n_data=3000, w_floor=1e-10,
                    compress_mode=0, flags=1, rot_chunk=0, n_cand=0, model=0, sigma=1.0)
        base.update(kw)
        assert libemc.emc_workspace_size(ctypes.byref(emc.Config(**base)), ctypes.byref(nb)) == 0
        return nb.value

    pruned, dense = ws(), ws(flags=1 | 8)
    frames = 2 * 3072 * 128  # BF16 [ld_data][ld_pix]
    assert pruned - dense >= frames
    assert ws(flags=0) > ws(flags=8)                         # recomputed scores prune too
    assert ws(precision=1) == ws(precision=1, flags=9)       # plain BF16 (no hi plane): none
    assert ws(precision=0) == ws(precision=0, flags=9)       # FP32: none
    assert ws(precision=3) > ws(precision=3, flags=9)        # the FP16 split prunes
    assert ws(n_cand=8) > ws(n_cand=8, flags=9)              # with candidate sets too
    assert ws(model=2) > ws(model=2, flags=9)                # and the fluence model
