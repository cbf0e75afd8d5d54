"""Host logic of the c-step's pixel groups (csrc/pixel_groups.h), on CPU.

A small driver is compiled with g++ against the header (no CUDA) and run on
the detectors of the workloads and on scattered pixels. Checked: the groups
partition the pixels (every index exactly once), no group exceeds the size
limit (one pixel per lane of a warp) or the extent limit along q_x and q_y,
pixels keep their index order within a group, and the split wastes few lanes:
the groups number at most a few more than the fewest that could hold the
pixels. For the detector sheets, the rotated groups' corner boxes are measured
against the shared-memory capacity the kernel uses (576 slots).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1409_4256_gb300", "csrc")
EXTENT, GROUP, CAP = 8.0, 32, 576

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "pixel_groups.h"
int main(int argc, char** argv) {
  long n = atol(argv[1]);
  double extent = atof(argv[2]);
  int gmax = atoi(argv[3]);
  std::vector<double> q(3 * n);
  for (long i = 0; i < 3 * n; i++)
    if (scanf("%lf", &q[i]) != 1) return 2;
  std::vector<int32_t> order, start;
  emc::build_pixel_groups(q.data(), n, extent, gmax, order, start);
  printf("%zu\n", start.size());
  for (size_t g = 0; g < start.size(); g++) printf("%d\n", start[g]);
  for (long p = 0; p < n; p++) printf("%d\n", order[p]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("groups")
    src = d / "groups.cpp"
    src.write_text(DRIVER)
    exe = d / "groups"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", HEADER_DIR, str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def run_groups(exe, q, extent=EXTENT, gmax=GROUP):
    inp = "\n".join(" ".join(repr(float(x)) for x in row) for row in q)
    out = subprocess.run([exe, str(q.shape[0]), repr(extent), str(gmax)], input=inp,
                         capture_output=True, text=True, check=True).stdout.split()
    ns = int(out[0])
    start = np.array(out[1:1 + ns], dtype=np.int64)
    order = np.array(out[1 + ns:], dtype=np.int64)
    return start, order


def check_invariants(q, start, order, extent=EXTENT, gmax=GROUP):
    n = q.shape[0]
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) > 0)
    assert np.array_equal(np.sort(order), np.arange(n))
    sizes = np.diff(start)
    assert sizes.max() <= gmax
    for g in range(len(sizes)):
        idx = order[start[g]:start[g + 1]]
        assert np.all(np.diff(idx) > 0)                  # index order kept
        if len(idx) > 1:                                 # within the extent limit
            span = q[idx, :2].max(0) - q[idx, :2].min(0)
            assert span.max() <= extent
    return sizes


@pytest.mark.parametrize("workload", ["emc32", "emc64", "emc128", "emc160"])
def test_detector_groups(driver, workload):
    from paper_1409_4256_gb300 import synth
    cfg = synth.WORKLOADS[workload]
    det = synth.make_detector(cfg["D"], cfg["N"], cfg["masked_fraction"])
    q = det.q
    start, order = run_groups(driver, q)
    sizes = check_invariants(q, start, order)
    # few idle lanes: nearly every group is full
    assert len(sizes) <= 1.15 * np.ceil(len(q) / GROUP), (len(sizes), len(q))
    # rotated corner boxes of the groups fit the kernel's capacity
    rng = np.random.default_rng(5)
    A = rng.standard_normal((20, 4))
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    over = 0
    total = 0
    for w, x, y, z in A:
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        f = np.floor(q @ R.T + cfg["N"] / 2).astype(np.int64)
        for g in range(len(start) - 1):
            fs = f[order[start[g]:start[g + 1]]]
            vol = np.prod(fs.max(0) - fs.min(0) + 2)
            over += vol > CAP
            total += 1
    assert over <= 0.005 * total


def test_scattered_pixels(driver):
    rng = np.random.default_rng(6)
    q = rng.uniform(-20, 20, (3000, 3))
    start, order = run_groups(driver, q)
    check_invariants(q, start, order)


def test_dense_cluster_is_cut_into_full_groups(driver):
    # 200 pixels within 6 voxels: no extent cut, so the split leaves groups of
    # 32 (a multiple of 32 on the first side of every cut) and one of 8
    rng = np.random.default_rng(7)
    q = rng.uniform(0.0, 5.9, (200, 3))
    start, order = run_groups(driver, q)
    check_invariants(q, start, order)
    assert sorted(np.diff(start)) == [8] + [32] * 6


def test_wide_pairs_are_split_by_extent(driver):
    # two pixels 20 voxels apart make two groups; a single pixel is one group
    q = np.array([[0.0, 0.0, 0.0], [20.0, 0.0, 0.0]])
    start, order = run_groups(driver, q)
    assert list(start) == [0, 1, 2]
    start, order = run_groups(driver, q[:1])
    assert list(start) == [0, 1] and list(order) == [0]
