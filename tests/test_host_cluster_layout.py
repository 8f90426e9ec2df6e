"""Host-compiled check of the work split and hand-over layout of the c64
cluster lattice transforms (csrc/lattice_cluster.cuh; the 2D transforms of
Eq. 2 on the circulant grid of Eq. 3): for every instantiated grid and lane
split, every lattice height and each of F2, I2 and I2MF2, the stores of the
eight CTAs of a cluster stay in bounds, never hit a location twice, and
cover every location the second axis reads.  The GPU parity tests compare
the transforms' results bitwise with the per-axis passes."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_17844_b300", "csrc")
EXE = os.path.join(ROOT, "paper_2608_17844_b300", "_build", "cluster_layout_check")


@pytest.fixture(scope="module")
def exe():
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-I", CSRC, "-I",
                    os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "native", "cluster_layout_check.cu"),
                    "-o", EXE, "-gencode", "arch=compute_103a,code=sm_103a"], check=True, capture_output=True)
    return EXE


def test_cluster_hand_over_layout(exe):
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    # 2 lane splits x (16 + 24 + 32 lattice heights) x 3 transforms
    assert int(r.stdout.split()[1]) == 2 * 3 * (16 + 24 + 32)
