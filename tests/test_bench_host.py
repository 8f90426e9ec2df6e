"""Host-side logic of bench.py, on the CPU: the algorithmic-byte count the
roofline divides by, the scaling of the committed ncu traffic record, and
the reference arm's JSON line (the oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

import bench
from synth import LatticeSpec


def _smooth(n):
    """Smallest 2^a 3^b 5^c >= n, by direct search over the exponents."""
    best = None
    for a in range(12):
        for b in range(8):
            for c in range(6):
                v = 2 ** a * 3 ** b * 5 ** c
                if v >= n and (best is None or v < best):
                    best = v
    return best


@pytest.mark.parametrize("nx,ny,b,nr", [(32, 32, 128, 2), (24, 24, 256, 64), (5, 3, 7, 1)])
def test_bin_product_bytes_counts_each_pair_once(nx, ny, b, nr):
    spec = LatticeSpec(nx, ny, b, 0.5, 0)
    alg, pairs, nbins = bench.bin_product_bytes(spec, nr)
    mx, my = _smooth(2 * nx - 1), _smooth(2 * ny - 1)
    # {k, -k} classes of the 2D circulant frequencies, counted as sets.
    classes = {frozenset({(kx, ky), ((-kx) % mx, (-ky) % my)}) for kx in range(mx) for ky in range(my)}
    assert nbins == mx * my and pairs == len(classes)
    ldb = b + b % 2
    assert alg == pairs * b * ldb * 8 + 2 * nbins * nr * b * 8


def test_c2_bin_product_bytes_value():
    spec = LatticeSpec(32, 32, 128, 0.5, 0)
    alg, pairs, nbins = bench.bin_product_bytes(spec, 2)
    # 64 x 64 bins, 4 of them self-paired: (4096 - 4) / 2 + 4 pairs.
    assert (nbins, pairs, alg) == (4096, 2050, 285474816)


def test_measured_traffic_follows_the_capture_and_its_source_hash(tmp_path, monkeypatch):
    spec = LatticeSpec(32, 32, 128, 0.5, 0)
    alg = bench.bin_product_bytes(spec, 2)[0]
    t = bench.measured_traffic(alg, spec, 2)
    assert t is not None and 0.99 * alg <= t <= 1.05 * alg  # the capture read each stored bin once
    # A copy of the tree whose kernel source differs from the captured one.
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2608_17844_b300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles" / "bin_pair_kernel_c64_traffic.txt").write_text(
        open(os.path.join(bench.ROOT, "profiles", "bin_pair_kernel_c64_traffic.txt")).read())
    (tmp_path / "paper_2608_17844_b300" / "csrc" / "binprod.cu").write_text("// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(alg, spec, 2) is None


def test_reference_arm_prints_its_line_on_the_cpu():
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--lattice", "3", "3", "8"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT,
                         env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm and prints."""
    env = {**os.environ, "CUDA_VISIBLE_DEVICES": "", "RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0", "--lattice", "3", "3", "8"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
