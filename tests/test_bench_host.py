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
@pytest.mark.parametrize("padded", [False, True])
def test_bin_product_bytes_counts_each_pair_once(nx, ny, b, nr, padded):
    spec = LatticeSpec(nx, ny, b, 0.5, 0)
    alg, pairs, nbins = bench.bin_product_bytes(spec, nr, padded=padded)
    mx, my = (_smooth(2 * nx - 1), _smooth(2 * ny - 1)) if padded else (2 * nx - 1, 2 * ny - 1)
    # {k, -k} classes of the 2D circulant frequencies, counted as sets.
    classes = {frozenset({(kx, ky), ((-kx) % mx, (-ky) % my)}) for kx in range(mx) for ky in range(my)}
    assert nbins == mx * my and pairs == len(classes)
    ldb = b + b % 2 if padded else b
    assert alg == pairs * b * ldb * 8 + 2 * nbins * nr * b * 8


def test_c2_bin_product_bytes_value():
    spec = LatticeSpec(32, 32, 128, 0.5, 0)
    # Algorithmic: the 63 x 63 circulant of Sec. II-A, (3969 + 1) / 2 pairs.
    assert bench.bin_product_bytes(spec, 2) == (276434944, 1985, 3969)
    # Streamed: 64 x 64 bins, 4 of them self-paired: (4096 - 4) / 2 + 4 pairs.
    assert bench.bin_product_bytes(spec, 2, padded=True) == (285474816, 2050, 4096)
    # One Z application adds the lattice vector in and out (2 x N x 2 RHS x 8 bytes).
    assert bench.matvec_bytes(spec, 2) == 276434944 + 2 * 131072 * 2 * 8


def test_measured_traffic_follows_the_capture_and_its_source_hash(tmp_path, monkeypatch):
    """The traffic record scales to a launch by streamed bytes while the
    kernel source it names is unchanged, and is withdrawn (None) after."""
    import hashlib
    spec = LatticeSpec(32, 32, 128, 0.5, 0)
    alg = bench.bin_product_bytes(spec, 2, padded=True)[0]
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_2608_17844_b300" / "csrc" / "kernel.cu"
    src.parent.mkdir(parents=True)
    src.write_text("// the captured kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    # a 24 x 24 capture that read each stored bin once plus 0.2 % extra
    cap_alg = 1154 * 128 * 128 * 8 + 2 * 2304 * 2 * 128 * 8
    (tmp_path / "profiles" / "bin_pair_kernel_c64_traffic.txt").write_text(
        f"kernel_source=paper_2608_17844_b300/csrc/kernel.cu\nkernel_source_sha256={sha}\npairs=1154\nbins=2304\n"
        f"nrhs=2\nb=128\ndram_read_bytes={int(cap_alg * 1.002)}\ndram_write_bytes=0\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t = bench.measured_traffic(alg, spec, 2)
    assert t == pytest.approx(1.002 * alg, rel=1e-6)
    src.write_text("// changed\n")
    assert bench.measured_traffic(alg, spec, 2) is None


def test_reference_arm_prints_its_line_on_the_cpu():
    """The reference arm times whole oracle solves only: the steps it
    reports ran, each solved every RHS to the 1e-10 residual."""
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "3", "--lattice", "3", "3", "8"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT,
                         env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["steps_requested"] == 2
    assert line["value"] == pytest.approx(2 * 1000.0 / line["ms_per_step"])  # 2 RHS per step
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "whole step" in line["cpu_baseline"]["sample"]
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["rhs_per_step"] == 2


def test_reference_arm_stops_at_its_budget_after_whole_steps():
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "50", "--warmup", "0", "--lattice", "3", "3", "8", "--ref-seconds", "0.01"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT,
                         env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["steps"] == 1 and line["steps_requested"] == 50


def test_serving_request_draw_follows_the_stated_distribution():
    reqs = bench.serve_requests(200.0, 2.0, 0)
    assert 300 <= len(reqs) <= 500  # Poisson(400)
    ts = [r[0] for r in reqs]
    assert ts == sorted(ts) and ts[-1] < 2.0
    nxs = [r[2].nx for r in reqs] + [r[2].ny for r in reqs]
    assert min(nxs) >= 4 and max(nxs) <= 40 and len(set(nxs)) > 25
    ds = [r[2].d for r in reqs]
    assert min(ds) >= 0.3 and max(ds) < 0.7 and len(set(ds)) == len(reqs)  # continuous: every request its own
    assert all(r[2].b == 128 and 1 <= len(r[3]) <= 32 for r in reqs)
    assert all(0 <= th <= 60 and 0 <= ph < 90 for r in reqs for th, ph in r[3])
    assert len({r[1] for r in reqs}) == len(reqs)
    keyed = bench.serve_requests(200.0, 2.0, 8)
    assert len({r[1] for r in keyed}) <= 8 and {r[2].d for r in keyed} <= {0.3, 0.4, 0.5, 0.6, 0.7}
    assert bench.serve_requests(200.0, 2.0, 0) == reqs  # seeded


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm and prints."""
    env = {**os.environ, "CUDA_VISIBLE_DEVICES": "", "RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0", "--lattice", "3", "3", "8"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
