"""Host-compiled check of the library's column FFT engine and plans against
numpy's FFT (no GPU needed): forward DIF, forward DIT and the fused
inverse-mask-forward pass used between the Z and Z^H legs."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_17844_b300", "csrc")
EXE = os.path.join(ROOT, "paper_2608_17844_b300", "_build", "fft_host_check")


@pytest.fixture(scope="module")
def exe():
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    cmd = [nvcc, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "native", "fft_host_check.cu"), os.path.join(CSRC, "fft.cu"),
           os.path.join(CSRC, "fftreg.cu"), "--expt-relaxed-constexpr", "-o", EXE,
           "-gencode", "arch=compute_103a,code=sm_103a"]
    subprocess.run(cmd, check=True, capture_output=True)
    return EXE


def _run(exe, x, mode, keep=0):
    inp = f"{len(x)} {mode} {keep}\n" + "\n".join("%.17g %.17g" % (v.real, v.imag) for v in x) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    vals = np.array([complex(*map(float, l.split())) for l in out[1:] if l.strip()])
    return int(out[0]), vals


SIZES = [1, 2, 3, 4, 5, 6, 8, 9, 12, 15, 16, 24, 25, 27, 32, 45, 48, 60, 63 + 1, 80, 96, 125, 128]


@pytest.mark.parametrize("M", SIZES)
@pytest.mark.parametrize("mode", ["dif", "dit"])
def test_forward_matches_numpy(exe, M, mode):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    _, y = _run(exe, x, mode)
    ref = np.fft.fft(x)
    assert np.allclose(y, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("M", [4, 15, 48, 64, 80, 96, 128])
@pytest.mark.parametrize("mode", ["difcoop", "ditcoop"])
@pytest.mark.parametrize("ng", [2, 3, 4, 8])
def test_cooperative_stage_split(exe, M, mode, ng):
    """Stages split over ng cooperating threads give the same transform."""
    rng = np.random.default_rng(M + ng)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    _, y = _run(exe, x, mode, ng)
    ref = np.fft.fft(x)
    assert np.allclose(y, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("M,keep", [(8, 3), (48, 24), (64, 32), (96, 40), (5, 3), (1, 1)])
def test_inverse_mask_forward(exe, M, keep):
    rng = np.random.default_rng(7 + M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    _, y = _run(exe, x, "imf", keep)
    t = np.fft.ifft(x)
    t[keep:] = 0
    ref = np.fft.fft(t)
    assert np.allclose(y, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


def test_rejects_non_smooth_length(exe):
    r = subprocess.run([exe], input="7 dif 0\n" + "1 0\n" * 7, capture_output=True, text=True)
    assert r.returncode != 0
