"""Host-compiled check of the register-resident FFT core used by the c64
lattice passes (csrc/fftreg.cuh), against numpy's FFT in float64, for every
length the passes take (all 2, 3, 5-smooth M <= 64): the forward transform,
the inverse, and the inverse / truncate / forward sequence of the mask pass
between the Z and Z^H legs (Sec. III-A).  FP32 arithmetic: the bar is a
few units of FP32 rounding times log2(M), relative to the largest value.
The split transform (P lanes per line, a whole warp of lines emulated on
the host with the device's exchange-buffer layout) is checked the same way
for every (M, P) the passes instantiate."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_17844_b300", "csrc")
EXE = os.path.join(ROOT, "paper_2608_17844_b300", "_build", "fftreg_host_check")
SIZES = [1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64]


@pytest.fixture(scope="module")
def exe():
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-I", CSRC, "-I",
                    os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "native", "fftreg_host_check.cu"),
                    "-o", EXE, "-gencode", "arch=compute_103a,code=sm_103a"], check=True, capture_output=True)
    return EXE


@pytest.mark.parametrize("M", SIZES)
def test_register_fft_matches_numpy(exe, M):
    rng = np.random.default_rng(M)
    x = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
    keep = max(1, (M + 1) // 2)
    inp = f"{M} {keep} 1\n" + "\n".join("%.9g %.9g" % (v.real, v.imag) for v in x) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    vals = np.array([complex(*map(float, l.split())) for l in out if l.strip()])
    fwd, inv, mask = vals[:M], vals[M:2 * M], vals[2 * M:3 * M]
    xd = x.astype(np.complex128)
    ref_f = np.fft.fft(xd)
    ref_i = np.fft.ifft(xd)
    t = ref_i.copy()
    t[keep:] = 0
    ref_m = np.fft.fft(t)
    tol = 4e-7 * max(1.0, np.log2(M))
    for got, ref in ((fwd, ref_f), (inv, ref_i), (mask, ref_m)):
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (M, np.abs(got - ref).max() / np.abs(ref).max())


# (M, P) pairs with P^2 | M that the lane kernels of fftreg.cu instantiate.
LANE_CASES = [(4, 2), (8, 2), (12, 2), (16, 2), (20, 2), (24, 2), (32, 2), (36, 2), (40, 2), (48, 2), (60, 2),
              (64, 2), (16, 4), (32, 4), (48, 4), (64, 4), (64, 8)]


@pytest.mark.parametrize("M,P", LANE_CASES)
def test_split_transform_matches_numpy(exe, M, P):
    rng = np.random.default_rng(1000 * M + P)
    x = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
    keep = max(1, (M + 1) // 2)
    inp = f"{M} {keep} {P}\n" + "\n".join("%.9g %.9g" % (v.real, v.imag) for v in x) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    vals = np.array([complex(*map(float, l.split())) for l in out if l.strip()])
    L = 32 // P
    assert vals.size == 3 * L * M
    tol = 4e-7 * max(1.0, np.log2(M))
    for l in range(L):
        xd = np.roll(x.astype(np.complex128), -l)  # line l holds x[(m + l) mod M]
        ref_f = np.fft.fft(xd)
        ref_i = np.fft.ifft(xd)
        t = ref_i.copy()
        t[keep:] = 0
        ref_m = np.fft.fft(t)
        base = 3 * M * l
        for o, ref in enumerate((ref_f, ref_i, ref_m)):
            got = vals[base + o * M: base + (o + 1) * M]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= tol, (M, P, l, o, err)
