"""Argument rules of the allocation-free product, checked on the host
without a GPU: the rules live in csrc/noalloc_check.h, a CUDA-free header
that the library and this test's small C++ driver both compile.  Buffers on
a device other than the array's are rejected before any launch (the product
would otherwise read another GPU's copy of the scratch array)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_17844_b300", "csrc")
EXE = os.path.join(ROOT, "paper_2608_17844_b300", "_build", "noalloc_check")
CAP = 32 << 20


@pytest.fixture(scope="module")
def exe():
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "native", "noalloc_check.cpp"), "-o", EXE],
                   check=True, capture_output=True)
    return EXE


def run(exe, rows):
    inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.strip().split("\n")
    return [(int(l.split(" ", 1)[0]), l.split(" ", 1)[1]) for l in out]


def need(nr, ny, mx, B, b, esz):
    a = lambda n: (n + 255) // 256 * 256  # noqa: E731
    return a(nr * ny * mx * b * esz) + 2 * a(B * nr * b * esz)


def test_accepts_buffers_on_the_arrays_device(exe):
    (n, msg), = run(exe, [(1, 1, 1, 1, 1, 3, 5, 15, 135, 12, 16, CAP)])
    assert msg == "OK" and n == need(3, 5, 15, 135, 12, 16)


@pytest.mark.parametrize("xd,yd", [(1, 0), (0, 1), (2, 2)])
def test_rejects_buffers_on_another_device(exe, xd, yd):
    (_, msg), = run(exe, [(0, 1, xd, 1, yd, 3, 5, 15, 135, 12, 16, CAP)])
    assert "array's device 0" in msg, msg


def test_rejects_host_buffers(exe):
    rows = [(0, 0, -1, 1, 0, 1, 5, 15, 135, 12, 8, CAP), (0, 1, 0, 0, -1, 1, 5, 15, 135, 12, 8, CAP)]
    assert all(m == "x and y must be device memory" for _, m in run(exe, rows))


def test_cap_boundary(exe):
    # 7x5 lattice, b = 12: Mx = 15, My = 9, B = 135; c128 values.
    per = need(1, 5, 15, 135, 12, 16)
    nmax = max(n for n in range(1, 4096) if need(n, 5, 15, 135, 12, 16) <= CAP)
    res = run(exe, [(0, 1, 0, 1, 0, nmax, 5, 15, 135, 12, 16, CAP), (0, 1, 0, 1, 0, nmax + 1, 5, 15, 135, 12, 16, CAP)])
    assert res[0][1] == "OK" and CAP - per < res[0][0] <= CAP
    assert res[1][0] > CAP and "fixed maximum is %d" % CAP in res[1][1]
