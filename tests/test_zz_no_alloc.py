"""moma_matvec_noalloc: the Z / Z^H product for callers that cannot let the
library allocate device memory at call time (another framework's caching
allocator may hold the free memory, or a latency-bound loop cannot take an
allocation's implicit synchronisation).  Its scratch is a fixed device array
compiled into the library.

Checked here: its output against the ordinary moma_matvec and against the
oracle's direct offset-sum product (Eq. 1, Sec. II-A), on two calls in a row
(the shared scratch keeps the previous call's contents, which must not leak
into the next result), for a MIXED array (c64 and double-FP32 c128 products),
an FP64 array (FP64 product), a request just under the 32 MiB scratch cap,
and 16 RHS, where moma_matvec switches to the tensor cores.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from oracle import mbt
from synth import LatticeSpec, offset_blocks

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}  # the matvec parity tolerances of the suite
CAP = 32 << 20


def scratch_need(nr, spec, mx, my, esz):
    """Bytes of scratch a call needs (the formula include/moma.h states)."""
    a = lambda n: (n + 255) // 256 * 256  # noqa: E731
    return a(nr * spec.ny * mx * spec.b * esz) + 2 * a(mx * my * nr * spec.b * esz)


def smooth(n):
    m = n
    while True:
        k = m
        for r in (2, 3, 5):
            while k % r == 0:
                k //= r
        if k == 1:
            return m
        m += 1


@pytest.fixture(scope="module", params=["mixed", "fp64"])
def handle(request, moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(7, 5, 12, 0.5, 2)
    prec = m.MOMA_PREC_MIXED if request.param == "mixed" else m.MOMA_PREC_FP64
    blocks = offset_blocks(spec, np.complex64 if request.param == "mixed" else np.complex128)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    m.moma_set_blocks(h, blocks)
    yield m, spec, h, request.param, blocks.astype(np.complex128)
    m.moma_destroy(h)


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("op", [0, 1])
def test_noalloc_matches_matvec_and_oracle_twice(handle, cuda, dtype, op):
    m, spec, h, prec, b128 = handle
    if prec == "fp64" and dtype == "c64":
        pytest.skip("c64 products need a MIXED array")
    torch = cuda
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    g = torch.Generator(device="cpu").manual_seed(11 + op)
    for call in range(2):
        x = torch.randn((3, spec.ny, spec.nx, spec.b), dtype=tdt, generator=g).cuda()
        y_ref = torch.zeros_like(x)
        m.moma_matvec(h, op, x, y_ref)
        y = torch.full_like(x, float("nan"))
        m.moma_matvec_noalloc(h, op, x, y)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        xo = x.cpu().numpy().astype(np.complex128)
        want = mbt.matvec(b128, spec.nx, spec.ny, xo) if op == 0 else mbt.matvec_h(b128, spec.nx, spec.ny, xo)
        assert np.all(np.isfinite(a)), call
        assert _max_rel(a, b) <= TOL[dtype], (call, _max_rel(a, b))
        assert _max_rel(a, want) <= TOL[dtype], (call, _max_rel(a, want))


def test_noalloc_just_under_the_cap(handle, cuda):
    m, spec, h, prec, b128 = handle
    torch = cuda
    mx, my = smooth(2 * spec.nx - 1), smooth(2 * spec.ny - 1)
    nmax = max(n for n in range(1, 4096) if scratch_need(n, spec, mx, my, 16) <= CAP)
    assert scratch_need(nmax, spec, mx, my, 16) > CAP - scratch_need(1, spec, mx, my, 16)
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn((nmax, spec.ny, spec.nx, spec.b), dtype=torch.complex128, generator=g).cuda()
    y = torch.full_like(x, float("nan"))
    m.moma_matvec_noalloc(h, 0, x, y)
    torch.cuda.synchronize()
    want = mbt.matvec(b128, spec.nx, spec.ny, x.cpu().numpy())
    assert _max_rel(y.cpu().numpy(), want) <= TOL["c128"]
    big = torch.zeros((nmax + 1, spec.ny, spec.nx, spec.b), dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 0, big, torch.zeros_like(big))
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_rejects_host_buffers_and_bad_ops(handle, cuda):
    m, spec, h, prec, _ = handle
    torch = cuda
    xh = np.zeros((1, spec.ny, spec.nx, spec.b), np.complex128)
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 0, xh, xh.copy())
    assert e.value.status == 1
    x = torch.zeros((1, spec.ny, spec.nx, spec.b), dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 2, x, torch.zeros_like(x))
    assert e.value.status == 1


def test_noalloc_16_rhs_against_tensor_core_matvec(moma_lib, cuda):
    """From 16 RHS moma_matvec's c64 product runs on the tensor cores
    (3xTF32, ~2e-6); the allocation-free product stays on the CUDA cores."""
    m, torch = moma_lib, cuda
    spec = LatticeSpec(4, 4, 128, 0.5, 0)
    blocks = offset_blocks(spec, np.complex64)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, m.MOMA_PREC_MIXED)
    try:
        m.moma_set_blocks(h, blocks)
        g = torch.Generator(device="cpu").manual_seed(3)
        for call in range(2):
            x = torch.randn((16, spec.ny, spec.nx, spec.b), dtype=torch.complex64, generator=g).cuda()
            y_ref = torch.zeros_like(x)
            m.moma_matvec(h, 0, x, y_ref)
            y = torch.full_like(x, float("nan"))
            m.moma_matvec_noalloc(h, 0, x, y)
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            want = mbt.matvec(blocks.astype(np.complex128), spec.nx, spec.ny, x.cpu().numpy().astype(np.complex128))
            assert _max_rel(a, b) <= 1e-5, (call, _max_rel(a, b))
            assert _max_rel(a, want) <= 1e-5, (call, _max_rel(a, want))
    finally:
        m.moma_destroy(h)
