"""moma_matvec_noalloc: the Z / Z^H product for callers that cannot let the
library allocate device memory at call time (its scratch is a fixed device
array compiled into the library).  Its output must match the ordinary
moma_matvec, on two calls in a row (the shared scratch keeps the previous
call's contents, which must not leak into the next result).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}  # the matvec parity tolerances of the suite


@pytest.fixture(scope="module")
def handle(moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(7, 5, 12, 0.5, 2)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, m.MOMA_PREC_MIXED)
    m.moma_set_blocks(h, offset_blocks(spec, np.complex64))
    yield m, spec, h
    m.moma_destroy(h)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("op", [0, 1])
def test_noalloc_matches_matvec_twice(handle, cuda, dtype, op):
    m, spec, h = handle
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
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert np.all(np.isfinite(a)) and err <= TOL[dtype], (call, err)


def test_noalloc_rejects_host_buffers_and_oversized_requests(handle, cuda):
    m, spec, h = handle
    torch = cuda
    xh = np.zeros((1, spec.ny, spec.nx, spec.b), np.complex64)
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 0, xh, xh.copy())
    assert e.value.status == 1
    big = torch.zeros((4096, spec.ny, spec.nx, spec.b), dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 0, big, torch.zeros_like(big))
    assert e.value.status == 1 and "scratch" in str(e.value)
    with pytest.raises(m.MomaError) as e:
        m.moma_matvec_noalloc(h, 2, big[:1], torch.zeros_like(big[:1]))
    assert e.value.status == 1
