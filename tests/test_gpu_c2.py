"""Full-size parity on the 32 x 32 lattice, b = 128 (N = 131072), blocks
stored complex64, broadside + 45 degree E-plane RHS -- the workload the
benchmark times, in the same launch configuration.

The dense oracle cannot hold this Z (275 GB), so the checks are:
  * the residual certificate: ||V - Z I|| / ||V|| recomputed on the CPU in
    complex128 with the oracle's direct offset sum (no FFT) <= 1e-10;
  * Z_a of the centre, edge and corner elements against oracle-I (GMRES on
    the original system, tol 1e-13) within 1e-8;
  * Z_a of every port within 1e-8 of oracle-I (the bar is per port), and
    the same two checks for the plain FP64 solve, the mixed path with FP64
    residual arithmetic and the PCG solver.
"""
import numpy as np
import pytest

from synth import config_c2, offset_blocks, excitation
from oracle import mbt, ports, iterative

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    spec, angles = config_c2()
    blocks64 = offset_blocks(spec, np.complex64)
    return spec, blocks64, excitation(spec, angles)


@pytest.fixture(scope="module")
def oracle_c2(c2):
    """oracle-I (GMRES on Z I = V, direct offset sums, tol 1e-13): currents
    and active impedances of every port, both RHS."""
    spec, blocks64, V = c2
    i_ref, _ = iterative.gmres(blocks64.astype(np.complex128), spec.nx, spec.ny, V, tol=1e-13, restart=60)
    return i_ref, ports.active_impedance(i_ref, V)


def _solve(m, spec, blocks64, V, prec, solver=0, flags=0):
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec, flags=flags)
    try:
        m.moma_set_blocks(h, blocks64)
        I = np.zeros_like(V)
        rr = np.zeros(V.shape[0])
        info = m.moma_solve(h, V, I, rel_residual=rr, solver=solver)
        za = np.zeros(V.shape[:3], np.complex128)
        gam = np.zeros_like(za)
        m.moma_active_impedance(h, I, V, za, gam)
        return I, za, gam, info, rr
    finally:
        m.moma_destroy(h)


def _certify(name, spec, blocks64, V, I, za, za_ref):
    """The GPU currents' residual recomputed by the oracle's FP64 direct
    offset sum, and Z_a of every port against oracle-I."""
    res = V - mbt.matvec(blocks64.astype(np.complex128), spec.nx, spec.ny, I)
    cert = np.linalg.norm(res.reshape(V.shape[0], -1), axis=1) / np.linalg.norm(V.reshape(V.shape[0], -1), axis=1)
    err = np.abs(za - za_ref) / np.abs(za_ref)
    print(f"C2 {name}: certified residual {cert}, max per-port Z_a rel err {err.max():.3g}")
    for pname, (ex, ey) in ports.named_elements(spec.nx, spec.ny).items():
        print(f"   {pname}: Za={za[:, ey, ex]} rel err {err[:, ey, ex]}")
    assert cert.max() <= 1e-10
    assert err.max() <= 1e-8


def test_c2_mixed_certified_and_ports_match_oracle(moma_lib, cuda, c2, oracle_c2):
    spec, blocks64, V = c2
    I, za, gam, info, rr = _solve(moma_lib, spec, blocks64, V, 1)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    _certify("mixed", spec, blocks64, V, I, za, oracle_c2[1])
    assert np.allclose(gam, ports.reflection(za), rtol=1e-12)


def test_c2_mixed_fp64_residual_certified(moma_lib, cuda, c2, oracle_c2):
    """The mixed path with its FP64-class stages (block-bin transform,
    refinement residual Z I, block Cholesky) in FP64 instead of double-FP32."""
    m = moma_lib
    spec, blocks64, V = c2
    I, za, gam, info, rr = _solve(m, spec, blocks64, V, 1, flags=m.MOMA_FLAG_FP64_RESIDUAL)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    _certify("mixed, FP64 residual", spec, blocks64, V, I, za, oracle_c2[1])


def test_c2_plain_fp64_certified(moma_lib, cuda, c2, oracle_c2):
    spec, blocks64, V = c2
    I, za, gam, info, rr = _solve(moma_lib, spec, blocks64, V, 0)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    _certify("plain FP64", spec, blocks64, V, I, za, oracle_c2[1])


def test_c2_pcg_certified(moma_lib, cuda, c2, oracle_c2):
    """The paper's PCG solver on the full-size problem."""
    spec, blocks64, V = c2
    I, za, gam, info, rr = _solve(moma_lib, spec, blocks64, V, 1, solver=1)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    _certify("pcg", spec, blocks64, V, I, za, oracle_c2[1])
