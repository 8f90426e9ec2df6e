"""GPU parity with an array margin (Eq. 1: Z = [Z_A, Z_B^T; Z_B, Z_C]):
Z and Z^H products, the preconditioner with its margin block (Eq. 38), and
full solves (GMRES and PCG, mixed and FP64) against the dense oracle; and
removing the margin restores the margin-free results exactly."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, margin_blocks, excitation
from oracle import dense, mbt, ports

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _case(nx=4, ny=3, b=8, seed=1, bm=2):
    spec = LatticeSpec(nx, ny, b, 0.5, seed)
    blocks = offset_blocks(spec)
    zb, zc = margin_blocks(spec, bm=bm)
    return spec, blocks, zb, zc


def _vec(spec, nm, nr, seed=3):
    rng = np.random.default_rng(seed)
    n = spec.n + nm
    return rng.standard_normal((nr, n)) + 1j * rng.standard_normal((nr, n))


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_margin_products_match_dense(moma_lib, cuda, prec):
    m = moma_lib
    spec, blocks, zb, zc = _case()
    nm = zc.shape[0]
    z = dense.assemble_with_margin(blocks, spec.nx, spec.ny, zb, zc)
    x = _vec(spec, nm, 3)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    try:
        m.moma_set_blocks(h, blocks)
        m.moma_set_margin(h, zb, zc)
        for op, ref in ((m.MOMA_OP_Z, x @ z.T), (m.MOMA_OP_ZH, x @ z.conj())):
            y = np.zeros_like(x)
            m.moma_matvec(h, op, x, y)
            e = relerr(y, ref)
            print(f"margin prec={prec} op={op}: c128 err {e:.3g}")
            assert e <= 1e-12
            if prec == MIXED:
                x32 = x.astype(np.complex64)
                y32 = np.zeros_like(x32)
                m.moma_matvec(h, op, x32, y32)
                ref32 = x32.astype(np.complex128) @ (z.T if op == m.MOMA_OP_Z else z.conj())
                assert relerr(y32, ref32) <= 1e-5
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_margin_preconditioner_matches_oracle(moma_lib, cuda, prec):
    m = moma_lib
    spec, blocks, zb, zc = _case(5, 2, 6)
    nm = zc.shape[0]
    p = mbt.precond_blocks(blocks, spec.nx, spec.ny)
    pc = mbt.precond_margin(zb, zc)
    x = _vec(spec, nm, 2)
    ref = mbt.precond_solve_margin(p, pc, x, spec.n)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    try:
        m.moma_set_blocks(h, blocks)
        m.moma_set_margin(h, zb, zc)
        xx = x if prec == FP64 else x.astype(np.complex64)
        y = np.zeros_like(xx)
        m.moma_apply_precond(h, xx, y)
    finally:
        m.moma_destroy(h)
    e = relerr(y.astype(np.complex128), ref)
    print(f"margin precond prec={prec}: err {e:.3g}")
    assert e <= (1e-11 if prec == FP64 else 1e-5)


@pytest.mark.parametrize("prec,solver", [(MIXED, 0), (FP64, 0), (MIXED, 1)])
def test_margin_solve_matches_dense_lu(moma_lib, cuda, prec, solver):
    m = moma_lib
    spec, blocks, zb, zc = _case(5, 4, 12, seed=2, bm=3)
    nm, n = zc.shape[0], spec.n
    z = dense.assemble_with_margin(blocks, spec.nx, spec.ny, zb, zc)
    va = excitation(spec, [(0.0, 0.0), (30.0, 45.0)]).reshape(2, n)
    V = np.concatenate([va, np.zeros((2, nm))], axis=1)  # ports on the elements only
    i_ref = dense.solve(z, V)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    try:
        m.moma_set_blocks(h, blocks if prec == FP64 else blocks)
        m.moma_set_margin(h, zb, zc)
        I = np.zeros_like(V)
        rr = np.zeros(2)
        info = m.moma_solve(h, V, I, rel_residual=rr, solver=solver)
        za = np.zeros((2, spec.ny, spec.nx), np.complex128)
        m.moma_active_impedance(h, I, V, za)
    finally:
        m.moma_destroy(h)
    print(f"margin solve prec={prec} solver={solver}:", info)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    assert dense.relative_residual(z, I, V).max() <= 1e-10
    za_ref = ports.active_impedance(i_ref[:, :n].reshape(2, spec.ny, spec.nx, spec.b),
                                    va.reshape(2, spec.ny, spec.nx, spec.b))
    assert relerr(za, za_ref) <= 1e-8


def test_removing_the_margin_restores_plain_results(moma_lib, cuda):
    m = moma_lib
    spec, blocks, zb, zc = _case()
    V = excitation(spec, [(0.0, 0.0)])
    out = []
    for with_margin in (False, True):
        h = m.moma_create_array(spec.nx, spec.ny, spec.b, MIXED)
        try:
            m.moma_set_blocks(h, blocks)
            if with_margin:
                m.moma_set_margin(h, zb, zc)
                m.moma_set_margin(h, None, None)
            I = np.zeros_like(V)
            m.moma_solve(h, V, I)
            out.append(I)
        finally:
            m.moma_destroy(h)
    assert np.array_equal(out[0], out[1])
