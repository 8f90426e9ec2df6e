"""GPU parity of the error predictors (Sec. II-E, Eqs. 23-36) against the
predictor oracle: the column coupling C_n from a phase sweep solved on the
GPU vs dense solves + the oracle's quadrature; S -> Z (Eq. 31) and its
round trip through the GPU all-port Z_p; S_ideal and xi_S (Eq. 36); the
xi_Z family (Eqs. 23-25) from a GPU Z_p.  FP64 results: <= 1e-10 relative
(the solves themselves are certified to 1e-10)."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks
from oracle import dense, ports, predictors as pr

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.mark.parametrize("nx,ny,b,nq,nmax,prec", [(6, 3, 8, 16, 5, 1), (9, 1, 4, 24, 8, 0), (5, 4, 128, 20, 4, 1)])
def test_column_coupling_matches_dense_sweep(moma_lib, cuda, nx, ny, b, nq, nmax, prec):
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 4)
    blocks = offset_blocks(spec)
    z = dense.assemble(blocks, nx, ny)
    v = pr.row_phase_excitation(nx, ny, b, pr.psi_samples(nq))
    za = ports.active_impedance(dense.solve(z, v), v)
    g_ref = ports.reflection(za[:, ny // 2, nx // 2])
    c_ref = pr.column_coupling(g_ref, nmax)
    h = m.moma_create_array(nx, ny, b, prec)
    try:
        m.moma_set_blocks(h, blocks if prec == 0 else blocks.astype(np.complex64))
        C = np.zeros(2 * nmax + 1, np.complex128)
        g = np.zeros(nq, np.complex128)
        m.moma_column_coupling(h, nq, nmax, C, g)
    finally:
        m.moma_destroy(h)
    if prec == 1:  # the c64-stored blocks define the mixed problem
        z = dense.assemble(blocks.astype(np.complex64).astype(np.complex128), nx, ny)
        za = ports.active_impedance(dense.solve(z, v), v)
        g_ref = ports.reflection(za[:, ny // 2, nx // 2])
        c_ref = pr.column_coupling(g_ref, nmax)
    print(f"C_n {nx}x{ny}x{b}: Gamma err {relerr(g, g_ref):.3g}, C err {relerr(C, c_ref):.3g}, |C| {np.abs(C).round(5)}")
    assert relerr(g, g_ref) <= 1e-9
    assert np.abs(C - c_ref).max() <= 1e-9 * np.abs(c_ref).max()


def test_s_to_z_and_round_trip_through_gpu_zp(moma_lib, cuda):
    import torch
    m = moma_lib
    spec = LatticeSpec(5, 4, 6, 0.5, 2)
    blocks = offset_blocks(spec)
    h = m.moma_create_array(5, 4, 6, 0)
    try:
        m.moma_set_blocks(h, blocks)
        zp = np.zeros((20, 20), np.complex128)
        m.moma_port_impedance(h, zp)
    finally:
        m.moma_destroy(h)
    s = pr.s_from_z(zp, 50.0)
    z_gpu = np.zeros_like(s)
    m.moma_s_to_z(s, z_gpu, 50.0)
    assert relerr(z_gpu, pr.z_from_s(s, 50.0)) <= 1e-12
    assert relerr(z_gpu, zp) <= 1e-10
    # device buffers
    s_d = torch.from_numpy(s).cuda()
    z_d = torch.zeros_like(s_d)
    m.moma_s_to_z(s_d, z_d, 50.0)
    assert np.array_equal(z_d.cpu().numpy(), z_gpu)
    with pytest.raises(m.MomaError):
        m.moma_s_to_z(np.eye(4, dtype=np.complex128), np.zeros((4, 4), np.complex128))  # I - S singular


def test_s_ideal_and_xi_s(moma_lib, cuda):
    m = moma_lib
    kd = 2 * np.pi * 0.6
    S = np.zeros((30, 30), np.complex128)
    m.moma_s_ideal(6, 5, 0.12 + 0.04j, -0.15 + 0.07j, kd, S)
    ref = pr.s_ideal(6, 5, 0.12 + 0.04j, -0.15 + 0.07j, kd)
    assert relerr(S, ref) <= 1e-15
    xs = m.moma_xi_s(6, 5, 0.12 + 0.04j, -0.15 + 0.07j, kd, 50.0)
    xs_ref = pr.xi_s(6, 5, 0.12 + 0.04j, -0.15 + 0.07j, kd, 50.0)
    print("xi_S", xs, xs_ref)
    assert abs(xs - xs_ref) <= 1e-12 * xs_ref


def test_xi_z_family_from_gpu_zp(moma_lib, cuda):
    m = moma_lib
    for nx, ny in ((5, 5), (6, 4)):
        spec = LatticeSpec(nx, ny, 5, 0.5, 1)
        blocks = offset_blocks(spec)
        h = m.moma_create_array(nx, ny, 5, 0)
        try:
            m.moma_set_blocks(h, blocks)
            zp = np.zeros((nx * ny, nx * ny), np.complex128)
            m.moma_port_impedance(h, zp)
        finally:
            m.moma_destroy(h)
        xz, xmax, bound = m.moma_xi_z(zp, nx, ny)
        assert abs(xz - pr.xi_z(zp, nx, ny)) <= 1e-15 * xz
        assert abs(xmax - pr.xi_z_max(zp, nx, ny)) <= 1e-15 * xmax
        assert abs(bound - pr.border_bound(zp, nx, ny)) <= 1e-13 * bound
