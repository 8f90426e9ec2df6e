"""GPU parity of the all-port passive impedance matrix Z_p (Eq. 18) against
the oracle's dense definition Y_p = [Z^{-1}]_{ports,ports}, Z_p = Y_p^{-1}.

Checks: Y_p and Z_p element by element (chunks with a ragged tail, both
precisions and both inner solvers), reciprocity Z_p = Z_p^T, and Eq. 17:
the port currents of a scanned solve satisfy Z_p I_p = V_p, i.e. the
active impedance obtained from Z_p equals the one obtained from the solve.
"""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense, ports

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("nx,ny,b,prec,chunk,solver,pb", [
    (4, 3, 8, 0, 5, 0, 0),      # 12 ports in chunks 5, 5, 2
    (5, 4, 16, 1, 0, 0, 3),     # one chunk, non-zero port basis
    (6, 5, 6, 1, 7, 1, 0),      # PCG inner solver, ragged tail
    (1, 1, 3, 1, 0, 0, 1),      # single element
])
def test_port_matrix_matches_dense_definition(moma_lib, cuda, nx, ny, b, prec, chunk, solver, pb):
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 0)
    blocks = offset_blocks(spec)
    z = dense.assemble(blocks, nx, ny)
    ports_idx = np.arange(nx * ny) * b + pb
    yp_ref = np.linalg.inv(z)[np.ix_(ports_idx, ports_idx)]
    zp_ref = ports.port_impedance_matrix(z, nx, ny, b, pb)
    h = m.moma_create_array(nx, ny, b, prec)
    try:
        m.moma_set_blocks(h, blocks)
        n = nx * ny
        zp = np.zeros((n, n), np.complex128)
        yp = np.zeros((n, n), np.complex128)
        m.moma_port_impedance(h, zp, yp, port_basis=pb, chunk=chunk, solver=solver)
    finally:
        m.moma_destroy(h)
    ey, ez = relerr(yp, yp_ref), relerr(zp, zp_ref)
    print(f"Z_p {nx}x{ny}x{b}: Y_p err {ey:.3g}, Z_p err {ez:.3g}")
    assert ey <= 1e-9 and ez <= 1e-8
    assert relerr(zp, zp.T) <= 1e-8


def test_port_matrix_reproduces_active_impedance(moma_lib, cuda):
    """Eq. 17: Z_a = diag(I_p)^{-1} Z_p I_p equals V_p / I_p of a solve."""
    m = moma_lib
    spec = LatticeSpec(8, 6, 12, 0.5, 3)
    blocks = offset_blocks(spec)
    V = excitation(spec, [(0.0, 0.0), (30.0, 45.0), (50.0, 90.0)])
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, 1)
    try:
        m.moma_set_blocks(h, blocks)
        I = np.zeros_like(V)
        m.moma_solve(h, V, I)
        za = np.zeros(V.shape[:3], np.complex128)
        m.moma_active_impedance(h, I, V, za)
        zp = np.zeros((spec.n_el, spec.n_el), np.complex128)
        m.moma_port_impedance(h, zp, chunk=16)
    finally:
        m.moma_destroy(h)
    ip = ports.port_currents(I).reshape(3, -1)
    za_zp = ports.active_impedance_from_zp(zp, ip).reshape(za.shape)
    print("Eq. 17 via Z_p vs solve:", relerr(za_zp, za))
    assert relerr(za_zp, za) <= 1e-8


def test_port_matrix_device_buffers_and_errors(moma_lib, cuda):
    import torch
    m = moma_lib
    spec = LatticeSpec(3, 3, 4, 0.5, 0)
    blocks = offset_blocks(spec)
    h = m.moma_create_array(3, 3, 4, 0)
    try:
        with pytest.raises(m.MomaError):
            m.moma_port_impedance(h, np.zeros((9, 9), np.complex128))  # no blocks yet
        m.moma_set_blocks(h, blocks)
        with pytest.raises(m.MomaError):
            m.moma_port_impedance(h, np.zeros((9, 9), np.complex128), port_basis=4)
        zp_h = np.zeros((9, 9), np.complex128)
        m.moma_port_impedance(h, zp_h)
        zp_d = torch.zeros((9, 9), dtype=torch.complex128, device="cuda")
        m.moma_port_impedance(h, zp_d)
        assert np.array_equal(zp_d.cpu().numpy(), zp_h)
    finally:
        m.moma_destroy(h)
