"""Pins of the MBT-operator oracle: the direct offset sum against the dense
assembly, Z^H against the dense adjoint and the reciprocity identity, the
preconditioner blocks against the dense Z^H Z, and the circulant bins
against the circulant-embedding identity (Eq. 3), the Hermitian commutation
theorem (Eq. 6) and the pairing Zhat_{-k} = Zhat_k^T."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks
from oracle import dense, mbt


def _rand_vec(rng, nrhs, ny, nx, b):
    return rng.standard_normal((nrhs, ny, nx, b)) + 1j * rng.standard_normal((nrhs, ny, nx, b))


CASES = [(1, 1, 3), (2, 1, 2), (3, 2, 4), (2, 4, 3), (5, 3, 2)]


@pytest.mark.parametrize("nx,ny,b", CASES)
def test_matvec_and_adjoint_match_dense(nx, ny, b):
    spec = LatticeSpec(nx, ny, b, 0.5, 3)
    blocks = offset_blocks(spec)
    z = dense.assemble(blocks, nx, ny)
    x = _rand_vec(np.random.default_rng(1), 2, ny, nx, b)
    y = mbt.matvec(blocks, nx, ny, x)
    assert np.allclose(y.reshape(2, -1), (z @ x.reshape(2, -1).T).T, rtol=1e-13, atol=1e-13)
    yh = mbt.matvec_h(blocks, nx, ny, x)
    assert np.allclose(yh.reshape(2, -1), (z.conj().T @ x.reshape(2, -1).T).T, rtol=1e-13, atol=1e-13)
    # Z symmetric => Z^H x = conj(Z conj(x))
    assert np.allclose(yh, np.conj(mbt.matvec(blocks, nx, ny, np.conj(x))), rtol=1e-13, atol=1e-13)


def test_matvec_nonsymmetric_blocks_still_match_dense():
    """The offset sum must not rely on reciprocity: random blocks."""
    nx, ny, b = 3, 2, 3
    rng = np.random.default_rng(5)
    blocks = rng.standard_normal((2 * ny - 1, 2 * nx - 1, b, b)) + 1j * rng.standard_normal((2 * ny - 1, 2 * nx - 1, b, b))
    z = dense.assemble(blocks, nx, ny)
    x = _rand_vec(rng, 1, ny, nx, b)
    assert np.allclose(mbt.matvec(blocks, nx, ny, x).ravel(), z @ x.ravel(), rtol=1e-13, atol=1e-12)
    assert np.allclose(mbt.matvec_h(blocks, nx, ny, x).ravel(), z.conj().T @ x.ravel(), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("nx,ny,b", [(1, 1, 3), (3, 2, 4), (2, 3, 3)])
def test_precond_blocks_are_block_diagonal_of_normal_matrix(nx, ny, b):
    spec = LatticeSpec(nx, ny, b, 0.5, 4)
    blocks = offset_blocks(spec)
    z = dense.assemble(blocks, nx, ny)
    zhz = z.conj().T @ z
    p = mbt.precond_blocks(blocks, nx, ny)
    for iy in range(ny):
        for ix in range(nx):
            e = ix + nx * iy
            assert np.allclose(p[iy, ix], zhz[e * b:(e + 1) * b, e * b:(e + 1) * b], rtol=1e-13, atol=1e-12)
            assert np.allclose(p[iy, ix], p[iy, ix].conj().T, rtol=1e-14, atol=1e-12)
            np.linalg.cholesky(p[iy, ix])  # Hermitian positive definite


def test_normal_operator_and_equal_spectra():
    """P^{-1} Z^H Z against dense, and sigma(P^{-1} Z^H Z) = sigma(L^{-1} Z^H Z L^{-H})
    with P = L L^H, real and positive (Sec. III-A)."""
    nx, ny, b = 3, 2, 3
    spec = LatticeSpec(nx, ny, b, 0.5, 6)
    blocks = offset_blocks(spec)
    z = dense.assemble(blocks, nx, ny)
    p = mbt.precond_blocks(blocks, nx, ny)
    n = z.shape[0]
    pd = np.zeros((n, n), dtype=complex)
    for iy in range(ny):
        for ix in range(nx):
            e = ix + nx * iy
            pd[e * b:(e + 1) * b, e * b:(e + 1) * b] = p[iy, ix]
    a = np.linalg.solve(pd, z.conj().T @ z)
    x = _rand_vec(np.random.default_rng(2), 1, ny, nx, b)
    assert np.allclose(mbt.normal_operator(blocks, nx, ny, x, p).ravel(), a @ x.ravel(), rtol=1e-12, atol=1e-12)
    l = np.linalg.cholesky(pd)
    li = np.linalg.inv(l)
    s = li @ z.conj().T @ z @ li.conj().T
    ev1 = np.sort(np.linalg.eigvals(a).real)
    ev2 = np.linalg.eigvalsh(s)
    assert np.abs(np.linalg.eigvals(a).imag).max() < 1e-10
    assert np.allclose(ev1, ev2, rtol=1e-10)
    assert ev2.min() > 0


def _circulant_apply(bins, x, nx, ny):
    """IFFT(diag(bins) FFT(pad x)) truncated to the lattice (Eq. 3), written
    in the test only to check the oracle's bins."""
    my, mx = bins.shape[:2]
    nrhs, _, _, b = x.shape
    pad = np.zeros((nrhs, my, mx, b), dtype=complex)
    pad[:, :ny, :nx] = x
    xh = np.fft.fft2(pad, axes=(1, 2))
    yh = np.einsum("yxij,qyxj->qyxi", bins, xh)
    return np.fft.ifft2(yh, axes=(1, 2))[:, :ny, :nx]


@pytest.mark.parametrize("nx,ny,b,extra", [(1, 1, 2, 0), (2, 1, 2, 0), (3, 2, 3, 0), (3, 2, 3, 3), (4, 3, 2, 1)])
def test_circulant_bins_embedding_identity(nx, ny, b, extra):
    spec = LatticeSpec(nx, ny, b, 0.5, 8)
    blocks = offset_blocks(spec)
    mx, my = 2 * nx - 1 + extra, 2 * ny - 1 + (extra + 1) // 2
    bins = mbt.circulant_bins(blocks, nx, ny, mx, my)
    x = _rand_vec(np.random.default_rng(3), 2, ny, nx, b)
    assert np.allclose(_circulant_apply(bins, x, nx, ny), mbt.matvec(blocks, nx, ny, x), rtol=1e-12, atol=1e-12)


def test_circulant_bins_hermitian_commutation_and_pairing():
    """Eq. 6: the transformed first column of Z^H's embedding equals the
    per-bin conjugate transpose of Z's.  Z^H has offset blocks
    W_Delta = (Z_{-Delta})^H.  Also Zhat_{-k} = Zhat_k^T (reciprocity)."""
    nx, ny, b = 3, 4, 3
    spec = LatticeSpec(nx, ny, b, 0.5, 9)
    blocks = offset_blocks(spec)
    w = np.conj(np.transpose(blocks[::-1, ::-1], (0, 1, 3, 2)))
    mx, my = 2 * nx - 1, 2 * ny
    zb = mbt.circulant_bins(blocks, nx, ny, mx, my)
    wb = mbt.circulant_bins(w, nx, ny, mx, my)
    assert np.allclose(wb, np.conj(np.transpose(zb, (0, 1, 3, 2))), rtol=1e-12, atol=1e-12)
    for ky in range(my):
        for kx in range(mx):
            assert np.allclose(zb[(-ky) % my, (-kx) % mx], zb[ky, kx].T, rtol=1e-12, atol=1e-12)


def test_circulant_bin_by_explicit_sum():
    nx, ny, b = 2, 3, 2
    blocks = offset_blocks(LatticeSpec(nx, ny, b, 0.5, 1))
    mx, my = 4, 6
    zb = mbt.circulant_bins(blocks, nx, ny, mx, my)
    for (ky, kx) in [(0, 0), (1, 3), (5, 2)]:
        acc = np.zeros((b, b), dtype=complex)
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                acc += blocks[dy + ny - 1, dx + nx - 1] * np.exp(-2j * np.pi * (kx * dx / mx + ky * dy / my))
        assert np.allclose(zb[ky, kx], acc, rtol=1e-13, atol=1e-13)
