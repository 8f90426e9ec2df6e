"""The multilevel block-Toeplitz operator by its definition.

Blocks: [2Ny-1][2Nx-1][b][b], offset (dx, dy) at (dy+Ny-1, dx+Nx-1).
Vectors: [nrhs][Ny][Nx][b].
"""
import numpy as np


def _blk(blocks, nx, ny, dx, dy):
    return blocks[dy + ny - 1, dx + nx - 1]


def matvec(blocks, nx, ny, x):
    """y = Z x with y_m = sum_n Z_{m-n} x_n (Sec. II-A, Eq. 1: the block of
    observation element m and source element n depends only on m - n).

    Written as a direct sum over the offsets Delta = m - n; each term is one
    small matrix product over all elements m whose source m - Delta exists.
    """
    x = np.asarray(x, dtype=np.complex128)
    y = np.zeros_like(x)
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            zb = _blk(blocks, nx, ny, dx, dy).astype(np.complex128)
            oy0, oy1 = max(0, dy), min(ny, ny + dy)  # observation rows with a source
            ox0, ox1 = max(0, dx), min(nx, nx + dx)
            src = x[:, oy0 - dy:oy1 - dy, ox0 - dx:ox1 - dx, :]
            y[:, oy0:oy1, ox0:ox1, :] += src @ zb.T
    return y


def matvec_h(blocks, nx, ny, x):
    """y = Z^H x: (Z^H)_{m,n} = (Z_{n,m})^H = (Z_{n-m})^H, so
    y_m = sum_n (Z_{n-m})^H x_n (the operator applied first in the
    preconditioning strategy of Sec. II-B, Eq. 5)."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.zeros_like(x)
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            zh = _blk(blocks, nx, ny, dx, dy).astype(np.complex128).conj().T
            # term for offset Delta = n - m: y_m += Z_Delta^H x_{m + Delta}
            oy0, oy1 = max(0, -dy), min(ny, ny - dy)
            ox0, ox1 = max(0, -dx), min(nx, nx - dx)
            src = x[:, oy0 + dy:oy1 + dy, ox0 + dx:ox1 + dx, :]
            y[:, oy0:oy1, ox0:ox1, :] += src @ zh.T
    return y


def precond_blocks(blocks, nx, ny):
    """Diagonal blocks of Z_A^H Z_A (Sec. III-A, Eq. 37):

        [P_A]_{i,i} = sum_j ([Z_A]_{j,i})^H [Z_A]_{j,i},  [Z_A]_{j,i} = Z_{j-i},

    summed over every element j of the lattice.  Returns [Ny][Nx][b][b].
    (The printed index pattern of Eq. 37 is read as the block (j, i) of Z_A,
    which is what the block diagonal of Z^H Z contains.)
    """
    b = blocks.shape[-1]
    p = np.zeros((ny, nx, b, b), dtype=np.complex128)
    for iy in range(ny):
        for ix in range(nx):
            acc = np.zeros((b, b), dtype=np.complex128)
            for jy in range(ny):
                for jx in range(nx):
                    zji = _blk(blocks, nx, ny, jx - ix, jy - iy).astype(np.complex128)
                    acc += zji.conj().T @ zji
            p[iy, ix] = acc
    return p


def precond_solve(p, x):
    """P^{-1} x for the block-diagonal P (Eq. 38 without the margin part):
    one b x b dense solve per element."""
    ny, nx, b, _ = p.shape
    x = np.asarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    for iy in range(ny):
        for ix in range(nx):
            y[:, iy, ix, :] = np.linalg.solve(p[iy, ix], x[:, iy, ix, :].T).T
    return y


def normal_operator(blocks, nx, ny, x, p=None):
    """P^{-1} Z^H Z x, the operator of the GMRES form of the preconditioning
    strategy (Sec. III-A: P^{-1} Z^H Z I = P^{-1} Z^H V)."""
    if p is None:
        p = precond_blocks(blocks, nx, ny)
    return precond_solve(p, matvec_h(blocks, nx, ny, matvec(blocks, nx, ny, x)))


def circulant_bins(blocks, nx, ny, mx, my):
    """Transformed first column of the circulant embedding, Eqs. 3 and 11:

        Zhat[ky][kx] = sum_Delta Z_Delta exp(-2 pi i (kx dx / Mx + ky dy / My)),

    with the embedding placing offset Delta at circulant index Delta mod M.
    Any Mx >= 2Nx-1, My >= 2Ny-1 makes the embedding exact (Sec. II-A uses
    2N-1).  Returns [My][Mx][b][b]; numpy's FFT evaluates the sum.
    """
    assert mx >= 2 * nx - 1 and my >= 2 * ny - 1
    b = blocks.shape[-1]
    col = np.zeros((my, mx, b, b), dtype=np.complex128)
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            col[dy % my, dx % mx] = _blk(blocks, nx, ny, dx, dy)
    return np.fft.fft2(col, axes=(0, 1))


def precond_margin(zb, zc):
    """Margin block of the preconditioner (the matrix P_C of Eq. 38):
    P_C = conj(Z_B) Z_B^T + Z_C^H Z_C, the margin-margin block of Z^H Z."""
    zb = np.asarray(zb, dtype=np.complex128)
    zc = np.asarray(zc, dtype=np.complex128)
    return zb.conj() @ zb.T + zc.conj().T @ zc


def precond_solve_margin(p, pc, x, n):
    """blockdiag(P_A, P_C)^{-1} x (Eq. 38) for vectors [nrhs][N + nm]: the
    lattice part by the element blocks p [Ny][Nx][b][b], the margin part by
    P_C."""
    ny, nx, b, _ = p.shape
    x = np.asarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    y[:, :n] = precond_solve(p, x[:, :n].reshape(-1, ny, nx, b)).reshape(x.shape[0], n)
    y[:, n:] = np.linalg.solve(pc, x[:, n:].T).T
    return y

