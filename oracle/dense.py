"""Dense assembly and direct solve (oracle-L).

Sec. II-A, Eq. (1): the element block Z_A of a regular array is multilevel
block-Toeplitz -- the block coupling observation element m and source element
n depends only on the offset m - n, so it is one of the (2Nx-1)(2Ny-1) unique
b x b offset blocks.  Here the full matrix is written out explicitly from
those blocks, then Eq. (15), Z I = V, is solved by LU with partial pivoting.
"""
import numpy as np
import scipy.linalg


def element_index(mx, my, nx):
    """Element numbering of the two-level ordering of Eq. (2): x (level 1) fastest."""
    return mx + nx * my


def assemble(blocks, nx, ny):
    """Dense Z (N x N, complex128) with Z[(m,i),(n,j)] = Z_{m-n}[i][j].

    blocks: [2Ny-1][2Nx-1][b][b], offset (dx, dy) at (dy+Ny-1, dx+Nx-1).
    """
    b = blocks.shape[-1]
    nel = nx * ny
    z = np.zeros((nel * b, nel * b), dtype=np.complex128)
    for my in range(ny):
        for mx in range(nx):
            m = element_index(mx, my, nx)
            for sy in range(ny):
                for sx in range(nx):
                    n = element_index(sx, sy, nx)
                    blk = blocks[my - sy + ny - 1, mx - sx + nx - 1]
                    z[m * b:(m + 1) * b, n * b:(n + 1) * b] = blk
    return z


def assemble_with_margin(blocks, nx, ny, zb, zc):
    """Z = [Z_A, Z_B^T; Z_B, Z_C] (Eq. 1): the MBT element part from the
    offset blocks, the margin coupling Z_B (nm x N) below it and its
    transpose to the right (the MoM matrix is symmetric, Sec. II-D), the
    margin part Z_C in the corner.  Unknown order: lattice, then margin."""
    za = assemble(blocks, nx, ny)
    zb = np.asarray(zb, dtype=np.complex128)
    zc = np.asarray(zc, dtype=np.complex128)
    n, nm = za.shape[0], zc.shape[0]
    z = np.zeros((n + nm, n + nm), dtype=np.complex128)
    z[:n, :n] = za
    z[:n, n:] = zb.T
    z[n:, :n] = zb
    z[n:, n:] = zc
    return z


def solve(z, v):
    """Solve Z I = V for every RHS column by LU (LAPACK getrf/getrs).

    v: [nrhs][N] (or [nrhs][Ny][Nx][b]); returns I with the same shape.
    """
    shape = v.shape
    rhs = v.reshape(shape[0], -1).T.astype(np.complex128)
    lu, piv = scipy.linalg.lu_factor(z)
    return scipy.linalg.lu_solve((lu, piv), rhs).T.reshape(shape)


def relative_residual(z, i, v):
    """Per-RHS ||V - Z I||_2 / ||V||_2."""
    vv = v.reshape(v.shape[0], -1)
    ii = i.reshape(i.shape[0], -1)
    r = vv - (z @ ii.T).T
    return np.linalg.norm(r, axis=1) / np.linalg.norm(vv, axis=1)
