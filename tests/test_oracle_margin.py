"""Pins of the margin part of the oracle (Eq. 1 block form, Eq. 38 margin
preconditioner block) and of the synthetic margin generator."""
import numpy as np

from synth import LatticeSpec, offset_blocks, margin_blocks, margin_geometry
from oracle import dense, mbt


def _case():
    spec = LatticeSpec(3, 2, 4, 0.5, 1)
    blocks = offset_blocks(spec)
    zb, zc = margin_blocks(spec, bm=2)
    return spec, blocks, zb, zc


def test_margin_generator_shapes_and_ring():
    spec, blocks, zb, zc = _case()
    pos, w, a = margin_geometry(spec, 2)
    ring = (spec.nx + 2) * (spec.ny + 2) - spec.nx * spec.ny
    assert zb.shape == (2 * ring, spec.n) and zc.shape == (2 * ring, 2 * ring)
    # every margin basis lies outside the lattice's cells
    d = spec.d
    inside = (pos[:, 0] >= 0) & (pos[:, 0] < spec.nx * d) & (pos[:, 1] >= 0) & (pos[:, 1] < spec.ny * d)
    assert not inside.any()
    assert np.allclose(np.diag(zc).real > 40, True)  # self-loaded


def test_assembled_margin_matrix_is_reciprocal_and_keeps_blocks():
    spec, blocks, zb, zc = _case()
    z = dense.assemble_with_margin(blocks, spec.nx, spec.ny, zb, zc)
    n = spec.n
    assert np.abs(z - z.T).max() == 0.0  # Sec. II-D: the MoM matrix is symmetric
    assert np.array_equal(z[:n, :n], dense.assemble(blocks, spec.nx, spec.ny))
    assert np.array_equal(z[n:, :n], zb) and np.array_equal(z[n:, n:], zc)


def test_margin_preconditioner_block_is_block_of_normal_matrix():
    """Eq. 38: P_C is the margin-margin block of Z^H Z (formed here from the
    assembled dense Z, not from the formula)."""
    spec, blocks, zb, zc = _case()
    z = dense.assemble_with_margin(blocks, spec.nx, spec.ny, zb, zc)
    n = spec.n
    zhz = z.conj().T @ z
    pc = mbt.precond_margin(zb, zc)
    assert np.abs(pc - zhz[n:, n:]).max() <= 1e-12 * np.abs(pc).max()
    # P_A keeps only Z_A^H Z_A's diagonal blocks (the paper drops Z_B^H Z_B):
    za = z[:n, :n]
    zaha = za.conj().T @ za
    p = mbt.precond_blocks(blocks, spec.nx, spec.ny)
    b = spec.b
    for e in range(spec.n_el):
        ey, ex = divmod(e, spec.nx)
        assert np.abs(p[ey, ex] - zaha[e * b:(e + 1) * b, e * b:(e + 1) * b]).max() <= 1e-12 * np.abs(p).max()


def test_margin_precond_solve_inverts_block_diagonal():
    spec, blocks, zb, zc = _case()
    n, nm = spec.n, zc.shape[0]
    p = mbt.precond_blocks(blocks, spec.nx, spec.ny)
    pc = mbt.precond_margin(zb, zc)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, n + nm)) + 1j * rng.standard_normal((3, n + nm))
    y = mbt.precond_solve_margin(p, pc, x, n)
    # multiply back with the explicit block-diagonal P
    P = np.zeros((n + nm, n + nm), np.complex128)
    b = spec.b
    for e in range(spec.n_el):
        ey, ex = divmod(e, spec.nx)
        P[e * b:(e + 1) * b, e * b:(e + 1) * b] = p[ey, ex]
    P[n:, n:] = pc
    assert np.abs(y @ P.T - x).max() <= 1e-10 * np.abs(x).max()
