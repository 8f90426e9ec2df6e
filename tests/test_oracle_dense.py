"""Pins of the dense oracle (assembly, LU solve, port quantities) against
things other than itself: the lattice geometry entry by entry, exact
structural invariants, brute-force inversion, network-reduction closed forms
and an independent second route to Z_a."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation, element_geometry
from synth.lattice import SELF_LOAD
from oracle import dense, ports, mbt


def _entry_from_geometry(spec, m, i, n, j):
    """Z[(m,i),(n,j)] straight from the lattice positions (no offset table)."""
    p, w, al = element_geometry(spec.b, spec.d, spec.seed)
    mx, my = m % spec.nx, m // spec.nx
    sx, sy = n % spec.nx, n // spec.nx
    ro = np.array([mx * spec.d, my * spec.d]) + p[i]
    rs = np.array([sx * spec.d, sy * spec.d]) + p[j]
    r = max(np.linalg.norm(ro - rs), 0.01)
    val = w[i] * w[j] * np.cos(al[i] - al[j]) * np.exp(-2j * np.pi * r) / (4 * np.pi * r)
    if m == n and i == j:
        val += SELF_LOAD
    return val


@pytest.mark.parametrize("nx,ny,b", [(3, 2, 4), (2, 3, 3), (1, 4, 2)])
def test_assembly_matches_geometry(nx, ny, b):
    spec = LatticeSpec(nx, ny, b, 0.45, 5)
    z = dense.assemble(offset_blocks(spec), nx, ny)
    rng = np.random.default_rng(0)
    for _ in range(60):
        m, n = rng.integers(nx * ny, size=2)
        i, j = rng.integers(b, size=2)
        assert np.isclose(z[m * b + i, n * b + j], _entry_from_geometry(spec, m, i, n, j), rtol=1e-13, atol=0)


def test_toeplitz_and_reciprocity_exact():
    nx, ny, b = 4, 3, 3
    spec = LatticeSpec(nx, ny, b, 0.5, 2)
    z = dense.assemble(offset_blocks(spec), nx, ny)
    assert np.array_equal(z, z.T)  # reciprocity (Sec. II-D)
    def blk(mx, my, sx, sy):
        m, n = mx + nx * my, sx + nx * sy
        return z[m * b:(m + 1) * b, n * b:(n + 1) * b]
    for (mx, my, sx, sy) in [(0, 0, 1, 1), (1, 0, 2, 2), (2, 1, 0, 0), (3, 2, 1, 0)]:
        for tx, ty in [(0, 0), (-1, 0), (0, -1), (-1, -1)]:
            if all(0 <= c < nx for c in (mx + tx, sx + tx)) and all(0 <= c < ny for c in (my + ty, sy + ty)):
                assert np.array_equal(blk(mx, my, sx, sy), blk(mx + tx, my + ty, sx + tx, sy + ty))


def test_lu_solve_against_brute_force_inverse():
    spec = LatticeSpec(3, 3, 4, 0.5, 0)
    z = dense.assemble(offset_blocks(spec), 3, 3)
    v = excitation(spec, [(0, 0), (30, 45)])
    i = dense.solve(z, v)
    ibf = (np.linalg.inv(z) @ v.reshape(2, -1).T).T.reshape(v.shape)
    assert np.allclose(i, ibf, rtol=1e-12, atol=1e-15)
    assert dense.relative_residual(z, i, v).max() < 1e-14


def test_single_element_is_isolated_input_impedance():
    """1x1 array: Z_a equals the isolated element's input impedance, i.e. the
    Schur complement z_00 - z_0r Z_rr^{-1} z_r0 of the self block (network
    reduction onto the port)."""
    spec = LatticeSpec(1, 1, 6, 0.5, 3)
    blocks = offset_blocks(spec)
    z0 = blocks[0, 0]
    v = excitation(spec, [(0, 0)])
    za = ports.active_impedance(dense.solve(dense.assemble(blocks, 1, 1), v), v)[0, 0, 0]
    schur = z0[0, 0] - z0[0, 1:] @ np.linalg.solve(z0[1:, 1:], z0[1:, 0])
    assert np.isclose(za, schur, rtol=1e-13)


def test_two_element_even_odd_modes():
    """b = 1, 2x1 array: Z = [[z0, z1], [z1, z0]]; broadside gives z0 + z1,
    anti-phase gives z0 - z1."""
    spec = LatticeSpec(2, 1, 1, 0.5, 4)
    blocks = offset_blocks(spec)
    z0, z1 = blocks[0, 1, 0, 0], blocks[0, 2, 0, 0]
    z = dense.assemble(blocks, 2, 1)
    v = np.array([[[[1.0]], [[1.0]]], [[[1.0]], [[-1.0]]]], dtype=complex).reshape(2, 1, 2, 1)
    za = ports.active_impedance(dense.solve(z, v), v)
    assert np.allclose(za[0, 0], z0 + z1, rtol=1e-14)
    assert np.allclose(za[1, 0], z0 - z1, rtol=1e-14)


def test_uncoupled_lattice_gives_self_impedance():
    nx, ny = 3, 2
    blocks = np.zeros((2 * ny - 1, 2 * nx - 1, 1, 1), dtype=complex)
    blocks[ny - 1, nx - 1] = 42.0 - 7.0j
    v = excitation(LatticeSpec(nx, ny, 1), [(20, 30)])
    za = ports.active_impedance(dense.solve(dense.assemble(blocks, nx, ny), v), v)
    assert np.allclose(za, 42.0 - 7.0j, rtol=1e-15)


def test_two_routes_to_active_impedance_and_symmetric_zp():
    nx, ny, b = 3, 3, 4
    spec = LatticeSpec(nx, ny, b, 0.5, 1)
    z = dense.assemble(offset_blocks(spec), nx, ny)
    v = excitation(spec, [(0, 0), (40, 10)])
    i = dense.solve(z, v)
    za1 = ports.active_impedance(i, v)
    zp = ports.port_impedance_matrix(z, nx, ny, b)
    assert np.allclose(zp, zp.T, rtol=1e-12, atol=1e-12)
    ip = ports.port_currents(i).reshape(2, -1)
    za2 = ports.active_impedance_from_zp(zp, ip).reshape(za1.shape)
    assert np.allclose(za1, za2, rtol=1e-11)


def test_zp_equals_z_when_every_basis_is_a_port():
    spec = LatticeSpec(3, 2, 1, 0.5, 9)
    z = dense.assemble(offset_blocks(spec), 3, 2)
    assert np.allclose(ports.port_impedance_matrix(z, 3, 2, 1), z, rtol=1e-12)


def test_reflection_and_rrmse():
    assert ports.reflection(np.array(50.0 + 0j)) == 0
    assert np.isclose(ports.reflection(np.array(150.0 + 0j)), 0.5)
    assert np.isclose(ports.reflection(np.array(1j * 50.0)), 1j)  # |Gamma| = 1 for reactive load
    assert ports.rrmse([1.0 + 1e-3], [1.0]) == pytest.approx(1e-3)
    assert ports.named_elements(5, 4) == {"centre": (2, 2), "edge": (0, 2), "corner": (0, 0)}
