"""oracle-I (GMRES on the original system with the direct offset sum)
against oracle-L (dense LU) where both fit."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense, iterative, ports


@pytest.mark.parametrize("nx,ny,b,d", [(1, 1, 4, 0.5), (3, 2, 4, 0.3), (4, 4, 8, 0.5), (5, 3, 6, 0.7)])
def test_iterative_matches_dense(nx, ny, b, d):
    spec = LatticeSpec(nx, ny, b, d, 0)
    blocks = offset_blocks(spec)
    v = excitation(spec, [(0, 0), (45, 0)])
    i_l = dense.solve(dense.assemble(blocks, nx, ny), v)
    i_i, info = iterative.gmres(blocks, nx, ny, v, tol=1e-13, restart=8)
    assert all(x["rel_residual"] < 2e-13 for x in info)
    assert np.linalg.norm(i_i - i_l) / np.linalg.norm(i_l) < 1e-11
    za_l = ports.active_impedance(i_l, v)
    za_i = ports.active_impedance(i_i, v)
    assert np.max(np.abs(za_i - za_l) / np.abs(za_l)) < 1e-11
