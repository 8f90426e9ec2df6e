"""The ragged workload at its stated shapes: square lattices 2x2 .. 48x48
(step 2), b = 96, spacings 0.3 / 0.5 / 0.7 wavelengths, one broadside solve
each (72 problems, the centre-element active impedance vs array size sweep
of Sec. IV / Fig. 4), set up and solved as one ragged batch.

Checks, per problem: the solve converged; its residual recomputed by the
oracle's FP64 direct offset sum (Eq. 1, no FFT) is <= 1e-10; for N <= 3456
(lattices up to 6 x 6) the active impedance of every port matches the dense
LU oracle within 1e-8; for 16 x 16 and 32 x 32 at 0.5 wavelengths the centre
element's Z_a matches oracle-I (GMRES on Z I = V, tol 1e-13) within 1e-8."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks_torch, excitation
from oracle import dense, iterative, mbt, ports

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", [0.3, 0.5, 0.7])
def test_ragged_b96_sweep(moma_lib, cuda, d):
    m, torch = moma_lib, cuda
    specs = [LatticeSpec(n, n, 96, d, 0) for n in range(2, 49, 2)]
    blocks = [offset_blocks_torch(s, "cuda") for s in specs]  # c64, the problem definition
    Vs = [excitation(s, [(0.0, 0.0)]) for s in specs]
    Vd = [torch.from_numpy(v).cuda() for v in Vs]
    Id = [torch.zeros_like(v) for v in Vd]
    zad = [torch.zeros(v.shape[:3], dtype=torch.complex128, device="cuda") for v in Vd]
    hs = [m.moma_create_array(s.nx, s.ny, s.b) for s in specs]
    try:
        m.moma_set_blocks_batch(hs, blocks, release_setup=True, workers=8)
        infos = m.moma_solve_batch(hs, Vd, Id, workers=8)
        for h, I, V, za in zip(hs, Id, Vd, zad):
            m.moma_active_impedance(h, I, V, za)
        torch.cuda.synchronize()
    finally:
        for h in hs:
            m.moma_destroy(h)
    assert all(x["converged"] == 1 for x in infos), infos
    for s, bl, V, I, za in zip(specs, blocks, Vs, Id, zad):
        b128 = bl.cpu().numpy().astype(np.complex128)
        I = I.cpu().numpy()
        za = za.cpu().numpy()
        r = V - mbt.matvec(b128, s.nx, s.ny, I)
        cert = float(np.linalg.norm(r) / np.linalg.norm(V))
        assert cert <= 1e-10, (s, cert)
        if s.n_el * s.b <= 3456:
            z = dense.assemble(b128, s.nx, s.ny)
            za_ref = ports.active_impedance(dense.solve(z, V), V)
            err = float(np.max(np.abs(za - za_ref) / np.abs(za_ref)))
            assert err <= 1e-8, (s, err)
        elif d == 0.5 and s.nx in (16, 32):
            i_ref, _ = iterative.gmres(b128, s.nx, s.ny, V, tol=1e-13, restart=60)
            za_ref = ports.active_impedance(i_ref, V)
            c = (s.ny // 2, s.nx // 2)
            err = abs(za[0][c] - za_ref[0][c]) / abs(za_ref[0][c])
            print(f"{s.nx}x{s.ny}@{d}: centre Z_a {za[0][c]:.6f}, oracle-I {za_ref[0][c]:.6f}, rel err {err:.2e}")
            assert err <= 1e-8
        del b128
    print(f"d={d}: certified residuals <= 1e-10 for all {len(specs)} lattices; centre Z_a by size:",
          [f"{s.nx}: {complex(za[0, s.ny // 2, s.nx // 2]):.4f}" for s, za in zip(specs, [z.cpu().numpy() for z in zad])][::4])
