"""Ragged batches, CUDA-graph replay and the autotuner: none of them may
change a result.  Batched solves of uneven lattices equal stand-alone
solves bitwise and the dense oracle to the solve tolerance; graph replay
equals direct launches; the autotuner reports what it picked."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 5, 0.5), (2, 3, 8, 0.3), (6, 4, 12, 0.7), (5, 5, 9, 0.5), (8, 8, 16, 0.4), (3, 9, 6, 0.6)]


def test_ragged_batch_equals_single_solves(moma_lib, cuda):
    m = moma_lib
    specs = [LatticeSpec(nx, ny, b, d, 3) for nx, ny, b, d in SIZES]
    blocks = [offset_blocks(s, np.complex64) for s in specs]
    Vs = [excitation(s, [(0, 0), (35, 20)][: 1 + i % 2]) for i, s in enumerate(specs)]
    hs = [m.moma_create_array(s.nx, s.ny, s.b) for s in specs]
    try:
        m.moma_set_blocks_batch(hs, blocks, release_setup=True, workers=3)
        Is = [np.zeros_like(V) for V in Vs]
        infos = m.moma_solve_batch(hs, Vs, Is, workers=3)
        assert all(x["converged"] == 1 for x in infos)
    finally:
        for h in hs:
            m.moma_destroy(h)
    for s, bl, V, I in zip(specs, blocks, Vs, Is):
        h = m.moma_create_array(s.nx, s.ny, s.b)
        try:
            m.moma_set_blocks(h, bl)
            I1 = np.zeros_like(V)
            m.moma_solve(h, V, I1)
        finally:
            m.moma_destroy(h)
        assert np.array_equal(I, I1)
        z = dense.assemble(bl.astype(np.complex128), s.nx, s.ny)
        assert dense.relative_residual(z, I, V).max() <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_direct_launches(moma_lib, cuda, prec):
    m = moma_lib
    spec = LatticeSpec(7, 6, 10, 0.5, 8)
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, [(0, 0), (30, 45), (55, 5)])
    res = []
    for flags in (0, m.MOMA_FLAG_NO_GRAPHS):
        h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            for _ in range(2):  # the second solve replays the captured steps
                I = np.zeros_like(V)
                m.moma_solve(h, V, I)
            res.append(I)
        finally:
            m.moma_destroy(h)
    assert np.array_equal(res[0], res[1])


def test_autotuner_reports_choices(moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(6, 6, 16, 0.5, 1)
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, [(0, 0)])
    h = m.moma_create_array(spec.nx, spec.ny, spec.b)
    h2 = m.moma_create_array(spec.nx, spec.ny, spec.b, flags=m.MOMA_FLAG_NO_AUTOTUNE)
    try:
        assert m.moma_tuning_report(h) == ""
        for x in (h, h2):
            m.moma_set_blocks(x, blocks)
            I = np.zeros_like(V)
            m.moma_solve(x, V, I)
        rep = m.moma_tuning_report(h)
        # inner product in c64 (its lattice passes are register-resident:
        # no launch shape to tune); the refinement residual's per-axis
        # passes and product in double-FP32 pairs
        assert "bin_product<c64>" in rep and "bin_product<dfl>" in rep and "Fx<dfl>" in rep, rep
        # No timing trials without autotuning: the array takes the shapes the
        # first one tuned (process-wide cache for the same shape) or heuristics.
        rep2 = m.moma_tuning_report(h2)
        assert "bin_product" not in rep2 and "F2<" not in rep2
    finally:
        m.moma_destroy(h)
        m.moma_destroy(h2)


def test_tuned_shapes_are_shared_across_arrays_of_a_shape(moma_lib, cuda):
    """A second array of the same shape and RHS count takes the first one's
    tuned launch shapes from the process-wide cache (no timing trials), and
    its solution is bitwise the first one's."""
    m = moma_lib
    spec = LatticeSpec(9, 7, 24, 0.45, 2)
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, [(0, 0), (20, 70), (45, 10)])
    out, reps = [], []
    for flags in (0, 0, m.MOMA_FLAG_NO_AUTOTUNE):
        h = m.moma_create_array(spec.nx, spec.ny, spec.b, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            I = np.zeros_like(V)
            m.moma_solve(h, V, I)
            out.append(I)
            reps.append(m.moma_tuning_report(h))
        finally:
            m.moma_destroy(h)
    assert all("process-wide cache" in r for r in reps[1:]), reps
    assert all("bin_product" not in r for r in reps[1:])
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nx,ny,b,nr", [(7, 6, 10, 3), (16, 12, 32, 2), (1, 1, 4, 1)])
def test_fused_arnoldi_step_equals_separate_sweeps(moma_lib, cuda, prec, nx, ny, b, nr):
    """The cooperative Arnoldi step (three CGS2 sweeps, Givens update and
    scaling in one launch, grid barriers between the sweeps) reduces in the
    same fixed order as the separate sweep launches: bitwise the same
    solution, graphs on and off; and the solution matches the dense oracle."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 8)
    blocks = offset_blocks(spec, np.complex64 if prec else np.complex128)
    V = excitation(spec, [(0, 0), (30, 45), (55, 5)][:nr])
    res = []
    for flags in (0, m.MOMA_FLAG_SPLIT_ARNOLDI, m.MOMA_FLAG_NO_GRAPHS):
        h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            for _ in range(2):
                I = np.zeros_like(V)
                info = m.moma_solve(h, V, I)
            res.append(I)
        finally:
            m.moma_destroy(h)
        assert info["converged"] == 1
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
    z = dense.assemble(blocks.astype(np.complex128), spec.nx, spec.ny)
    assert dense.relative_residual(z, res[0], V).max() <= 1e-10


def test_fresh_arrays_on_worker_streams_never_skip_the_solve(moma_lib, cuda):
    """Many fresh arrays set up and solved concurrently on the batch's
    non-blocking worker streams (workspaces allocated and zeroed inside the
    calls): every solve must run (outer_iters >= 1 from the zero start),
    reach the tolerance, and return nonzero port currents.  A workspace
    zeroing that was not ordered on the array's stream once let a solve see
    ||V|| = 0 and stop at I = 0."""
    m, torch = moma_lib, cuda
    specs = [LatticeSpec(n, n + (k % 3), 12 + 2 * (k % 4), 0.3 + 0.1 * (k % 5), 0) for k, n in
             enumerate([2, 3, 4, 5, 6, 7, 8] * 6)]
    for rep in range(3):
        hs = [m.moma_create_array(s.nx, s.ny, s.b) for s in specs]
        try:
            blocks = [torch.from_numpy(offset_blocks(s, np.complex64)).cuda() for s in specs]
            Vs = [torch.from_numpy(excitation(s, [(0, 0)])).cuda() for s in specs]
            Is = [torch.zeros_like(v) for v in Vs]
            m.moma_set_blocks_batch(hs, blocks, workers=8)
            infos = m.moma_solve_batch(hs, Vs, Is, workers=8)
            torch.cuda.synchronize()
            for s, info, I in zip(specs, infos, Is):
                ip = I.cpu().numpy()[..., 0]
                assert info["converged"] == 1 and info["outer_iters"] >= 1 and 0 < info["max_rel_residual"] <= 1e-10, \
                    (rep, s, info)
                assert np.abs(ip).min() > 0, (rep, s)
        finally:
            for h in hs:
                m.moma_destroy(h)
