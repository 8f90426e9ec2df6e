"""GPU parity of the tensor-core (tcgen05, 3xTF32) bin product against the
oracle: Z x and Z^H x through the whole lattice-FFT path with the tensor
path forced (several RHS tile widths, ragged RHS tails, b not a multiple of
the 128-row MMA tile or of the 16-value K chunk), the normal operator, and
full solves that take the tensor path by default (>= 16 RHS).

Tolerance: the c64 products must stay within FP32-level error of the FP64
oracle (3xTF32 keeps ~22 significant bits per operand): <= 2e-5 relative;
the raw errors are printed.  Solves must still meet the 1e-10 residual and
the 1e-8 active-impedance bars.
"""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense, mbt, ports

pytestmark = pytest.mark.gpu

MIXED = 1


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rand_vec(nr, spec, seed=1):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((nr, spec.ny, spec.nx, spec.b)) + 1j * rng.standard_normal((nr, spec.ny, spec.nx, spec.b))
    return v.astype(np.complex64)


@pytest.mark.parametrize("nx,ny,b,nr", [
    (3, 2, 128, 20),   # 32-wide RHS tile, ragged
    (2, 2, 136, 5),    # 8-wide tile, b past one M tile, partial K chunk
    (4, 3, 160, 40),   # 64-wide tile, two M tiles
    (2, 3, 144, 70),   # two 64-wide RHS tiles
    (1, 1, 128, 16),   # single element, 16-wide tile
])
def test_tensor_products_match_oracle(moma_lib, cuda, nx, ny, b, nr):
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 2)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec)
    ref_z = mbt.matvec(b128, nx, ny, x.astype(np.complex128))
    ref_h = mbt.matvec_h(b128, nx, ny, x.astype(np.complex128))
    out = {}
    for name, flags in (("tensor", m.MOMA_FLAG_TENSOR_ALWAYS), ("cuda", m.MOMA_FLAG_NO_TENSOR)):
        h = m.moma_create_array(nx, ny, b, MIXED, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            m.moma_profile(h, 1)
            yz = np.zeros_like(x)
            yh = np.zeros_like(x)
            m.moma_matvec(h, m.MOMA_OP_Z, x, yz)
            m.moma_matvec(h, m.MOMA_OP_ZH, x, yh)
            n_tc = m.moma_kernel_stats(h, "bin_tc")[0]
            m.moma_profile(h, 0)
        finally:
            m.moma_destroy(h)
        out[name] = (yz, yh, n_tc)
    yz, yh, n_tc = out["tensor"]
    assert n_tc == 2 and out["cuda"][2] == 0
    ez, eh = relerr(yz, ref_z), relerr(yh, ref_h)
    cz, ch = relerr(out["cuda"][0], ref_z), relerr(out["cuda"][1], ref_h)
    print(f"tensor {nx}x{ny}x{b} nr={nr}: Z err {ez:.3g} (cuda cores {cz:.3g}), Z^H err {eh:.3g} (cuda cores {ch:.3g})")
    assert ez <= 2e-5 and eh <= 2e-5
    # Element-wise: every output entry, not only the norm.
    scale = np.abs(ref_z).max()
    assert np.abs(yz - ref_z).max() <= 1e-4 * scale


def test_tensor_normal_operator(moma_lib, cuda):
    """P^{-1} Z^H Z x (Sec. III-A) with the tensor path forced, element by
    element against the oracle's normal operator (dense-definition blocks of
    Eq. 37, direct offset sums), and against the CUDA-core path."""
    m = moma_lib
    spec = LatticeSpec(3, 3, 128, 0.5, 4)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(24, spec, seed=5)
    ref = mbt.normal_operator(b128, spec.nx, spec.ny, x.astype(np.complex128))
    ys = []
    for flags in (m.MOMA_FLAG_TENSOR_ALWAYS, m.MOMA_FLAG_NO_TENSOR):
        h = m.moma_create_array(3, 3, 128, MIXED, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            m.moma_profile(h, 1)
            y = np.zeros_like(x)
            m.moma_matvec(h, m.MOMA_OP_NORMAL, x, y)
            n_tc = m.moma_kernel_stats(h, "bin_tc")[0]
            m.moma_profile(h, 0)
            ys.append((y, n_tc))
        finally:
            m.moma_destroy(h)
    (yt, nt), (yc, nc) = ys
    assert nt == 2 and nc == 0
    scale = np.abs(ref).max()
    et, ec = np.abs(yt - ref).max() / scale, np.abs(yc - ref).max() / scale
    print(f"normal operator, max |y - oracle| / max |oracle|: tensor {et:.3g}, cuda cores {ec:.3g}")
    assert et <= 1e-4 and ec <= 1e-5
    assert relerr(yt, ref) <= 5e-5


def test_solve_takes_tensor_path_and_matches_dense(moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(4, 3, 128, 0.5, 1)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    angles = [(th, ph) for th in (0.0, 20.0, 40.0, 60.0) for ph in (0.0, 30.0, 60.0, 90.0)]
    V = excitation(spec, angles)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, MIXED)
    try:
        m.moma_set_blocks(h, blocks)
        m.moma_profile(h, 1)
        I = np.zeros_like(V)
        rr = np.zeros(len(angles))
        info = m.moma_solve(h, V, I, rel_residual=rr)
        n_tc = m.moma_kernel_stats(h, "bin_tc")[0]
        m.moma_profile(h, 0)
        za = np.zeros(V.shape[:3], np.complex128)
        m.moma_active_impedance(h, I, V, za)
    finally:
        m.moma_destroy(h)
    print("tensor-path solve:", info, "bin_tc launches", n_tc)
    assert n_tc > 0
    assert info["converged"] == 1 and rr.max() <= 1e-10
    z = dense.assemble(b128, spec.nx, spec.ny)
    i_ref = dense.solve(z, V)
    za_ref = ports.active_impedance(i_ref, V)
    # The Z_a bar is per port: the largest relative error over every port of every RHS.
    err = np.max(np.abs(za - za_ref) / np.abs(za_ref))
    print("tensor-path solve, max per-port Z_a rel err:", err)
    assert err <= 1e-8
    assert dense.relative_residual(z, I, V).max() <= 1e-10  # the oracle's own residual of the GPU currents


@pytest.mark.parametrize("nx,ny,b,nr", [(3, 2, 128, 20), (2, 2, 160, 33), (2, 1, 256, 16)])
def test_tensor_preconditioner_apply(moma_lib, cuda, nx, ny, b, nr):
    """y = P^{-1} x through X_e^H X_e on the tensor cores vs the oracle's
    direct block solve (Eq. 37 blocks, Cholesky)."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 3)
    blocks = offset_blocks(spec, np.complex64)
    x = rand_vec(nr, spec, seed=7)
    ref = mbt.precond_solve(mbt.precond_blocks(blocks.astype(np.complex128), nx, ny), x.astype(np.complex128))
    ys = {}
    for name, flags in (("tensor", m.MOMA_FLAG_TENSOR_ALWAYS), ("cuda", m.MOMA_FLAG_NO_TENSOR)):
        h = m.moma_create_array(nx, ny, b, MIXED, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            m.moma_profile(h, 1)
            y = np.zeros_like(x)
            m.moma_apply_precond(h, x, y)
            n_tc = m.moma_kernel_stats(h, "precond_tc")[0]
            m.moma_profile(h, 0)
        finally:
            m.moma_destroy(h)
        ys[name] = (y, n_tc)
    et, ec = relerr(ys["tensor"][0], ref), relerr(ys["cuda"][0], ref)
    print(f"precond {nx}x{ny}x{b} nr={nr}: tensor err {et:.3g}, cuda cores err {ec:.3g}")
    assert ys["tensor"][1] == 2 and ys["cuda"][1] == 0
    assert et <= 1e-4 and ec <= 1e-4


@pytest.mark.parametrize("prec,nr", [(MIXED, 16), (MIXED, 2), (0, 2)])
def test_wide_blocks_b256_solve_matches_dense(moma_lib, cuda, prec, nr):
    """b = 256 (preconditioner factors read from global memory): mixed with
    the tensor path (16 RHS), mixed on the CUDA cores (2 RHS), plain FP64."""
    m = moma_lib
    spec = LatticeSpec(3, 2, 256, 0.5, 5)
    blocks = offset_blocks(spec, np.complex64 if prec == MIXED else np.complex128)
    b128 = blocks.astype(np.complex128)
    angles = [(th, ph) for th in (0.0, 15.0, 30.0, 45.0) for ph in (0.0, 30.0, 60.0, 90.0)][:nr]
    V = excitation(spec, angles)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    try:
        m.moma_set_blocks(h, blocks)
        I = np.zeros_like(V)
        rr = np.zeros(nr)
        info = m.moma_solve(h, V, I, rel_residual=rr)
        za = np.zeros(V.shape[:3], np.complex128)
        m.moma_active_impedance(h, I, V, za)
    finally:
        m.moma_destroy(h)
    print(f"b=256 prec={prec} nr={nr}:", info)
    assert info["converged"] == 1 and rr.max() <= 1e-10
    z = dense.assemble(b128, spec.nx, spec.ny)
    i_ref = dense.solve(z, V)
    za_ref = ports.active_impedance(i_ref, V)
    assert np.max(np.abs(za - za_ref) / np.abs(za_ref)) <= 1e-8
    assert dense.relative_residual(z, I, V).max() <= 1e-10


@pytest.mark.parametrize("nx,ny,b", [(3, 2, 128), (2, 2, 160)])
def test_tensor_gram_preconditioner_blocks(moma_lib, cuda, nx, ny, b):
    """Set-up Gram products on the tensor cores (c64 blocks, mixed path):
    every P_e (Eq. 37) against the oracle's direct sum, and against the
    CUDA-core Gram products (MOMA_FLAG_NO_TENSOR).  3xTF32 products carry
    ~2e-6 relative error, so the bar is 2e-5 of the block's largest entry."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 8)
    blocks = offset_blocks(spec, np.complex64)
    P = mbt.precond_blocks(blocks.astype(np.complex128), nx, ny)
    got = {}
    for name, flags in (("tensor", 0), ("cuda", m.MOMA_FLAG_NO_TENSOR)):
        h = m.moma_create_array(nx, ny, b, MIXED, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            out = np.zeros((ny, nx, b, b), np.complex128)
            for ey in range(ny):
                for ex in range(nx):
                    blk = np.zeros((b, b), np.complex128)
                    m.moma_get_precond_block(h, ex, ey, blk)
                    out[ey, ex] = blk
            got[name] = out
        finally:
            m.moma_destroy(h)
    for name, out in got.items():
        err = max(np.abs(out[ey, ex] - P[ey, ex]).max() / np.abs(P[ey, ex]).max()
                  for ey in range(ny) for ex in range(nx))
        print(f"P_e {nx}x{ny}x{b} ({name} Gram): max rel err {err:.3g}")
        assert err <= 2e-5
    # Hermitian to the last bit is not required, but the factor must exist:
    # both arrays factorised (set_blocks raised no MOMA_ERR_NOT_PD).
