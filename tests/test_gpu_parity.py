"""GPU parity: every stage of the CUDA path against the CPU oracle, through
the C ABI, on seeded synthetic lattices (several tiles, ragged sizes, odd b,
degenerate 1x1 and single-row arrays, padded circulant sizes).

Tolerances: FP64 stages agree with the oracle to rounding (<= 1e-11
relative, FFT-based vs direct-sum evaluation order); c64 stages record their
raw error and must stay within FP32 rounding of well-conditioned data
(<= 1e-4); solves must reach relative residual <= 1e-10 and active
impedance within 1e-8 of the oracle.
"""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation, config_c1
from oracle import dense, mbt, ports

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
MIXED_F64R = 101  # a MIXED array with MOMA_FLAG_FP64_RESIDUAL (FP64 instead of double-FP32 residual stages)
RAW_ERRORS = {}


def smooth(n):
    m = max(n, 1)
    while True:
        k = m
        for r in (2, 3, 5):
            while k % r == 0:
                k //= r
        if k == 1:
            return m
        m += 1


def make(m, nx, ny, b, prec, d=0.5, seed=0, dtype=np.complex128, mx=0, my=0):
    spec = LatticeSpec(nx, ny, b, d, seed)
    blocks = offset_blocks(spec, dtype)
    if prec == MIXED_F64R:
        h = m.moma_create_array(nx, ny, b, MIXED, mx, my, flags=m.MOMA_FLAG_FP64_RESIDUAL)
    else:
        h = m.moma_create_array(nx, ny, b, prec, mx, my)
    m.moma_set_blocks(h, blocks)
    return spec, blocks.astype(np.complex128), h


def rand_vec(nr, spec, seed=1, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((nr, spec.ny, spec.nx, spec.b)) + 1j * rng.standard_normal((nr, spec.ny, spec.nx, spec.b))
    return v.astype(dtype)


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CASES = [(1, 1, 3), (2, 1, 1), (3, 2, 4), (4, 4, 32), (5, 3, 7), (7, 5, 6), (2, 6, 2), (6, 6, 33)]


@pytest.mark.parametrize("nx,ny,b", CASES)
def test_bins_match_circulant_definition(moma_lib, cuda, nx, ny, b):
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, MIXED)
    try:
        Mx, My = smooth(2 * nx - 1), smooth(2 * ny - 1)
        ref = mbt.circulant_bins(blocks, nx, ny, Mx, My)
        scale = np.abs(ref).max()
        out = np.zeros((b, b), np.complex128)
        out64 = np.zeros((b, b), np.complex64)
        worst64 = worst128 = 0.0
        for ky in range(My):
            for kx in range(Mx):
                m.moma_get_bin(h, kx, ky, out)
                assert np.abs(out - ref[ky, kx]).max() <= 1e-12 * scale
                worst128 = max(worst128, np.abs(out - ref[ky, kx]).max() / scale)
                m.moma_get_bin(h, kx, ky, out64)
                worst64 = max(worst64, np.abs(out64 - ref[ky, kx]).max() / scale)
        assert worst64 < 1e-6
        RAW_ERRORS[f"bins_c64 {nx}x{ny}x{b}"] = worst64
        RAW_ERRORS[f"bins_dfl {nx}x{ny}x{b}"] = worst128  # c128-class bins of a MIXED array (double-FP32)
    finally:
        m.moma_destroy(h)


def test_padded_circulant_sizes(moma_lib, cuda):
    """Any M >= 2N-1 embeds Z exactly (Eq. 3): a padded 3x4 lattice."""
    m = moma_lib
    spec, blocks, h = make(m, 3, 4, 5, FP64, mx=8, my=10)
    try:
        x = rand_vec(2, spec)
        y = np.zeros_like(x)
        m.moma_matvec(h, m.MOMA_OP_Z, x, y)
        assert relerr(y, mbt.matvec(blocks, 3, 4, x)) < 1e-12
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("nx,ny,b", CASES)
@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("prec", [MIXED, MIXED_F64R])
def test_matvec_fp64_and_c64(moma_lib, cuda, nx, ny, b, op, prec):
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, prec)
    try:
        x = rand_vec(3, spec)
        ref = mbt.matvec(blocks, nx, ny, x) if op == 0 else mbt.matvec_h(blocks, nx, ny, x)
        y = np.zeros_like(x)
        m.moma_matvec(h, op, x, y)
        assert relerr(y, ref) < 1e-12
        RAW_ERRORS[f"matvec{'H' if op else ''}_{'fp64' if prec == MIXED_F64R else 'dfl'} {nx}x{ny}x{b}"] = \
            relerr(y, ref)
        assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()
        x32 = x.astype(np.complex64)
        y32 = np.zeros_like(x32)
        m.moma_matvec(h, op, x32, y32)
        e = relerr(y32.astype(np.complex128), mbt.matvec(blocks, nx, ny, x32.astype(np.complex128)) if op == 0
                   else mbt.matvec_h(blocks, nx, ny, x32.astype(np.complex128)))
        RAW_ERRORS[f"matvec{'H' if op else ''}_c64 {nx}x{ny}x{b}"] = e
        assert e < 1e-5
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("nx,ny,b", [(1, 1, 3), (3, 2, 4), (4, 4, 32), (5, 3, 7), (6, 6, 33), (3, 1, 96), (2, 2, 128),
                                      (1, 2, 160), (1, 1, 256)])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_preconditioner_blocks_and_apply(moma_lib, cuda, nx, ny, b, prec):
    """Every P_e (Eq. 37) and the apply of P^{-1} against the oracle, for
    each launch shape of the block factorisation: the whole triangle in
    shared memory (b <= 33), four CTAs per SM with the first 24 / 48 / 80
    columns factored in global memory (b = 96, 128, 160), one CTA per SM
    (b = 256)."""
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, prec)
    try:
        P = mbt.precond_blocks(blocks, nx, ny)
        tol_blk = 1e-12 if prec == FP64 else 1e-5
        out = np.zeros((b, b), np.complex128)
        for ey in range(ny):
            for ex in range(nx):
                m.moma_get_precond_block(h, ex, ey, out)
                assert np.abs(out - P[ey, ex]).max() <= tol_blk * np.abs(P[ey, ex]).max()
        dt = np.complex128 if prec == FP64 else np.complex64
        x = rand_vec(2, spec, dtype=dt)
        y = np.zeros_like(x)
        m.moma_apply_precond(h, x, y)
        ref = mbt.precond_solve(P, x.astype(np.complex128))
        e = relerr(y.astype(np.complex128), ref)
        RAW_ERRORS[f"precond_{'c128' if prec == FP64 else 'c64'} {nx}x{ny}x{b}"] = e
        assert e < (1e-11 if prec == FP64 else 1e-5)
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("nx,ny,b", [(1, 1, 3), (3, 2, 4), (4, 4, 32), (7, 5, 6)])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_normal_operator(moma_lib, cuda, nx, ny, b, prec):
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, prec)
    try:
        dt = np.complex128 if prec == FP64 else np.complex64
        x = rand_vec(2, spec, dtype=dt)
        y = np.zeros_like(x)
        m.moma_matvec(h, m.MOMA_OP_NORMAL, x, y)
        ref = mbt.normal_operator(blocks, nx, ny, x.astype(np.complex128))
        e = relerr(y.astype(np.complex128), ref)
        RAW_ERRORS[f"normal_{'c128' if prec == FP64 else 'c64'} {nx}x{ny}x{b}"] = e
        assert e < (1e-11 if prec == FP64 else 1e-4)
    finally:
        m.moma_destroy(h)


def _check_solution(spec, blocks, V, I, za, gam, z0=50.0):
    z = dense.assemble(blocks, spec.nx, spec.ny)
    i_ref = dense.solve(z, V)
    rr = dense.relative_residual(z, I, V)
    assert rr.max() <= 1e-10, rr
    za_ref = ports.active_impedance(i_ref, V)
    assert np.max(np.abs(za - za_ref) / np.abs(za_ref)) <= 1e-8
    assert np.allclose(gam, ports.reflection(za_ref, z0), rtol=1e-8, atol=1e-10)


SOLVE_CASES = [(1, 1, 3, 0.5), (2, 1, 1, 0.5), (3, 2, 4, 0.3), (4, 4, 32, 0.5), (5, 3, 7, 0.7), (7, 5, 6, 0.5),
               (6, 6, 33, 0.4)]


@pytest.mark.parametrize("nx,ny,b,d", SOLVE_CASES)
@pytest.mark.parametrize("prec", [FP64, MIXED, MIXED_F64R])
def test_solve_matches_dense_lu(moma_lib, cuda, nx, ny, b, d, prec):
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, prec, d=d)
    try:
        V = excitation(spec, [(0, 0), (45, 0), (30, 60)])
        I = np.zeros_like(V)
        rr = np.zeros(V.shape[0])
        info = m.moma_solve(h, V, I, rel_residual=rr)
        assert info["converged"] == 1 and rr.max() <= 1e-10
        za = np.zeros(V.shape[:3], np.complex128)
        gam = np.zeros_like(za)
        m.moma_active_impedance(h, I, V, za, gam)
        _check_solution(spec, blocks, V, I, za, gam)
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_config_c1(moma_lib, cuda, prec):
    m = moma_lib
    spec, angles = config_c1()
    blocks = offset_blocks(spec)
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, prec)
    try:
        m.moma_set_blocks(h, blocks)
        V = excitation(spec, angles)
        I = np.zeros_like(V)
        info = m.moma_solve(h, V, I)
        za = np.zeros(V.shape[:3], np.complex128)
        gam = np.zeros_like(za)
        m.moma_active_impedance(h, I, V, za, gam)
        _check_solution(spec, blocks, V, I, za, gam)
        RAW_ERRORS[f"c1_first_inner_reduction prec={prec}"] = info["first_inner_reduction"]
    finally:
        m.moma_destroy(h)


def test_device_buffers_match_host_buffers(moma_lib, cuda):
    torch = cuda
    m = moma_lib
    spec = LatticeSpec(5, 4, 8, 0.5, 3)
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, [(0, 0), (20, 30)])
    h1 = m.moma_create_array(5, 4, 8, MIXED)
    h2 = m.moma_create_array(5, 4, 8, MIXED)
    try:
        m.moma_set_blocks(h1, blocks)
        m.moma_set_blocks(h2, torch.from_numpy(blocks).cuda())
        I1 = np.zeros_like(V)
        m.moma_solve(h1, V, I1)
        Vd = torch.from_numpy(V).cuda()
        Id = torch.zeros_like(Vd)
        m.moma_solve(h2, Vd, Id)
        assert np.array_equal(I1, Id.cpu().numpy())
    finally:
        m.moma_destroy(h1)
        m.moma_destroy(h2)


def test_warm_start_converges_immediately(moma_lib, cuda):
    m = moma_lib
    spec, blocks, h = make(m, 4, 3, 6, MIXED)
    try:
        V = excitation(spec, [(10, 10)])
        I = np.zeros_like(V)
        m.moma_solve(h, V, I)
        info = m.moma_solve(h, V, I, warm_start=True)
        assert info["outer_iters"] == 0 and info["converged"] == 1
    finally:
        m.moma_destroy(h)


def test_error_statuses(moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(3, 3, 4, 0.5, 0)
    h = m.moma_create_array(3, 3, 4, MIXED)
    try:
        V = excitation(spec, [(0, 0)])
        I = np.zeros_like(V)
        with pytest.raises(m.MomaError) as e:
            m.moma_solve(h, V, I)
        assert e.value.status == 2  # MOMA_ERR_STATE: no blocks yet
        bad = offset_blocks(spec)
        bad[3, 2, 0, 1] = np.nan  # a row the host ingest reads (dy >= 0)
        with pytest.raises(m.MomaError) as e:
            m.moma_set_blocks(h, bad)
        assert e.value.status == 8  # MOMA_ERR_NONFINITE
        m.moma_set_blocks(h, offset_blocks(spec))
        Vn = V.copy()
        Vn[0, 1, 1, 0] = np.inf
        with pytest.raises(m.MomaError) as e:
            m.moma_solve(h, Vn, I)
        assert e.value.status == 8
        za = np.zeros(V.shape[:3], np.complex128)
        with pytest.raises(m.MomaError) as e:
            m.moma_active_impedance(h, np.zeros_like(V), V, za)  # I_p = 0
        assert e.value.status == 8
        assert np.isnan(za).all()
    finally:
        m.moma_destroy(h)


def test_not_positive_definite_is_reported(moma_lib, cuda):
    """All-zero blocks make every P_e zero: the Cholesky pivot check fires."""
    m = moma_lib
    h = m.moma_create_array(2, 2, 3, FP64)
    try:
        with pytest.raises(m.MomaError) as e:
            m.moma_set_blocks(h, np.zeros((3, 3, 3, 3), np.complex128))
        assert e.value.status == 5
    finally:
        m.moma_destroy(h)


def test_zz_report_raw_errors():
    """Print the raw error of every reduced-precision stage seen above."""
    for k in sorted(RAW_ERRORS):
        print(f"RAW_ERROR {k}: {RAW_ERRORS[k]:.3e}")


def test_solves_are_deterministic(moma_lib, cuda):
    """Fixed reduction orders everywhere: fresh handles and repeated solves
    on one handle give bitwise identical currents (needed for the
    alone-versus-in-a-batch comparisons)."""
    m = moma_lib
    spec = LatticeSpec(6, 5, 10, 0.5, 4)
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, [(0, 0), (25, 40), (50, 10)])
    outs = []
    for _ in range(3):
        h = m.moma_create_array(spec.nx, spec.ny, spec.b, MIXED)
        try:
            m.moma_set_blocks(h, blocks)
            for _ in range(2):
                I = np.zeros_like(V)
                m.moma_solve(h, V, I)
                outs.append(I)
        finally:
            m.moma_destroy(h)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


PCG_CASES = [(1, 1, 3, 0.5), (2, 1, 1, 0.5), (3, 2, 4, 0.3), (4, 4, 32, 0.5), (5, 3, 7, 0.7), (6, 6, 33, 0.4)]


@pytest.mark.parametrize("nx,ny,b,d", PCG_CASES)
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_pcg_solve_matches_dense_lu(moma_lib, cuda, nx, ny, b, d, prec):
    """The paper's PCG form (Sec. II-C): CG on Z^H Z with preconditioner P,
    inside the same FP64 refinement, reaches the plain solution."""
    m = moma_lib
    spec, blocks, h = make(m, nx, ny, b, prec, d=d)
    try:
        V = excitation(spec, [(0, 0), (45, 0), (30, 60)])
        I = np.zeros_like(V)
        rr = np.zeros(V.shape[0])
        info = m.moma_solve(h, V, I, rel_residual=rr, solver=m.MOMA_SOLVER_PCG)
        assert info["converged"] == 1 and rr.max() <= 1e-10
        za = np.zeros(V.shape[:3], np.complex128)
        gam = np.zeros_like(za)
        m.moma_active_impedance(h, I, V, za, gam)
        _check_solution(spec, blocks, V, I, za, gam)
        RAW_ERRORS[f"pcg_first_inner_reduction {nx}x{ny}x{b} prec={prec}"] = info["first_inner_reduction"]
    finally:
        m.moma_destroy(h)


@pytest.mark.parametrize("nx,ny,b,prec", [(5, 4, 12, MIXED), (3, 1, 8, FP64), (4, 2, 6, MIXED), (6, 7, 5, FP64)])
def test_host_blocks_read_only_upper_rows(moma_lib, cuda, nx, ny, b, prec):
    """From host memory only the offsets with dy >= 0 are read; the rows
    dy < 0 are completed by reciprocity.  Overwriting them with unrelated
    finite values changes nothing, and host and device inputs agree."""
    m = moma_lib
    import torch
    spec = LatticeSpec(nx, ny, b, 0.5, 6)
    dt = np.complex128 if prec == FP64 else np.complex64
    blocks = offset_blocks(spec, dt)
    junk = blocks.copy()
    rng = np.random.default_rng(9)
    junk[:ny - 1] = (rng.standard_normal(junk[:ny - 1].shape) + 1j * rng.standard_normal(junk[:ny - 1].shape)).astype(dt)
    V = excitation(spec, [(0.0, 0.0), (30.0, 20.0)])
    out = []
    for src in (blocks, junk, torch.from_numpy(blocks).cuda()):
        h = m.moma_create_array(nx, ny, b, prec)
        try:
            m.moma_set_blocks(h, src)
            I = np.zeros_like(V)
            m.moma_solve(h, V, I)
            out.append(I)
        finally:
            m.moma_destroy(h)
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0], out[2])


@pytest.mark.parametrize("nx,ny,b,nr", [(1, 1, 16, 1), (2, 1, 18, 2), (5, 3, 32, 3), (7, 5, 24, 2), (6, 6, 48, 5),
                                         (16, 12, 32, 2), (40, 40, 16, 3), (4, 3, 128, 2), (3, 3, 160, 15)])
def test_fused_transforms_and_streaming_preconditioner(moma_lib, cuda, nx, ny, b, nr):
    """The 2D lattice transforms (one launch per transform) and the
    streaming preconditioner apply against the per-axis passes and the
    per-element apply (MOMA_FLAG_AXIS_FFT | MOMA_FLAG_PRECOND_PER_ELEMENT),
    and both against the oracle: Z x, Z^H x, P^{-1} x and P^{-1} Z^H Z x
    (Sec. III-A), c64, element by element.  (40, 40, 16) has 1600 elements,
    so every persistent CTA of the streaming apply wraps its copy ring."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 6)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec, seed=9, dtype=np.complex64)
    xo = x.astype(np.complex128)
    p = mbt.precond_blocks(b128, nx, ny)
    ref = {"z": mbt.matvec(b128, nx, ny, xo), "zh": mbt.matvec_h(b128, nx, ny, xo),
           "p": mbt.precond_solve(p, xo), "n": mbt.normal_operator(b128, nx, ny, xo, p)}
    out = {}
    for name, flags in (("fused", m.MOMA_FLAG_NO_TENSOR),
                        ("split", m.MOMA_FLAG_NO_TENSOR | m.MOMA_FLAG_AXIS_FFT | m.MOMA_FLAG_PRECOND_PER_ELEMENT)):
        h = m.moma_create_array(nx, ny, b, MIXED, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            res = {}
            for key, fn in (("z", lambda y: m.moma_matvec(h, 0, x, y)), ("zh", lambda y: m.moma_matvec(h, 1, x, y)),
                            ("p", lambda y: m.moma_apply_precond(h, x, y)),
                            ("n", lambda y: m.moma_matvec(h, 2, x, y))):
                y = np.full_like(x, np.nan)
                fn(y)
                res[key] = y.astype(np.complex128)
            out[name] = res
        finally:
            m.moma_destroy(h)
    for key in ("z", "zh", "p", "n"):
        scale = np.abs(ref[key]).max()
        ef = np.abs(out["fused"][key] - ref[key]).max() / scale
        es = np.abs(out["split"][key] - ref[key]).max() / scale
        RAW_ERRORS[f"fused_{key} {nx}x{ny}x{b} nr={nr}"] = ef
        print(f"{key} {nx}x{ny}x{b} nr={nr}: fused {ef:.3g}, per-axis/per-element {es:.3g}")
        assert np.all(np.isfinite(out["fused"][key]))
        assert ef <= 1e-5 and es <= 1e-5


@pytest.mark.parametrize("nx,ny,b,nr", [(3, 2, 64, 1), (2, 3, 96, 2), (4, 3, 128, 3), (3, 3, 160, 5), (2, 2, 192, 4),
                                         (2, 3, 224, 2), (2, 2, 256, 6), (1, 1, 128, 2)])
@pytest.mark.parametrize("op", [0, 1])
def test_row_column_warp_bin_product(moma_lib, cuda, nx, ny, b, nr, op):
    """The c64 per-bin product for b a multiple of 32 (row warps for the
    Zhat x leg, column warps for the Zhat^T x leg, Eqs. 3 and 6): Z x and
    Z^H x on the CUDA cores, element by element against the oracle's direct
    offset sums, for every column-group / row-slice split (b = 64 .. 256)
    and RHS chunks of 1, 2 and 4 with a ragged tail."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 11)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec, seed=4, dtype=np.complex64)
    ref = (mbt.matvec if op == 0 else mbt.matvec_h)(b128, nx, ny, x.astype(np.complex128))
    h = m.moma_create_array(nx, ny, b, MIXED, flags=m.MOMA_FLAG_NO_TENSOR)
    try:
        m.moma_set_blocks(h, blocks)
        y = np.full_like(x, np.nan)
        m.moma_matvec(h, op, x, y)
    finally:
        m.moma_destroy(h)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    RAW_ERRORS[f"rc_bin{'H' if op else ''} {nx}x{ny}x{b} nr={nr}"] = err
    assert np.all(np.isfinite(y)) and err <= 1e-5, err


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,b,nr", [(32, 3, 8, 1), (24, 20, 4, 2), (16, 30, 6, 1), (10, 32, 5, 3)])
def test_split_lattice_transforms(moma_lib, cuda, nx, ny, b, nr):
    """Lattice axes whose circulant length takes the split register
    transform (2 or 4 lanes per line: M = 64, 48 and 32 -> 4 lanes, 60, 40
    and 20 -> 2 at these line counts) beside an axis on one thread per line
    (M = 5): Z x, Z^H x and P^{-1} Z^H Z x (Eq. 3, Eq. 6, Sec. III-A; the
    last includes the inverse / lattice mask / forward pass) element by
    element against the oracle's direct offset sums, c64.  Eight lanes per
    line (never chosen by the rule) are checked on the host."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 12)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec, seed=21, dtype=np.complex64)
    xo = x.astype(np.complex128)
    p = mbt.precond_blocks(b128, nx, ny)
    ref = {0: mbt.matvec(b128, nx, ny, xo), 1: mbt.matvec_h(b128, nx, ny, xo),
           2: mbt.normal_operator(b128, nx, ny, xo, p)}
    h = m.moma_create_array(nx, ny, b, MIXED, flags=m.MOMA_FLAG_NO_TENSOR)
    try:
        m.moma_set_blocks(h, blocks)
        for op in (0, 1, 2):
            y = np.full_like(x, np.nan)
            m.moma_matvec(h, op, x, y)
            err = np.abs(y - ref[op]).max() / np.abs(ref[op]).max()
            RAW_ERRORS[f"split_fft op{op} {nx}x{ny}x{b} nr={nr}"] = err
            assert np.all(np.isfinite(y)) and err <= 1e-5, (op, err)
    finally:
        m.moma_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,b,nr,M", [(3, 3, 24, 1, 64), (32, 32, 8, 2, 0), (5, 4, 20, 3, 48), (4, 4, 12, 2, 32),
                                           (3, 3, 128, 4, 64), (24, 24, 8, 1, 0)])
def test_cluster_lattice_transforms(moma_lib, cuda, nx, ny, b, nr, M):
    """The c64 2D lattice transforms on thread-block clusters (F2, I2 and the
    inverse / mask / forward pass between the Z and Z^H legs, Eq. 2, Eq. 3,
    Sec. III-A) on square circulants M = 64, 48, 32: Z x, Z^H x and
    P^{-1} Z^H Z x bitwise equal to the per-axis passes (MOMA_FLAG_AXIS_FFT:
    the same line transforms, handed over through L2 between launches) and
    element by element against the oracle's direct offset sums.  b = 20 and
    12 leave the last group of eight basis indices ragged; four RHS at
    b = 128 take two lanes per y line."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 14)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec, seed=23, dtype=np.complex64)
    xo = x.astype(np.complex128)
    p = mbt.precond_blocks(b128, nx, ny)
    ref = {0: mbt.matvec(b128, nx, ny, xo), 1: mbt.matvec_h(b128, nx, ny, xo),
           2: mbt.normal_operator(b128, nx, ny, xo, p)}
    out = {}
    for name, flags in (("cluster", m.MOMA_FLAG_NO_TENSOR), ("axis", m.MOMA_FLAG_NO_TENSOR | m.MOMA_FLAG_AXIS_FFT)):
        h = m.moma_create_array(nx, ny, b, MIXED, mx=M, my=M, flags=flags)
        try:
            m.moma_set_blocks(h, blocks)
            m.moma_profile(h, 1)
            for op in (0, 1, 2):
                n0 = m.moma_kernel_stats(h, "fft_c64")[0]
                y = np.full_like(x, np.nan)
                m.moma_matvec(h, op, x, y)
                out[name, op] = y
                # Lattice-transform launches of the c64 product: one per 2D
                # transform on the clusters, one per axis pass otherwise.
                nt = m.moma_kernel_stats(h, "fft_c64")[0] - n0
                assert nt == {"cluster": (2, 2, 3), "axis": (4, 4, 7)}[name][op], (name, op, nt)
        finally:
            m.moma_destroy(h)
    for op in (0, 1, 2):
        y = out["cluster", op]
        err = np.abs(y - ref[op]).max() / np.abs(ref[op]).max()
        RAW_ERRORS[f"cluster_fft op{op} {nx}x{ny}x{b} M={M} nr={nr}"] = err
        assert np.all(np.isfinite(y)) and err <= 1e-5, (op, err)
        assert np.array_equal(y, out["axis", op]), op


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,b,nr", [(3, 2, 64, 1), (2, 3, 96, 3), (4, 3, 128, 2), (2, 2, 160, 5),
                                         (2, 2, 192, 3), (1, 2, 224, 1), (2, 1, 256, 2)])
@pytest.mark.parametrize("op", [0, 1])
def test_double_fp32_row_column_bin_product(moma_lib, cuda, nx, ny, b, nr, op):
    """The double-FP32 per-bin product of the refinement residual (Eq. 3,
    the row/column-warp layout: 32-row tiles for b = 64 .. 160, 16-row tiles
    above; two RHS per launch with a ragged last one): Z x and Z^H x of c128
    vectors on a MIXED array,
    element by element against the oracle's FP64 direct offset sums at the
    FP64-class bar of the residual path."""
    m = moma_lib
    spec = LatticeSpec(nx, ny, b, 0.5, 13)
    blocks = offset_blocks(spec, np.complex64)
    b128 = blocks.astype(np.complex128)
    x = rand_vec(nr, spec, seed=5)
    ref = (mbt.matvec if op == 0 else mbt.matvec_h)(b128, nx, ny, x)
    h = m.moma_create_array(nx, ny, b, MIXED, flags=m.MOMA_FLAG_NO_TENSOR)
    try:
        m.moma_set_blocks(h, blocks)
        y = np.full_like(x, np.nan)
        m.moma_matvec(h, op, x, y)
    finally:
        m.moma_destroy(h)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    RAW_ERRORS[f"dfl_rc_bin{'H' if op else ''} {nx}x{ny}x{b} nr={nr}"] = err
    assert np.all(np.isfinite(y)) and err <= 1e-11, err
