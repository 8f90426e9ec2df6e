"""Input generator: stream definition, determinism and the structure the
paper's matrices have (reciprocity, Sec. II-D)."""
import os

import numpy as np

from synth import SplitMix64, splitmix64_stream, LatticeSpec, offset_blocks, excitation, element_geometry
from synth.lattice import SELF_LOAD

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bigint_splitmix(seed, n):
    m = (1 << 64) - 1
    out, s = [], seed
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & m
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_values():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = splitmix64_stream(0, len(vals))
    assert [int(v) for v in got] == vals


def test_splitmix64_matches_bigint_and_offsets():
    for seed in (0, 7, 123456789, 2**63 + 5):
        ref = _bigint_splitmix(seed, 50)
        assert [int(v) for v in splitmix64_stream(seed, 50)] == ref
        assert [int(v) for v in splitmix64_stream(seed, 10, start=20)] == ref[20:30]
    g = SplitMix64(3)
    a = g.next_u64(5)
    b = g.next_u64(5)
    assert [int(v) for v in np.concatenate([a, b])] == _bigint_splitmix(3, 10)


def test_uniform_range():
    u = SplitMix64(1).uniform(10000, 0.5, 1.0)
    assert u.min() >= 0.5 and u.max() < 1.0
    assert abs(u.mean() - 0.75) < 0.01


def test_blocks_reciprocal_and_loaded():
    spec = LatticeSpec(3, 2, 5, 0.4, 11)
    z = offset_blocks(spec)
    nx, ny = spec.nx, spec.ny
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            a = z[dy + ny - 1, dx + nx - 1]
            bm = z[-dy + ny - 1, -dx + nx - 1]
            assert np.array_equal(a, bm.T)
    # self terms: r is floored at a = 0.01 and cos(0) = 1, plus the loading
    _, w, _ = element_geometry(5, 0.4, 11)
    k, a = 2 * np.pi, 0.01
    diag = w * w * np.exp(-1j * k * a) / (4 * np.pi * a) + SELF_LOAD
    assert np.allclose(np.diag(z[ny - 1, nx - 1]), diag, rtol=1e-14, atol=0)


def test_c64_rounding_is_single_rounding():
    spec = LatticeSpec(2, 2, 4, 0.5, 0)
    assert np.array_equal(offset_blocks(spec, np.complex64), offset_blocks(spec).astype(np.complex64))


def test_excitation_layout():
    spec = LatticeSpec(4, 3, 6, 0.5, 0)
    v = excitation(spec, [(0.0, 0.0), (30.0, 0.0)], port_basis=2)
    assert v.shape == (2, 3, 4, 6)
    assert np.all(v[0, :, :, 2] == 1.0)
    assert np.count_nonzero(v[:, :, :, [0, 1, 3, 4, 5]]) == 0
    ph = np.angle(v[1, 0, 1, 2] / v[1, 0, 0, 2])
    assert np.isclose(ph, -2 * np.pi * 0.5 * np.sin(np.pi / 6))


def test_torch_generator_matches_numpy():
    import torch
    from synth import offset_blocks_torch
    spec = LatticeSpec(4, 3, 7, 0.37, 5)
    a = offset_blocks(spec)
    t = offset_blocks_torch(spec, "cpu", torch.complex128).numpy()
    assert np.allclose(t, a, rtol=1e-13, atol=1e-15)
    c64 = offset_blocks_torch(spec, "cpu").numpy()
    assert c64.dtype == np.complex64 and np.allclose(c64, a, rtol=1e-6, atol=0)
