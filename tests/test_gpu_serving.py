"""Serving loop: continuous batching of solve requests.  Each result must be
the same alone (one slot, one request at a time) and in the mix (several
slots, all requests queued at once, a memory budget that forces evictions
and re-builds), and must match the dense oracle."""
import numpy as np
import pytest

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense, ports

pytestmark = pytest.mark.gpu

PROBLEMS = [(4, 4, 16, 0.5, 1), (5, 3, 8, 0.3, 2), (6, 6, 12, 0.7, 3), (3, 7, 10, 0.45, 4), (8, 5, 8, 0.5, 5),
            (2, 2, 20, 0.6, 6)]


def _requests():
    rng = np.random.default_rng(7)
    specs = [LatticeSpec(*p) for p in PROBLEMS]
    blocks = [offset_blocks(s, np.complex64) for s in specs]
    reqs = []
    for t in range(16):
        k = int(rng.integers(len(specs)))
        nr = int(rng.integers(1, 5))
        angles = [(float(rng.uniform(0, 60)), float(rng.uniform(0, 90))) for _ in range(nr)]
        reqs.append((k, excitation(specs[k], angles)))
    return specs, blocks, reqs


def _run(m, specs, blocks, reqs, slots, budget, all_at_once):
    s = m.moma_server_create(slots=slots, max_device_bytes=budget)
    outs = [None] * len(reqs)
    results = [None] * len(reqs)
    try:
        bufs = []
        tickets = []
        for i, (k, V) in enumerate(reqs):
            I = np.zeros_like(V)
            za = np.zeros(V.shape[:3], np.complex128)
            bufs.append((V, I, za))
            t = m.moma_server_submit(s, k + 1, blocks[k], V, I, Za=za)
            if all_at_once:
                tickets.append((i, t))
            else:
                results[i] = m.moma_server_wait(s, t, 120.0)
        for i, t in tickets:
            results[i] = m.moma_server_wait(s, t, 120.0)
        stats = m.moma_server_get_stats(s)
    finally:
        m.moma_server_destroy(s)
    for i, (V, I, za) in enumerate(bufs):
        outs[i] = (I, za)
    return outs, results, stats


def test_alone_equals_mix_and_oracle(moma_lib, cuda):
    m = moma_lib
    specs, blocks, reqs = _requests()
    alone, r_alone, st_alone = _run(m, specs, blocks, reqs, 1, 0, False)
    # A budget barely above one array's set-up footprint: a miss must evict
    # idle arrays, so arrays are rebuilt and results must not depend on it.
    budget = int(1.2 * max(m.moma_estimate_bytes(s.nx, s.ny, s.b, 4) for s in specs))
    mix, r_mix, st_mix = _run(m, specs, blocks, reqs, 4, budget, True)
    assert all(r["status"] == 0 for r in r_alone + r_mix), [r["message"] for r in r_alone + r_mix]
    for (ia, za_a), (im, za_m) in zip(alone, mix):
        assert np.array_equal(ia, im)
        assert np.array_equal(za_a, za_m)
    print("serving stats: alone", st_alone, "mix", st_mix)
    assert st_mix["completed"] == len(reqs) and st_alone["hits"] > 0
    assert st_mix["evictions"] > 0 and st_mix["resident_bytes"] <= budget
    for (k, V), (I, za) in zip(reqs, alone):
        z = dense.assemble(blocks[k].astype(np.complex128), specs[k].nx, specs[k].ny)
        assert dense.relative_residual(z, I, V).max() <= 1e-10
        za_ref = ports.active_impedance(dense.solve(z, V), V)
        assert np.max(np.abs(za - za_ref) / np.abs(za_ref)) <= 1e-8


def test_server_reports_per_request_errors(moma_lib, cuda):
    m = moma_lib
    spec = LatticeSpec(3, 3, 4, 0.5, 0)
    bad = offset_blocks(spec, np.complex64)
    bad[-1, 0, 0, 0] = np.nan  # a row the host ingest reads (dy >= 0)
    V = excitation(spec, [(0, 0)])
    I = np.zeros_like(V)
    s = m.moma_server_create(slots=2)
    try:
        t = m.moma_server_submit(s, 99, bad, V, I)
        r = m.moma_server_wait(s, t, 60.0)
        assert r["status"] == 8 and "non-finite" in r["message"]
        good = offset_blocks(spec, np.complex64)
        t = m.moma_server_submit(s, 100, good, V, I)
        assert m.moma_server_wait(s, t, 60.0)["status"] == 0
    finally:
        m.moma_server_destroy(s)


def test_alone_equals_mix_at_b128_with_tensor_core_requests(moma_lib, cuda):
    """Requests shaped like the serving workload (b = 128, 16-32 scan RHS,
    which take the tensor-core product and preconditioner, plus a few small
    ones on the CUDA cores), admitted concurrently: every result is bitwise
    the stand-alone one and matches the dense oracle per port."""
    m = moma_lib
    specs = [LatticeSpec(5, 4, 128, 0.45, 0), LatticeSpec(6, 3, 128, 0.62, 0), LatticeSpec(4, 4, 128, 0.33, 0)]
    blocks = [offset_blocks(s, np.complex64) for s in specs]
    rng = np.random.default_rng(17)
    reqs = []
    for i in range(7):
        k = i % len(specs)
        nr = int(rng.integers(16, 33)) if i < 5 else int(rng.integers(1, 4))
        angles = [(float(rng.uniform(0, 60)), float(rng.uniform(0, 90))) for _ in range(nr)]
        reqs.append((k, excitation(specs[k], angles)))
    alone, r_alone, _ = _run(m, specs, blocks, reqs, 1, 0, False)
    mix, r_mix, st_mix = _run(m, specs, blocks, reqs, 4, 0, True)
    assert all(r["status"] == 0 for r in r_alone + r_mix), [r["message"] for r in r_alone + r_mix]
    assert st_mix["completed"] == len(reqs)
    for (ia, za_a), (im, za_m) in zip(alone, mix):
        assert np.array_equal(ia, im) and np.array_equal(za_a, za_m)
    for (k, V), (I, za) in zip(reqs, alone):
        z = dense.assemble(blocks[k].astype(np.complex128), specs[k].nx, specs[k].ny)
        assert dense.relative_residual(z, I, V).max() <= 1e-10
        za_ref = ports.active_impedance(dense.solve(z, V), V)
        err = np.max(np.abs(za - za_ref) / np.abs(za_ref))
        print(f"b=128 request {specs[k].nx}x{specs[k].ny}, {V.shape[0]} RHS: max per-port Z_a rel err {err:.3g}")
        assert err <= 1e-8
