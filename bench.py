"""Benchmark: solves/s of the MBT array solver on one B300 (or N replicas).

Workload: the 32 x 32 lattice, b = 128 basis functions per element
(N = 131072 unknowns), offset blocks stored complex64, two right-hand sides
(broadside and a 45 degree E-plane scan), restarted GMRES(50) on the
preconditioned normal equations with FP64 refinement to a relative residual
of 1e-10.  One step = the whole hot path on one problem: block ingest, the
block-bin transform, preconditioner build and factorisation, the solve and
the port quantities.  value = right-hand sides solved per second (solves/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the problem (the work
shards by independent problems; no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at rel. Z_a err <=1e-8 vs plain FP64 GPU solve; p50/p99 latency; HBM GB/s"
WORKLOAD = ("32x32 lattice, b=128 (N=131072), offset blocks complex64, 2 RHS (broadside, 45deg E-plane), "
            "preconditioned GMRES(50) + FP64 refinement to rel. residual 1e-10")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-lanes", type=int, default=4,
                    help="array handles (each on its own stream and host thread) of the end-to-end leg")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="timed steps of the plain FP64 solve and of the FP64-residual variant "
                         "(-1 = same as --steps, 0 = skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg (cpu_baseline)")
    ap.add_argument("--ref-seconds", type=float, default=200.0,
                    help="reference arm: wall-time budget for whole oracle solves (at least one step runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="headline workload only (no scan / ragged / serving sub-measurements)")
    ap.add_argument("--ragged", action="store_true",
                    help="ragged batch: 24 square lattices 2x2..48x48, b=96, x 3 spacings, one broadside solve each")
    ap.add_argument("--scan", action="store_true",
                    help="scan workload: 24x24, b=256, 64 scan-angle RHS at spacings 0.3/0.5/0.7 (tensor cores)")
    ap.add_argument("--predictors", action="store_true",
                    help="all-port Z_p (16x16, b=128) + xi_Z, column coupling (32x32, b=128, 64 phase samples), xi_S")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: Poisson request stream through the continuous-batching server")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-keys", type=int, default=0,
                    help="0: every request draws its own lattice and spacing; K > 0: K resident lattice keys")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--nrhs", type=int, default=0,
                    help="profiling: this many scan-angle RHS instead of the workload's two")
    ap.add_argument("--lattice", type=int, nargs=3, metavar=("NX", "NY", "B"), default=None,
                    help="override the lattice (profiling of smaller cases; not the benchmark workload)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)
        self.lines.clear()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(lattice=None, nrhs=0):
    from synth import config_c2, offset_blocks, excitation, LatticeSpec, config_c3_angles
    spec, angles = config_c2()
    if lattice:
        spec = LatticeSpec(lattice[0], lattice[1], lattice[2], spec.d, spec.seed)
    if nrhs:
        angles = (config_c3_angles() * (nrhs // 64 + 1))[:nrhs]
    blocks = offset_blocks(spec, np.complex64)
    V = excitation(spec, angles)
    return spec, blocks, V


def smooth235(n):
    """Smallest 2^a 3^b 5^c >= n (the library's default circulant size)."""
    m = max(1, n)
    while True:
        k = m
        for r in (2, 3, 5):
            while k % r == 0:
                k //= r
        if k == 1:
            return m
        m += 1


def pair_count(mx, my):
    """Number of {k, -k} classes of the Mx x My circulant frequencies (one
    stored b x b block per class)."""
    return sum(1 for ky in range(my) for kx in range(mx)
               if ky * mx + kx <= ((my - ky) % my) * mx + ((mx - kx) % mx))


def bin_product_bytes(spec, nr, padded=False):
    """Bytes of one c64 bin-product launch: the transformed blocks once (one
    b x b block per {k,-k} pair) plus the bin vectors in and out.

    padded=False: the algorithmic count, on the paper's circulant size
    M = 2N - 1 per axis (Sec. II-A), whatever size the library pads to.
    padded=True: the bytes the kernel really streams, on the library's
    padded sizes (smallest 2^a 3^b 5^c >= 2N - 1) and rows of even length."""
    if padded:
        mx, my = smooth235(2 * spec.nx - 1), smooth235(2 * spec.ny - 1)
        ldb = spec.b + (spec.b % 2)
    else:
        mx, my = 2 * spec.nx - 1, 2 * spec.ny - 1
        ldb = spec.b
    B = mx * my
    pairs = pair_count(mx, my)
    return pairs * spec.b * ldb * 8 + 2 * B * nr * spec.b * 8, pairs, B


def matvec_bytes(spec, nr):
    """Algorithmic bytes of one Z application, c64 (the MLFFT product of
    Eq. 3): the transformed blocks once (pair storage on M = 2N - 1), the bin
    vectors in and out of the per-bin product, and the lattice vector in and
    out."""
    alg_bin, _, _ = bin_product_bytes(spec, nr, padded=False)
    return alg_bin + 2 * spec.nx * spec.ny * spec.b * nr * 8


def measured_traffic(alg_bytes_padded, spec, nr):
    """DRAM bytes per launch of the c64 bin product from the committed ncu
    capture (profiles/bin_pair_kernel_c64_traffic.txt), scaled from the
    captured lattice to this launch by the streamed (padded) bytes; None if
    the kernel source the record names changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "bin_pair_kernel_c64_traffic.txt")
    try:
        kv = dict(l.strip().split("=", 1) for l in open(path) if "=" in l and not l.startswith("#"))
        src = os.path.join(ROOT, kv.get("kernel_source", "paper_2608_17844_b300/csrc/binprod.cu"))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if kv.get("kernel_source_sha256") != sha:
        return None
    pairs, bins, nrc, b = (int(kv[k]) for k in ("pairs", "bins", "nrhs", "b"))
    alg_captured = pairs * b * (b + b % 2) * 8 + 2 * bins * nrc * b * 8
    measured = int(kv["dram_read_bytes"]) + int(kv["dram_write_bytes"])
    return measured / alg_captured * alg_bytes_padded


def named_elements(nx, ny):
    """(mx, my) of the centre (floor(Nx/2), floor(Ny/2)), edge (0, floor(Ny/2))
    and corner (0, 0) elements."""
    return {"centre": (nx // 2, ny // 2), "edge": (0, ny // 2), "corner": (0, 0)}


def oracle_solves(spec, blocks, V, qs):
    """The CPU oracle (oracle-I: restarted GMRES on Z I = V with the direct
    offset-sum product and block Jacobi, complex128) run to a relative
    residual of 1e-10 on the RHS columns qs, one complete solve each.
    Returns (seconds per solve, currents [len(qs)][Ny][Nx][b], iterations,
    residuals)."""
    from oracle import iterative
    b128 = blocks.astype(np.complex128)
    secs, cur, its, res = [], [], [], []
    for q in qs:
        t0 = time.perf_counter()
        I, info = iterative.gmres(b128, spec.nx, spec.ny, V[q:q + 1], tol=1e-10, restart=60, max_iter=500)
        secs.append(time.perf_counter() - t0)
        cur.append(I[0])
        its.append(info[0]["iters"])
        res.append(info[0]["rel_residual"])
    return secs, np.array(cur), its, res


def cpu_baseline_leg(spec, blocks, V, I_gpu):
    """cpu_baseline: one complete oracle solve (RHS 0 of the workload),
    timed on the host cores.  The same leg certifies the GPU result it is
    handed: the oracle's Z_a against the GPU's for RHS 0 (every port), and
    the GPU currents' residual recomputed by the oracle's FP64 direct
    offset sum for every RHS."""
    from oracle import mbt
    cores = len(os.sched_getaffinity(0))
    secs, I0, its, res = oracle_solves(spec, blocks, V, [0])
    b128 = blocks.astype(np.complex128)
    za_o = V[0, ..., 0] / I0[0, ..., 0]
    za_g = V[0, ..., 0] / I_gpu[0, ..., 0]
    za_err = float(np.max(np.abs(za_g - za_o) / np.abs(za_o)))
    cert = []
    for q in range(V.shape[0]):
        r = V[q] - mbt.matvec(b128, spec.nx, spec.ny, I_gpu[q:q + 1])[0]
        cert.append(float(np.linalg.norm(r) / np.linalg.norm(V[q])))
    return {"value": 1.0 / secs[0], "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle-I (complex128 GMRES(60), direct offset-sum product, block Jacobi) on RHS 0 of the "
                       f"same {spec.nx}x{spec.ny} b={spec.b} problem, run to convergence: {its[0]} iterations, "
                       f"{secs[0]:.1f} s, final residual {res[0]:.2e} (converged)"),
            "seconds": secs[0], "iterations": its[0], "oracle_rel_residual": res[0],
            "certify_gpu": {"za_rel_err_rhs0_all_ports": za_err, "za_bar": 1e-8,
                            "direct_sum_rel_residual": cert, "residual_bar": 1e-10}}


def serve_requests(rate, seconds, keys, seed=7):
    """Request stream of the serving workload: Poisson arrivals at `rate`
    per second for `seconds`.  Per request, in this order: inter-arrival
    time, Nx ~ U{4..40}, Ny ~ U{4..40}, spacing d ~ U(0.3, 0.7) wavelengths
    (keys = 0) or one of `keys` resident lattices with d on the 5-point grid
    0.3..0.7 (keys > 0), nrhs ~ U{1..32}, then nrhs scan angles
    (theta ~ U[0, 60], phi ~ U[0, 90) degrees).  b = 128, block seed 0."""
    from synth import LatticeSpec
    rng = np.random.default_rng(seed)
    pool = []
    for _ in range(keys):
        nx, ny = int(rng.integers(4, 41)), int(rng.integers(4, 41))
        pool.append(LatticeSpec(nx, ny, 128, float(rng.choice([0.3, 0.4, 0.5, 0.6, 0.7])), 0))
    reqs, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= seconds:
            break
        if keys:
            k = int(rng.integers(len(pool)))
            spec = pool[k]
        else:
            nx, ny = int(rng.integers(4, 41)), int(rng.integers(4, 41))
            d = float(rng.uniform(0.3, 0.7))
            spec, k = LatticeSpec(nx, ny, 128, d, 0), len(reqs)
        nr = int(rng.integers(1, 33))
        angles = [(float(rng.uniform(0, 60)), float(rng.uniform(0, 90))) for _ in range(nr)]
        reqs.append((t, k, spec, angles))
    return reqs


def serve_stream(rate, seconds, keys, slots):
    """One serving run: the request blocks (c64, generated on the GPU before
    the clock starts; each request of the continuous draw has its own
    lattice and spacing, hence its own blocks) are submitted at their
    arrival times to the continuous-batching server; each request's latency
    is submit -> result.  Returns a dict of the run's figures."""
    import torch
    import paper_2608_17844_b300 as m
    from synth import offset_blocks_torch, excitation
    torch.cuda.set_device(0)
    reqs = serve_requests(rate, seconds, keys)
    blocks, seen = {}, {}
    for (_, k, spec, _) in reqs:
        if k not in blocks:
            blocks[k] = offset_blocks_torch(spec, "cuda")
    torch.cuda.synchronize()
    gen_bytes = sum(b.numel() * 8 for b in blocks.values())
    s = m.moma_server_create(slots=slots)
    outstanding, lat, qms, hits, solved, errors = [], [], [], 0, 0, 0
    t0 = time.perf_counter()

    def collect(block):
        nonlocal hits, solved, errors
        while outstanding and (block or outstanding[0][0] is None):
            tk, bufs = outstanding.pop(0)
            r = m.moma_server_wait(s, tk, -1.0)
            lat.append(r["total_ms"])
            qms.append(r["queue_ms"])
            hits += r["resident_hit"]
            if r["status"] == 0:
                solved += bufs[0].shape[0]
            else:
                errors += 1

    for (ta, k, spec, angles) in reqs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        V = excitation(spec, angles)
        I = np.zeros_like(V)
        tk = m.moma_server_submit(s, k + 1, blocks[k], V, I)
        outstanding.append((tk, (V, I)))
    collect(True)
    wall = time.perf_counter() - t0
    stats = m.moma_server_get_stats(s)
    m.moma_server_destroy(s)
    del blocks
    torch.cuda.empty_cache()
    lat = np.array(lat)
    n_rhs = sum(len(r[3]) for r in reqs)
    return {"offered_req_per_s": len(reqs) / seconds, "requests": len(reqs), "rhs": n_rhs,
            "completed_req_per_s": len(reqs) / wall, "solves_per_s": solved / wall, "wall_s": wall,
            "errors": errors, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(qms, 50)), "resident_hit_rate": hits / len(reqs),
            "slots": slots, "request_blocks_gb": gen_bytes / 1e9, "server": stats}


def run_serving(args, sub=False):
    """Serving workload: Poisson arrivals (seed 7) of requests with
    Nx, Ny ~ U{4..40}, b = 128, spacing d ~ U(0.3, 0.7), 1-32 scan-angle
    RHS, through the continuous-batching server (HBM-footprint admission,
    resident arrays, LRU eviction).  Reported at the offered rate (200/s
    default) and below saturation; plus the residency variant (d on a
    5-point grid, a few lattice keys, so arrays are served resident)."""
    runs = {}
    if sub:
        plan = [("continuous_200", args.serve_rate, 1.5, 0), ("continuous_below_saturation", 15.0, 4.0, 0),
                ("resident_keys_200", args.serve_rate, 1.5, 8)]
    else:
        plan = [(f"{'keys%d' % args.serve_keys if args.serve_keys else 'continuous'}_{args.serve_rate:g}",
                 args.serve_rate, args.serve_seconds, args.serve_keys)]
    for name, rate, secs, keys in plan:
        runs[name] = serve_stream(rate, secs, keys, args.serve_slots)
    head = runs[plan[0][0]]
    return {"metric": "serving: solves/s with p50/p99 request latency", "mode": "serve",
            "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "runs": runs, "data": "synthetic",
            "config": {"workload": "Poisson arrivals (seed 7); per request Nx,Ny~U{4..40}, b=128, d~U(0.3,0.7) "
                                   "(or 8 keys with d on a 5-point grid), 1-32 scan RHS; c64 blocks",
                       "slots": args.serve_slots}}


def run_ragged(args, sub=False):
    """Ragged workload: square lattices 2x2 .. 48x48 (step 2), b = 96,
    spacings 0.3 / 0.5 / 0.7, one broadside solve each (72 problems).  One
    step = batched set-up (block transform, preconditioner) of all 72 arrays
    + batched solve + port quantities.  Blocks are generated on the GPU
    (synth.offset_blocks_torch, c64)."""
    import torch
    import paper_2608_17844_b300 as m
    from synth import LatticeSpec, offset_blocks_torch, excitation
    torch.cuda.set_device(0)
    specs = [LatticeSpec(n, n, 96, d, 0) for d in (0.3, 0.5, 0.7) for n in range(2, 49, 2)]
    blocks = [offset_blocks_torch(s, "cuda") for s in specs]
    Vs = [torch.from_numpy(excitation(s, [(0.0, 0.0)])).cuda() for s in specs]
    Is = [torch.zeros_like(v) for v in Vs]
    zas = [torch.zeros(v.shape[:3], dtype=torch.complex128, device="cuda") for v in Vs]
    hs = [m.moma_create_array(s.nx, s.ny, s.b) for s in specs]

    def step():
        m.moma_set_blocks_batch(hs, blocks, release_setup=False, workers=8)
        infos = m.moma_solve_batch(hs, Vs, Is, workers=8)
        for h, I, V, za in zip(hs, Is, Vs, zas):
            m.moma_active_impedance(h, I, V, za)
        return infos

    for _ in range(max(1, min(args.warmup, 2))):
        infos = step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3 if sub else 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        infos = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    centre = {f"{s.nx}x{s.ny}@{s.d}": complex(za[0, s.ny // 2, s.nx // 2].item()) for s, za in zip(specs, zas)}
    line = {"metric": "ragged batch: solves/s (set-up + solve per problem)", "mode": "ragged",
            "value": len(specs) / dt, "unit": "solves/s", "ms_per_step": 1000 * dt, "steps": steps,
            "problems": len(specs), "converged": sum(x["converged"] for x in infos),
            "max_rel_residual": max(x["max_rel_residual"] for x in infos),
            "inner_iters": [x["inner_iters"] for x in infos],
            "device_bytes": sum(m.moma_device_bytes(h) for h in hs), "data": "synthetic",
            "config": {"workload": "2x2..48x48 step 2, b=96, d in {0.3,0.5,0.7}, broadside, c64 blocks"},
            "centre_Za": {k: f"{v.real:.6f}{v.imag:+.6f}j" for k, v in list(centre.items())[::6]}}
    for h in hs:
        m.moma_destroy(h)
    del blocks
    torch.cuda.empty_cache()
    return line


def tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst peak times the nominal
    tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)["bf16_tflops"] * 1.1 / 2.25, "of measured (bf16 burst x nominal tf32/bf16)"


def run_scan(args, sub=False):
    """Scan workload: 24 x 24 lattice, b = 256 (N = 147456), 64 RHS per
    array (8 x 8 grid of scan angles, theta in [0, 60], phi in [0, 90)) at
    three element spacings (0.3, 0.5, 0.7 wavelengths: three arrays, c64
    blocks generated on the GPU).  One step = set-up of the three arrays +
    three 64-RHS solves (bin products and preconditioner on the tensor
    cores) + port quantities.  value = RHS solved per second."""
    import torch
    import paper_2608_17844_b300 as m
    from synth import LatticeSpec, offset_blocks_torch, excitation, config_c3_angles
    torch.cuda.set_device(0)
    angles = config_c3_angles()
    specs = [LatticeSpec(24, 24, 256, d, 0) for d in (0.3, 0.5, 0.7)]
    blocks = [offset_blocks_torch(s, "cuda") for s in specs]
    Vs = [torch.from_numpy(excitation(s, angles)).cuda() for s in specs]
    Is = [torch.zeros_like(v) for v in Vs]
    zas = [torch.zeros(v.shape[:3], dtype=torch.complex128, device="cuda") for v in Vs]
    hs = [m.moma_create_array(s.nx, s.ny, s.b) for s in specs]
    nr = len(angles)

    def step():
        m.moma_set_blocks_batch(hs, blocks, release_setup=False, workers=3)
        infos = m.moma_solve_batch(hs, Vs, Is, workers=3)
        for h, I, V, za in zip(hs, Is, Vs, zas):
            m.moma_active_impedance(h, I, V, za)
        return infos

    for _ in range(max(1, min(args.warmup, 2))):
        infos = step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3 if sub else 5))
    clk = ClockSampler(0)
    clk.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        infos = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    clocks = clk.stop()
    # One profiled step, arrays one after another, for the per-kernel split.
    for h in hs:
        m.moma_profile(h, 1)
    for h, b, V, I in zip(hs, blocks, Vs, Is):
        m.moma_set_blocks(h, b)
        m.moma_solve(h, V, I)
    torch.cuda.synchronize()
    fam = {}
    for name in m.KERNEL_IDS:
        n = sum(m.moma_kernel_stats(h, name)[0] for h in hs)
        ms = sum(m.moma_kernel_stats(h, name)[1] for h in hs)
        if n:
            fam[name] = {"launches": n, "ms": round(ms, 3)}
    for h in hs:
        m.moma_profile(h, 0)
    spec = specs[0]
    mxp, myp = smooth235(2 * spec.nx - 1), smooth235(2 * spec.ny - 1)
    flops_launch = 8.0 * (2 * spec.nx - 1) * (2 * spec.ny - 1) * spec.b * spec.b * nr  # on M = 2N-1 bins
    tc = fam.get("bin_tc", {"launches": 0, "ms": 0.0})
    peak, peak_src = tf32_peak()
    us = 1000.0 * tc["ms"] / tc["launches"] if tc["launches"] else None
    achieved = flops_launch / (us * 1e-6) / 1e12 if us else None
    alg_bytes = bin_product_bytes(spec, nr)[0]
    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6400.0)
    line = {"metric": "scan workload: RHS solved/s (set-up + solve, 3 spacings x 64 RHS)", "mode": "scan",
            "value": len(specs) * nr / dt, "unit": "solves/s", "ms_per_step": 1000 * dt, "steps": steps,
            "converged": sum(x["converged"] for x in infos),
            "max_rel_residual": max(x["max_rel_residual"] for x in infos),
            "inner_iters": [x["inner_iters"] for x in infos], "outer_iters": [x["outer_iters"] for x in infos],
            "device_bytes": sum(m.moma_device_bytes(h) for h in hs), "data": "synthetic", "dtype": "c64+c128",
            "config": {"workload": "24x24 lattice, b=256 (N=147456), 64 RHS (8x8 scan grid), d in {0.3,0.5,0.7}, "
                                   "c64 blocks, GMRES(50) + FP64 refinement to 1e-10",
                       "circulant": f"{mxp}x{myp} (padded from {2 * spec.nx - 1})"},
            "kernels_profiled_step": fam,
            "roofline": {"kernel": "bin_mma_kernel (tcgen05 kind::tf32, 3xTF32)", "bound": "hbm",
                         "achieved": alg_bytes / (us * 1e-6) / 1e9 if us else None, "peak": hbm_peak,
                         "unit": "GB/s", "frac": alg_bytes / (us * 1e-6) / 1e9 / hbm_peak if us else None,
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_us": us,
                         "alg_basis": "c64 pair store on M = 2N-1 + bin vectors in and out",
                         "tensor": {"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                    "frac": achieved / peak if achieved else None,
                                    "issued_frac": 3 * achieved / peak if achieved else None,
                                    "flops_per_launch": flops_launch, "peak_source": peak_src}},
            "clocks": clocks,
            "centre_Za_broadside": {f"d={s.d}": f"{complex(za[0, 12, 12].item()):.6f}" for s, za in zip(specs, zas)}}
    for h in hs:
        m.moma_destroy(h)
    del blocks
    torch.cuda.empty_cache()
    return line


def run_predictors(args, sub=False):
    """Analysis workloads on top of the solver (Sec. II-E): the all-port
    passive impedance matrix Z_p of a 16 x 16 lattice (b = 128, 256 unit
    port excitations in RHS chunks of 64 on the tensor-core path, FP64
    Gauss-Jordan inverse) with the xi_Z family; the column coupling C_n of
    the 32 x 32 lattice from 64 row-phase samples; xi_S from S_ideal for the
    32 x 32 lattice.  Timed with CUDA events / host clock, after one warm-up."""
    import torch
    import paper_2608_17844_b300 as m
    from synth import LatticeSpec, offset_blocks_torch
    torch.cuda.set_device(0)
    out = {"metric": "analysis: all-port Z_p, column coupling, xi_S", "mode": "predictors", "data": "synthetic"}
    # Z_p
    spec = LatticeSpec(16, 16, 128, 0.5, 0)
    blocks = offset_blocks_torch(spec, "cuda")
    h = m.moma_create_array(spec.nx, spec.ny, spec.b)
    m.moma_set_blocks(h, blocks)
    n = spec.n_el
    zp = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    m.moma_port_impedance(h, zp, chunk=64)  # warm-up (builds the tensor-core store)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.moma_port_impedance(h, zp, chunk=64)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    zpn = zp.cpu().numpy()
    xz, xmax, bound = m.moma_xi_z(zpn, spec.nx, spec.ny)
    out["zp"] = {"lattice": "16x16, b=128", "ports": n, "seconds": dt, "ports_per_s": n / dt,
                 "symmetry_rel": float(np.linalg.norm(zpn - zpn.T) / np.linalg.norm(zpn)),
                 "xi_z": xz, "xi_z_max": xmax, "border_bound_ohm": bound}
    m.moma_destroy(h)
    # column coupling
    spec = LatticeSpec(32, 32, 128, 0.5, 0)
    blocks = offset_blocks_torch(spec, "cuda")
    h = m.moma_create_array(spec.nx, spec.ny, spec.b)
    m.moma_set_blocks(h, blocks)
    C = torch.zeros(2 * 10 + 1, dtype=torch.complex128, device="cuda")
    g = torch.zeros(64, dtype=torch.complex128, device="cuda")
    m.moma_column_coupling(h, 64, 10, C, g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.moma_column_coupling(h, 64, 10, C, g)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c = C.cpu().numpy()
    out["column_coupling"] = {"lattice": "32x32, b=128", "samples": 64, "seconds": dt,
                              "abs_C_n": {str(k - 10): float(abs(c[k])) for k in range(10, 21)}}
    m.moma_destroy(h)
    t0 = time.perf_counter()
    xs = m.moma_xi_s(32, 32, 0.1 + 0.05j, -0.15 + 0.07j, np.pi, 50.0)
    out["xi_s"] = {"lattice": "32x32", "value": xs, "seconds": time.perf_counter() - t0}
    return out


def headline_config(args, nr, world):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD if not (args.lattice or args.nrhs)
            else f"profiling lattice {args.lattice or 'C2'}, {nr} RHS",
            "rhs_per_step": nr * world, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (c64 blocks 520 MB; stored bins 269 MB c64 + 537 MB c128)"}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle as it stands, on the host cores.  One
    step = the workload's RHS columns each solved to completion by oracle-I
    (the paper publishes no implementation to install).  Whole steps run
    until --steps are done or the next one would pass --ref-seconds (at
    least one step runs); the line reports the steps actually timed."""
    if rank != 0:
        return
    spec, blocks, V = make_inputs(args.lattice, args.nrhs)
    nr = V.shape[0]
    cores = len(os.sched_getaffinity(0))
    # Warm-up: one oracle product (thread pools, page-in), untimed.
    warm = min(args.warmup, 1)
    if warm:
        from oracle import mbt
        mbt.matvec(blocks.astype(np.complex128), spec.nx, spec.ny, V[:1])
    step_s, iters = [], []
    t_all = time.perf_counter()
    while len(step_s) < max(1, args.steps):
        if step_s and (time.perf_counter() - t_all) + float(np.mean(step_s)) > args.ref_seconds:
            break
        t0 = time.perf_counter()
        _, _, its, _ = oracle_solves(spec, blocks, V, list(range(nr)))
        step_s.append(time.perf_counter() - t0)
        iters.append(its)
    total = float(np.sum(step_s))
    value = nr * len(step_s) / total
    sample = (f"oracle-I (complex128 GMRES(60), direct offset-sum product, block Jacobi): {len(step_s)} whole "
              f"step(s) of {nr} RHS each solved to rel. residual 1e-10 ({iters} iterations), {total:.1f} s on "
              f"{cores} host cores; {args.steps} steps requested, whole steps only")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(step_s), "steps_requested": args.steps, "warmup": warm, "warmup_requested": args.warmup,
            "ms_per_step": 1000.0 * total / len(step_s), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": headline_config(args, nr, 1),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_variant(m, torch, spec, blocks_d, V_d, za_d, gam_d, stream, steps, warmup, precision, flags=0,
                  solver=0):
    """Whole steps (set-up + solve + port quantities) of one solver variant
    on the headline problem, CUDA events on the stream around `steps` steps
    after `warmup` untimed ones.  Returns (ms per step, last solve info,
    currents)."""
    h = m.moma_create_array(spec.nx, spec.ny, spec.b, precision, stream=stream, flags=flags)
    I = torch.zeros_like(V_d)
    info = None
    try:
        for _ in range(max(1, warmup)):
            m.moma_set_blocks(h, blocks_d)
            info = m.moma_solve(h, V_d, I, solver=solver)
        torch.cuda.synchronize()
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(steps):
            m.moma_set_blocks(h, blocks_d)
            info = m.moma_solve(h, V_d, I, solver=solver)
            m.moma_active_impedance(h, I, V_d, za_d, gam_d)
        b_.record(stream)
        torch.cuda.synchronize()
        ms = a_.elapsed_time(b_) / steps
    finally:
        m.moma_destroy(h)
    return ms, info, I


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    modes = [("serve", run_serving), ("ragged", run_ragged), ("scan", run_scan), ("predictors", run_predictors)]
    for flag, fn in modes:
        if getattr(args, flag):
            if rank == 0:
                print(json.dumps(fn(args), default=str), flush=True)
            return
    import torch
    import paper_2608_17844_b300 as m
    from paper_2608_17844_b300 import replicas

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    spec, blocks, V = make_inputs(args.lattice, args.nrhs)
    nr = V.shape[0]
    stream = torch.cuda.current_stream()
    blocks_d = torch.from_numpy(blocks).cuda()
    V_d = torch.from_numpy(V).cuda()
    I_d = torch.zeros_like(V_d)
    za_d = torch.zeros(V.shape[:3], dtype=torch.complex128, device="cuda")
    gam_d = torch.zeros_like(za_d)

    h = m.moma_create_array(spec.nx, spec.ny, spec.b, m.MOMA_PREC_MIXED, stream=stream)
    infos = []

    def step():
        m.moma_set_blocks(h, blocks_d)
        infos.append(m.moma_solve(h, V_d, I_d))
        m.moma_active_impedance(h, I_d, V_d, za_d, gam_d)

    for _ in range(args.warmup):
        step()
    barrier()

    def timed_region(profile):
        """K steps between CUDA events on torch's stream (the library's own
        streams are ordered into it), barrier + synchronize on both sides."""
        m.moma_profile(h, profile)
        launches0 = m.moma_launch_count(h)
        marks = []
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            step()
            e_b.record(stream)
            marks.append((e_a, e_b))
        ev1.record(stream)
        barrier()
        total = ev0.elapsed_time(ev1)
        launches = m.moma_launch_count(h) - launches0
        stats = {k: m.moma_kernel_stats(h, k) for k in m.KERNEL_IDS} if profile else None
        m.moma_profile(h, False)
        return total, [a.elapsed_time(b) for a, b in marks], launches, stats

    # Headline: graphs replayed, no per-kernel events.
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    clocks.wait_first()
    total_ms, steps_ms, launches, _ = timed_region(False)
    clk = clocks.stop()
    dev = "cuda" if dist is not None else "cpu"
    value = replicas.aggregate_throughput(nr * args.steps, total_ms / 1000.0, device=dev)
    total_ms = 1000.0 * replicas.max_over_ranks(total_ms / 1000.0, device=dev)
    I_head = I_d.cpu().numpy()
    za_head = za_d.cpu().numpy()
    # Same steps again with CUDA events around every kernel launch (graphs
    # off): per-kernel durations for the roofline and the breakdown.
    prof_total_ms, _, _, stats = timed_region(True)

    # Phase breakdown of one step (set-up vs solve), same stream, events.
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    m.moma_set_blocks(h, blocks_d)
    e[1].record(stream)
    info = m.moma_solve(h, V_d, I_d)
    e[2].record(stream)
    m.moma_active_impedance(h, I_d, V_d, za_d, gam_d)
    e[3].record(stream)
    torch.cuda.synchronize()
    phases = {"set_blocks_ms": e[0].elapsed_time(e[1]), "solve_ms": e[1].elapsed_time(e[2]),
              "ports_ms": e[2].elapsed_time(e[3]), "solve_info": info}

    # Roofline of the dominant kernel: the c64 bin product.
    n_bin, ms_bin = stats["bin_c64"]
    n_fft, ms_fft = stats["fft_c64"]
    alg_bytes, pairs, B = bin_product_bytes(spec, nr)
    pad_bytes = bin_product_bytes(spec, nr, padded=True)[0]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.4 TB/s (of fallback)"
    achieved = alg_bytes / (ms_bin / n_bin / 1000.0) / 1e9 if n_bin else None
    traffic = measured_traffic(pad_bytes, spec, nr)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak if achieved else None,
                "traffic": int(traffic) if traffic else None,
                "traffic_source": "ncu dram bytes of the 24x24 capture scaled by streamed bytes" if traffic
                else "kernel changed since the ncu capture",
                "kernel": "bin_rc_kernel (c64 per-bin product, Z and Z^H legs, row and column warps)",
                "alg_bytes_per_launch": alg_bytes, "alg_basis": f"{pairs} pairs of the {2 * spec.nx - 1}x"
                f"{2 * spec.ny - 1} circulant (M = 2N-1), {nr} RHS",
                "streamed_bytes_per_launch": pad_bytes, "launches": n_bin,
                "avg_launch_us": 1000.0 * ms_bin / n_bin if n_bin else None, "peak_source": peak_src}
    # Back-to-back device time per application (50 applications captured as
    # one CUDA graph, as the solve replays its steps; CUDA events around the
    # replay, no per-launch events in between).
    b2b = {k: m.moma_time_operator(h, w, nr, 50) for k, w in
           (("z", m.MOMA_TIME_Z), ("bin", m.MOMA_TIME_BIN), ("precond", m.MOMA_TIME_PRECOND),
            ("normal", m.MOMA_TIME_NORMAL))}
    b2b_timing = "back-to-back, 50 applications replayed as one CUDA graph, CUDA events around the replay"
    roofline["b2b_launch_us"] = b2b["bin"]
    roofline["b2b_frac"] = alg_bytes / (b2b["bin"] * 1e-6) / 1e9 / hbm_peak
    # The whole Z application (lattice FFT passes + bin product).
    mv_bytes = matvec_bytes(spec, nr)
    mv_us = b2b["z"]
    ev_us = 1000.0 * (ms_bin + ms_fft) / n_bin if n_bin else None
    matvec_roofline = {"bound": "hbm", "alg_bytes_per_application": mv_bytes,
                       "us_per_application": mv_us, "timing": b2b_timing,
                       "event_timed_us_per_application": ev_us,
                       "event_timed_bin_us": 1000.0 * ms_bin / n_bin if n_bin else None,
                       "event_timed_fft_us": 1000.0 * ms_fft / n_bin if n_bin else None,
                       "fft_launches_per_application": n_fft / n_bin if n_bin else None,
                       "achieved": mv_bytes / (mv_us * 1e-6) / 1e9, "peak": hbm_peak,
                       "unit": "GB/s", "frac": mv_bytes / (mv_us * 1e-6) / 1e9 / hbm_peak,
                       "floor_us": mv_bytes / (hbm_peak * 1e9) * 1e6, "peak_source": peak_src}
    # The block preconditioner apply (Eq. 38 through X_e^H X_e): the packed
    # c64 factor triangles once plus x in and y out, per launch.
    n_pre, ms_pre = stats["precond"]
    pre_bytes = spec.nx * spec.ny * (spec.b * (spec.b + 1) // 2) * 8 + 2 * spec.nx * spec.ny * spec.b * nr * 8
    pre_us = b2b["precond"]
    precond_roofline = {"bound": "hbm",
                        "kernel": "precond_blk_kernel (c64 P_e^{-1} = X_e^H X_e stored Hermitian, one pass)",
                        "alg_bytes_per_launch": pre_bytes, "avg_launch_us": pre_us, "timing": b2b_timing,
                        "event_timed_us": 1000.0 * ms_pre / n_pre if n_pre else None, "launches": n_pre,
                        "achieved": pre_bytes / (pre_us * 1e-6) / 1e9, "peak": hbm_peak,
                        "unit": "GB/s", "frac": pre_bytes / (pre_us * 1e-6) / 1e9 / hbm_peak,
                        "peak_source": peak_src}
    # One inner-iteration operator P^{-1} Z^H Z (Sec. III-A): both bin
    # product legs with their lattice vectors, and the preconditioner.
    nm_bytes = 2 * mv_bytes + pre_bytes
    nm_us = b2b["normal"]
    normal_roofline = {"bound": "hbm", "alg_bytes_per_application": nm_bytes, "us_per_application": nm_us,
                       "timing": b2b_timing, "achieved": nm_bytes / (nm_us * 1e-6) / 1e9, "peak": hbm_peak,
                       "unit": "GB/s", "frac": nm_bytes / (nm_us * 1e-6) / 1e9 / hbm_peak,
                       "floor_us": nm_bytes / (hbm_peak * 1e9) * 1e6, "peak_source": peak_src}
    kernel_share = {k: {"launches": n, "ms": ms} for k, (n, ms) in stats.items()}
    m.moma_destroy(h)

    fp_steps = args.steps if args.fp64_steps < 0 else args.fp64_steps
    fp64 = fp64r = pcg = None
    if fp_steps > 0:
        # Plain FP64 GPU solve on the same problem (the comparison solver).
        ms64, inf64, _ = timed_variant(m, torch, spec, blocks_d, V_d, za_d, gam_d, stream, fp_steps, args.warmup,
                                       m.MOMA_PREC_FP64)
        v64 = nr / (ms64 / 1000.0)
        fp64 = {"value": v64, "unit": "solves/s", "ms_per_step": ms64, "steps": fp_steps, "info": inf64,
                "speedup_mixed_vs_fp64": value / world / v64}
        # Mixed path with its FP64-class stages (block-bin transform,
        # refinement residual Z I, block Cholesky) in FP64 instead of
        # double-FP32.
        msr, infr, Ir = timed_variant(m, torch, spec, blocks_d, V_d, za_d, gam_d, stream, fp_steps, args.warmup,
                                      m.MOMA_PREC_MIXED, flags=m.MOMA_FLAG_FP64_RESIDUAL)
        za_r = za_d.cpu().numpy()
        fp64r = {"value": nr / (msr / 1000.0), "unit": "solves/s", "ms_per_step": msr, "steps": fp_steps,
                 "info": infr, "speedup_vs_fp64": (nr / (msr / 1000.0)) / v64,
                 "za_max_rel_diff_vs_headline": float(np.max(np.abs(za_r - za_head) / np.abs(za_head))),
                 "dtype": "c64 inner; block-bin transform, refinement residual Z I and block Cholesky in FP64"}
        # The paper's PCG solver (Sec. II-C) on the same problem and path.
        msp, infp, _ = timed_variant(m, torch, spec, blocks_d, V_d, za_d, gam_d, stream, fp_steps, args.warmup,
                                     m.MOMA_PREC_MIXED, solver=m.MOMA_SOLVER_PCG)
        pcg = {"value": nr / (msp / 1000.0), "unit": "solves/s", "ms_per_step": msp, "steps": fp_steps,
               "info": infp}

    # End to end through the C ABI with host buffers (pinned), copies inside:
    # every step uploads its blocks and V and reads back I, Z_a and Gamma.
    # Measured twice: one handle, steps one after another ("serial"); and
    # --e2e-lanes handles (default 4) on their own streams, each driven by
    # its own host thread, the steps split between them, so that one step's
    # block upload overlaps the others' solves -- how a caller with a stream
    # of independent problems keeps the copy engine and the SMs busy at once
    # (the line's value).  (2 / 3 / 4 handles measured 186 / 195 / 214
    # solves/s on the C2 workload.)
    e2e = None
    if not args.no_e2e:
        import threading
        hb = torch.from_numpy(blocks).pin_memory()

        def make_lane(st):
            lane = {"h": m.moma_create_array(spec.nx, spec.ny, spec.b, m.MOMA_PREC_MIXED, stream=st),
                    "V": torch.from_numpy(V).pin_memory(), "I": torch.zeros(V.shape, dtype=torch.complex128).pin_memory(),
                    "z": torch.zeros(V.shape[:3], dtype=torch.complex128).pin_memory()}
            lane["g"] = torch.zeros_like(lane["z"]).pin_memory()
            return lane

        def host_step(lane):
            m.moma_set_blocks(lane["h"], hb)
            m.moma_solve(lane["h"], lane["V"], lane["I"])
            m.moma_active_impedance(lane["h"], lane["I"], lane["V"], lane["z"], lane["g"])

        nl = max(1, args.e2e_lanes)
        lanes = [make_lane(stream)] + [make_lane(torch.cuda.Stream()) for _ in range(nl - 1)]
        for _ in range(args.warmup):
            for ln in lanes:
                host_step(ln)
        # serial: one handle
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step(lanes[0])
        barrier()
        dt_serial = time.perf_counter() - t0
        # pipelined: nl handles, nl host threads, steps split between them
        counts = [args.steps // nl + (1 if i < args.steps % nl else 0) for i in range(nl)]
        errors = []

        def run_lane(i):
            try:
                for _ in range(counts[i]):
                    host_step(lanes[i])
            except Exception as ex:  # reported after the join
                errors.append(ex)

        barrier()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=run_lane, args=(i,)) for i in range(nl)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        torch.cuda.synchronize()
        barrier()
        dt = time.perf_counter() - t0
        if errors:
            raise errors[0]
        for ln in lanes:
            m.moma_destroy(ln["h"])
        # Host blocks: the library copies the offsets with dy >= 0 (Ny of the
        # 2Ny-1 rows; the rest follow from reciprocity); V goes in twice
        # (solve, port quantities) and I once.
        e2e = {"value": replicas.aggregate_throughput(nr * args.steps, dt, device=dev), "unit": "solves/s",
               "h2d_bytes_per_step": int(blocks.nbytes // (2 * spec.ny - 1) * spec.ny + 2 * V.nbytes + V.nbytes),
               "d2h_bytes_per_step": int(V.nbytes + 2 * lanes[0]["z"].numel() * 16),
               "pipeline": f"{nl} handles on {nl} streams, {nl} host threads, steps split between them",
               "serial": replicas.aggregate_throughput(nr * args.steps, dt_serial, device=dev)}

    ports = {n: [complex(za_head[q, ey, ex]) for q in range(nr)]
             for n, (ex, ey) in named_elements(spec.nx, spec.ny).items()}

    subs = {}
    if rank == 0 and not args.quick and not (args.lattice or args.nrhs):
        sub_args = argparse.Namespace(**vars(args))
        for name, fn in (("scan", run_scan), ("ragged", run_ragged), ("serve", run_serving),
                         ("predictors", run_predictors)):
            try:
                subs[name] = fn(sub_args, sub=True)
            except Exception as ex:  # a failed sub-measurement is reported, not hidden
                subs[name] = {"error": repr(ex)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_leg(spec, blocks, V, I_head)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 inner (FP32 FFTs, bin products, GMRES vectors); refinement residual Z I, block-bin "
                     "transform and block Cholesky in double-FP32 (~48 bit); FP64 residual subtraction, "
                     "Hessenberg/Givens, factor storage",
            "data": "synthetic",
            "config": headline_config(args, nr, world),
            "step_ms": {"p50": statistics.median(steps_ms), "p99": float(np.percentile(steps_ms, 99)),
                        "min": min(steps_ms), "max": max(steps_ms)},
            "profiled_ms_per_step": prof_total_ms / args.steps,
            "phases": phases, "roofline": roofline, "matvec_roofline": matvec_roofline,
            "precond_roofline": precond_roofline, "normal_roofline": normal_roofline, "kernels": kernel_share,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_plain": fp64,
            "mixed_fp64_residual": fp64r, "pcg_mixed": pcg,
            "ports_Za": {k: [f"{z.real:.10f}{z.imag:+.10f}j" for z in v] for k, v in ports.items()},
        }
        line.update(subs)
        print(json.dumps(line, default=str), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
