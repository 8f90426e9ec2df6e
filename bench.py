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
    ap.add_argument("--fp64-steps", type=int, default=2, help="steps of the plain FP64 solve (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="bounded oracle sample (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
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
    ap.add_argument("--serve-keys", type=int, default=8)
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


def bin_product_bytes(spec, nr):
    """Algorithmic bytes of one c64 bin-product launch: the stored bins once
    (one b x b block per {k,-k} pair) plus the bin vectors in and out."""
    def smooth(n):
        m = n
        while True:
            k = m
            for r in (2, 3, 5):
                while k % r == 0:
                    k //= r
            if k == 1:
                return m
            m += 1
    mx, my = smooth(2 * spec.nx - 1), smooth(2 * spec.ny - 1)
    B = mx * my
    pairs = sum(1 for ky in range(my) for kx in range(mx)
                if ky * mx + kx <= ((my - ky) % my) * mx + ((mx - kx) % mx))
    ldb = spec.b + (spec.b % 2)
    return pairs * spec.b * ldb * 8 + 2 * B * nr * spec.b * 8, pairs, B


def measured_traffic(alg_bytes, spec, nr):
    """DRAM bytes per launch of the c64 bin product from the committed ncu
    capture (profiles/bin_pair_kernel_c64_traffic.txt), scaled from the
    captured lattice to this launch by the algorithmic bytes; None if the
    kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "bin_pair_kernel_c64_traffic.txt")
    src = os.path.join(ROOT, "paper_2608_17844_b300", "csrc", "binprod.cu")
    try:
        kv = dict(l.strip().split("=", 1) for l in open(path) if "=" in l and not l.startswith("#"))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if kv.get("kernel_source_sha256") != sha:
        return None
    pairs, bins, nrc, b = (int(kv[k]) for k in ("pairs", "bins", "nrhs", "b"))
    alg_captured = pairs * b * (b + b % 2) * 8 + 2 * bins * nrc * b * 8
    measured = int(kv["dram_read_bytes"]) + int(kv["dram_write_bytes"])
    return measured / alg_captured * alg_bytes


def cpu_oracle_sample(spec, blocks, V, seconds):
    """Time the oracle (oracle-I: GMRES on Z I = V with the direct offset-sum
    product, complex128) on RHS 0 of the workload for a bounded wall time;
    extrapolate to one full solve from the measured time per iteration and
    the observed geometric residual reduction per iteration."""
    from oracle import iterative
    cores = len(os.sched_getaffinity(0))
    b128 = blocks.astype(np.complex128)
    hist = []
    t0 = time.perf_counter()

    class Stop(Exception):
        pass

    def cb(q, it, rel):
        hist.append((time.perf_counter() - t0, it, rel))
        if time.perf_counter() - t0 > seconds:
            raise Stop()

    try:
        iterative.gmres(b128, spec.nx, spec.ny, V[:1], tol=1e-10, restart=60, max_iter=500, callback=cb)
        converged = True
    except Stop:
        converged = False
    if not hist:
        return None
    t_iter = hist[-1][0] / hist[-1][1]
    if converged:
        iters = hist[-1][1]
    else:
        rho = hist[-1][2] ** (1.0 / hist[-1][1])
        iters = int(np.ceil(np.log(1e-10) / np.log(rho))) if 0 < rho < 1 else float("inf")
    per_solve = t_iter * iters
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle-I (complex128 GMRES, direct offset-sum product, block Jacobi) on RHS 0 of the same "
                       f"{spec.nx}x{spec.ny} b={spec.b} problem for {hist[-1][0]:.1f} s: {hist[-1][1]} iterations at "
                       f"{t_iter:.2f} s each, residual {hist[-1][2]:.2e}; "
                       + ("converged" if converged else f"extrapolated to {iters} iterations for 1e-10")),
            "s_per_iteration": t_iter, "iterations_for_1e-10": iters}


def run_serving(args):
    """Serving stream shaped like BASELINE config 5: Poisson arrivals
    (rate --serve-rate, seed 7) of requests with Nx, Ny ~ U{4..40}, b = 128,
    1-32 scan-angle RHS.  Blocks come from a pool of --serve-keys lattices
    (spacing on the 5-point grid 0.3..0.7) generated once on the host, so
    arrays are built on first use and then served from residency."""
    import torch
    import paper_2608_17844_b300 as m
    from synth import LatticeSpec, offset_blocks, excitation
    rng = np.random.default_rng(7)
    pool = []
    for k in range(args.serve_keys):
        nx, ny = int(rng.integers(4, 41)), int(rng.integers(4, 41))
        d = float(rng.choice([0.3, 0.4, 0.5, 0.6, 0.7]))
        spec = LatticeSpec(nx, ny, 128, d, 0)
        pool.append((spec, offset_blocks(spec, np.complex64)))
    reqs = []
    t = 0.0
    while t < args.serve_seconds:
        t += float(rng.exponential(1.0 / args.serve_rate))
        k = int(rng.integers(len(pool)))
        nr = int(rng.integers(1, 33))
        angles = [(float(rng.uniform(0, 60)), float(rng.uniform(0, 90))) for _ in range(nr)]
        reqs.append((t, k, angles))
    torch.cuda.set_device(0)
    s = m.moma_server_create(slots=args.serve_slots)
    max_outstanding = 64
    outstanding = []
    lat, hits, solved, errors = [], 0, 0, 0
    t0 = time.perf_counter()

    def collect(block):
        nonlocal hits, solved, errors
        while outstanding and (block or len(outstanding) >= max_outstanding):
            tk, bufs = outstanding.pop(0)
            r = m.moma_server_wait(s, tk, -1.0)
            lat.append(r["total_ms"])
            hits += r["resident_hit"]
            if r["status"] == 0:
                solved += bufs[0].shape[0]
            else:
                errors += 1
            block = block and bool(outstanding)

    for (ta, k, angles) in reqs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        spec, blocks = pool[k]
        V = excitation(spec, angles)
        I = np.zeros_like(V)
        tk = m.moma_server_submit(s, k + 1, blocks, V, I)
        outstanding.append((tk, (V, I)))
        collect(False)
    collect(True)
    wall = time.perf_counter() - t0
    stats = m.moma_server_get_stats(s)
    m.moma_server_destroy(s)
    lat = np.array(lat)
    line = {"metric": "serving: solves/s with p50/p99 request latency", "mode": "serve",
            "value": solved / wall, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "offered_req_per_s": len(reqs) / reqs[-1][0], "achieved_req_per_s": len(reqs) / wall,
            "requests": len(reqs), "errors": errors, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "resident_hit_rate": hits / len(reqs),
            "slots": args.serve_slots, "server": stats, "data": "synthetic",
            "config": {"workload": f"Poisson {args.serve_rate}/s, {args.serve_keys} lattice keys Nx,Ny~U{{4..40}}, "
                                   f"b=128, d on 0.3..0.7 grid, 1-32 RHS", "max_outstanding": max_outstanding}}
    print(json.dumps(line, default=str), flush=True)


def run_ragged(args):
    """Ragged batch shaped like BASELINE config 4: square lattices 2x2 ..
    48x48 (step 2), b = 96, spacings 0.3 / 0.5 / 0.7, one broadside solve
    each (72 problems).  One step = batched set-up (block transform,
    preconditioner) of all 72 arrays + batched solve + port quantities.
    Blocks are generated on the GPU (synth.offset_blocks_torch, c64)."""
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

    for _ in range(max(1, args.warmup)):
        infos = step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        infos = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    centre = {f"{s.nx}x{s.ny}@{s.d}": complex(za[0, s.ny // 2, s.nx // 2].item()) for s, za in zip(specs, zas)}
    line = {"metric": "ragged batch: solves/s (set-up + solve per problem)", "mode": "ragged",
            "value": len(specs) / dt, "unit": "solves/s", "ms_per_step": 1000 * dt, "steps": steps,
            "problems": len(specs), "converged": sum(x["converged"] for x in infos),
            "inner_iters": [x["inner_iters"] for x in infos],
            "device_bytes": sum(m.moma_device_bytes(h) for h in hs), "data": "synthetic",
            "config": {"workload": "2x2..48x48 step 2, b=96, d in {0.3,0.5,0.7}, broadside, c64 blocks"},
            "centre_Za": {k: f"{v.real:.6f}{v.imag:+.6f}j" for k, v in list(centre.items())[::6]}}
    for h in hs:
        m.moma_destroy(h)
    print(json.dumps(line, default=str), flush=True)


def tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst peak times the nominal
    tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)["bf16_tflops"] * 1.1 / 2.25, "of measured (bf16 burst x nominal tf32/bf16)"


def run_scan(args):
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

    for _ in range(max(1, args.warmup)):
        infos = step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
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
    B = 48 * 48
    flops_launch = 8.0 * B * spec.b * spec.b * nr  # complex b x b by b x nr per bin
    tc = fam.get("bin_tc", {"launches": 0, "ms": 0.0})
    peak, peak_src = tf32_peak()
    achieved = flops_launch / (tc["ms"] / tc["launches"] * 1e-3) / 1e12 if tc["launches"] else None
    line = {"metric": "scan workload: RHS solved/s (set-up + solve, 3 spacings x 64 RHS)", "mode": "scan",
            "value": len(specs) * nr / dt, "unit": "solves/s", "ms_per_step": 1000 * dt, "steps": steps,
            "converged": sum(x["converged"] for x in infos),
            "max_rel_residual": max(x["max_rel_residual"] for x in infos),
            "inner_iters": [x["inner_iters"] for x in infos], "outer_iters": [x["outer_iters"] for x in infos],
            "device_bytes": sum(m.moma_device_bytes(h) for h in hs), "data": "synthetic", "dtype": "c64+c128",
            "config": {"workload": "24x24 lattice, b=256 (N=147456), 64 RHS (8x8 scan grid), d in {0.3,0.5,0.7}, "
                                   "c64 blocks, GMRES(50) + FP64 refinement to 1e-10"},
            "kernels_profiled_step": fam,
            "roofline": {"kernel": "bin_mma_kernel (tcgen05 kind::tf32, 3xTF32)", "bound": "tensor",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if achieved else None,
                         "issued_frac": 3 * achieved / peak if achieved else None,
                         "flops_per_launch": flops_launch, "peak_source": peak_src},
            "clocks": clocks,
            "centre_Za_broadside": {f"d={s.d}": f"{complex(za[0, 12, 12].item()):.6f}" for s, za in zip(specs, zas)}}
    for h in hs:
        m.moma_destroy(h)
    print(json.dumps(line, default=str), flush=True)


def run_predictors(args):
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
    print(json.dumps(out, default=str), flush=True)


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    spec, blocks, V = make_inputs(args.lattice)
    per_step = max(5.0, min(30.0, 120.0 / max(1, args.steps + args.warmup)))
    vals = []
    cb = None
    for s in range(args.warmup + args.steps):
        cb = cpu_oracle_sample(spec, blocks, V, per_step)
        if s >= args.warmup and cb:
            vals.append(cb["value"])
    value = float(np.mean(vals)) if vals else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 2 / value if value else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.lattice else f"profiling lattice {args.lattice}, 1 RHS sampled",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample")} | {"value": value} if cb else None,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.serve:
        if rank == 0:
            run_serving(args)
        return
    if args.ragged:
        if rank == 0:
            run_ragged(args)
        return
    if args.scan:
        if rank == 0:
            run_scan(args)
        return
    if args.predictors:
        if rank == 0:
            run_predictors(args)
        return
    import torch
    import paper_2608_17844_b300 as m

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
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * nr * args.steps / (total_ms / 1000.0)
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
    alg_bytes, pairs, B = bin_product_bytes(spec, nr)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = alg_bytes / (ms_bin / n_bin / 1000.0) / 1e9 if n_bin else None
    traffic = measured_traffic(alg_bytes, spec, nr)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak if achieved else None,
                "traffic": int(traffic) if traffic else None,
                "traffic_source": "ncu dram bytes of the 24x24 capture scaled by algorithmic bytes" if traffic
                else "kernel changed since the ncu capture",
                "kernel": "bin_pair_kernel<float> (c64 per-bin product, Z and Z^H legs)",
                "alg_bytes_per_launch": alg_bytes, "launches": n_bin, "avg_launch_us": 1000.0 * ms_bin / n_bin if n_bin else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"}
    kernel_share = {k: {"launches": n, "ms": ms} for k, (n, ms) in stats.items()}

    # Plain FP64 GPU solve on the same problem (the comparison solver).
    fp64 = None
    if args.fp64_steps > 0:
        h64 = m.moma_create_array(spec.nx, spec.ny, spec.b, m.MOMA_PREC_FP64, stream=stream)
        I64 = torch.zeros_like(V_d)
        m.moma_set_blocks(h64, blocks_d)
        m.moma_solve(h64, V_d, I64)
        torch.cuda.synchronize()
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(args.fp64_steps):
            m.moma_set_blocks(h64, blocks_d)
            inf64 = m.moma_solve(h64, V_d, I64)
            m.moma_active_impedance(h64, I64, V_d, za_d, gam_d)
        b_.record(stream)
        torch.cuda.synchronize()
        ms64 = a_.elapsed_time(b_) / args.fp64_steps
        m.moma_destroy(h64)
        fp64 = {"value": nr / (ms64 / 1000.0), "unit": "solves/s", "ms_per_step": ms64, "info": inf64,
                "speedup_mixed_vs_fp64": value / world / (nr / (ms64 / 1000.0))}

    # The paper's PCG solver (Sec. II-C) on the same problem and path.
    pcg = None
    if args.fp64_steps > 0:
        infos_pcg = []
        for _ in range(2):
            m.moma_set_blocks(h, blocks_d)
            infos_pcg.append(m.moma_solve(h, V_d, I_d, solver=m.MOMA_SOLVER_PCG))
        torch.cuda.synchronize()
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(args.fp64_steps + 1):
            m.moma_set_blocks(h, blocks_d)
            inf_pcg = m.moma_solve(h, V_d, I_d, solver=m.MOMA_SOLVER_PCG)
            m.moma_active_impedance(h, I_d, V_d, za_d, gam_d)
        b_.record(stream)
        torch.cuda.synchronize()
        ms_pcg = a_.elapsed_time(b_) / (args.fp64_steps + 1)
        pcg = {"value": nr / (ms_pcg / 1000.0), "unit": "solves/s", "ms_per_step": ms_pcg, "info": inf_pcg}

    # End to end through the C ABI with host buffers (pinned), copies inside.
    e2e = None
    if not args.no_e2e:
        hb = torch.from_numpy(blocks).pin_memory()
        hV = torch.from_numpy(V).pin_memory()
        hI = torch.zeros_like(hV).pin_memory()
        hz = torch.zeros(V.shape[:3], dtype=torch.complex128).pin_memory()
        hg = torch.zeros_like(hz).pin_memory()

        def host_step():
            m.moma_set_blocks(h, hb)
            m.moma_solve(h, hV, hI)
            m.moma_active_impedance(h, hI, hV, hz, hg)

        host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        barrier()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        # Host blocks: the library copies the offsets with dy >= 0 (Ny of the
        # 2Ny-1 rows; the rest follow from reciprocity); V goes in twice
        # (solve, port quantities) and I once.
        e2e = {"value": world * nr * args.steps / dt, "unit": "solves/s",
               "h2d_bytes_per_step": int(blocks.nbytes // (2 * spec.ny - 1) * spec.ny + 2 * V.nbytes + V.nbytes),
               "d2h_bytes_per_step": int(V.nbytes + 2 * hz.numel() * 16)}

    za = za_d.cpu().numpy()
    from oracle.ports import named_elements
    ports = {n: [complex(za[q, ey, ex]) for q in range(nr)] for n, (ex, ey) in named_elements(spec.nx, spec.ny).items()}
    m.moma_destroy(h)

    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        cpu = cpu_oracle_sample(spec, blocks, V, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (FP32) inner + f64 refinement",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not (args.lattice or args.nrhs)
                       else f"profiling lattice {args.lattice or 'C2'}, {nr} RHS",
                       "rhs_per_step": nr * world, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (c64 blocks 520 MB; stored bins 269 MB c64 + 537 MB c128)"},
            "step_ms": {"p50": statistics.median(steps_ms), "p99": float(np.percentile(steps_ms, 99)),
                        "min": min(steps_ms), "max": max(steps_ms)},
            "profiled_ms_per_step": prof_total_ms / args.steps,
            "phases": phases, "roofline": roofline, "kernels": kernel_share, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_plain": fp64, "pcg_mixed": pcg,
            "ports_Za": {k: [f"{z.real:.10f}{z.imag:+.10f}j" for z in v] for k, v in ports.items()},
        }
        print(json.dumps(line, default=str), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
