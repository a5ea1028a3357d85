"""Benchmark of the ISDF-xTC kernel path on B300 (one JSON line on stdout).

Workload (default): linear H50 chain at 1.8 bohr, 550 seeded random s/p/d
contracted Gaussians -> 400 orbitals, Becke grid 50 x 40 x 50 = 100,000
points, N_mu = 2000, radial e-e Jastrow u = r/(2(1+r)).  A step is one pass
of the whole path: orbitals -> pivoted-Cholesky points -> ISDF fit -> W
kernels (u1x, u1y, u1z, u3) -> xTC D and occupied X -> test energies, with
the inputs resident on the device.

value = algorithmic W-build flops (8 N_mu N_g^2 + 8 N_mu^2 N_g) / device time
of the W build inside each step (CUDA events on the launching stream);
ms_per_step is the whole step.  e2e repeats the step through the public
Python API from pinned host inputs with the copies inside the timed region.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the W build for a slice of outer grid points).
"""
from __future__ import annotations

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

METRIC = "W_munu build TFLOP/s (algorithmic 8 N_mu N_g^2 + 8 N_mu^2 N_g), tensor-core vs FP64 GPU"
L2_BYTES = 126e6  # B300's L2; operands above it are not served from L2 between steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "bf16x6", "tf32x3"])
    ap.add_argument("--workload", default="h50_chain")
    ap.add_argument("--fp64-rows", type=int, default=1024,
                    help="outer grid points of the FP64 GPU comparison slice")
    ap.add_argument("--cpu-rows", type=int, default=64,
                    help="outer grid points of the CPU oracle sample")
    ap.add_argument("--validate", action="store_true",
                    help="instead of the bench line: the whole workload once on the tensor-core "
                         "path and once on the FP64 GPU path from the same orbitals, pivots and "
                         "fit; full W, D, X and energy differences (minutes at the H50 size)")
    ap.add_argument("--assembly", action="store_true",
                    help="instead of the bench line: the full X (every orbital pair) and the "
                         "four-index assembly (one K/DeltaU panel of --panel-rows rows, Delta h, "
                         "f^xTC, E0) at the workload's size, timed")
    ap.add_argument("--panel-rows", type=int, default=512)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--w-only", action="store_true",
                    help="profiling mode: time only the W build on an H50-chain grid with "
                         "--w-nrad radial shells and seeded random xi (N_mu = --w-nmu)")
    ap.add_argument("--streamed", action="store_true",
                    help="the W build with xi in pinned host memory, streamed in grid batches")
    ap.add_argument("--bra", type=int, default=25000)
    ap.add_argument("--ket", type=int, default=25024)
    ap.add_argument("--adjoint", action="store_true",
                    help="adjoint dW/dtheta on the H20 chain (FP32 and FP64) instead of the main line")
    ap.add_argument("--proposer", action="store_true",
                    help="learned proposer on perturbed H30 chains (60,000 points, 240 orbitals, "
                         "N_mu = 1200): train on --n-train, report on --n-test held-out chains")
    ap.add_argument("--vmc", action="store_true",
                    help="VMC optimisation of the correlator (Sec. II.C) on an H20 chain: "
                         "Metropolis sweeps, then Gauss-Newton iterations on the fixed sample")
    ap.add_argument("--fit-mode", type=int, default=1, choices=[0, 1],
                    help="the FP64 products of the orbitals and the fit: 0 on CUDA cores, "
                         "1 emulated on the tensor cores")
    ap.add_argument("--emu64", action="store_true",
                    help="the fit on the H50 chain with FP64 on CUDA cores and with the FP64 "
                         "products emulated on the tensor cores, and one emulated GEMM")
    ap.add_argument("--emu-n", type=int, default=100000)
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--sweeps", type=int, default=40)
    ap.add_argument("--n-train", type=int, default=24)
    ap.add_argument("--n-test", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--kappa", type=str, default="3,6",
                    help="candidate budgets (multiples of N_mu), comma separated")
    ap.add_argument("--kchunk", type=int, default=0,
                    help="stage-1 fold interval in inner points (0: the library default)")
    ap.add_argument("--w-nrad", type=int, default=16)
    ap.add_argument("--w-nmu", type=int, default=1024)
    ap.add_argument("--w-nang", type=int, default=50)
    ap.add_argument("--w-geom", default="h50_chain", choices=["h50_chain", "benzene"])
    ap.add_argument("--w-fp64-rows", type=int, default=0,
                    help="--w-only: also time the FP64 GPU path on this many outer points")
    ap.add_argument("--w-slice", type=int, default=0,
                    help="--w-only: outer grid points of the W build (0: all)")
    return ap.parse_args()


def w_flops(n_mu, n_rows, n_g):
    """Algorithmic flops of the W build over n_rows outer points."""
    return 8.0 * n_mu * n_rows * n_g + 8.0 * n_mu * n_mu * n_rows


FALLBACK_BF16_SUSTAINED_TFLOPS = 1400.0

# ncu counters of the current stage-1 kernel (the CTA-pair kernel), from its
# small-case capture (H50-chain geometry, 40,000 points, N_mu = 1024, one
# launch): dram__bytes_read.sum + dram__bytes_write.sum divided by N_mu x n_g
# (the launch's compulsory traffic, FP64 calG writes and the (w xi) limb reads,
# scales with it), and sm__pipe_tensor_cycles_active as a fraction of elapsed
# cycles.  Empty for a kernel not yet captured.
S1_NCU = {"bf16x3": {"dram_bytes_per_mu_g": 50.2, "tensor_pipe_active": 0.608}}


def tensor_peak(root=None):
    """Dense BF16 peak (TFLOP/s) for a kernel timed inside a long step, and
    where it came from: the sustained figure of the measured-peaks file, else
    its burst figure, else the fallback.  A missing or malformed file gives the
    fallback, never an error."""
    path = os.path.join(ROOT if root is None else root, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        d = None
    if isinstance(d, dict):
        for key, kind in (("bf16_tflops_sustained", "measured bf16 sustained"),
                          ("bf16_tflops", "measured bf16 burst")):
            v = d.get(key)
            if isinstance(v, (int, float)) and not isinstance(v, bool) and v > 0:
                return float(v), kind
    return FALLBACK_BF16_SUSTAINED_TFLOPS, "fallback bf16 sustained"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name):
    from synth import workloads as wl
    fn = {"h50_chain": wl.h50_chain, "h6_chain": wl.h6_chain,
          "benzene_c6h6": wl.benzene_c6h6}[name]
    return fn()


def sampled_energy_error(api, inp, out, J, precision, n_slices=8, width=128):
    """Error of the tensor-core energies against the FP64 GPU path, estimated
    from outer-grid slices.  W, D and X are sums over outer grid points and the
    energies are linear in them, so each slice's error contribution is exact:
    both paths build W, calG, D and X over the slice (same xi, pivots and
    orbitals) and the energies of the partial sums are differenced.  The total
    is extrapolated by n_g / (n_slices width), with the standard error of that
    extrapolation from the spread over the slices."""
    import torch
    n_g, n_occ = inp.n_g, inp.n_occ
    xi, xig, phiP, dphiP = out["xi"], out["xig"], out["phiP"], out["dphiP"]
    diffs = []
    for i in range(n_slices):
        g0 = max(0, min(n_g - width, int((i + 0.5) * n_g / n_slices) - width // 2))
        g1 = min(n_g, g0 + width)
        xs = xi[:, g0:g1].contiguous()
        ws = inp.w[g0:g1].contiguous()
        E = {}
        for prec in ("fp64", precision):
            W, calG = api.tc_kernel_build(inp.grid, inp.w, xi, xig, J, prec, g_begin=g0, g_end=g1)
            D, Xp = api.xtc_density_contract(phiP, n_occ, xs, ws, calG, n_occ, precision=prec)
            E[prec] = api.tc_energies(W, D, Xp, phiP, dphiP, n_occ)
            del W, calG, D, Xp
        diffs.append([a - b for a, b in zip(E[precision], E["fp64"])])
    torch.cuda.empty_cache()
    d = np.array(diffs)
    scale = n_g / (n_slices * width)
    est = scale * d.sum(axis=0)
    se = scale * np.sqrt(n_slices) * d.std(axis=0, ddof=1)
    keys = ("E_K", "E_dU", "E0")
    return {"estimate": dict(zip(keys, map(float, est))),
            "std_error": dict(zip(keys, map(float, se))),
            "sample": f"{n_slices} outer slices x {width} points spread over the grid, exact "
                      f"per-slice differences of W, D, X and the energies, extrapolated by "
                      f"n_g/{n_slices * width}"}


def cpu_sample(wlw, rows, xi, xit):
    """FP64 oracle W build for `rows` outer points (all inner points)."""
    from oracle import wbuild
    t0 = time.perf_counter()
    g_rows = np.arange(rows)
    calG = wbuild.stage1(wlw.grid_xyz, wlw.grid_w, xi, wlw.jastrow, g_rows=g_rows, batch=16)
    wbuild.stage2(wlw.grid_w, xi, xit, calG, g_rows=g_rows)
    dt = time.perf_counter() - t0
    return dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def aggregate_times(a4_ms, ms_step, world, device):
    """Max over ranks of the per-replica W-build and step times: the slowest
    replica sets the pace of the whole job."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([a4_ms, ms_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t[0]), float(t[1])
    return a4_ms, ms_step


def job_tflops(world, flops_per_replica, ms):
    """Whole-job throughput: every replica's work over the slowest replica's time."""
    return world * flops_per_replica / (ms * 1e-3) / 1e12


def run_config(args, wlw, world):
    """The workload config shared by both arms' lines."""
    n_mu, n_g = wlw.n_mu, wlw.n_g
    limbs = 2 if args.precision == "bf16x3" else 3
    limb_bytes = limbs * 2 * n_mu * n_g
    l2 = (f"inputs larger than L2 (w xi limbs {limb_bytes / 1e9:.2f} GB)" if limb_bytes > L2_BYTES
          else f"inputs fit in L2 (w xi limbs {limb_bytes / 1e6:.1f} MB): not a timing size")
    return {"workload": args.workload, "n_g": n_g, "n_mu": n_mu, "n_orb": wlw.n_orb,
            "n_occ": wlw.n_occ, "jastrow": "radial u=r/(2(1+r))",
            "precision": args.precision,
            "l2": l2,
            "parallelism": f"replicas{world}",
            "fp64_products": ("orbitals and fit: emulated on the tensor cores"
                              if getattr(args, "fit_mode", 0) else "FP64 on CUDA cores"),
            "value_basis": "W build (stage 1 + stage 2 + operand prep) inside each full-path step"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wlw = make_workload(args.workload)
    # inputs of the workload's shape (the oracle's cost does not depend on
    # the values); each step is the W build for a slice of outer points
    rng = np.random.default_rng(0)
    n_mu, n_g = wlw.n_mu, wlw.n_g
    xi = rng.standard_normal((n_mu, n_g)) * 1e-3
    xit = rng.standard_normal((3, n_mu, n_g)) * 1e-3
    times = []
    for _ in range(args.warmup):
        cpu_sample(wlw, args.cpu_rows, xi, xit)
    for _ in range(args.steps):
        times.append(cpu_sample(wlw, args.cpu_rows, xi, xit))
    dt = statistics.mean(times)
    val = w_flops(n_mu, args.cpu_rows, n_g) / dt / 1e12
    unit = "TFLOP/s"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": unit,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(args, wlw, world),
            "cpu_baseline": {"value": val, "unit": unit, "cores": host_cores(), "kind": "oracle",
                             "sample": f"W build (stages 1+2) for {args.cpu_rows} of {n_g} outer "
                                       f"grid points, all {n_g} inner points, N_mu={n_mu}; "
                                       f"random xi of the workload's shape"},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_w_only(args):
    """The W build alone (kernel profiles; the benzene-geometry timing): the
    H50-chain geometry with the radial correlator, or the benzene geometry
    with its two-type multi-centre correlator; seeded random xi."""
    import numpy as np
    import torch
    from synth import workloads as wl
    from paper_2607_17314_b300 import api, build
    build.build()
    if args.w_geom == "benzene":
        atoms, xyz = wl.benzene()
        grid, w = wl.becke_grid(xyz, args.w_nrad, args.w_nang)
        jas = wl.bh_jastrow(atoms, xyz, wl.BH_TERMS_C3, np.random.default_rng(3001))
    else:
        _, xyz = wl.h_chain(50, 1.8)
        grid, w = wl.becke_grid(xyz, args.w_nrad, args.w_nang)
        jas = wl.radial_jastrow(xyz)
    n_g, n_mu = grid.shape[0], args.w_nmu
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    g = torch.tensor(grid, device="cuda")
    wt = torch.tensor(w, device="cuda")
    xi = torch.randn((n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    xig = torch.randn((3, n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    g1 = n_g if args.w_slice <= 0 else min(n_g, args.w_slice)
    kb = api.KernelBuilder(g, wt, xi, xig, api.jastrow_from(jas), args.precision, g_end=g1,
                           kchunk=args.kchunk, time_stages=True)
    for _ in range(max(args.warmup, 1)):
        kb()
    s1, s2 = [], []
    for _ in range(args.steps):
        kb()
        s1.append(kb.stage_ms[0]); s2.append(kb.stage_ms[1])
    fl1 = 8.0 * n_mu * n_g * g1
    out = {"mode": "w_only", "geometry": args.w_geom, "n_g": n_g, "outer_points": g1,
           "n_mu": n_mu, "precision": args.precision, "s1_ms": s1, "s2_ms": s2,
           "s1_alg_tflops": fl1 / (min(s1) * 1e-3) / 1e12}
    if args.w_fp64_rows > 0:
        # the FP64 GPU path and the tensor-core path on the same outer slice
        rows = min(args.w_fp64_rows, g1)
        J = api.jastrow_from(jas)
        k64 = api.KernelBuilder(g, wt, xi, xig, J, "fp64", g_end=rows)
        k16 = api.KernelBuilder(g, wt, xi, xig, J, args.precision, g_end=rows)
        k64()
        k16()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        k64()
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        fl64 = 8.0 * n_mu * n_g * rows + 8.0 * n_mu * n_mu * rows
        err = [float(torch.linalg.norm(k16.W[c] - k64.W[c]) / torch.linalg.norm(k64.W[c]))
               for c in range(4)]
        out["fp64_gpu"] = {"outer_points": rows, "ms": t64, "tflops": fl64 / (t64 * 1e-3) / 1e12,
                           "w_rel_err_tc_vs_fp64": err}
        out["speedup_tc_over_fp64"] = out["s1_alg_tflops"] / out["fp64_gpu"]["tflops"]
    print(json.dumps(out), flush=True)


def run_streamed(args):
    """The W build with xi and xi~ in pinned host memory (Sec. II.D grid-batched
    streaming, depth-one prefetch) against the resident build, H50-chain
    geometry (--w-nrad/--w-nmu), radial correlator, seeded random xi."""
    import torch
    from synth import workloads as wl
    from paper_2607_17314_b300 import api, build
    build.build()
    _, xyz = wl.h_chain(50, 1.8)
    grid, w = wl.becke_grid(xyz, args.w_nrad, args.w_nang)
    jas = api.jastrow_from(wl.radial_jastrow(xyz))
    n_g, n_mu = grid.shape[0], args.w_nmu
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    g = torch.tensor(grid, device="cuda")
    wt = torch.tensor(w, device="cuda")
    xi = torch.randn((n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    xig = torch.randn((3, n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    xi_h = xi.cpu().pin_memory()
    xig_h = xig.cpu().pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            out = fn()
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, ts

    kb = api.KernelBuilder(g, wt, xi, xig, jas, args.precision, kchunk=args.kchunk)
    _, tr = timed(lambda: kb())
    Ws, tsd = timed(lambda: api.tc_kernel_build_streamed(g, wt, xi_h, xig_h, jas, args.precision,
                                                        bra=args.bra, ket=args.ket,
                                                        kchunk=args.kchunk))
    n_bra = -(-n_g // args.bra)
    h2d = 8 * n_mu * n_g * (n_bra + 4)
    fl = 8.0 * n_mu * n_g * n_g + 8.0 * n_mu * n_mu * n_g
    rel = [float(torch.linalg.norm(Ws[c] - kb.W[c]) / torch.linalg.norm(kb.W[c])) for c in range(4)]
    print(json.dumps({"mode": "streamed", "n_g": n_g, "n_mu": n_mu, "precision": args.precision,
                      "bra": args.bra, "ket": args.ket, "resident_ms": tr, "streamed_ms": tsd,
                      "resident_tflops": fl / (min(tr) * 1e-3) / 1e12,
                      "streamed_tflops": fl / (min(tsd) * 1e-3) / 1e12,
                      "h2d_bytes": h2d, "h2d_gbs_needed": h2d / (min(tsd) * 1e-3) / 1e9,
                      "w_rel_diff_streamed_vs_resident": rel}), flush=True)


def run_adjoint(args):
    """The adjoint dL/dtheta on the H20-chain workload (40,000 points, N_mu = 800,
    28-term one-type correlator + d + b = 30 parameters; seeded xi and seed
    Wbar of the workload's shapes): the FP32 adjoint kernel, with the FP64
    forward W build of the same correlator on a 512-point outer slice for
    comparison (the full FP64 forward and the FP64 adjoint take minutes at this
    size; their agreement with the FP32 adjoint is tested on smaller cases)."""
    import numpy as np
    import torch
    from synth import workloads as wl
    from paper_2607_17314_b300 import api, build
    build.build()
    w = wl.h20_chain_bh()
    n_g, n_mu = w.grid_xyz.shape[0], w.n_mu
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4321)
    g = torch.tensor(w.grid_xyz, device="cuda")
    wt = torch.tensor(w.grid_w, device="cuda")
    xi = torch.randn((n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    xig = torch.randn((3, n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    Wbar = torch.tensor(wl.seeded_matrix((4, n_mu, n_mu), 77), device="cuda")
    J = api.jastrow_from(w.jastrow)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            fn()
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, ts

    d32, t32 = timed(lambda: api.tc_kernel_adjoint(g, wt, xi, xig, J, Wbar, "fp32"))
    rows = 512
    _, tw = timed(lambda: api.tc_kernel_build(g, wt, xi, xig, J, "fp64", g_end=rows))
    pair_flops = 8.0 * n_mu * n_g * n_g  # the recomputed M tiles, 4 channels
    print(json.dumps({"mode": "adjoint", "workload": "h20_chain (28-term correlator, 30 parameters)",
                      "n_g": n_g, "n_mu": n_mu, "n_params": int(d32.numel()),
                      "fp32_ms": t32,
                      "fp32_m_tile_tflops": pair_flops / (min(t32) * 1e-3) / 1e12,
                      "forward_fp64_slice": {"outer_points": rows, "ms": tw,
                                             "tflops": 8.0 * n_mu * n_g * rows / (min(tw) * 1e-3) / 1e12},
                      "dtheta_finite": bool(torch.isfinite(d32).all())}), flush=True)


def fit_backward_errors(out, cols_n=128, seed=2):
    """Backward error of the fit's normal equations on sampled grid columns,
    ||A X - B|| / (||A|| ||X||) per channel, from the GPU's orbitals at the
    pivots and at the columns (host FP64 GEMMs; A includes the jitter used)."""
    phi, dphi, piv = out["phi"], out["dphi"], out["pivots"]
    n_g = phi.shape[1]
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(n_g, cols_n, replace=False))
    P = piv.cpu().numpy().astype(np.int64)
    import torch
    it = torch.as_tensor(cols, device=phi.device)
    pc = phi[:, it].cpu().numpy()
    dc = dphi[:, :, it].cpu().numpy()
    phiP = out["phiP"].cpu().numpy()             # [n_mu][n_orb]
    dphiP = out["dphiP"].cpu().numpy()           # [3][n_mu][n_orb]
    GPP = phiP @ phiP.T
    G = phiP @ pc
    X = [out["xi"][:, it].cpu().numpy()] + [out["xig"][c][:, it].cpu().numpy() for c in range(3)]
    res = []
    for c in range(4):
        if c == 0:
            A, B = GPP * GPP, G * G
        else:
            A, B = (dphiP[c - 1] @ dphiP[c - 1].T) * GPP, (dphiP[c - 1] @ dc[c - 1]) * G
        A = A + out["jitter"][c] * np.eye(A.shape[0])
        res.append(float(np.linalg.norm(A @ X[c] - B) / (np.linalg.norm(A) * np.linalg.norm(X[c]))))
        del A, B
    return res, int(len(P))


def run_validate_sampled(args):
    """The benzene workload end to end at full size (271,800 points, 1200
    orbitals, N_mu = 8000, two-type correlator): one pass of the path with CUDA
    event stage times, the fit's backward error on sampled grid columns, and
    the energies' error against the FP64 GPU path from outer-grid slices (a
    full FP64 W build with this correlator would take hours)."""
    import torch
    from paper_2607_17314_b300 import api, build, pipeline
    build.build()
    wlw = make_workload(args.workload)
    b = wlw.basis
    J = api.jastrow_from(wlw.jastrow)
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, wlw.mo_coef, wlw.grid_xyz,
                          wlw.grid_w, wlw.n_mu, wlw.n_occ, J)
    events = {}
    stage_ms = []
    out = pipeline.run(inp, precision=args.precision, events=events, stage_ms=stage_ms,
                       kchunk=args.kchunk, fit_mode=args.fit_mode)
    torch.cuda.synchronize()
    st = {k: float(v[0].elapsed_time(v[1])) for k, v in events.items()}
    back, n_piv = fit_backward_errors(out)
    n_g, n_mu = inp.n_g, inp.n_mu
    s1 = stage_ms[0][0] if stage_ms else float("nan")
    err = sampled_energy_error(api, inp, out, J, args.precision)
    keys = ("E_K", "E_dU", "E0")
    print(json.dumps({
        "mode": "validate_sampled", "workload": args.workload, "precision": args.precision,
        "n_g": n_g, "n_mu": n_mu, "n_orb": int(out["phi"].shape[0]), "n_occ": inp.n_occ,
        "pivots": n_piv, "jitter": list(map(float, out["jitter"])), "stages_ms": st,
        "s1_ms": s1, "s1_alg_tflops": 8.0 * n_mu * n_g * n_g / (s1 * 1e-3) / 1e12,
        "fit_backward_error_sampled_cols": back,
        "energies_ha": dict(zip(keys, out["E"])),
        "energies_err_ha_vs_fp64_gpu": err,
    }), flush=True)


def run_validate(args):
    """Full-size accuracy of the tensor-core path against the FP64 GPU path (the
    FP64 GPU path is checked against the FP64 oracle at 1e-10 on the smaller
    configurations): one pass of the path at the requested precision, then W,
    D, X and the energies rebuilt in FP64 on the GPU from the same orbitals,
    pivots and fit."""
    import torch
    from paper_2607_17314_b300 import api, build, pipeline
    if args.workload == "benzene_c6h6":
        return run_validate_sampled(args)
    build.build()
    wlw = make_workload(args.workload)
    b = wlw.basis
    J = api.jastrow_from(wlw.jastrow)
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, wlw.mo_coef, wlw.grid_xyz,
                          wlw.grid_w, wlw.n_mu, wlw.n_occ, J)
    out = pipeline.run(inp, precision=args.precision, kchunk=args.kchunk, fit_mode=args.fit_mode)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W64, calG64 = api.tc_kernel_build(inp.grid, inp.w, out["xi"], out["xig"], J, "fp64")
    torch.cuda.synchronize()
    t_w = time.perf_counter() - t0
    D64, X64 = api.xtc_density_contract(out["phiP"], inp.n_occ, out["xi"], inp.w, calG64,
                                        inp.n_occ, precision="fp64")
    E64 = api.tc_energies(W64, D64, X64, out["phiP"], out["dphiP"], inp.n_occ)
    # the xTC arithmetic alone: FP64 D and X from the tensor-core calG
    D6c, X6c = api.xtc_density_contract(out["phiP"], inp.n_occ, out["xi"], inp.w, out["calG"],
                                        inp.n_occ, precision="fp64")
    E_xtc_arith = api.tc_energies(out["W"], D6c, X6c, out["phiP"], out["dphiP"], inp.n_occ)
    relf = lambda a, r: float(torch.linalg.norm(a - r) / torch.linalg.norm(r))
    keys = ("E_K", "E_dU", "E0")
    print(json.dumps({
        "mode": "validate", "workload": args.workload, "precision": args.precision,
        "n_g": inp.n_g, "n_mu": inp.n_mu, "n_occ": inp.n_occ,
        "fp64_w_build_s": t_w,
        "w_rel_err": [relf(out["W"][c], W64[c]) for c in range(4)],
        "w_max_err_over_max": [float((out["W"][c] - W64[c]).abs().max() / W64[c].abs().max())
                               for c in range(4)],
        "calG_rel_err": [relf(out["calG"][c], calG64[c]) for c in range(4)],
        "D_rel_err": relf(out["D"], D64), "X_rel_err": relf(out["Xp"], X64),
        "energies_ha": dict(zip(keys, out["E"])), "energies_fp64_ha": dict(zip(keys, E64)),
        "energies_err_ha": {k: a - b for k, a, b in zip(keys, out["E"], E64)},
        "energies_err_ha_from_xtc_arithmetic": {k: a - b for k, a, b in
                                                zip(keys, out["E"], E_xtc_arith)},
        "energies_err_ha_from_w_and_calG": {k: a - b for k, a, b in zip(keys, E_xtc_arith, E64)},
    }), flush=True)


def run_assembly(args):
    """The xTC X over every orbital pair and the four-index assembly at the
    workload's size: one pass of the path, then X with n_orb_x = n_orb, one
    panel of K and DeltaU rows (tensor cores, three limbs), and Delta h,
    f^xTC, E0 for every orbital pair; device times by CUDA events."""
    import torch
    from paper_2607_17314_b300 import api, build, pipeline
    build.build()
    wlw = make_workload(args.workload)
    b = wlw.basis
    J = api.jastrow_from(wlw.jastrow)
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, wlw.mo_coef, wlw.grid_xyz,
                          wlw.grid_w, wlw.n_mu, wlw.n_occ, J)
    out = pipeline.run(inp, precision=args.precision, kchunk=args.kchunk, fit_mode=args.fit_mode)
    n_orb, n_mu, n_g, n_occ = wlw.n_orb, wlw.n_mu, inp.n_g, wlw.n_occ

    def timed(fn, reps=2):
        fn()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(); e0.record(); r = fn(); e1.record(); torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return r, min(ts)

    (D, Xp), t_x = timed(lambda: api.xtc_density_contract(out["phiP"], n_occ, out["xi"], inp.w,
                                                          out["calG"], n_orb,
                                                          precision=args.precision), reps=1)
    x_flops = 4.0 * n_g * n_mu * n_orb * n_orb
    rows = min(args.panel_rows, n_orb * n_orb)
    (Kp, Up), t_p = timed(lambda: api.tc_two_body_panel(out["W"], D, Xp, out["phiP"],
                                                        out["dphiP"], 0, rows,
                                                        precision=args.precision), reps=1)
    p_flops = 12.0 * rows * n_mu * n_orb * n_orb
    (dh, f, e0), t_1 = timed(lambda: api.tc_xtc_one_body(out["W"], D, Xp, out["phiP"],
                                                         out["dphiP"], n_occ))
    # the occupied block of the panel against the occupied-only energies call
    print(json.dumps({
        "mode": "assembly", "workload": args.workload, "precision": args.precision,
        "n_g": n_g, "n_mu": n_mu, "n_orb": n_orb, "n_occ": n_occ,
        "x_full_ms": t_x, "x_full_alg_tflops": x_flops / (t_x * 1e-3) / 1e12,
        "panel_rows": rows, "panel_ms": t_p, "panel_alg_tflops": p_flops / (t_p * 1e-3) / 1e12,
        "panels_for_all_rows_s_extrapolated": t_p * 1e-3 * n_orb * n_orb / rows,
        "one_body_ms": t_1, "e0_ha": e0, "e0_occupied_energies_call_ha": out["E"][2],
    }), flush=True)


def _chain(k):
    from synth import workloads as wl
    return wl.perturbed_chain(k)


def run_proposer(args):
    """Learned interpolation-point proposer at the perturbed-H30 scale."""
    import multiprocessing as mp
    ks = list(range(args.n_train)) + list(range(1000, 1000 + args.n_test))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        chains = pool.map(_chain, ks)
    import torch
    from paper_2607_17314_b300 import api, build, proposer as PR
    build.build()

    def cu(a, dt=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    samples, plain_ms = [], []
    for w in chains:
        b = w.basis
        phi, dphi = api.isdf_eval_orbitals(cu(b.center), cu(b.powers, torch.int32), cu(b.exps),
                                           cu(b.coefs), cu(w.mo_coef), cu(w.grid_xyz))
        wt = cu(w.grid_w)
        e0 = ev()
        plain = api.isdf_points(phi, dphi, wt, w.n_mu)
        e1 = ev()
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
        labels = torch.zeros(w.n_g, dtype=torch.float32, device="cuda")
        labels[plain.long()] = 1.0
        feat = PR.features(phi, dphi, wt, cu(w.grid_xyz), w.xyz)
        samples.append(PR.Sample(feat=feat, labels=labels, phi=phi, dphi=dphi, w=wt, plain=plain,
                                 n_mu=w.n_mu))
    train, test = samples[:args.n_train], samples[args.n_train:]
    prop = PR.Proposer(seed=0, lr=3e-3)
    e0 = ev()
    losses = [prop.train_epoch(train) for _ in range(args.epochs)]
    e1 = ev()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    kappas = [float(k) for k in str(args.kappa).split(",")]
    summary = {}
    for kappa in kappas:
        rows = []
        for smp, pm in zip(test, plain_ms[args.n_train:]):
            e0 = ev()
            piv = prop.propose(smp, kappa)
            e1 = ev()
            torch.cuda.synchronize()
            ep = PR.fit_error(smp.phi, smp.w, piv)
            el = PR.fit_error(smp.phi, smp.w, smp.plain)
            c_net = prop.candidates(smp, kappa)
            c_diag = PR.diagonal_candidates(smp, kappa)
            ed = PR.fit_error(smp.phi, smp.w,
                              PR.points_restricted(smp.phi, smp.dphi, smp.w, c_diag, smp.n_mu))
            rows.append({"plain_ms": pm, "proposal_ms": e0.elapsed_time(e1), "eps_plain": el,
                         "eps_proposal": ep, "eps_diagonal_budget": ed, "ratio": ep / el,
                         "recall_network": PR.recall(c_net, smp.plain),
                         "recall_diagonal": PR.recall(c_diag, smp.plain)})
        summary[str(kappa)] = {
            "median_selection_speedup": float(np.median([r["plain_ms"] / r["proposal_ms"]
                                                         for r in rows])),
            "median_fit_error_ratio_vs_plain": float(np.median([r["ratio"] for r in rows])),
            "median_fit_error_ratio_vs_diagonal_budget": float(np.median(
                [r["eps_proposal"] / r["eps_diagonal_budget"] for r in rows])),
            "mean_recall_network": float(np.mean([r["recall_network"] for r in rows])),
            "mean_recall_diagonal": float(np.mean([r["recall_diagonal"] for r in rows])),
            "per_chain": rows}
    line = {"mode": "proposer", "workload": "perturbed H30 chains", "n_g": int(test[0].feat.shape[0]),
            "n_mu": test[0].n_mu, "n_train": args.n_train, "n_test": args.n_test,
            "epochs": args.epochs, "train_ms": train_ms,
            "loss_first": losses[0], "loss_last": losses[-1], "by_kappa": summary}
    print(json.dumps(line), flush=True)


def run_vmc(args):
    """Reference-variance VMC optimisation of the correlator (Sec. II.C) on an
    H20 chain (s/p basis, 80 functions, 10 doubly occupied orbitals, the
    28-term one-type BH correlator: 30 parameters).  --walkers walkers start
    around the nuclei, take --sweeps Metropolis sweeps of |Phi_0|^2 (random
    numbers drawn on the device and passed in), then each timed step is one
    Gauss-Newton iteration on that fixed sample: local energies with their
    parameter Jacobian, then the step of Eq. gn applied to theta.  The
    oracle's local energy and Jacobian are timed on a few walkers."""
    import numpy as np
    import torch
    from synth import workloads as wl
    from paper_2607_17314_b300 import api, build
    build.build()
    atoms, xyz, basis, C, n_occ, jas = wl.vmc_chain(20, terms=wl.bh_terms_c4(), jscale=0.05)
    N, Nw = 2 * n_occ, args.walkers
    Z = np.ones(len(atoms))
    B = tuple(torch.as_tensor(np.ascontiguousarray(a)).cuda()
              for a in (basis.center, basis.powers.astype(np.int32), basis.exps, basis.coefs))
    Cg = torch.as_tensor(np.ascontiguousarray(C)).cuda()
    R = torch.as_tensor(wl.vmc_walkers(xyz, Nw, N, seed=61)).cuda()
    J = api.jastrow_from(jas)
    theta0 = np.concatenate([[jas.d], np.asarray(jas.b, float), np.asarray(jas.coef, float).ravel()])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(62)
    normals = torch.randn((args.sweeps, N, Nw, 3), dtype=torch.float64, device="cuda", generator=gen)
    uniforms = torch.rand((args.sweeps, N, Nw), dtype=torch.float64, device="cuda", generator=gen)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    half = args.sweeps // 2
    api.isdf_vmc_sample(B, Cg, n_occ, R, normals[:half], uniforms[:half], 0.5)  # burn-in
    torch.cuda.synchronize()
    e0.record()
    acc = api.isdf_vmc_sample(B, Cg, n_occ, R, normals[half:], uniforms[half:], 0.5)
    e1.record()
    torch.cuda.synchronize()
    sample_ms = e0.elapsed_time(e1)
    timed_sweeps = args.sweeps - half
    theta = torch.as_tensor(theta0.copy()).cuda()
    opt = api.VmcOptimizer(B, Cg, n_occ, R, J, Z, theta)
    var = [opt.var]
    lams = []
    for _ in range(max(args.warmup, 3)):
        v, lam, _ = opt.step()
        var.append(v)
        lams.append(lam)
    ts = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0.record()
        v, lam, _ = opt.step()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        var.append(v)
        lams.append(lam)
    # one local energy + Jacobian pass alone
    torch.cuda.synchronize()
    e0.record()
    api.isdf_vmc_local_energy(B, Cg, n_occ, R, J, Z, theta=theta)
    e1.record()
    torch.cuda.synchronize()
    jac_ms = e0.elapsed_time(e1)
    # energies alone (no Jacobian)
    torch.cuda.synchronize()
    e0.record()
    api.isdf_vmc_local_energy(B, Cg, n_occ, R, J, Z, theta=theta, grad=False)
    e1.record()
    torch.cuda.synchronize()
    eloc_ms = e0.elapsed_time(e1)
    # the warm-up / refinement schedule: each step continues the chains for 10
    # sweeps, then one Gauss-Newton step; Polyak-Ruppert average of the last 4
    th_s = torch.as_tensor(theta0.copy()).cuda()
    torch.cuda.synchronize()
    e0.record()
    avg, sched = api.vmc_schedule(B, Cg, n_occ, R, J, Z, th_s, n_warm=4, n_refine=8, window=4,
                                  sweeps=10, sigma=0.5, generator=gen)
    e1.record()
    torch.cuda.synchronize()
    sched_ms = e0.elapsed_time(e1)
    R2 = torch.as_tensor(wl.vmc_walkers(xyz, Nw, N, seed=64)).cuda()
    n2 = torch.randn((args.sweeps, N, Nw, 3), dtype=torch.float64, device="cuda", generator=gen)
    u2 = torch.rand((args.sweeps, N, Nw), dtype=torch.float64, device="cuda", generator=gen)
    api.isdf_vmc_sample(B, Cg, n_occ, R2, n2, u2, 0.5)
    th0 = torch.as_tensor(theta0.copy()).cuda()
    v_start = float(api.isdf_vmc_objective(
        api.isdf_vmc_local_energy(B, Cg, n_occ, R2, J, Z, theta=th0, grad=False))[1])
    v_avg = float(api.isdf_vmc_objective(
        api.isdf_vmc_local_energy(B, Cg, n_occ, R2, J, Z, theta=avg, grad=False))[1])
    # parity on seeded walkers (oracle inputs from the generator, not the GPU)
    from oracle import vmc as ovmc
    Rs = wl.vmc_walkers(xyz, 4, N, seed=63)
    t0 = time.time()
    refE = ovmc.local_energies(Rs, basis, C[:, :n_occ], jas, xyz, Z)
    refJ = ovmc.energy_jacobian_fd(Rs, basis, C[:, :n_occ], jas, xyz, Z)
    oracle_s = time.time() - t0
    Eg, dEg = api.isdf_vmc_local_energy(B, Cg, n_occ, torch.as_tensor(Rs).cuda(), J, Z)
    line = {"mode": "vmc", "workload": "H20 chain, s/p basis (80 functions), 20 electrons, "
                                       "28-term BH correlator (30 parameters)",
            "walkers": Nw, "sweeps": args.sweeps, "timed_sweeps": timed_sweeps,
            "sample_ms": sample_ms,
            "moves_per_s": timed_sweeps * N * Nw / (sample_ms * 1e-3),
            "acceptance": acc / float(timed_sweeps * N * Nw),
            "gn_iteration_ms": ts, "walker_iterations_per_s": Nw / (min(ts) * 1e-3),
            "local_energy_only_ms": eloc_ms, "local_energy_and_jacobian_ms": jac_ms,
            "variance_per_iteration": var, "lambda_per_iteration": lams,
            "schedule": {"warm_up": 4, "refinement": 8, "polyak_window": 4, "sweeps_per_step": 10,
                         "ms_per_step": sched_ms / 12,
                         "variance_per_step": [h[0] for h in sched],
                         "fresh_sample_variance": {"start": v_start, "polyak_average": v_avg}},
            "oracle": {"walkers": 4, "energy_and_jacobian_s": oracle_s,
                       "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))},
            "oracle_ratio_per_walker": (oracle_s / 4) / (jac_ms * 1e-3 / Nw),
            "parity": {"E_max_abs": float(np.max(np.abs(Eg.cpu().numpy() - refE))),
                       "dE_max_abs": float(np.max(np.abs(dEg.cpu().numpy() - refJ))),
                       "dE_scale": float(np.max(np.abs(refJ)))}}
    print(json.dumps(line), flush=True)


def run_emu64(args):
    """The ISDF fit of the H50 chain (100,000 points, 400 orbitals, N_mu = 2000)
    with fit_mode 0 (FP64 on CUDA cores) and 1 (FP64 products emulated on the
    tensor cores), and one emulated GEMM of the solves' update shape (2000 x
    --emu-n x 128) against torch's FP64 matmul; CUDA events."""
    import torch
    from paper_2607_17314_b300 import api, build, pipeline
    build.build()
    wlw = make_workload("h50_chain")
    b = wlw.basis
    J = api.jastrow_from(wlw.jastrow)
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, wlw.mo_coef, wlw.grid_xyz,
                          wlw.grid_w, wlw.n_mu, wlw.n_occ, J)
    phi, dphi = api.isdf_eval_orbitals(inp.center, inp.powers, inp.exps, inp.coefs, inp.mo_coef,
                                       inp.grid)
    piv = api.isdf_points(phi, dphi, inp.w, inp.n_mu)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        ts, out = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, ts
    (x0, g0, _), t0 = timed(lambda: api.isdf_fit(phi, dphi, piv, fit_mode=0), 1)
    (x1, g1, _), t1 = timed(lambda: api.isdf_fit(phi, dphi, piv, fit_mode=1),
                            max(args.steps, 1) + 1)
    diff = [float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0))] + \
        [float(torch.linalg.norm(g1[c] - g0[c]) / torch.linalg.norm(g0[c])) for c in range(3)]
    del x0, g0, x1, g1
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    A = torch.randn((2000, 128), dtype=torch.float64, device="cuda", generator=gen)
    B = torch.randn((128, args.emu_n), dtype=torch.float64, device="cuda", generator=gen)
    C, tg = timed(lambda: api.isdf_dgemm_emulated(A, B), max(args.warmup, 1) + max(args.steps, 1))
    C0, tr = timed(lambda: A @ B, 3)
    flops = 2.0 * 2000 * args.emu_n * 128
    print(json.dumps({"mode": "emu64", "workload": "h50_chain fit (N_mu = 2000, 400 orbitals, "
                                                   "100,000 points)",
                      "fit_fp64_ms": t0, "fit_emulated_ms": t1[1:],
                      "fit_rel_diff": diff,
                      "gemm": {"shape": [2000, args.emu_n, 128], "emulated_ms": tg[-1],
                               "emulated_tflops_fp64_equiv": flops / (min(tg[1:]) * 1e-3) / 1e12,
                               "torch_fp64_ms": min(tr[1:]),
                               "rel_diff": float(torch.linalg.norm(C - C0) / torch.linalg.norm(C0))}}),
          flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.w_only:
        return run_w_only(args)
    if args.streamed:
        return run_streamed(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.proposer:
        return run_proposer(args)
    if args.vmc:
        return run_vmc(args)
    if args.emu64:
        return run_emu64(args)
    if args.validate:
        return run_validate(args)
    if args.assembly:
        return run_assembly(args)

    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2607_17314_b300 import api, build, pipeline
    build.build()
    wlw = make_workload(args.workload)
    b = wlw.basis
    J = api.jastrow_from(wlw.jastrow)
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, wlw.mo_coef, wlw.grid_xyz,
                          wlw.grid_w, wlw.n_mu, wlw.n_occ, J)
    n_g, n_mu = wlw.n_g, wlw.n_mu
    stream = torch.cuda.current_stream()

    def step(events=None, stage_ms=None):
        return pipeline.run(inp, precision=args.precision, events=events, stage_ms=stage_ms,
                            kchunk=args.kchunk, fit_mode=args.fit_mode)

    for _ in range(max(args.warmup, 0)):
        out = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    events = {}
    stage_ms = []
    launches0 = api.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            out = step(events, stage_ms)
        t_end.record(stream)
        barrier()
    launches = api.kernel_launches() - launches0
    total_ms = t_start.elapsed_time(t_end)

    def stage(name):
        ev = events.get(name, [])
        return [ev[i].elapsed_time(ev[i + 1]) for i in range(0, len(ev), 2)]

    stages = {k: statistics.mean(stage(k)) for k in ("a1", "a2", "a3", "a4", "a5", "a6")}
    a4_ms = stages["a4"]
    ms_step = total_ms / max(args.steps, 1)
    a4_ms, ms_step = aggregate_times(a4_ms, ms_step, world, "cuda")
    flops = w_flops(n_mu, n_g, n_g)
    value = job_tflops(world, flops, a4_ms)

    # dominant kernel: stage-1 tcgen05 contraction (device time from events
    # recorded by the library on the launching stream)
    s1_ms = statistics.mean(x[0] for x in stage_ms)
    s2_ms = statistics.mean(x[1] for x in stage_ms)
    peak, peak_kind = tensor_peak()
    if args.precision == "tf32x3":
        # dense TF32 runs at half the BF16 rate (1.1 vs 2.25 PFLOP/s nominal)
        peak, peak_kind = peak * 0.5, peak_kind + " x 0.5 (nominal TF32/BF16 ratio)"
    s1_tflops = 8.0 * n_mu * n_g * n_g / (s1_ms * 1e-3) / 1e12
    products = 6 if args.precision == "bf16x6" else 3
    ncu = S1_NCU.get(args.precision)
    # DRAM traffic of one launch: the per-(mu, g) figure of the ncu capture of
    # the current kernel (reads of the w xi limbs and the FP64 calG writes both
    # scale with N_mu n_g), or null when the current kernel has not been captured
    traffic = ncu["dram_bytes_per_mu_g"] * n_mu * n_g if ncu else None
    roofline = {"bound": "tensor", "achieved": s1_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": s1_tflops / peak, "traffic": traffic,
                "products_frac": s1_tflops * products / peak,
                "ncu_tensor_pipe_active": ncu["tensor_pipe_active"] if ncu else None,
                "kernel": f"s1_pair_kernel ({args.precision}: {products} tensor-core products per "
                          f"algorithmic MAC)",
                "peak_kind": peak_kind}

    # FP64 GPU path on an outer-grid slice (same inner sum), and accuracy of
    # the tensor-core W over that slice against it
    rows = min(args.fp64_rows, n_g)
    xi, xig = out["xi"], out["xig"]
    ms64 = []
    kb64 = api.KernelBuilder(inp.grid, inp.w, xi, xig, J, "fp64", 0, rows)
    kb64()
    torch.cuda.synchronize()
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); kb64(); e1.record(stream); torch.cuda.synchronize()
        ms64.append(e0.elapsed_time(e1))
    fp64_tflops = w_flops(n_mu, rows, n_g) / (min(ms64) * 1e-3) / 1e12
    kbt = api.KernelBuilder(inp.grid, inp.w, xi, xig, J, args.precision, 0, rows)
    kbt()
    errs = [float(torch.linalg.norm(kbt.W[c] - kb64.W[c]) / torch.linalg.norm(kb64.W[c]))
            for c in range(4)]
    # the TF32 tensor-core arm of the same build (stage 1 kind::tf32 with two
    # TF32 limbs), timed over the whole grid and checked on the FP64 slice
    tf32_arm = None
    if args.precision != "tf32x3":
        kb32 = api.KernelBuilder(inp.grid, inp.w, xi, xig, J, "tf32x3", time_stages=True)
        kb32()
        t32 = []
        for _ in range(2):
            kb32()
            t32.append(float(kb32.stage_ms[0]) + float(kb32.stage_ms[1]))
        del kb32
        kbs = api.KernelBuilder(inp.grid, inp.w, xi, xig, J, "tf32x3", 0, rows)
        kbs()
        e32 = [float(torch.linalg.norm(kbs.W[c] - kb64.W[c]) / torch.linalg.norm(kb64.W[c]))
               for c in range(4)]
        del kbs
        tf32_arm = {"w_build_ms_stages": min(t32),
                    "tflops": w_flops(n_mu, n_g, n_g) / (min(t32) * 1e-3) / 1e12,
                    "w_rel_err_vs_fp64": e32}
    del kbt, kb64
    e_err = sampled_energy_error(api, inp, out, J, args.precision)

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        host = [np.ascontiguousarray(a) for a in (b.center, b.powers, b.exps, b.coefs,
                                                  wlw.mo_coef, wlw.grid_xyz, wlw.grid_w)]
        pinned = [torch.as_tensor(a).pin_memory() for a in host]
        h2d = sum(t.numel() * t.element_size() for t in pinned)
        W_host = torch.empty((4, n_mu, n_mu), dtype=torch.float64).pin_memory()
        d2h = W_host.numel() * 8 + 3 * 8
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            dev = [t.to("cuda", non_blocking=True) for t in pinned]
            inp2 = pipeline.Inputs(dev[0], dev[1].to(torch.int32), dev[2], dev[3], dev[4], dev[5],
                                   dev[6], n_mu, wlw.n_occ, J)
            o2 = pipeline.run(inp2, precision=args.precision, kchunk=args.kchunk,
                              fit_mode=args.fit_mode)
            W_host.copy_(o2["W"], non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms, _ = aggregate_times(e0.elapsed_time(e1) / max(args.steps, 1), 0.0, world, "cuda")
        e2e = {"value": job_tflops(world, flops, e2e_ms), "unit": "TFLOP/s",
               "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        xi_h = out["xi"].cpu().numpy()
        xit_h = out["xig"].cpu().numpy()
        cpu_sample(wlw, 4, xi_h, xit_h)
        dt = cpu_sample(wlw, args.cpu_rows, xi_h, xit_h)
        cpu = {"value": w_flops(n_mu, args.cpu_rows, n_g) / dt / 1e12, "unit": "TFLOP/s",
               "cores": host_cores(), "kind": "oracle",
               "sample": f"FP64 oracle W build (stages 1+2) for {args.cpu_rows} of {n_g} outer grid "
                         f"points x all {n_g} inner points, N_mu={n_mu}, {dt:.1f} s"}

    if rank == 0:
        E = out["E"]
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": run_config(args, wlw, world),
            "stages_ms": stages, "w_build_ms": a4_ms, "s1_ms": s1_ms, "s2_ms": s2_ms,
            "fp64_gpu": {"tflops": fp64_tflops, "slice_outer_points": rows,
                         "speedup_tc_over_fp64": value / fp64_tflops,
                         "w_rel_err_tc_vs_fp64": errs},
            "tf32x3_arm": tf32_arm,
            "energies_ha": {"E_K": E[0], "E_dU": E[1], "E0": E[2]},
            "energies_err_ha_vs_fp64_gpu": e_err,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
