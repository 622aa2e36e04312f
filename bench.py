"""Benchmark of the ISIS force step on one GB300 (or N independent replicas).

One step is the whole hot path at 512^3 in a 256 Mpc/h box:
  CIC deposit of 512^3 Zel'dovich-displaced particles (seeded, P(k) ~ k^-2,
  0.5-cell rms displacement) -> Poisson solve -> symmetron FAS solve
  (a = 1, a_SSB = 0.5, lambda0 = 1 Mpc/h, beta = 1) -> Hu-Sawicki f(R) FAS
  solve (n = 1, |f_R0| = 1e-5) -> forces of both models on every particle.
The three solves run the FP32 correction cycles inside the FP64 defect-
correction loop to a relative residual of 1e-8.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "symmetron/f(R) 512³ FAS solve time to residual 1e-8; smoother HBM GB/s"
# The arithmetic of the step: FP32 V-cycles; the fine-grid residual of the defect correction and the field it
# carries in float-float (pairs of FP32 numbers, about 48 significant bits; FP32 instructions); the coarsest
# Newton solves and the returned fields in FP64.
DTYPE = "f32 (V-cycles) + float-float ~48-bit (outer residual, carried field) + f64 (coarsest Newton, returned field)"
L2_BYTES = 129 * 2 ** 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--box", type=float, default=256.0)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-poisson", type=int, default=4, help="FP32 cycles per FP64 outer iteration")
    ap.add_argument("--inner-sym", type=int, default=4)
    ap.add_argument("--inner-fofr", type=int, default=4)
    ap.add_argument("--ncoarse", type=int, default=2, help="coarsest grid (dense Newton): 2 or 4")
    ap.add_argument("--nu1", type=int, default=2, help="pre-smoothing sweeps per level")
    ap.add_argument("--nu2", type=int, default=1, help="post-smoothing sweeps per level")
    ap.add_argument("--sample-N", type=int, default=128, help="grid of the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-ref", action="store_true", help="skip the FP64-solver comparison")
    ap.add_argument("--fmg", type=int, default=1, choices=[0, 1],
                    help="start the FP32 phase of each solve with nested iteration (full multigrid)")
    ap.add_argument("--guess", default="background", choices=["net", "background"],
                    help="symmetron initial guess of the timed step: the background field (the faster start on this "
                         "density, see the learned_guess record) or the trained U-Net")
    ap.add_argument("--no-halo-record", action="store_true",
                    help="skip the solves on the lognormal-plus-halo density (outside the timed region)")
    ap.add_argument("--no-guess-record", action="store_true",
                    help="skip the learned guess's record (net start against background start)")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1307_6748_gb300", "weights", "unet_symmetron.npz"))
    return ap.parse_args(argv)


def workload(args):
    return {"workload": f"force step: CIC deposit of {args.N}^3 Zel'dovich particles, Poisson + symmetron + "
                        f"f(R) FAS solves (FP32 cycles in FP64 defect correction, residual {args.tol:g}), "
                        f"forces of both models",
            "N": args.N, "box_mpc_h": args.box, "particles": args.N ** 3, "tol": args.tol,
            "residual_floor": "float-float residual: about 1e-9 of ref for f(R) (u held to 48 bits), far below "
                              "for Poisson and the symmetron",
            "symmetron": {"a": 1.0, "a_ssb": 0.5, "lambda0": 1.0, "beta": 1.0},
            "fofr": {"n": 1, "fR0_abs": 1e-5}, "cycle": f"V({args.nu1},{args.nu2}), coarsest {args.ncoarse}^3 dense Newton"
                                                        + (", FP32 phase started by nested iteration" if args.fmg else ""),
            "inner_cycles": {"poisson": args.inner_poisson, "symmetron": args.inner_sym, "fofr": args.inner_fofr},
            "initial_guess": {"symmetron": "U-Net (trained at 1 Mpc/h cells) on the 8-cell mean density, "
                                           "prolongated trilinearly" if args.guess == "net" else "background",
                              "fofr": "background field", "poisson": "zero"},
            "l2": "inputs larger than L2 (each 512^3 field is 0.5-1 GB), no flush",
            "parallelism": "replicas (one independent problem per GPU)"}


# ---------------------------------------------------------------------------
# Ranks (one process per GPU): each rank solves its own seeded problem (replicas)
# ---------------------------------------------------------------------------

def replica_seed(rank: int) -> int:
    """Seed of rank `rank`'s Zel'dovich particles: every replica solves its own problem."""
    return 3 + 1000 * rank


def max_over_ranks(v: float, dist, dev) -> float:
    """The largest v over all ranks (v itself without a process group)."""
    if dist is None:
        return v
    import torch
    tt = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# ---------------------------------------------------------------------------
# The timed step
# ---------------------------------------------------------------------------

class ForceStep:
    """One force step on device-resident particles: CIC deposit, the Poisson, symmetron and f(R) solves (FP32
    cycles in FP64 defect correction), the forces of both models.  The solver options here are the launch
    configuration the benchmark times; the full-size GPU test runs the same object."""

    def __init__(self, args, dev, npart: int):
        import torch

        from paper_1307_6748_gb300 import isis, unet
        self.isis = isis
        N, box = args.N, args.box
        self.tol = args.tol
        self.grid = isis.Grid(N, box)
        self.psym = isis.Params(lambda0=1.0, beta=1.0, a_ssb=0.5)
        self.pfr = isis.Params(n=1, fR0_abs=1e-5)
        self.a = 1.0
        f64 = dict(dtype=torch.float64, device=dev)
        self.eta, self.Phi, self.chi, self.u = (torch.empty((N,) * 3, **f64) for _ in range(4))
        self.g = [torch.empty(npart, device=dev, dtype=torch.float32) for _ in range(6)]

        def opts(inner, init=isis.ISIS_INIT_BACKGROUND):
            return isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=inner, init=init, n_coarsest=args.ncoarse,
                             fmg=args.fmg, nu1=args.nu1, nu2=args.nu2)
        self.o_poi, self.o_sym, self.o_fr = opts(args.inner_poisson), opts(args.inner_sym), opts(args.inner_fofr)
        self.net, self.pooled = None, False
        if args.guess == "net":
            # the net is convolutional: it runs at its training cell size (1 Mpc/h), here on 8-cell means
            meta = unet.UNet.meta(args.weights)
            h, h_net = box / N, float(meta.get("h", 1.0))
            if abs(2 * h - h_net) < 1e-9 * h_net:
                self.pooled = True
            elif abs(h - h_net) > 1e-9 * h_net:
                raise SystemExit(f"bench: the net was trained at {h_net} Mpc/h cells; this grid has {h} Mpc/h")
            self.net = unet.UNet.load(args.weights, device=dev)
            self.o_sym = opts(args.inner_sym, isis.ISIS_INIT_INPUT)
        self.stream = torch.cuda.current_stream()
        self.infos = {}

    def __call__(self, xx, yy, zz, ev=None):
        isis, st, infos = self.isis, self.stream, self.infos
        grid, a, eta, Phi, chi, u, g = self.grid, self.a, self.eta, self.Phi, self.chi, self.u, self.g
        if ev:
            ev[0].record(st)
        isis.isis_cic_deposit(grid, xx, yy, zz, eta)
        if ev:
            ev[1].record(st)
        infos["poisson"] = isis.isis_poisson_solve(grid, a, eta, Phi, tol=self.tol, opts=self.o_poi)
        if ev:
            ev[2].record(st)
        if self.net is not None:
            self.net.guess(eta, a, self.psym.a_ssb, chi, pooled=self.pooled)
        if ev:
            ev[3].record(st)
        infos["symmetron"] = isis.isis_scalar_solve(isis.ISIS_SYMMETRON, self.psym, grid, a, eta, chi, tol=self.tol,
                                                    opts=self.o_sym)
        if ev:
            ev[4].record(st)
        infos["fofr"] = isis.isis_scalar_solve(isis.ISIS_FOFR_HS, self.pfr, grid, a, eta, u, tol=self.tol,
                                               opts=self.o_fr)
        if ev:
            ev[5].record(st)
        isis.isis_fifth_force(isis.ISIS_SYMMETRON, self.psym, grid, a, Phi, chi, xx, yy, zz, out=g[0:3])
        isis.isis_fifth_force(isis.ISIS_FOFR_HS, self.pfr, grid, a, Phi, u, xx, yy, zz, out=g[3:6])
        if ev:
            ev[6].record(st)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.stop = threading.Event()
        self.th = threading.Thread(target=self.run, daemon=True)

    def run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                return
            self.stop.wait(0.2)

    def __enter__(self):
        self.th.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return None
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[4:8]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# The oracle as CPU baseline / reference arm
# ---------------------------------------------------------------------------

def oracle_step(sample_N: int, box_full: float, N_full: int, tol: float, cache={}):
    """One oracle force step on a sample grid with the same cell size; returns seconds."""
    import numpy as np

    import oracle
    from paper_1307_6748_gb300 import isis, synth
    box = box_full * sample_N / N_full
    if sample_N not in cache:
        cache[sample_N] = tuple(v.numpy() for v in synth.zeldovich(sample_N, box, seed=3))
    x, y, z = cache[sample_N]
    t0 = time.perf_counter()
    eta = oracle.cic_deposit(sample_N, x, y, z)
    Pp = oracle.Problem(oracle.POISSON, sample_N, box)
    Ps = oracle.Problem(oracle.SYMMETRON, sample_N, box, a=1.0, a_ssb=0.5)
    Pf = oracle.Problem(oracle.FOFR, sample_N, box, a=1.0, fR0_abs=1e-5)
    shape = (sample_N,) * 3
    rp = oracle.solve(Pp, eta, np.zeros(shape), tol=tol)
    rs = oracle.solve(Ps, eta, np.full(shape, oracle.background_field(oracle.SYMMETRON, 1.0, a_ssb=0.5)), tol=tol)
    rf = oracle.solve(Pf, eta, np.full(shape, oracle.background_field(oracle.FOFR, 1.0, fR0_abs=1e-5)), tol=tol)
    oracle.fifth_force(Ps, rp.phi, rs.phi, x, y, z)
    oracle.fifth_force(Pf, rp.phi, rf.phi, x, y, z)
    return time.perf_counter() - t0


def oracle_threads() -> int:
    n = os.environ.get("OMP_NUM_THREADS")
    if not n:
        n = str(os.cpu_count() or 1)
        os.environ["OMP_NUM_THREADS"] = n  # read by libgomp when the oracle library loads
    return int(n)


def cpu_baseline(args, steps=1):
    cores = oracle_threads()
    import oracle
    oracle.build()
    scale = (args.N / args.sample_N) ** 3
    times = [oracle_step(args.sample_N, args.box, args.N, args.tol) for _ in range(steps)]
    v = statistics.median(times) * 1e3 * scale
    return {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"estimate: {args.sample_N}^3 sample x {scale:g}. The full oracle force step (deposit, "
                      f"3 FP64 FAS solves to {args.tol:g}, forces) timed on {args.sample_N}^3 with the same "
                      f"recipe and cell size (median of {steps}), scaled by cell count to {args.N}^3"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = oracle_threads()
    import oracle
    oracle.build()
    scale = (args.N / args.sample_N) ** 3
    for _ in range(args.warmup):
        oracle_step(args.sample_N, args.box, args.N, args.tol)
    ts = [oracle_step(args.sample_N, args.box, args.N, args.tol) for _ in range(args.steps)]
    ms = statistics.mean(ts) * 1e3 * scale
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload(args),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"estimate: {args.sample_N}^3 sample x {scale:g}. Each step runs the oracle "
                                       f"force step on {args.sample_N}^3 (same recipe, same cell size); value = "
                                       f"mean of {args.steps} x {scale:g} by cell count",
                             "sample_ms_per_step": ms / scale},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def copy_times(cev: dict, steps: int) -> dict:
    """Per loop (serial, pipelined) and direction: the copies' event time per step (mean) and the slowest step's.
    Against the step time they show whether the link, not the schedule, set the end-to-end figure: a copy that
    outlasts a step cannot hide behind it."""
    out = {}
    for loop, evs in cev.items():
        for kind in ("h2d", "d2h"):
            ts = [a.elapsed_time(b) for k, a, b in evs if k == kind]
            if not ts:
                continue
            # the d2h of one step is two groups in the pipelined loop (each model's forces)
            per = len(ts) / steps
            steps_ms = [sum(ts[i:i + round(per)]) for i in range(0, len(ts), max(1, round(per)))]
            out[f"{loop}_{kind}"] = {"mean": sum(ts) / steps, "max_step": max(steps_ms)}
    return out


def copy_rates(h_src, d_dst, h_dst, d_src, stream) -> dict:
    """This box's pinned-host link, measured with the step's own buffers (one particle coordinate, one force
    component): GB/s host-to-device, device-to-host, and both directions at once on two streams."""
    import torch
    nb = d_dst.numel() * d_dst.element_size()
    other = torch.cuda.Stream()

    def timed(fn, reps=3):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
        return best

    def both():
        other.wait_stream(stream)
        with torch.cuda.stream(other):
            h_dst.copy_(d_src, non_blocking=True)
        d_dst.copy_(h_src, non_blocking=True)
        stream.wait_stream(other)

    h2d = timed(lambda: d_dst.copy_(h_src, non_blocking=True))
    d2h = timed(lambda: h_dst.copy_(d_src, non_blocking=True))
    bo = timed(both)
    return {"h2d": nb / h2d / 1e9, "d2h": nb / d2h / 1e9, "both": 2 * nb / bo / 1e9, "bytes": nb}


def learned_guess(args, dev, S, barrier) -> dict:
    """The step's symmetron solve started from the trained U-Net's guess against the background start, on the
    step's own density and solver options, outside the timed region (CUDA events, one warm-up of each): the
    inference time, and the cycles and solve time of each start."""
    import torch

    from paper_1307_6748_gb300 import isis, unet
    meta = unet.UNet.meta(args.weights)
    h, h_net = args.box / args.N, float(meta.get("h", 1.0))
    pooled = abs(2 * h - h_net) < 1e-9 * h_net
    if not pooled and abs(h - h_net) > 1e-9 * h_net:
        return {"skipped": f"the net was trained at {h_net} Mpc/h cells; this grid has {h} Mpc/h"}
    net = unet.UNet.load(args.weights, device=dev)
    st = S.stream

    def opts(init):
        return isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=args.inner_sym, init=init,
                         n_coarsest=args.ncoarse, fmg=args.fmg, nu1=args.nu1, nu2=args.nu2)
    rec = {}
    for rep in range(2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        barrier()
        ev[0].record(st)
        net.guess(S.eta, S.a, S.psym.a_ssb, S.chi, pooled=pooled)
        ev[1].record(st)
        i_net = isis.isis_scalar_solve(isis.ISIS_SYMMETRON, S.psym, S.grid, S.a, S.eta, S.chi, tol=S.tol,
                                       opts=opts(isis.ISIS_INIT_INPUT))
        ev[2].record(st)
        barrier()
        ev[3].record(st)
        i_bg = isis.isis_scalar_solve(isis.ISIS_SYMMETRON, S.psym, S.grid, S.a, S.eta, S.chi, tol=S.tol,
                                      opts=opts(isis.ISIS_INIT_BACKGROUND))
        ev[4].record(st)
        barrier()
        rec = {"inference_ms": ev[0].elapsed_time(ev[1]), "net_solve_ms": ev[1].elapsed_time(ev[2]),
               "net_cycles": i_net.cycles, "background_solve_ms": ev[3].elapsed_time(ev[4]),
               "background_cycles": i_bg.cycles}
    rec["net_total_ms"] = rec["inference_ms"] + rec["net_solve_ms"]
    rec["net_saves_ms"] = rec["background_solve_ms"] - rec["net_total_ms"]
    rec["cycles_saved"] = rec["background_cycles"] - rec["net_cycles"]
    return rec


def halo_record(args, dev, S, barrier, peak: float) -> dict:
    """The metric's solves on the lognormal-plus-halo density (sigma 1.5, 32 NFW haloes of 1e13-1e15 Msun/h,
    c = 5) at the step's grid and box: the symmetron at a = 1.0 and 0.6 (close to symmetry breaking) from its
    background field, and f(R) from the cell-wise uniform-density solution (ISIS_INIT_LOCAL: from the background
    the f(R) iterate overshoots without bound inside the haloes), with the step's options, timed after one warm-up
    with CUDA events, outside the timed region.  solve_frac as in the roofline record."""
    import torch

    from paper_1307_6748_gb300 import isis, synth
    eta = synth.nfw_eta(args.N, args.box, 1.5, seed=11).to(device=dev, dtype=torch.float64)
    phi = torch.empty_like(eta)
    per_cycle = 6 * 4 * (8.0 / 7.0) * args.N ** 3
    out = {"density": "lognormal sigma 1.5 (seed 11) plus 32 NFW haloes (seed 2)"}
    cases = (("symmetron_a1.0", isis.ISIS_SYMMETRON, S.psym, 1.0, args.inner_sym, isis.ISIS_INIT_BACKGROUND),
             ("symmetron_a0.6", isis.ISIS_SYMMETRON, S.psym, 0.6, args.inner_sym, isis.ISIS_INIT_BACKGROUND),
             ("fofr", isis.ISIS_FOFR_HS, S.pfr, 1.0, args.inner_fofr, isis.ISIS_INIT_LOCAL))
    for name, model, par, a, inner, init in cases:
        o = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=inner, init=init,
                      n_coarsest=args.ncoarse, fmg=args.fmg, nu1=args.nu1, nu2=args.nu2)
        try:
            for _ in range(2):
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(S.stream)
                info = isis.isis_scalar_solve(model, par, S.grid, a, eta, phi, tol=args.tol, opts=o)
                e1.record(S.stream)
                barrier()
            ms = e0.elapsed_time(e1)
            out[name] = {"ms": ms, "cycles": info.cycles, "outer": info.outer,
                         "res_rel": info.res_final / info.res_ref,
                         "solve_frac": per_cycle * info.cycles / (ms * 1e-3 * peak * 1e9)}
        except isis.IsisError as err:
            out[name] = {"error": str(err)}
    return out


# ---------------------------------------------------------------------------
# Roofline figures
# ---------------------------------------------------------------------------

# Sources of the fine-grid smoother and its operators: the DRAM traffic recorded in profiles/ holds only while
# they are unchanged.
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1307_6748_gb300", "csrc", f) for f in ("isis_kernels.cuh", "isis_model.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_smooth_fine_512.md")


def sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind: str):
    """DRAM bytes per launch of `kind` at 512^3 from the committed ncu summary, or None when the summary has no
    figure for it or the kernel sources changed since it was taken.  The summary's machine-readable lines read
    `traffic: <kind> <bytes per launch> <sources sha>`."""
    try:
        with open(TRAFFIC_FILE) as f:
            lines = [ln.split() for ln in f if ln.startswith("traffic: ")]
    except OSError:
        return None
    sha = sources_sha()
    for parts in lines:
        if len(parts) == 4 and parts[1] == kind and parts[3] == sha:
            return float(parts[2])
    return None


def roofline_line(prof: dict, peak: float, peak_source: str, steps: int) -> dict:
    """The dominant kernel (by summed event time, each model and form apart) against the HBM peak, and every
    instantiation of the fine-grid smoother beside it.  achieved = algorithmic bytes / event time."""
    name, (nl, kms, kbytes) = max(prof.items(), key=lambda kv: kv[1][1])
    achieved = kbytes / (kms * 1e-3) / 1e9
    per = {}
    for k, (n, ms, by) in sorted(prof.items()):
        if k.startswith("smooth_fine[") and ms > 0:
            a = by / (ms * 1e-3) / 1e9
            per[k] = {"achieved": a, "frac": a / peak, "launches_per_step": n / steps, "ms_per_step": ms / steps,
                      "avg_launch_us": ms * 1e3 / n, "bytes_per_launch": by / n,
                      "traffic": recorded_traffic(k)}
    allf = [v for k, v in prof.items() if k.startswith("smooth_fine[")]
    agg = None
    if allf:
        ms = sum(v[1] for v in allf)
        by = sum(v[2] for v in allf)
        agg = {"achieved": by / (ms * 1e-3) / 1e9, "frac": by / (ms * 1e-3) / 1e9 / peak}
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": recorded_traffic(name), "launches": nl,
            "avg_launch_us": kms * 1e3 / nl, "bytes_per_launch": kbytes / nl, "peak_source": peak_source,
            "measured": f"CUDA events around every launch (on its stream) in {steps} steps run right after the timed "
                        f"region; algorithmic bytes from the library's per-launch accounting",
            "smooth_fine_by_instantiation": per, "smooth_fine_all": agg}


def solve_fractions(N: int, infos: dict, breakdown: dict, peak: float) -> dict:
    """Solve-level roofline: the algorithmic minimum of a V-cycle in FP32 (two fused passes per level visit, each
    reading x and eta and writing x: 6 x 4 bytes per cell, x 8/7 over the levels) times the cycles, over the
    solve's time (CUDA events in the timed region) times the HBM peak.  The FP64 outer residual and update
    passes are not in the minimum, so they count against the fraction."""
    per_cycle = 6 * 4 * (8.0 / 7.0) * N ** 3
    out = {}
    for k, info in infos.items():
        t = breakdown[k] * 1e-3
        out[k] = {"cycles": info.cycles, "bytes_per_cycle": per_cycle, "ms": breakdown[k],
                  "frac": per_cycle * info.cycles / (t * peak * 1e9)}
    return out


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_1307_6748_gb300 import build, isis, synth
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    N, box = args.N, args.box
    x, y, z = synth.zeldovich(N, box, seed=replica_seed(rank), device=dev)
    npart = x.numel()
    S = ForceStep(args, dev, npart)
    grid, psym, pfr, a = S.grid, S.psym, S.pfr, S.a
    eta, Phi, chi, u, g = S.eta, S.Phi, S.chi, S.u, S.g
    o_poi, o_sym, o_fr, net, pooled = S.o_poi, S.o_sym, S.o_fr, S.net, S.pooled
    stream, infos, step = S.stream, S.infos, S

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(x, y, z)
    barrier()

    # timed region: device-resident inputs, no per-launch events (they add about 6% to a step)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    isis.prof_reset()
    with ClockSampler(local) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(args.steps):
            step(x, y, z, evs[s])
        t1.record(stream)
        barrier()
    launches = isis.launch_count()
    # per-kernel durations: the same steps again, every launch bracketed by CUDA events on its stream
    isis.prof_reset()
    isis.prof_enable(True)
    for s in range(args.steps):
        step(x, y, z)
    barrier()
    isis.prof_enable(False)
    prof = isis.prof_read()
    total_ms = t0.elapsed_time(t1)
    ms = max_over_ranks(total_ms / args.steps, dist, dev)
    parts = ["deposit", "poisson", "guess", "symmetron", "fofr", "forces"]
    breakdown = {p: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, p in enumerate(parts)}

    # end to end: positions from pinned host memory, forces back to pinned host memory, every step
    e2e = None
    if not args.no_e2e:
        # the library's page-locked host buffers (huge-page backed where the kernel grants it)
        hx, hy, hz = (isis.host_empty(npart) for _ in range(3))
        for h, v in zip((hx, hy, hz), (x, y, z)):
            h.copy_(v)
        hg = [isis.host_empty(npart) for _ in range(6)]
        pos = [tuple(torch.empty_like(x) for _ in range(3)) for _ in range(2)]
        gb = [g, [torch.empty_like(t) for t in g]]

        def tev():
            return torch.cuda.Event(enable_timing=True)

        # copy groups of each loop, bracketed by events on the copying stream: (kind, start, end)
        cev = {"serial": [], "pipelined": []}

        def copies(loop, kind, st, pairs):
            a, b = tev(), tev()
            a.record(st)
            for dst, src in pairs:
                dst.copy_(src, non_blocking=True)
            b.record(st)
            cev[loop].append((kind, a, b))

        # one untimed pass of every copy first: the first DMA to or from a freshly pinned buffer runs slow
        for bufs in pos:
            for dst, src in zip(bufs, (hx, hy, hz)):
                dst.copy_(src, non_blocking=True)
        for bufs in gb:
            for dst, src in zip(hg, bufs):
                dst.copy_(src, non_blocking=True)

        # serial: every copy on the compute stream, before and after its step
        barrier()
        e0, e1 = tev(), tev()
        e0.record(stream)
        for s in range(args.steps):
            copies("serial", "h2d", stream, zip(pos[0], (hx, hy, hz)))
            step(*pos[0])
            copies("serial", "d2h", stream, zip(hg, g))
        e1.record(stream)
        barrier()
        serial = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)

        # pipelined: copies on a second stream, positions and forces double-buffered; step s's positions
        # arrive while step s-1 computes, and each model's forces leave as soon as they exist
        cs = torch.cuda.Stream()
        h2d = [torch.cuda.Event() for _ in range(2)]
        pos_free = [torch.cuda.Event() for _ in range(2)]
        g_free = [torch.cuda.Event() for _ in range(2)]
        barrier()
        e0.record(stream)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            copies("pipelined", "h2d", cs, zip(pos[0], (hx, hy, hz)))
            h2d[0].record(cs)
        for s in range(args.steps):
            b = s % 2
            if s + 1 < args.steps:
                with torch.cuda.stream(cs):
                    if s >= 1:
                        cs.wait_event(pos_free[1 - b])
                    copies("pipelined", "h2d", cs, zip(pos[1 - b], (hx, hy, hz)))
                    h2d[1 - b].record(cs)
            stream.wait_event(h2d[b])
            if s >= 2:
                stream.wait_event(g_free[b])
            xx, yy, zz = pos[b]
            isis.isis_cic_deposit(grid, xx, yy, zz, eta)
            infos["poisson"] = isis.isis_poisson_solve(grid, a, eta, Phi, tol=args.tol, opts=o_poi)
            if net is not None:
                net.guess(eta, a, psym.a_ssb, chi, pooled=pooled)
            infos["symmetron"] = isis.isis_scalar_solve(isis.ISIS_SYMMETRON, psym, grid, a, eta, chi, tol=args.tol,
                                                        opts=o_sym)
            isis.isis_fifth_force(isis.ISIS_SYMMETRON, psym, grid, a, Phi, chi, xx, yy, zz, out=gb[b][0:3])
            ev = torch.cuda.Event()
            ev.record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev)
                copies("pipelined", "d2h", cs, zip(hg[0:3], gb[b][0:3]))
            infos["fofr"] = isis.isis_scalar_solve(isis.ISIS_FOFR_HS, pfr, grid, a, eta, u, tol=args.tol, opts=o_fr)
            isis.isis_fifth_force(isis.ISIS_FOFR_HS, pfr, grid, a, Phi, u, xx, yy, zz, out=gb[b][3:6])
            pos_free[b].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(pos_free[b])
                copies("pipelined", "d2h", cs, zip(hg[3:6], gb[b][3:6]))
                g_free[b].record(cs)
        stream.wait_stream(cs)
        e1.record(stream)
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
        e2e = {"value": ems, "unit": "ms", "h2d_bytes_per_step": 3 * npart * 4, "d2h_bytes_per_step": 6 * npart * 4,
               "copies": "on a second stream, positions and forces double-buffered: step s's positions are copied "
                         "while step s-1 computes, each model's forces are read back while the next solve runs; "
                         "host buffers from isis_host_alloc (page-locked, huge-page backed)",
               "serial_value": serial, "copy_ms_per_step": copy_times(cev, args.steps),
               "copy_rates_gbs": copy_rates(hx, x, hg[0], g[0], stream)}

    # roofline of the dominant kernel (kind and instantiation, by summed event time)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    roofline = roofline_line(prof, hbm_peak, "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks
                             else "fallback 6800 GB/s", args.steps)
    roofline["solve_frac"] = solve_fractions(args.N, infos, breakdown, hbm_peak)
    kernels = {k: {"launches": v[0], "ms_per_step": v[1] / args.steps,
                   "GBps": (v[2] / (v[1] * 1e-3) / 1e9) if v[1] > 0 else None} for k, v in prof.items()}

    # the mixed-precision solves against the plain FP64 solver on the same GPU and density (outside the timed
    # region; each solve once after one of its own warm-ups).  Arms: the FP64 solver in V(2,2) and in the
    # benchmark's own cycle shape V(nu1,nu2); the mixed path in that shape without and with the nested-iteration
    # start.  speedup_same_cycle compares the FP64 and mixed arms of one cycle shape, neither with nested
    # iteration (which only the mixed path has); speedup is the FP64 V(2,2) arm against the benchmarked setting.
    vs_fp64 = None
    if not args.no_fp64_ref:
        vs_fp64 = {"cycle": f"V({args.nu1},{args.nu2})"}
        arms = (("fp64_v22", isis.ISIS_F64, 2, 2, 0), ("fp64", isis.ISIS_F64, args.nu1, args.nu2, 0),
                ("refine64_nofmg", isis.ISIS_F32_REFINE64, args.nu1, args.nu2, 0),
                ("refine64", isis.ISIS_F32_REFINE64, args.nu1, args.nu2, args.fmg))
        for name, prec_inner in (("poisson", args.inner_poisson), ("symmetron", args.inner_sym),
                                 ("fofr", args.inner_fofr)):
            row = {}
            for label, prec, nu1, nu2, fmg in arms:
                o = isis.Opts(prec=prec, inner_cycles=prec_inner, init=isis.ISIS_INIT_BACKGROUND,
                              n_coarsest=args.ncoarse, max_cycles=60, fmg=fmg, nu1=nu1, nu2=nu2)
                out = {"poisson": Phi, "symmetron": chi, "fofr": u}[name]
                for rep in range(2):
                    barrier()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    if name == "poisson":
                        info = isis.isis_poisson_solve(grid, a, eta, out, tol=args.tol, opts=o)
                    else:
                        m = isis.ISIS_SYMMETRON if name == "symmetron" else isis.ISIS_FOFR_HS
                        info = isis.isis_scalar_solve(m, psym if name == "symmetron" else pfr, grid, a, eta, out,
                                                      tol=args.tol, opts=o)
                    e1.record(stream)
                    barrier()
                row[label + "_ms"] = e0.elapsed_time(e1)
                row[label + "_cycles"] = info.cycles
            row["speedup"] = row["fp64_v22_ms"] / row["refine64_ms"]
            row["speedup_same_cycle"] = row["fp64_ms"] / row["refine64_nofmg_ms"]
            vs_fp64[name] = row

    guess_rec = None
    if not args.no_guess_record and os.path.exists(args.weights):
        guess_rec = learned_guess(args, dev, S, barrier)
    halo_rec = None
    if not args.no_halo_record:
        halo_rec = halo_record(args, dev, S, barrier, hbm_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE, "data": "synthetic", "config": workload(args),
                "breakdown_ms": breakdown,
                "solves": {k: {"cycles": v.cycles, "outer": v.outer, "res_rel": v.res_final / v.res_ref}
                           for k, v in infos.items()},
                "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary()}
        if vs_fp64 is not None:
            line["vs_fp64_solver"] = vs_fp64
        if guess_rec is not None:
            line["learned_guess"] = guess_rec
        if halo_rec is not None:
            line["halo_density_solves"] = halo_rec
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
