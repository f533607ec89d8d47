#!/usr/bin/env python
"""Benchmark of the residual / RK-stage path: grid-point-stage updates per second.

One step = one low-storage RK3 step (3 stages of: ghost fill, primitives, characteristic TENO5
flux differences in x, y, z, viscous fluxes, viscous divergence fused with the register update)
over the whole grid.  Workload: 3D Taylor-Green vortex, 256^3 periodic, Ma 1.25, Re 1600,
Pr 0.72, TENO5 characteristic reconstruction in all directions + 4th-order central viscous
terms, analytic initial field.  Three forms are timed on the same workload: mixed precision with
the learned TENO/central gate (the headline ``value``; the sensor is first trained on the GPU from
TENO labels of coarse TGV snapshots), mixed precision alone (FP32 reconstruction arithmetic, FP64
state and RK registers), and plain FP64, with the relative L2 difference of each state against the
FP64 state after the same steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 256]
                    [--workload tgv|sbli]

``--workload ensemble`` times 64 seeded four-quadrant 2D Riemann problems (sizes drawn from
128^2..1024^2, TENO5, mixed precision) advanced together through osbli_ensemble_* (one launch per
phase over all members, one graph per step, autotuned chunk), beside the same members stepped on
their own handles one after another and the batched plain FP64 form.

``--workload sbli`` times the shock / boundary-layer box instead (512x256x64, Mach 2, Re 1e4,
tanh-stretched wall-normal grid, isothermal wall, similarity inflow, 10-degree oblique shock on
the top boundary, periodic span), with the sensor trained on TGV and reduced-box snapshots.

Prints one JSON line (rank 0).  ``value`` is device-timed (CUDA events on the solver's stream,
inputs resident in HBM); ``e2e`` repeats the metric through the C ABI with page-locked host
buffers, host<->device copies inside the timed region.  Under torchrun every rank runs its own
replica on its own GPU (the method has no data exchange between replicas): ``value`` is the
sum over ranks of points x stages / max-over-ranks time.  ``--impl reference`` times the CPU
oracle on the host cores (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2007_14933_b300 import inputs as I  # noqa: E402

METRIC = "Mpoint-stage updates/s, mixed+learned vs plain FP64 at matched L2 error"
UNIT = "Mpoint-stage/s"
# Algorithmic FP64 operations per grid point per direction of one convective launch (interface
# flux + flux difference), counted from the arithmetic of the method (fma = 2, div/sqrt/rsqrt =
# 1; comparisons and abs not counted).  Breakdown in the design notes.
FLOPS_CONV_POINT_DIR = {I.TENO5: 1379.0, I.WENO5JS: 1279.0, I.WENO5Z: 1359.0, I.CENTRAL4: 63.0,
                        I.TENO6: 1889.0}
# central 4th-order interface flux in delta form (three node flux differences by the product
# rule, the 5-point combination) + flux difference
FLOPS_CENTRAL_DELTA = 135.0
SCHEME_NAME = {I.TENO5: "TENO5", I.WENO5JS: "WENO5-JS", I.WENO5Z: "WENO5-Z", I.CENTRAL4: "central4",
               I.TENO6: "TENO6"}


def max_over_ranks(x, dist, device):
    """The job's time is its slowest rank's: the largest x over the ranks (x itself when dist is
    None).  device: where the reduction tensor lives (cuda for NCCL, cpu for gloo)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points_per_rank, steps, world, seconds, stages=3):
    """Whole-job Mpoint-stage/s: every rank advances its own replica of points_per_rank points
    (weak scaling) by `steps` RK steps of `stages` stages in `seconds` (the slowest rank's)."""
    return points_per_rank * stages * steps * world / seconds / 1e6


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0     # the profiling recipe's fallback


HBM_GBS = _measured_hbm()

# dram__bytes_read.sum + dram__bytes_write.sum per interior point of one launch, from ncu captures
# of the same kernel on a smaller grid (traffic grows with the points processed)
DRAM_BYTES_PER_POINT = {
    "k_conv_delta_tile": (104.8, "ncu capture of k_conv_delta_tile<2,2> in the bench at --n 160 (learned "
                                 "form, 5.2 % of cells gated): dram__bytes_read.sum 358.8 MB + "
                                 "dram__bytes_write.sum 70.2 MB per launch over 4.096 M points, scaled to "
                                 "this grid"),
    "k_conv_delta_xy": (90.4, "ncu capture of k_conv_delta_xy in the bench at --n 160 (learned form, 5.2 % "
                              "of cells gated): dram__bytes_read.sum 294.0 MB + dram__bytes_write.sum 76.3 "
                              "MB per launch over 4.096 M points, scaled to this grid"),
    "k_conv_delta_x_win": (78.2, "ncu capture of k_conv_delta_x_win<2> in the bench at --n 160 (learned "
                                 "form): dram__bytes_read.sum 251.0 MB + dram__bytes_write.sum 69.1 MB per "
                                 "launch over 4.096 M points, scaled to this grid"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv", choices=["tgv", "sbli", "ensemble"],
                    help="tgv: Taylor-Green vortex n^3 (headline); sbli: shock / boundary-layer box "
                         "512x256x64; ensemble: 64 seeded 2D Riemann problems 128^2..1024^2")
    ap.add_argument("--seed", type=int, default=0, help="ensemble seed")
    ap.add_argument("--n", type=int, default=256, help="TGV grid points per direction")
    ap.add_argument("--scheme", type=int, default=I.TENO5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain", action="store_true", help="time the plain FP64 form only")
    ap.add_argument("--mixed", action="store_true", help="time the mixed form only")
    ap.add_argument("--no-sensor", action="store_true", help="skip the learned-sensor form")
    ap.add_argument("--forms", default=None, help="comma list of forms to time (learned, mixed, fp64)")
    ap.add_argument("--sensor-steps", type=int, default=3000, help="Adam steps of the sensor training")
    ap.add_argument("--train-fine", type=int, default=1,
                    help="TGV: add TENO labels of the run's own grid at t = 1.5 and 2.0 to the training set")
    ap.add_argument("--accuracy-steps", type=int, default=100,
                    help="steps from the initial field after which the forms' states are compared "
                         "(the timed steps count; the rest run after the timed region)")
    ap.add_argument("--shock-t", type=float, default=2.5,
                    help="TGV: time the learned form also from the shocklet phase, reached by "
                         "advancing the mixed form to at least this time (0: skip)")
    ap.add_argument("--shock-steps-max", type=int, default=1500)
    ap.add_argument("--slabs", type=int, default=0,
                    help="TGV: also time the grid split into this many z-slabs with halo exchanges "
                         "(osbli_domain_*, one device), mixed and FP64 forms, against the whole grid")
    return ap.parse_args()


SBLI_N = (512, 256, 64)


def workload(n, scheme, kind="tgv"):
    if kind == "sbli":
        cfg, U = I.sbli(n=SBLI_N, scheme=scheme)
        name = "sbli%dx%dx%d_%s_viscous" % (SBLI_N + (SCHEME_NAME[scheme].lower().replace("-", ""),))
        conf = {"workload": name, "grid": list(SBLI_N), "points": int(np.prod(SBLI_N)),
                "scheme": "%s characteristic (Roe average, LLF) in x, y, z" % SCHEME_NAME[scheme],
                "viscous": "4th-order central, Re=1e4 (displacement thickness), Pr=0.72, Sutherland "
                           "110.4 K / 288 K",
                "Ma": 2.0, "gamma": 1.4, "dt": cfg["dt"],
                "domain": "300 x 60 x 20, tanh wall-normal stretching 3.0 (rectilinear)",
                "boundaries": "similarity inflow / zero-gradient outlet, isothermal wall at the "
                              "adiabatic-wall temperature / Dirichlet top with a 10 deg oblique "
                              "shock from x=20, periodic span",
                "initial": "similarity profile everywhere (analytic)",
                "time_integration": "low-storage RK3, 3 stages per step",
                "l2": "inputs larger than L2: state %.0f MB" % (5 * np.prod(SBLI_N) * 8 / 1e6),
                "parallelism": "one replica per GPU"}
        return cfg, U, conf
    Ma = 1.25 if scheme != I.CENTRAL4 else 0.1
    cfg, U = I.tgv(n, Ma=Ma, Re=1600.0, scheme=scheme)
    name = "tgv%d_%s_viscous" % (n, SCHEME_NAME[scheme].lower().replace("-", ""))
    conf = {"workload": name, "grid": [n, n, n], "points": n ** 3,
            "scheme": "%s characteristic (Roe average, LLF) in x, y, z" % SCHEME_NAME[scheme]
            if scheme != I.CENTRAL4 else "central 4th order",
            "viscous": "4th-order central, Re=1600, Pr=0.72, mu=1", "Ma": Ma, "gamma": 1.4,
            "dt": cfg["dt"], "time_integration": "low-storage RK3, 3 stages per step",
            "precision": "fp64 state and arithmetic",
            "l2": "inputs larger than L2: state %.0f MB, resident working set > 4 GB"
                  % (5 * n ** 3 * 8 / 1e6),
            "parallelism": "one replica per GPU"}
    return cfg, U, conf


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_sbli(scheme, target_s=12.0):
    """The oracle on every host core, one RK step of the shock / boundary-layer physics on a box
    with the same domain and set-up at reduced resolution (~10-30 s of CPU work)."""
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    f = 8
    while True:
        n = tuple(max(8, v // f) for v in SBLI_N)
        cfg, U = I.sbli(n=n, scheme=scheme)
        o = O.Oracle(cfg)
        o.set_state(U)
        t = time.perf_counter()
        o.step(1)
        el = time.perf_counter() - t
        if el > target_s / 8 or f <= 2:
            break
        f //= 2
    npts = int(np.prod(n))
    return {"value": npts * 3 / el / 1e6, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
            "sample": "one RK3 step (3 stages) of the same %s shock / boundary-layer set-up on a "
                      "%dx%dx%d grid (%.1f s)" % ((SCHEME_NAME[scheme],) + n + (el,))}


def cpu_baseline(scheme, target_s=12.0):
    """The oracle as it stands, on every host core, one RK step of the same TGV physics on a
    smaller grid sized for ~10-30 s of CPU work."""
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    n = 24
    Ma = 1.25 if scheme != I.CENTRAL4 else 0.1
    cfg, U = I.tgv(n, Ma=Ma, scheme=scheme)
    o = O.Oracle(cfg)
    o.set_state(U)
    t = time.perf_counter()
    o.step(1)
    per_pt = (time.perf_counter() - t) / n ** 3
    n = int(min(128, max(24, round((target_s / per_pt) ** (1.0 / 3.0)))))
    cfg, U = I.tgv(n, Ma=Ma, scheme=scheme)
    o = O.Oracle(cfg)
    o.set_state(U)
    t = time.perf_counter()
    o.step(1)
    el = time.perf_counter() - t
    return {"value": n ** 3 * 3 / el / 1e6, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
            "sample": "one RK3 step (3 stages) of the same TGV %s + viscous physics on a %d^3 grid "
                      "(%.1f s)" % (SCHEME_NAME[scheme], n, el)}


def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    if args.workload == "ensemble":
        mem = I.riemann_ensemble(args.seed, scheme=args.scheme)
        cfg, U = min(mem, key=lambda m: int(np.prod(m[0]["n"])))
        nn = tuple(int(x) for x in cfg["n"])
        sample = "each step: one RK3 step of the oracle on the smallest ensemble member (%dx%d)" % nn[:2]
    elif args.workload == "sbli":
        nn = tuple(v // 8 for v in SBLI_N)
        cfg, U = I.sbli(n=nn, scheme=args.scheme)
        sample = ("each step: one RK3 step of the oracle on the same shock / boundary-layer set-up "
                  "at %dx%dx%d" % nn)
    else:
        n = 32
        nn = (n, n, n)
        Ma = 1.25 if args.scheme != I.CENTRAL4 else 0.1
        cfg, U = I.tgv(n, Ma=Ma, scheme=args.scheme)
        sample = "each step: one RK3 step of the oracle on a %d^3 sample of the workload's physics" % n
    o = O.Oracle(cfg)
    o.set_state(U)
    o.step(max(args.warmup, 0))
    t = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t
    val = int(np.prod(nn)) * 3 * args.steps / el / 1e6
    if args.workload == "ensemble":
        conf = {"workload": "riemann2d_ensemble64_seed%d_%s" % (args.seed, SCHEME_NAME[args.scheme].lower().replace("-", "")),
                "members": len(mem), "points": int(sum(np.prod(c["n"]) for c, _ in mem))}
    else:
        _, _, conf = workload(args.n, args.scheme, args.workload)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic (analytic initial field)", "config": conf,
                      "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)
    return 0


def run_ensemble(args, world, rank, local):
    """64 seeded 2D Riemann problems: batched mixed (headline), separate handles, batched FP64."""
    import torch
    from paper_2007_14933_b300 import build, osbli
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    osbli.load()

    def barrier():
        if dist:
            dist.barrier()
    mem = I.riemann_ensemble(args.seed, scheme=args.scheme)
    cfgs = [c for c, _ in mem]
    npts = int(sum(np.prod(c["n"]) for c in cfgs))
    stream = torch.cuda.current_stream()
    sizes = [int(c["n"][0]) for c in cfgs]
    conf = {"workload": "riemann2d_ensemble64_seed%d_%s" % (args.seed, SCHEME_NAME[args.scheme].lower().replace("-", "")),
            "members": len(cfgs), "points": npts, "sizes": sizes,
            "scheme": "%s characteristic (Roe average, LLF) in x, y, inviscid" % SCHEME_NAME[args.scheme],
            "states": "four quadrants, rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1] (numpy PCG64, seed %d)" % args.seed,
            "dt": "per member, CFL 0.4 on the initial state", "boundaries": "zero-gradient",
            "time_integration": "low-storage RK3, 3 stages per step",
            "l2": "inputs larger than L2: states %.0f MB" % (5 * npts * 8 / 1e6),
            "parallelism": "one replica per GPU"}

    def make(prec):
        e = osbli.Ensemble(cfgs, precision=prec, cuda_stream=stream.cuda_stream)
        for p, (_, U) in enumerate(mem):
            e.set_state(p, U)
        return e

    def timed(fn):
        fn(args.warmup)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(args.steps)
        e1.record(stream)
        e1.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, "cuda")

    gpu_index = torch.cuda.current_device()
    res = {}
    with ClockSampler(gpu_index) as clk:
        ens = make(osbli.OSBLI_MIXED)
        chunk, _ = ens.autotune(reps=2)
        res["ensemble"] = timed(ens.step)
        launches = ens.launches_per_step() * args.steps
        # the persistent form: one cooperative launch for all the timed steps of every member
        pers = make(osbli.OSBLI_MIXED)
        pers.set_chunk(chunk)
        pers.set_persistent(True)
        res["persistent"] = timed(pers.step)
        pers_grid = pers.persistent_grid()
        pers_same = all(np.array_equal(pers.get_state(p), ens.get_state(p)) for p in range(len(cfgs)))
        pers.close()
        sep = [osbli.Solver(c, precision=osbli.OSBLI_MIXED, cuda_stream=stream.cuda_stream) for c in cfgs]
        for s_, (_, U) in zip(sep, mem):
            s_.set_state(U)

        def sep_step(k):
            for _ in range(k):
                for s_ in sep:
                    s_.step(1)
        res["separate"] = timed(sep_step)
        sep_launches = sum(s_.launches_per_step() for s_ in sep)
        for s_ in sep:
            s_.close()
        e64 = make(osbli.OSBLI_FP64)
        res["fp64"] = timed(e64.step)
    clocks = clk.summary()
    forms = {f: {"value": job_rate(npts, args.steps, world, ms / 1e3), "ms_per_step": ms / args.steps}
             for f, ms in res.items()}
    l2 = 0.0
    for p in range(len(cfgs)):
        a, b = ens.get_state(p), e64.get_state(p)
        nb = [float(np.linalg.norm(b[v])) for v in range(5)]
        nb[1] = nb[2] = nb[3] = max(nb[1:4])
        l2 = max(l2, max(float(np.linalg.norm(a[v] - b[v])) / nb[v] for v in range(5) if nb[v] > 0))
    e2e = None
    if not args.no_e2e:
        hosts = [torch.from_numpy(np.ascontiguousarray(U)).pin_memory() for _, U in mem]
        outs = [torch.empty_like(h) .pin_memory() for h in hosts]
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for p, h in enumerate(hosts):
                osbli.osbli_ensemble_set_state(ens.e, p, h)
            ens.step(1)
            for p, o in enumerate(outs):
                osbli.osbli_ensemble_get_state(ens.e, p, o)
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        byt = int(sum(h.numel() for h in hosts) * 8)
        e2e = {"value": job_rate(npts, args.steps, world, el), "unit": UNIT, "h2d_bytes_per_step": byt,
               "d2h_bytes_per_step": byt,
               "api": "osbli_ensemble_set_state(host) x64 + osbli_ensemble_step(1) + osbli_ensemble_get_state(host) x64"}
    ens.close()
    e64.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    out = {"metric": METRIC, "value": forms["ensemble"]["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms["ensemble"]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic (seeded four-quadrant Riemann states)", "config": conf,
           "roofline": None, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
           "forms": forms, "autotuned_chunk": chunk,
           "gpu_launches_separate_per_step": sep_launches,
           "speedup_ensemble_vs_separate": forms["ensemble"]["value"] / forms["separate"]["value"],
           "persistent": {"blocks": pers_grid, "launches_per_call": 1,
                          "bitwise_equal_to_graph_form": pers_same,
                          "speed_vs_graph_form": forms["persistent"]["value"] / forms["ensemble"]["value"]},
           "speedup_ensemble_vs_fp64": forms["ensemble"]["value"] / forms["fp64"]["value"],
           "l2_ensemble_vs_fp64": l2,
           "variant": "mixed precision, batched members (osbli_ensemble_step)"}
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        cores = len(os.sched_getaffinity(0))
        O.set_threads(cores)
        done, el, used = 0, 0.0, []
        for cfg, U in sorted(mem, key=lambda m: int(np.prod(m[0]["n"]))):
            o = O.Oracle(cfg)
            o.set_state(U)
            t = time.perf_counter()
            o.step(1)
            el += time.perf_counter() - t
            done += int(np.prod(cfg["n"]))
            used.append(int(cfg["n"][0]))
            if el > 10.0:
                break
        out["cpu_baseline"] = {"value": done * 3 / el / 1e6, "unit": UNIT, "cores": O.get_threads(),
                               "kind": "oracle", "sample": "one RK3 step of the %d smallest members (N = %s), %.1f s"
                               % (len(used), used, el)}
    print(json.dumps(out), flush=True)
    return 0


def time_form(osbli, torch, cfg, U, precision, args, stream, barrier, dist, sensor=None, tag=""):
    """Warm up, then time args.steps RK steps of one form with CUDA events on its stream."""
    s = osbli.Solver(dict(cfg, sensor=1 if sensor else 0), precision=precision,
                     cuda_stream=stream.cuda_stream)
    if sensor:
        s.set_sensor(sensor[0], sensor[1])
    s.set_state(U)
    s.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed%s_%s" % (tag, "learned" if sensor else ("mixed" if precision else "fp64")))
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    return s, max_over_ranks(e0.elapsed_time(e1), dist, "cuda")


def l2_vs(Uf, Up):
    """Relative L2 difference, max over the conserved variables (momentum components share one
    scale)."""
    nb = [float(np.linalg.norm(Up[v])) for v in range(5)]
    nb[1] = nb[2] = nb[3] = max(nb[1:4])
    return max(float(np.linalg.norm(Uf[v] - Up[v])) / nb[v] for v in range(5) if nb[v] > 0)


_CALIB = {}


def SN_threshold(sensor, recall):
    """Threshold of the trained sensor for another recall target on its training set (kept by
    main() while the training set is alive)."""
    f = _CALIB.get("fn")
    return f(recall) if f else None


def shocked_phase(osbli, torch, cfg, U, sensor, args, stream, barrier, dist, npts, world, prec):
    """The learned form where its gate acts: the TGV is advanced with the mixed form (outside any
    timed region) into its shocklet phase -- past args.shock_t and until TENO cut-off labels mark
    at least 1 % of the cells -- and the learned, mixed and FP64 forms are then timed from that
    state exactly as from the initial field, and compared after the same steps."""
    s = osbli.Solver(cfg, precision=osbli.OSBLI_MIXED, cuda_stream=stream.cuda_stream)
    s.set_state(U)
    done, lab_frac = 0, 0.0
    lab = torch.empty(npts, dtype=torch.uint8, device="cuda")
    while done < args.shock_steps_max:
        s.step(100)
        done += 100
        osbli.osbli_sensor_labels(s.h, lab)
        lab_frac = float(lab.float().mean().item())
        if done * cfg["dt"] >= args.shock_t and lab_frac >= 0.01:
            break
    Us = s.get_state()
    s.close()
    # the gate's recall of the labels at the start state
    g = osbli.Solver(dict(cfg, sensor=1), precision=osbli.OSBLI_MIXED, cuda_stream=stream.cuda_stream)
    g.set_sensor(sensor[0], sensor[1])
    g.set_state(Us)
    probs = torch.empty(npts, dtype=torch.float32, device="cuda")
    osbli.osbli_sensor_probs(g.h, probs)
    flagged = probs >= sensor[1]
    pos = lab.bool()
    recall = float((flagged & pos).sum().item()) / max(1, int(pos.sum().item()))
    g.close()
    del probs, flagged, pos
    res = {f: time_form(osbli, torch, cfg, Us, prec[f], args, stream, barrier, dist,
                        sensor if f == "learned" else None, tag="_shocklet") for f in ("learned", "mixed", "fp64")}
    dg = res["learned"][0].diagnostics()
    prof = res["learned"][0].profile_residual(reps=2)
    out = {"t_start": done * cfg["dt"], "steps_advanced": done, "label_fraction": lab_frac,
           "gate_recall_of_labels": recall,
           "gated": {"cells": float(dg[9]), "interfaces_x": float(dg[10]), "interfaces_y": float(dg[11]),
                     "interfaces_z": float(dg[12])},
           "forms": {f: {"value": job_rate(npts, args.steps, world, ms / 1e3), "ms_per_step": ms / args.steps}
                     for f, (_, ms) in res.items()},
           "kernels_ms": {nm: t_ for nm, t_ in prof}}
    Up = res["fp64"][0].get_state()
    for f in ("learned", "mixed"):
        out["l2_%s_vs_fp64" % f] = l2_vs(res[f][0].get_state(), Up)
        out["speedup_%s_vs_fp64" % f] = out["forms"][f]["value"] / out["forms"]["fp64"]["value"]
    # a stricter threshold (the calibration's recall target 0.99): more cells on the characteristic
    # flux, closer to the FP64 result, at its cost
    thr2 = SN_threshold(sensor, 0.99)
    if thr2 is not None:
        s2, ms2 = time_form(osbli, torch, cfg, Us, prec["learned"], args, stream, barrier, dist, (sensor[0], thr2),
                            tag="_shocklet_strict")
        dg2 = s2.diagnostics()
        out["stricter_gate"] = {"threshold": thr2, "recall_target": 0.99, "gated_cells": float(dg2[9]),
                                "value": job_rate(npts, args.steps, world, ms2 / 1e3),
                                "ms_per_step": ms2 / args.steps, "l2_vs_fp64": l2_vs(s2.get_state(), Up)}
        s2.close()
    out["note"] = ("state advanced %d steps (t = %.2f) with the mixed form, then each form timed over "
                   "%d steps after %d warm-up steps from it; L2 against the FP64 form after those %d steps"
                   % (done, done * cfg["dt"], args.steps, args.warmup, args.warmup + args.steps))
    for f in res:
        res[f][0].close()
    return out


def split_grid(osbli, torch, cfg, U, args, stream, barrier, dist, npts, world, prec, res, done):
    """The same workload as args.slabs z-slabs with halo exchanges on this device (the layout a
    decomposed run uses), mixed and FP64 forms, timed like the whole grid; states compared
    bitwise with the whole grid's after the same steps."""
    out = {"slabs": args.slabs}
    for f in ("mixed", "fp64"):
        if f not in res:
            continue
        d = osbli.Domain(cfg, args.slabs, precision=prec[f], cuda_stream=stream.cuda_stream)
        d.set_state(U)
        d.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        launches, copies = d.launches_per_step()
        d.step(done - args.warmup - args.steps)      # as many steps as the whole grid's solver took
        Ud, Uw = d.get_state(), res[f][0].get_state()
        same = bool(np.array_equal(Ud, Uw))
        l2d = l2_vs(Ud, Uw)
        del Ud, Uw
        d.close()
        out[f] = {"value": job_rate(npts, args.steps, world, ms / 1e3), "ms_per_step": ms / args.steps,
                  "launches_per_step": launches, "halo_copies_per_step": copies,
                  "bitwise_equal_to_whole_grid": same, "l2_vs_whole_grid": l2d}
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "ensemble":
        return run_ensemble(args, world, rank, local)

    import torch
    from paper_2007_14933_b300 import build, osbli
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    osbli.load()

    def barrier():
        if dist:
            dist.barrier()

    cfg, U, conf = workload(args.n, args.scheme, args.workload)
    npts = int(conf["points"])
    stream = torch.cuda.current_stream()
    forms = ["learned", "mixed", "fp64"]
    if args.plain or args.scheme == I.CENTRAL4:
        forms = ["fp64"]
    elif args.mixed:
        forms = ["mixed"]
    elif args.no_sensor:
        forms = ["mixed", "fp64"]
    if args.forms:
        forms = [f for f in args.forms.split(",") if f in ("learned", "mixed", "fp64")]
    head = forms[0]
    prec = {"learned": osbli.OSBLI_MIXED, "mixed": osbli.OSBLI_MIXED, "fp64": osbli.OSBLI_FP64}
    sensor = None
    sensor_info = None
    if "learned" in forms:
        # train the sensor on the GPU from TENO labels of coarse TGV snapshots (same physics)
        from paper_2007_14933_b300 import sensor as SN
        t0 = time.perf_counter()
        feats, labels, _ = SN.tgv_training_set(N=64, Ma=1.25, nsnap=6, steps_between=12)
        train_set = "TGV 64^3 Ma 1.25, 6 snapshots every 12 steps"
        if args.workload == "tgv":
            f2, l2_, desc = SN.tgv_shocklet_training_set(N=128, Ma=1.25, times=(1.0, 1.5, 2.0, 2.5, 3.0, 3.5))
            feats, labels = torch.cat([feats, f2]), torch.cat([labels, l2_])
            train_set += " + " + desc
            del f2, l2_
            if args.n >= 256 and args.train_fine:
                # the run's own resolution, before the timed windows (t <= 2): the sensor learns from
                # the TENO labels of the run it gates (a snapshot at t = 2.25 as well raised the gated
                # fraction of the smooth phase to 2.4 % for 3 points of recall at t = 2.5)
                f2, l2_, desc = SN.tgv_shocklet_training_set(N=args.n, Ma=1.25, times=(1.5, 2.0))
                feats, labels = torch.cat([feats, f2]), torch.cat([labels, l2_])
                train_set += " + " + desc
                del f2, l2_
        if args.workload == "sbli":
            f2, l2_, _ = SN.sbli_training_set()
            feats, labels = torch.cat([feats, f2]), torch.cat([labels, l2_])
            train_set += " + " + SN.SBLI_TRAIN_DESC
            del f2, l2_
        w, hist = SN.train(feats, labels, steps=args.sensor_steps, batch=4096)
        thr = SN.calibrate_threshold(w, feats, labels, recall=0.9)
        sensor = (w, thr)
        _CALIB["thr"] = {r: SN.calibrate_threshold(w, feats, labels, recall=r) for r in (0.99,)}
        _CALIB["fn"] = lambda r: _CALIB["thr"].get(r)
        sensor_info = {"train_set": "%s, %d cells, label fraction %.3f"
                                    % (train_set, int(labels.numel()), float(labels.float().mean().item())),
                       "train_steps": args.sensor_steps, "batch": 4096, "loss_first": float(hist[:20].mean()),
                       "loss_last": float(hist[-20:].mean()), "threshold": thr,
                       "recall_target": 0.9, "train_s": time.perf_counter() - t0}
        del feats, labels

    gpu_index = torch.cuda.current_device()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except (ValueError, IndexError):
            pass
    res = {}
    with ClockSampler(gpu_index) as clk:
        for f in forms:
            res[f] = time_form(osbli, torch, cfg, U, prec[f], args, stream, barrier, dist,
                               sensor if f == "learned" else None)
    clocks = clk.summary()
    sh, ms_max = res[head]
    value = job_rate(npts, args.steps, world, ms_max / 1e3)
    launches = sh.launches_per_step() * args.steps

    # per-kernel durations of one residual evaluation of the headline form (CUDA events)
    prof = sh.profile_residual(reps=2)
    conv = [(nm, t_) for nm, t_ in prof if nm.startswith("conv_")]
    dom_name, dom_ms = max(conv, key=lambda x: x[1])
    # directions the dominant launch forms (the learned form's fused x + y pass: two)
    ndir = len(dom_name) - len("conv_")
    flops = FLOPS_CONV_POINT_DIR[args.scheme] * npts * ndir
    gated = None
    if head == "learned":
        dg = sh.diagnostics()
        gated = {"cells": float(dg[9]), "interfaces_x": float(dg[10]),
                 "interfaces_y": float(dg[11]), "interfaces_z": float(dg[12])}
        f_int = sum(float(dg[10 + "xyz".index(c)]) for c in dom_name[5:]) / ndir
        flops = (f_int * FLOPS_CONV_POINT_DIR[args.scheme] + (1.0 - f_int) * FLOPS_CENTRAL_DELTA) * npts * ndir
    if head in ("mixed", "learned"):
        peak, pdt = osbli.osbli_fp32_peak(), "fp32"
        if head == "learned":
            kern = {"conv_x": "k_conv_delta_x_win", "conv_xy": "k_conv_delta_xy"}.get(dom_name, "k_conv_delta_tile")
        else:
            kern = "k_conv_char_delta" if dom_name != "conv_x" else "k_conv_char_delta_x"
        src = "FP32 FMA throughput measured in this run (osbli_fp32_peak)"
    else:
        peak, pdt, kern = osbli.osbli_fp64_peak(), "fp64", "k_conv_char"
        src = "FP64 FMA throughput measured in this run (osbli_fp64_peak)"
    achieved = flops / (dom_ms * 1e-3) / 1e12
    alu = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": None, "kernel": "%s (%s)" % (kern, dom_name),
           "dtype": pdt, "peak_source": src, "flops_per_launch": flops}
    roofline = alu
    if head in ("mixed", "learned"):
        # the same launch against HBM: algorithmic bytes per point of one delta-form pass (one
        # direction, or x and y fused) = FP32 hi/lo state (40 B) + u, v, w, p (16 B) + residual
        # write (20 B) and read when it accumulates (20 B, not the first pass) + gate byte;
        # a, sqrt(rho), H (12 B) only for characteristic interfaces (fraction f_int)
        f_c = f_int if head == "learned" else 1.0
        acc = 0 if dom_name in ("conv_x", "conv_xy") else 1
        bpp = 40.0 + 16.0 + 20.0 + 20.0 * acc + (1.0 if head == "learned" else 0.0) + 12.0 * f_c
        hbm_bytes = bpp * npts
        gbs = hbm_bytes / (dom_ms * 1e-3) / 1e9
        hbm = {"bound": "hbm", "achieved": gbs, "peak": HBM_GBS, "unit": "GB/s", "frac": gbs / HBM_GBS,
               "traffic": None, "kernel": "%s (%s)" % (kern, dom_name),
               "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "bytes_per_launch": hbm_bytes}
        if kern in DRAM_BYTES_PER_POINT:
            # DRAM traffic of the kernel per point from its ncu capture, scaled to this launch
            hbm["traffic"] = DRAM_BYTES_PER_POINT[kern][0] * npts
            hbm["traffic_source"] = DRAM_BYTES_PER_POINT[kern][1]
        # the binding roofline is the one the launch comes closest to
        roofline = dict(hbm if hbm["frac"] > alu["frac"] else alu)
        roofline["other"] = alu if roofline["bound"] == "hbm" else hbm

    out_forms = {}
    for f in forms:
        s_, ms_ = res[f]
        out_forms[f] = {"value": job_rate(npts, args.steps, world, ms_ / 1e3),
                        "ms_per_step": ms_ / args.steps}
    extra = {"forms": out_forms}
    if "fp64" in forms and len(forms) > 1:
        # accuracy at matched work: every form advanced to the same step count from the same
        # state (the steps beyond warmup + steps run after the timed region)
        acc_steps = max(args.accuracy_steps, args.warmup + args.steps)
        for f in forms:
            res[f][0].step(acc_steps - args.warmup - args.steps)
        Up = res["fp64"][0].get_state()
        for f in forms:
            if f == "fp64":
                continue
            extra["l2_%s_vs_fp64" % f] = l2_vs(res[f][0].get_state(), Up)
            extra["speedup_%s_vs_fp64" % f] = out_forms[f]["value"] / out_forms["fp64"]["value"]
        extra["accuracy_note"] = ("relative L2 (max over conserved variables) of each form's state "
                                  "against the FP64 form after %d steps from the same initial "
                                  "field; the FP64 form is parity-checked against the CPU oracle"
                                  % acc_steps)
        del Up
        if head == "learned":
            dg = res["learned"][0].diagnostics()
            extra["gated_after_accuracy_steps"] = {"cells": float(dg[9]), "interfaces_x": float(dg[10]),
                                                   "interfaces_y": float(dg[11]),
                                                   "interfaces_z": float(dg[12])}
    if args.slabs > 1 and args.workload == "tgv":
        done = (max(args.accuracy_steps, args.warmup + args.steps) if ("fp64" in forms and len(forms) > 1)
                else args.warmup + args.steps)
        extra["split_grid"] = split_grid(osbli, torch, cfg, U, args, stream, barrier, dist, npts, world, prec, res,
                                         done)
    if "learned" in forms and args.workload == "tgv" and args.shock_t > 0:
        extra["shocklet_phase"] = shocked_phase(osbli, torch, cfg, U, sensor, args, stream, barrier, dist,
                                                npts, world, prec)
    if sensor_info:
        sensor_info["gated"] = gated
        extra["sensor"] = sensor_info

    e2e = None
    launches_e2e = None
    if not args.no_e2e:
        Uh = torch.from_numpy(np.ascontiguousarray(U)).pin_memory()
        Uo = torch.empty_like(Uh).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            osbli.osbli_set_state(sh.h, Uh)
            osbli.osbli_rk_step(sh.h, 1)
            osbli.osbli_get_state(sh.h, Uo)
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": job_rate(npts, args.steps, world, el), "unit": UNIT,
               "h2d_bytes_per_step": int(Uh.numel() * 8), "d2h_bytes_per_step": int(Uo.numel() * 8),
               "api": "osbli_set_state(host) + osbli_rk_step(1) + osbli_get_state(host)"}
        launches_e2e = (sh.launches_per_step() + 2) * args.steps
    for f in forms:
        res[f][0].close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    mixed_desc = ("mixed: FP32 reconstruction / weights / projections / viscous terms, FP64 state, "
                  "RK registers, metrics and strong-jump interfaces")
    conf = dict(conf, precision=mixed_desc if head in ("mixed", "learned") else "fp64 state and arithmetic",
                form={"learned": "mixed precision + learned TENO/central gate", "mixed": "mixed precision",
                      "fp64": "plain FP64"}[head])
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if head in ("mixed", "learned") else "f64",
           "data": "synthetic (analytic %s initial field)" % ("similarity-profile" if args.workload == "sbli"
                                                               else "TGV"), "config": conf,
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
           "kernels_ms": {nm: t_ for nm, t_ in prof},
           "variant": {"learned": "mixed precision + learned sensor (headline form)",
                       "mixed": "mixed precision", "fp64": "plain FP64"}[head]}
    out.update(extra)
    if launches_e2e is not None:
        out["gpu_launches_e2e"] = launches_e2e
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = (cpu_baseline_sbli(args.scheme) if args.workload == "sbli"
                               else cpu_baseline(args.scheme))
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
