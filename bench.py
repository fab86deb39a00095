"""Benchmark of the split-operator propagation (arXiv:1306.3247) on GB300.

Headline (`value`): the plain FP64 form on the 3-D workload. One bench step = one
complete propagation job: a Gaussian packet (sigma 1.5, p0 = (2,0,0), centred at
(-3,0,0)) on a 256^3 grid over [-30,30)^3 scattering off the time-dependent spherical
barrier 1.5 (1 + 0.3 sin 2t) exp(-|r|^2), dt = 0.002, 200 Strang steps, observables
(norm, <x>, <p>, <x^2>, energies) every 20 steps. Metric: grid-point steps per second
over all ranks.

  value   -- device-resident input: the initial state already in HBM, each timed job
             starts from a device-to-device copy of it.
  e2e     -- the same job through the C ABI with host buffers: host-to-device copy of
             psi(0) from pinned memory, the run, device-to-host copy of psi(T) and of the
             observables, all inside the timed region.
  forms   -- the same job in the float-float complex128-accuracy form and in complex64.
  batched -- 4096 uneven 1-D/2-D driven-trap instances advanced together (complex64,
             chunks of 20 steps replayed as CUDA graphs), next to the plain per-instance
             FP64 form on a seeded sample of 256 of the same instances.
  served  -- the seeded Poisson request stream (2000 requests of 1-D/2-D/3-D jobs,
             complex64) through the continuous-batching server under an 80 GB budget:
             p50/p99 latency, offered and achieved rates; then its first 500 and its
             first 120 requests offered below the achieved rate.

--impl reference times the FP64 CPU oracle on a bounded sample of the
3-D workload on the host cores. With --gpus N > 1 (torchrun) every rank runs an
independent replica ("replicas only": the method has no exchange step).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1306_3247_gb300 import workloads as W  # noqa: E402

METRIC = "grid-point·steps/s (256³ c128 plain vs batched c64) + served p50/p99 ms"
UNIT = "grid-point·steps/s"
# FP64 operations per clock per SM on GB300: 2 FP64 fused multiply-adds (the nominal
# 1.25 TFLOP/s over 152 SMs at 2070 MHz).
FP64_FLOP_PER_CLOCK_PER_SM = 4

# DRAM bytes (read + write) per launch of each pass class on the 256^3 workload, from one
# ncu capture of the current kernels (dram__bytes_read.sum + dram__bytes_write.sum). Valid
# for grid 256 only; any other grid reports null.
TRAFFIC_256 = {
    "c128": {"pass_contig": 480336128, "pass_strided": 472172288, "pass_kinetic": 477476096},
    "c64": {"pass_contig": 206836992, "pass_strided": 205500416, "pass_kinetic": 209300736},
    "c128f": {"pass_contig": 474867456, "pass_strided": 471806464, "pass_kinetic": 477838592},
}


def traffic_of(grid, precision, kernel_class):
    return TRAFFIC_256.get(precision, {}).get(kernel_class) if grid == 256 else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, ("fallback: 6.8 TB/s HBM, 1.9 PFLOP/s bf16 from one "
                                                            "earlier GB300 measurement (no MEASURED_PEAKS.json)")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if s[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl != "reference":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline_run(cfg, nsteps):
    """Time the oracle as it stands on nsteps Strang steps of the workload."""
    from oracle import oracle as O
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    t0 = time.perf_counter()
    O.propagate(pb, terms, psi0, nsteps)
    dt = time.perf_counter() - t0
    npts = math.prod(pb["n"][: pb["ndim"]])
    return npts * nsteps / dt, dt, O.num_threads()


def reference_arm(args, world, rank):
    """The oracle, on the host cores, as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle as O
    cfg = W.config_3d_barrier(n=args.grid)
    pb, terms = cfg["problem"], cfg["terms"]
    psi = O.gaussian(pb, **cfg["init"])
    npts = args.grid ** 3
    for k in range(args.warmup):
        psi = O.step(pb, terms, psi, k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        psi = O.step(pb, terms, psi, args.warmup + k)
    el = time.perf_counter() - t0
    v = npts * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"] + " VKV (FP64 CPU oracle: one Strang step per bench step)",
                       "grid": [args.grid] * 3, "dt": 0.002},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"one Strang step of the {args.grid}^3 barrier workload per bench step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def probe_rate(WPK, fp64):
    """FMA throughput of the device in TFLOP/s, measured by the library's probe."""
    import ctypes
    lib = WPK.load_library()
    lib.wp_probe_fma_rate.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    lib.wp_probe_fma_rate.restype = ctypes.c_int
    out = ctypes.c_double(0.0)
    st = lib.wp_probe_fma_rate(1 if fp64 else 0, None, ctypes.byref(out))
    if st != WPK.WP_OK:
        raise RuntimeError("wp_probe_fma_rate failed with status %d" % st)
    return out.value


def pass_flops_per_point(logn, kind):
    """Algorithmic FLOPs per grid point of one pass: 5 log2 n per axis transform (the
    standard radix-2 count) and 6 per complex multiply by a phase factor."""
    fft = 5 * logn
    return {"pass_contig": 2 * fft + 6, "pass_kinetic": 2 * fft + 6, "pass_strided": fft}.get(kind, fft)


def bench_3d(args, WPK, precision, world, local, steps, warmup, nt, with_e2e=True, with_clocks=False, order="vkv",
             keep_state=False):
    import torch
    cfg = W.config_3d_barrier(n=args.grid, order=order)
    pb, terms = cfg["problem"], cfg["terms"]
    nprint = cfg["nprint"]
    npts = math.prod(pb["n"][: pb["ndim"]])
    stream = torch.cuda.Stream()
    P = WPK.Propagator(pb, terms, precision, stream=stream.cuda_stream)
    P.init_gaussian(**cfg["init"])
    tuned = None
    if args.autotune:
        sched, ms, ncand = P.autotune(steps=2)
        tuned = {"schedule": sched, "ms_per_step": ms, "schedules_timed": ncand}
    psi0_dev = torch.empty(P.shape, dtype=torch.complex128, device="cuda")
    P.get_state_device(psi0_dev)
    torch.cuda.synchronize()
    host_in = torch.empty(P.shape, dtype=torch.complex128, pin_memory=True)
    host_in.copy_(psi0_dev.cpu())
    host_out = torch.empty(P.shape, dtype=torch.complex128, pin_memory=True)

    def job_device():
        P.set_state(psi0_dev)
        P.step_index = 0
        return P.run(nt, nprint)

    def job_e2e():
        WPK.wp_set_state(P.h, host_in.data_ptr(), False)
        P.step_index = 0
        obs = P.run(nt, nprint)
        WPK.wp_get_state(P.h, host_out.data_ptr(), False)
        return obs

    for _ in range(warmup):
        job_device()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if with_clocks else None
    if clocks:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = P.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        obs = job_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    dev_ms = ev0.elapsed_time(ev1)
    launches = P.launches - launches0
    barrier(world)
    clk = clocks.stop() if clocks else None
    dev_ms = max_over_ranks(world, dev_ms)
    out = {"value": world * npts * nt * steps / (dev_ms / 1e3), "ms_per_job": dev_ms / steps, "launches": launches,
           "clocks": clk, "final_norm": float(obs["norm"][-1]),
           "norm_drift": float(abs(obs["norm"][-1] - obs["norm"][0])), "autotune": tuned}
    if with_e2e:
        job_e2e()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            job_e2e()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        out["e2e"] = {"value": world * npts * nt * steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": npts * 16,
                      "d2h_bytes_per_step": npts * 16 + 128 * (1 + nt // nprint)}
    # per-kernel durations with CUDA events on the launching stream (one more job)
    P.profile(True)
    job_device()
    prof = P.profile_read()
    P.profile(False)
    out["kernels"] = {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in prof.items() if v[0]}
    if keep_state:  # the final state of the job just run, for the error of the other forms
        out["state"] = P.get_state_device(torch.empty(P.shape, dtype=torch.complex128, device="cuda"))
    P.close()
    return out


def bench_batched(WPK, precision, count, chunk, steps, warmup, plain_subset, autotune=True, job_steps=None):
    """The uneven-instance batch: all instances advance `chunk` steps per graph replay; a
    bench step is `job_steps` steps (a whole job of job_steps / chunk replays) or one chunk.
    With autotune, one instance of every distinct 1-D shape is tuned first; the cached
    schedules then apply to all instances of that shape. 2-D instances keep the default
    schedule: the batched 2-D passes run the 2048-element-tile kernels, and an instance
    tuned to another tiling would leave the batched launch for its own sequence."""
    import torch
    inst = W.batched_instances(count=count)
    pts = [math.prod(c["problem"]["n"][: c["problem"]["ndim"]]) for c in inst]
    tuned = {}
    if autotune:
        for c in inst:
            key = tuple(c["problem"]["n"][: c["problem"]["ndim"]])
            if key in tuned or c["problem"]["ndim"] != 1:
                continue
            with WPK.Propagator(c["problem"], c["terms"], precision) as T:
                T.init_gaussian(**c["init"])
                sched, ms, ncand = T.autotune(steps=3)
            tuned[key] = sched
    B = WPK.Batch(precision)
    for c in inst:
        k = B.add(c["problem"], c["terms"])
        B.init_gaussian(k, **c["init"])
    per = (job_steps // chunk) if job_steps else 1
    for _ in range(warmup):
        B.step(chunk, use_graph=True)
    torch.cuda.synchronize()
    l0 = B.launches
    t0 = time.perf_counter()
    for _ in range(steps * per):
        B.step(chunk, use_graph=True)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    launches = B.launches - l0
    finite = bool(np.isfinite(B.get_state(0)).all())
    B.close()
    out = {"value": sum(pts) * chunk * per * steps / el, "instances": count, "points": int(sum(pts)),
           "steps_per_bench_step": chunk * per, "graph_chunk_steps": chunk, "ms_per_bench_step": el / steps * 1e3,
           "graph_launches_issued": launches,
           "n1d": sum(1 for c in inst if c["problem"]["ndim"] == 1), "finite": finite, "precision": precision,
           "autotuned_shapes": {"x".join(map(str, k)): v for k, v in tuned.items()}}
    if plain_subset <= 0:
        return out
    # The plain per-instance FP64 form on a seeded sample of the same instances: every
    # instance its own handle, spread over 16 streams so that instances overlap on the
    # device, chunks replayed as CUDA graphs (two warm-up chunks: direct, then capture).
    rng = np.random.default_rng(7)
    pick = sorted(rng.choice(len(inst), size=min(plain_subset, len(inst)), replace=False).tolist())
    streams = [torch.cuda.Stream() for _ in range(16)]
    handles = []
    for k, i in enumerate(pick):
        c = inst[i]
        P = WPK.Propagator(c["problem"], c["terms"], "c128", stream=streams[k % 16].cuda_stream)
        P.init_gaussian(**c["init"])
        handles.append(P)
    for _ in range(2):
        for P in handles:
            P.step(chunk)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for P in handles:
        P.step(chunk)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    for P in handles:
        P.close()
    out["plain_fp64_per_instance"] = {"value": sum(pts[i] for i in pick) * chunk / el, "instances": len(pick),
                                      "sample": "seeded random sample of the batch's instances, 16 streams, "
                                                "CUDA-graph replay"}
    return out


def bench_served(WPK, nreq, precision, nreq_below=(500, 120)):
    """The seeded Poisson stream at its own rate (200 req/s offered: far above capacity, so
    latency is mostly queueing), then its first 500 and its first 120 requests with arrivals
    stretched so that the offered rate is 0.7 of the rate achieved at saturation. The large
    3-D jobs (256^3, up to 2000 steps, about 0.5 s alone) share the GPU with the others
    while they run, so the tail latency below capacity is mostly their shared service
    time."""
    from paper_1306_3247_gb300 import serving as S
    reqs = W.request_stream()[:nreq]
    summary, _ = S.serve(reqs, budget_bytes=80e9, nslots=32, chunk_steps=50, precision=precision)
    summary["precision"] = precision
    if summary.get("achieved_rate"):
        for k, nb in enumerate(nreq_below):
            sub = reqs[:min(nb, len(reqs))]
            target = 0.7 * summary["achieved_rate"]
            offered = len(sub) / sub[-1][0] if sub and sub[-1][0] > 0 else None
            scale = offered / target if offered else 1.0
            under, _ = S.serve(sub, budget_bytes=80e9, nslots=32, chunk_steps=50, precision=precision,
                               time_scale=max(1.0, scale))
            under["time_scale"] = max(1.0, scale)
            summary["below_capacity" if k == 0 else "below_capacity_first%d" % nb] = under
    return summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="c128", choices=["c128", "c64", "c128f"])
    ap.add_argument("--grid", type=int, default=256, help="points per axis of the 3-D workload")
    ap.add_argument("--nt", type=int, default=200)
    ap.add_argument("--cpu-steps", type=int, default=25, help="oracle steps of the CPU baseline sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="headline only (no forms, batch, serving)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the seeded stream served at its own rate (the first 500 and the first "
                         "120 of them also below capacity)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="run the default schedule instead of the autotuned one")
    ap.add_argument("--only", choices=["batch", "serve"], default=None,
                    help="time only the uneven-instance batch (complex64) or only the served stream, and print "
                         "its record")
    args = ap.parse_args()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    import torch
    from paper_1306_3247_gb300 import wavepacket as WPK

    torch.cuda.set_device(local)
    if args.only == "batch":
        r = bench_batched(WPK, "c64", args.batch_count, chunk=20, steps=args.steps, warmup=args.warmup,
                          plain_subset=0, autotune=args.autotune)
        if rank == 0:
            print(json.dumps({"batched": r}))
        return
    if args.only == "serve":
        t0 = time.perf_counter()
        r = bench_served(WPK, args.serve_requests, "c64")
        r["bench_wall_s"] = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"served": r}))
        return
    head = bench_3d(args, WPK, args.precision, world, local, args.steps, args.warmup, args.nt, with_e2e=True,
                    with_clocks=True, keep_state=(args.precision == "c128" and not args.no_extra and rank == 0))
    ref_state = head.pop("state", None)
    pk, src = peaks()
    npts = args.grid ** 3
    logn = int(math.log2(args.grid))
    dom = max(head["kernels"].items(), key=lambda kv: kv[1]["launches"] * kv[1]["avg_ms"])
    dom_name, dom_v = dom
    avg_s = dom_v["avg_ms"] / 1e3
    elem = 8 if args.precision == "c64" else 16
    if args.precision == "c128":
        # the FP64 pipe bounds this form: peak derived from the unit counts and the clock
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = pk.get("sm_max_mhz") or 2070.0  # else GB300's maximum SM clock
        fp64_peak = nsm * FP64_FLOP_PER_CLOCK_PER_SM * mhz * 1e6 / 1e12
        flops = pass_flops_per_point(logn, dom_name) * npts
        roof = {"bound": "alu", "kernel": dom_name, "achieved": flops / avg_s / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": flops / avg_s / 1e12 / fp64_peak,
                "traffic": traffic_of(args.grid, args.precision, dom_name),
                "peak_source": f"derived: {nsm} SMs x 2 FP64 FMA per clock x 2 FLOP x {mhz:.0f} MHz "
                               f"(GB300 nominal FP64 1.25 TFLOP/s); clock and HBM peak: {src}",
                "probe_fp64_fma_tflops": probe_rate(WPK, True),
                "probe_fp32_fma_tflops": probe_rate(WPK, False),
                "avg_launch_ms": dom_v["avg_ms"], "launches": dom_v["launches"],
                "hbm_frac": 2 * npts * elem / avg_s / 1e9 / pk["hbm_gbs"]}
    else:
        achieved = 2 * npts * elem / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": traffic_of(args.grid, args.precision, dom_name),
                "peak_source": src,
                "avg_launch_ms": dom_v["avg_ms"], "launches": dom_v["launches"]}
    extra = {}
    if not args.no_extra and rank == 0:
        for form in ("c128f", "c64"):
            if form == args.precision:
                continue
            r = bench_3d(args, WPK, form, 1, local, args.steps, args.warmup, args.nt, with_e2e=False,
                         keep_state=ref_state is not None)
            kd = max(r["kernels"].items(), key=lambda kv: kv[1]["launches"] * kv[1]["avg_ms"])
            el = 8 if form == "c64" else 16
            r["roofline"] = {"bound": "hbm", "kernel": kd[0],
                             "achieved": 2 * npts * el / (kd[1]["avg_ms"] / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                             "unit": "GB/s", "traffic": traffic_of(args.grid, form, kd[0]), "peak_source": src}
            r["roofline"]["frac"] = r["roofline"]["achieved"] / pk["hbm_gbs"]
            r["dtype"] = {"c128f": "f32x2", "c64": "f32"}[form]
            st = r.pop("state", None)
            if st is not None and ref_state is not None:
                # error of the form against the native FP64 GPU result of the same job; the
                # parity tests compare every form with the FP64 CPU oracle on this job
                r["rel_l2_vs_native_fp64_gpu"] = float(torch.linalg.vector_norm(st - ref_state) /
                                                       torch.linalg.vector_norm(ref_state))
            extra.setdefault("forms", {})[form] = r
        # the paper's K-V-K order (eq. splitop, Algorithm 1) on the same job, native FP64
        r = bench_3d(args, WPK, "c128", 1, local, args.steps, min(args.warmup, 3), args.nt, with_e2e=False,
                     order="kvk")
        extra["orders"] = {"kvk": {"value": r["value"], "ms_per_job": r["ms_per_job"], "precision": "c128",
                                   "kernels": r["kernels"]}}
        extra["batched"] = bench_batched(WPK, "c64", args.batch_count, chunk=20, steps=1, warmup=3,
                                         plain_subset=256, autotune=args.autotune, job_steps=2000)
        # the same batch in the complex128-accuracy forms (native FP64 and float-float)
        extra["batched_forms"] = {}
        for form in ("c128", "c128f"):
            r = bench_batched(WPK, form, args.batch_count, chunk=20, steps=3, warmup=1, plain_subset=0,
                              autotune=args.autotune)
            extra["batched_forms"][form] = {k: r[k] for k in ("value", "ms_per_bench_step", "precision")}
        extra["served"] = bench_served(WPK, args.serve_requests, "c64")
    cpu = None
    if rank == 0 and not args.no_cpu:
        v, dt, cores = cpu_baseline_run(W.config_3d_barrier(n=args.grid), args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} Strang step(s) of the {args.grid}^3 workload ({dt:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_job"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"c128": "f64", "c64": "f32", "c128f": "f32x2"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"3d_barrier_{args.grid}^3 {args.precision} VKV, {args.nt} steps per job, "
                                   f"observables every 20",
                       "grid": [args.grid] * 3, "dt": 0.002, "steps_per_job": args.nt, "parallelism": "replicas",
                       "l2": "state larger than the 129 MB L2 (268 MB complex128), no flush needed",
                       "schedule": head["autotune"]},
            "e2e": head["e2e"], "gpu_launches": int(head["launches"]), "roofline": roof,
            "kernels": head["kernels"], "clocks": head["clocks"], "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
