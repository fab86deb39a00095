"""Benchmark of the split-operator propagation (arXiv:1306.3247) on GB300.

One bench step = one complete propagation job of the 3-D workload: a Gaussian packet
(sigma 1.5, p0 = (2,0,0), centred at (-3,0,0)) on a 256^3 grid over [-30,30)^3
scattering off the time-dependent spherical barrier 1.5 (1 + 0.3 sin 2t) exp(-|r|^2),
dt = 0.002, 200 Strang steps, observables (norm, <x>, <p>, <x^2>, energies) every 20
steps. Metric: grid-point steps per second over all ranks.

  value  -- device-resident input: the initial state already in HBM, the timed job
            starts from a device-to-device copy of it.
  e2e    -- the same job through the C ABI with host buffers: host-to-device copy of
            psi(0) from pinned memory, the run, device-to-host copy of psi(T) and of
            the observables, all inside the timed region.

--impl reference times the FP64 CPU oracle (the checker) on a bounded sample of the
same workload on the host cores. With --gpus N > 1 (torchrun) every rank runs an
independent replica of the job ("replicas only": the method has no exchange step).
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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

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
        sm = []
        mx = []
        reasons = set()
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
    cfg = W.config_3d_barrier(n=256)
    if rank != 0:
        return
    from oracle import oracle as O
    pb, terms = cfg["problem"], cfg["terms"]
    psi = O.gaussian(pb, **cfg["init"])
    npts = 256 ** 3
    for _ in range(args.warmup):
        psi = O.step(pb, terms, psi, 0)
    t0 = time.perf_counter()
    for k in range(args.steps):
        psi = O.step(pb, terms, psi, k)
    el = time.perf_counter() - t0
    v = npts * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"] + " c128 VKV (oracle: 1 Strang step per bench step)",
                       "grid": [256, 256, 256], "dt": 0.002},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "one Strang step of the 256^3 barrier workload per bench step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="c128", choices=["c128", "c64", "c128f"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nt", type=int, default=200)
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    import torch
    from paper_1306_3247_gb300 import wavepacket as WPK

    torch.cuda.set_device(local)
    cfg = W.config_3d_barrier(n=args.n)
    pb, terms = cfg["problem"], cfg["terms"]
    nt, nprint = args.nt, cfg["nprint"]
    npts = math.prod(pb["n"][: pb["ndim"]])
    stream = torch.cuda.Stream()
    P = WPK.Propagator(pb, terms, args.precision, stream=stream.cuda_stream)
    # resident initial state (complex128) and pinned host buffers
    P.init_gaussian(**cfg["init"])
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

    for _ in range(args.warmup):
        job_device()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = P.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        obs = job_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    dev_ms = ev0.elapsed_time(ev1)
    launches = P.launches - launches0
    barrier(world)
    clk = clocks.stop()
    dev_ms = max_over_ranks(world, dev_ms)
    value = world * npts * nt * args.steps / (dev_ms / 1e3)

    # end to end through the C ABI with host buffers
    job_e2e()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        job_e2e()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = world * npts * nt * args.steps / e2e_s

    # per-kernel durations with CUDA events on the launching stream (one extra job)
    P.profile(True)
    job_device()
    prof = P.profile_read()
    P.profile(False)
    elem = 8 if args.precision == "c64" else 16
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_n, dom_ms) = dom
    avg_s = dom_ms / max(1, dom_n) / 1e3
    bytes_per_launch = 2 * npts * elem  # one read and one write of the state
    achieved = bytes_per_launch / avg_s / 1e9
    pk, src = peaks()

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, dt, cores = cpu_baseline_run(cfg, args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} Strang step(s) of the {args.n}^3 workload ({dt:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"c128": "f64", "c64": "f32", "c128f": "f32x2"}[args.precision],
            "data": "synthetic",
            "config": {"workload": cfg["name"] + f" {args.precision} VKV, {nt} steps, observables every {nprint}",
                       "grid": pb["n"], "dt": pb["dt"], "steps_per_job": nt, "parallelism": "replicas",
                       "l2": "state 268 MB > 129 MB L2 (c128)"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": npts * 16, "d2h_bytes_per_step": npts * 16
                    + 16 * 8 * (1 + nt // nprint)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None,
                         "peak_source": src, "avg_launch_ms": avg_s * 1e3, "launches": dom_n},
            "kernels": {k: {"launches": v[0], "total_ms": v[1]} for k, v in prof.items() if v[0]},
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    P.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
