"""Serving driver: replays a timed request stream against the continuous-batching server.

Requests are submitted when their arrival time comes (wall clock from the start of the
run, optionally compressed by time_scale), the server is polled, and every request's
latency runs from its arrival to the moment its completion is seen. The scheduling itself
(admission by the memory budget, per-request streams, chunk issue) is the library's
wp_server_*; this module only feeds it and measures.
"""
import math
import time

import numpy as np

from . import wavepacket as WPK


def serve(requests, budget_bytes=80e9, nslots=32, chunk_steps=50, precision="c64", time_scale=1.0,
          want_states=False, poll_sleep=2e-4):
    """requests: list of (arrival_s, job dict) sorted by arrival. Returns a summary dict and,
    per request id, (observables record, state or None, latency_s)."""
    results = {}
    lat = []
    failed = []
    points_steps = 0
    with WPK.Server(budget_bytes, nslots, chunk_steps) as srv:
        t0 = time.perf_counter()
        arrivals = {}
        i = 0
        n = len(requests)
        while i < n or srv.pending > 0:
            now = time.perf_counter() - t0
            while i < n and requests[i][0] * time_scale <= now:
                arr, job = requests[i]
                srv.submit(i, job["problem"], job["terms"], job["init"], job["nt"], precision)
                arrivals[i] = t0 + arr * time_scale
                i += 1
            done = srv.progress()
            seen = time.perf_counter()
            for rid in done:
                try:
                    psi, obs, _ = srv.fetch(rid, want_states)
                except WPK.WavepacketError as e:
                    failed.append((rid, e.status))
                    continue
                job = requests[rid][1]
                latency = seen - arrivals[rid]
                lat.append(latency)
                points_steps += math.prod(job["problem"]["n"][: job["problem"]["ndim"]]) * job["nt"]
                results[rid] = (obs, psi, latency)
            if not done:
                time.sleep(poll_sleep)
        wall = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3
    span = requests[-1][0] * time_scale if requests else 0.0
    summary = {
        "requests": n,
        "completed": len(lat),
        "failed": len(failed),
        "wall_s": wall,
        "offered_rate": n / span if span > 0 else None,
        "achieved_rate": n / wall if wall > 0 else None,
        "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat) else None,
        "grid_point_steps_per_s": points_steps / wall if wall > 0 else None,
    }
    return summary, results
