"""Thin driver of the library's serving core (sacd_server_* in include/sacd.h).

``Server`` wraps the C API; ``run_arrivals`` replays a seeded Poisson arrival stream of jobs in
wall-clock time: a job is submitted when its arrival time has passed, the server steps (one outer
iteration of every admitted job per step), and each result's latency is arrival -> result.
"""

from __future__ import annotations

import time

import numpy as np

from . import sacd as S

__all__ = ["Server", "poisson_arrivals", "run_arrivals", "latency_summary"]


class Server:
    def __init__(self, hbm_budget_bytes, max_active=1024, max_admit_per_step=16, stream=None):
        self.s = S.sacd_server_create(hbm_budget_bytes, max_active, max_admit_per_step, stream)
        self._keep = {}
        self._shapes = {}

    def submit(self, spec, iters):
        jid, keep = S.sacd_server_submit(self.s, spec, iters)
        self._keep[jid] = (keep, spec)  # inputs stay alive until the result is drained
        self._shapes[jid] = [(d, spec["rank"]) for d in spec["dims"]]
        return jid

    def step(self):
        return S.sacd_server_step(self.s)

    def results(self):
        res = S.sacd_server_results(self.s)
        for r in res:
            self._keep.pop(r["job_id"], None)
        return res

    def factors(self, job_id):
        return [S.sacd_server_get_factor(self.s, job_id, n, shp) for n, shp in enumerate(self._shapes[job_id])]

    def release(self, job_id):
        S.sacd_server_release(self.s, job_id)
        self._shapes.pop(job_id, None)

    def stats(self):
        return S.sacd_server_stats(self.s)

    def close(self):
        if self.s:
            S.sacd_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def poisson_arrivals(rate, n, seed):
    """n arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_arrivals(server, specs, arrivals, iters, keep_factors=False, timeout_s=3600.0, keep_for=()):
    """Drive `server` with jobs `specs[i]` arriving at `arrivals[i]` (seconds from now).

    Returns (results, wall seconds): results carry latency = result time - arrival time."""
    t0 = time.perf_counter()
    nxt = 0
    pending = {}
    out = []
    n = len(specs)
    while len(out) < n:
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError("serving run exceeded its time limit")
        while nxt < n and arrivals[nxt] <= now:
            jid = server.submit(specs[nxt], iters)
            pending[jid] = (nxt, arrivals[nxt])
            nxt += 1
        active, waiting = server.step()
        for r in server.results():
            i, arr = pending.pop(r["job_id"])
            r["index"] = i
            r["arrival"] = arr
            r["latency"] = (time.perf_counter() - t0) - arr
            if (keep_factors or i in keep_for) and r["status"] == 0:
                r["factors"] = server.factors(r["job_id"])
            server.release(r["job_id"])
            out.append(r)
        if active == 0 and waiting == 0 and nxt < n:
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.01)))
    return out, time.perf_counter() - t0


def latency_summary(results):
    lat = np.array([r["latency"] for r in results if r["status"] == 0])
    if lat.size == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
