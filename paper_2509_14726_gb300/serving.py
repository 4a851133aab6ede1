"""Serving driver: many simulated drones requesting MPPI solves at their own rates.

Each drone issues solve requests at Poisson-jittered times around its control
rate (50, 100 or 200 Hz by drone id), with K and N drawn per request from the
given choices.  The requests are replayed in wall-clock time, optionally with
simulated time running slower than wall time (``time_scale`` < 1 scales every
rate down), against

* the served path: one ``mppi_server`` (continuous batching: requests are
  admitted as slots and scratch memory free up, batches overlap on the device);
* the plain path: one ``mppi_solve`` per request in arrival order on per-drone
  handles (one solve per launch sequence).

Latency of a request = time its result is available on the host - its
scheduled arrival time.  Both paths see the same arrival schedule.  With a
deadline of d control periods, a request that has not started d periods after
its arrival is refused (load shedding: its drone has already moved on); the
served path leaves that to the server (mppi_server_submit_deadline), the plain
path skips it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from . import mppi as M
from . import workloads as W


@dataclasses.dataclass
class Schedule:
    t: np.ndarray        # arrival time, s (wall-clock offset from the start)
    drone: np.ndarray    # drone index
    K: np.ndarray
    N: np.ndarray
    period: np.ndarray   # the requesting drone's control period (wall clock), s


def make_schedule(fleet: Sequence[W.ServeDrone], duration_s: float, time_scale: float, K_choices, N_choices,
                  seed: int = 0) -> Schedule:
    """Poisson-jittered arrivals: exponential gaps with mean 1 / (rate x time_scale)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5E7, int(seed)]))
    ts, ds = [], []
    for i, d in enumerate(fleet):
        t = W.poisson_arrivals(d.rate_hz * time_scale, duration_s, rng)
        ts.append(t)
        ds.append(np.full(len(t), i, np.int32))
    t = np.concatenate(ts)
    dr = np.concatenate(ds)
    order = np.argsort(t, kind="stable")
    n = len(t)
    K = rng.choice(np.asarray(K_choices, np.int32), n)
    N = rng.choice(np.asarray(N_choices, np.int32), n)
    period = np.array([1.0 / (fleet[i].rate_hz * time_scale) for i in dr[order]])
    return Schedule(t[order], dr[order], K, N, period)


def _stats(lat: np.ndarray, done: int, wall: float, steps: float) -> dict:
    if len(lat) == 0:
        return {"finished": 0}
    return {"finished": int(done), "wall_s": wall, "solves_per_s": done / wall, "rollout_steps_per_s": steps / wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p90_ms": float(np.percentile(lat, 90) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3)}


def _load(out: dict, n: int, refused: int, window: float) -> dict:
    """Offered, achieved and refused request rates over the arrival window."""
    out.update({"offered": n, "offered_per_s": n / window, "achieved_per_s": out.get("finished", 0) / window,
                "refused": int(refused), "refused_per_s": refused / window})
    return out


def run_served(fleet, sched: Schedule, budget_bytes: int = 40 << 30, n_slots: int = 3, max_batch: int = 512,
               K_cap: int = 16384, N_cap: int = 80, dt: float = 0.02, drain_s: float = 30.0,
               deadline_periods: Optional[float] = None) -> dict:
    """Replays the schedule against one mppi_server; returns latency
    statistics of the served requests and the offered / achieved / refused
    rates (refusals only with deadline_periods)."""
    srv = M.Server(len(fleet), budget_bytes, n_slots, max_batch)
    ids = []
    for d in fleet:
        sc = W.SolveConfig(objective=d.objective, K=min(1024, K_cap), N=min(30, N_cap), dt=dt, drone_id=d.drone_id)
        ids.append(srv.add_drone(W.ModelConfig(), sc, d.track, K_cap, N_cap))
    X0 = np.array([d.x0 for d in fleet], np.float32)
    n = len(sched.t)
    lat = np.zeros(n)
    seen = np.zeros(n, bool)
    sid = np.zeros(n, np.int64)
    t_start = M.mppi_clock()
    i = 0
    finished = 0
    refused = 0
    id_to_idx = {}
    steps_done = 0.0
    while finished < n:
        now = M.mppi_clock() - t_start
        j = int(np.searchsorted(sched.t, now, side="right"))
        if j > i:
            sl = slice(i, j)
            dl = None
            if deadline_periods is not None:
                dl = t_start + sched.t[sl] + deadline_periods * sched.period[sl]
            got = srv.submit(sched.drone[sl], X0[sched.drone[sl]], sched.t[sl], sched.K[sl], sched.N[sl], dl)
            for q, rid in enumerate(got):
                id_to_idx[int(rid)] = i + q
            i = j
        while srv.step() > 0:
            pass
        res = srv.poll()
        for r in res:
            k = id_to_idx.pop(int(r["request"]))
            if int(r["status"]) == M.MPPI_ERR_NOT_ADMITTED:
                refused += 1
                continue
            lat[k] = (r["t_done"] - t_start) - sched.t[k]
            seen[k] = True
            steps_done += float(r["K"]) * float(r["N"])
        finished += len(res)
        if now > sched.t[-1] + drain_s:
            break
    wall = M.mppi_clock() - t_start
    st = srv.stats()
    srv.close()
    out = _stats(lat[seen], int(seen.sum()), wall, steps_done)
    out.update({"batches": st["batches"], "scratch_peak_gb": st["scratch_peak"] / 1e9,
                "mean_batch": st["finished"] / max(st["batches"], 1)})
    return _load(out, n, refused, max(float(sched.t[-1]), 1e-9))


def run_plain(fleet, sched: Schedule, K_cap: int = 16384, N_cap: int = 80, dt: float = 0.02,
              time_limit_s: Optional[float] = None, deadline_periods: Optional[float] = None) -> dict:
    """The same schedule, one mppi_solve per request in arrival order (a
    request past its deadline when its turn comes is refused)."""
    ctl = []
    for d in fleet:
        sc = W.SolveConfig(objective=d.objective, K=1024, N=30, dt=dt, drone_id=d.drone_id)
        ctl.append(M.Controller(W.ModelConfig(), sc, d.track, K_cap=K_cap, N_cap=N_cap))
    shape = [(1024, 30)] * len(fleet)
    X0 = [d.x0 for d in fleet]
    n = len(sched.t)
    lat = np.zeros(n)
    steps = 0.0
    t_start = M.mppi_clock()
    done = 0
    refused = 0
    last = n
    for k in range(n):
        now = M.mppi_clock() - t_start
        if time_limit_s is not None and now > time_limit_s:
            last = k
            break
        if now < sched.t[k]:
            while M.mppi_clock() - t_start < sched.t[k]:
                pass
        elif deadline_periods is not None and now > sched.t[k] + deadline_periods * sched.period[k]:
            refused += 1
            lat[k] = -1.0
            continue
        d = int(sched.drone[k])
        if shape[d] != (int(sched.K[k]), int(sched.N[k])):
            ctl[d].set_shape(int(sched.K[k]), int(sched.N[k]))
            shape[d] = (int(sched.K[k]), int(sched.N[k]))
        ctl[d].solve(X0[d], float(sched.t[k]))
        lat[k] = (M.mppi_clock() - t_start) - sched.t[k]
        steps += float(sched.K[k]) * float(sched.N[k])
        done += 1
    wall = M.mppi_clock() - t_start
    for c in ctl:
        c.close()
    served = lat[:last]
    out = _stats(served[served >= 0], done, wall, steps)
    # requests the time limit left unstarted count as refused too
    return _load(out, n, refused + (n - last), max(float(sched.t[-1]), 1e-9))
