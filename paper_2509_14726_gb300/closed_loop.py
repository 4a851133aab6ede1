"""Closed-loop flights of the three objectives over several laps (the
comparison protocol of Sec. V-A: completion time of three laps, lap times,
waypoint-pass error, tracking RMSE).

The simulated quadrotor is the library's own model (the RK4 step of Eq. 2 that
the controller rolls out, run through ``mppi_rollout_states``), as in the
paper's simulation study where one dynamics model serves plant and
controller.  The controller is a ``Controller`` solving once per control
period and applying u0 for one period (50 Hz at dt = 0.02 s).

Gate passes are detected on the flown trajectory with the crossing rule of
Sec. IV-A: the segment between two control steps crosses the gate plane from
the front and the crossing point lies inside the opening.  Gates count in
order (a lap is the full sequence).  The waypoint-pass error of a pass is the
smallest distance of the flown states to the gate centre within half a second
of the crossing (the state with the minimal distance to the waypoint).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

from . import mppi as M
from . import workloads as W


class Plant:
    """The library's model stepped one control period at a time on the GPU."""

    def __init__(self, mc: W.ModelConfig, dt: float):
        import torch
        self.torch = torch
        self.model = M.make_model(W.f32_model(mc))
        self.rotor = int(mc.kind) == 1
        self.dt = float(dt)
        self.dx0 = torch.zeros(13, dtype=torch.float32, device="cuda")
        self.dU = torch.zeros(4, dtype=torch.float32, device="cuda")
        self.dX = torch.zeros((2, 13), dtype=torch.float32, device="cuda")
        self.dT0 = torch.zeros(4, dtype=torch.float32, device="cuda")
        self.dT = torch.zeros((2, 4), dtype=torch.float32, device="cuda")

    def step(self, x: np.ndarray, u: np.ndarray, T: Optional[np.ndarray] = None):
        t = self.torch
        self.dx0.copy_(t.from_numpy(np.float32(x)))
        self.dU.copy_(t.from_numpy(np.float32(u[:4])))
        if self.rotor:
            self.dT0.copy_(t.from_numpy(np.float32(T)))
            M.mppi_rollout_states_rotor(self.model, self.dt, 1, 1, self.dx0.data_ptr(), self.dT0.data_ptr(),
                                        self.dU.data_ptr(), self.dX.data_ptr(), self.dT.data_ptr())
            X, Tn = self.dX.cpu().numpy(), self.dT.cpu().numpy()
            return X[1].astype(np.float64), Tn[1].astype(np.float64)
        M.mppi_rollout_states(self.model, self.dt, 1, 1, self.dx0.data_ptr(), self.dU.data_ptr(),
                              self.dX.data_ptr())
        return self.dX.cpu().numpy()[1].astype(np.float64), None


def _gate_frame(g):
    n = np.array([math.cos(g[3]), math.sin(g[3]), 0.0])
    lat = np.array([-math.sin(g[3]), math.cos(g[3]), 0.0])
    return np.asarray(g[:3], float), n, lat


def crossing(g, pa: np.ndarray, pb: np.ndarray):
    """Sec. IV-A crossing of gate g by the segment pa -> pb: returns the
    fraction along the segment, or None."""
    c, n, lat = _gate_frame(g)
    sa, sb = float(n @ (pa - c)), float(n @ (pb - c))
    if not (sa < 0.0 <= sb):
        return None
    a = sa / (sa - sb)
    e = pa + a * (pb - pa) - c
    if abs(float(lat @ e)) <= g[4] and abs(e[2]) <= g[5]:
        return a
    return None


@dataclasses.dataclass
class Flight:
    objective: int
    model: str
    completed: bool
    gates_passed: int
    time_s: float
    lap_times_s: List[float]
    waypoint_error_m: float
    tracking_rmse_m: Optional[float]
    mean_speed_mps: float
    max_speed_mps: float
    solve_ms_p50: float

    def as_dict(self) -> Dict:
        return dataclasses.asdict(self)


def fly(mc: W.ModelConfig, sc: W.SolveConfig, track: W.Track, x0: np.ndarray, laps: int = 3,
        t_max: float = 60.0, noise_gen: Optional[int] = None, t_ref0: float = 0.0) -> Flight:
    """Flies the controller in closed loop until `laps` laps of the gate
    sequence are complete or t_max seconds have passed.  t_ref0 offsets the
    reference clock (tracking: the reference time at the start)."""
    import time as _time
    ctl = M.Controller(mc, sc, track, noise_gen=noise_gen)
    plant = Plant(mc, sc.dt)
    rotor = int(mc.kind) == 1
    T = np.full(4, mc.mass * mc.gravity / 4) if rotor else None
    gates = np.asarray(track.gates, float)
    n_g = len(gates)
    target = laps * n_g
    x = np.asarray(x0, float).copy()
    t = 0.0
    P: List[np.ndarray] = [x[:3].copy()]
    V: List[float] = [float(np.linalg.norm(x[3:6]))]
    times: List[float] = [0.0]
    passes: List[float] = []
    gi = 0
    solve_ms: List[float] = []
    while t < t_max and len(passes) < target:
        t0 = _time.perf_counter()
        u0, _ = ctl.solve(x, t + t_ref0)
        solve_ms.append((_time.perf_counter() - t0) * 1e3)
        xn, T = plant.step(x, np.asarray(u0, float), T)
        a = crossing(gates[gi % n_g], x[:3], xn[:3])
        if a is not None:
            passes.append(t + a * sc.dt)
            gi += 1
        x, t = xn, t + sc.dt
        P.append(x[:3].copy())
        V.append(float(np.linalg.norm(x[3:6])))
        times.append(t)
        if not np.all(np.isfinite(x)) or x[2] < -5.0:
            break
    ctl.close()
    P_a, T_a = np.array(P), np.array(times)
    # waypoint-pass error: closest flown state to the gate centre near each pass
    errs = []
    for i, tp in enumerate(passes):
        c = gates[i % n_g][:3]
        win = np.abs(T_a - tp) <= 0.5
        errs.append(float(np.min(np.linalg.norm(P_a[win] - c, axis=1))))
    lap_ends = [passes[k * n_g - 1] for k in range(1, len(passes) // n_g + 1)]
    laps_t = [lap_ends[0]] + [lap_ends[k] - lap_ends[k - 1] for k in range(1, len(lap_ends))] if lap_ends else []
    rmse = None
    if sc.objective == W.OBJ_TRACK:
        ref_p = np.array([_ref_position(track, tt + t_ref0) for tt in T_a])
        rmse = float(math.sqrt(np.mean(np.sum((P_a - ref_p) ** 2, axis=1))))
    return Flight(objective=sc.objective, model="rotor" if rotor else "ctbr", completed=len(passes) >= target,
                  gates_passed=len(passes), time_s=passes[-1] if len(passes) >= target else float(t),
                  lap_times_s=laps_t, waypoint_error_m=float(np.mean(errs)) if errs else float("nan"),
                  tracking_rmse_m=rmse, mean_speed_mps=float(np.mean(V)), max_speed_mps=float(np.max(V)),
                  solve_ms_p50=float(np.percentile(solve_ms, 50)) if solve_ms else float("nan"))


def reference_time_before_gate(track: W.Track, back: float) -> float:
    """Reference time at which the reference is `back` metres (of path) before
    gate 0, where it starts (the reference flies the closed spline from gate
    0 at constant speed)."""
    period = track.ref.shape[0] * track.dt_ref
    speed = track.L / period
    return period - back / speed


def _ref_state(track: W.Track, t: float) -> np.ndarray:
    T = track.ref.shape[0]
    s = (t / track.dt_ref) % T
    i = int(math.floor(s))
    f = s - i
    x = (1.0 - f) * track.ref[i % T] + f * track.ref[(i + 1) % T]
    x[6:10] /= np.linalg.norm(x[6:10])
    return x


def _ref_position(track: W.Track, t: float) -> np.ndarray:
    """Position of the periodic reference table at time t (linear)."""
    T = track.ref.shape[0]
    s = (t / track.dt_ref) % T
    i = int(math.floor(s))
    f = s - i
    return (1.0 - f) * track.ref[i % T, :3] + f * track.ref[(i + 1) % T, :3]


def comparison(tracks: Dict[str, W.Track], laps: int = 3, K: int = 4096, N: int = 50, dt: float = 0.02,
               t_max: float = 60.0, models=("ctbr",)) -> Dict[str, Dict]:
    """Each objective on each track (and each input model): the table of the
    paper's comparison, with synthetic tracks standing in for its own."""
    out: Dict[str, Dict] = {}
    for name, tr in tracks.items():
        for model in models:
            for obj in (W.OBJ_GATE, W.OBJ_CONTOUR, W.OBJ_TRACK):
                mc = W.ModelConfig() if model == "ctbr" else W.rotor_model()
                sc = W.SolveConfig(objective=obj, K=K, N=N, dt=dt, lam=1.0, seed=0)
                if model == "rotor":
                    sc = W.rotor_solve(sc)
                # all start 1 m before gate 0: gate progress and contouring from
                # hover, tracking on its reference (flying start at 8 m/s)
                x0, t_ref0 = W.hover_state_before_gate(tr.gates, 0, 1.0), 0.0
                if obj == W.OBJ_TRACK:
                    t_ref0 = reference_time_before_gate(tr, 1.0)
                    x0 = _ref_state(tr, t_ref0)
                f = fly(mc, sc, tr, x0, laps=laps, t_max=t_max, t_ref0=t_ref0)
                out[f"{name}/{model}/{W.OBJECTIVE_NAMES[obj]}"] = f.as_dict()
    return out
