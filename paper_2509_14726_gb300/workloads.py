"""Seeded synthetic inputs for the MPPI racing solve.

This module builds the *inputs* of the controller (Algorithm 1 of arXiv
2509.14726 lists them: the waypoints W, the arc-length path P_arc and the
time-parameterised reference tau_ref) and the configuration values of the
workloads.  It holds none of the controller's own arithmetic: no sampling,
no dynamics integration of samples, no costs and no weights.  Both the CUDA
path and the FP64 oracle consume the tables built here.

Tracks
  * ``circle_track``: gates on a circle, yaw tangent to it (counter-clockwise).
  * ``random_course``: gate centres rejection-sampled in a box with a minimum
    spacing, ordered by polar angle around the box centre so that they form a
    loop, gate yaw = heading of (c[i+1] - c[i-1]) plus a uniform jitter.
The paper's own tracks (Circle, Figure-8, Split-S, Sec. V-A) are not given as
data; these synthetic tracks stand in for them.

Path (Sec. IV-B, Eq. 9 needs P_arc(theta)): a closed cubic spline through the
gate centres with chord-length knots, its arc length integrated by 16-point
Gauss-Legendre on sub-intervals, resampled at S uniform arc-length nodes that
store position and unit tangent.

Reference (Sec. IV-B, Eq. 8 needs x_ref(t)): the path flown at a constant
speed; velocity along the tangent, attitude from the thrust direction
(a + g e_z) with the body x axis along the horizontal heading, body rates from
a central difference of the attitude.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

GRAVITY = 9.81
MASS = 0.85
INERTIA = (0.0025, 0.0025, 0.0043)

OBJ_GATE, OBJ_CONTOUR, OBJ_TRACK = 0, 1, 2
OBJECTIVE_NAMES = {OBJ_GATE: "gate", OBJ_CONTOUR: "contour", OBJ_TRACK: "track"}


# --------------------------------------------------------------------------
# configuration values
# --------------------------------------------------------------------------

@dataclasses.dataclass
class ModelConfig:
    """Quadrotor with collective-thrust / body-rate input (Eq. 2 with CTBR)."""
    mass: float = MASS
    inertia: Tuple[float, float, float] = INERTIA
    gravity: float = GRAVITY
    k_omega: float = 20.0
    drag: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    u_min: Tuple[float, ...] = (0.0, -10.0, -10.0, -10.0, -20.0)
    u_max: Tuple[float, ...] = (4 * MASS * GRAVITY, 10.0, 10.0, 10.0, 20.0)
    omega_max: float = 10.0
    z_floor: float = 0.0
    kind: int = 0              # 0: collective thrust + body rates, 1: rotor-thrust rates
    arm: float = 0.15          # rotor model: arm length l, m
    c_tau: float = 0.01        # rotor model: drag-torque coefficient, m
    thrust_min: float = 0.0    # rotor model: per-rotor thrust range, N (Table I)
    thrust_max: float = 10.0

    @property
    def hover(self) -> float:
        return self.mass * self.gravity


@dataclasses.dataclass
class SolveConfig:
    """Sampling, objective and weighting parameters of one controller."""
    objective: int = OBJ_GATE
    K: int = 256
    N: int = 20
    dt: float = 0.05
    lam: float = 1.0
    sigma: Tuple[float, ...] = (0.3 * MASS * GRAVITY, 1.0, 1.0, 1.0, 5.0)
    seed: int = 0
    drone_id: int = 0
    w_limit: float = 1.0e3
    q_near: float = 0.05
    r_near: float = 1.5
    temporal_rule: int = 1
    q_lag: float = 1.0
    q_cont: float = 10.0
    q_omega: Tuple[float, float, float] = (0.001, 0.001, 0.001)
    r_dv: float = 0.001
    r_dthrust: float = 0.001
    mu: float = 0.1
    v_theta_max: float = 20.0
    theta_back: float = 2.0
    theta_ahead: float = 10.0
    Q: Tuple[float, ...] = (10.0,) * 3 + (0.1,) * 3 + (1.0,) * 4 + (0.01,) * 3
    QN: Tuple[float, ...] = (20.0,) * 3 + (0.2,) * 3 + (2.0,) * 4 + (0.02,) * 3
    R: Tuple[float, float, float, float] = (0.001, 0.01, 0.01, 0.01)
    flag_eps: float = 1.0e-5
    nominal_sample: int = 0  # 1: sample 0 is the unperturbed nominal
    warm_start: int = 0      # 0: shift by one step, 1: keep the complete sequence


@dataclasses.dataclass
class Track:
    gates: np.ndarray            # [n][6] cx cy cz yaw half_w half_h
    closed: bool
    path: np.ndarray             # [S][6] p, unit tangent
    L: float
    ref: np.ndarray              # [T][13] p v q(wxyz) omega
    dt_ref: float

    @property
    def n_gates(self) -> int:
        return int(self.gates.shape[0])

    def as_f32(self) -> "Track":
        """The same track with every table rounded to binary32."""
        r = lambda a: np.asarray(a, np.float32).astype(np.float64)
        return Track(r(self.gates), self.closed, r(self.path), float(np.float32(self.L)),
                     r(self.ref), float(np.float32(self.dt_ref)))


def _r32(v):
    if isinstance(v, (tuple, list)):
        return tuple(float(np.float32(x)) for x in v)
    if isinstance(v, float):
        return float(np.float32(v))
    return v


def f32_model(mc: ModelConfig) -> ModelConfig:
    """The same model with every real parameter rounded to binary32 (what the
    CUDA path receives)."""
    return ModelConfig(**{f.name: _r32(getattr(mc, f.name)) for f in dataclasses.fields(mc)})


def f32_solve(sc: SolveConfig) -> SolveConfig:
    """The same solve parameters with every real value rounded to binary32."""
    return SolveConfig(**{f.name: _r32(getattr(sc, f.name)) for f in dataclasses.fields(sc)})


# --------------------------------------------------------------------------
# gates
# --------------------------------------------------------------------------

def circle_gates(n: int = 4, radius: float = 5.0, height: float = 2.0,
                 size: float = 1.5) -> np.ndarray:
    g = np.zeros((n, 6))
    for i in range(n):
        phi = 2.0 * math.pi * i / n
        g[i] = (radius * math.cos(phi), radius * math.sin(phi), height,
                phi + 0.5 * math.pi, 0.5 * size, 0.5 * size)
    return g


def figure8_gates(n: int = 8, a: float = 12.0, height: float = 3.0, size: float = 1.5) -> np.ndarray:
    """Gates on the lemniscate (a sin t, a sin t cos t) at equal parameter
    steps, facing along the curve (a stand-in for a figure-8 race track; the
    crossing at the centre is flown twice per lap)."""
    g = np.zeros((n, 6))
    for i in range(n):
        t = 2.0 * math.pi * (i + 0.5) / n
        x, y = a * math.sin(t), a * math.sin(t) * math.cos(t)
        dx, dy = a * math.cos(t), a * math.cos(2.0 * t)
        g[i] = (x, y, height, math.atan2(dy, dx), 0.5 * size, 0.5 * size)
    return g


def figure8_track(n: int = 8, a: float = 12.0, height: float = 3.0, S: int = 1024) -> Track:
    key = ("figure8", n, a, height, S)
    if key not in _TRACK_CACHE:
        _TRACK_CACHE[key] = build_track(figure8_gates(n, a, height), S)
    return _TRACK_CACHE[key]


def random_gates(seed: int, n: int, box=(30.0, 30.0, 6.0), z_low: float = 1.0,
                 min_spacing: float = 6.0, yaw_jitter_deg: float = 45.0,
                 size: float = 1.5) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([0x6A7E, int(seed)]))
    pts: List[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place gates with the requested spacing")
        c = np.array([rng.uniform(-box[0] / 2, box[0] / 2), rng.uniform(-box[1] / 2, box[1] / 2),
                      rng.uniform(z_low, z_low + box[2])])
        if all(np.linalg.norm(c - p) >= min_spacing for p in pts):
            pts.append(c)
    P = np.array(pts)
    order = np.argsort(np.arctan2(P[:, 1], P[:, 0]))
    P = P[order]
    g = np.zeros((n, 6))
    for i in range(n):
        d = P[(i + 1) % n] - P[(i - 1) % n]
        yaw = math.atan2(d[1], d[0]) + math.radians(rng.uniform(-yaw_jitter_deg, yaw_jitter_deg))
        g[i] = (P[i, 0], P[i, 1], P[i, 2], yaw, 0.5 * size, 0.5 * size)
    return g


# --------------------------------------------------------------------------
# closed cubic spline through the gate centres, arc-length resampled
# --------------------------------------------------------------------------

class ClosedSpline:
    """C2 closed cubic spline with chord-length knots (piecewise on [t_i, t_i+1]).

    Arc length is integrated by 16-point Gauss-Legendre on 64 sub-intervals
    per segment; the inverse (parameter at a given arc length) takes the
    bracketing sub-interval and refines with vectorised Newton steps."""

    SUB = 64

    def __init__(self, pts: np.ndarray):
        pts = np.asarray(pts, float)
        n = pts.shape[0]
        h = np.linalg.norm(np.roll(pts, -1, axis=0) - pts, axis=1)
        A = np.zeros((n, n))
        rhs = np.zeros((n, 3))
        for i in range(n):
            hm, hi = h[i - 1], h[i]
            A[i, (i - 1) % n] += hm
            A[i, i] += 2.0 * (hm + hi)
            A[i, (i + 1) % n] += hi
            rhs[i] = 6.0 * ((pts[(i + 1) % n] - pts[i]) / hi - (pts[i] - pts[i - 1]) / hm)
        M = np.linalg.solve(A, rhs)
        self.n, self.h, self.y, self.M = n, h, pts, M
        y1, m1 = np.roll(pts, -1, axis=0), np.roll(M, -1, axis=0)
        self.ca = pts
        self.cb = (y1 - pts) / h[:, None] - h[:, None] * (2.0 * M + m1) / 6.0
        self.cc = 0.5 * M
        self.cd = (m1 - M) / (6.0 * h[:, None])
        self._glx, self._glw = np.polynomial.legendre.leggauss(16)
        # arc length at the sub-interval edges of every segment
        edges = h[:, None] * np.linspace(0.0, 1.0, self.SUB + 1)[None, :]      # [n][SUB+1]
        a, b = edges[:, :-1], edges[:, 1:]
        x = 0.5 * (b - a)[..., None] * self._glx + 0.5 * (a + b)[..., None]    # [n][SUB][16]
        seg = np.repeat(np.arange(n)[:, None], self.SUB, axis=1)
        sp = np.linalg.norm(self.d1(seg[..., None], x), axis=-1)
        sub_len = 0.5 * (b - a) * np.einsum("ijk,k->ij", sp, self._glw)
        self.sub_edges = edges
        self.sub_s = np.concatenate([np.zeros((n, 1)), np.cumsum(sub_len, axis=1)], axis=1)
        self.seg_len = self.sub_s[:, -1]
        self.s_knot = np.concatenate([[0.0], np.cumsum(self.seg_len)])
        self.L = float(self.s_knot[-1])

    def d0(self, i, tau):
        tau = np.asarray(tau)[..., None]
        return self.ca[i] + tau * (self.cb[i] + tau * (self.cc[i] + tau * self.cd[i]))

    def d1(self, i, tau):
        tau = np.asarray(tau)[..., None]
        return self.cb[i] + tau * (2.0 * self.cc[i] + 3.0 * tau * self.cd[i])

    def d2(self, i, tau):
        tau = np.asarray(tau)[..., None]
        return 2.0 * self.cc[i] + 6.0 * tau * self.cd[i]

    def locate(self, s):
        """Segment index and local parameter at arc length(s) s (array)."""
        s = np.mod(np.asarray(s, float), self.L)
        i = np.clip(np.searchsorted(self.s_knot, s, side="right") - 1, 0, self.n - 1)
        r = s - self.s_knot[i]
        j = np.clip(np.array([np.searchsorted(self.sub_s[ii], rr, side="right") - 1
                              for ii, rr in zip(np.atleast_1d(i), np.atleast_1d(r))]), 0, self.SUB - 1)
        j = j.reshape(np.shape(s))
        a = self.sub_edges[i, j]
        b = self.sub_edges[i, j + 1]
        target = r - self.sub_s[i, j]
        tau = a + (b - a) * target / np.maximum(self.sub_s[i, j + 1] - self.sub_s[i, j], 1e-300)
        for _ in range(6):
            x = 0.5 * (tau - a)[..., None] * self._glx + 0.5 * (tau + a)[..., None]
            sp = np.linalg.norm(self.d1(np.asarray(i)[..., None], x), axis=-1)
            arc = 0.5 * (tau - a) * (sp @ self._glw)
            f = arc - target
            tau = np.clip(tau - f / np.linalg.norm(self.d1(i, tau), axis=-1), a, b)
        return i, tau

    def frame(self, s):
        """Position, unit tangent and curvature vector dT/ds at arc length(s) s."""
        i, tau = self.locate(s)
        p = self.d0(i, tau)
        d1 = self.d1(i, tau)
        d2 = self.d2(i, tau)
        sp = np.linalg.norm(d1, axis=-1)[..., None]
        T = d1 / sp
        kappa = (d2 - np.sum(d2 * T, axis=-1)[..., None] * T) / (sp * sp)
        return p, T, kappa


def path_table(spline: ClosedSpline, S: int = 1024) -> Tuple[np.ndarray, float]:
    L = spline.L
    p, T, _ = spline.frame(np.arange(S) * L / S)
    return np.concatenate([p, T], axis=1), L


def _rot_to_quat(R: np.ndarray) -> np.ndarray:
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    if tr > 0:
        s = 2.0 * math.sqrt(tr + 1.0)
        q = np.array([0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s])
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = 2.0 * math.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2])
        q = np.array([(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s])
    elif R[1, 1] > R[2, 2]:
        s = 2.0 * math.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2])
        q = np.array([(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s])
    else:
        s = 2.0 * math.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1])
        q = np.array([(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s])
    return q / np.linalg.norm(q)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def yaw_quat(yaw: float) -> np.ndarray:
    return np.array([math.cos(0.5 * yaw), 0.0, 0.0, math.sin(0.5 * yaw)])


def reference_table(spline: ClosedSpline, speed: float = 8.0, dt_nominal: float = 0.005,
                    gravity: float = GRAVITY) -> Tuple[np.ndarray, float]:
    """Full-state reference of the closed path flown at constant speed."""
    L = spline.L
    T = int(math.ceil(L / (speed * dt_nominal)))
    dt = L / (speed * T)
    p, Tn, kap = spline.frame(speed * dt * np.arange(T))
    a = speed * speed * kap
    zb = a + np.array([0.0, 0.0, gravity])
    zb /= np.linalg.norm(zb, axis=1, keepdims=True)
    xc = np.stack([Tn[:, 0], Tn[:, 1], np.zeros(T)], axis=1)
    xc /= np.linalg.norm(xc, axis=1, keepdims=True)
    yb = np.cross(zb, xc)
    yb /= np.linalg.norm(yb, axis=1, keepdims=True)
    xb = np.cross(yb, zb)
    Qs = np.zeros((T, 4))
    for i in range(T):
        q = _rot_to_quat(np.column_stack([xb[i], yb[i], zb[i]]))
        if i and np.dot(q, Qs[i - 1]) < 0:
            q = -q
        Qs[i] = q
    rows = np.zeros((T, 13))
    rows[:, 0:3] = p
    rows[:, 3:6] = speed * Tn
    rows[:, 6:10] = Qs
    for i in range(T):
        qp, qm = Qs[(i + 1) % T], Qs[(i - 1) % T]
        if np.dot(qp, Qs[i]) < 0:
            qp = -qp
        if np.dot(qm, Qs[i]) < 0:
            qm = -qm
        qdot = (qp - qm) / (2.0 * dt)
        conj = Qs[i] * np.array([1.0, -1.0, -1.0, -1.0])
        rows[i, 10:13] = 2.0 * _qmul(conj, qdot)[1:]
    return rows, dt


def build_track(gates: np.ndarray, S: int = 1024, speed: float = 8.0,
                dt_ref: float = 0.005, with_reference: bool = True) -> Track:
    spline = ClosedSpline(gates[:, :3])
    path, L = path_table(spline, S)
    if with_reference:
        ref, dtr = reference_table(spline, speed, dt_ref)
    else:
        ref, dtr = np.zeros((1, 13)), 1.0
        ref[0, 6] = 1.0
    return Track(np.asarray(gates, float), True, path, L, ref, dtr)


_TRACK_CACHE = {}


def circle_track(n: int = 4, radius: float = 5.0, height: float = 2.0, S: int = 1024,
                 with_reference: bool = True) -> Track:
    key = ("circle", n, radius, height, S, with_reference)
    if key not in _TRACK_CACHE:
        _TRACK_CACHE[key] = build_track(circle_gates(n, radius, height), S, with_reference=with_reference)
    return _TRACK_CACHE[key]


def random_course(seed: int, n_gates: int = 7, S: int = 1024, with_reference: bool = True) -> Track:
    key = ("course", seed, n_gates, S, with_reference)
    if key not in _TRACK_CACHE:
        _TRACK_CACHE[key] = build_track(random_gates(seed, n_gates), S, with_reference=with_reference)
    return _TRACK_CACHE[key]


def hover_state_before_gate(gates: np.ndarray, gate: int = 0, back: float = 1.0) -> np.ndarray:
    """Hover 1 m in front of a gate, facing through it."""
    g = gates[gate]
    n = np.array([math.cos(g[3]), math.sin(g[3]), 0.0])
    x = np.zeros(13)
    x[0:3] = g[:3] - back * n
    x[6:10] = yaw_quat(g[3])
    return x


def perturbed_states(base: np.ndarray, count: int, seed: int, sigma_p: float = 0.1,
                     sigma_v: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([0x51A7, int(seed)]))
    X = np.repeat(base[None, :], count, axis=0)
    X[:, 0:3] += rng.normal(0.0, sigma_p, (count, 3))
    X[:, 3:6] += rng.normal(0.0, sigma_v, (count, 3))
    return X


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def c1_single_gate():
    """Plain single solve, gate progress: K=256, N=20, dt=0.05, 4-gate circle."""
    tr = circle_track(4, 5.0, 2.0)
    cfg = SolveConfig(objective=OBJ_GATE, K=256, N=20, dt=0.05, lam=1.0, seed=0)
    return ModelConfig(), cfg, tr, hover_state_before_gate(tr.gates, 0, 1.0)


def c2_full_scale(objective: int = OBJ_GATE, seed: int = 7):
    """Single drone, full scale: K=4096, N=50, dt=0.02, seeded 7-gate course."""
    tr = random_course(seed, 7)
    cfg = SolveConfig(objective=objective, K=4096, N=50, dt=0.02, lam=1.0, seed=0)
    return ModelConfig(), cfg, tr, hover_state_before_gate(tr.gates, 0, 1.0)


def rotor_model() -> ModelConfig:
    """The input parameterisation of Eq. 2 as printed: rotor-thrust rates
    u = dT_s/dt in [-10, 10] per rotor and thrusts T_s in [0, 10] N (Table I);
    the 5th input (progress acceleration, contouring) keeps its range."""
    return ModelConfig(kind=1, u_min=(-10.0, -10.0, -10.0, -10.0, -20.0), u_max=(10.0, 10.0, 10.0, 10.0, 20.0))


def rotor_solve(sc: SolveConfig) -> SolveConfig:
    """A solve configuration for the rotor model: the same weights, noise of
    5 N/s per rotor rate (Table I gives the range, not the spread)."""
    return dataclasses.replace(sc, sigma=(5.0, 5.0, 5.0, 5.0, sc.sigma[4]))


def paper_table1(objective: int = OBJ_GATE, K: int = 8192, seed: int = 7):
    """The solve size of the paper's simulation parameters (Table I): 8192
    samples, horizon 20, dt 0.03 s, temperature 0.01, on the seeded 7-gate
    course (the paper's tracks are not available).  K=2048 is the sample count
    of its onboard flights at 50 Hz (Sec. V-C)."""
    tr = random_course(seed, 7)
    cfg = SolveConfig(objective=objective, K=K, N=20, dt=0.03, lam=0.01, seed=0)
    return ModelConfig(), cfg, tr, hover_state_before_gate(tr.gates, 0, 1.0)


@dataclasses.dataclass
class BatchItem:
    drone_id: int
    objective: int
    K: int
    N: int
    n_gates: int
    track: Track
    x0: np.ndarray


def c3_batch(n_drones: int = 256, seed: int = 3, K_lo: int = 1024, K_hi: int = 16384,
             N_lo: int = 20, N_hi: int = 80, S: int = 1024) -> List[BatchItem]:
    """Uneven batch: K log-uniform, N uniform, 5-9 gates, objective = id mod 3."""
    rng = np.random.default_rng(np.random.SeedSequence([0xC3, int(seed)]))
    items = []
    for d in range(n_drones):
        K = int(round(math.exp(rng.uniform(math.log(K_lo), math.log(K_hi)))))
        N = int(rng.integers(N_lo, N_hi + 1))
        ng = int(rng.integers(5, 10))
        tr = random_course(1000 + d, ng, S)
        x0 = hover_state_before_gate(tr.gates, 0, 1.0)
        items.append(BatchItem(d, d % 3, K, N, ng, tr, x0))
    return items


def c4_precision(seed: int = 7):
    """Large single solve: K=65536, N=100, dt=0.01, gate progress, 7-gate course."""
    tr = random_course(seed, 7)
    cfg = SolveConfig(objective=OBJ_GATE, K=65536, N=100, dt=0.01, lam=1.0, seed=0)
    return ModelConfig(), cfg, tr, hover_state_before_gate(tr.gates, 0, 1.0)


@dataclasses.dataclass
class ServeDrone:
    drone_id: int
    rate_hz: float
    objective: int
    n_gates: int
    track: Track
    x0: np.ndarray


def c5_fleet(n_drones: int = 2000, seed: int = 5, S: int = 1024,
             distinct_tracks: int = 64) -> List[ServeDrone]:
    """Serving fleet: rate class id mod 3 -> 50/100/200 Hz, 5-9 gate tracks.

    Tracks are drawn from a pool of ``distinct_tracks`` seeded courses so that
    building the tables stays quick; drones on the same course still have
    their own key, nominal, counters and state.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0xC5, int(seed)]))
    rates = (50.0, 100.0, 200.0)
    out = []
    for d in range(n_drones):
        t_id = d % distinct_tracks
        ng = 5 + (t_id % 5)
        tr = random_course(5000 + t_id, ng, S)
        x0 = hover_state_before_gate(tr.gates, 0, 1.0)
        out.append(ServeDrone(d, rates[d % 3], int(rng.integers(0, 3)), ng, tr, x0))
    return out


def poisson_arrivals(rate_hz: float, horizon_s: float, rng: np.random.Generator,
                     start: Optional[float] = None) -> np.ndarray:
    """Request times jittered around a nominal rate: exponential gaps, mean 1/rate."""
    t = rng.uniform(0.0, 1.0 / rate_hz) if start is None else start
    ts = []
    while t < horizon_s:
        ts.append(t)
        t += rng.exponential(1.0 / rate_hz)
    return np.array(ts)
