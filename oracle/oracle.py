"""ctypes front end of the FP64 CPU oracle (``mppi_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference leg may load this module; the product path
never does.  It marshals numpy arrays into the oracle's own C structs and
back; all arithmetic happens in ``mppi_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MPPI_ORACLE_LIB") or os.path.join(HERE, "liboracle.so")
SRC_PATH = os.path.join(HERE, "mppi_oracle.c")

D = C.c_double
I32 = C.c_int32
U32 = C.c_uint32
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int32)


class OrModel(C.Structure):
    _fields_ = [("mass", D), ("inertia", D * 3), ("gravity", D), ("k_omega", D), ("drag", D * 3),
                ("u_min", D * 5), ("u_max", D * 5), ("omega_max", D), ("z_floor", D), ("kind", I32), ("arm", D),
                ("c_tau", D), ("thrust_min", D), ("thrust_max", D)]


class OrParams(C.Structure):
    _fields_ = [("objective", I32), ("K", I32), ("N", I32), ("dt", D), ("lam", D), ("sigma", D * 5),
                ("seed", U32), ("drone_id", U32), ("w_limit", D), ("q_near", D), ("r_near", D),
                ("temporal_rule", I32), ("q_lag", D), ("q_cont", D), ("q_omega", D * 3), ("r_dv", D),
                ("r_dthrust", D), ("mu", D), ("v_theta_max", D), ("theta_back", D), ("theta_ahead", D),
                ("Q", D * 13), ("QN", D * 13), ("R", D * 4), ("flag_eps", D), ("nominal_sample", I32),
                ("warm_start", I32)]


class OrTrack(C.Structure):
    _fields_ = [("n_gates", I32), ("closed", I32), ("gates", PD), ("S", I32), ("L", D), ("path", PD),
                ("T", I32), ("dt_ref", D), ("ref", PD)]


class OrState(C.Structure):
    _fields_ = [("U", PD), ("n_nom", I32), ("cap", I32), ("iter", U32), ("gate", I32), ("prevcnt", PI),
                ("n_prev", I32), ("prev_x0", D * 13), ("has_prev", I32), ("theta", D), ("v_theta", D),
                ("c_last", D), ("has_theta", I32), ("rotor", D * 4), ("has_rotor", I32)]


class OrOut(C.Structure):
    _fields_ = [("Z_in", PD), ("Z", PD), ("J", PD), ("Jabs", PD), ("npass", PI), ("first_pass", PI),
                ("near_flag", PI), ("w", PD), ("Unew", PD), ("u0", PD), ("passcnt", PI), ("theta0", PD),
                ("xref", PD), ("Xnom", PD), ("gate_at_start", I32), ("status", I32), ("Us", PD)]


LIB_OMP_PATH = os.path.join(HERE, "liboracle_omp.so")

_libs = {}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no vector intrinsics).
    omp: the same source with OpenMP over the samples of a solve, used only to
    time the oracle on all host cores (the parity checks use the plain build)."""
    path = LIB_OMP_PATH if omp else LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SRC_PATH):
        extra = ["-fopenmp"] if omp else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", *extra,
                               "-o", path, SRC_PATH, "-lm"])
    return path


def lib(omp: bool = False):
    if omp not in _libs:
        L = C.CDLL(build(omp=omp))
        L.or_philox4x32_10.argtypes = [C.POINTER(U32), C.POINTER(U32), C.POINTER(U32)]
        L.or_uniform.argtypes = [U32]
        L.or_uniform.restype = D
        L.or_box_muller.argtypes = [U32, U32, PD]
        L.or_normals4.argtypes = [U32, U32, U32, U32, U32, U32, PD]
        L.or_deriv.argtypes = [C.POINTER(OrModel), PD, PD, PD]
        L.or_rk4_step.argtypes = [C.POINTER(OrModel), PD, PD, D, C.c_int, PD]
        L.or_penalty.argtypes = [C.POINTER(OrModel), C.POINTER(OrParams), PD]
        L.or_penalty.restype = D
        L.or_gate_crossing.argtypes = [PD, PD, PD, PD]
        L.or_gate_crossing.restype = C.c_int
        L.or_path_eval.argtypes = [C.POINTER(OrTrack), D, PD, PD]
        L.or_path_project.argtypes = [C.POINTER(OrTrack), PD, I32, I32]
        L.or_path_project.restype = D
        L.or_ref_eval.argtypes = [C.POINTER(OrTrack), D, PD]
        L.or_solve.argtypes = [C.POINTER(OrModel), C.POINTER(OrParams), C.POINTER(OrTrack),
                               C.POINTER(OrState), PD, D, C.POINTER(OrOut)]
        L.or_solve.restype = C.c_int
        L.or_rollout.argtypes = [C.POINTER(OrModel), C.POINTER(OrParams), C.POINTER(OrTrack), PD, PD, I32,
                                 PI, I32, D, D, D, PD, PD, PI, PD, PD]
        L.or_deriv_rotor.argtypes = [C.POINTER(OrModel), PD, PD, PD]
        L.or_rotor_at.argtypes = [C.POINTER(OrModel), PD, PD, D, PD]
        L.or_rk4_step_rotor.argtypes = [C.POINTER(OrModel), PD, PD, PD, D, C.c_int, PD, PD]
        L.or_rollout.restype = D
        L.or_threads.restype = C.c_int
        _libs[omp] = L
    return _libs[omp]


def threads(omp: bool = False) -> int:
    """Threads the sample loop of a solve runs on."""
    return int(lib(omp).or_threads())


def _pd(a: np.ndarray):
    return a.ctypes.data_as(PD)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(PI)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------
# struct builders
# ----------------------------------------------------------------------------

def make_model(mc) -> OrModel:
    m = OrModel()
    m.mass = mc.mass
    m.inertia[:] = list(mc.inertia)
    m.gravity = mc.gravity
    m.k_omega = mc.k_omega
    m.drag[:] = list(mc.drag)
    m.u_min[:] = list(mc.u_min)
    m.u_max[:] = list(mc.u_max)
    m.kind = int(getattr(mc, "kind", 0))
    m.arm, m.c_tau = getattr(mc, "arm", 0.15), getattr(mc, "c_tau", 0.01)
    m.thrust_min, m.thrust_max = getattr(mc, "thrust_min", 0.0), getattr(mc, "thrust_max", 10.0)
    m.omega_max = mc.omega_max
    m.z_floor = mc.z_floor
    return m


def make_params(sc) -> OrParams:
    p = OrParams()
    p.objective, p.K, p.N = sc.objective, sc.K, sc.N
    p.dt, p.lam = sc.dt, sc.lam
    p.sigma[:] = list(sc.sigma)
    p.seed, p.drone_id = sc.seed & 0xFFFFFFFF, sc.drone_id & 0xFFFFFFFF
    p.w_limit, p.q_near, p.r_near, p.temporal_rule = sc.w_limit, sc.q_near, sc.r_near, sc.temporal_rule
    p.q_lag, p.q_cont = sc.q_lag, sc.q_cont
    p.q_omega[:] = list(sc.q_omega)
    p.r_dv, p.r_dthrust, p.mu, p.v_theta_max = sc.r_dv, sc.r_dthrust, sc.mu, sc.v_theta_max
    p.theta_back, p.theta_ahead = sc.theta_back, sc.theta_ahead
    p.Q[:] = list(sc.Q)
    p.QN[:] = list(sc.QN)
    p.R[:] = list(sc.R)
    p.flag_eps = sc.flag_eps
    p.nominal_sample = getattr(sc, "nominal_sample", 0)
    p.warm_start = getattr(sc, "warm_start", 0)
    return p


class TrackView:
    """Keeps the numpy tables alive for as long as the C struct points at them."""

    def __init__(self, track):
        self.gates = _f64(track.gates)
        self.path = _f64(track.path)
        self.ref = _f64(track.ref)
        t = OrTrack()
        t.n_gates, t.closed = self.gates.shape[0], int(bool(track.closed))
        t.gates = _pd(self.gates)
        t.S, t.L, t.path = self.path.shape[0], float(track.L), _pd(self.path)
        t.T, t.dt_ref, t.ref = self.ref.shape[0], float(track.dt_ref), _pd(self.ref)
        self.c = t


# ----------------------------------------------------------------------------
# function-level access (used by the pin tests)
# ----------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    c = (U32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (U32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (U32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(x: int) -> float:
    return lib().or_uniform(int(x) & 0xFFFFFFFF)


def box_muller(xa: int, xb: int) -> np.ndarray:
    z = np.zeros(2)
    lib().or_box_muller(int(xa) & 0xFFFFFFFF, int(xb) & 0xFFFFFFFF, _pd(z))
    return z


def normals4(seed, drone, m, k, it, blk) -> np.ndarray:
    z = np.zeros(4)
    lib().or_normals4(seed, drone, m, k, it, blk, _pd(z))
    return z


def deriv(mc, x, u) -> np.ndarray:
    m = make_model(mc)
    x, u = _f64(x), _f64(u)
    dx = np.zeros(13)
    lib().or_deriv(C.byref(m), _pd(x), _pd(u), _pd(dx))
    return dx


def rk4_step(mc, x, u, h, renormalise=True) -> np.ndarray:
    m = make_model(mc)
    x, u = _f64(x), _f64(u)
    xn = np.zeros(13)
    lib().or_rk4_step(C.byref(m), _pd(x), _pd(u), float(h), int(renormalise), _pd(xn))
    return xn


def deriv_rotor(mc, x, T) -> np.ndarray:
    m = make_model(mc)
    x, T = _f64(x), _f64(T)
    dx = np.zeros(13)
    lib().or_deriv_rotor(C.byref(m), _pd(x), _pd(T), _pd(dx))
    return dx


def rotor_at(mc, T0, u, t) -> np.ndarray:
    m = make_model(mc)
    T0, u = _f64(T0), _f64(u)
    T = np.zeros(4)
    lib().or_rotor_at(C.byref(m), _pd(T0), _pd(u), float(t), _pd(T))
    return T


def rk4_step_rotor(mc, x, T0, u, h, renormalise=True):
    """One RK4 step of the rotor model; returns (x_next, T_next)."""
    m = make_model(mc)
    x, T0, u = _f64(x), _f64(T0), _f64(u)
    xn, Tn = np.zeros(13), np.zeros(4)
    lib().or_rk4_step_rotor(C.byref(m), _pd(x), _pd(T0), _pd(u), float(h), int(renormalise), _pd(xn), _pd(Tn))
    return xn, Tn


def penalty(mc, sc, x) -> float:
    m, p = make_model(mc), make_params(sc)
    x = _f64(x)
    return lib().or_penalty(C.byref(m), C.byref(p), _pd(x))


def gate_crossing(gate, pa, pb):
    g, a, b = _f64(gate), _f64(pa), _f64(pb)
    info = np.zeros(4)
    r = lib().or_gate_crossing(_pd(g), _pd(a), _pd(b), _pd(info))
    return bool(r), info


def path_eval(track, theta):
    tv = TrackView(track)
    P, T = np.zeros(3), np.zeros(3)
    lib().or_path_eval(C.byref(tv.c), float(theta), _pd(P), _pd(T))
    return P, T


def path_project(track, p, jlo, jhi) -> float:
    tv = TrackView(track)
    p = _f64(p)
    return lib().or_path_project(C.byref(tv.c), _pd(p), int(jlo), int(jhi))


def ref_eval(track, t) -> np.ndarray:
    tv = TrackView(track)
    xr = np.zeros(13)
    lib().or_ref_eval(C.byref(tv.c), float(t), _pd(xr))
    return xr


def rollout(mc, sc, track, x0, U, gate0=0, prev=None, theta0=0.0, vth0=0.0, c_last=None, xref=None, T0=None,
            want_T=False):
    """Rolls one sequence U[N][5] out from x0 (and rotor thrusts T0 for the
    rotor model); returns (J, X[N+1][13], passcnt[N+1]) (+ T[N+1][4] with
    want_T)."""
    m, p, tv = make_model(mc), make_params(sc), TrackView(track)
    N = sc.N
    U = _f64(np.asarray(U).reshape(N, -1))
    if U.shape[1] < 5:
        U = np.ascontiguousarray(np.pad(U, ((0, 0), (0, 5 - U.shape[1]))))
    x0 = _f64(x0)
    X = np.zeros((N + 1, 13))
    pc = np.zeros(N + 1, dtype=np.int32)
    prev_a = np.ascontiguousarray(np.asarray(prev if prev is not None else [0], dtype=np.int32))
    n_prev = 0 if prev is None else len(prev_a)
    if c_last is None:
        c_last = mc.mass * mc.gravity
    xr = _f64(xref) if xref is not None else np.zeros((N + 1, 13))
    if T0 is None:
        T0 = np.full(4, 0.25 * mc.mass * mc.gravity)
    T0 = _f64(T0)
    Tr = np.zeros((N + 1, 4))
    J = lib().or_rollout(C.byref(m), C.byref(p), C.byref(tv.c), _pd(x0), _pd(U), int(gate0), _pi(prev_a),
                         int(n_prev), float(theta0), float(vth0), float(c_last), _pd(xr), _pd(X), _pi(pc),
                         _pd(T0), _pd(Tr))
    if want_T:
        return J, X, pc, Tr
    return J, X, pc


# ----------------------------------------------------------------------------
# the controller: resident state + one solve per call (Algorithm 1)
# ----------------------------------------------------------------------------

class OracleController:
    """FP64 controller that carries the same per-drone state between solves
    as the CUDA library's handle: nominal U*, Philox iteration, gate index,
    pass counts of the previous nominal, last x0, progress state, last thrust."""

    def __init__(self, mc, sc, track, cap: Optional[int] = None, omp: bool = False):
        self.mc, self.sc, self.track = mc, sc, track
        self.omp = omp
        self.m, self.p = make_model(mc), make_params(sc)
        self.tv = TrackView(track)
        self.cap = int(cap or sc.N)
        self.U = np.zeros((self.cap, 5))
        self.prevcnt = np.zeros(self.cap, dtype=np.int32)
        st = OrState()
        st.U, st.n_nom, st.cap = _pd(self.U), 0, self.cap
        st.iter, st.gate, st.prevcnt, st.n_prev, st.has_prev = 0, 0, _pi(self.prevcnt), 0, 0
        st.theta = st.v_theta = 0.0
        st.c_last = mc.mass * mc.gravity
        st.has_theta = 0
        st.has_rotor = 0
        self.st = st

    # state access, so a test can start both sides from the same state
    def set_state(self, U=None, n_nom=None, iter=None, gate=None, prevcnt=None, prev_x0=None,
                  theta=None, v_theta=None, c_last=None, has_theta=None, rotor=None):
        st = self.st
        if rotor is not None:
            st.rotor[:] = [float(v) for v in rotor]
            st.has_rotor = 1
        if U is not None:
            U = np.asarray(U, float)
            self.U[:] = 0.0
            self.U[:U.shape[0], :U.shape[1]] = U
            st.n_nom = U.shape[0] if n_nom is None else n_nom
        if iter is not None:
            st.iter = int(iter)
        if gate is not None:
            st.gate = int(gate)
        if prevcnt is not None:
            pc = np.asarray(prevcnt, np.int32)
            self.prevcnt[:] = 0
            self.prevcnt[:len(pc)] = pc
            st.n_prev = len(pc)
        if prev_x0 is not None:
            st.prev_x0[:] = list(np.asarray(prev_x0, float))
            st.has_prev = 1
        if theta is not None:
            st.theta = float(theta)
            st.has_theta = 1 if has_theta is None else int(has_theta)
        if v_theta is not None:
            st.v_theta = float(v_theta)
        if c_last is not None:
            st.c_last = float(c_last)

    def solve(self, x0, t0: float = 0.0, Z_in: Optional[np.ndarray] = None, want_Z: bool = False,
              want_Us: Optional[bool] = None) -> dict:
        """One solve; want_Us (default: when K N <= 4e6) also returns the
        clamped sampled sequences as "Us" [K][N][5]."""
        K, N = self.sc.K, self.sc.N
        if want_Us is None:
            want_Us = K * N <= 4_000_000
        x0 = _f64(x0)
        o = OrOut()
        res = {
            "J": np.zeros(K), "Jabs": np.zeros(K), "npass": np.zeros(K, np.int32),
            "first_pass": np.zeros(K, np.int32), "near_flag": np.zeros(K, np.int32), "w": np.zeros(K),
            "Unew": np.zeros((N, 5)), "u0": np.zeros(5), "passcnt": np.zeros(N + 1, np.int32),
            "theta0": np.zeros(2), "xref": np.zeros((N + 1, 13)), "Xnom": np.zeros((N + 1, 13)),
        }
        if want_Z:
            res["Z"] = np.zeros((N, K, 5))
            o.Z = _pd(res["Z"])
        if want_Us:
            res["Us"] = np.zeros((K, N, 5))
            o.Us = _pd(res["Us"])
        zin = None
        if Z_in is not None:
            zin = _f64(Z_in)
            o.Z_in = _pd(zin)
        o.J, o.Jabs, o.npass = _pd(res["J"]), _pd(res["Jabs"]), _pi(res["npass"])
        o.first_pass, o.near_flag, o.w = _pi(res["first_pass"]), _pi(res["near_flag"]), _pd(res["w"])
        o.Unew, o.u0, o.passcnt = _pd(res["Unew"]), _pd(res["u0"]), _pi(res["passcnt"])
        o.theta0, o.xref, o.Xnom = _pd(res["theta0"]), _pd(res["xref"]), _pd(res["Xnom"])
        rc = lib(self.omp).or_solve(C.byref(self.m), C.byref(self.p), C.byref(self.tv.c), C.byref(self.st), _pd(x0),
                            float(t0), C.byref(o))
        if rc < 0:
            raise ValueError("oracle solve rejected its arguments")
        res["status"] = int(o.status)
        res["gate_at_start"] = int(o.gate_at_start)
        return res

    @property
    def nominal(self) -> np.ndarray:
        return self.U[: self.st.n_nom].copy()

    @property
    def rotor(self) -> np.ndarray:
        """Rotor thrusts the next solve starts from (rotor model)."""
        if self.st.has_rotor:
            return np.array(list(self.st.rotor))
        return np.full(4, 0.25 * self.mc.mass * self.mc.gravity)

    @property
    def gate(self) -> int:
        return int(self.st.gate)

    @property
    def iter(self) -> int:
        return int(self.st.iter)
