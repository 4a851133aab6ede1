"""Python binding of libmppi (include/mppi.h): argument marshalling only.

Every function here converts Python / numpy / torch arguments into the C ABI's
plain structs and pointers and calls the shared library; all arithmetic of the
solve runs in the library's CUDA kernels.  There is no fallback: if the
library is not built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MPPI_LIB") or os.path.join(HERE, "lib", "libmppi.so")

MPPI_OK, MPPI_ERR_ARG, MPPI_ERR_OOM, MPPI_ERR_CUDA, MPPI_ERR_TIMEOUT, MPPI_ERR_NOT_ADMITTED, MPPI_WARN_DEGENERATE = range(7)
NOISE_F32, NOISE_BF16 = 0, 1
NOISEGEN_KERNEL, NOISEGEN_FUSED, NOISEGEN_REGEN, NOISEGEN_SMEM, NOISEGEN_AHEAD = 0, 1, 2, 3, 4
NOISEGEN_DEFAULT = NOISEGEN_KERNEL
ACC_KAHAN32, ACC_F64, ACC_F32 = 0, 1, 2
F = C.c_float
I32 = C.c_int32
U32 = C.c_uint32
PF = C.POINTER(C.c_float)


class MppiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmppi error {code}: {msg}")
        self.code = code


class Model(C.Structure):
    _fields_ = [("kind", I32), ("mass", F), ("inertia", F * 3), ("gravity", F), ("k_omega", F), ("drag", F * 3),
                ("u_min", F * 5), ("u_max", F * 5), ("omega_max", F), ("z_floor", F), ("arm", F), ("c_tau", F),
                ("thrust_min", F), ("thrust_max", F)]


class Params(C.Structure):
    _fields_ = [("objective", I32), ("K", I32), ("N", I32), ("dt", F), ("lam", F), ("sigma", F * 5),
                ("seed", U32), ("drone_id", U32), ("w_limit", F), ("q_near", F), ("r_near", F),
                ("temporal_rule", I32), ("q_lag", F), ("q_cont", F), ("q_omega", F * 3), ("r_dv", F),
                ("r_dthrust", F), ("mu", F), ("v_theta_max", F), ("theta_back", F), ("theta_ahead", F),
                ("Q", F * 13), ("QN", F * 13), ("R", F * 4), ("noise_dtype", I32), ("accum", I32), ("block", I32),
                ("N_cap", I32), ("K_cap", I32), ("noise_gen", I32), ("nominal_sample", I32), ("warm_start", I32),
                ("samples_per_thread", I32)]


class TrackC(C.Structure):
    _fields_ = [("n_gates", I32), ("closed", I32), ("gates", PF), ("S", I32), ("L", F), ("path", PF), ("T", I32),
                ("dt_ref", F), ("ref", PF)]


_lib = None


def load():
    """Loads libmppi.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmppi is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, sz = C.c_void_p, C.c_size_t
    sig = {
        "mppi_default_model": ([C.POINTER(Model)], C.c_int),
        "mppi_default_params": ([C.POINTER(Params), I32, I32, I32, F], C.c_int),
        "mppi_create": ([C.POINTER(Model), C.POINTER(Params), C.POINTER(TrackC), C.POINTER(vp)], C.c_int),
        "mppi_destroy": ([vp], C.c_int),
        "mppi_solve": ([vp, PF, C.c_double, vp, PF], C.c_int),
        "mppi_solve_async": ([vp, vp, C.c_double, vp, vp], C.c_int),
        "mppi_solve_batch": ([I32, C.POINTER(vp), PF, C.POINTER(C.c_double), vp, PF], C.c_int),
        "mppi_batch_create": ([I32, C.POINTER(vp), I32, C.POINTER(vp)], C.c_int),
        "mppi_batch_solve": ([vp, PF, C.POINTER(C.c_double), vp, PF], C.c_int),
        "mppi_batch_solve_async": ([vp, vp, vp, vp, vp], C.c_int),
        "mppi_batch_destroy": ([vp], C.c_int),
        "mppi_batch_profile": ([vp, I32, vp, PF], C.c_int),
        "mppi_set_shape": ([vp, I32, I32], C.c_int),
        "mppi_get_nominal": ([vp, PF], C.c_int),
        "mppi_get_unew": ([vp, PF], C.c_int),
        "mppi_get_costs": ([vp, C.POINTER(C.c_double)], C.c_int),
        "mppi_get_sample_info": ([vp, C.POINTER(I32), C.POINTER(I32)], C.c_int),
        "mppi_get_noise": ([vp, PF], C.c_int),
        "mppi_get_passcnt": ([vp, C.POINTER(I32)], C.c_int),
        "mppi_get_info": ([vp, C.POINTER(I32)], C.c_int),
        "mppi_get_solve_scalars": ([vp, C.POINTER(C.c_double)], C.c_int),
        "mppi_get_xref": ([vp, PF], C.c_int),
        "mppi_export_state": ([vp, vp, C.POINTER(sz)], C.c_int),
        "mppi_import_state": ([vp, vp, sz], C.c_int),
        "mppi_set_gate_index": ([vp, I32], C.c_int),
        "mppi_set_rotor_thrusts": ([vp, PF], C.c_int),
        "mppi_rollout_states_rotor": ([C.POINTER(Model), F, I32, I32, vp, vp, vp, vp, vp, vp], C.c_int),
        "mppi_get_rotor_thrusts": ([vp, PF], C.c_int),
        "mppi_set_noise": ([vp, vp, vp, vp], C.c_int),
        "mppi_philox": ([U32, U32, U32, U32, U32, U32, I32, vp, vp], C.c_int),
        "mppi_normals": ([U32, U32, U32, U32, U32, I32, vp, vp], C.c_int),
        "mppi_rollout_states": ([C.POINTER(Model), F, I32, I32, vp, vp, vp, vp], C.c_int),
        "mppi_device_bytes": ([vp, C.POINTER(sz)], C.c_int),
        "mppi_estimate_bytes": ([C.POINTER(Params), C.POINTER(TrackC), C.POINTER(sz)], C.c_int),
        "mppi_kernel_launches": ([], C.c_uint64),
        "mppi_abi_sizes": ([C.POINTER(sz)], C.c_int),
        "mppi_clock": ([], C.c_double),
        "mppi_server_create": ([I32, sz, I32, I32, C.POINTER(vp)], C.c_int),
        "mppi_server_add_drone": ([vp, C.POINTER(Model), C.POINTER(Params), C.POINTER(TrackC), C.POINTER(I32)], C.c_int),
        "mppi_server_submit": ([vp, I32, vp, vp, vp, vp, vp, vp], C.c_int),
        "mppi_server_submit_deadline": ([vp, I32, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "mppi_server_step": ([vp, C.POINTER(I32)], C.c_int),
        "mppi_server_poll": ([vp, vp, I32, C.POINTER(I32)], C.c_int),
        "mppi_server_stats": ([vp, C.POINTER(C.c_double)], C.c_int),
        "mppi_server_export_drone": ([vp, I32, vp, C.POINTER(sz)], C.c_int),
        "mppi_server_destroy": ([vp], C.c_int),
        "mppi_server_fail_next_launch": ([vp], C.c_int),
        "mppi_set_copy_wait": ([vp, C.c_uint32, I32], C.c_int),
        "mppi_solve_noalloc": ([C.POINTER(Model), C.POINTER(Params), C.POINTER(TrackC), vp, C.c_double, vp, U32, I32,
                                vp, vp, vp], C.c_int),
        "mppi_last_error": ([], C.c_char_p),
        "mppi_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc: int, allow_degenerate: bool = True) -> int:
    if rc == MPPI_OK or (allow_degenerate and rc == MPPI_WARN_DEGENERATE):
        return rc
    raise MppiError(rc, load().mppi_last_error().decode())


def _pf(a: np.ndarray):
    return a.ctypes.data_as(PF)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _stream_ptr(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))


# ---------------------------------------------------------------------------
# struct builders
# ---------------------------------------------------------------------------

def make_model(mc: W.ModelConfig) -> Model:
    m = Model()
    m.kind = int(mc.kind)
    m.mass, m.gravity, m.k_omega = mc.mass, mc.gravity, mc.k_omega
    m.arm, m.c_tau, m.thrust_min, m.thrust_max = mc.arm, mc.c_tau, mc.thrust_min, mc.thrust_max
    m.inertia[:] = list(mc.inertia)
    m.drag[:] = list(mc.drag)
    m.u_min[:] = list(mc.u_min)
    m.u_max[:] = list(mc.u_max)
    m.omega_max, m.z_floor = mc.omega_max, mc.z_floor
    return m


def make_params(sc: W.SolveConfig, noise_dtype: int = NOISE_F32, accum: int = ACC_KAHAN32, block: int = 128,
                N_cap: int = 0, K_cap: int = 0, noise_gen: Optional[int] = None, spt: int = 1) -> Params:
    p = Params()
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
    p.noise_dtype, p.accum, p.block, p.N_cap, p.K_cap = noise_dtype, accum, block, N_cap, K_cap
    p.noise_gen = NOISEGEN_DEFAULT if noise_gen is None else noise_gen
    p.nominal_sample, p.warm_start = int(sc.nominal_sample), int(sc.warm_start)
    p.samples_per_thread = int(spt)
    return p


class TrackArrays:
    """float32 copies of a track's tables plus the C struct that points at them."""

    def __init__(self, track: W.Track):
        self.gates = _f32(track.gates)
        self.path = _f32(track.path)
        self.ref = _f32(track.ref)
        t = TrackC()
        t.n_gates, t.closed = self.gates.shape[0], int(bool(track.closed))
        t.gates = _pf(self.gates)
        t.S, t.L, t.path = self.path.shape[0], float(track.L), _pf(self.path)
        t.T, t.dt_ref, t.ref = self.ref.shape[0], float(track.dt_ref), _pf(self.ref)
        self.c = t


# ---------------------------------------------------------------------------
# C-ABI functions, same names
# ---------------------------------------------------------------------------

def mppi_create(model: Model, params: Params, track: TrackArrays) -> int:
    h = C.c_void_p()
    _check(load().mppi_create(C.byref(model), C.byref(params), C.byref(track.c), C.byref(h)))
    return h.value


def mppi_destroy(h: int) -> None:
    _check(load().mppi_destroy(C.c_void_p(h)))


def mppi_solve(h: int, x0, t0: float = 0.0, stream=None):
    """Returns (u0[5], status)."""
    x = _f32(x0)
    u = np.zeros(5, np.float32)
    rc = _check(load().mppi_solve(C.c_void_p(h), _pf(x), float(t0), _stream_ptr(stream), _pf(u)))
    return u, rc


def mppi_solve_async(h: int, d_x0_ptr: int, t0: float, stream, d_u0_ptr: int) -> None:
    _check(load().mppi_solve_async(C.c_void_p(h), C.c_void_p(d_x0_ptr), float(t0), _stream_ptr(stream),
                                   C.c_void_p(d_u0_ptr)))


def _handles(hs: Sequence[int]):
    arr = (C.c_void_p * len(hs))(*hs)
    return arr


def mppi_solve_batch(hs: Sequence[int], x0s, t0s=None, stream=None):
    n = len(hs)
    x = _f32(np.asarray(x0s).reshape(n, 13))
    t = np.ascontiguousarray(np.zeros(n) if t0s is None else np.asarray(t0s, np.float64))
    u = np.zeros((n, 5), np.float32)
    rc = _check(load().mppi_solve_batch(n, _handles(hs), _pf(x), t.ctypes.data_as(C.POINTER(C.c_double)),
                                        _stream_ptr(stream), _pf(u)))
    return u, rc


def mppi_batch_create(hs: Sequence[int], use_graph: bool = True) -> int:
    b = C.c_void_p()
    _check(load().mppi_batch_create(len(hs), _handles(hs), int(use_graph), C.byref(b)))
    return b.value


def mppi_batch_solve(b: int, n: int, x0s, t0s=None, stream=None):
    x = _f32(np.asarray(x0s).reshape(n, 13))
    t = np.ascontiguousarray(np.zeros(n) if t0s is None else np.asarray(t0s, np.float64))
    u = np.zeros((n, 5), np.float32)
    rc = _check(load().mppi_batch_solve(C.c_void_p(b), _pf(x), t.ctypes.data_as(C.POINTER(C.c_double)),
                                        _stream_ptr(stream), _pf(u)))
    return u, rc


def mppi_batch_solve_async(b: int, d_x0s: int, d_t0s: int, stream, d_u0s: int) -> None:
    _check(load().mppi_batch_solve_async(C.c_void_p(b), C.c_void_p(d_x0s), C.c_void_p(d_t0s), _stream_ptr(stream),
                                         C.c_void_p(d_u0s)))


def mppi_batch_profile(b: int, n_iters: int, stream=None) -> np.ndarray:
    """Mean ms per iteration of [noise, rollout gate, rollout contour, rollout
    track, nominal, total] (launched without the graph, with CUDA events)."""
    ms = np.zeros(6, np.float32)
    _check(load().mppi_batch_profile(C.c_void_p(b), int(n_iters), _stream_ptr(stream), _pf(ms)))
    return ms


def mppi_batch_destroy(b: int) -> None:
    _check(load().mppi_batch_destroy(C.c_void_p(b)))


def mppi_set_shape(h: int, K: int, N: int) -> None:
    _check(load().mppi_set_shape(C.c_void_p(h), K, N))


def mppi_get_nominal(h: int, N: int) -> np.ndarray:
    U = np.zeros((N, 5), np.float32)
    _check(load().mppi_get_nominal(C.c_void_p(h), _pf(U)))
    return U


def mppi_get_unew(h: int, N: int) -> np.ndarray:
    U = np.zeros((N, 5), np.float32)
    _check(load().mppi_get_unew(C.c_void_p(h), _pf(U)))
    return U


def mppi_get_costs(h: int, K: int) -> np.ndarray:
    J = np.zeros(K, np.float64)
    _check(load().mppi_get_costs(C.c_void_p(h), J.ctypes.data_as(C.POINTER(C.c_double))))
    return J


def mppi_get_sample_info(h: int, K: int):
    npass = np.zeros(K, np.int32)
    first = np.zeros(K, np.int32)
    _check(load().mppi_get_sample_info(C.c_void_p(h), npass.ctypes.data_as(C.POINTER(I32)),
                                       first.ctypes.data_as(C.POINTER(I32))))
    return npass, first


def mppi_get_noise(h: int, N: int, K: int) -> np.ndarray:
    Z = np.zeros((N, K, 5), np.float32)
    _check(load().mppi_get_noise(C.c_void_p(h), _pf(Z)))
    return Z


def mppi_get_passcnt(h: int, N: int) -> np.ndarray:
    p = np.zeros(N + 1, np.int32)
    _check(load().mppi_get_passcnt(C.c_void_p(h), p.ctypes.data_as(C.POINTER(I32))))
    return p


def mppi_get_info(h: int) -> np.ndarray:
    a = np.zeros(4, np.int32)
    _check(load().mppi_get_info(C.c_void_p(h), a.ctypes.data_as(C.POINTER(I32))))
    return a


def mppi_get_solve_scalars(h: int) -> np.ndarray:
    a = np.zeros(4, np.float64)
    _check(load().mppi_get_solve_scalars(C.c_void_p(h), a.ctypes.data_as(C.POINTER(C.c_double))))
    return a


def mppi_get_xref(h: int, N: int) -> np.ndarray:
    a = np.zeros((N + 1, 13), np.float32)
    _check(load().mppi_get_xref(C.c_void_p(h), _pf(a)))
    return a


def mppi_export_state(h: int) -> bytes:
    n = C.c_size_t(0)
    _check(load().mppi_export_state(C.c_void_p(h), None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(load().mppi_export_state(C.c_void_p(h), C.cast(buf, C.c_void_p), C.byref(n)))
    return buf.raw


def mppi_import_state(h: int, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().mppi_import_state(C.c_void_p(h), C.cast(buf, C.c_void_p), len(blob)))


def mppi_set_gate_index(h: int, gate: int) -> None:
    _check(load().mppi_set_gate_index(C.c_void_p(h), int(gate)))


def mppi_rollout_states_rotor(model: Model, dt: float, N: int, B: int, d_x0: int, d_T0: int, d_U: int, d_X: int,
                              d_T: int, stream=None):
    _check(load().mppi_rollout_states_rotor(C.byref(model), float(dt), N, B, C.c_void_p(d_x0), C.c_void_p(d_T0),
                                            C.c_void_p(d_U), C.c_void_p(d_X), C.c_void_p(d_T), _stream_ptr(stream)))


def mppi_set_rotor_thrusts(h: int, T) -> None:
    a = (C.c_float * 4)(*[float(v) for v in T])
    _check(load().mppi_set_rotor_thrusts(C.c_void_p(h), a))


def mppi_get_rotor_thrusts(h: int) -> np.ndarray:
    a = (C.c_float * 4)()
    _check(load().mppi_get_rotor_thrusts(C.c_void_p(h), a))
    return np.array(list(a), np.float32)


def mppi_set_noise(h: int, d_Z: int, d_Z5: Optional[int], stream=None) -> None:
    _check(load().mppi_set_noise(C.c_void_p(h), C.c_void_p(d_Z), C.c_void_p(d_Z5 or 0), _stream_ptr(stream)))


def mppi_philox(k0, k1, c0, c1, c2, c3, n: int, d_out: int, stream=None) -> None:
    _check(load().mppi_philox(k0, k1, c0, c1, c2, c3, n, C.c_void_p(d_out), _stream_ptr(stream)))


def mppi_normals(seed, drone, k, it, blk, n: int, d_out: int, stream=None) -> None:
    _check(load().mppi_normals(seed, drone, k, it, blk, n, C.c_void_p(d_out), _stream_ptr(stream)))


def mppi_rollout_states(model: Model, dt: float, N: int, B: int, d_x0: int, d_U: int, d_X: int, stream=None):
    _check(load().mppi_rollout_states(C.byref(model), float(dt), N, B, C.c_void_p(d_x0), C.c_void_p(d_U),
                                      C.c_void_p(d_X), _stream_ptr(stream)))


def mppi_solve_noalloc(model: Model, params: Params, d_track: TrackC, d_x0: int, t0: float, d_U: int, it: int,
                       gate: int, stream, d_Unew: int, d_u0: int) -> None:
    """Stateless solve whose scratch is the library's static device array
    (no device allocation); d_track holds device pointers."""
    _check(load().mppi_solve_noalloc(C.byref(model), C.byref(params), C.byref(d_track), C.c_void_p(d_x0), float(t0),
                                     C.c_void_p(d_U), int(it) & 0xFFFFFFFF, int(gate), _stream_ptr(stream),
                                     C.c_void_p(d_Unew), C.c_void_p(d_u0)))


def mppi_device_bytes(h: int) -> int:
    n = C.c_size_t(0)
    _check(load().mppi_device_bytes(C.c_void_p(h), C.byref(n)))
    return n.value


def mppi_estimate_bytes(params: Params, track: TrackArrays) -> int:
    n = C.c_size_t(0)
    _check(load().mppi_estimate_bytes(C.byref(params), C.byref(track.c), C.byref(n)))
    return n.value


def mppi_kernel_launches() -> int:
    return int(load().mppi_kernel_launches())


def mppi_version() -> str:
    return load().mppi_version().decode()


# ---------------------------------------------------------------------------
# convenience wrapper: one controller handle
# ---------------------------------------------------------------------------

class Controller:
    """Owns one libmppi handle for one drone."""

    def __init__(self, mc: W.ModelConfig, sc: W.SolveConfig, track: W.Track, noise_dtype: int = NOISE_F32,
                 accum: int = ACC_KAHAN32, block: int = 128, N_cap: int = 0, K_cap: int = 0,
                 noise_gen: Optional[int] = None, spt: int = 1):
        self.mc, self.sc, self.track = mc, sc, track
        self.model = make_model(mc)
        self.params = make_params(sc, noise_dtype, accum, block, N_cap, K_cap, noise_gen, spt)
        self.tables = TrackArrays(track)
        self.h = mppi_create(self.model, self.params, self.tables)
        self.K, self.N = sc.K, sc.N

    def close(self):
        if self.h:
            mppi_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, x0, t0: float = 0.0, stream=None):
        return mppi_solve(self.h, x0, t0, stream)

    def set_shape(self, K: int, N: int):
        mppi_set_shape(self.h, K, N)
        self.K, self.N = K, N

    def set_copy_wait(self, limit_ns: int, unreachable: bool = False) -> None:
        """Bound of the rollout's wait for its bulk copies; unreachable makes
        that wait target a barrier nothing completes (testing the timeout)."""
        _check(load().mppi_set_copy_wait(C.c_void_p(self.h), int(limit_ns), int(bool(unreachable))))

    def rotor_thrusts(self) -> np.ndarray:
        """Rotor model: the rotor thrusts the next solve starts from."""
        return mppi_get_rotor_thrusts(self.h)

    def set_rotor_thrusts(self, T) -> None:
        mppi_set_rotor_thrusts(self.h, T)

    def nominal(self):
        return mppi_get_nominal(self.h, self.N)

    def unew(self):
        return mppi_get_unew(self.h, self.N)

    def costs(self):
        return mppi_get_costs(self.h, self.K)

    def sample_info(self):
        return mppi_get_sample_info(self.h, self.K)

    def noise(self):
        return mppi_get_noise(self.h, self.N, self.K)

    def passcnt(self):
        return mppi_get_passcnt(self.h, self.N)

    def info(self):
        return mppi_get_info(self.h)

    def scalars(self):
        return mppi_get_solve_scalars(self.h)

    def xref(self):
        return mppi_get_xref(self.h, self.N)

    def export_state(self) -> bytes:
        return mppi_export_state(self.h)

    def import_state(self, blob: bytes):
        mppi_import_state(self.h, blob)


# DevState: 10 int32, theta, v_theta, c_last + prev_x0[13], scal[4], rotor[4], rotor_prev[4], has_rotor,
# timeouts_seen
_DEVSTATE_FMT = "<10i2d14f4d8f2i"


def decode_state(blob: bytes, N_cap: int) -> dict:
    """Reads the fields of an exported state blob (layout of mppi_export_state)."""
    import struct
    magic, version, ncap, nu = struct.unpack_from("<4I", blob, 0)
    vals = struct.unpack_from(_DEVSTATE_FMT, blob, 16)
    i32 = vals[:10]
    d = {"gate": i32[0], "iter": i32[1] & 0xFFFFFFFF, "has_prev": i32[2], "has_theta": i32[3], "n_nom": i32[4],
         "n_prev": i32[5], "gate0": i32[6], "adv": i32[7], "status": i32[8], "timeouts": i32[9],
         "theta": vals[10], "v_theta": vals[11], "c_last": vals[12], "prev_x0": np.array(vals[13:26]),
         "scal": np.array(vals[26:30]), "rotor": np.array(vals[30:34]), "rotor_prev": np.array(vals[34:38]),
         "has_rotor": vals[38], "nu": nu}
    off = 16 + struct.calcsize(_DEVSTATE_FMT)
    d["U"] = np.frombuffer(blob, np.float32, count=N_cap * 5, offset=off).reshape(N_cap, 5).astype(np.float64)
    off += 4 * N_cap * 5
    d["prevcnt"] = np.frombuffer(blob, np.int32, count=N_cap, offset=off).copy()
    return d


def encode_state(N_cap: int, nu: int, U, iter: int = 0, gate: int = 0, prevcnt=None, prev_x0=None,
                 theta: float = 0.0, v_theta: float = 0.0, c_last: float = 0.0, has_theta: int = 0,
                 n_nom: Optional[int] = None, rotor=None) -> bytes:
    """Builds a state blob for mppi_import_state.  U rows beyond its length
    repeat its last row; pass counts beyond theirs repeat the last count."""
    import struct
    U = np.asarray(U, np.float64).reshape(-1, 5)
    Uf = np.zeros((N_cap, 5), np.float32)
    Uf[:U.shape[0]] = U[:N_cap]
    if U.shape[0] < N_cap:
        Uf[U.shape[0]:] = U[-1]
    pc = np.zeros(N_cap, np.int32)
    n_prev = 0
    if prevcnt is not None and len(prevcnt):
        p = np.asarray(prevcnt, np.int32)
        n_prev = len(p)
        pc[:min(n_prev, N_cap)] = p[:N_cap]
        if n_prev < N_cap:
            pc[n_prev:] = p[-1]
    has_prev = 1 if prev_x0 is not None else 0
    x0 = np.zeros(13) if prev_x0 is None else np.asarray(prev_x0, np.float64)
    dev = struct.pack(_DEVSTATE_FMT, int(gate), int(iter) & 0x7FFFFFFF if iter < 2 ** 31 else int(iter) - 2 ** 32,
                      has_prev, int(has_theta), int(U.shape[0] if n_nom is None else n_nom), n_prev, int(gate), 0, 0, 0,
                      float(theta), float(v_theta), float(c_last), *[float(v) for v in x0], 0.0, 0.0, 0.0, 0.0,
                      *[float(v) for v in (rotor if rotor is not None else np.zeros(4))], 0.0, 0.0, 0.0, 0.0,
                      1 if rotor is not None else 0, 0)
    return struct.pack("<4I", 0x4D505049, 1, N_cap, nu) + dev + Uf.tobytes() + pc.tobytes()


# ---------------------------------------------------------------------------
# serving (continuous batching): thin wrappers of mppi_server_*
# ---------------------------------------------------------------------------

RESULT_DTYPE = np.dtype([("request", np.int64), ("drone", np.int32), ("status", np.int32), ("K", np.int32),
                         ("N", np.int32), ("u0", np.float32, 5), ("t_submit", np.float64), ("t_launch", np.float64),
                         ("t_done", np.float64)], align=True)


def mppi_clock() -> float:
    return float(load().mppi_clock())


class Server:
    """One mppi_server: resident state of many drones plus a scratch pool."""

    def __init__(self, max_drones: int, budget_bytes: int, n_slots: int = 3, max_batch: int = 512):
        h = C.c_void_p()
        _check(load().mppi_server_create(int(max_drones), C.c_size_t(int(budget_bytes)), int(n_slots),
                                         int(max_batch), C.byref(h)))
        self.h = h.value
        self._keep = []

    def add_drone(self, mc, sc, track, K_cap: int, N_cap: int, block: int = 128, noise_gen: Optional[int] = None,
                  spt: int = 1) -> int:
        tables = TrackArrays(track)
        self._keep.append(tables)
        d = I32()
        _check(load().mppi_server_add_drone(C.c_void_p(self.h), C.byref(make_model(mc)),
                                            C.byref(make_params(sc, block=block, N_cap=N_cap, K_cap=K_cap,
                                                                noise_gen=noise_gen, spt=spt)),
                                            C.byref(tables.c), C.byref(d)))
        return int(d.value)

    def submit(self, drones, x0s, t0s, Ks, Ns, deadlines=None) -> np.ndarray:
        """Queues requests; deadlines (mppi_clock() times, optional): a
        request still queued then is dropped (status MPPI_ERR_NOT_ADMITTED)."""
        n = len(drones)
        dr = np.ascontiguousarray(drones, np.int32)
        x = _f32(np.asarray(x0s).reshape(n, 13))
        t = np.ascontiguousarray(t0s, np.float64)
        k = np.ascontiguousarray(Ks, np.int32)
        nn = np.ascontiguousarray(Ns, np.int32)
        ids = np.zeros(n, np.int64)
        if deadlines is None:
            _check(load().mppi_server_submit(C.c_void_p(self.h), n, dr.ctypes.data, x.ctypes.data, t.ctypes.data,
                                             k.ctypes.data, nn.ctypes.data, ids.ctypes.data))
        else:
            dl = np.ascontiguousarray(deadlines, np.float64)
            _check(load().mppi_server_submit_deadline(C.c_void_p(self.h), n, dr.ctypes.data, x.ctypes.data,
                                                      t.ctypes.data, k.ctypes.data, nn.ctypes.data, dl.ctypes.data,
                                                      ids.ctypes.data))
        return ids

    def step(self) -> int:
        n = I32()
        _check(load().mppi_server_step(C.c_void_p(self.h), C.byref(n)))
        return int(n.value)

    def poll(self, cap: int = 8192) -> np.ndarray:
        out = np.zeros(cap, RESULT_DTYPE)
        n = I32()
        _check(load().mppi_server_poll(C.c_void_p(self.h), out.ctypes.data, int(cap), C.byref(n)))
        return out[: n.value]

    def fail_next_launch(self) -> None:
        """Testing hook: the next step that admits a batch fails on the host."""
        _check(load().mppi_server_fail_next_launch(C.c_void_p(self.h)))

    def stats(self) -> dict:
        a = (C.c_double * 8)()
        _check(load().mppi_server_stats(C.c_void_p(self.h), a))
        keys = ("queued", "in_flight", "scratch_used", "scratch_peak", "batches", "finished", "drones", "pool")
        return dict(zip(keys, list(a)))

    def export_drone(self, d: int) -> bytes:
        n = C.c_size_t(0)
        _check(load().mppi_server_export_drone(C.c_void_p(self.h), int(d), None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().mppi_server_export_drone(C.c_void_p(self.h), int(d), C.cast(buf, C.c_void_p), C.byref(n)))
        return buf.raw

    def close(self):
        if self.h:
            _check(load().mppi_server_destroy(C.c_void_p(self.h)))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
