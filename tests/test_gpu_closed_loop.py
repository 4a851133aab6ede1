"""Closed-loop sanity of the CUDA controller (not parity: FP32 and FP64 closed
loops drift apart chaotically).  The plant is the oracle's FP64 RK4 model,
applying u0 for one control period.

C1: 4-gate circle, K=256, N=20, dt=0.05, 100 steps from hover 1 m before
    the first gate: every gate is passed.
C2: seeded 7-gate course, K=4096, N=50, dt=0.02, 20 s at 50 Hz, each
    objective: gate progress keeps passing gates (the reading of the gate
    objective can stall at some yawed, stacked gates of random courses; the
    FP64 closed loop passes 8 gates on this course), contouring advances
    along the path, tracking stays near its 8 m/s reference.
"""
import math

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    from oracle import oracle as O
    from paper_2509_14726_gb300 import mppi as M
    return O, M


def _fly(O, M, mc, sc, tr, x0, steps, t0=0.0):
    ctl = M.Controller(mc, sc, tr)
    x, t = x0.copy(), t0
    X = [x.copy()]
    for _ in range(steps):
        u0, _ = ctl.solve(x, t)
        x = O.rk4_step(mc, x, np.asarray(u0[:4], np.float64), sc.dt)
        t += sc.dt
        X.append(x.copy())
    info = ctl.info()
    ctl.close()
    return np.array(X), int(info[3])


def test_c1_passes_every_gate(env):
    O, M = env
    mc, sc, tr, x0 = W.c1_single_gate()
    X, gates = _fly(O, M, mc, sc, tr, x0, 100)
    assert gates >= 4, f"passed {gates} gates in 100 steps"
    assert np.all(X[:, 2] > 0.0)


def test_c2_gate_progress_laps(env):
    O, M = env
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_GATE)
    X, gates = _fly(O, M, mc, sc, tr, x0, 1000)
    assert gates >= 3, f"passed {gates} of {tr.n_gates} gates in 20 s"


def test_c2_contouring_advances(env):
    O, M = env
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_CONTOUR)
    X, _ = _fly(O, M, mc, sc, tr, x0, 1000)
    S = tr.path.shape[0]
    th = [O.path_project(tr, x, 0, S - 1) for x in X[::10]]
    prog = np.mod(np.diff(th) + tr.L / 2, tr.L) - tr.L / 2
    dist = [np.linalg.norm(O.path_eval(tr, a)[0] - x[:3]) for a, x in zip(th, X[::10])]
    assert prog.sum() > 0.5 * tr.L, f"progress {prog.sum():.1f} m of a {tr.L:.1f} m lap"
    assert np.mean(dist) < 1.0


def test_c2_tracking_follows_reference(env):
    O, M = env
    mc, sc, tr, _ = W.c2_full_scale(W.OBJ_TRACK)
    x0 = O.ref_eval(tr, 0.0)
    X, _ = _fly(O, M, mc, sc, tr, x0, 1000)
    err = [np.linalg.norm(X[k, :3] - O.ref_eval(tr, k * sc.dt)[:3]) for k in range(0, 1001, 5)]
    rmse = math.sqrt(np.mean(np.square(err)))
    assert rmse < 1.0, f"tracking RMSE {rmse:.3f} m"


def test_lap_protocol_on_the_circle(env):
    """The comparison protocol (Sec. V-A): one lap of the 4-gate circle with
    each objective, the library's model as the plant.  Every objective
    completes the lap through the gates, gate progress is the fastest and
    tracking stays on its reference."""
    from paper_2509_14726_gb300 import closed_loop as CL
    out = CL.comparison({"circle": W.circle_track(4, 5.0)}, laps=1, K=2048, N=40, t_max=20.0)
    g, c, t = (out[f"circle/ctbr/{n}"] for n in ("gate", "contour", "track"))
    assert g["completed"] and c["completed"] and t["completed"], out
    assert g["time_s"] < t["time_s"]
    assert t["tracking_rmse_m"] < 0.2
    assert all(r["waypoint_error_m"] <= 0.75 * 2 ** 0.5 for r in (g, c, t))
