"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than the oracle
itself: a closed-form solution, an invariant, a brute-force search, or an
independent implementation (cuRAND's host Philox4x32-10 generator).  The
tests are chosen so that a plausible slip (a dropped term, a flipped sign, a
transposed operand, an off-by-one step index) breaks at least one of them.
"""
import ctypes
import math
import os

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W

HOVER_M = W.ModelConfig()


def _mc(**kw):
    m = W.ModelConfig()
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _axis_quat(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * a])


def _state(p=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0), w=(0, 0, 0)):
    return np.concatenate([p, v, q, w]).astype(float)


# ---------------------------------------------------------------------------
# Philox4x32-10 and Box-Muller (Eq. 3 sampling)
# ---------------------------------------------------------------------------

def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10",
              "/usr/local/cuda/targets/sbsa-linux/lib/libcurand.so", "libcurand.so"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x1234_5678, 0xDEAD_BEEF_0BAD_F00D])
def test_philox_matches_curand_host_generator(oracle_mod, seed):
    """cuRAND's host PHILOX4_32_10 generator is an independent implementation.
    Seeded with s, its output block j (words 4j..4j+3) is
    philox(ctr = (a_lo, a_hi, b, 0), key = (s_lo, s_hi)) with j = 65536 a + b
    (65536 interleaved subsequences); generator offsets reach any j."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    key = (seed & 0xFFFFFFFF, seed >> 32)

    def block_at(j, nb):
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * j)) == 0
        out = np.zeros(4 * nb, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
        return out.reshape(nb, 4)

    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        for j0, nb in ((0, 64), (65536 * 3 + 11, 4), (1 << 48, 2), ((5 << 48) + 65536 * 7 + 40000, 2)):
            blocks = block_at(j0, nb)
            for i in range(nb):
                a, b = divmod(j0 + i, 65536)
                ctr = (a & 0xFFFFFFFF, a >> 32, b, 0)
                np.testing.assert_array_equal(oracle_mod.philox(ctr, key), blocks[i])
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox((5, 6, 7, 8), (9, 10))
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] += 1
        assert not np.array_equal(oracle_mod.philox(c, (9, 10)), base)
    assert not np.array_equal(oracle_mod.philox((5, 6, 7, 8), (9, 11)), base)
    assert not np.array_equal(oracle_mod.philox((5, 6, 7, 8), (10, 10)), base)


def test_uniform_map_is_exact_and_in_half_open_unit_interval(oracle_mod):
    assert oracle_mod.uniform(0) == 2.0 ** -24
    assert oracle_mod.uniform(0xFF) == 2.0 ** -24
    assert oracle_mod.uniform(0x100) == 2.0 ** -23
    assert oracle_mod.uniform(0xFFFFFFFF) == 1.0
    xs = np.random.default_rng(0).integers(0, 2 ** 32, 2000, dtype=np.uint64)
    us = np.array([oracle_mod.uniform(int(x)) for x in xs])
    assert np.all((us > 0) & (us <= 1))
    # every value is an integer multiple of 2^-24, so binary32 holds it exactly
    assert np.all(np.float32(us).astype(np.float64) == us)


def test_box_muller_special_angles(oracle_mod):
    # u_a = 1 gives radius 0
    np.testing.assert_allclose(oracle_mod.box_muller(0xFFFFFFFF, 12345), [0.0, 0.0], atol=0)
    # u_a = 2^-24 * (2^24 * e^-0.5 rounded) gives radius ~ 1; pick u_a exactly
    xa = (int(round(math.exp(-0.5) * 2 ** 24)) - 1) << 8
    ua = ((xa >> 8) + 1) / 2 ** 24
    r = math.sqrt(-2 * math.log(ua))
    # u_b = 1/4 -> angle pi/2 ; u_b = 1/2 -> angle pi ; u_b = 1 -> angle 2 pi
    for ub_num, (c, s) in [(2 ** 22, (0.0, 1.0)), (2 ** 23, (-1.0, 0.0)), (2 ** 24, (1.0, 0.0))]:
        xb = (ub_num - 1) << 8
        z = oracle_mod.box_muller(xa, xb)
        np.testing.assert_allclose(z, [r * c, r * s], atol=1e-12)


def test_normals_are_standard_normal(oracle_mod):
    from math import erf
    zs = np.array([oracle_mod.normals4(0, 3, m, k, 2, 0) for m in range(1500) for k in range(8)]).ravel()
    assert abs(zs.mean()) < 0.015
    assert abs(zs.var() - 1.0) < 0.03
    # Kolmogorov-Smirnov distance to the normal CDF
    s = np.sort(zs)
    cdf = 0.5 * (1 + np.vectorize(erf)(s / math.sqrt(2)))
    n = len(s)
    d = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(0, n) / n))
    assert d < 1.63 / math.sqrt(n)  # 1% level
    # the four outputs of one draw are uncorrelated
    z4 = zs.reshape(-1, 4)
    c = np.corrcoef(z4.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.05


# ---------------------------------------------------------------------------
# Quadrotor model (Eq. 2) and RK4
# ---------------------------------------------------------------------------

def test_hover_is_an_equilibrium(oracle_mod):
    mc = _mc()
    for yaw in (0.0, 1.1, -2.7):
        x = _state(p=(3, -4, 2), q=W.yaw_quat(yaw))
        y = x.copy()
        for _ in range(200):
            y = oracle_mod.rk4_step(mc, y, [mc.hover, 0, 0, 0], 0.02)
        np.testing.assert_allclose(y, x, atol=1e-12)


def test_free_fall_is_exact(oracle_mod):
    """c = 0: p(t) = p0 + v0 t - g t^2 / 2 e_z; RK4 integrates quadratics exactly."""
    mc = _mc()
    p0, v0 = np.array([1.0, 2.0, 30.0]), np.array([0.5, -1.0, 3.0])
    x = _state(p=p0, v=v0, q=_axis_quat([1, 2, 3], 0.7))
    h, n = 0.013, 150
    for _ in range(n):
        x = oracle_mod.rk4_step(mc, x, [0, 0, 0, 0], h)
    t = h * n
    np.testing.assert_allclose(x[:3], p0 + v0 * t + 0.5 * t * t * np.array([0, 0, -mc.gravity]), atol=1e-10)
    np.testing.assert_allclose(x[3:6], v0 + t * np.array([0, 0, -mc.gravity]), atol=1e-11)


@pytest.mark.parametrize("axis,ang", [([1, 0, 0], 0.4), ([0, 1, 0], -0.6), ([1, 1, 0], 0.3)])
def test_constant_thrust_along_body_z(oracle_mod, axis, ang):
    """Fixed attitude, no rates: acceleration is (c/m) R(q) e_z + g, a constant,
    so the motion is an exact parabola.  R(q) about x by +a maps e_z to
    (0, -sin a, cos a), about y to (sin a, 0, cos a)."""
    mc = _mc()
    q = _axis_quat(axis, ang)
    c = 12.0
    x = _state(p=(0, 0, 5), q=q)
    h, n = 0.02, 60
    for _ in range(n):
        x = oracle_mod.rk4_step(mc, x, [c, 0, 0, 0], h)
    a_ = np.asarray(axis, float) / np.linalg.norm(axis)
    # Rodrigues: R e_z
    ez = np.array([0, 0, 1.0])
    Rez = ez * math.cos(ang) + np.cross(a_, ez) * math.sin(ang) + a_ * np.dot(a_, ez) * (1 - math.cos(ang))
    acc = c / mc.mass * Rez + np.array([0, 0, -mc.gravity])
    t = h * n
    np.testing.assert_allclose(x[:3], np.array([0, 0, 5.0]) + 0.5 * acc * t * t, atol=1e-10)
    np.testing.assert_allclose(x[6:10], q, atol=1e-14)
    if axis == [1, 0, 0]:
        assert Rez[1] < 0  # a positive roll tilts thrust toward -y


def test_body_rate_integrates_in_body_frame(oracle_mod):
    """With rates held (w_cmd = w, gyroscopic term zero for rotation about a
    principal axis), q(t) = q0 * exp(w t / 2) -- a body-frame rotation."""
    mc = _mc()
    q0 = _axis_quat([1, 0, 0], 0.5 * math.pi)
    Om = 2.0
    x = _state(q=q0, w=(0, 0, Om))
    h, n = 0.005, 200
    for _ in range(n):
        x = oracle_mod.rk4_step(mc, x, [mc.hover, 0, 0, Om], h)
    t = h * n
    expect = _qmul(q0, np.array([math.cos(Om * t / 2), 0, 0, math.sin(Om * t / 2)]))
    np.testing.assert_allclose(x[6:10], expect, atol=1e-9)
    world_frame = _qmul(np.array([math.cos(Om * t / 2), 0, 0, math.sin(Om * t / 2)]), q0)
    assert np.max(np.abs(world_frame - expect)) > 0.1  # the test tells the frames apart


def test_rate_loop_is_first_order_with_exact_rk4_factor(oracle_mod):
    """About one principal axis dw = k (w_cmd - w); RK4 multiplies the error
    by P(-k h) = 1 - kh + (kh)^2/2 - (kh)^3/6 + (kh)^4/24 per step."""
    mc = _mc()
    h, cmd, w0 = 0.01, 3.0, -1.0
    for axis in range(3):
        w = [0.0, 0.0, 0.0]
        w[axis] = w0
        x = _state(w=w)
        u = [mc.hover, 0, 0, 0]
        u[1 + axis] = cmd
        n = 40
        for _ in range(n):
            x = oracle_mod.rk4_step(mc, x, u, h, renormalise=False)
        z = -mc.k_omega * h
        P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        assert abs(x[10 + axis] - (cmd + (w0 - cmd) * P ** n)) < 1e-12


def test_gyroscopic_precession_of_a_symmetric_body(oracle_mod):
    """k_omega = 0, J = diag(a, a, b): w_z is constant and (w_x, w_y) turns at
    Omega = (b - a)/a * w_z (Euler's equations)."""
    mc = _mc(k_omega=0.0)
    a, b = mc.inertia[0], mc.inertia[2]
    wz = 6.0
    x = _state(w=(1.0, 0.0, wz))
    h, n = 0.001, 500
    for _ in range(n):
        x = oracle_mod.rk4_step(mc, x, [mc.hover, 0, 0, 0], h)
    Om = (b - a) / a * wz
    t = h * n
    np.testing.assert_allclose(x[10:13], [math.cos(Om * t), math.sin(Om * t), wz], atol=1e-9)


def test_drag_acts_in_the_body_frame(oracle_mod):
    """D = diag(d1, d2, 0) in the body; with yaw 90 deg body x is world y, so a
    world-y velocity decays with d1, exactly by P(-d1 h) per RK4 step."""
    d1, d2 = 0.8, 0.1
    mc = _mc(drag=(d1, d2, 0.0))
    x = _state(v=(0, 2.0, 0), q=W.yaw_quat(0.5 * math.pi))
    h, n = 0.02, 30
    for _ in range(n):
        x = oracle_mod.rk4_step(mc, x, [mc.hover, 0, 0, 0], h)
    z = -d1 * h
    P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert abs(x[4] - 2.0 * P ** n) < 1e-12
    assert abs(x[3]) < 1e-12


def test_rk4_is_fourth_order(oracle_mod):
    mc = _mc()
    x0 = _state(p=(0, 0, 2), v=(1, -2, 0.5), q=_axis_quat([0.3, -0.2, 1], 0.8), w=(2.0, -1.5, 3.0))
    u = [14.0, 4.0, -3.0, 6.0]
    T = 0.4

    def run(h):
        x = x0.copy()
        for _ in range(int(round(T / h))):
            x = oracle_mod.rk4_step(mc, x, u, h, renormalise=False)
        return x

    ref = run(T / 2048)
    e1 = np.max(np.abs(run(T / 16) - ref))
    e2 = np.max(np.abs(run(T / 32) - ref))
    e3 = np.max(np.abs(run(T / 64) - ref))
    assert 12 < e1 / e2 < 20 and 12 < e2 / e3 < 20


def test_quaternion_norm(oracle_mod):
    mc = _mc()
    x = _state(q=_axis_quat([1, 2, 3], 1.0), w=(3, -4, 5))
    xr = x.copy()
    for _ in range(300):
        x = oracle_mod.rk4_step(mc, x, [10, 5, -5, 2], 0.02)
        xr = oracle_mod.rk4_step(mc, xr, [10, 5, -5, 2], 0.002, renormalise=False)
    assert abs(np.linalg.norm(x[6:10]) - 1) < 1e-14
    # without renormalisation the drift per step is O(h^5): tiny at h = 0.002
    assert abs(np.linalg.norm(xr[6:10]) - 1) < 1e-9


def test_penalty_closed_form(oracle_mod):
    mc, sc = _mc(), W.SolveConfig()
    assert oracle_mod.penalty(mc, sc, _state(p=(0, 0, 1), w=(9.9, -10, 0))) == 0.0
    v = oracle_mod.penalty(mc, sc, _state(p=(0, 0, -0.5), w=(11.0, -12.0, 0)))
    assert abs(v - sc.w_limit * (1.0 + 4.0 + 0.25)) < 1e-9


# ---------------------------------------------------------------------------
# gate geometry and the gate-progress objective (Eq. 6, Eq. 7, Sec. IV-A)
# ---------------------------------------------------------------------------

GATE = np.array([2.0, 1.0, 3.0, 0.3, 0.75, 0.75])


def _gate_frame(g):
    n = np.array([math.cos(g[3]), math.sin(g[3]), 0.0])
    l = np.array([-math.sin(g[3]), math.cos(g[3]), 0.0])
    return g[:3], n, l


def test_gate_crossing_geometry(oracle_mod):
    c, n, l = _gate_frame(GATE)
    ok, info = oracle_mod.gate_crossing(GATE, c - 0.3 * n, c + 0.2 * n)
    assert ok and abs(info[0] + 0.3) < 1e-15 and abs(info[1] - 0.2) < 1e-15
    # through the opening near its edge, and just outside it
    assert oracle_mod.gate_crossing(GATE, c - 0.3 * n + 0.74 * l, c + 0.2 * n + 0.74 * l)[0]
    assert not oracle_mod.gate_crossing(GATE, c - 0.3 * n + 0.76 * l, c + 0.2 * n + 0.76 * l)[0]
    assert not oracle_mod.gate_crossing(GATE, c - 0.3 * n + [0, 0, 0.8], c + 0.2 * n + [0, 0, 0.8])[0]
    # backwards and parallel motion are not passes
    assert not oracle_mod.gate_crossing(GATE, c + 0.2 * n, c - 0.3 * n)[0]
    assert not oracle_mod.gate_crossing(GATE, c - 0.3 * n, c - 0.3 * n + l)[0]
    # landing exactly on the plane counts; starting on it does not
    assert oracle_mod.gate_crossing(GATE, c - 0.3 * n, c)[0]
    assert not oracle_mod.gate_crossing(GATE, c, c + 0.3 * n)[0]
    # the interpolated point is used, not either end point
    ok, info = oracle_mod.gate_crossing(GATE, c - 0.5 * n - 1.0 * l, c + 0.5 * n + 1.0 * l)
    assert ok and abs(info[2]) < 1e-12


def _line_track(n_gates=2, spacing=6.0, closed=True):
    gates = np.zeros((n_gates, 6))
    for i in range(n_gates):
        gates[i] = (spacing * (i + 1), 0.0, 2.0, 0.0, 0.75, 0.75)
    path = np.zeros((4, 6))
    path[:, 3] = 1.0
    ref = np.zeros((2, 13))
    ref[:, 6] = 1.0
    return W.Track(gates, closed, path, 100.0, ref, 1.0)


def _straight_flight_J(track, p0, vx, h, N, sc, first_gate, cross_ok):
    P = [np.array(p0) + np.array([vx * h * k, 0, 0]) for k in range(N + 1)]
    g0 = track.gates[first_gate, :3]
    gi = first_gate
    J = 0.0
    for k in range(N):
        g = track.gates[gi % track.n_gates, :3]
        J += np.sum((P[k + 1] - g) ** 2) - np.sum((P[k] - g) ** 2)
        d0 = np.linalg.norm(P[k] - g0)
        if d0 < sc.r_near:
            J += sc.q_near * d0 * d0
        gx = track.gates[gi % track.n_gates, 0]
        if P[k][0] < gx <= P[k + 1][0] and cross_ok(k):
            gi += 1
    return J, gi - first_gate


def test_gate_progress_closed_form_straight_line(oracle_mod):
    """Level hover thrust, zero rates, constant velocity through two gates in a
    row: the cost is Eq. 7 evaluated on the closed-form positions with the
    target switching to the next gate right after each crossing."""
    tr = _line_track(2, spacing=4.0)
    mc = _mc()
    N, h, vx = 40, 0.05, 5.0
    sc = W.SolveConfig(objective=0, K=1, N=N, dt=h, q_near=0.7, r_near=1.5, temporal_rule=1)
    x0 = _state(p=(1.2, 0.1, 2.05), v=(vx, 0, 0))
    U = np.tile([mc.hover, 0, 0, 0, 0], (N, 1))
    J, X, pc = oracle_mod.rollout(mc, sc, tr, x0, U, gate0=0)
    Jc, passed = _straight_flight_J(tr, x0[:3], vx, h, N, sc, 0, lambda k: True)
    assert passed == 2 and pc[-1] == 2
    assert abs(J - Jc) < 1e-9
    # with no gate reached the sum telescopes to ||p_N - g||^2 - ||p_0 - g||^2
    sc5 = W.SolveConfig(objective=0, K=1, N=5, dt=h, q_near=0.0, r_near=1.5)
    J5, X5, _ = oracle_mod.rollout(mc, sc5, tr, x0, U[:5], gate0=0)
    g = tr.gates[0, :3]
    assert abs(J5 - (np.sum((X5[5, :3] - g) ** 2) - np.sum((X5[0, :3] - g) ** 2))) < 1e-12


def test_near_gate_term_uses_p_k_for_k_below_N(oracle_mod):
    """Eq. 7 sums Q_near ||p_k - g0||^2 over k = 0..N-1: the start state counts,
    the final state does not."""
    tr = _line_track(2, spacing=4.0)
    mc = _mc()
    N, h, vx = 6, 0.05, 2.0
    sc = W.SolveConfig(objective=0, K=1, N=N, dt=h, q_near=0.7, r_near=1.5)
    x0 = _state(p=(3.3, 0.0, 2.0), v=(vx, 0, 0))
    U = np.tile([mc.hover, 0, 0, 0, 0], (N, 1))
    J, X, _ = oracle_mod.rollout(mc, sc, tr, x0, U, gate0=0)
    Jc, _ = _straight_flight_J(tr, x0[:3], vx, h, N, sc, 0, lambda k: True)
    assert abs(J - Jc) < 1e-12


def test_temporal_rule_rejects_passes_later_than_the_previous_nominal(oracle_mod):
    """Sec. IV-A: a pass at step k counts only if the previous iteration's
    nominal had not yet passed that gate at the same time (counts aligned to
    this solve's steps)."""
    tr = _line_track(2, spacing=6.0)
    mc = _mc()
    N, h, vx = 30, 0.05, 5.0
    sc = W.SolveConfig(objective=0, K=1, N=N, dt=h, q_near=0.0, temporal_rule=1)
    x0 = _state(p=(1.2, 0.1, 2.05), v=(vx, 0, 0))
    U = np.tile([mc.hover, 0, 0, 0, 0], (N, 1))
    # geometric crossing of gate 0 happens on step k* with x in (k* h vx, (k*+1) h vx]
    kstar = int(math.floor((6.0 - 1.2) / (vx * h) - 1e-12))
    for prev_pass_step in (kstar - 3, kstar, kstar + 1, kstar + 5):
        prev = np.array([1 if k >= prev_pass_step else 0 for k in range(N)], np.int32)
        J, X, pc = oracle_mod.rollout(mc, sc, tr, x0, U, gate0=0, prev=prev)
        accepted = prev_pass_step > kstar
        Jc, passed = _straight_flight_J(tr, x0[:3], vx, h, N, sc, 0,
                                        lambda k: prev[k] <= 0)
        assert (pc[-1] >= 1) == accepted
        assert abs(J - Jc) < 1e-9
    # rule off: always accepted
    sc.temporal_rule = 0
    prev = np.ones(N, np.int32)
    _, _, pc = oracle_mod.rollout(mc, sc, tr, x0, U, gate0=0, prev=prev)
    assert pc[-1] >= 1


def test_open_track_stops_after_last_gate(oracle_mod):
    tr = _line_track(2, spacing=3.0, closed=False)
    mc = _mc()
    N, h, vx = 60, 0.05, 5.0
    sc = W.SolveConfig(objective=0, K=1, N=N, dt=h, q_near=0.0)
    x0 = _state(p=(1.0, 0.0, 2.0), v=(vx, 0, 0))
    U = np.tile([mc.hover, 0, 0, 0, 0], (N, 1))
    _, _, pc = oracle_mod.rollout(mc, sc, tr, x0, U, gate0=0)
    assert pc[-1] == 2


# ---------------------------------------------------------------------------
# tracking (Eq. 8)
# ---------------------------------------------------------------------------

def test_tracking_cost_of_the_reference_itself(oracle_mod):
    """x_ref = rollout of a known U: that U scores sum ||u - u_hover||^2_R and
    a perturbed U scores more."""
    mc = _mc()
    N, h = 12, 0.04
    rng = np.random.default_rng(3)
    U = np.zeros((N, 5))
    U[:, 0] = mc.hover + rng.normal(0, 1.5, N)
    U[:, 1:4] = rng.normal(0, 1.0, (N, 3))
    x0 = _state(p=(1, 2, 3), v=(1, 0, 0), q=W.yaw_quat(0.4))
    sc = W.SolveConfig(objective=2, K=1, N=N, dt=h)
    _, X, _ = oracle_mod.rollout(mc, sc, _line_track(), x0, U)
    ref = np.vstack([X, X[-1:]])  # T = N + 2 rows, dt_ref = h; t0 = 0 hits rows exactly
    tr = W.Track(_line_track().gates, True, _line_track().path, 100.0, ref, h)
    xref = np.array([oracle_mod.ref_eval(tr, k * h) for k in range(N + 1)])
    np.testing.assert_allclose(xref, X, atol=1e-12)
    J, _, _ = oracle_mod.rollout(mc, sc, tr, x0, U, xref=xref)
    du = U[:, :4].copy()
    du[:, 0] -= mc.hover
    expect = float(np.sum(np.asarray(sc.R) * du * du))
    assert abs(J - expect) < 1e-9
    # the quaternion error uses the nearer sign: -q is the same attitude
    xref_neg = xref.copy()
    xref_neg[:, 6:10] *= -1
    J_neg, _, _ = oracle_mod.rollout(mc, sc, tr, x0, U, xref=xref_neg)
    assert abs(J_neg - expect) < 1e-9
    # one state weight at a time: a position offset dp costs Q_p dp^2 per stage
    xref_off = xref.copy()
    xref_off[:, 0] += 0.1
    J_off, _, _ = oracle_mod.rollout(mc, sc, tr, x0, U, xref=xref_off)
    assert abs(J_off - expect - (N * sc.Q[0] + sc.QN[0]) * 0.01) < 1e-9


def test_reference_interpolation(oracle_mod):
    T, dt = 10, 0.1
    ref = np.zeros((T, 13))
    for i in range(T):
        ref[i, 0:3] = (i, 2 * i, -i)
        ref[i, 3:6] = (1, 2, -1)
        ref[i, 6:10] = _axis_quat([0, 0, 1], 0.1 * i)
        ref[i, 10:13] = (0.5 * i, 0, 0)
    tr = W.Track(np.zeros((1, 6)), True, np.zeros((2, 6)), 1.0, ref, dt)
    xr = oracle_mod.ref_eval(tr, 0.35)
    np.testing.assert_allclose(xr[0:3], (3.5, 7.0, -3.5), atol=1e-12)
    np.testing.assert_allclose(xr[10], 1.75, atol=1e-12)
    q = 0.5 * (_axis_quat([0, 0, 1], 0.3) + _axis_quat([0, 0, 1], 0.4))
    np.testing.assert_allclose(xr[6:10], q / np.linalg.norm(q), atol=1e-12)
    # periodic: t + period gives the same row; between the last and the first row it blends them
    np.testing.assert_allclose(oracle_mod.ref_eval(tr, 0.35 + T * dt), xr, atol=1e-12)
    xw = oracle_mod.ref_eval(tr, 0.95)
    np.testing.assert_allclose(xw[0:3], 0.5 * (ref[9, 0:3] + ref[0, 0:3]), atol=1e-12)


# ---------------------------------------------------------------------------
# contouring (Eq. 9)
# ---------------------------------------------------------------------------

def _square_path(side=40.0, S=400):
    L = 4 * side
    pts = np.zeros((S, 6))
    corners = [np.array([0, 0, 2.0]), np.array([side, 0, 2.0]), np.array([side, side, 2.0]), np.array([0, side, 2.0])]
    for j in range(S):
        s = j * L / S
        e = int(s // side)
        f = s - e * side
        a, b = corners[e], corners[(e + 1) % 4]
        t = (b - a) / side
        pts[j, :3] = a + f * t
        pts[j, 3:] = t
    return pts, L


def test_contouring_on_the_path_scores_only_progress(oracle_mod):
    path, L = _square_path()
    ref = np.zeros((2, 13))
    ref[:, 6] = 1
    tr = W.Track(np.zeros((1, 6)), True, path, L, ref, 1.0)
    mc = _mc()
    N, h, v = 20, 0.05, 6.0
    sc = W.SolveConfig(objective=1, K=1, N=N, dt=h)
    x0 = _state(p=(5.0, 0.0, 2.0), v=(v, 0, 0))
    U = np.tile([mc.hover, 0, 0, 0, 0.0], (N, 1))
    J, _, _ = oracle_mod.rollout(mc, sc, tr, x0, U, theta0=5.0, vth0=v, c_last=mc.hover)
    assert abs(J - (-sc.mu * v * N)) < 1e-9
    # a lateral offset d is pure contouring error, a lag of theta is pure lag error
    d = 0.3
    x1 = x0.copy()
    x1[1] = d
    J1, _, _ = oracle_mod.rollout(mc, sc, tr, x1, U, theta0=5.0, vth0=v, c_last=mc.hover)
    assert abs(J1 - (-sc.mu * v * N + N * sc.q_cont * d * d)) < 1e-9
    J2, _, _ = oracle_mod.rollout(mc, sc, tr, x0, U, theta0=5.0 - d, vth0=v, c_last=mc.hover)
    assert abs(J2 - (-sc.mu * v * N + N * sc.q_lag * d * d)) < 1e-9
    # progress acceleration: v' = clamp(v + a dt), theta by the trapezoid;
    # input terms r a^2 and thrust change against the last applied thrust
    Ua = U.copy()
    Ua[:, 4] = 2.0
    Ua[0, 0] = mc.hover + 1.0
    Ja, _, _ = oracle_mod.rollout(mc, sc, tr, x0, Ua, theta0=5.0, vth0=v, c_last=mc.hover)
    assert Ja > J  # lag builds up and the input terms are positive


def test_path_eval_and_projection(oracle_mod):
    path, L = _square_path()
    tr = W.Track(np.zeros((1, 6)), True, path, L, np.zeros((2, 13)), 1.0)
    P, T = oracle_mod.path_eval(tr, 10.25)
    np.testing.assert_allclose(P, [10.25, 0, 2], atol=1e-12)
    np.testing.assert_allclose(T, [1, 0, 0], atol=1e-12)
    P, T = oracle_mod.path_eval(tr, 10.25 + 3 * L)
    np.testing.assert_allclose(P, [10.25, 0, 2], atol=1e-12)
    # at a corner the tangent blends and is renormalised
    P, T = oracle_mod.path_eval(tr, 40.0 - 0.2)
    assert abs(np.linalg.norm(T) - 1) < 1e-14
    # projection equals a brute-force search over a fine sampling of the path
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = np.array([rng.uniform(-5, 45), rng.uniform(-5, 45), rng.uniform(0, 4)])
        th = oracle_mod.path_project(tr, p, 0, 399)
        grid = np.linspace(0, L, 16001)[:-1]
        d = [np.sum((oracle_mod.path_eval(tr, s)[0] - p) ** 2) for s in grid[::10]]
        best = grid[::10][int(np.argmin(d))]
        Pp, _ = oracle_mod.path_eval(tr, th)
        Pb, _ = oracle_mod.path_eval(tr, best)
        assert np.sum((Pp - p) ** 2) <= np.sum((Pb - p) ** 2) + 1e-9


# ---------------------------------------------------------------------------
# weights and update (Eq. 4, Eq. 5) and the warm start
# ---------------------------------------------------------------------------

def _small_case(obj=0, K=48, N=8, lam=1.0, seed=0):
    mc, sc, tr, x0 = W.c1_single_gate()
    sc.objective, sc.K, sc.N, sc.lam, sc.seed = obj, K, N, lam, seed
    return mc, sc, tr, x0


def test_weights_sum_to_one_and_update_is_the_weighted_mean(oracle_mod):
    mc, sc, tr, x0 = _small_case()
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r = ctl.solve(x0, 0.0, want_Z=True)
    assert abs(r["w"].sum() - 1) < 1e-14
    Jmin = r["J"].min()
    w = np.exp(-(r["J"] - Jmin) / sc.lam)
    np.testing.assert_allclose(r["w"], w / w.sum(), rtol=1e-13)
    # rebuild the clamped samples from the reported normals and average them
    hover = mc.hover
    U0 = np.zeros((sc.N, 5))
    U0[:, 0] = hover
    us = np.clip(U0[None] + np.asarray(sc.sigma) * r["Z"].transpose(1, 0, 2), mc.u_min, mc.u_max)
    us[:, :, 4] = 0
    np.testing.assert_allclose(r["Unew"], np.einsum("m,mkj->kj", r["w"], us), atol=1e-12)
    # each sample's cost equals a plain rollout of its clamped sequence
    for m in (0, 7, 31):
        J, _, _ = oracle_mod.rollout(mc, sc, tr, x0, us[m], gate0=0)
        assert abs(J - r["J"][m]) < 1e-9
    # warm start: shifted by one, last row repeated
    np.testing.assert_array_equal(ctl.nominal[:-1], r["Unew"][1:])
    np.testing.assert_array_equal(ctl.nominal[-1], r["Unew"][-1])
    assert ctl.iter == 1


def test_clamped_samples_are_rolled_out_and_averaged(oracle_mod):
    """Samples leave the input box often when the box is tight: both the
    rollout and the average (Eq. 5) use the clamped values."""
    mc, sc, tr, x0 = _small_case(K=40, N=6)
    mc.u_min = (5.0, -0.4, -0.4, -0.4, -20.0)
    mc.u_max = (10.0, 0.4, 0.4, 0.4, 20.0)
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r = ctl.solve(x0, 0.0, want_Z=True)
    U0 = np.zeros((sc.N, 5))
    U0[:, 0] = mc.hover
    raw = U0[None] + np.asarray(sc.sigma) * r["Z"].transpose(1, 0, 2)
    us = np.clip(raw, mc.u_min, mc.u_max)
    us[:, :, 4] = 0
    assert np.mean(raw[:, :, 1:4] != us[:, :, 1:4]) > 0.3
    np.testing.assert_allclose(r["Unew"], np.einsum("m,mkj->kj", r["w"], us), atol=1e-12)
    for m in (0, 9, 39):
        J, _, _ = oracle_mod.rollout(mc, sc, tr, x0, us[m], gate0=0)
        assert abs(J - r["J"][m]) < 1e-9


def test_lambda_to_zero_selects_the_argmin_sample(oracle_mod):
    mc, sc, tr, x0 = _small_case(lam=1e-9)
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r = ctl.solve(x0, 0.0, want_Z=True)
    m = int(np.argmin(r["J"]))
    U0 = np.zeros((sc.N, 5))
    U0[:, 0] = mc.hover
    us = np.clip(U0 + np.asarray(sc.sigma) * r["Z"][:, m, :], mc.u_min, mc.u_max)
    np.testing.assert_allclose(r["Unew"][:, :4], us[:, :4], atol=1e-12)


def test_lambda_to_infinity_gives_the_sample_mean(oracle_mod):
    mc, sc, tr, x0 = _small_case(lam=1e12)
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r = ctl.solve(x0, 0.0, want_Z=True)
    U0 = np.zeros((sc.N, 5))
    U0[:, 0] = mc.hover
    us = np.clip(U0[None] + np.asarray(sc.sigma) * r["Z"].transpose(1, 0, 2), mc.u_min, mc.u_max)
    np.testing.assert_allclose(r["Unew"][:, :4], us[:, :, :4].mean(0), atol=1e-9)


def _hover_reference(p=(1.0, 2.0, 3.0), h=0.04):
    """A tracking reference that hovers at p (two equal rows)."""
    x = _state(p=p)
    base = _line_track()
    return W.Track(base.gates, True, base.path, 100.0, np.vstack([x, x]), h), x


def test_nominal_sample_is_the_unperturbed_nominal(oracle_mod):
    """nominal_sample = 1 makes candidate 0 the nominal itself (no
    perturbation, Eq. 3 with du = 0).  Hovering on a hover reference, the
    hover nominal costs 0 (Eq. 8: no state error, u = u_hover) and every
    perturbed candidate costs more, so as lambda -> 0 the update (Eq. 4, 5)
    returns the hover sequence exactly; without the nominal candidate it
    returns a perturbed sample."""
    mc = _mc()
    tr, x0 = _hover_reference()
    sc = W.SolveConfig(objective=2, K=64, N=8, dt=0.04, lam=1e-9, nominal_sample=1)
    r = oracle_mod.OracleController(mc, sc, tr).solve(x0, 0.0, want_Z=True)
    assert np.all(r["Z"][:, 0, :] == 0)
    assert r["J"][0] < 1e-20 and np.all(r["J"][1:] > 1e-6)
    np.testing.assert_array_equal(r["Unew"][:, 0], np.full(sc.N, mc.hover))
    np.testing.assert_array_equal(r["Unew"][:, 1:4], 0.0)
    sc.nominal_sample = 0
    r0 = oracle_mod.OracleController(mc, sc, tr).solve(x0, 0.0)
    assert np.max(np.abs(r0["Unew"][:, 1:4])) > 1e-3


def test_warm_start_keeps_the_whole_sequence(oracle_mod):
    """warm_start = 1 (the complete new sequence is the next nominal, no
    shift): the nominal equals U*_new row for row, and the next solve samples
    around it -- its update is the weighted mean of clamp(U*_new + sigma z)."""
    mc, sc, tr, x0 = _small_case()
    sc.warm_start = 1
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r = ctl.solve(x0, 0.0)
    np.testing.assert_array_equal(ctl.nominal, r["Unew"])
    r2 = ctl.solve(x0, 0.0, want_Z=True)
    us = np.clip(r["Unew"][None] + np.asarray(sc.sigma) * r2["Z"].transpose(1, 0, 2), mc.u_min, mc.u_max)
    us[:, :, 4] = 0
    np.testing.assert_allclose(r2["Unew"], np.einsum("m,mkj->kj", r2["w"], us), atol=1e-12)


def test_noise_stream_and_iteration_counter(oracle_mod):
    mc, sc, tr, x0 = _small_case()
    ctl = oracle_mod.OracleController(mc, sc, tr)
    r0 = ctl.solve(x0, 0.0, want_Z=True)
    r1 = ctl.solve(x0, 0.0, want_Z=True)
    for m, k in ((0, 0), (5, 3), (47, 7)):
        np.testing.assert_array_equal(r0["Z"][k, m, :4], oracle_mod.normals4(sc.seed, sc.drone_id, m, k, 0, 0))
        np.testing.assert_array_equal(r1["Z"][k, m, :4], oracle_mod.normals4(sc.seed, sc.drone_id, m, k, 1, 0))


def test_fifth_normals_take_four_steps_from_one_draw(oracle_mod):
    """Contouring's 5th normals of steps 4j .. 4j+3 are the four normals of
    Philox block 1 at step 4j, in order: each block-1 draw is used once, and
    the stream of a sample never repeats a value across steps."""
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_CONTOUR)
    sc.K, sc.N = 8, 10
    r = oracle_mod.OracleController(mc, sc, tr).solve(x0, 0.0, want_Z=True)
    for m in range(sc.K):
        col = r["Z"][:, m, 4]
        for j in range(0, sc.N, 4):
            draw = oracle_mod.normals4(sc.seed, sc.drone_id, m, j, 0, 1)
            np.testing.assert_array_equal(col[j:j + 4], draw[: len(col[j:j + 4])])
        assert len(set(col.tolist())) == sc.N


def test_plant_crossing_advances_the_gate_and_shifts_counts(oracle_mod):
    mc, sc, tr, x0 = _small_case()
    ctl = oracle_mod.OracleController(mc, sc, tr)
    g = tr.gates[0]
    c, n, l = _gate_frame(g)
    before, after = c - 0.1 * n, c + 0.1 * n
    xa = x0.copy()
    xa[:3] = before
    xb = x0.copy()
    xb[:3] = after
    ctl.set_state(prevcnt=[0, 1, 1, 2, 2, 2, 2, 2], prev_x0=xa)
    r = ctl.solve(xb, 0.0)
    assert r["gate_at_start"] == 1
    # a non-crossing move does not advance
    ctl2 = oracle_mod.OracleController(mc, sc, tr)
    ctl2.set_state(prev_x0=xa)
    r2 = ctl2.solve(xa, 0.0)
    assert r2["gate_at_start"] == 0


def test_nonfinite_costs_get_zero_weight(oracle_mod):
    mc, sc, tr, x0 = _small_case()
    ctl = oracle_mod.OracleController(mc, sc, tr)
    x_bad = x0.copy()
    x_bad[3] = np.nan
    r = ctl.solve(x_bad, 0.0)
    assert r["status"] == 1
    np.testing.assert_allclose(r["Unew"][:, 0], mc.hover)


# ---------------------------------------------------------------------------
# the rotor-thrust-rate model (Eq. 2 as printed: u = dT_s/dt, torque map)
# ---------------------------------------------------------------------------

def _rotor_mc(**kw):
    mc = W.rotor_model()
    for k, v in kw.items():
        setattr(mc, k, v)
    return mc


def test_rotor_hover_is_an_equilibrium(oracle_mod):
    mc = _rotor_mc()
    x = _state(p=(1, -2, 3), q=W.yaw_quat(0.7))
    T = np.full(4, mc.hover / 4)
    x1, T1 = x.copy(), T.copy()
    for _ in range(50):
        x1, T1 = oracle_mod.rk4_step_rotor(mc, x1, T1, np.zeros(4), 0.02)
    np.testing.assert_allclose(x1, x, atol=1e-12)
    np.testing.assert_array_equal(T1, T)


def test_rotor_free_fall_is_exact(oracle_mod):
    mc = _rotor_mc()
    x = _state(p=(0, 0, 50), v=(1, 2, 3))
    T = np.zeros(4)
    h, n = 0.05, 20
    for _ in range(n):
        x, T = oracle_mod.rk4_step_rotor(mc, x, T, np.zeros(4), h)
    t = h * n
    np.testing.assert_allclose(x[:3], [t, 2 * t, 50 + 3 * t - 0.5 * mc.gravity * t * t], atol=1e-11)
    np.testing.assert_allclose(x[3:6], [1, 2, 3 - mc.gravity * t], atol=1e-12)


def test_rotor_thrust_ramp_is_exact(oracle_mod):
    """Level attitude, all rotors ramping at the same rate r from a: the
    collective thrust 4 (a + r t) is linear in t, so v_z is quadratic and p_z
    cubic -- RK4 with the exact stage thrusts reproduces both exactly."""
    mc = _rotor_mc()
    a, r, m, g = 1.5, 2.0, mc.mass, mc.gravity
    x = _state(p=(0, 0, 5))
    T = np.full(4, a)
    h, n = 0.03, 40
    for _ in range(n):
        x, T = oracle_mod.rk4_step_rotor(mc, x, T, np.full(4, r), h)
    t = h * n
    vz = (4 * a / m - g) * t + 2 * r * t * t / m
    pz = 5 + 0.5 * (4 * a / m - g) * t * t + 2 * r * t ** 3 / (3 * m)
    assert abs(x[5] - vz) < 1e-11 and abs(x[2] - pz) < 1e-11
    np.testing.assert_allclose(T, a + r * t, atol=1e-12)


def test_rotor_thrust_saturates_in_its_range(oracle_mod):
    mc = _rotor_mc()
    T0 = np.array([9.0, 0.5, 5.0, 9.9])
    u = np.array([10.0, -10.0, 0.0, 10.0])
    for t, expect in ((0.04, [9.4, 0.1, 5.0, 10.0]), (0.1, [10.0, 0.0, 5.0, 10.0]), (0.5, [10.0, 0.0, 5.0, 10.0])):
        np.testing.assert_allclose(oracle_mod.rotor_at(mc, T0, u, t), expect, atol=1e-15)


@pytest.mark.parametrize("pattern,axis", [((1, 1, -1, -1), 0), ((-1, 1, 1, -1), 1), ((1, -1, 1, -1), 2)])
def test_rotor_torque_map(oracle_mod, pattern, axis):
    """Differential thrust patterns of the torque map in Eq. 2: each excites
    one body axis only; the collective thrust is the rotor sum."""
    mc = _rotor_mc()
    a, d = 2.0, 0.3
    T = a + d * np.asarray(pattern, float)
    dx = oracle_mod.deriv_rotor(mc, _state(), T)
    l2 = mc.arm / math.sqrt(2.0)
    tau = [l2 * 4 * d, l2 * 4 * d, mc.c_tau * 4 * d][axis]
    expect = np.zeros(3)
    expect[axis] = tau / mc.inertia[axis]
    np.testing.assert_allclose(dx[10:13], expect, atol=1e-14)
    assert abs(dx[5] - (4 * a / mc.mass - mc.gravity)) < 1e-14


def test_rotor_yaw_spin_up(oracle_mod):
    """A constant yaw torque from rest: omega_z grows linearly (exact) and
    the attitude follows the yaw angle psi = alpha t^2 / 2 (RK4 order)."""
    mc = _rotor_mc()
    a, d = mc.hover / 4, 0.2
    T = a + d * np.array([1.0, -1.0, 1.0, -1.0])
    alpha = 4 * mc.c_tau * d / mc.inertia[2]
    x = _state()
    h, n = 0.01, 30
    for _ in range(n):
        x, T = oracle_mod.rk4_step_rotor(mc, x, T, np.zeros(4), h)
    t = h * n
    assert abs(x[12] - alpha * t) < 1e-12
    psi = 0.5 * alpha * t * t
    np.testing.assert_allclose(x[6:10], [math.cos(psi / 2), 0, 0, math.sin(psi / 2)], atol=1e-9)


def test_rotor_tracking_effort_is_on_the_rates(oracle_mod):
    """Tracking a reference that is the rollout of a known rate sequence: the
    cost is sum ||u||^2_R on the rates themselves (no hover offset)."""
    mc = _rotor_mc()
    N, h = 10, 0.03
    rng = np.random.default_rng(8)
    U = np.zeros((N, 5))
    U[:, :4] = rng.normal(0, 3.0, (N, 4))
    x0 = _state(p=(1, 2, 3), q=W.yaw_quat(-0.3))
    T0 = np.array([2.0, 2.2, 1.9, 2.1])
    sc = W.SolveConfig(objective=2, K=1, N=N, dt=h)
    _, X, _, Tr = oracle_mod.rollout(mc, sc, _line_track(), x0, U, T0=T0, want_T=True)
    np.testing.assert_allclose(Tr[1], T0 + U[0, :4] * h, atol=1e-14)
    xref = np.vstack([X])
    J, _, _ = oracle_mod.rollout(mc, sc, _line_track(), x0, U, xref=xref, T0=T0)
    expect = float(np.sum(np.asarray(sc.R) * U[:, :4] ** 2))
    assert abs(J - expect) < 1e-9


def test_rotor_controller_state(oracle_mod):
    """The nominal starts at zero rates (Algorithm 1's U = 0) and the rotor
    thrusts advance by the applied u0 over one control period."""
    mc = _rotor_mc()
    _, sc, tr, x0 = W.c1_single_gate()
    sc = W.rotor_solve(sc)
    sc.K, sc.N = 32, 6
    ctl = oracle_mod.OracleController(mc, sc, tr)
    T0 = ctl.rotor.copy()
    np.testing.assert_allclose(T0, mc.hover / 4)
    r = ctl.solve(x0, 0.0, want_Z=True)
    us = np.clip(np.asarray(sc.sigma) * r["Z"].transpose(1, 0, 2), mc.u_min, mc.u_max)
    us[:, :, 4] = 0
    np.testing.assert_allclose(r["Unew"], np.einsum("m,mkj->kj", r["w"], us), atol=1e-12)
    np.testing.assert_allclose(ctl.rotor, np.clip(T0 + r["u0"][:4] * sc.dt, mc.thrust_min, mc.thrust_max),
                               atol=1e-14)


# ---------------------------------------------------------------------------
# outputs that scale or filter the parity tests: near-boundary flags and the
# cost-term magnitude J_abs (relative-error denominator)
# ---------------------------------------------------------------------------

def _line_solve(oracle_mod, x0, N, **kw):
    """One solve of a single unperturbed sample (K = 1, caller normals all
    zero) on the straight two-gate line: the hover input keeps the velocity,
    so p_k = p_0 + k h v in closed form."""
    tr = _line_track(2, spacing=6.0)
    mc = _mc()
    sc = W.SolveConfig(objective=kw.pop("objective", 0), K=1, N=N, dt=0.05, **kw)
    ctl = oracle_mod.OracleController(mc, sc, tr)
    return ctl.solve(np.asarray(x0, float), 0.0, Z_in=np.zeros((N, 1, 5))), tr, sc


@pytest.mark.parametrize("ds,expect", [(3e-6, 1), (3e-4, 0)])
def test_near_plane_flag(oracle_mod, ds, expect):
    """A state within flag_eps (1e-5 m) of the gate plane sets bit 0; one
    3e-4 m away sets nothing."""
    vx, h = 5.0, 0.05
    r, _, _ = _line_solve(oracle_mod, _state(p=(6.0 - 3 * vx * h + ds, 0.1, 2.05), v=(vx, 0, 0)), 8)
    assert r["near_flag"][0] == expect
    assert r["npass"][0] == 1


@pytest.mark.parametrize("lat,expect_flag,expect_pass", [(0.75 - 3e-6, 2, 1), (0.75 + 3e-6, 2, 0),
                                                         (-0.75 + 3e-6, 2, 1), (-0.75 - 3e-6, 2, 0),
                                                         (0.75 - 3e-4, 0, 1), (0.75 + 3e-4, 0, 0)])
def test_near_edge_flag(oracle_mod, lat, expect_flag, expect_pass):
    """A crossing point within flag_eps of the opening's edge sets bit 1,
    inside (counted pass) or outside (no pass); 3e-4 m from it, nothing."""
    r, _, _ = _line_solve(oracle_mod, _state(p=(6.0 - 0.65, lat, 2.0), v=(5.0, 0, 0)), 8, q_near=0.0)
    assert r["near_flag"][0] == expect_flag
    assert r["npass"][0] == expect_pass


@pytest.mark.parametrize("dr,expect", [(3e-6, 4), (-3e-6, 4), (3e-4, 0)])
def test_near_sphere_flag(oracle_mod, dr, expect):
    """A state p_k (k < N) within flag_eps of the near-gate sphere's radius
    sets bit 2 (Eq. 7's conditional term switches there)."""
    vx, h = 5.0, 0.05
    r_near = 1.5
    p0 = (6.0 - (r_near + dr) - 2 * vx * h, 0.0, 2.0)
    r, _, _ = _line_solve(oracle_mod, _state(p=p0, v=(vx, 0, 0)), 6, r_near=r_near, q_near=0.5)
    assert r["near_flag"][0] == expect


def test_gate_cost_scale_closed_form(oracle_mod):
    """J_abs of the gate objective is sum_k (||p_{k+1} - g||^2 + ||p_k - g||^2
    + |near_k|) + penalties: on the straight line, without the near term and
    before the gate, it follows from the closed-form positions."""
    vx, h, N = 5.0, 0.05, 6
    p0 = np.array([1.0, 0.3, 2.2])
    r, tr, _ = _line_solve(oracle_mod, _state(p=p0, v=(vx, 0, 0)), N, q_near=0.0)
    g = tr.gates[0, :3]
    P = [p0 + np.array([vx * h * k, 0, 0]) for k in range(N + 1)]
    expect = sum(np.sum((P[k + 1] - g) ** 2) + np.sum((P[k] - g) ** 2) for k in range(N))
    assert abs(r["Jabs"][0] - expect) < 1e-9 * expect
    # the cost itself telescopes
    assert abs(r["J"][0] - (np.sum((P[N] - g) ** 2) - np.sum((P[0] - g) ** 2))) < 1e-9


def test_tracking_cost_scale_equals_cost(oracle_mod):
    """Every Eq. 8 term is non-negative, so J_abs = J for tracking."""
    tr = W.random_course(7)
    mc = _mc()
    sc = W.SolveConfig(objective=2, K=16, N=10, dt=0.02)
    x0 = oracle_mod.ref_eval(tr, 0.2)
    x0[0:3] += 0.3
    r = oracle_mod.OracleController(mc, sc, tr).solve(x0, 0.2)
    assert np.all(r["J"] > 0)
    np.testing.assert_allclose(r["Jabs"], r["J"], rtol=1e-14)


def test_contouring_cost_scale_counts_the_progress_reward_positive(oracle_mod):
    """Eq. 9's only negative term is the progress reward -mu v_theta, so
    J_abs - J = 2 mu sum_k v_{k+1}; with a constant progress acceleration a
    from rest, v_{k+1} = (k + 1) a h."""
    N, h = 8, 0.05
    tr = _line_track(2)
    mc = _mc()
    sc = W.SolveConfig(objective=1, K=1, N=N, dt=h, mu=0.7)
    z5 = 0.2
    Z = np.zeros((N, 1, 5))
    Z[:, 0, 4] = z5
    a = sc.sigma[4] * z5
    r = oracle_mod.OracleController(mc, sc, tr).solve(_state(p=(0.0, 0.2, 2.0)), 0.0, Z_in=Z)
    expect = 2 * sc.mu * sum((k + 1) * a * h for k in range(N))
    assert abs((r["Jabs"][0] - r["J"][0]) - expect) < 1e-12


def test_binary32_floor_closed_form():
    """The conditioning floor of two samples: with the costs (0, D) and only
    the second one perturbed (J_abs = (0, A)), the floor is the larger change
    of U = (u1 + e u2) / (1 + e), e = exp(-D / lambda), over the signs drawn."""
    from oracle.conditioning import U32, binary32_floor
    lam, D, A = 0.7, 0.3, 250.0
    u1, u2 = np.array([[1.0, -2.0]]), np.array([[4.0, 1.0]])
    Us = np.stack([u1, u2])
    J = np.array([0.0, D])

    def U(d):
        e = math.exp(-d / lam)
        return (u1 + e * u2) / (1 + e)
    r = {"J": J, "Jabs": np.array([0.0, A]), "Us": Us, "Unew": U(D)}
    rng = np.random.default_rng(12345)
    signs = {int(rng.choice([-1.0, 1.0], size=2)[1]) for _ in range(8)}
    expect = max(np.max(np.abs(U(D + s * U32 * A) - U(D))) for s in signs)
    assert abs(binary32_floor(r, lam, 2) - expect) < 1e-15
    # first order: |u2 - u1| w1 w2 u A / lambda
    w2 = math.exp(-D / lam) / (1 + math.exp(-D / lam))
    assert abs(expect - np.max(np.abs(u2 - u1)) * (1 - w2) * w2 * U32 * A / lam) < 1e-3 * expect


# ---------------------------------------------------------------------------
# whole solves: the C oracle against an independent NumPy statement
# ---------------------------------------------------------------------------

def _cross_cases():
    mc, sc, tr, x0 = W.c1_single_gate()
    sc.K, sc.N = 48, 8
    x0 = np.array(x0, float)
    g = tr.gates[0]
    x0[3:6] = 4.0 * np.array([math.cos(g[3]), math.sin(g[3]), 0.0])  # flies through gate 0
    yield "gate", mc, sc, tr, x0, [0.05 * i for i in range(7)]
    for obj, name in ((1, "contour"), (2, "track")):
        mc, sc, tr, x0 = W.c2_full_scale(obj, 7)
        sc.K, sc.N = 48, 8
        yield name, mc, sc, tr, np.array(x0, float), [0.3, 0.32, 0.34]


@pytest.mark.parametrize("name", ["gate", "contour", "track"])
def test_c_oracle_equals_numpy_solve(oracle_mod, name):
    """Consecutive solves (K = 48, N = 8, the plant stepping with u0 between
    them: warm start, temporal rule, gate advance, progress state) agree with
    tests/numpy_solve.py: costs and their term magnitudes to 1e-12 relative,
    the new nominal to 1e-12, gate decisions exactly."""
    import numpy_solve as NS
    case = [c for c in _cross_cases() if c[0] == name][0]
    _, mc, sc, tr, x, t0s = case
    if name == "track":
        x = oracle_mod.ref_eval(tr, t0s[0])
        x[0:3] += 0.1
    a, b = oracle_mod.OracleController(mc, sc, tr), NS.NumpyController(mc, sc, tr)
    passes = 0
    for t0 in t0s:
        ra, rb = a.solve(x, t0), b.solve(x, t0)
        ok = ra["near_flag"] == 0
        assert ok.sum() >= sc.K - 2
        den = np.maximum(np.abs(ra["J"]), ra["Jabs"])
        assert np.max(np.abs(ra["J"] - rb["J"])[ok] / den[ok]) < 1e-12
        np.testing.assert_allclose(rb["Jabs"][ok], ra["Jabs"][ok], rtol=1e-12)
        np.testing.assert_allclose(rb["Unew"], ra["Unew"], rtol=0, atol=1e-12)
        np.testing.assert_array_equal(rb["npass"][ok], ra["npass"][ok])
        np.testing.assert_array_equal(rb["first_pass"][ok], ra["first_pass"][ok])
        passes += int(ra["npass"].max())
        x = oracle_mod.rk4_step(mc, x, ra["u0"][:4], sc.dt)
    if name == "gate":
        assert passes > 0 and a.gate == b.gate == 1  # samples pass, and so does the plant
