"""The rotor-thrust-rate input model (Eq. 2 as printed: u = dT_s/dt, the
torque map, saturating rotor thrusts) on the CUDA path against the FP64 oracle.

Covered: rollouts of given rate sequences (states and thrusts, with
saturation), whole solves of each objective at full scale, a closed-loop
sequence with the rotor thrusts carried between solves, the batched launch
mixing both models and the server.  Tolerances are those of the parity tests
(per-sample cost 1e-4 relative, nominal 1e-5 scaled by the conditioning).
"""
import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W
from parity_util import compare, f32_case, make_pair, push_oracle_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    from paper_2509_14726_gb300 import mppi
    return mppi


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _rotor_case(objective, K=4096, N=50, seed=7):
    _, sc, tr, x0 = W.c2_full_scale(objective, seed)
    sc = W.rotor_solve(sc)
    sc.K, sc.N = K, N
    return f32_case(W.rotor_model(), sc, tr, x0)


def test_rotor_rollout_states_match_oracle(O, M):
    mc = W.f32_model(W.rotor_model())
    rng = np.random.default_rng(1)
    B, N, dt = 64, 50, np.float32(0.02)
    x0 = np.zeros(13)
    x0[0:3] = (3.0, -2.0, 2.0)
    x0[3:6] = (1.0, 0.5, -0.2)
    x0[6:10] = W.yaw_quat(0.7)
    x0 = np.float32(x0).astype(np.float64)
    # rates about hover; half the batch starts with all four rotors next to
    # the same thrust bound and drives into it for ten steps, so that many
    # steps saturate without an extreme torque (differential saturation
    # tumbles the body within a fraction of a second, a chaotic regime where
    # binary32 and FP64 trajectories part for physical reasons)
    T0 = rng.uniform(1.9, 2.3, (B, 4))
    U = np.clip(rng.normal(0, 1.0, (B, N, 4)), -10, 10)
    hi = rng.random(B // 2) < 0.5
    T0[: B // 2] = np.where(hi, 9.8, 0.2)[:, None] + rng.uniform(-0.02, 0.02, (B // 2, 4))
    U[: B // 2, :10] = np.where(hi, 10.0, -10.0)[:, None, None] + rng.normal(0, 0.2, (B // 2, 10, 4))
    T0, U = np.float32(T0), np.float32(np.clip(U, -10, 10))
    dx0 = torch.tensor(np.float32(x0), device="cuda")
    dT0 = torch.tensor(T0, device="cuda")
    dU = torch.tensor(U, device="cuda")
    dX = torch.zeros((B, N + 1, 13), dtype=torch.float32, device="cuda")
    dT = torch.zeros((B, N + 1, 4), dtype=torch.float32, device="cuda")
    M.mppi_rollout_states_rotor(M.make_model(mc), float(dt), N, B, dx0.data_ptr(), dT0.data_ptr(), dU.data_ptr(),
                                dX.data_ptr(), dT.data_ptr())
    torch.cuda.synchronize()
    X = dX.cpu().numpy().astype(np.float64)
    T = dT.cpu().numpy().astype(np.float64)
    sc = W.SolveConfig(N=N, dt=float(dt))
    saturated = 0
    for b in range(B):
        Ub = np.zeros((N, 5))
        Ub[:, :4] = U[b]
        _, Xo, _, To = O.rollout(mc, sc, W.circle_track(), x0, Ub, gate0=0, T0=T0[b].astype(np.float64),
                                 want_T=True)
        saturated += int(np.sum((To == mc.thrust_min) | (To == mc.thrust_max)))
        # the compensated thrust ramp: one rounding of the returned thrust
        assert np.max(np.abs(T[b] - To)) <= 2.0 ** -23 * mc.thrust_max
        # undamped body rates (no rate loop in this model) keep the binary32
        # roundings of every step, about six per state: over N = 50 steps
        # 50 * 6 * 2^-24 ~ 2e-5 of the largest size each state component
        # reaches along the trajectory
        scale = np.max(np.abs(Xo), axis=0)
        bound = 2e-5 + N * 6 * 2.0 ** -24 * scale[None, :]
        assert np.all(np.abs(X[b] - Xo) <= bound), np.max(np.abs(X[b] - Xo) / bound)
    assert saturated > 100


@pytest.mark.parametrize("objective", [0, 1, 2])
def test_rotor_full_scale_each_objective(O, M, objective):
    case = _rotor_case(objective)
    gpu, ora = make_pair(case)
    t0 = 0.37
    x0 = case.x0
    if objective == 2:
        x0 = np.float32(O.ref_eval(case.tr, t0)).astype(np.float64)
        x0[0:3] += 0.1
    gpu.solve(x0, t0)
    r = ora.solve(x0, t0)
    st = compare(gpu, r, f"rotor model, objective {objective}")
    print(f"\nrotor objective {objective}: {st}")
    # the handle's rotor thrusts advance by u0 over one control period
    np.testing.assert_allclose(gpu.rotor_thrusts(), ora.rotor, atol=2e-5)
    gpu.close()


@pytest.mark.parametrize("objective", [0, 1, 2])
def test_rotor_closed_loop_sequence(O, M, objective):
    """Several solves in closed loop with the FP64 rotor-model plant; the GPU
    handle starts from the oracle's state (nominal, counters, rotor thrusts)
    at every step."""
    case = _rotor_case(objective, K=1024, N=30)
    gpu, ora = make_pair(case)
    x = case.x0.copy() if objective != 2 else O.ref_eval(case.tr, 0.0)
    T = ora.rotor.copy()
    t = 0.0
    for step in range(4):
        push_oracle_state(gpu, ora)
        xs = np.float32(x).astype(np.float64)
        gpu.solve(xs, t)
        r = ora.solve(xs, t)
        compare(gpu, r, f"rotor objective {objective} step {step}")
        x, T = O.rk4_step_rotor(case.mc, x, T, r["u0"][:4], case.sc.dt)
        np.testing.assert_allclose(ora.rotor, T, atol=1e-12)
        t += case.sc.dt
    gpu.close()


def test_rotor_thrust_setter(M):
    case = _rotor_case(0, K=256, N=10)
    gpu = M.Controller(case.mc, case.sc, case.tr)
    np.testing.assert_allclose(gpu.rotor_thrusts(), np.float32(case.mc.mass * case.mc.gravity / 4), rtol=1e-6)
    gpu.set_rotor_thrusts([1.0, 2.0, 3.0, 4.0])
    np.testing.assert_array_equal(gpu.rotor_thrusts(), np.float32([1, 2, 3, 4]))
    ctbr = M.Controller(W.ModelConfig(), case.sc, case.tr)
    with pytest.raises(M.MppiError):
        ctbr.rotor_thrusts()
    with pytest.raises(M.MppiError):
        M.Controller(case.mc, case.sc, case.tr, noise_dtype=M.NOISE_BF16)
    gpu.close()
    ctbr.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_mixing_models_equals_alone(M, use_graph):
    items = W.c3_batch(n_drones=8, K_lo=300, K_hi=2000, N_lo=5, N_hi=30)
    pairs = []
    for i, it in enumerate(items):
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
        mc = W.ModelConfig()
        if i % 2:
            mc, sc = W.rotor_model(), W.rotor_solve(sc)
        case = f32_case(mc, sc, it.track, it.x0)
        pairs.append((M.Controller(case.mc, case.sc, case.tr), M.Controller(case.mc, case.sc, case.tr), case))
    X0 = np.array([c.x0 for _, _, c in pairs])
    b = M.mppi_batch_create([g1.h for g1, _, _ in pairs], use_graph=use_graph)
    for rep in range(2):
        ub, _ = M.mppi_batch_solve(b, len(pairs), X0, np.full(len(pairs), 0.3))
        for i, (g1, g2, c) in enumerate(pairs):
            ua, _ = g2.solve(c.x0, 0.3)
            np.testing.assert_array_equal(ub[i], ua)
            np.testing.assert_array_equal(g1.costs(), g2.costs())
            assert g1.export_state() == g2.export_state()
    M.mppi_batch_destroy(b)
    for g1, g2, _ in pairs:
        g1.close()
        g2.close()


def test_server_with_rotor_drones(M):
    fleet = W.c5_fleet(n_drones=4, distinct_tracks=2)
    srv = M.Server(len(fleet), 1 << 30, n_slots=2, max_batch=4)
    alone = []
    for i, d in enumerate(fleet):
        sc = W.SolveConfig(objective=d.objective, K=1024, N=30, dt=0.02, drone_id=d.drone_id)
        mc = W.ModelConfig()
        if i % 2 == 0:
            mc, sc = W.rotor_model(), W.rotor_solve(sc)
        srv.add_drone(mc, sc, d.track, 1024, 30)
        alone.append(M.Controller(mc, sc, d.track, K_cap=1024, N_cap=30))
    X0 = np.array([d.x0 for d in fleet])
    n = len(fleet)
    for rnd in range(2):
        ids = srv.submit(np.arange(n), X0, np.full(n, 0.1 * rnd), np.full(n, 1024), np.full(n, 30))
        got = {}
        while len(got) < n:
            while srv.step() > 0:
                pass
            for r in srv.poll().tolist():
                got[int(r[0])] = r
        for i, c in enumerate(alone):
            u, _ = c.solve(X0[i], 0.1 * rnd)
            np.testing.assert_array_equal(np.asarray(got[int(ids[i])][5], np.float32), u)
    for i, c in enumerate(alone):
        assert srv.export_drone(i) == c.export_state()
        c.close()
    srv.close()
