"""CUDA path against the FP64 oracle, element by element, on seeded inputs.

Every test here calls libmppi through its C ABI (the ctypes binding) on
cuda:0.  Tolerances: Philox words bit-exact; standard normals within the
rounding of binary32 log/sqrt/sincospi (6 ulp relative); per-sample cost
relative error <= 1e-4; nominal control absolute error <= 1e-5 (N, rad/s);
gate-crossing decisions identical except for samples the oracle flags as
within 1e-5 m of a gate plane, an opening edge or the near-gate sphere.
"""
import math

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W
from parity_util import Case, compare, f32_case, make_pair, push_oracle_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def M():
    from paper_2509_14726_gb300 import mppi
    return mppi


# ---------------------------------------------------------------------------
# Philox4x32-10 and Box-Muller
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((7, 3), (123, 45, 6, 1)),
                                     ((0xFFFFFFFF, 0xDEADBEEF), (0xFFFFFF00, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF))])
def test_philox_bit_exact(O, M, key, ctr):
    n = 4096
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    M.mppi_philox(key[0], key[1], ctr[0], ctr[1], ctr[2], ctr[3], n, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    for i in list(range(0, 64)) + list(range(n - 64, n)) + list(range(64, n - 64, 97)):
        c0 = (ctr[0] + i) & 0xFFFFFFFF
        np.testing.assert_array_equal(got[i], O.philox((c0, ctr[1], ctr[2], ctr[3]), key))


def test_normals_within_binary32_rounding(O, M):
    n = 20000
    out = torch.zeros(4 * n, dtype=torch.float32, device="cuda")
    M.mppi_normals(11, 5, 3, 2, 0, n, out.data_ptr())
    torch.cuda.synchronize()
    z = out.cpu().numpy().astype(np.float64).reshape(n, 4)
    ref = np.array([O.normals4(11, 5, m, 3, 2, 0) for m in range(n)])
    err = np.abs(z - ref)
    assert np.all(err <= 6 * 2.0 ** -23 * np.abs(ref) + 1e-7), err.max()


@pytest.mark.parametrize("K,N,noise_gen", [(300, 11, 0), (40000, 11, 0), (300, 11, 1), (5000, 23, 1)])
def test_fifth_normal_stream(O, M, K, N, noise_gen):
    """Contouring's 5th normals: step k uses normal k mod 4 of Philox block 1
    at step 4 floor(k / 4).  Checked on every step against the oracle's draw,
    for the separate pass split along the horizon (few tiles) and in one span
    (many tiles), and for the draw inside the rollout."""
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_CONTOUR)
    sc.K, sc.N = K, N
    case = f32_case(mc, sc, tr, x0)
    gpu = M.Controller(case.mc, case.sc, case.tr, noise_gen=noise_gen)
    gpu.solve(case.x0, 0.0)
    Z5 = gpu.noise()[:, :, 4]
    ms = sorted(set(list(range(0, 5)) + list(range(0, K, max(1, K // 97))) + [K - 1]))
    ref = np.array([[O.normals4(sc.seed, sc.drone_id, m, k - k % 4, 0, 1)[k % 4] for m in ms] for k in range(N)])
    err = np.abs(Z5[:, ms] - ref)
    assert np.all(err <= 6 * 2.0 ** -23 * np.abs(ref) + 1e-7), err.max()
    gpu.close()


# ---------------------------------------------------------------------------
# the model: RK4 rollouts of given sequences
# ---------------------------------------------------------------------------

def test_rollout_states_match_oracle(O, M):
    mc = W.f32_model(W.ModelConfig())
    rng = np.random.default_rng(0)
    B, N, dt = 64, 50, np.float32(0.02)
    x0 = np.zeros(13)
    x0[0:3] = (3.0, -2.0, 2.0)
    x0[3:6] = (1.0, 0.5, -0.2)
    x0[6:10] = W.yaw_quat(0.7)
    x0 = np.float32(x0).astype(np.float64)
    U = np.zeros((B, N, 4))
    U[:, :, 0] = mc.mass * mc.gravity + rng.normal(0, 2.5, (B, N))
    U[:, :, 1:] = rng.normal(0, 1.0, (B, N, 3))
    U = np.clip(U, mc.u_min[:4], mc.u_max[:4]).astype(np.float32)
    dx0 = torch.tensor(np.float32(x0), device="cuda")
    dU = torch.tensor(U, device="cuda")
    dX = torch.zeros((B, N + 1, 13), dtype=torch.float32, device="cuda")
    M.mppi_rollout_states(M.make_model(mc), float(dt), N, B, dx0.data_ptr(), dU.data_ptr(), dX.data_ptr())
    torch.cuda.synchronize()
    X = dX.cpu().numpy().astype(np.float64)
    sc = W.SolveConfig(N=N, dt=float(dt))
    for b in range(B):
        _, Xo, _ = O.rollout(mc, sc, W.circle_track(), x0, U[b].astype(np.float64), gate0=0)
        assert np.max(np.abs(X[b, :, 0:3] - Xo[:, 0:3])) < 2e-5
        assert np.max(np.abs(X[b, :, 3:6] - Xo[:, 3:6])) < 2e-5
        assert np.max(np.abs(X[b, :, 6:13] - Xo[:, 6:13])) < 2e-5


# ---------------------------------------------------------------------------
# whole solves
# ---------------------------------------------------------------------------

def c1_case(**kw):
    mc, sc, tr, x0 = W.c1_single_gate()
    for k, v in kw.items():
        setattr(sc, k, v)
    return f32_case(mc, sc, tr, x0)


def test_c1_first_solve(O, M):
    case = c1_case()
    gpu, ora = make_pair(case)
    u0, rc = gpu.solve(case.x0, 0.0)
    r = ora.solve(case.x0, 0.0)
    st = compare(gpu, r, "C1")
    np.testing.assert_allclose(u0[:4], r["u0"][:4], atol=1e-5)
    # the warm start and the counters
    np.testing.assert_allclose(gpu.nominal()[:, :4], ora.nominal[:, :4], atol=1e-5)
    info = gpu.info()
    assert info[2] == 1 and info[3] == 0 and info[1] == 0
    np.testing.assert_array_equal(gpu.passcnt(), r["passcnt"])
    # the sampled noise itself
    Z = gpu.noise()
    zo = np.array([[O.normals4(0, 0, m, k, 0, 0) for m in range(0, case.sc.K, 37)] for k in range(case.sc.N)])
    assert np.max(np.abs(Z[:, ::37, :4] - zo)) < 5e-6
    gpu.close()


@pytest.mark.parametrize("K,N,block", [(1, 1, 32), (33, 3, 32), (1000, 13, 128), (3000, 20, 64), (5000, 7, 128),
                                     (20000, 5, 64), (2100, 30, 64), (8192, 25, 128)])
def test_ragged_tiles_and_merge_levels(O, M, K, N, block):
    """K not a multiple of the block, one tile, several tiles, and enough
    tiles for the two-level merge (more than 16), with short and long
    horizons (one and several of the N x 5 sums per thread)."""
    case = c1_case(K=K, N=N)
    gpu, ora = make_pair(case, block=block)
    gpu.solve(case.x0, 0.0)
    r = ora.solve(case.x0, 0.0)
    compare(gpu, r, f"K={K} N={N} block={block}")
    gpu.close()


def test_closed_loop_sequence_from_oracle_states(O, M):
    """Ten consecutive solves along the oracle's own closed loop; before each
    solve the GPU handle starts from the oracle's controller state, so every
    solve is compared from identical inputs (gate index, pass counts of the
    previous nominal, RNG iteration, nominal)."""
    case = c1_case()
    gpu, ora = make_pair(case)
    x, t = case.x0.copy(), 0.0
    decisions = 0
    for step in range(10):
        push_oracle_state(gpu, ora)
        xs = np.float32(x).astype(np.float64)
        gpu.solve(xs, t)
        r = ora.solve(xs, t)
        st = compare(gpu, r, f"step {step}")
        decisions += st["decision_mismatch_flagged"]
        np.testing.assert_array_equal(gpu.passcnt(), r["passcnt"])
        assert gpu.info()[0] == r["gate_at_start"]
        x = O.rk4_step(case.mc, x, r["u0"][:4], case.sc.dt)
        t += case.sc.dt
    gpu.close()


def test_gpu_state_evolves_like_the_oracle(O, M):
    """Without any state transfer: both sides evolve their own controller
    state over five solves from the same x0 sequence."""
    case = c1_case()
    gpu, ora = make_pair(case)
    x, t = case.x0.copy(), 0.0
    for step in range(5):
        xs = np.float32(x).astype(np.float64)
        gpu.solve(xs, t)
        r = ora.solve(xs, t)
        compare(gpu, r, f"step {step}")
        x = O.rk4_step(case.mc, x, r["u0"][:4], case.sc.dt)
        t += case.sc.dt
    gpu.close()


def c2_case(objective, K=4096, N=50, seed=7):
    mc, sc, tr, x0 = W.c2_full_scale(objective, seed)
    sc.K, sc.N = K, N
    return f32_case(mc, sc, tr, x0)


@pytest.mark.parametrize("objective", [0, 1, 2])
def test_c2_full_scale_each_objective(O, M, objective):
    case = c2_case(objective)
    gpu, ora = make_pair(case)
    t0 = 0.37
    x0 = case.x0
    if objective == 2:
        # start near the reference so that the tracking cost is moderate
        x0 = np.float32(O.ref_eval(case.tr, t0)).astype(np.float64)
        x0[0:3] += 0.1
    gpu.solve(x0, t0)
    r = ora.solve(x0, t0)
    compare(gpu, r, f"C2 objective {objective}")
    if objective == 1:
        sc = gpu.scalars()
        assert abs(sc[0] - r["theta0"][0]) < 1e-4
    if objective == 2:
        np.testing.assert_allclose(gpu.xref(), r["xref"], atol=2e-5)
    gpu.close()


@pytest.mark.parametrize("objective", [1, 2])
def test_objective_sequences(O, M, objective):
    """Several solves with the progress state (contouring) or the reference
    time (tracking) moving on; GPU started from the oracle's state each time."""
    case = c2_case(objective, K=1024, N=30)
    gpu, ora = make_pair(case)
    t = 0.0
    x = case.x0.copy() if objective == 1 else O.ref_eval(case.tr, 0.0)
    for step in range(4):
        push_oracle_state(gpu, ora)
        xs = np.float32(x).astype(np.float64)
        gpu.solve(xs, t)
        r = ora.solve(xs, t)
        compare(gpu, r, f"objective {objective} step {step}")
        x = O.rk4_step(case.mc, x, r["u0"][:4], case.sc.dt)
        t += case.sc.dt
    gpu.close()


@pytest.mark.parametrize("accum", [1, 2])
def test_accumulation_modes(O, M, accum):
    case = c2_case(0, K=4096, N=50)
    gpu, ora = make_pair(case, accum=accum)
    gpu.solve(case.x0, 0.0)
    r = ora.solve(case.x0, 0.0)
    compare(gpu, r, f"accum {accum}")
    gpu.close()


def test_caller_noise_bf16(O, M):
    """BF16 noise storage: the noise is a seeded input (bf16 values drawn by
    the input generator), given to both sides."""
    case = c2_case(0, K=2048, N=40)
    rng = np.random.default_rng(99)
    z = rng.standard_normal((case.sc.N, case.sc.K, 4)).astype(np.float32)
    zb = torch.tensor(z).to(torch.bfloat16)
    z_dec = zb.float().numpy().astype(np.float64)
    gpu, ora = make_pair(case, noise_dtype=M.NOISE_BF16)
    dz = zb.cuda().contiguous()
    M.mppi_set_noise(gpu.h, dz.data_ptr(), None)
    gpu.solve(case.x0, 0.0)
    Zin = np.zeros((case.sc.N, case.sc.K, 5))
    Zin[:, :, :4] = z_dec
    r = ora.solve(case.x0, 0.0, Z_in=Zin)
    compare(gpu, r, "bf16 caller noise")
    # the next solve goes back to Philox; its stored bf16 noise is the
    # round-to-nearest-even of the binary32 normals
    gpu.solve(case.x0, 0.0)
    Zg = gpu.noise()[:, :, :4]
    zo = np.array([[O.normals4(0, 0, m, k, 1, 0) for m in range(0, case.sc.K, 101)] for k in range(case.sc.N)])
    assert np.max(np.abs(Zg[:, ::101] - zo)) <= 2.0 ** -8 * np.max(np.abs(zo)) + 1e-6
    gpu.close()


def test_batch_equals_alone(O, M):
    """Uneven solves in one batched launch give exactly what each gives alone."""
    items = W.c3_batch(n_drones=9, K_lo=300, K_hi=3000, N_lo=5, N_hi=40)
    gpus, alone = [], []
    for it in items:
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
        case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
        g1, _ = make_pair(case)
        g2, _ = make_pair(case)
        gpus.append((g1, g2, case))
    X0 = np.array([c.x0 for _, _, c in gpus])
    t0 = np.full(len(items), 0.3)
    for rep in range(2):
        ub, _ = M.mppi_solve_batch([g1.h for g1, _, _ in gpus], X0, t0)
        for i, (g1, g2, c) in enumerate(gpus):
            ua, _ = g2.solve(c.x0, 0.3)
            np.testing.assert_array_equal(ub[i], ua)
            np.testing.assert_array_equal(g1.costs(), g2.costs())
            np.testing.assert_array_equal(g1.nominal(), g2.nominal())
    for g1, g2, _ in gpus:
        g1.close()
        g2.close()


def test_batch_against_oracle(O, M):
    items = W.c3_batch(n_drones=6, K_lo=500, K_hi=2000, N_lo=10, N_hi=30)
    pairs = []
    for it in items:
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
        case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
        pairs.append((case,) + make_pair(case))
    t0 = 0.25
    X0 = []
    for case, _, _ in pairs:
        x = case.x0
        if case.sc.objective == 2:
            x = np.float32(W_ref(case.tr, t0)).astype(np.float64)
        X0.append(x)
    b = M.mppi_batch_create([g.h for _, g, _ in pairs], use_graph=True)
    u, _ = M.mppi_batch_solve(b, len(pairs), np.array(X0), np.full(len(pairs), t0))
    for i, (case, g, o) in enumerate(pairs):
        r = o.solve(X0[i], t0)
        compare(g, r, f"batch item {i} objective {case.sc.objective}")
        np.testing.assert_allclose(u[i, :4], r["u0"][:4], atol=1e-5)
    M.mppi_batch_destroy(b)
    for _, g, _ in pairs:
        g.close()


def W_ref(tr, t):
    from oracle import oracle as O
    return O.ref_eval(tr, t)


def test_degenerate_costs_keep_the_nominal(O, M):
    case = c1_case(K=64, N=8)
    gpu, ora = make_pair(case)
    x = case.x0.copy()
    x[3] = np.nan
    u0, rc = gpu.solve(x, 0.0)
    r = ora.solve(x, 0.0)
    assert rc == M.MPPI_WARN_DEGENERATE and r["status"] == 1
    np.testing.assert_allclose(u0[:4], r["u0"][:4], atol=1e-5)
    gpu.close()


def test_longest_horizon_and_state_roundtrip(O, M):
    case = c1_case(K=512, N=128, dt=0.01)
    gpu, ora = make_pair(case)
    gpu.solve(case.x0, 0.0)
    r = ora.solve(case.x0, 0.0)
    compare(gpu, r, "N=128")
    blob = gpu.export_state()
    u_a, _ = gpu.solve(case.x0, 0.0)
    gpu.import_state(blob)
    u_b, _ = gpu.solve(case.x0, 0.0)
    np.testing.assert_array_equal(u_a, u_b)
    gpu.close()


def test_async_solve_on_torch_stream(O, M):
    case = c1_case()
    gpu, ora = make_pair(case)
    s = torch.cuda.Stream()
    dx = torch.tensor(np.float32(case.x0), device="cuda")
    du = torch.zeros(5, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        M.mppi_solve_async(gpu.h, dx.data_ptr(), 0.0, s, du.data_ptr())
    s.synchronize()
    r = ora.solve(case.x0, 0.0)
    np.testing.assert_allclose(du.cpu().numpy()[:4], r["u0"][:4], atol=1e-5)
    gpu.close()


def test_set_shape_changes_K_and_N(O, M):
    case = c1_case(K=256, N=20)
    gpu, _ = make_pair(case, K_cap=2048, N_cap=40)
    gpu.solve(case.x0, 0.0)
    gpu.set_shape(1500, 33)
    sc2 = W.f32_solve(case.sc)
    sc2.K, sc2.N = 1500, 33
    from oracle import oracle as O_
    ora = O_.OracleController(case.mc, sc2, case.tr, cap=40)
    push_oracle_state(gpu, ora)
    gpu.solve(case.x0, 0.0)
    r = ora.solve(case.x0, 0.0)
    compare(gpu, r, "after set_shape")
    gpu.close()


@pytest.mark.parametrize("objective", [0, 1, 2])
@pytest.mark.parametrize("K", [8192, 2048])
def test_paper_table1_size(O, M, objective, K):
    """The paper's simulation parameters (Table I): 8192 samples (2048 on its
    onboard computer), horizon 20, dt 0.03, temperature 0.01 -- a much sharper
    weighting than lambda = 1; the conditioning-aware tolerance of the nominal
    scales with it."""
    mc, sc, tr, x0 = W.paper_table1(objective, K)
    case = f32_case(mc, sc, tr, x0)
    gpu, ora = make_pair(case)
    t0 = 0.21
    x = case.x0
    if objective == 2:
        x = np.float32(O.ref_eval(case.tr, t0)).astype(np.float64)
        x[0:3] += 0.1
    gpu.solve(x, t0)
    r = ora.solve(x, t0)
    st = compare(gpu, r, f"Table I size, K {K}, objective {objective}")
    print(f"\nTable I K={K} objective {objective}: {st}")
    gpu.close()


@pytest.mark.parametrize("variant", [{"nominal_sample": 1}, {"warm_start": 1}, {"temporal_rule": 2},
                                     {"temporal_rule": 0}, {"nominal_sample": 1, "warm_start": 1}],
                         ids=["nominal_candidate", "warm_keep", "same_index_rule", "no_rule", "both"])
def test_gate_logic_variants(O, M, variant):
    """Variants of the sampling, the warm start and the temporal rule, over a
    short closed-loop sequence (GPU started from the oracle's state at every
    step): per-sample costs and gate decisions, the update, and the next
    nominal (U*_new shifted by one step, or kept whole)."""
    mc, sc, tr, x0 = W.c2_full_scale(0)
    sc.K, sc.N = 2048, 30
    for k, v in variant.items():
        setattr(sc, k, v)
    case = f32_case(mc, sc, tr, x0)
    gpu, ora = make_pair(case)
    x = case.x0.copy()
    for step in range(3):
        push_oracle_state(gpu, ora)
        xs = np.float32(x).astype(np.float64)
        gpu.solve(xs, 0.02 * step)
        r = ora.solve(xs, 0.02 * step)
        compare(gpu, r, f"variant {variant} step {step}")
        unew = gpu.unew()
        expect = unew if sc.warm_start == 1 else np.vstack([unew[1:], unew[-1:]])
        np.testing.assert_array_equal(gpu.nominal(), expect)
        x = O.rk4_step(case.mc, x, r["u0"][:4], sc.dt)
    gpu.close()


@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_batch_mixing_variants_equals_alone(M, use_graph):
    """A plan mixing solves with and without the nominal candidate and with
    either warm start gives each solve exactly what it gets alone."""
    items = W.c3_batch(n_drones=8, K_lo=300, K_hi=2000, N_lo=5, N_hi=30)
    pairs = []
    for i, it in enumerate(items):
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id,
                           nominal_sample=i % 2, warm_start=(i // 2) % 2)
        case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
        pairs.append((M.Controller(case.mc, case.sc, case.tr), M.Controller(case.mc, case.sc, case.tr), case))
    X0 = np.array([c.x0 for _, _, c in pairs])
    b = M.mppi_batch_create([g1.h for g1, _, _ in pairs], use_graph=use_graph)
    for rep in range(2):
        ub, _ = M.mppi_batch_solve(b, len(pairs), X0, np.full(len(pairs), 0.3))
        for i, (g1, g2, c) in enumerate(pairs):
            ua, _ = g2.solve(c.x0, 0.3)
            np.testing.assert_array_equal(ub[i], ua)
            np.testing.assert_array_equal(g1.costs(), g2.costs())
            np.testing.assert_array_equal(g1.nominal(), g2.nominal())
            if c.sc.nominal_sample:
                assert np.all(g1.noise()[:, 0, :] == 0)
    M.mppi_batch_destroy(b)
    for g1, g2, _ in pairs:
        g1.close()
        g2.close()


@pytest.mark.parametrize("spt", [1, 2])
def test_full_bench_batch_sampled_against_oracle(O, M, spt):
    """The bench's own workload and launch: the 256-drone uneven batch (K
    log-uniform in [1024, 16384], N in [20, 80], 1/3 each objective), solved
    once through a captured batch plan with concurrent branches, at one and at
    two samples per thread (the autotuned launch shape).  Sampled
    solves -- the first two of each objective, the largest K and the longest
    N -- against the oracle on the same inputs.  The nominal tolerance takes
    the measured cost error of the weighted samples (long horizons and large
    tracking costs carry a larger absolute binary32 error)."""
    items = W.c3_batch(n_drones=256, seed=3)
    t0 = 0.3
    cases, ctls, X0 = [], [], []
    for it in items:
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, lam=1.0, seed=0, drone_id=it.drone_id)
        x = it.x0.copy()
        if it.objective == 2:
            x = it.track.ref[int(round(t0 / it.track.dt_ref)) % it.track.ref.shape[0]].copy()
        case = f32_case(W.ModelConfig(), sc, it.track, x)
        cases.append(case)
        ctls.append(M.Controller(case.mc, case.sc, case.tr, spt=spt))
        X0.append(case.x0)
    plan = M.mppi_batch_create([c.h for c in ctls], use_graph=1)
    M.mppi_batch_solve(plan, len(items), np.array(X0), np.full(len(items), t0))
    picked = []
    for obj in (0, 1, 2):
        picked += [i for i, it in enumerate(items) if it.objective == obj][:2]
    picked += [int(np.argmax([it.K for it in items])), int(np.argmax([it.N for it in items]))]
    for i in dict.fromkeys(picked):
        c = cases[i]
        r = O.OracleController(c.mc, c.sc, c.tr).solve(c.x0, t0)
        st = compare(ctls[i], r, f"bench drone {i} (objective {c.sc.objective}, K {c.sc.K}, N {c.sc.N})")
        print(f"\nbench drone {i}: {st}")
    M.mppi_batch_destroy(plan)
    for c in ctls:
        c.close()


def test_solve_batch_cache_under_threads(M):
    """mppi_solve_batch from several threads at once, with more distinct
    handle sets than its plan cache holds, so that plans leave the cache
    while other calls run them: every result equals the same solves made
    one handle at a time."""
    import threading
    items = W.c3_batch(n_drones=24, K_lo=256, K_hi=1024, N_lo=5, N_hi=15)
    errors = []

    def worker(tid):
        try:
            sets = []
            for s in range(3):
                its = items[tid * 6 + 2 * s: tid * 6 + 2 * s + 2]
                pair = []
                for it in its:
                    sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
                    case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
                    pair.append((M.Controller(case.mc, case.sc, case.tr), M.Controller(case.mc, case.sc, case.tr),
                                 case))
                sets.append(pair)
            for rep in range(4):
                for pair in sets:
                    X0 = np.array([c.x0 for _, _, c in pair])
                    ub, _ = M.mppi_solve_batch([g.h for g, _, _ in pair], X0, np.full(len(pair), 0.1 * rep))
                    for i, (_, alone, c) in enumerate(pair):
                        ua, _ = alone.solve(c.x0, 0.1 * rep)
                        if not np.array_equal(ub[i], ua):
                            errors.append((tid, rep, i, ub[i], ua))
            for pair in sets:
                for g, alone, _ in pair:
                    g.close()
                    alone.close()
        except Exception as e:  # reported below
            errors.append((tid, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors[:3]


def test_bounded_wait_reports_a_timeout_and_keeps_the_nominal(O, M):
    """The rollout's wait for its bulk copies is bounded.  Pointed at a barrier
    that nothing completes (a 1 ms limit), it gives up: the solve returns
    MPPI_ERR_TIMEOUT, no sample is used and the nominal is kept (U*_new = U*,
    u0 = U*[0]), the context stays usable, and with the normal wait the next
    solve matches the oracle."""
    case = c1_case()
    gpu, ora = make_pair(case)
    U_before = gpu.nominal().copy()
    gpu.set_copy_wait(1_000_000, unreachable=True)
    with pytest.raises(M.MppiError) as e:
        gpu.solve(case.x0, 0.0)
    assert e.value.code == M.MPPI_ERR_TIMEOUT
    np.testing.assert_array_equal(gpu.unew(), U_before)
    assert M.decode_state(gpu.export_state(), case.sc.N)["status"] == M.MPPI_ERR_TIMEOUT
    # the same handle, normal wait: the oracle's solve from the state the failed
    # solve left (its iteration counter advanced, the nominal shifted)
    gpu.set_copy_wait(200_000_000, unreachable=False)
    after = M.decode_state(gpu.export_state(), case.sc.N)
    assert after["iter"] == 1
    ora.set_state(U=after["U"][: case.sc.N], iter=after["iter"])
    x = case.x0
    gpu.solve(x, 0.0)
    r = ora.solve(x, 0.0)
    compare(gpu, r, "after a timed-out solve")
    gpu.close()


def test_reference_rows_staged_or_read_give_the_same_solve(M):
    """A tracking block stages the reference rows its window needs in shared
    memory by bulk copies (two when the window wraps past the end of the
    table) unless they would not fit, and then reads the table directly.  On
    a reference ten times finer than usual (dt_ref / 10), a handle of horizon
    cap 20 stages its rows and one of cap 128 cannot; the same solves,
    including windows across the wrap, agree bit for bit."""
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_TRACK)
    sc.K, sc.N = 1024, 20
    fine = 10
    T = tr.ref.shape[0]
    ref = np.zeros((T * fine, 13))
    for j in range(fine):
        a, b = tr.ref, np.roll(tr.ref, -1, axis=0)
        f = j / fine
        ref[j::fine] = (1 - f) * a + f * b
    ref[:, 6:10] /= np.linalg.norm(ref[:, 6:10], axis=1, keepdims=True)
    tr = W.Track(tr.gates, tr.closed, tr.path, tr.L, ref, tr.dt_ref / fine)
    case = f32_case(mc, sc, tr, x0)
    staged = M.Controller(case.mc, case.sc, case.tr)
    direct = M.Controller(case.mc, case.sc, case.tr, N_cap=128)
    period = T * fine * float(np.float32(tr.dt_ref))
    for t0 in (0.3, period - 0.1, period - 0.01):
        x = np.float32(tr.ref[int(t0 / tr.dt_ref) % (T * fine)]).astype(np.float64)
        ua, _ = staged.solve(x, t0)
        ub, _ = direct.solve(x, t0)
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(staged.costs(), direct.costs())
        np.testing.assert_array_equal(staged.xref(), direct.xref()[: sc.N + 1])
    staged.close()
    direct.close()
