"""Noise drawn inside the rollout -- stored (MPPI_NOISEGEN_FUSED) or drawn
again by the update and never stored (MPPI_NOISEGEN_REGEN) -- and noise drawn
by the separate pass after the previous solve (MPPI_NOISEGEN_AHEAD), against
the separate Philox pass and against the FP64 oracle.

Both evaluate the same Philox4x32-10 / Box-Muller arithmetic on the same
counters (Sec. III-B, Eq. 3), so the fused path's stored noise is
bit-identical to the two-kernel path's.  The rest of the rollout is a separate compilation
whose floating-point contractions the compiler chooses on its own, so costs
and the update agree to binary32 rounding (observed: 1e-8 relative in J),
not bit for bit; the same mode is bit-exact between the single, batched and
served paths.  Against the oracle the fused path is held to the parity
tolerances.  Covered: every objective, both noise storages, ragged tiles,
consecutive solves (the iteration counter moves), the batched launch (all
graph forms, both modes mixed in one plan), the server and caller noise (the
allocation-free entry point is covered in its own file).
"""
import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W
from parity_util import U_ABS_TOL, compare, f32_case, make_pair

# costs of the two compilations: binary32 rounding of a 13..50-step sum
J_ROUND_TOL = 1e-6

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


def _case(objective, K, N, seed=7):
    mc, sc, tr, x0 = W.c2_full_scale(objective, seed)
    sc.K, sc.N = K, N
    return f32_case(mc, sc, tr, x0)


def _x0(O, case, t0):
    if case.sc.objective == 2:
        x = np.float32(O.ref_eval(case.tr, t0)).astype(np.float64)
        x[0:3] += 0.1
        return x
    return case.x0


def _same(a, b):
    np.testing.assert_array_equal(a.costs(), b.costs())
    np.testing.assert_array_equal(a.unew(), b.unew())
    np.testing.assert_array_equal(a.nominal(), b.nominal())
    if a.params.noise_gen in (0, 1):
        np.testing.assert_array_equal(a.noise(), b.noise())
    assert a.export_state() == b.export_state()


def _close(a, b):
    """Same noise bit for bit (where a stores it); costs and update to
    binary32 rounding."""
    if a.params.noise_gen in (0, 1):
        np.testing.assert_array_equal(a.noise(), b.noise())
    na, fa = a.sample_info()
    nb, fb = b.sample_info()
    same = (na == nb) & (fa == fb)
    assert same.mean() >= 0.999
    Ja, Jb = a.costs(), b.costs()
    rel = np.abs(Ja - Jb) / np.maximum(np.abs(Jb), 1e-30)
    assert rel[same].max() <= J_ROUND_TOL, rel.max()
    assert np.abs(a.unew() - b.unew()).max() <= U_ABS_TOL
    assert np.abs(a.nominal() - b.nominal()).max() <= U_ABS_TOL


GEN_CASES = [(1, 0), (1, 1), (2, 0), (3, 0), (3, 1)]  # (noise generation, bf16 storage)


@pytest.mark.parametrize("objective", [0, 1, 2])
@pytest.mark.parametrize("gen,bf16", GEN_CASES)
@pytest.mark.parametrize("K,N,block", [(1000, 13, 128), (3001, 20, 64), (33, 3, 32)])
def test_drawn_in_rollout_matches_separate(O, M, objective, gen, bf16, K, N, block):
    case = _case(objective, K, N)
    kw = dict(noise_dtype=bf16, block=block)
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=gen, **kw)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL, **kw)
    t0 = 0.37
    x0 = _x0(O, case, t0)
    for rep in range(3):
        ua, _ = a.solve(x0, t0 + 0.02 * rep)
        ub, _ = b.solve(x0, t0 + 0.02 * rep)
        assert np.abs(ua - ub).max() <= U_ABS_TOL
        _close(a, b)
        assert a.info()[2] == b.info()[2] == rep + 1
    a.close()
    b.close()


@pytest.mark.parametrize("objective", [0, 1, 2])
@pytest.mark.parametrize("gen", [1, 2, 3])
def test_drawn_in_rollout_against_oracle(O, M, objective, gen):
    case = _case(objective, 4096, 50 if gen != 3 else 20)
    gpu, ora = make_pair(case, noise_gen=gen)
    t0 = 0.37
    x0 = _x0(O, case, t0)
    gpu.solve(x0, t0)
    r = ora.solve(x0, t0)
    compare(gpu, r, f"noise generation {gen}, objective {objective}")
    if gen in (2, 3):
        gpu.close()
        return
    # the stored normals are the oracle's Philox / Box-Muller draws
    Zg = gpu.noise()
    ms = range(0, case.sc.K, 257)
    zo = np.array([[O.normals4(case.sc.seed, case.sc.drone_id, m, k, 0, 0) for m in ms] for k in range(case.sc.N)])
    assert np.max(np.abs(Zg[:, ::257, :4] - zo)) <= 6 * 2.0 ** -23 * np.max(np.abs(zo)) + 1e-6
    gpu.close()


@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_batch_with_mixed_noise_modes(M, use_graph):
    """A plan holding handles of every noise generation mode and objective
    gives each solve exactly what it gets alone in the same mode."""
    items = W.c3_batch(n_drones=8, K_lo=300, K_hi=3000, N_lo=5, N_hi=40)
    trip = []
    for i, it in enumerate(items):
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
        case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
        mode = i % 5  # separate pass, fused, regenerated, kept in shared memory, drawn ahead
        g1 = M.Controller(case.mc, case.sc, case.tr, noise_gen=mode)
        g2 = M.Controller(case.mc, case.sc, case.tr, noise_gen=mode)
        trip.append((g1, g2, case))
    X0 = np.array([c.x0 for _, _, c in trip])
    t0 = np.full(len(trip), 0.3)
    b = M.mppi_batch_create([g1.h for g1, _, _ in trip], use_graph=use_graph)
    for rep in range(2):
        ub, _ = M.mppi_batch_solve(b, len(trip), X0, t0)
        for i, (g1, g2, c) in enumerate(trip):
            ua, _ = g2.solve(c.x0, 0.3)
            np.testing.assert_array_equal(ub[i], ua)
            _same(g1, g2)
    M.mppi_batch_destroy(b)
    for g1, g2, _ in trip:
        g1.close()
        g2.close()


def test_server_with_fused_noise(M):
    fleet = W.c5_fleet(n_drones=6, distinct_tracks=4)
    srv = M.Server(len(fleet), 1 << 30, n_slots=2, max_batch=4)
    alone = []
    for i, d in enumerate(fleet):
        sc = W.SolveConfig(objective=d.objective, K=1024, N=30, dt=0.02, drone_id=d.drone_id)
        mode = i % 3
        srv.add_drone(W.ModelConfig(), sc, d.track, 2048, 30, noise_gen=mode)
        alone.append(M.Controller(W.ModelConfig(), sc, d.track, K_cap=2048, N_cap=30, noise_gen=mode))
    X0 = np.array([d.x0 for d in fleet])
    n = len(fleet)
    for rnd in range(2):
        ids = srv.submit(np.arange(n), X0, np.full(n, 0.1 * rnd), np.full(n, 2048), np.full(n, 30))
        got = {}
        while len(got) < n:
            while srv.step() > 0:
                pass
            for r in srv.poll().tolist():
                got[int(r[0])] = r
        for i, c in enumerate(alone):
            c.set_shape(2048, 30)
            u, _ = c.solve(X0[i], 0.1 * rnd)
            np.testing.assert_array_equal(np.asarray(got[int(ids[i])][5], np.float32), u)
    for i, c in enumerate(alone):
        assert srv.export_drone(i) == c.export_state()
        c.close()
    srv.close()


def test_caller_noise_on_a_fused_handle(M):
    """mppi_set_noise on a fused handle: that solve uses the caller's normals
    (the rollout loads them, as the separate path does), the next one draws
    its own again."""
    case = _case(0, 2048, 40)
    rng = np.random.default_rng(5)
    z = torch.tensor(rng.standard_normal((40, 2048, 4)).astype(np.float32), device="cuda").contiguous()
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_FUSED)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL)
    for c in (a, b):
        M.mppi_set_noise(c.h, z.data_ptr(), None)
    for rep in range(2):
        ua, _ = a.solve(case.x0, 0.0)
        ub, _ = b.solve(case.x0, 0.0)
        if rep == 0:
            # both ran the loading kernel on the same normals
            np.testing.assert_array_equal(ua, ub)
            np.testing.assert_array_equal(a.costs(), b.costs())
            np.testing.assert_array_equal(a.noise()[:, :, :4], z.cpu().numpy())
        else:
            assert np.abs(ua - ub).max() <= U_ABS_TOL
            _close(a, b)
    a.close()
    b.close()


def test_regenerated_noise_has_no_buffer(M):
    """REGEN stores no noise: the handle is smaller by the noise buffer, the
    noise getters refuse, and bfloat16 storage is refused at creation."""
    case = _case(1, 4096, 50)
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_REGEN)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL)
    saved = M.mppi_device_bytes(b.h) - M.mppi_device_bytes(a.h)
    # 16 B + the 5th plane's 4 B per rollout step, less two 256-B placeholders
    assert saved >= 4096 * 50 * 20 - 512
    with pytest.raises(M.MppiError) as e:
        a.noise()
    assert e.value.code == M.MPPI_ERR_ARG
    z = torch.zeros((50, 4096, 4), device="cuda")
    with pytest.raises(M.MppiError):
        M.mppi_set_noise(a.h, z.data_ptr(), z.data_ptr())
    with pytest.raises(M.MppiError) as e:
        M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_REGEN, noise_dtype=M.NOISE_BF16)
    assert e.value.code == M.MPPI_ERR_ARG
    a.close()
    b.close()


def test_noise_kept_in_shared_memory(M):
    """MPPI_NOISEGEN_SMEM needs no noise buffer and refuses the noise getters;
    a horizon whose normals do not fit a block's shared memory is refused at
    creation."""
    case = _case(0, 2048, 20)
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_SMEM)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL)
    assert M.mppi_device_bytes(b.h) - M.mppi_device_bytes(a.h) >= 2048 * 20 * 16 - 512
    with pytest.raises(M.MppiError) as e:
        a.noise()
    assert e.value.code == M.MPPI_ERR_ARG
    big = _case(1, 2048, 128)
    with pytest.raises(M.MppiError) as e:
        M.Controller(big.mc, big.sc, big.tr, noise_gen=M.NOISEGEN_SMEM)
    assert e.value.code == M.MPPI_ERR_ARG
    a.close()
    b.close()


def _equal_solves(a, b, x0, t0):
    ua, _ = a.solve(x0, t0)
    ub, _ = b.solve(x0, t0)
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(a.costs(), b.costs())
    np.testing.assert_array_equal(a.unew(), b.unew())
    np.testing.assert_array_equal(a.nominal(), b.nominal())
    assert a.export_state() == b.export_state()


@pytest.mark.parametrize("objective", [0, 1, 2])
@pytest.mark.parametrize("bf16", [0, 1])
def test_noise_drawn_ahead_equals_separate(O, M, objective, bf16):
    """MPPI_NOISEGEN_AHEAD draws the next solve's normals after each solve.
    Every result is the separate pass's, bit for bit, over consecutive
    solves, a change of shape, caller noise for one solve and an imported
    state; after a solve the buffer holds the normals the next solve uses."""
    case = _case(objective, 3001, 20)
    kw = dict(noise_dtype=bf16, block=128, K_cap=4096, N_cap=30)
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_AHEAD, **kw)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL, **kw)
    t0 = 0.37
    x0 = _x0(O, case, t0)
    ahead = None
    for rep in range(3):
        _equal_solves(a, b, x0, t0 + 0.02 * rep)
        if ahead is not None:
            # what a drew after its previous solve is what b drew for this one
            np.testing.assert_array_equal(ahead, b.noise())
        ahead = a.noise()
    # a change of shape: the next solve draws first
    for c in (a, b):
        c.set_shape(4096, 30)
    _equal_solves(a, b, x0, t0 + 0.1)
    if not bf16:
        # caller noise for one solve, then the draws resume
        rng = np.random.default_rng(11)
        z = torch.tensor(rng.standard_normal((30, 4096, 4)).astype(np.float32), device="cuda").contiguous()
        z5 = torch.tensor(rng.standard_normal((30, 4096)).astype(np.float32), device="cuda").contiguous()
        for c in (a, b):
            M.mppi_set_noise(c.h, z.data_ptr(), z5.data_ptr() if objective == 1 else None)
        _equal_solves(a, b, x0, t0 + 0.12)
        _equal_solves(a, b, x0, t0 + 0.14)
    # an imported state moves the iteration counter: the next solve draws first
    b.solve(x0, t0 + 0.16)
    a.import_state(b.export_state())
    _equal_solves(a, b, x0, t0 + 0.18)
    _equal_solves(a, b, x0, t0 + 0.2)
    a.close()
    b.close()


def test_noise_drawn_ahead_is_for_single_solves(M):
    """The server refuses MPPI_NOISEGEN_AHEAD; a batch draws the normals of
    such a handle itself, and the next single solve draws first again (the
    batch moved the counter)."""
    fleet = W.c5_fleet(n_drones=2, distinct_tracks=2)
    srv = M.Server(len(fleet), 1 << 28, n_slots=1, max_batch=2)
    d = fleet[0]
    sc = W.SolveConfig(objective=d.objective, K=1024, N=20, dt=0.02, drone_id=d.drone_id)
    with pytest.raises(M.MppiError) as e:
        srv.add_drone(W.ModelConfig(), sc, d.track, 1024, 20, noise_gen=M.NOISEGEN_AHEAD)
    assert e.value.code == M.MPPI_ERR_ARG
    srv.close()
    case = _case(0, 2048, 20)
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_AHEAD)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL)
    _equal_solves(a, b, case.x0, 0.0)
    plan_a = M.mppi_batch_create([a.h], use_graph=0)
    plan_b = M.mppi_batch_create([b.h], use_graph=0)
    X0 = np.array([case.x0])
    ua, _ = M.mppi_batch_solve(plan_a, 1, X0, np.zeros(1))
    ub, _ = M.mppi_batch_solve(plan_b, 1, X0, np.zeros(1))
    np.testing.assert_array_equal(ua, ub)
    M.mppi_batch_destroy(plan_a)
    M.mppi_batch_destroy(plan_b)
    _equal_solves(a, b, case.x0, 0.02)
    a.close()
    b.close()


def test_noise_drawn_ahead_across_streams(O, M):
    """A noise-ahead handle whose solves move between streams, then into a
    batch on a third: each call waits for the draw the previous one left
    running, so every result is the separate pass's, bit for bit."""
    case = _case(1, 3001, 20)  # contouring: the 5th normals too
    a = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_AHEAD)
    b = M.Controller(case.mc, case.sc, case.tr, noise_gen=M.NOISEGEN_KERNEL)
    streams = [torch.cuda.Stream() for _ in range(3)]
    x0 = case.x0
    for rep in range(4):
        ua, _ = a.solve(x0, 0.02 * rep, stream=streams[rep % 2])
        ub, _ = b.solve(x0, 0.02 * rep)
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(a.unew(), b.unew())
    plan_a = M.mppi_batch_create([a.h], use_graph=1)
    plan_b = M.mppi_batch_create([b.h], use_graph=1)
    ua, _ = M.mppi_batch_solve(plan_a, 1, np.array([x0]), np.full(1, 0.1), stream=streams[2])
    ub, _ = M.mppi_batch_solve(plan_b, 1, np.array([x0]), np.full(1, 0.1))
    np.testing.assert_array_equal(ua, ub)
    torch.cuda.synchronize()
    assert a.export_state() == b.export_state()
    M.mppi_batch_destroy(plan_a)
    M.mppi_batch_destroy(plan_b)
    a.close()
    b.close()
