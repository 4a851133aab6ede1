"""Serving (continuous batching) gives each drone the result it gets alone.

Requests from several drones with different objectives, K and N go through
one mppi_server (batched, overlapping slots, scratch from a shared pool); the
same request sequence per drone goes through its own handle (mppi_solve).  u0
and the resident controller state must be identical: the server runs the same
kernels with the same per-solve reduction order.
"""
import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W

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


def _fleet(n):
    return W.c5_fleet(n_drones=n, distinct_tracks=4)


def _drain(srv, n_expected, timeout_s=60.0):
    import time
    got = []
    t0 = time.time()
    while len(got) < n_expected and time.time() - t0 < timeout_s:
        while srv.step() > 0:
            pass
        got.extend(srv.poll().tolist())
    return got


def test_served_results_equal_alone(M):
    fleet = _fleet(6)
    K_cap, N_cap = 4096, 40
    srv = M.Server(len(fleet), 1 << 30, n_slots=2, max_batch=4)
    alone = []
    for d in fleet:
        sc = W.SolveConfig(objective=d.objective, K=1024, N=30, dt=0.02, drone_id=d.drone_id)
        srv.add_drone(W.ModelConfig(), sc, d.track, K_cap, N_cap)
        alone.append(M.Controller(W.ModelConfig(), sc, d.track, K_cap=K_cap, N_cap=N_cap))
    rng = np.random.default_rng(4)
    X0 = np.array([d.x0 for d in fleet])
    for rnd in range(3):
        Ks = rng.choice([300, 1024, 4096], len(fleet)).astype(np.int32)
        Ns = rng.choice([12, 30, 40], len(fleet)).astype(np.int32)
        t0 = np.full(len(fleet), 0.1 * rnd)
        ids = srv.submit(np.arange(len(fleet)), X0, t0, Ks, Ns)
        res = _drain(srv, len(fleet))
        assert len(res) == len(fleet)
        by_id = {int(r[0]): r for r in res}
        for i, c in enumerate(alone):
            c.set_shape(int(Ks[i]), int(Ns[i]))
            u, _ = c.solve(X0[i], float(t0[i]))
            r = by_id[int(ids[i])]
            np.testing.assert_array_equal(np.asarray(r[5], np.float32), u)
            assert r[2] == 0
    for i, c in enumerate(alone):
        assert srv.export_drone(i) == c.export_state()
        c.close()
    st = srv.stats()
    assert st["batches"] >= 6 and st["finished"] == 3 * len(fleet) and st["scratch_used"] == 0
    srv.close()


def test_admission_waits_for_scratch_and_refuses_oversize(M):
    fleet = _fleet(8)
    # one request of K=4096, N=40 needs ~2.7 MB of scratch: a 6 MB pool holds two
    srv = M.Server(len(fleet), 6 << 20, n_slots=4, max_batch=8)
    for d in fleet:
        sc = W.SolveConfig(objective=0, K=1024, N=30, dt=0.02, drone_id=d.drone_id)
        srv.add_drone(W.ModelConfig(), sc, d.track, 4096, 40)
    X0 = np.array([d.x0 for d in fleet])
    n = len(fleet)
    srv.submit(np.arange(n), X0, np.zeros(n), np.full(n, 4096), np.full(n, 40))
    res = _drain(srv, n)
    assert len(res) == n and all(r[2] == 0 for r in res)
    st = srv.stats()
    assert st["scratch_peak"] <= st["pool"] and st["batches"] >= n // 2
    with pytest.raises(M.MppiError) as e:
        srv.submit([0], X0[:1], [0.0], [4096], [41])  # beyond the drone's N cap
    assert e.value.code == M.MPPI_ERR_NOT_ADMITTED
    srv.close()
    small = M.Server(1, 1 << 20, n_slots=1, max_batch=1)
    sc = W.SolveConfig(objective=0, K=1024, N=30, dt=0.02)
    small.add_drone(W.ModelConfig(), sc, fleet[0].track, 4096, 40)
    with pytest.raises(M.MppiError) as e:
        small.submit([0], X0[:1], [0.0], [4096], [40])  # needs more than the whole pool
    assert e.value.code == M.MPPI_ERR_NOT_ADMITTED
    small.close()


def test_serving_loop_runs_a_fleet(M):
    from paper_2509_14726_gb300 import serving
    fleet = _fleet(40)
    sched = serving.make_schedule(fleet, duration_s=0.5, time_scale=1.0, K_choices=[1024, 4096],
                                  N_choices=[30, 50], seed=1)
    out = serving.run_served(fleet, sched, budget_bytes=2 << 30, n_slots=3, max_batch=256, K_cap=4096, N_cap=50)
    assert out["finished"] == out["offered"]
    assert out["p99_ms"] < 1000.0


def test_failed_launch_hands_the_batch_back(M):
    """A batch whose launch fails (injected on the host, before any transfer
    or launch) returns its requests to the queue: the step reports
    MPPI_ERR_CUDA, no scratch stays in use, no drone stays busy, and the next
    steps serve every request with the result it gets alone."""
    fleet = _fleet(4)
    srv = M.Server(len(fleet), 1 << 30, n_slots=2, max_batch=8)
    alone = []
    for d in fleet:
        sc = W.SolveConfig(objective=d.objective, K=1024, N=20, dt=0.02, drone_id=d.drone_id)
        srv.add_drone(W.ModelConfig(), sc, d.track, 2048, 30)
        alone.append(M.Controller(W.ModelConfig(), sc, d.track, K_cap=2048, N_cap=30))
    X0 = np.array([d.x0 for d in fleet])
    n = len(fleet)
    ids = srv.submit(np.arange(n), X0, np.zeros(n), np.full(n, 1024), np.full(n, 20))
    srv.fail_next_launch()
    with pytest.raises(M.MppiError) as e:
        srv.step()
    assert e.value.code == M.MPPI_ERR_CUDA
    st = srv.stats()
    assert st["queued"] == n and st["in_flight"] == 0 and st["scratch_used"] == 0
    res = _drain(srv, n)
    assert len(res) == n
    by_id = {int(r[0]): r for r in res}
    for i, c in enumerate(alone):
        u, _ = c.solve(X0[i], 0.0)
        np.testing.assert_array_equal(np.asarray(by_id[int(ids[i])][5], np.float32), u)
        c.close()
    srv.close()

