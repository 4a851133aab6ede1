"""The device-side batched solve (mppi_batch_solve_async) against the host
entry point (mppi_batch_solve).

With a graph plan, the async form captures one graph per set of caller
buffers (x0, t0, u0) and launches it with no copies; a plan keeps four such
graphs and sends calls with further buffer sets through its own buffers.
Every form runs the same kernels on the same inputs, so each call must give
the host path's u0 bit for bit, and both plans' handles must end in the same
state.  Covered: the three plan forms, alternating buffer sets, a fifth set
(the copy path) and buffers that are reused after other sets ran.
"""
import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W
from parity_util import f32_case

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


@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_async_buffer_sets_equal_host_path(M, use_graph):
    items = W.c3_batch(n_drones=7, K_lo=300, K_hi=2500, N_lo=5, N_hi=40)
    a_ctl, h_ctl = [], []
    for it in items:
        sc = W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, drone_id=it.drone_id)
        case = f32_case(W.ModelConfig(), sc, it.track, it.x0)
        a_ctl.append(M.Controller(case.mc, case.sc, case.tr))
        h_ctl.append(M.Controller(case.mc, case.sc, case.tr))
    n = len(items)
    X0 = np.float32([it.x0 for it in items])
    pa = M.mppi_batch_create([c.h for c in a_ctl], use_graph=use_graph)
    ph = M.mppi_batch_create([c.h for c in h_ctl], use_graph=use_graph)
    # six buffer sets: the plan keeps graphs for four, the rest take the copy path
    sets = []
    for _ in range(6):
        sets.append((torch.tensor(X0, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda"),
                     torch.zeros((n, 5), dtype=torch.float32, device="cuda")))
    order = [0, 1, 0, 2, 3, 4, 5, 1, 4, 0]
    s = torch.cuda.Stream()
    rng = np.random.default_rng(3)
    for call, p in enumerate(order):
        x0 = X0 + np.float32(rng.normal(0, 0.05, X0.shape)) * np.float32([1] * 3 + [0] * 10)
        t0 = np.full(n, 0.3 + 0.02 * call)
        dx, dt, du = sets[p]
        dx.copy_(torch.from_numpy(x0))
        dt.copy_(torch.from_numpy(t0))
        with torch.cuda.stream(s):
            M.mppi_batch_solve_async(pa, dx.data_ptr(), dt.data_ptr(), s, du.data_ptr())
        s.synchronize()
        uh, _ = M.mppi_batch_solve(ph, n, x0, t0)
        np.testing.assert_array_equal(du.cpu().numpy(), np.asarray(uh, np.float32), err_msg=f"call {call} set {p}")
    for ca, ch in zip(a_ctl, h_ctl):
        assert ca.export_state() == ch.export_state()
        np.testing.assert_array_equal(ca.nominal(), ch.nominal())
    M.mppi_batch_destroy(pa)
    M.mppi_batch_destroy(ph)
    for c in a_ctl + h_ctl:
        c.close()
