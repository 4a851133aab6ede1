"""The allocation-free solve gives the handle API's result.

mppi_solve_noalloc exists for callers that may not allocate device memory
while they run (a control loop that allocates only at start-up, a process
whose GPU memory belongs to another allocator, a loop that cannot absorb the
synchronisation an allocation may bring).  It keeps its scratch in the
library's static device array.  This test runs two solves in a row through it
and through a handle (mppi_create + mppi_solve_async) with the same inputs and
checks that u0 and the weighted nominal agree within the parity tolerance.
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U_TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    from paper_2509_14726_gb300 import mppi
    return mppi


def _device_track(M, tr):
    gates = torch.tensor(np.float32(tr.gates), device="cuda").contiguous()
    path = torch.tensor(np.float32(tr.path), device="cuda").contiguous()
    ref = torch.tensor(np.float32(tr.ref), device="cuda").contiguous()
    t = M.TrackC()
    t.n_gates, t.closed = gates.shape[0], int(bool(tr.closed))
    t.gates = C.cast(C.c_void_p(gates.data_ptr()), M.PF)
    t.S, t.L, t.path = path.shape[0], float(tr.L), C.cast(C.c_void_p(path.data_ptr()), M.PF)
    t.T, t.dt_ref, t.ref = ref.shape[0], float(tr.dt_ref), C.cast(C.c_void_p(ref.data_ptr()), M.PF)
    return t, (gates, path, ref)


@pytest.mark.parametrize("noise", ["f32", "bf16"])
@pytest.mark.parametrize("objective", [W.OBJ_GATE, W.OBJ_CONTOUR, W.OBJ_TRACK])
def test_noalloc_matches_the_handle_path_twice(M, objective, noise):
    """Two calls in a row (the second warm-started from the first's result)
    against a handle put in the same state before each of its solves: the
    nominal, the Philox iteration and no other history (the allocation-free
    call is stateless).  Each objective, with float32 and bfloat16 noise
    storage, on one stream."""
    mc, sc, tr, x0 = W.c2_full_scale(objective)
    sc.K, sc.N = 2048, 40
    sc.temporal_rule = 0  # stateless call: no pass counts of a previous nominal
    mc, sc, tr = W.f32_model(mc), W.f32_solve(sc), tr.as_f32()
    t0 = 0.3
    if objective == W.OBJ_TRACK:
        x0 = tr.ref[int(round(t0 / tr.dt_ref)) % tr.ref.shape[0]].copy()
    nu = 5 if objective == W.OBJ_CONTOUR else 4
    ctl = M.Controller(mc, sc, tr, noise_dtype=M.NOISE_BF16 if noise == "bf16" else M.NOISE_F32)
    d_track, keep = _device_track(M, tr)
    stream = torch.cuda.Stream()
    d_x0 = torch.tensor(np.float32(x0), device="cuda")
    d_u0_h = torch.zeros(5, dtype=torch.float32, device="cuda")
    d_u0_s = torch.zeros(5, dtype=torch.float32, device="cuda")
    U = np.zeros((sc.N, 5), np.float32)
    U[:, 0] = np.float32(mc.mass) * np.float32(mc.gravity)
    d_Unew = torch.zeros((sc.N, 5), dtype=torch.float32, device="cuda")
    free_before_second = None
    for call in range(2):
        d_U = torch.tensor(U, device="cuda")
        ctl.import_state(M.encode_state(sc.N, nu, U, iter=call, n_nom=sc.N if call else 0))
        with torch.cuda.stream(stream):
            M.mppi_solve_async(ctl.h, d_x0.data_ptr(), t0, stream, d_u0_h.data_ptr())
            if call == 1:
                torch.cuda.synchronize()
                free_before_second = torch.cuda.mem_get_info()[0]
            M.mppi_solve_noalloc(ctl.model, ctl.params, d_track, d_x0.data_ptr(), t0, d_U.data_ptr(), call, 0,
                                 stream, d_Unew.data_ptr(), d_u0_s.data_ptr())
        stream.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before_second
        u_h = d_u0_h.cpu().numpy()
        u_s = d_u0_s.cpu().numpy()
        U_h = ctl.unew()
        U_s = d_Unew.cpu().numpy()
        assert np.max(np.abs(u_s[:nu] - u_h[:nu])) <= U_TOL, (call, u_s, u_h)
        assert np.max(np.abs(U_s[:, :nu] - U_h[:, :nu])) <= U_TOL, call
        # warm start for the next call: shift by one row, repeat the last
        U = np.vstack([U_s[1:], U_s[-1:]]).astype(np.float32)
    ctl.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(M):
    mc, sc, tr, x0 = W.c4_precision()
    p = M.make_params(sc)
    d_track, keep = _device_track(M, tr)
    dummy = torch.zeros(1024, dtype=torch.float32, device="cuda")
    rc = M.load().mppi_solve_noalloc(C.byref(M.make_model(mc)), C.byref(p), C.byref(d_track),
                                     C.c_void_p(dummy.data_ptr()), 0.0, C.c_void_p(dummy.data_ptr()), 0, 0, None,
                                     C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()))
    assert rc == M.MPPI_ERR_ARG
    assert b"static maximum" in M.load().mppi_last_error()


def test_noalloc_refuses_noise_drawn_ahead(M):
    """MPPI_NOISEGEN_AHEAD draws for a handle's next solve; a call that keeps
    nothing between calls refuses it before touching any buffer."""
    mc, sc, tr, x0 = W.c4_precision()
    sc.K, sc.N = 1024, 20
    p = M.make_params(sc, noise_gen=M.NOISEGEN_AHEAD)
    d_track, keep = _device_track(M, tr)
    dummy = torch.zeros(1024, dtype=torch.float32, device="cuda")
    rc = M.load().mppi_solve_noalloc(C.byref(M.make_model(mc)), C.byref(p), C.byref(d_track),
                                     C.c_void_p(dummy.data_ptr()), 0.0, C.c_void_p(dummy.data_ptr()), 0, 0, None,
                                     C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()))
    assert rc == M.MPPI_ERR_ARG
    assert b"noise drawn ahead" in M.load().mppi_last_error()


def test_noalloc_fused_noise_equals_separate_pass(M):
    """Noise drawn inside the rollout (stored, or drawn again by the update)
    gives the two-kernel result to binary32 rounding (the draws are
    bit-identical; the rollout is another compilation)."""
    mc, sc, tr, x0 = W.c2_full_scale(W.OBJ_CONTOUR)
    sc.K, sc.N = 3000, 40
    mc, sc, tr = W.f32_model(mc), W.f32_solve(sc), tr.as_f32()
    d_track, keep = _device_track(M, tr)
    model = M.make_model(mc)
    d_x0 = torch.tensor(np.float32(x0), device="cuda")
    d_U = torch.zeros((sc.N, 5), dtype=torch.float32, device="cuda")
    d_U[:, 0] = float(np.float32(mc.mass) * np.float32(mc.gravity))
    out = []
    for mode in (M.NOISEGEN_KERNEL, M.NOISEGEN_FUSED, M.NOISEGEN_REGEN):
        p = M.make_params(sc, noise_gen=mode)
        d_Unew = torch.zeros((sc.N, 5), dtype=torch.float32, device="cuda")
        d_u0 = torch.zeros(5, dtype=torch.float32, device="cuda")
        M.mppi_solve_noalloc(model, p, d_track, d_x0.data_ptr(), 0.0, d_U.data_ptr(), 3, 0, None,
                             d_Unew.data_ptr(), d_u0.data_ptr())
        torch.cuda.synchronize()
        out.append((d_u0.cpu().numpy(), d_Unew.cpu().numpy()))
    for other in out[1:]:
        assert np.max(np.abs(out[0][0] - other[0])) <= U_TOL
        assert np.max(np.abs(out[0][1] - other[1])) <= U_TOL
