"""Precision study on the large single solve: K=65536, N=100, dt=0.01, gate
progress on the seeded 7-gate course.

Variants of the CUDA path against the FP64 oracle on the same inputs:
  (a) all-fp32: float32 noise, plain float32 weighted sums;
  (b) bfloat16-stored noise, float32 rollout, float64 weighted sums -- the
      noise is a seeded input (bfloat16 values drawn by the input generator)
      given to both sides, so parity is exact in the inputs;
  (c) float32 with compensated (Kahan / TwoSum) weighted sums (the default).
Each reports max |dU|, max |du0|, the largest per-sample cost relative error,
the samples the oracle flags near a gate plane / edge / sphere and gate
decision mismatches.  (b) also reports how far bfloat16 storage moves the
result from full-precision noise (not a parity bound: a precision cost).
"""
import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W
from parity_util import compare, f32_case, make_pair

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
    mc, sc, tr, x0 = W.c4_precision()
    case = f32_case(mc, sc, tr, x0)
    ora = O.OracleController(case.mc, case.sc, case.tr)
    ref = ora.solve(case.x0, 0.0)
    return O, M, case, ref


@pytest.mark.parametrize("accum,label", [(2, "a: all fp32"), (0, "c: fp32 + Kahan")])
def test_c4_float32_variants(env, accum, label):
    O, M, case, ref = env
    gpu, _ = make_pair(case, accum=accum)
    gpu.solve(case.x0, 0.0)
    st = compare(gpu, ref, label)
    print(f"\nC4 {label}: {st}")
    gpu.close()


def test_c4_bf16_noise_fp64_sums(env):
    O, M, case, ref = env
    K, N = case.sc.K, case.sc.N
    rng = np.random.default_rng(2026)
    z = rng.standard_normal((N, K, 4)).astype(np.float32)
    zb = torch.tensor(z).to(torch.bfloat16)
    z_dec = zb.float().numpy().astype(np.float64)
    gpu, _ = make_pair(case, noise_dtype=M.NOISE_BF16, accum=M.ACC_F64)
    dz = zb.cuda().contiguous()
    M.mppi_set_noise(gpu.h, dz.data_ptr(), None)
    gpu.solve(case.x0, 0.0)
    ora = O.OracleController(case.mc, case.sc, case.tr)
    Zin = np.zeros((N, K, 5))
    Zin[:, :, :4] = z_dec
    r = ora.solve(case.x0, 0.0, Z_in=Zin)
    st = compare(gpu, r, "b: bf16 noise + fp64 sums")
    # precision cost of bfloat16 storage: the same draws at full precision
    ora2 = O.OracleController(case.mc, case.sc, case.tr)
    Zf = np.zeros((N, K, 5))
    Zf[:, :, :4] = z.astype(np.float64)
    r2 = ora2.solve(case.x0, 0.0, Z_in=Zf)
    st["bf16_vs_full_noise_max_dU"] = float(np.max(np.abs(r["Unew"][:, :4] - r2["Unew"][:, :4])))
    print(f"\nC4 b: bf16 noise + fp64 sums: {st}")
    gpu.close()
