"""The autotuner times the real entry points and caches its choice."""
import json

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_tune_single_picks_a_measured_block_and_caches_it(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2509_14726_gb300 import autotune as AT
    mc, sc, tr, x0 = W.c1_single_gate()
    cache = AT.Cache(str(tmp_path / "tune.json"))
    out = AT.tune_single(mc, sc, tr, blocks=(32, 128), cache=cache, x0=x0)
    assert out["block"] in (32, 128) and out["noise_gen"] in (0, 1, 2)
    # blocks x noise generation forms
    assert len(out["table"]) == 6 and all(r["ms"] > 0 for r in out["table"])
    assert {(r["block"], r["noise_gen"]) for r in out["table"]} == {(b, g) for b in (32, 128) for g in (0, 1, 2)}
    assert out["ms"] == min(r["ms"] for r in out["table"])
    saved = json.load(open(tmp_path / "tune.json"))
    assert AT.bucket_key(sc.objective, sc.K, sc.N) in saved
    again = AT.tune_single(mc, sc, tr, blocks=(32, 128), cache=AT.Cache(str(tmp_path / "tune.json")))
    assert again["block"] == out["block"]


def test_tune_batch_searches_samples_per_thread():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2509_14726_gb300 import autotune as AT, mppi as M, workloads as W
    items = W.c3_batch(n_drones=4, K_lo=500, K_hi=2000, N_lo=10, N_hi=20)
    X0 = np.array([it.x0 for it in items])

    def make_handles(block, noise_gen=None, spt=1):
        return [M.Controller(W.ModelConfig(), W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02,
                                                            drone_id=it.drone_id), it.track, block=block,
                             noise_gen=noise_gen, spt=spt) for it in items]

    out = AT.tune_batch(make_handles, X0, 0.3, blocks=(64, 128), modes=(1,), spts=(1, 2, 4),
                        noise_gens=(M.NOISEGEN_KERNEL,))
    spts = sorted(r["spt"] for r in out["table"])
    assert spts == [1, 1, 2, 2, 4, 4]  # (2 blocks at spt 1) + each block at spt 2 and 4
    best = min(out["table"], key=lambda r: r["ms"])
    assert (out["block"], out["spt"], out["ms"]) == (best["block"], best["spt"], best["ms"])
