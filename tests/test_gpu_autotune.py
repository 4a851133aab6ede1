"""The autotuner times the real entry points and caches its choice."""
import json

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
