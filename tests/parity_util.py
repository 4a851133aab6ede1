"""Shared helpers of the GPU parity tests.

The oracle always receives the binary32-rounded inputs that the CUDA path
receives (model, parameters, track tables, x0), so both sides solve the same
problem; the CUDA path's results never flow into the oracle.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from paper_2509_14726_gb300 import workloads as W

# tolerances stated for this path: per-sample cost relative error, absolute
# error of the nominal control (N or rad/s)
J_REL_TOL = 1e-4
U_ABS_TOL = 1e-5
# Binary32 rollouts carry a per-sample cost error; it reaches the nominal
# through the weights (Eq. 4): dU_kj = (1/lambda) sum_m w_m (dJbar - dJ_m)
# (u_mkj - U_kj), so |dU_kj| <= 2 DJ32 sens_kj with sens_kj the oracle's
# (1/lambda) sum_m w_m |u_mkj - U_kj|.  DJ32 is the binary32 cost error of a
# sample: trajectory error floor 2.5e-7 m rms / 6.5e-7 m max over 50 RK4
# steps times the cost gradient (2 |p - target| q, about 10 for these
# weights) -> 2.5e-6 .. 6.5e-6; measured on significantly weighted samples
# up to 5e-6.  Where sens_kj < 1 this leaves U_ABS_TOL.
DJ32 = 5e-6


@dataclasses.dataclass
class Case:
    mc: W.ModelConfig
    sc: W.SolveConfig
    tr: W.Track
    x0: np.ndarray


def f32_case(mc, sc, tr, x0) -> Case:
    return Case(W.f32_model(mc), W.f32_solve(sc), tr.as_f32(), np.float32(x0).astype(np.float64))


def make_pair(case: Case, **gpu_kw):
    from oracle import oracle as O
    from paper_2509_14726_gb300 import mppi
    gpu = mppi.Controller(case.mc, case.sc, case.tr, **gpu_kw)
    ora = O.OracleController(case.mc, case.sc, case.tr, cap=max(case.sc.N, gpu_kw.get("N_cap", 0) or 0))
    return gpu, ora


def push_oracle_state(gpu, ora) -> None:
    """Starts the GPU handle from the oracle's current controller state
    (binary32-rounded): oracle -> CUDA only."""
    from paper_2509_14726_gb300 import mppi
    st = ora.st
    N_cap = gpu.params.N_cap or gpu.params.N
    nu = 5 if gpu.sc.objective == 1 else 4
    prev = ora.prevcnt[: st.n_prev].copy() if st.n_prev else None
    rotor = gpu.mc.kind == 1
    hover_row = [0.0 if rotor else gpu.mc.mass * gpu.mc.gravity, 0, 0, 0, 0]
    U = ora.U[: st.n_nom] if st.n_nom else np.tile(hover_row, (1, 1))
    blob = mppi.encode_state(N_cap, nu, U, iter=st.iter, gate=st.gate, prevcnt=prev,
                             prev_x0=np.array(st.prev_x0[:]) if st.has_prev else None, theta=st.theta,
                             v_theta=st.v_theta, c_last=st.c_last, has_theta=st.has_theta,
                             n_nom=st.n_nom, rotor=ora.rotor if rotor else None)
    gpu.import_state(blob)


def compare(gpu, r: dict, label: str = "", j_tol: float = J_REL_TOL, u_tol: float = U_ABS_TOL,
            check_decisions: bool = True, measured_cost_bound: bool = False) -> dict:
    """Element-wise comparison of one solve; returns the statistics and
    asserts the tolerances (samples the oracle flags as within 1e-5 m of a
    gate plane, opening edge or near-gate sphere are counted and excluded).

    measured_cost_bound: the nominal tolerance takes the largest absolute
    cost error of the weighted, unflagged samples in place of DJ32 when that
    is larger (long horizons and large costs carry a larger absolute binary32
    cost error; their relative error is still held to j_tol)."""
    K = gpu.K
    nu = 5 if gpu.sc.objective == 1 else 4
    J = gpu.costs()
    flag = r["near_flag"] != 0
    ok = ~flag
    denom = np.maximum(np.abs(r["J"]), r["Jabs"])
    rel = np.abs(J - r["J"]) / np.where(denom > 0, denom, 1.0)
    stats = {"K": K, "flagged": int(flag.sum()), "max_rel_J": float(rel[ok].max()) if ok.any() else 0.0}
    npass, first = gpu.sample_info()
    if gpu.sc.objective == 0:
        mism = (npass != r["npass"]) | (first != r["first_pass"])
        stats["decision_mismatch_unflagged"] = int((mism & ok).sum())
        stats["decision_mismatch_flagged"] = int((mism & flag).sum())
    Unew = gpu.unew()
    dU = np.abs(Unew[:, :nu] - r["Unew"][:, :nu])
    dj = DJ32
    if measured_cost_bound:
        wsig = ok & (r["w"] > 1e-8)
        if wsig.any():
            dj = max(DJ32, float(np.max(np.abs(J - r["J"])[wsig])))
        stats["cost_error_bound"] = dj
    tolU = np.maximum(u_tol, 2.0 * dj * r["sens"][:, :nu])
    stats["max_dU"] = float(dU.max())
    stats["max_du0"] = float(dU[0].max())
    stats["max_dU_over_tol"] = float((dU / tolU).max())
    stats["well_conditioned_share"] = float(np.mean(tolU == u_tol))
    # the weight mass on samples whose decision differs (if any) explains a dU excess
    assert stats["max_rel_J"] <= j_tol, f"{label} J rel err {stats}"
    if gpu.sc.objective == 0 and check_decisions:
        assert stats["decision_mismatch_unflagged"] == 0, f"{label} gate decisions differ {stats}"
    assert stats["max_dU_over_tol"] <= 1.0, f"{label} nominal differs {stats}"
    return stats
