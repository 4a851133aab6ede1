"""Conditioning of a solve's nominal, from FP64 oracle outputs only.

TEST INFRASTRUCTURE ONLY (the tests and the bench's CPU-baseline leg use it;
the product path never does).  The nominal of Eq. 5 depends on the costs
through the exponential weights of Eq. 4, which can amplify a cost error by
orders of magnitude where a few samples share the weight.  binary32_floor
measures that amplification on the oracle's own samples: each FP64 cost J_m
moves by one binary32 unit roundoff of its term magnitude (u * J_abs_m, u =
2^-24, random signs from a fixed seed), Eq. 4 and Eq. 5 are evaluated again,
and the largest change of the nominal is returned.  A binary32 rollout
carries at least that much cost error, so a solve whose floor is a sizeable
fraction of the 1e-5 nominal bound cannot be held to that bound in binary32.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

U32 = 2.0 ** -24


def eq45(J: np.ndarray, Us: np.ndarray, lam: float) -> np.ndarray:
    """Eq. 4 (weights exp(-(J - J_min) / lambda), normalised) and Eq. 5 (the
    weighted sum of the clamped sequences Us [K][N][nu]) in FP64."""
    w = np.exp(-(J - np.min(J)) / lam)
    w /= w.sum()
    return np.einsum("m,mkj->kj", w, Us)


def binary32_floor(r: dict, lam: float, nu: int, seeds: int = 8) -> Optional[float]:
    """Largest change of the oracle's nominal when each cost moves by one
    binary32 unit roundoff of its term magnitude.  r: an oracle solve with
    "Us" (OracleController.solve exports it for K N <= 4e6).  None when the
    solve has no samples exported or a non-finite cost."""
    if "Us" not in r or not np.all(np.isfinite(r["J"])):
        return None
    Us = r["Us"][:, :, :nu]
    J = r["J"]
    U0 = eq45(J, Us, lam)
    assert np.max(np.abs(U0 - r["Unew"][:, :nu])) < 1e-9, "Eq. 4/5 restatement disagrees with the oracle"
    rng = np.random.default_rng(12345)
    floor = 0.0
    for _ in range(seeds):
        s = rng.choice([-1.0, 1.0], size=J.shape[0])
        floor = max(floor, float(np.max(np.abs(eq45(J + s * U32 * r["Jabs"], Us, lam) - U0))))
    return floor
