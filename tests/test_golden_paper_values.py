"""The workload configuration against the values the paper prints.

tests/golden/paper_table1_parameters.json holds Table I of the paper (Sec.
V-A): the solve size, temperature and step of its simulation study, and the
ranges of the inputs and states.  The input generators that feed both the
oracle and the CUDA path must reproduce them where the workload claims to be
the paper's configuration.
"""
import json
import os

import numpy as np

from paper_2509_14726_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table1_parameters.json")


def _table1():
    with open(GOLDEN) as f:
        return json.load(f)


def test_table1_solve_size_temperature_and_step():
    t = _table1()
    for obj in (W.OBJ_GATE, W.OBJ_CONTOUR, W.OBJ_TRACK):
        mc, sc, tr, x0 = W.paper_table1(obj)
        assert (sc.K, sc.N) == (t["samples_M"], t["horizon_K"])
        assert sc.lam == t["lambda"] and sc.dt == t["dt_s"]


def test_table1_input_and_state_ranges():
    t = _table1()
    ctbr, rotor = W.ModelConfig(), W.rotor_model()
    # rotor model: rotor-thrust rates and the rotor thrusts they integrate
    np.testing.assert_array_equal(rotor.u_min[:4], [t["rotor_thrust_rate_range"][0]] * 4)
    np.testing.assert_array_equal(rotor.u_max[:4], [t["rotor_thrust_rate_range"][1]] * 4)
    assert (rotor.thrust_min, rotor.thrust_max) == tuple(t["rotor_thrust_range_N"])
    # contouring's progress acceleration, both models
    for mc in (ctbr, rotor):
        assert (mc.u_min[4], mc.u_max[4]) == tuple(t["progress_acceleration_range"])
    # body rates: the collective-thrust model's rate commands and the state
    # penalty's limit
    lo, hi = t["body_rate_range_rad_s"]
    np.testing.assert_array_equal(ctbr.u_min[1:4], [lo] * 3)
    np.testing.assert_array_equal(ctbr.u_max[1:4], [hi] * 3)
    for mc in (ctbr, rotor):
        assert mc.omega_max == hi
