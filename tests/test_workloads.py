"""The seeded input generators build the tracks the paper's experiments need
(gates, arc-length path P_arc, constant-speed reference tau_ref)."""
import math

import numpy as np
import pytest

from paper_2509_14726_gb300 import workloads as W


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_circle_gates_are_tangent():
    g = W.circle_gates(4, 5.0, 2.0)
    for i in range(4):
        c = g[i, :3]
        n = np.array([math.cos(g[i, 3]), math.sin(g[i, 3]), 0])
        assert abs(np.linalg.norm(c[:2]) - 5.0) < 1e-12 and c[2] == 2.0
        assert abs(np.dot(n[:2], c[:2])) < 1e-12  # normal tangent to the circle
        assert c[0] * n[1] - c[1] * n[0] > 0  # counter-clockwise
    assert np.all(g[:, 4:] == 0.75)


@pytest.mark.parametrize("seed,n", [(7, 7), (11, 5), (12, 9)])
def test_random_course_spacing_and_box(seed, n):
    g = W.random_gates(seed, n)
    d = np.linalg.norm(g[:, None, :3] - g[None, :, :3], axis=-1)
    assert np.min(d[np.triu_indices(n, 1)]) >= 6.0
    assert np.all(np.abs(g[:, :2]) <= 15.0) and np.all((g[:, 2] >= 1.0) & (g[:, 2] <= 7.0))
    np.testing.assert_array_equal(g, W.random_gates(seed, n))  # seeded


def test_spline_path_is_arc_length_parameterised():
    tr = W.random_course(7, 7)
    S = tr.path.shape[0]
    ds = tr.L / S
    P, T = tr.path[:, :3], tr.path[:, 3:]
    np.testing.assert_allclose(np.linalg.norm(T, axis=1), 1.0, atol=1e-12)
    chord = np.linalg.norm(np.roll(P, -1, axis=0) - P, axis=1)
    assert np.all(chord <= ds * (1 + 1e-9)) and np.all(chord >= 0.99 * ds)
    # the path goes through every gate centre
    for c in tr.gates[:, :3]:
        assert np.min(np.linalg.norm(P - c, axis=1)) <= 0.5 * ds + 1e-9
    # tangent is the direction of motion between nodes
    dirs = (np.roll(P, -1, axis=0) - P) / chord[:, None]
    assert np.min(np.sum(dirs * T, axis=1)) > 0.95


def test_reference_is_flown_at_constant_speed_with_consistent_attitude():
    tr = W.circle_track(4, 5.0, 2.0)
    ref, dt = tr.ref, tr.dt_ref
    np.testing.assert_allclose(np.linalg.norm(ref[:, 3:6], axis=1), 8.0, atol=1e-9)
    assert abs(ref.shape[0] * dt * 8.0 - tr.L) < 1e-9
    np.testing.assert_allclose(np.linalg.norm(ref[:, 6:10], axis=1), 1.0, atol=1e-12)
    # position difference matches the velocity (central difference)
    dp = (np.roll(ref[:, :3], -1, axis=0) - np.roll(ref[:, :3], 1, axis=0)) / (2 * dt)
    assert np.max(np.linalg.norm(dp - ref[:, 3:6], axis=1)) < 1e-2
    # thrust axis is along a + g e_z, body x points along the heading
    acc = (np.roll(ref[:, 3:6], -1, axis=0) - np.roll(ref[:, 3:6], 1, axis=0)) / (2 * dt)
    for i in range(0, ref.shape[0], 17):
        R = _rot(ref[i, 6:10])
        f = acc[i] + np.array([0, 0, 9.81])
        assert np.dot(R[:, 2], f / np.linalg.norm(f)) > 0.999
        assert np.dot(R[:, 0][:2], ref[i, 3:5]) > 0
    # body rates integrate the attitude: q_{i+1} ~ q_i * exp(w dt / 2)
    i = 10
    w = ref[i, 10:13]
    q = ref[i, 6:10]
    half = 0.5 * w * dt
    dq = np.concatenate([[1.0], half])
    qn = np.array([q[0] * dq[0] - np.dot(q[1:], dq[1:]),
                   *(q[0] * dq[1:] + dq[0] * q[1:] + np.cross(q[1:], dq[1:]))])
    assert np.linalg.norm(qn / np.linalg.norm(qn) - ref[i + 1, 6:10]) < 1e-4


def test_hover_start_is_one_metre_before_the_gate():
    g = W.circle_gates()
    x = W.hover_state_before_gate(g, 0, 1.0)
    n = np.array([math.cos(g[0, 3]), math.sin(g[0, 3]), 0])
    np.testing.assert_allclose(x[:3], g[0, :3] - n, atol=1e-12)
    np.testing.assert_allclose(_rot(x[6:10])[:, 0], n, atol=1e-12)


def test_batch_workload_shape():
    items = W.c3_batch(n_drones=64)
    Ks = np.array([it.K for it in items])
    Ns = np.array([it.N for it in items])
    assert Ks.min() >= 1024 and Ks.max() <= 16384
    assert Ns.min() >= 20 and Ns.max() <= 80
    assert set(it.objective for it in items) == {0, 1, 2}
    assert all(5 <= it.n_gates <= 9 for it in items)
