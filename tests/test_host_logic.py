"""Host-side serving and tuning logic (CPU): the fleet's request schedule
(Poisson-jittered arrivals at each drone's rate class, time-ordered,
reproducible from the seed, with K and N drawn from the configured choices),
the autotuner's JSON cache, and the lap counter of the closed-loop flights."""
import numpy as np

from paper_2509_14726_gb300 import serving as SV, workloads as W


def _fleet(n):
    return W.c5_fleet(n_drones=n, distinct_tracks=3)


def test_arrival_counts_follow_the_rate_classes():
    fleet = _fleet(60)
    duration, scale = 4.0, 0.5
    sched = SV.make_schedule(fleet, duration, scale, (1024, 4096), (30, 50), seed=1)
    assert np.all(np.diff(sched.t) >= 0.0)
    assert sched.t.min() >= 0.0 and sched.t.max() < duration
    for rate in (50.0, 100.0, 200.0):
        ids = [d.drone_id for d in fleet if d.rate_hz == rate]
        n = int(np.isin(sched.drone, ids).sum())
        expected = len(ids) * rate * scale * duration
        # Poisson count: within five standard deviations of its mean
        assert abs(n - expected) <= 5.0 * np.sqrt(expected), (rate, n, expected)


def test_gaps_are_exponential_with_the_class_mean():
    fleet = _fleet(3)  # one drone per rate class
    sched = SV.make_schedule(fleet, 40.0, 1.0, (1024,), (30,), seed=2)
    for d in fleet:
        t = sched.t[sched.drone == d.drone_id]
        gaps = np.diff(t)
        mean = 1.0 / d.rate_hz
        # sample mean of n exponential gaps: standard error mean / sqrt(n)
        assert abs(gaps.mean() - mean) <= 5.0 * mean / np.sqrt(len(gaps))
        # exponential: standard deviation equals the mean
        assert abs(gaps.std() - mean) <= 0.15 * mean


def test_schedule_is_reproducible_and_uses_the_choices():
    fleet = _fleet(12)
    a = SV.make_schedule(fleet, 2.0, 0.3, (1024, 4096, 16384), (30, 50, 80), seed=7)
    b = SV.make_schedule(fleet, 2.0, 0.3, (1024, 4096, 16384), (30, 50, 80), seed=7)
    c = SV.make_schedule(fleet, 2.0, 0.3, (1024, 4096, 16384), (30, 50, 80), seed=8)
    for f in ("t", "drone", "K", "N"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.t, c.t)
    assert set(np.unique(a.K)) <= {1024, 4096, 16384}
    assert set(np.unique(a.N)) <= {30, 50, 80}
    assert len(np.unique(a.K)) == 3 and len(np.unique(a.N)) == 3


def test_autotune_cache_round_trip_and_corrupt_file(tmp_path):
    """The autotuner's JSON cache (no device): entries persist across
    instances, and an unreadable file starts an empty cache."""
    from paper_2509_14726_gb300 import autotune as AT
    path = str(tmp_path / "sub" / "tune.json")
    c = AT.Cache(path)
    assert c.get("k") is None
    c.put("k", {"block": 128, "spt": 2})
    assert AT.Cache(path).get("k") == {"block": 128, "spt": 2}
    with open(path, "w") as f:
        f.write("{not json")
    assert AT.Cache(path).get("k") is None


def test_closed_loop_gate_crossing_rule():
    """closed_loop.crossing (the lap counter of the comparison flights):
    front-to-back through the opening counts, at the interpolated point;
    outside the opening, backwards, or not reaching the plane does not."""
    from paper_2509_14726_gb300 import closed_loop as CL
    # gate at the origin facing +x (yaw 0), half-width 0.75, half-height 0.75
    g = np.array([0.0, 0.0, 2.0, 0.0, 0.75, 0.75])
    a = CL.crossing(g, np.array([-1.0, 0.2, 2.1]), np.array([3.0, 0.2, 2.1]))
    assert a is not None and abs(a - 0.25) < 1e-12
    assert CL.crossing(g, np.array([-1.0, 0.0, 2.0]), np.array([0.0, 0.0, 2.0])) == 1.0  # s = 0 counts
    assert CL.crossing(g, np.array([-1.0, 0.9, 2.0]), np.array([1.0, 0.9, 2.0])) is None  # beside the opening
    assert CL.crossing(g, np.array([-1.0, 0.0, 2.9]), np.array([1.0, 0.0, 2.9])) is None  # above it
    assert CL.crossing(g, np.array([1.0, 0.0, 2.0]), np.array([-1.0, 0.0, 2.0])) is None  # backwards
    assert CL.crossing(g, np.array([-2.0, 0.0, 2.0]), np.array([-1.0, 0.0, 2.0])) is None  # short of the plane
    # a yawed gate: normal along +y
    g90 = np.array([5.0, 5.0, 2.0, np.pi / 2, 0.75, 0.75])
    assert CL.crossing(g90, np.array([5.3, 4.0, 2.0]), np.array([5.3, 6.0, 2.0])) is not None
    assert CL.crossing(g90, np.array([6.0, 4.0, 2.0]), np.array([6.0, 6.0, 2.0])) is None
