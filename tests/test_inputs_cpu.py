"""The seeded input module against the recipes it states: near-cubic boxes,
the batched-solve instances, the Poisson arrival stream, the smooth random
right-hand sides and the i.i.d. fields.  Every generator is reproducible
from its seed."""

import math

import numpy as np

from paper_2110_01716_gb300 import inputs


def _near_cubic_triples(limit):
    for ex in range(1, limit):
        for ey in (ex, ex + 1):
            for ez in (ey, ey + 1):
                if ez - ex <= 1:
                    yield ex, ey, ez


def test_near_cube_factors_is_the_closest_near_cubic_box():
    triples = list(_near_cubic_triples(60))
    for E in list(range(1, 400)) + [512, 1000, 4095, 8192, 32767, 65536]:
        ex, ey, ez = inputs.near_cube_factors(E)
        assert max(ex, ey, ez) - min(ex, ey, ez) <= 1
        best = min(abs(a * b * c - E) for a, b, c in triples)
        assert abs(ex * ey * ez - E) == best, (E, (ex, ey, ez))


def test_batch_instances_follow_the_recipe():
    a = inputs.batch_instances(4)
    assert a == inputs.batch_instances(4)                 # reproducible
    assert a != inputs.batch_instances(5)
    assert len(a) == 64
    assert {p["N"] for p in a} <= {5, 7, 9} and len({p["N"] for p in a}) == 3
    assert len({p["seed"] for p in a}) == 64               # one mesh seed each
    E = np.array([p["ex"] * p["ey"] * p["ez"] for p in a])
    for p in a:
        f = (p["ex"], p["ey"], p["ez"])
        assert max(f) - min(f) <= 1
    # log-uniform in [64, 8192] (nearest near-cubic box: within 15 % of the range)
    assert E.min() >= 64 * 0.85 and E.max() <= 8192 * 1.15
    logs = np.log(E)
    assert abs(logs.mean() - 0.5 * (math.log(64) + math.log(8192))) < 0.6
    assert (logs < math.log(724)).sum() > 16 and (logs > math.log(724)).sum() > 16


def test_arrival_stream_is_poisson_at_the_rate():
    rate = 14.0
    s = inputs.arrival_stream(5, 1000, rate)
    assert s == inputs.arrival_stream(5, 1000, rate)
    t = np.array([q["t"] for q in s])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate, coefficient of variation 1 (1000 draws)
    assert abs(gaps.mean() * rate - 1.0) < 0.12
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15
    assert {q["N"] for q in s} == {7}
    assert {q["tol"] for q in s} == {1e-6, 1e-8, 1e-10}
    E = np.array([q["ex"] * q["ey"] * q["ez"] for q in s])
    assert E.min() >= 512 * 0.85 and E.max() <= 65536 * 1.15


def test_fourier_modes_and_sequence():
    a, k, phi = inputs.fourier_modes(3)
    a2, k2, phi2 = inputs.fourier_modes(3)
    assert np.array_equal(a, a2) and np.array_equal(k, k2) and np.array_equal(phi, phi2)
    assert k.shape == (8, 3) and np.all((k >= 0) & (k <= 3)) and np.all(k.any(axis=1))
    assert np.all((phi >= 0) & (phi < 2 * math.pi))
    # a_m |k_m|^2 are the standard normal draws: finite, of both signs here
    z = a * np.sum(k * k, axis=1)
    assert np.all(np.isfinite(z)) and np.abs(z).max() < 6
    a3, k3, phi3, om = inputs.fourier_sequence(3)
    assert np.array_equal(a3, a) and np.array_equal(k3, k) and np.array_equal(phi3, phi)
    assert om.shape == (8,) and np.all((om >= 0.02) & (om < 0.1))


def test_random_field_is_iid_uniform_and_seeded():
    u = inputs.random_field(200000, 7)
    assert np.array_equal(u, inputs.random_field(200000, 7))
    assert not np.array_equal(u, inputs.random_field(200000, 8))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
