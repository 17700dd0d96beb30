"""The paper's performance model (section 4.1, Eq. 2-7): sem_perf_model (the
library's exact minimiser, host code) against the brute-force element-split
search of oracle/perf_model.py, and the oracle against closed forms."""
import math

import numpy as np
import pytest

from oracle import perf_model as om
from paper_2405_05640_gb300 import binding


# ---- the oracle against the model's closed forms
def test_oracle_single_device_and_additive_performance():
    T, sp = om.tmin_search(120, 0.5, [3.0])
    assert sp == (120,) and T == pytest.approx(120 * 0.5 / 3.0, rel=1e-15)
    # unconstrained: performances add, T_min = C / sum P, split proportional to P
    T, sp = om.tmin_search(400, 1.0, [3.0, 1.0])
    assert sp == (300, 100) and T == pytest.approx(400 / 4.0, rel=1e-15)


def test_oracle_capacity_binds_and_superlinear():
    # the fast device holds only 200 elements: it is filled, the slow one takes the rest
    T, sp = om.tmin_search(400, 1.0, [3.0, 1.0], [200.0, 0])
    assert sp == (200, 200) and T == pytest.approx(200.0)
    # two devices that cannot hold the problem alone: together they can (the
    # superlinear regime of the paper: alone the run time is unbounded)
    T1, _ = om.tmin_search(100, 1.0, [2.0], [60.0])
    T2, sp = om.tmin_search(100, 1.0, [2.0, 2.0], [60.0, 60.0])
    assert math.isinf(T1) and sp in ((50, 50),) and T2 == pytest.approx(25.0)
    T, sp = om.tmin_search(100, 1.0, [2.0, 2.0], [40.0, 40.0])
    assert math.isinf(T) and sp is None


# ---- the library against the oracle
def test_perf_model_closed_form_unconstrained():
    P = np.array([7.5, 0.25, 1.0])
    T, sp = binding.perf_model(P, 1000.0)
    assert T == pytest.approx(1000.0 / P.sum(), rel=1e-15)
    np.testing.assert_allclose(sp, 1000.0 * P / P.sum(), rtol=1e-14)


@pytest.mark.parametrize("seed", range(12))
def test_perf_model_matches_element_search(seed):
    rng = np.random.default_rng(seed)
    n = 2 if seed < 8 else 3
    E = int(rng.integers(20, 90 if n == 3 else 400))
    c = float(rng.uniform(0.5, 2.0))
    P = rng.uniform(0.1, 10.0, n)
    cap = [float(rng.uniform(0.2, 1.0) * E * c) if rng.random() < 0.6 else 0.0 for _ in range(n)]
    To, spo = om.tmin_search(E, c, list(P), cap)
    if math.isinf(To):
        # no integer split fits; the continuous model may still fit only if the
        # capacities hold the cost
        if sum(x if x > 0 else math.inf for x in cap) < E * c:
            with pytest.raises(binding.SemError) as ei:
                binding.perf_model(P, E * c, cap)
            assert ei.value.status == binding.SEM_ERR_WORKSPACE
        return
    T, sp = binding.perf_model(P, E * c, cap)
    # the continuous optimum bounds the element-granular one from below; rounding
    # its split to whole elements leaves fewer than n elements to place, at most
    # n - 1 element-times on one device
    assert T <= To * (1 + 1e-12)
    assert To <= T + (n - 1) * max(c / p for p in P) * (1 + 1e-12)
    assert sp.sum() == pytest.approx(E * c, rel=1e-12)
    for i in range(n):
        if cap[i] > 0:
            assert sp[i] <= cap[i] * (1 + 1e-12)
        assert sp[i] / P[i] <= T * (1 + 1e-12)


def test_perf_model_errors():
    with pytest.raises(binding.SemError) as ei:
        binding.perf_model([1.0, 0.0], 10.0)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    with pytest.raises(binding.SemError) as ei:
        binding.perf_model([1.0, 2.0], 10.0, [3.0, 3.0])
    assert ei.value.status == binding.SEM_ERR_WORKSPACE
    T, sp = binding.perf_model([1.0, 2.0], 0.0)
    assert T == 0.0 and not sp.any()
