"""The oracle's step against closed forms (CPU only). See ``tests/pins.py``."""
import numpy as np
import pytest

from paper_1203_2394_gb300 import workloads
from tests import pins
from tests.kalman import dense_posterior, kalman


def test_kalman_filter_matches_dense_conditioning():
    spec = workloads.make_model("lg4", 0)
    _, ys = workloads.simulate(spec, 6, 0)
    km, _, kll = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    dm, dll = dense_posterior(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    np.testing.assert_allclose(km, dm, rtol=1e-9, atol=1e-9)
    assert kll.sum() == pytest.approx(dll, rel=1e-10)


@pytest.mark.parametrize("growth", [False, True])
def test_lookahead_weight_is_unbiased_for_exact_predictive(oracle_lib, growth):
    ok, info = pins.pin_lookahead_weight(oracle_lib, growth=growth)
    assert ok, info


def test_inner_step_targets_mixture_posterior(oracle_lib):
    ok, info = pins.pin_inner_step(oracle_lib)
    assert ok, info


def test_filter_tracks_kalman(oracle_lib):
    ok, info = pins.pin_kalman(oracle_lib)
    assert ok, info
