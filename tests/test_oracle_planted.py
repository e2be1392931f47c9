"""Planted mistakes: each deliberate error, compiled into a copy of the oracle,
must make at least one closed-form pin fail. This shows the pins can see the
kinds of mistake a restatement of the method is likely to contain."""
import pytest

from oracle import oracle
from tests import pins

PLANTS = {
    "PLANT_NO_QNOBAR": [pins.pin_inner_step, pins.pin_lookahead_weight],
    "PLANT_AZZ_T": [pins.pin_inner_step, pins.pin_lookahead_weight],
    "PLANT_NO_PROJ_NOISE": [pins.pin_lookahead_weight, pins.pin_kalman],
    "PLANT_GROWTH_SIGN": [lambda lib: pins.pin_lookahead_weight(lib, growth=True)],
    "PLANT_MEAN_NO_GAIN": [pins.pin_kalman],
    "PLANT_NO_AVERAGE": [pins.pin_lookahead_weight],
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_mistake_is_caught(plant):
    lib = oracle.load(oracle.build(extra_flags=(f"-D{plant}",)))
    results = [f(lib)[0] for f in PLANTS[plant]]
    assert not all(results), f"{plant} passed every pin"
