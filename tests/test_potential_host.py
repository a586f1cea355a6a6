"""Host-side logic of the learned-potential module (no GPU): the parameter vector's
layout and initialisation agree with the oracle's (W1, b1, W2, b2, W3, b3, c)."""
import numpy as np

from oracle import mlp
from paper_1711_05095_gb300 import potential


def test_parameter_layout_matches_oracle():
    assert potential.N_PARAMS == mlp.N_PARAMS == 17922
    for seed in (0, 7):
        a = potential.init_params(seed)
        b = mlp.init_params(seed)
        assert a.dtype == np.float32 and a.shape == (potential.N_PARAMS,)
        np.testing.assert_array_equal(a, b)
    parts = mlp.unpack(potential.init_params(1))
    assert parts["W1"].shape == (128, 9) and parts["W2"].shape == (128, 128)
    assert np.all(parts["b1"] == 0) and np.all(parts["b2"] == 0) and parts["c"] == 0
    assert np.abs(parts["W2"]).max() <= 1 / np.sqrt(128)
