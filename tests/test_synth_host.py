"""Host checks of the input generators that a tolerance relies on (no method arithmetic)."""
import numpy as np

import synth


def test_householder_inverse_from_the_same_reflectors():
    # the kappa_inf of the mixed-precision parity tolerance is built from this inverse
    n = 300
    A = synth.householder_spd(n, seed=5).numpy()
    Ai = synth.householder_spd(n, seed=5, inverse=True).numpy()
    assert np.abs(A @ Ai - np.eye(n)).max() <= 1e-9
    assert np.linalg.cond(A) == np.float64(1e6) or abs(np.linalg.cond(A) / 1e6 - 1) <= 1e-8
