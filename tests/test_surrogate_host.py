"""Host-side mapping of the crater surrogate's outputs: the network regresses the profile in
km and the logarithms of the transient depth and the diameter, so a unit error in those two
outputs is a relative error; the mapping and its inverse round-trip, and an equal error in
the network's space is the same relative error at any crater size."""
import numpy as np

from paper_2403_04267_gb300 import surrogate as S


def _targets(rng, n):
    prof = rng.uniform(-2.0, 0.5, (n, S.N_PROFILE)) * S.DEPTH_SCALE
    depth = rng.uniform(50.0, 3000.0, n)
    diam = rng.uniform(200.0, 9000.0, n)
    return np.stack([S.targets(prof[k], depth[k], diam[k]) for k in range(n)])


def test_network_mapping_round_trips():
    T = _targets(np.random.default_rng(1), 50)
    back = S.from_network(S.to_network(T))
    assert np.allclose(back, T, rtol=2e-6, atol=2e-6)


def test_a_network_error_in_depth_and_diameter_is_relative():
    T = _targets(np.random.default_rng(2), 20)
    Y = S.to_network(T).astype(np.float64)
    Y[:, S.N_PROFILE:] += 0.01 * S.OUT_WEIGHT[S.N_PROFILE:]      # +0.01 in log units
    ed, eD = S.crater_errors(S.from_network(Y), T)
    assert np.allclose(ed, np.expm1(0.01), rtol=1e-5) and np.allclose(eD, np.expm1(0.01), rtol=1e-5)
