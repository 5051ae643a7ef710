"""Seeded input generators: SplitMix64 against its published reference outputs,
and the shapes / parameter ranges of the synthetic workloads."""
import numpy as np

import workloads as W


def test_splitmix64_reference_outputs():
    # first five outputs of SplitMix64 seeded with 1234567 (reference implementation)
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [int(x) for x in W.splitmix64(1234567, 5)] == ref


def test_uniform01_range_and_determinism():
    a = W.uniform01(0, 100000)
    assert a.min() >= 0.0 and a.max() < 1.0 and abs(a.mean() - 0.5) < 5e-3
    assert np.array_equal(a, W.uniform01(0, 100000))


def test_thermal_decay_fields():
    c = W.thermal_decay(n=64)
    assert c.rho.shape == (64, 64) and c.u.shape == (2, 64, 64)
    assert np.allclose((c.rho * c.theta), 1.0, atol=2e-6)   # isobaric up to the noise
    assert c.params["H"] and c.params["Pr"] == 0.71


def test_batched_domain_list():
    cases = W.batched(256, seed=0)
    sizes = np.array([c.nx for c in cases])
    assert len(cases) == 256 and sizes.min() >= 32 and sizes.max() <= 256
    total = sum(c.nodes for c in cases)
    assert 5.0e6 < total < 8.0e6
    taus = np.array([c.tau_hat for c in cases])
    assert taus.min() >= 0.55 and taus.max() <= 1.2
    assert all(c.params["SC"] for c in cases[1::2]) and all(c.params["H"] for c in cases[0::2])
