"""Pins of the oracle's Philox4x64-10 and uniform conversion (model: Philox keyed by
(seed, event id, draw block), replacing the paper's CURAND states, §3.1)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("key", [(0, 0), (7, 0), (2**64 - 1, 12345), (0xDEADBEEF, 2**63)])
@pytest.mark.parametrize("counter", [(0, 0, 0, 0), (5, 9, 0, 0), (2**64 - 2, 1, 2, 3)])
def test_philox_matches_numpy(key, counter):
    # numpy's Philox advances its 256-bit counter by one before producing each block of 4
    g = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(counter, np.uint64))
    ref = g.random_raw(12)
    mine = []
    c = list(counter)
    for _ in range(3):
        # add one with carry across the four 64-bit words
        for k in range(4):
            c[k] = (c[k] + 1) % 2**64
            if c[k] != 0:
                break
        mine.extend(int(x) for x in oracle.philox4x64_10(c, key))
    assert [int(x) for x in ref] == mine


def test_uniform_conversion_exact_open_interval():
    assert oracle.uniform(0) == 0.5 * 2.0**-52
    assert oracle.uniform(2**64 - 1) == 1.0 - 0.5 * 2.0**-52
    w = 0x0123456789ABCDEF
    assert oracle.uniform(w) == ((w >> 12) + 0.5) / 2.0**52


def test_event_streams_are_uniform_and_independent():
    # partner-momentum cos(theta) = 2u - 1 exposes the raw uniforms of one event's stream
    d = oracle.sample_fermi(1.0, 20000, seed=3, event=11)
    u = (d[:, 2] / np.linalg.norm(d, axis=1) + 1) / 2
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = ((h - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
    d2 = oracle.sample_fermi(1.0, 20000, seed=3, event=12)
    assert abs(np.corrcoef(d[:, 2], d2[:, 2])[0, 1]) < 0.03
