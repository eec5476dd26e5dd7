"""Pins of the oracle's Philox4x64-10, uniform conversion and draw order (model: Philox keyed
by (seed, event id, draw block), each uniform one 32-bit half of a word, replacing the
paper's CURAND states, §3.1)."""
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
    assert oracle.uniform(0) == 0.5 * 2.0**-32
    assert oracle.uniform(2**32 - 1) == 1.0 - 0.5 * 2.0**-32
    h = 0x89ABCDEF
    assert oracle.uniform(h) == (h + 0.5) / 2.0**32


@pytest.mark.parametrize("seed,event", [(0, 0), (5, 11), (2**64 - 1, 2**40 + 3)])
def test_draw_stream_is_the_half_words_of_numpy_philox(seed, event):
    """Draw d of an event is half d % 2 (high first) of word (d / 2) % 4 of the Philox block
    with counter (d / 8, event, 0, 0) and key (seed, 0): numpy's Philox, whose counter is
    incremented before each block, started one below (d / 8, event, 0, 0)."""
    n = 40  # five blocks
    draws = oracle.stream_draws(seed, event, n)
    # the counter (0, event, 0, 0) minus one, borrowing across the four 64-bit words
    start, borrow = [0, event, 0, 0], 1
    for k in range(4):
        start[k] -= borrow
        borrow = 1 if start[k] < 0 else 0
        start[k] %= 2**64
    g = np.random.Philox(key=np.array([seed, 0], np.uint64), counter=np.array(start, np.uint64))
    words = [int(x) for x in g.random_raw(n // 2)]
    halves = [h for w in words for h in (w >> 32, w & 0xFFFFFFFF)]
    assert [float(d) for d in draws] == [(h + 0.5) / 2.0**32 for h in halves]


def test_event_streams_are_uniform_and_independent():
    # partner-momentum cos(theta) = 2u - 1 exposes the raw uniforms of one event's stream
    d = oracle.sample_fermi(1.0, 20000, seed=3, event=11)
    u = (d[:, 2] / np.linalg.norm(d, axis=1) + 1) / 2
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = ((h - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
    d2 = oracle.sample_fermi(1.0, 20000, seed=3, event=12)
    assert abs(np.corrcoef(d[:, 2], d2[:, 2])[0, 1]) < 0.03
