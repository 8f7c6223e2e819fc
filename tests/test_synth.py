"""The seeded input generator: published reference outputs, determinism,
and the shape of what it draws (Algorithms 1 and 3 input distributions)."""
import numpy as np
import pytest

import oracle
import synth


def test_splitmix64_reference_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    got = [int(x) for x in synth.splitmix_raw(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_xoshiro256ss_reference_outputs():
    # xoshiro256** (Blackman, Vigna 2018) from state {1, 2, 3, 4}
    got = [int(x) for x in synth.xoshiro_raw([1, 2, 3, 4], 4)]
    assert got == [11520, 0, 1509978240, 1215971899390074240]


@pytest.mark.parametrize("level", [1, 3, 5])
def test_keys_and_ciphertext_randomness(level):
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, 5)
    h2, x2, y2 = synth.keys(S, 2, first=3)
    assert (h[3:] == h2).all() and (x[3:] == x2).all() and (y[3:] == y2).all()
    for row in np.concatenate([x, y]):
        assert len(set(row.tolist())) == P.w and row.max() < P.n
    nb = P.n % 64
    assert (h[:, P.W_u - 1] >> np.uint64(nb) == 0).all()
    assert (h[:, P.W_u:] == 0).all()
    m, r1, r2, e = synth.ciphertext_randomness(S, 64)
    for row in np.concatenate([r1, r2]):
        assert len(set(row.tolist())) == P.wr and row.max() < P.n
    for row in e:
        assert len(set(row.tolist())) == P.we
    assert m.shape == (64, P.k)
    assert 100 < m.mean() < 155


def test_key_assignment_balanced_and_shuffled():
    idx = synth.key_assignment(1000, 16, tag=3)
    assert sorted(np.bincount(idx).tolist()) == [62] * 8 + [63] * 8
    assert not (idx == np.arange(1000) % 16).all()
    assert (synth.key_assignment(1000, 16, tag=3) == idx).all()


def test_uniform_below_range():
    v = synth.below(17669, 20000, tag=1)
    assert v.max() < 17669 and v.min() >= 0
    assert abs(v.mean() / 17669 - 0.5) < 0.02
