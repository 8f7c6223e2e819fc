"""The open-loop burst trace used by the serving benchmark (host only)."""
import numpy as np

import synth


def test_burst_trace_rate_and_bursts():
    t = synth.burst_trace(2e5, 2.0, tag=9)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] < 2e9
    assert abs(len(t) / 2.0 / 2e5 - 1) < 0.15
    _, sizes = np.unique(t, return_counts=True)
    assert sizes.min() >= 1 and sizes.max() <= 512
    # log-uniform sizes: P(B = 1) = ln 2 / ln 513 ~ 0.111
    assert abs((sizes == 1).mean() - np.log(2) / np.log(513)) < 0.03
    assert (synth.burst_trace(2e5, 2.0, tag=9) == t).all()


def test_level_mix_shares():
    lv = synth.level_mix(10000, ((1, 0.4), (3, 0.35), (5, 0.25)), tag=1)
    assert (np.bincount(lv)[[1, 3, 5]] == [4000, 3500, 2500]).all()
    assert not (lv[:4000] == 1).all()
