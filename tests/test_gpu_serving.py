"""The continuous-batching service loop (hqc_serve_run) on the GPU.

Requests reference a pinned host ring of oracle-built ciphertexts of all
three levels; the expected result of every ring entry is its message.
"""
import numpy as np
import pytest

import synth
from workloads import honest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = ((1, 0.40), (3, 0.35), (5, 0.25))


@pytest.fixture(scope="module")
def hqc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2512_12904_gb300 as lib
    lib.load()
    return lib


def make_ring(hqc, period, tag, entries=None):
    """Ring of `period` requests (levels 40/35/25 %) with their messages."""
    levels = synth.level_mix(period, MIX, tag=tag)
    pools = {l: honest(l, 4, max(1, int((levels == l).sum())), first_ct=70000 + 1000 * tag, tag=tag)
             for l in (1, 3, 5)}
    used = {1: 0, 3: 0, 5: 0}
    rows, keys_, woff, moff, want = [], [], [0], [0], []
    for l in levels:
        wl, i = pools[int(l)], used[int(l)]
        used[int(l)] += 1
        rows += [wl.u[i], wl.v[i]]
        keys_.append(wl.key_idx[i])
        woff.append(woff[-1] + wl.P.W_u_pitch + wl.P.W_v)
        moff.append(moff[-1] + wl.P.k)
        want.append(wl.m[i])
    ks = [hqc.Keyset(l, pools[l].y) for l in (1, 3, 5)]
    words = torch.from_numpy(np.concatenate(rows).view(np.int64)).pin_memory()
    return dict(keys=ks, level=levels, key=np.array(keys_, np.int32), word_off=np.array(woff, np.int64),
                words=words, m_off=np.array(moff, np.int64), want=np.concatenate(want), pools=pools)


def run(hqc, R, arrivals, level=None, key=None, **kw):
    return hqc.hqc_serve_run(R["keys"], R["level"] if level is None else level, R["key"] if key is None else key,
                             R["word_off"], R["words"], R["m_off"], arrivals, **kw)


@pytest.mark.parametrize("transfer", [1, 2])
def test_results_alone_and_in_the_mix(hqc, transfer):
    """Copy mode (1) and in-place reads of the ring (2): every request's
    result is its message, in a burst mix, spread out, and alone."""
    R = make_ring(hqc, 300, tag=1)
    # everything at once (a burst mix), then spread out one by one
    st, lat, m_mix, stats = run(hqc, R, np.zeros(300, np.int64), streams=3, max_batch=64, transfer=transfer)
    assert (st == 0).all() and (lat >= 0).all() and stats["completed"] == 300
    assert (m_mix == R["want"]).all() and stats["batches"] >= 5
    assert stats["in_place"] == (transfer == 2)
    st2, lat2, m_spread, _ = run(hqc, R, np.arange(300, dtype=np.int64) * 20000, streams=2, transfer=transfer)
    assert (st2 == 0).all() and (m_spread == R["want"]).all()
    # large batches take the per-level persistent kernels
    st3, _, m_big, stats3 = run(hqc, R, np.zeros(300, np.int64), streams=1, max_batch=4096, transfer=transfer)
    assert (st3 == 0).all() and (m_big == R["want"]).all() and stats3["batches"] == 1
    # a few entries alone: a one-entry ring holding the same ciphertext
    for j in (0, 7, 123, 299):
        w0, w1 = R["word_off"][j], R["word_off"][j + 1]
        m0, m1 = R["m_off"][j], R["m_off"][j + 1]
        one = torch.from_numpy(R["words"][w0:w1].numpy().copy()).pin_memory()
        st1, _, m1_out, _ = hqc.hqc_serve_run(R["keys"], R["level"][j:j + 1], R["key"][j:j + 1],
                                              np.array([0, w1 - w0], np.int64), one,
                                              np.array([0, m1 - m0], np.int64), np.zeros(1, np.int64),
                                              transfer=transfer)
        assert st1[0] == 0 and (m1_out == m_mix[m0:m1]).all()


def test_invalid_requests_are_answered_and_the_rest_decrypts(hqc):
    R = make_ring(hqc, 60, tag=2)
    level = R["level"].copy()
    key = R["key"].copy()
    level[3] = 2          # no such level
    key[10] = 10 ** 6     # key index out of range
    st, lat, m, stats = run(hqc, R, np.zeros(60, np.int64), level=level, key=key)
    assert st[3] == 4 and st[10] == 4 and stats["rejected_invalid"] == 2
    ok = np.ones(60, bool)
    ok[[3, 10]] = False
    assert (st[ok] == 0).all() and (lat[ok] >= 0).all() and (lat[~ok] == -1).all()
    for j in np.nonzero(ok)[0]:
        assert (m[R["m_off"][j]:R["m_off"][j + 1]] == R["want"][R["m_off"][j]:R["m_off"][j + 1]]).all()


def test_memory_budget_admission(hqc):
    R = make_ring(hqc, 80, tag=3)
    # 8 KB per stream holds one HQC-1 request but no HQC-3/5 request
    st, _, m, stats = run(hqc, R, np.zeros(80, np.int64), streams=2, budget_bytes=2 * 8192)
    big = R["level"] != 1
    assert (st[big] == 5).all() and (st[~big] == 0).all()
    assert stats["rejected_size"] == int(big.sum()) and stats["items_per_slot"] == 1
    for j in np.nonzero(~big)[0]:
        assert (m[R["m_off"][j]:R["m_off"][j + 1]] == R["want"][R["m_off"][j]:R["m_off"][j + 1]]).all()


@pytest.mark.parametrize("transfer", [0, 1])
def test_queue_limit_rejects_and_the_admitted_decrypt(hqc, transfer):
    R = make_ring(hqc, 200, tag=4)
    arr = np.zeros(1000, np.int64)     # 1000 requests at once, ring entries reused
    st, lat, m, stats = run(hqc, R, arr, streams=1, max_batch=32, max_queue=100, transfer=transfer)
    assert stats["rejected_queue"] > 0 and stats["completed"] + stats["rejected_queue"] == 1000
    assert set(np.unique(st)) <= {0, 3}
    assert (lat[st == 0] >= 0).all()
    for i in np.nonzero(st == 0)[0]:
        j = i % 200
        assert (m[R["m_off"][j]:R["m_off"][j + 1]] == R["want"][R["m_off"][j]:R["m_off"][j + 1]]).all()


def test_a_batch_past_its_stall_limit_ends_the_call_with_a_timeout(hqc):
    """A batch still incomplete stall_ms after its launch ends the call with
    HQC_ETIMEOUT; the batch in flight is waited for and freed, its requests
    are reported as still running, and the library keeps working.  A slow
    batch stands in for a stuck one: 32,768 HQC-5 requests in one batch
    need more than 1 ms for the upload of their 472 MB alone at the host
    link's rate, and about as long again to decrypt."""
    P = hqc.hqc_get_params(5)
    n, per = 32768, P.W_u_pitch + P.W_v
    wl = honest(5, 1, 1, first_ct=99000, tag=93)
    keys = [None, None, hqc.Keyset(5, wl.y)]
    words = torch.from_numpy(synth.words(n * per, tag=94).view(np.int64)).pin_memory()
    level = np.full(n, 5, np.int32)
    key = np.zeros(n, np.int32)
    woff = np.arange(n + 1, dtype=np.int64) * per
    moff = np.arange(n + 1, dtype=np.int64) * P.k
    with pytest.raises(hqc.HqcError) as info:
        hqc.hqc_serve_run(keys, level, key, woff, words, moff, np.zeros(n, np.int64), streams=1, max_batch=n,
                          budget_bytes=512 << 20, stall_ms=1)
    err = info.value
    assert err.code == hqc.HQC_ETIMEOUT and "did not complete" in str(err)
    st, lat, _, stats = err.partial
    assert (st == 2).all() and (lat == -1).all() and stats["completed"] == 0 and stats["batches"] == 1
    keys[2].free()
    # the same library and device serve a normal trace afterwards
    R = make_ring(hqc, 40, tag=5)
    st2, _, m2, stats2 = run(hqc, R, np.zeros(40, np.int64), streams=2)
    assert (st2 == 0).all() and (m2 == R["want"]).all() and stats2["completed"] == 40
