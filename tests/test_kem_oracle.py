"""Pins of the KEM oracle (kem_oracle.c): SHAKE256 against Python's
hashlib (an independent FIPS 202 implementation), the fixed-weight sampler
against Floyd's uniformity theorem by exhaustive enumeration, and the KEM
readings A19-A22 assembled from those pinned parts."""
import hashlib
import itertools
from collections import Counter

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("length", [0, 1, 31, 32, 135, 136, 137, 271, 272, 273, 4450])
def test_shake256_matches_hashlib(length):
    msg = synth.words((length + 7) // 8 + 1, tag=77, index=length).tobytes()[:length]
    for outlen in (1, 32, 135, 136, 137, 1200):
        assert oracle.shake256(msg, outlen) == hashlib.shake_256(msg).digest(outlen), (length, outlen)


def test_keccak_permutation_is_the_one_inside_shake():
    # one block: the output of SHAKE256("") is the permuted padded block
    st = bytearray(200)
    st[0] ^= 0x1F
    st[135] ^= 0x80
    assert oracle.keccak_f1600(bytes(st))[:136] == hashlib.shake_256(b"").digest(136)
    # squeezing: the next 136 bytes are one more permutation of that state
    s1 = oracle.keccak_f1600(bytes(st))
    assert oracle.keccak_f1600(s1)[:136] == hashlib.shake_256(b"").digest(272)[136:]


def _draw_for(t, span):
    """A 32-bit word R with floor(R * span / 2^32) = t."""
    R = -(-(t << 32) // span)
    assert (R * span) >> 32 == t and R < 2 ** 32
    return R


@pytest.mark.parametrize("n,w", [(5, 2), (7, 3), (8, 4), (9, 2)])
def test_fixed_weight_is_uniform_over_subsets(n, w):
    """Floyd: with uniform draws every w-subset comes out equally often."""
    counts = Counter()
    for ts in itertools.product(*[range(n - i) for i in range(w)]):
        R = [_draw_for(t, n - i) for i, t in enumerate(ts)]
        pos = oracle.fixed_weight(n, w, R)
        assert len(set(pos.tolist())) == w and pos.max() < n
        counts[tuple(sorted(pos.tolist()))] += 1
    total = int(np.prod([n - i for i in range(w)]))
    from math import comb
    assert len(counts) == comb(n, w)
    assert set(counts.values()) == {total // comb(n, w)}


@pytest.mark.parametrize("level", [1, 3, 5])
def test_fixed_weight_full_size_invariants(level):
    P = oracle.params(level)
    for idx in range(20):
        R = synth.words(P.we, tag=91, index=idx).astype(np.uint32)
        pos = oracle.fixed_weight(P.n, P.we, R)
        assert len(set(pos.tolist())) == P.we and int(pos.max()) < P.n
    # all-equal draws force the collision rule on every entry but the last
    pos = oracle.fixed_weight(P.n, P.w, np.zeros(P.w, np.uint32))
    assert pos.tolist() == list(range(P.w))


def _words_le(b):
    return np.frombuffer(b, "<u4").astype(np.uint32)


def _seeds(nkeys, tag):
    return (synth.words(4 * nkeys, tag=tag).view(np.uint8).reshape(nkeys, 32).copy(),
            synth.words(4 * nkeys, tag=tag + 1).view(np.uint8).reshape(nkeys, 32).copy())


@pytest.mark.parametrize("level", [1, 3, 5])
def test_kem_readings_from_pinned_parts(level):
    P = oracle.params(level)
    sk, pk = _seeds(2, tag=300 + level)
    h, x, y, s = oracle.kem_keygen(level, sk, pk)
    # A22: h from the seed_pk stream, x / y through the sampler, s = x + h y
    hb = hashlib.shake_256(pk[1].tobytes() + b"\x02").digest(8 * P.W_u)
    hw = np.frombuffer(hb, "<u8").copy()
    if P.n % 64:
        hw[-1] &= np.uint64((1 << (P.n % 64)) - 1)
    assert (h[1, :P.W_u] == hw).all() and (h[1, P.W_u:] == 0).all()
    R = _words_le(hashlib.shake_256(sk[1].tobytes() + b"\x01").digest(8 * P.w))
    assert (x[1] == oracle.fixed_weight(P.n, P.w, R[:P.w])).all()
    assert (y[1] == oracle.fixed_weight(P.n, P.w, R[P.w:])).all()
    assert (s == oracle.keygen(level, h, x, y)).all()
    # A19 / A18
    m = synth.words(4, tag=310 + level).view(np.uint8)[:P.k].copy()
    salt = synth.words(2, tag=320 + level).view(np.uint8).copy()
    theta = oracle.kem_theta(level, m.tobytes(), salt.tobytes())
    assert theta == hashlib.shake_256(m.tobytes() + salt.tobytes() + b"\x03").digest(32)
    r1, r2, e = oracle.kem_randomness(level, theta)
    Rr = _words_le(hashlib.shake_256(theta + b"\x01").digest(4 * (2 * P.wr + P.we)))
    assert (r1 == oracle.fixed_weight(P.n, P.wr, Rr[:P.wr])).all()
    assert (r2 == oracle.fixed_weight(P.n, P.wr, Rr[P.wr:2 * P.wr])).all()
    assert (e == oracle.fixed_weight(P.n, P.we, Rr[2 * P.wr:])).all()
    # Encaps = Encrypt with that randomness, K over the canonical bytes (A20)
    kidx = np.array([1], np.int32)
    u, v, K = oracle.kem_encaps(level, h, s, kidx, m[None], salt[None])
    u2, v2 = oracle.encrypt(level, h, s, kidx, m[None], r1[None], r2[None], e[None])
    assert (u == u2).all() and (v == v2).all()
    U = u[0].tobytes()[:(P.n + 7) // 8]
    V = v[0].tobytes()
    assert K[0].tobytes() == hashlib.shake_256(m.tobytes() + U + V + salt.tobytes() + b"\x04").digest(32)


@pytest.mark.parametrize("level", [1, 3, 5])
def test_decaps_accepts_honest_and_rejects_implicitly(level):
    P = oracle.params(level)
    sk, pk = _seeds(3, tag=400 + level)
    h, x, y, s = oracle.kem_keygen(level, sk, pk)
    sigma = synth.words(3 * 4, tag=410 + level).view(np.uint8).reshape(3, 32)[:, :P.k].copy()
    cnt = 6
    kidx = (np.arange(cnt) % 3).astype(np.int32)
    m = synth.words(cnt * 4, tag=420 + level).view(np.uint8).reshape(cnt, 32)[:, :P.k].copy()
    salt = synth.words(cnt * 2, tag=430 + level).view(np.uint8).reshape(cnt, 16).copy()
    u, v, K = oracle.kem_encaps(level, h, s, kidx, m, salt)
    Kd, ok = oracle.kem_decaps(level, h, s, y, sigma, kidx, u, v, salt)
    assert ok.all() and (Kd == K).all()
    # padding bits of u do not change anything
    ug = u.copy()
    ug[:, P.W_u - 1] |= np.uint64(~((1 << (P.n % 64)) - 1) & (2 ** 64 - 1))
    ug[:, P.W_u:] = np.uint64(0x5A5A5A5A5A5A5A5A)
    Kg, okg = oracle.kem_decaps(level, h, s, y, sigma, kidx, ug, v, salt)
    assert okg.all() and (Kg == K).all()
    # tampering: one flipped bit of v (still decodes to m, re-encryption differs),
    # another salt, a ciphertext under the wrong key
    vt = v.copy()
    vt[:, 3] ^= np.uint64(1 << 5)
    Kt, okt = oracle.kem_decaps(level, h, s, y, sigma, kidx, u, vt, salt)
    assert not okt.any()
    for i in range(cnt):
        U = u[i].tobytes()[:(P.n + 7) // 8]
        want = hashlib.shake_256(sigma[kidx[i]].tobytes() + U + vt[i].tobytes() + salt[i].tobytes()
                                 + b"\x04").digest(32)
        assert Kt[i].tobytes() == want
    st = salt.copy()
    st[:, 0] ^= 1
    _, oks = oracle.kem_decaps(level, h, s, y, sigma, kidx, u, v, st)
    assert not oks.any()
    _, okk = oracle.kem_decaps(level, h, s, y, sigma, (kidx + 1) % 3, u, v, salt)
    assert not okk.any()


def test_fixed_weight_full_size_marginals_are_uniform():
    """At full size (HQC-1, w_e = 75 of n = 17,669) every position is in the
    support with probability w / n: over 3,000 supports drawn from seeded
    32-bit words, the counts in 32 equal bins pass a chi-square test, and
    both ends of [0, n) occur (an off-by-one in pos_i = i + floor(R_i (n - i)
    / 2^32) would lose n - 1 or shift mass between the bins)."""
    from scipy.stats import chi2
    P = oracle.params(1)
    n, w, trials = P.n, P.we, 3000
    counts = np.zeros(n, np.int64)
    for idx in range(trials):
        R = synth.words(w, tag=93, index=idx).astype(np.uint32)
        counts[oracle.fixed_weight(n, w, R)] += 1
    assert counts.sum() == trials * w
    assert counts[0] > 0 and counts[n - 1] > 0
    edges = np.linspace(0, n, 33).astype(np.int64)
    observed = np.array([counts[a:b].sum() for a, b in zip(edges[:-1], edges[1:])], np.float64)
    expected = trials * w * np.diff(edges) / n
    stat = float(((observed - expected) ** 2 / expected).sum())
    assert chi2.sf(stat, df=31) > 1e-4, stat
