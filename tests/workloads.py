"""Seeded workloads for the tests: keys and ciphertexts built by the CPU
oracle from the synthetic input generator, plus adversarial variants.

Recipe (Table I sizes, Algorithms 1 and 3): per key h uniform over n bits,
x and y uniform weight-w supports, s = x + h*y; per ciphertext m uniform
over k bytes, r1, r2 weight w_r, e weight w_e, key (i mod nkeys) shuffled.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
import synth


@dataclass
class Workload:
    level: int
    P: object
    h: np.ndarray
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    key_idx: np.ndarray
    m: np.ndarray
    u: np.ndarray
    v: np.ndarray

    @property
    def y_rows(self):
        return self.y[self.key_idx]


def honest(level: int, nkeys: int, count: int, first_key: int = 0, first_ct: int = 0, tag: int = 0) -> Workload:
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, nkeys, first=first_key)
    s = oracle.keygen(level, h, x, y)
    m, r1, r2, e = synth.ciphertext_randomness(S, count, first=first_ct)
    kidx = synth.key_assignment(count, nkeys, tag=1000 + level + tag)
    u, v = oracle.encrypt(level, h, s, kidx, m, r1, r2, e)
    return Workload(level, P, h, x, y, s, kidx, m, u, v)


def with_garbage_padding(P, u: np.ndarray, tag: int) -> np.ndarray:
    """Random bits above bit n and in the pad word (they must be ignored)."""
    g = synth.words(u.size, tag=tag).reshape(u.shape)
    out = u.copy()
    nb = P.n % 64
    out[:, P.W_u - 1] |= g[:, P.W_u - 1] & np.uint64(((1 << 64) - 1) ^ ((1 << nb) - 1))
    out[:, P.W_u:] = g[:, P.W_u:]
    return out


def adversarial(level: int, tag: int = 0):
    """(u, v, y) rows that stress every branch-free path of the decoder:
    random v (far beyond delta errors), all-zero and all-one u, garbage
    padding, supports with repeats and entries >= n."""
    P = oracle.params(level)
    base = honest(level, 4, 8, tag=tag)
    rows_u, rows_v, rows_y = [], [], []
    nw = P.W_u_pitch
    full = np.zeros(nw, np.uint64)
    for i in range(P.n):
        full[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    for i in range(4):
        rows_u.append(base.u[i]); rows_v.append(synth.words(P.W_v, tag=50 + tag, index=i)); rows_y.append(base.y_rows[i])
    rows_u.append(np.zeros(nw, np.uint64)); rows_v.append(base.v[0]); rows_y.append(base.y_rows[0])
    rows_u.append(full.copy()); rows_v.append(base.v[1]); rows_y.append(base.y_rows[1])
    rows_u.append(with_garbage_padding(P, base.u[2:3], tag=60 + tag)[0]); rows_v.append(base.v[2]); rows_y.append(base.y_rows[2])
    dup = base.y_rows[3].copy(); dup[1] = dup[0]; dup[5] = dup[4]
    rows_u.append(base.u[3]); rows_v.append(base.v[3]); rows_y.append(dup)
    bad = base.y_rows[4].copy(); bad[0] = P.n; bad[2] = 0xFFFFFFFF; bad[3] = P.n + 12345
    rows_u.append(base.u[4]); rows_v.append(base.v[4]); rows_y.append(bad)
    rows_u.append(with_garbage_padding(P, base.u[5:6], tag=70 + tag)[0]); rows_v.append(synth.words(P.W_v, tag=80 + tag)); rows_y.append(base.y_rows[5])
    u = np.stack(rows_u); v = np.stack(rows_v); y = np.stack(rows_y).astype(np.uint32)
    # a few honest ciphertexts with heavy extra noise on some RM blocks
    extra = honest(level, 2, 6, first_ct=100, tag=tag + 7)
    vv = extra.v.copy()
    for i in range(6):
        nblocks = [P.delta - 1, P.delta, P.delta + 1, P.delta + 2, P.n1 // 2, 3][i]
        blocks = synth.support(P.n1, nblocks, tag=90 + tag, index=i)
        for j in blocks:
            lo = int(j) * P.n2 // 64
            vv[i, lo: lo + P.n2 // 64] ^= synth.words(P.n2 // 64, tag=95 + tag, index=i * 1000 + int(j))
    u = np.concatenate([u, extra.u]); v = np.concatenate([v, vv]); y = np.concatenate([y, extra.y_rows])
    return P, u, v, y


def noisy_keyed(level: int, nkeys: int, count: int, first_ct: int, tag: int):
    """Honest ciphertexts under nkeys valid keys, a fifth of them made hard:
    random v (far beyond delta errors), heavy noise on delta-1 .. n1/2 RM
    blocks, all-zero u, or garbage in u's padding.  Returns (workload, u, v);
    the supports stay valid, so the rows suit the keyed entry points."""
    wl = honest(level, nkeys, count, first_ct=first_ct, tag=tag)
    P = wl.P
    u, v = wl.u.copy(), wl.v.copy()
    for i in range(0, count, 5):
        kind = (i // 5) % 4
        if kind == 0:
            v[i] = synth.words(P.W_v, tag=tag + 1, index=i)
        elif kind == 1:
            nb = [P.delta - 1, P.delta, P.delta + 1, P.n1 // 2][(i // 20) % 4]
            for j in synth.support(P.n1, nb, tag=tag + 2, index=i):
                lo = int(j) * P.n2 // 64
                v[i, lo:lo + P.n2 // 64] ^= synth.words(P.n2 // 64, tag=tag + 3, index=i * 1000 + int(j))
        elif kind == 2:
            u[i] = 0
        else:
            u[i] = with_garbage_padding(P, u[i:i + 1], tag=tag + 4 + i)[0]
    return wl, u, v
