"""Seeded synthetic inputs for HQC.PKE (keys, messages, sparse supports).

Random numbers only -- this module holds none of the scheme's arithmetic, so
the CPU oracle (tests) and the CUDA library (tests, bench) can both consume
its output.  The C file ``synth.c`` does the drawing (SplitMix64 seeding,
xoshiro256** streams, rejection sampling); this module marshals numpy arrays.

Input recipe (Algorithms 1 and 3 of the paper, Table I sizes):
  * per key i: h uniform over n bits, x and y uniform weight-w supports;
  * per ciphertext j: m uniform over k bytes, r1 and r2 uniform weight-w_r
    supports, e a uniform weight-w_e support;
  * ciphertext j uses key (j mod nkeys), then the key order is shuffled with
    a seeded Fisher-Yates pass.
Every stream is keyed by (master seed, level, kind, index), so any item can
be regenerated on its own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 2512129040

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhqc_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u64, i64, c_int = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
            u32 = ctypes.c_uint32
            sig = {
                "synth_keys": [u64, c_int, i64, i64, c_int, c_int, c_int, P, P, P],
                "synth_ciphertexts": [u64, c_int, i64, i64, c_int, c_int, c_int, c_int, P, P, P, P],
                "synth_shuffle_i32": [u64, c_int, P, i64],
                "synth_words": [u64, c_int, u64, P, i64],
                "synth_below": [u64, c_int, u64, u32, P, i64],
                "synth_support": [u64, c_int, u64, u32, c_int, P],
                "synth_xoshiro_raw": [P, P, c_int],
                "synth_splitmix_raw": [u64, P, c_int],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.restype = None
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Shape:
    """Sizes the generator needs; filled from either side's parameter table."""
    level: int
    n: int
    k: int
    w: int
    wr: int
    we: int
    W_u_pitch: int

    @classmethod
    def of(cls, p) -> "Shape":
        return cls(level=int(p.level), n=int(p.n), k=int(p.k), w=int(p.w),
                   wr=int(p.wr), we=int(p.we), W_u_pitch=int(p.W_u_pitch))


def keys(shape: Shape, nkeys: int, first: int = 0, master: int = MASTER_SEED):
    """(h [nkeys][W_u_pitch] uint64, x [nkeys][w], y [nkeys][w] uint32)."""
    h = np.zeros((nkeys, shape.W_u_pitch), np.uint64)
    x = np.zeros((nkeys, shape.w), np.uint32)
    y = np.zeros((nkeys, shape.w), np.uint32)
    _load().synth_keys(master, shape.level, first, nkeys, shape.n, shape.w,
                       shape.W_u_pitch, _p(h), _p(x), _p(y))
    return h, x, y


def ciphertext_randomness(shape: Shape, count: int, first: int = 0,
                          master: int = MASTER_SEED):
    """(m [count][k] uint8, r1, r2 [count][wr], e [count][we] uint32)."""
    m = np.zeros((count, shape.k), np.uint8)
    r1 = np.zeros((count, shape.wr), np.uint32)
    r2 = np.zeros((count, shape.wr), np.uint32)
    e = np.zeros((count, shape.we), np.uint32)
    _load().synth_ciphertexts(master, shape.level, first, count, shape.n, shape.k,
                              shape.wr, shape.we, _p(m), _p(r1), _p(r2), _p(e))
    return m, r1, r2, e


def key_assignment(count: int, nkeys: int, tag: int, master: int = MASTER_SEED):
    """key_idx[j] = j mod nkeys, then a seeded shuffle."""
    idx = (np.arange(count, dtype=np.int64) % max(nkeys, 1)).astype(np.int32)
    if count > 1:
        _load().synth_shuffle_i32(master, tag, _p(idx), count)
    return idx


def shuffle(a: np.ndarray, tag: int, master: int = MASTER_SEED) -> np.ndarray:
    a = np.ascontiguousarray(a, np.int32).copy()
    if a.size > 1:
        _load().synth_shuffle_i32(master, tag, _p(a), a.size)
    return a


def words(n_words: int, tag: int, index: int = 0, master: int = MASTER_SEED) -> np.ndarray:
    out = np.zeros(n_words, np.uint64)
    if n_words:
        _load().synth_words(master, tag, index, _p(out), n_words)
    return out


def below(n: int, length: int, tag: int, index: int = 0, master: int = MASTER_SEED) -> np.ndarray:
    out = np.zeros(length, np.uint32)
    if length:
        _load().synth_below(master, tag, index, n, _p(out), length)
    return out


def support(n: int, w: int, tag: int, index: int = 0, master: int = MASTER_SEED) -> np.ndarray:
    out = np.zeros(w, np.uint32)
    _load().synth_support(master, tag, index, n, w, _p(out))
    return out


def xoshiro_raw(state, length: int) -> np.ndarray:
    s = np.ascontiguousarray(np.asarray(state, np.uint64))
    out = np.zeros(length, np.uint64)
    _load().synth_xoshiro_raw(_p(s), _p(out), length)
    return out


def splitmix_raw(seed: int, length: int) -> np.ndarray:
    out = np.zeros(length, np.uint64)
    _load().synth_splitmix_raw(seed, _p(out), length)
    return out


def burst_trace(rate_per_s: float, duration_s: float, tag: int, max_burst: int = 512,
                master: int = MASTER_SEED) -> np.ndarray:
    """Open-loop arrival times (ns, non-decreasing) of single requests.

    Bursts arrive as a Poisson process; a burst carries B requests with B a
    log-uniform integer in [1, max_burst] (B = floor(exp(U ln(max_burst+1))),
    U uniform in [0, 1)), all with the burst's arrival time.  The burst rate
    is rate_per_s / E[B], so requests arrive at rate_per_s on average."""
    ln = np.log(max_burst + 1.0)
    b = np.arange(1, max_burst + 1, dtype=np.float64)
    mean_b = float(((np.log(b + 1) - np.log(b)) / ln * b).sum())
    n_bursts = max(1, int(rate_per_s * duration_s / mean_b * 1.2) + 16)
    u = (words(2 * n_bursts, tag=tag, index=1, master=master) >> np.uint64(11)).astype(np.float64) / 2.0 ** 53
    gaps = -np.log1p(-u[:n_bursts]) / (rate_per_s / mean_b)
    sizes = np.floor(np.exp(u[n_bursts:] * ln)).astype(np.int64).clip(1, max_burst)
    t = np.cumsum(gaps)
    keep = t < duration_s
    t, sizes = t[keep], sizes[keep]
    return np.repeat((t * 1e9).astype(np.int64), sizes)


def level_mix(n: int, shares, tag: int, master: int = MASTER_SEED) -> np.ndarray:
    """n levels drawn with the given {level: share} weights, shuffled."""
    levels = []
    for lvl, share in shares:
        levels += [lvl] * int(round(n * share))
    levels = np.array((levels + [shares[0][0]] * n)[:n], np.int32)
    return shuffle(levels, tag=tag, master=master)
