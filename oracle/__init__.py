"""CPU oracle for batched HQC.PKE decryption -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The CUDA library never calls it
and has no CPU fallback.

This module is argument marshalling around ``hqc_oracle.c`` (plain C, built
with gcc on first use).  Every function cites the paper passage it follows;
the arithmetic itself lives in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hqc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "kem_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhqc_oracle.so")
_lock = threading.Lock()
_lib = None

LEVELS = (1, 3, 5)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libhqc_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread"] + _SRCS + ["-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            sig = {
                "oracle_params": (ctypes.c_int, [ctypes.c_int, P]),
                "oracle_gf_mul": (ctypes.c_uint8, [ctypes.c_uint8, ctypes.c_uint8]),
                "oracle_rs_generator": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P]),
                "oracle_rs_encode": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P]),
                "oracle_rs_syndromes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P]),
                "oracle_rs_decode": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P]),
                "oracle_rm_encode_byte": (None, [ctypes.c_uint8, P]),
                "oracle_rm_transform": (None, [ctypes.c_int, P, P]),
                "oracle_rm_decode_block": (ctypes.c_uint8, [ctypes.c_int, P]),
                "oracle_ring_mul_sparse": (None, [ctypes.c_int, P, P, ctypes.c_int, P]),
                "oracle_ring_mul_packed": (None, [ctypes.c_int, P, P, ctypes.c_int, P]),
                "oracle_keygen_batch": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, ctypes.c_int]),
                "oracle_encrypt_batch": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, P, P, P, P, P, ctypes.c_int]),
                "oracle_decrypt_batch": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, ctypes.c_int]),
                "oracle_decrypt_dump": (ctypes.c_int, [ctypes.c_int] + [P] * 14),
                "oracle_concat_encode": (ctypes.c_int, [ctypes.c_int, P, P]),
                "oracle_keccak_f1600": (None, [P]),
                "oracle_shake256": (None, [P, i64, P, i64]),
                "oracle_fixed_weight": (None, [ctypes.c_int, ctypes.c_int, P, P]),
                "oracle_kem_theta": (None, [ctypes.c_int, P, P, P]),
                "oracle_kem_randomness": (ctypes.c_int, [ctypes.c_int, P, P, P, P]),
                "oracle_kem_keygen": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, P, P]),
                "oracle_kem_encaps": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, P, P, P, P]),
                "oracle_kem_decaps": (ctypes.c_int, [ctypes.c_int, i64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            del i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


# --------------------------------------------------------------------------
# Parameters (Table I)
# --------------------------------------------------------------------------
class Params:
    """Table I row plus derived sizes, as the oracle computes them."""

    def __init__(self, level: int):
        out = np.zeros(9, np.int32)
        if _load().oracle_params(level, _p(out)) != 0:
            raise ValueError("unknown HQC level %r" % (level,))
        (self.n, self.w, self.wr, self.we, self.n1, self.k, self.delta,
         self.n2, self.mult) = (int(x) for x in out)
        self.level = level
        self.W_u = (self.n + 63) // 64
        self.W_u_pitch = self.W_u + (self.W_u & 1)
        self.W_v = (self.n1 * self.n2 + 63) // 64


def params(level: int) -> Params:
    return Params(level)


# --------------------------------------------------------------------------
# GF(2^8), RS, RM pieces (Sec. II-A, Sec. III-D; readings A3-A11)
# --------------------------------------------------------------------------
def gf_mul(a: int, b: int) -> int:
    """GF(2^8) product modulo x^8+x^4+x^3+x^2+1 (reading A3)."""
    return int(_load().oracle_gf_mul(a, b))


def rs_generator(n1: int, k: int) -> np.ndarray:
    """g(x) = prod_{i=1}^{n1-k} (x - alpha^i), coefficients low to high (A4)."""
    g = np.zeros(n1 - k + 1, np.uint8)
    assert _load().oracle_rs_generator(n1, k, _p(g)) == 0
    return g


def rs_encode(n1: int, k: int, m: np.ndarray) -> np.ndarray:
    """Systematic RS codeword (parity || m), reading A6."""
    m = np.ascontiguousarray(m, np.uint8)
    c = np.zeros(n1, np.uint8)
    assert _load().oracle_rs_encode(n1, k, _p(m), _p(c)) == 0
    return c


def rs_syndromes(n1: int, k: int, r: np.ndarray) -> np.ndarray:
    """S_1..S_{n1-k} of a received word (Sec. III-D)."""
    r = np.ascontiguousarray(r, np.uint8)
    S = np.zeros(n1 - k, np.uint8)
    _load().oracle_rs_syndromes(n1, k, _p(r), _p(S))
    return S


def rs_decode(n1: int, k: int, r: np.ndarray) -> dict:
    """BM + Chien + Forney decode of one received word (readings A9-A11)."""
    r = np.ascontiguousarray(r, np.uint8)
    nr = n1 - k
    S = np.zeros(nr, np.uint8)
    lam = np.zeros(nr + 1, np.uint8)
    L = np.zeros(1, np.int32)
    em = np.zeros(n1, np.uint8)
    ev = np.zeros(n1, np.uint8)
    cw = np.zeros(n1, np.uint8)
    fl = np.zeros(1, np.int32)
    assert _load().oracle_rs_decode(n1, k, _p(r), _p(S), _p(lam), _p(L), _p(em),
                                    _p(ev), _p(cw), _p(fl)) == 0
    return dict(S=S, lam=lam, L=int(L[0]), errmask=em, errval=ev, cw=cw,
                flag=int(fl[0]))


def rm_encode_byte(b: int) -> np.ndarray:
    """128 codeword bits of one byte (reading A7)."""
    bits = np.zeros(128, np.uint8)
    _load().oracle_rm_encode_byte(b, _p(bits))
    return bits


def rm_transform(mult: int, bits: np.ndarray) -> np.ndarray:
    """F(a) = sum_i s_i (-1)^{<a,i>} from its definition (Sec. II-A)."""
    bits = np.ascontiguousarray(bits, np.uint8)
    assert bits.size == 128 * mult
    F = np.zeros(128, np.int32)
    _load().oracle_rm_transform(mult, _p(bits), _p(F))
    return F


def rm_decode_block(mult: int, bits: np.ndarray) -> int:
    """Byte decoded from 128*mult received bits (reading A8)."""
    bits = np.ascontiguousarray(bits, np.uint8)
    assert bits.size == 128 * mult
    return int(_load().oracle_rm_decode_block(mult, _p(bits)))


# --------------------------------------------------------------------------
# Ring product (Eq. 1)
# --------------------------------------------------------------------------
def ring_mul_sparse_bits(n: int, a2_bits: np.ndarray, supp) -> np.ndarray:
    """XOR of x^p * a2 over p in supp, on unpacked bits (Eq. 1)."""
    a2 = np.ascontiguousarray(a2_bits, np.uint8)
    s = np.ascontiguousarray(np.asarray(supp, np.uint32))
    out = np.zeros(n, np.uint8)
    _load().oracle_ring_mul_sparse(n, _p(a2), _p(s), int(s.size), _p(out))
    return out


def ring_mul_packed(n: int, a2_words: np.ndarray, supp) -> np.ndarray:
    """Eq. 1 on packed LSB-first words (reading A5); ceil(n/64) words out."""
    a2 = np.ascontiguousarray(a2_words, np.uint64)
    s = np.ascontiguousarray(np.asarray(supp, np.uint32))
    out = np.zeros((n + 63) // 64, np.uint64)
    _load().oracle_ring_mul_packed(n, _p(a2), _p(s), int(s.size), _p(out))
    return out


# --------------------------------------------------------------------------
# PKE (Algorithms 1-3)
# --------------------------------------------------------------------------
def keygen(level: int, h: np.ndarray, x: np.ndarray, y: np.ndarray,
           nthreads=None) -> np.ndarray:
    """s = x + h*y for each key (Algorithm 3 core).  h: [nkeys][W_u_pitch]."""
    P = Params(level)
    h = np.ascontiguousarray(h, np.uint64)
    x = np.ascontiguousarray(x, np.uint32)
    y = np.ascontiguousarray(y, np.uint32)
    nk = h.shape[0]
    assert h.shape == (nk, P.W_u_pitch) and x.shape == (nk, P.w) and y.shape == (nk, P.w)
    s = np.zeros_like(h)
    assert _load().oracle_keygen_batch(level, nk, _p(h), _p(x), _p(y), _p(s),
                                       _threads(nthreads)) == 0
    return s


def encrypt(level: int, h: np.ndarray, s: np.ndarray, key_idx: np.ndarray,
            m: np.ndarray, r1: np.ndarray, r2: np.ndarray, e: np.ndarray,
            nthreads=None):
    """(u, v) per ciphertext (Algorithm 1, v truncated per reading A2)."""
    P = Params(level)
    h = np.ascontiguousarray(h, np.uint64)
    s = np.ascontiguousarray(s, np.uint64)
    key_idx = np.ascontiguousarray(key_idx, np.int32)
    m = np.ascontiguousarray(m, np.uint8)
    r1 = np.ascontiguousarray(r1, np.uint32)
    r2 = np.ascontiguousarray(r2, np.uint32)
    e = np.ascontiguousarray(e, np.uint32)
    cnt = m.shape[0]
    assert m.shape == (cnt, P.k) and r1.shape == (cnt, P.wr) and r2.shape == (cnt, P.wr)
    assert e.shape == (cnt, P.we) and key_idx.shape == (cnt,)
    assert key_idx.size == 0 or (key_idx.min() >= 0 and key_idx.max() < h.shape[0])
    u = np.zeros((cnt, P.W_u_pitch), np.uint64)
    v = np.zeros((cnt, P.W_v), np.uint64)
    assert _load().oracle_encrypt_batch(level, cnt, _p(h), _p(s), _p(key_idx), _p(m),
                                        _p(r1), _p(r2), _p(e), _p(u), _p(v),
                                        _threads(nthreads)) == 0
    return u, v


def decrypt(level: int, u: np.ndarray, v: np.ndarray, y: np.ndarray,
            nthreads=None) -> np.ndarray:
    """m' per ciphertext (Algorithm 2 with reading A1); y: [count][w]."""
    P = Params(level)
    u = np.ascontiguousarray(u, np.uint64)
    v = np.ascontiguousarray(v, np.uint64)
    y = np.ascontiguousarray(y, np.uint32)
    cnt = u.shape[0]
    assert u.shape == (cnt, P.W_u_pitch) and v.shape == (cnt, P.W_v) and y.shape == (cnt, P.w)
    m = np.zeros((cnt, P.k), np.uint8)
    assert _load().oracle_decrypt_batch(level, cnt, _p(u), _p(v), _p(y), _p(m),
                                        _threads(nthreads)) == 0
    return m


def decrypt_dump(level: int, u: np.ndarray, v: np.ndarray, y: np.ndarray) -> dict:
    """Every intermediate of Algorithm 2 for ONE ciphertext.

    Keys: t, w (W_v words), r (n1 bytes), S (2 delta), lam (2 delta + 1),
    L, errmask, errval, cw (n1 each), m (k), flag.
    """
    P = Params(level)
    u = np.ascontiguousarray(u, np.uint64).reshape(P.W_u_pitch)
    v = np.ascontiguousarray(v, np.uint64).reshape(P.W_v)
    y = np.ascontiguousarray(y, np.uint32).reshape(P.w)
    nr = 2 * P.delta
    d = dict(t=np.zeros(P.W_v, np.uint64), w=np.zeros(P.W_v, np.uint64),
             r=np.zeros(P.n1, np.uint8), S=np.zeros(nr, np.uint8),
             lam=np.zeros(nr + 1, np.uint8), L=np.zeros(1, np.int32),
             errmask=np.zeros(P.n1, np.uint8), errval=np.zeros(P.n1, np.uint8),
             cw=np.zeros(P.n1, np.uint8), m=np.zeros(P.k, np.uint8),
             flag=np.zeros(1, np.int32))
    order = ["t", "w", "r", "S", "lam", "L", "errmask", "errval", "cw", "m", "flag"]
    assert _load().oracle_decrypt_dump(level, _p(u), _p(v), _p(y),
                                       *[_p(d[k]) for k in order]) == 0
    d["L"] = int(d["L"][0])
    d["flag"] = int(d["flag"][0])
    return d


def concat_encode(level: int, m: np.ndarray) -> np.ndarray:
    """C.Encode(m) as W_v packed words (Sec. II-A, readings A6-A7)."""
    P = Params(level)
    m = np.ascontiguousarray(m, np.uint8).reshape(P.k)
    out = np.zeros(P.W_v, np.uint64)
    assert _load().oracle_concat_encode(level, _p(m), _p(out)) == 0
    return out


# --------------------------------------------------------------------------
# SHAKE256, fixed-weight sampling and the KEM (kem_oracle.c, readings A16-A22)
# --------------------------------------------------------------------------
def keccak_f1600(state: bytes) -> bytes:
    """Keccak-f[1600] on a 200-byte state (FIPS 202 Sec. 3)."""
    st = np.frombuffer(bytes(state), np.uint8).copy()
    assert st.size == 200
    _load().oracle_keccak_f1600(_p(st))
    return st.tobytes()


def shake256(msg: bytes, outlen: int) -> bytes:
    """SHAKE256 (FIPS 202 Sec. 6.2, reading A16)."""
    m = np.frombuffer(bytes(msg) + b"\0", np.uint8).copy()
    out = np.zeros(max(outlen, 1), np.uint8)
    _load().oracle_shake256(_p(m), len(msg), _p(out), outlen)
    return out[:outlen].tobytes()


def fixed_weight(n: int, w: int, R) -> np.ndarray:
    """Floyd / Sendrier constant-weight sampler on 32-bit draws (A17)."""
    R = np.ascontiguousarray(R, np.uint32)
    assert R.size == w
    pos = np.zeros(w, np.uint32)
    _load().oracle_fixed_weight(n, w, _p(R), _p(pos))
    return pos


def kem_theta(level: int, m: bytes, salt: bytes) -> bytes:
    """theta = G(m, salt) (A19)."""
    P = params(level)
    mm = np.frombuffer(bytes(m), np.uint8).copy()
    ss = np.frombuffer(bytes(salt), np.uint8).copy()
    assert mm.size == P.k and ss.size == 16
    th = np.zeros(32, np.uint8)
    _load().oracle_kem_theta(P.k, _p(mm), _p(ss), _p(th))
    return th.tobytes()


def kem_randomness(level: int, theta: bytes):
    """(r1, r2, e) supports drawn from theta (A17, A18)."""
    P = params(level)
    th = np.frombuffer(bytes(theta), np.uint8).copy()
    r1 = np.zeros(P.wr, np.uint32)
    r2 = np.zeros(P.wr, np.uint32)
    e = np.zeros(P.we, np.uint32)
    assert _load().oracle_kem_randomness(level, _p(th), _p(r1), _p(r2), _p(e)) == 0
    return r1, r2, e


def kem_keygen(level: int, seed_sk: np.ndarray, seed_pk: np.ndarray):
    """(h, x, y, s) from 32-byte seeds [nkeys][32] (A22, Algorithm 3)."""
    P = params(level)
    seed_sk = np.ascontiguousarray(seed_sk, np.uint8)
    seed_pk = np.ascontiguousarray(seed_pk, np.uint8)
    nk = seed_sk.shape[0]
    h = np.zeros((nk, P.W_u_pitch), np.uint64)
    s = np.zeros((nk, P.W_u_pitch), np.uint64)
    x = np.zeros((nk, P.w), np.uint32)
    y = np.zeros((nk, P.w), np.uint32)
    assert _load().oracle_kem_keygen(level, nk, _p(seed_sk), _p(seed_pk), _p(h), _p(x), _p(y), _p(s)) == 0
    return h, x, y, s


def kem_encaps(level: int, h, s, key_idx, m, salt):
    """(u, v, K) per item (A18-A20, Algorithm 1)."""
    P = params(level)
    key_idx = np.ascontiguousarray(key_idx, np.int32)
    m = np.ascontiguousarray(m, np.uint8)
    salt = np.ascontiguousarray(salt, np.uint8)
    cnt = key_idx.size
    u = np.zeros((cnt, P.W_u_pitch), np.uint64)
    v = np.zeros((cnt, P.W_v), np.uint64)
    K = np.zeros((cnt, 32), np.uint8)
    assert _load().oracle_kem_encaps(level, cnt, _p(np.ascontiguousarray(h, np.uint64)),
                                     _p(np.ascontiguousarray(s, np.uint64)), _p(key_idx), _p(m), _p(salt),
                                     _p(u), _p(v), _p(K)) == 0
    return u, v, K


def kem_decaps(level: int, h, s, y, sigma, key_idx, u, v, salt, nthreads=1):
    """(K, ok) per item: decrypt, re-encrypt, compare, implicit rejection (A21)."""
    P = params(level)
    key_idx = np.ascontiguousarray(key_idx, np.int32)
    cnt = key_idx.size
    K = np.zeros((cnt, 32), np.uint8)
    ok = np.zeros(cnt, np.int32)
    args = [np.ascontiguousarray(h, np.uint64), np.ascontiguousarray(s, np.uint64), np.ascontiguousarray(y, np.uint32),
            np.ascontiguousarray(sigma, np.uint8), key_idx, np.ascontiguousarray(u, np.uint64),
            np.ascontiguousarray(v, np.uint64), np.ascontiguousarray(salt, np.uint8)]
    assert _load().oracle_kem_decaps(level, cnt, *[_p(a) for a in args], _p(K), _p(ok), int(nthreads)) == 0
    return K, ok.astype(bool)
