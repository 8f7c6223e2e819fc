"""Python binding of the GB300 batched HQC.PKE library (include/hqc_gb300.h).

Argument marshalling only: every function below checks tensor dtypes,
shapes and devices, then calls the C entry point of the same name in
``libhqc_gb300.so``.  PyTorch supplies device memory and streams; all
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback:
without the compiled library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import functools
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = [
    "HqcError", "Params", "Keyset", "load", "hqc_get_params", "hqc_decrypt_batch",
    "hqc_keys_register", "hqc_decrypt_batch_keyed", "hqc_staged_workspace_bytes",
    "hqc_decrypt_batch_staged", "hqc_decrypt_batch_staged_noalloc", "hqc_decrypt_debug", "hqc_mixed_workspace_bytes",
    "hqc_decrypt_mixed", "hqc_set_launch_config", "hqc_get_launch_shape", "hqc_keygen_batch",
    "hqc_encrypt_batch", "hqc_count_bad_key_idx", "hqc_rm_decode_batch", "hqc_rm_tc_timeouts", "hqc_decrypt_debug_team", "LEVELS", "Plan", "PLAN_VARIANTS", "PLAN_FORMS", "hqc_plan_create_keyed", "hqc_plan_create_mixed", "hqc_serve_run",
    "SERVE_STATUS", "hqc_decrypt_host_keyed", "hqc_host_workspace_bytes", "hqc_shake256_batch",
    "hqc_kem_keygen", "hqc_kem_workspace_bytes", "hqc_kem_encaps", "hqc_kem_decaps",
    "hqc_kem_host_workspace_bytes", "hqc_kem_decaps_host", "hqc_mixed_host_workspace_bytes",
    "hqc_decrypt_mixed_host", "HQC_OK", "HQC_EINVAL", "HQC_ENOMEM", "HQC_ECUDA", "HQC_ETIMEOUT", "HQC_EBUSY",
    "HQC_EINTERNAL",
]

LEVELS = (1, 3, 5)
_lock = threading.Lock()
_lib = None


HQC_OK, HQC_EINVAL, HQC_ENOMEM, HQC_ECUDA, HQC_ETIMEOUT, HQC_EBUSY, HQC_EINTERNAL = 0, -1, -2, -3, -4, -5, -6


class HqcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("HQC error %d: %s" % (code, msg))
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("level", "n", "n1", "k", "delta", "n2", "mult", "w", "wr", "we", "W_u", "W_u_pitch", "W_v")]


class _Dump(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("t", "w", "r", "S", "lam", "L", "errmask", "errval", "cw", "flag")]


class _LaunchCfg(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


ITEM_DTYPE = np.dtype([("level", "<i4"), ("key", "<i4"), ("u_off", "<i8"), ("v_off", "<i8"), ("m_off", "<i8")])


def load(build_if_missing: bool = True):
    """Load libhqc_gb300.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libhqc_gb300.so is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "hqc_get_params": (i32, [i32, P]),
            "hqc_last_error": (ctypes.c_char_p, []),
            "hqc_decrypt_batch": (i32, [i32, i64, P, P, P, P, P]),
            "hqc_keys_register": (i32, [i32, i64, P, P]),
            "hqc_keys_free": (i32, [P]),
            "hqc_keys_info": (i32, [P, P, P, P]),
            "hqc_decrypt_batch_keyed": (i32, [i32, i64, P, P, P, P, P, P]),
            "hqc_staged_workspace_bytes": (sz, [i32, i64]),
            "hqc_decrypt_batch_staged": (i32, [i32, i64, P, P, P, P, P, P, sz, P, P]),
            "hqc_decrypt_batch_staged_noalloc": (i32, [i32, i64, P, P, P, P, P, P, P]),
            "hqc_decrypt_debug": (i32, [i32, i64, P, P, P, P, P, P]),
            "hqc_mixed_workspace_bytes": (sz, []),
            "hqc_decrypt_mixed": (i32, [i64, P, P, i64, P, P, i64, P, sz, P]),
            "hqc_set_launch_config": (i32, [i32, P]),
            "hqc_get_launch_shape": (i32, [i32, i32, P, P, P]),
            "hqc_plan_create_keyed": (i32, [i32, i64, P, P, P, P, P, i32, P, P]),
            "hqc_plan_create_mixed": (i32, [i64, P, P, i64, P, P, i64, i32, P, P]),
            "hqc_plan_launch": (i32, [P, P]),
            "hqc_plan_info": (i32, [P, P, P, P, P]),
            "hqc_plan_destroy": (i32, [P]),
            "hqc_serve_run": (i32, [P, P, P, i64, P, P, P, P, P]),
            "hqc_host_workspace_bytes": (sz, [i32, i64]),
            "hqc_decrypt_host_keyed": (i32, [i32, i64, P, P, P, P, P, i64, P, sz, P]),
            "hqc_shake256_batch": (i32, [i64, P, i32, P, i32, P]),
            "hqc_kem_keygen": (i32, [i32, i64, P, P, P, P, P, P, P]),
            "hqc_kem_workspace_bytes": (sz, [i32, i64]),
            "hqc_kem_encaps": (i32, [i32, i64, P, P, i64, P, P, P, P, P, P, P, sz, P]),
            "hqc_kem_decaps": (i32, [i32, i64, P, P, P, P, P, P, P, P, P, P, P, sz, P]),
            "hqc_kem_host_workspace_bytes": (sz, [i32, i64]),
            "hqc_mixed_host_workspace_bytes": (sz, [i64, P, i64]),
            "hqc_decrypt_mixed_host": (i32, [i64, P, P, i64, P, P, i64, i64, P, sz, P]),
            "hqc_kem_decaps_host": (i32, [i32, i64, P, P, P, P, P, P, P, P, P, P, i64, P, sz, P]),
            "hqc_keygen_batch": (i32, [i32, i64, P, P, P, P, P]),
            "hqc_count_bad_key_idx": (i32, [i64, P, i64, P, P]),
            "hqc_rm_decode_batch": (i32, [i32, i64, P, P, i32, P]),
            "hqc_rm_tc_timeouts": (i32, [P]),
            "hqc_decrypt_debug_team": (i32, [i32, i32, i64, P, P, P, P, P, P]),
            "hqc_plan_describe": (i32, [P, P, sz]),
            "hqc_plan_create_keyed_fixed": (i32, [i32, i64, P, P, P, P, P, i32, P, P, P]),
            "hqc_plan_create_mixed_fixed": (i32, [i64, P, P, i64, P, P, i64, i32, P, P, P, P, P]),
            "hqc_encrypt_batch": (i32, [i32, i64, P, P, i64, P, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise HqcError(rc, load().hqc_last_error().decode(errors="replace"))


# ---------------------------------------------------------------------------
# marshalling helpers (torch is imported lazily so the CPU tests can load
# the library without touching CUDA)
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _dev_ptr(t, dtype, shape=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s (got %s)" % (name, tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


@dataclass(frozen=True)
class Params:
    level: int
    n: int
    n1: int
    k: int
    delta: int
    n2: int
    mult: int
    w: int
    wr: int
    we: int
    W_u: int
    W_u_pitch: int
    W_v: int


@functools.lru_cache(maxsize=None)
def hqc_get_params(level: int) -> Params:
    """Table I parameters and derived sizes (constant per level, so cached;
    a bad level raises every time)."""
    p = _Params()
    _check(load().hqc_get_params(level, ctypes.byref(p)))
    return Params(*(int(getattr(p, f)) for f, _ in _Params._fields_))


def _as_u64(t):
    """View a uint64 tensor as int64 (torch's 64-bit integer type of choice)."""
    torch = _torch()
    return t.view(torch.int64) if t.dtype == torch.uint64 else t


def hqc_decrypt_batch(level, u, v, y, m_out=None, stream=None):
    """Fused decryption with literal supports y [count][w] (int32/uint32 view)."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    cnt = u.shape[0]
    if m_out is None:
        m_out = torch.empty((cnt, P.k), dtype=torch.uint8, device=u.device)
    y = y.view(torch.int32) if y.dtype == torch.uint32 else y
    _check(load().hqc_decrypt_batch(level, cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                    _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"),
                                    _dev_ptr(y, torch.int32, (cnt, P.w), "y"),
                                    _dev_ptr(m_out, torch.uint8, (cnt, P.k), "m_out"), _stream(stream)))
    return m_out


class Keyset:
    """Secret supports registered on the current device (hqc_keys_register)."""

    def __init__(self, level: int, y_host):
        y = np.ascontiguousarray(np.asarray(y_host, dtype=np.uint32))
        P = hqc_get_params(level)
        if y.ndim != 2 or y.shape[1] != P.w:
            raise ValueError("y_host must be [nkeys][%d]" % P.w)
        self.level = level
        self.nkeys = y.shape[0]
        self._h = ctypes.c_void_p()
        _check(load().hqc_keys_register(level, self.nkeys, y.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self._h)))

    @property
    def handle(self):
        if not self._h:
            raise ValueError("keyset was freed")
        return self._h

    def free(self):
        if self._h:
            _check(load().hqc_keys_free(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hqc_keys_register(level, y_host) -> Keyset:
    return Keyset(level, y_host)


def hqc_decrypt_batch_keyed(level, u, v, keys: Keyset, key_idx, m_out=None, stream=None):
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    cnt = u.shape[0]
    if m_out is None:
        m_out = torch.zeros((cnt, P.k), dtype=torch.uint8, device=u.device)
    _check(load().hqc_decrypt_batch_keyed(level, cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                          _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"), keys.handle,
                                          _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"),
                                          _dev_ptr(m_out, torch.uint8, (cnt, P.k), "m_out"), _stream(stream)))
    return m_out


def hqc_count_bad_key_idx(key_idx, nkeys: int, stream=None) -> int:
    """How many entries of key_idx (a device int32 tensor) lie outside
    [0, nkeys): the items every keyed entry point skips.  Counted on the
    device by hqc_count_bad_key_idx; this wrapper waits for the result."""
    torch = _torch()
    cnt = key_idx.numel()
    out = torch.empty((1,), dtype=torch.int32, device=key_idx.device)
    _check(load().hqc_count_bad_key_idx(cnt, _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"), int(nkeys),
                                        _dev_ptr(out, torch.int32, (1,), "out"), _stream(stream)))
    if stream is not None:
        stream.synchronize()
    return int(out.item()) & 0xFFFFFFFF


def hqc_rm_decode_batch(level, w, r_out=None, tensor_cores=False, stream=None):
    """S5-S7 alone: the n1 RM bytes of each received word of w (int64
    [count, W_v], device), by the register butterflies or, with
    tensor_cores, by the tensor-core product (hqc_rm_decode_batch)."""
    torch = _torch()
    P = hqc_get_params(level)
    cnt = w.shape[0]
    if r_out is None:
        r_out = torch.zeros((cnt, P.n1), dtype=torch.uint8, device=w.device)
    _check(load().hqc_rm_decode_batch(level, cnt, _dev_ptr(w, torch.int64, (cnt, P.W_v), "w"),
                                      _dev_ptr(r_out, torch.uint8, (cnt, P.n1), "r_out"), 1 if tensor_cores else 0,
                                      _stream(stream)))
    return r_out


def hqc_rm_tc_timeouts() -> int:
    """Timed-out tensor-core waits since the last call (0 normally)."""
    out = ctypes.c_int(0)
    _check(load().hqc_rm_tc_timeouts(ctypes.byref(out)))
    return out.value


def hqc_staged_workspace_bytes(level: int, count: int) -> int:
    return int(load().hqc_staged_workspace_bytes(level, count))


def hqc_decrypt_batch_staged(level, u, v, y=None, keys: Keyset = None, key_idx=None, workspace=None,
                             m_out=None, stream=None):
    """Plain per-stage form (three kernels, intermediates in `workspace`)."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    cnt = u.shape[0]
    if m_out is None:
        m_out = torch.zeros((cnt, P.k), dtype=torch.uint8, device=u.device)
    need = hqc_staged_workspace_bytes(level, cnt)
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=u.device)
    yp = ctypes.c_void_p()
    kp = ctypes.c_void_p()
    ip = ctypes.c_void_p()
    if keys is not None:
        kp = keys.handle
        ip = _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx")
    else:
        y = y.view(torch.int32) if y.dtype == torch.uint32 else y
        yp = _dev_ptr(y, torch.int32, (cnt, P.w), "y")
    _check(load().hqc_decrypt_batch_staged(level, cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                           _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"), yp, kp, ip,
                                           _dev_ptr(workspace, torch.uint8, None, "workspace"),
                                           workspace.numel(), _dev_ptr(m_out, torch.uint8, (cnt, P.k), "m_out"),
                                           _stream(stream)))
    return m_out


def hqc_decrypt_batch_staged_noalloc(level, u, v, y=None, keys: Keyset = None, key_idx=None, m_out=None,
                                     stream=None):
    """Per-stage decryption whose scratch is the library's compiled-in array
    (no device allocation by the library; m_out may be passed in by a caller
    that allocates nothing either).  Calls overlapping on the GPU race on
    that array."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    cnt = u.shape[0]
    if m_out is None:
        m_out = torch.zeros((cnt, P.k), dtype=torch.uint8, device=u.device)
    yp, kp, ip = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    if keys is not None:
        kp = keys.handle
        ip = _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx")
    else:
        y = y.view(torch.int32) if y.dtype == torch.uint32 else y
        yp = _dev_ptr(y, torch.int32, (cnt, P.w), "y")
    # the library resolves its compiled-in scratch on the current device:
    # make that the device the tensors live on
    with torch.cuda.device(u.device):
        _check(load().hqc_decrypt_batch_staged_noalloc(level, cnt,
                                                       _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                                       _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"), yp, kp, ip,
                                                       _dev_ptr(m_out, torch.uint8, (cnt, P.k), "m_out"),
                                                       _stream(stream)))
    return m_out


def hqc_decrypt_debug(level, u, v, y, stream=None):
    """Per-stage decryption returning every intermediate of Algorithm 2."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    y = y.view(torch.int32) if y.dtype == torch.uint32 else y
    cnt = u.shape[0]
    dev = u.device
    nr = 2 * P.delta
    out = dict(t=torch.zeros((cnt, P.W_v), dtype=torch.int64, device=dev),
               w=torch.zeros((cnt, P.W_v), dtype=torch.int64, device=dev),
               r=torch.zeros((cnt, P.n1), dtype=torch.uint8, device=dev),
               S=torch.zeros((cnt, nr), dtype=torch.uint8, device=dev),
               lam=torch.zeros((cnt, nr + 1), dtype=torch.uint8, device=dev),
               L=torch.zeros((cnt,), dtype=torch.int32, device=dev),
               errmask=torch.zeros((cnt, P.n1), dtype=torch.uint8, device=dev),
               errval=torch.zeros((cnt, P.n1), dtype=torch.uint8, device=dev),
               cw=torch.zeros((cnt, P.n1), dtype=torch.uint8, device=dev),
               flag=torch.zeros((cnt,), dtype=torch.int32, device=dev),
               m=torch.zeros((cnt, P.k), dtype=torch.uint8, device=dev))
    d = _Dump(*[ctypes.c_void_p(out[f].data_ptr()) for f, _ in _Dump._fields_])
    _check(load().hqc_decrypt_debug(level, cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                    _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"),
                                    _dev_ptr(y, torch.int32, (cnt, P.w), "y"), ctypes.byref(d),
                                    _dev_ptr(out["m"], torch.uint8, (cnt, P.k), "m"), _stream(stream)))
    return out


def hqc_decrypt_debug_team(level, u, v, y, form=0, stream=None):
    """The fused kernels' own intermediates (form 0: four-warp team per
    ciphertext, 1: cluster of four blocks, 2: the persistent throughput
    kernels' per-turn code): r, S, lam and m per ciphertext."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    y = y.view(torch.int32) if y.dtype == torch.uint32 else y
    cnt = u.shape[0]
    dev = u.device
    nr = 2 * P.delta
    out = dict(r=torch.zeros((cnt, P.n1), dtype=torch.uint8, device=dev),
               S=torch.zeros((cnt, nr), dtype=torch.uint8, device=dev),
               lam=torch.zeros((cnt, nr + 1), dtype=torch.uint8, device=dev),
               m=torch.zeros((cnt, P.k), dtype=torch.uint8, device=dev))
    ptrs = {f: ctypes.c_void_p(out[f].data_ptr()) if f in out else ctypes.c_void_p(0) for f, _ in _Dump._fields_}
    d = _Dump(*[ptrs[f] for f, _ in _Dump._fields_])
    _check(load().hqc_decrypt_debug_team(level, int(form), cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                         _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"),
                                         _dev_ptr(y, torch.int32, (cnt, P.w), "y"), ctypes.byref(d),
                                         _dev_ptr(out["m"], torch.uint8, (cnt, P.k), "m"), _stream(stream)))
    return out


def hqc_mixed_workspace_bytes() -> int:
    return int(load().hqc_mixed_workspace_bytes())


def hqc_decrypt_mixed(items, arena, keys, m_arena, workspace=None, stream=None):
    """One persistent launch over mixed-level items.

    items: uint8 CUDA tensor viewing an array of ITEM_DTYPE records;
    arena: int64 CUDA tensor of u/v words; keys: (Keyset|None) x 3 for
    levels 1, 3, 5; m_arena: uint8 CUDA tensor."""
    torch = _torch()
    if items.dtype != torch.uint8 or items.numel() % ITEM_DTYPE.itemsize:
        raise TypeError("items must be a uint8 tensor of packed ITEM_DTYPE records")
    cnt = items.numel() // ITEM_DTYPE.itemsize
    arena = _as_u64(arena)
    if workspace is None:
        workspace = torch.zeros(hqc_mixed_workspace_bytes(), dtype=torch.uint8, device=arena.device)
    karr = (ctypes.c_void_p * 3)(*[(k.handle if k is not None else None) for k in keys])
    _check(load().hqc_decrypt_mixed(cnt, _dev_ptr(items, torch.uint8, None, "items"),
                                    _dev_ptr(arena, torch.int64, None, "arena"), arena.numel(), karr,
                                    _dev_ptr(m_arena, torch.uint8, None, "m_arena"), m_arena.numel(),
                                    _dev_ptr(workspace, torch.uint8, None, "workspace"), workspace.numel(),
                                    _stream(stream)))
    return m_arena


def hqc_set_launch_config(level: int, warps_per_cta: int = 0, ctas_per_sm: int = 0):
    cfg = _LaunchCfg(warps_per_cta, ctas_per_sm)
    _check(load().hqc_set_launch_config(level, ctypes.byref(cfg)))


def hqc_get_launch_shape(level: int, keyed: bool = True):
    w, c, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().hqc_get_launch_shape(level, int(keyed), ctypes.byref(w), ctypes.byref(c), ctypes.byref(g)))
    return dict(warps_per_cta=w.value, ctas_per_sm=c.value, grid=g.value)


def hqc_keygen_batch(level, h, x, y, s_out=None, stream=None):
    torch = _torch()
    P = hqc_get_params(level)
    h = _as_u64(h)
    nk = h.shape[0]
    if s_out is None:
        s_out = torch.empty((nk, P.W_u_pitch), dtype=torch.int64, device=h.device)
    x = x.view(torch.int32) if x.dtype == torch.uint32 else x
    y = y.view(torch.int32) if y.dtype == torch.uint32 else y
    _check(load().hqc_keygen_batch(level, nk, _dev_ptr(h, torch.int64, (nk, P.W_u_pitch), "h"),
                                   _dev_ptr(x, torch.int32, (nk, P.w), "x"), _dev_ptr(y, torch.int32, (nk, P.w), "y"),
                                   _dev_ptr(s_out, torch.int64, (nk, P.W_u_pitch), "s_out"), _stream(stream)))
    return s_out


def hqc_encrypt_batch(level, h, s, key_idx, m, r1, r2, e, u_out=None, v_out=None, stream=None):
    torch = _torch()
    P = hqc_get_params(level)
    h, s = _as_u64(h), _as_u64(s)
    nk = h.shape[0]
    cnt = m.shape[0]
    dev = m.device
    if u_out is None:
        u_out = torch.zeros((cnt, P.W_u_pitch), dtype=torch.int64, device=dev)
    if v_out is None:
        v_out = torch.zeros((cnt, P.W_v), dtype=torch.int64, device=dev)
    r1, r2, e = [t.view(torch.int32) if t.dtype == torch.uint32 else t for t in (r1, r2, e)]
    _check(load().hqc_encrypt_batch(level, cnt, _dev_ptr(h, torch.int64, (nk, P.W_u_pitch), "h"),
                                    _dev_ptr(s, torch.int64, (nk, P.W_u_pitch), "s"), nk,
                                    _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"),
                                    _dev_ptr(m, torch.uint8, (cnt, P.k), "m"),
                                    _dev_ptr(r1, torch.int32, (cnt, P.wr), "r1"),
                                    _dev_ptr(r2, torch.int32, (cnt, P.wr), "r2"),
                                    _dev_ptr(e, torch.int32, (cnt, P.we), "e"),
                                    _dev_ptr(u_out, torch.int64, (cnt, P.W_u_pitch), "u_out"),
                                    _dev_ptr(v_out, torch.int64, (cnt, P.W_v), "v_out"), _stream(stream)))
    return u_out, v_out


class Plan:
    """A batch captured in a CUDA graph (hqc_plan_create_*); keeps the
    tensors it points at alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(load().hqc_plan_launch(self._h, _stream(stream)))

    def info(self):
        form = ctypes.c_int32()
        cfg = _LaunchCfg()
        grids = (ctypes.c_int32 * 3)()
        ms = ctypes.c_float()
        _check(load().hqc_plan_info(self._h, ctypes.byref(form), ctypes.byref(cfg), grids, ctypes.byref(ms)))
        return dict(form={0: "keyed", 1: "mixed-single-kernel", 2: "mixed-level-partitioned",
                          3: "mixed-per-level-sequential", 4: "mixed-one-launch-block-ranges"}[form.value],
                    warps_per_cta=cfg.warps_per_cta, ctas_per_sm=cfg.ctas_per_sm, grids=list(grids),
                    tuned_ms=ms.value)

    def describe(self):
        """The chosen form, kernel variant(s) and shape, and every candidate
        the tuner timed (fastest first), from hqc_plan_describe."""
        import json
        buf = ctypes.create_string_buffer(1 << 20)
        _check(load().hqc_plan_describe(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def destroy(self):
        if self._h:
            _check(load().hqc_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# kernel variants of the keyed and per-level plans (hqc_plan_create_*_fixed)
PLAN_VARIANTS = {"default": 0, "solo-G1": 1, "solo-G2": 2, "solo-G4": 3, "team2": 4}
PLAN_FORMS = {"mixed-single-kernel": 1, "mixed-level-partitioned": 2, "mixed-per-level-sequential": 3,
              "mixed-one-launch-block-ranges": 4}


def hqc_plan_create_keyed(level, u, v, keys: Keyset, key_idx, m_out, autotune=True, stream=None, variant=None,
                          warps_per_cta=0, ctas_per_sm=0) -> Plan:
    """Keyed plan: tuned (autotune), the library default, or -- with
    variant (a PLAN_VARIANTS name or number) -- that variant at the given
    shape (hqc_plan_create_keyed_fixed)."""
    torch = _torch()
    P = hqc_get_params(level)
    u, v = _as_u64(u), _as_u64(v)
    cnt = u.shape[0]
    h = ctypes.c_void_p()
    args = (level, cnt, _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"), _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"),
            keys.handle, _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"),
            _dev_ptr(m_out, torch.uint8, (cnt, P.k), "m_out"))
    if variant is None:
        _check(load().hqc_plan_create_keyed(*args, int(bool(autotune)), _stream(stream), ctypes.byref(h)))
    else:
        var = PLAN_VARIANTS[variant] if isinstance(variant, str) else int(variant)
        cfg = _LaunchCfg(warps_per_cta, ctas_per_sm)
        _check(load().hqc_plan_create_keyed_fixed(*args, var, ctypes.byref(cfg), _stream(stream), ctypes.byref(h)))
    return Plan(h, (u, v, keys, key_idx, m_out))


def hqc_plan_create_mixed(items, arena, keys, m_arena, autotune=True, stream=None, form=None, variants=None,
                          grids=None, warps_per_cta=0, ctas_per_sm=0) -> Plan:
    """Mixed plan: tuned (autotune) or the single mixed kernel, or -- with
    form (a PLAN_FORMS name or 1-4) -- that form with the given per-level
    variants (names or numbers) and blocks per level
    (hqc_plan_create_mixed_fixed)."""
    torch = _torch()
    if items.dtype != torch.uint8 or items.numel() % ITEM_DTYPE.itemsize:
        raise TypeError("items must be a uint8 tensor of packed ITEM_DTYPE records")
    cnt = items.numel() // ITEM_DTYPE.itemsize
    arena = _as_u64(arena)
    karr = (ctypes.c_void_p * 3)(*[(k.handle if k is not None else None) for k in keys])
    h = ctypes.c_void_p()
    args = (cnt, _dev_ptr(items, torch.uint8, None, "items"), _dev_ptr(arena, torch.int64, None, "arena"),
            arena.numel(), karr, _dev_ptr(m_arena, torch.uint8, None, "m_arena"), m_arena.numel())
    if form is None:
        _check(load().hqc_plan_create_mixed(*args, int(bool(autotune)), _stream(stream), ctypes.byref(h)))
    else:
        f = PLAN_FORMS[form] if isinstance(form, str) else int(form)
        vs = (ctypes.c_int32 * 3)(*[(PLAN_VARIANTS[x] if isinstance(x, str) else int(x))
                                    for x in (variants or (0, 0, 0))])
        gs = (ctypes.c_int32 * 3)(*(grids or (0, 0, 0)))
        cfg = _LaunchCfg(warps_per_cta, ctas_per_sm)
        _check(load().hqc_plan_create_mixed_fixed(*args, f, ctypes.byref(cfg), vs, gs, _stream(stream),
                                                  ctypes.byref(h)))
    return Plan(h, (items, arena, keys, m_arena))


class _ServeCfg(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("max_queue", ctypes.c_int64), ("warps_per_cta", ctypes.c_int32), ("stall_ms", ctypes.c_int32),
                ("transfer", ctypes.c_int32)]


class _ServeRing(ctypes.Structure):
    _fields_ = [("period", ctypes.c_int64), ("level", ctypes.c_void_p), ("key", ctypes.c_void_p),
                ("word_off", ctypes.c_void_p), ("words", ctypes.c_void_p), ("m_off", ctypes.c_void_p)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected_queue", ctypes.c_int64),
                ("rejected_invalid", ctypes.c_int64), ("rejected_size", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mean_batch", ctypes.c_double), ("wall_ns", ctypes.c_int64),
                ("items_per_slot", ctypes.c_int64), ("in_place", ctypes.c_int64)]


SERVE_STATUS = {0: "done", 1: "queued", 2: "running", 3: "rejected", 4: "invalid", 5: "too_large"}


def hqc_serve_run(keys, ring_level, ring_key, ring_word_off, ring_words, ring_m_off, arrival_ns, streams=4,
                  max_batch=8192, budget_bytes=256 << 20, max_queue=1 << 20, warps_per_cta=0, want_m=True,
                  stall_ms=0, transfer=0):
    """Run the continuous-batching loop over a request trace (hqc_serve_run).

    ring_words must be a PINNED uint64/int64 CPU tensor; the other ring
    arrays are numpy.  Returns (status, latency_ns, m_out or None, stats).
    A batch incomplete stall_ms after its launch (0: 10 s) raises HqcError
    with code HQC_ETIMEOUT.  transfer: 0 in place when possible, 1 copy
    engines, 2 in place (the kernels read the ring from host memory)."""
    torch = _torch()
    if not isinstance(ring_words, torch.Tensor) or ring_words.is_cuda or not ring_words.is_pinned():
        raise ValueError("ring_words must be a pinned CPU tensor")
    lvl = np.ascontiguousarray(ring_level, np.int32)
    key = np.ascontiguousarray(ring_key, np.int32)
    woff = np.ascontiguousarray(ring_word_off, np.int64)
    moff = np.ascontiguousarray(ring_m_off, np.int64)
    arr = np.ascontiguousarray(arrival_ns, np.int64)
    period = lvl.size
    if key.size != period or woff.size != period + 1 or moff.size != period + 1:
        raise ValueError("ring arrays disagree on the period")
    if woff[-1] > ring_words.numel():
        raise ValueError("ring_words is shorter than word_off says")
    cnt = arr.size
    status = np.zeros(cnt, np.int32)
    lat = np.zeros(cnt, np.int64)
    m_out = np.zeros(int(moff[-1]), np.uint8) if want_m else None
    cfg = _ServeCfg(streams, max_batch, budget_bytes, max_queue, warps_per_cta, stall_ms, transfer)
    ring = _ServeRing(period, lvl.ctypes.data_as(ctypes.c_void_p), key.ctypes.data_as(ctypes.c_void_p),
                      woff.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ring_words.data_ptr()),
                      moff.ctypes.data_as(ctypes.c_void_p))
    karr = (ctypes.c_void_p * 3)(*[(k.handle if k is not None else None) for k in keys])
    st = _ServeStats()
    rc = load().hqc_serve_run(ctypes.byref(cfg), karr, ctypes.byref(ring), cnt, arr.ctypes.data_as(ctypes.c_void_p),
                              status.ctypes.data_as(ctypes.c_void_p), lat.ctypes.data_as(ctypes.c_void_p),
                              m_out.ctypes.data_as(ctypes.c_void_p) if want_m else None, ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _ServeStats._fields_}
    if rc != 0:
        err = HqcError(rc, load().hqc_last_error().decode(errors="replace"))
        err.partial = (status, lat, m_out, stats)  # what was answered before the error
        raise err
    return status, lat, m_out, stats


def hqc_host_workspace_bytes(level: int, chunk: int) -> int:
    return int(load().hqc_host_workspace_bytes(level, chunk))


def hqc_decrypt_host_keyed(level, u_host, v_host, keys: Keyset, key_idx_host, m_host=None, chunk=0,
                           workspace=None, stream=None):
    """Decrypt from (pinned) HOST tensors with chunked copy/compute overlap.

    u_host [count][W_u_pitch] int64, v_host [count][W_v] int64, key_idx_host
    [count] int32, m_host [count][k] uint8 (CPU tensors); workspace: a CUDA
    uint8 tensor of at least hqc_host_workspace_bytes(level, chunk) bytes
    (allocated here when None; chunk 0 lets the library choose, bounded by
    the workspace).  Returns m_host (valid once the stream reaches the end
    of the call)."""
    torch = _torch()
    P = hqc_get_params(level)
    u_host, v_host = _as_u64(u_host), _as_u64(v_host)
    cnt = u_host.shape[0]
    for t, name in ((u_host, "u_host"), (v_host, "v_host"), (key_idx_host, "key_idx_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CPU tensor" % name)
    if tuple(u_host.shape) != (cnt, P.W_u_pitch) or tuple(v_host.shape) != (cnt, P.W_v):
        raise ValueError("u_host / v_host shapes")
    if key_idx_host.dtype != torch.int32 or tuple(key_idx_host.shape) != (cnt,):
        raise ValueError("key_idx_host must be int32 [count]")
    if m_host is None:
        m_host = torch.zeros((cnt, P.k), dtype=torch.uint8).pin_memory()
    if workspace is None:
        workspace = torch.empty(hqc_host_workspace_bytes(level, chunk if chunk > 0 else max(1, min(cnt, 16384))),
                                dtype=torch.uint8, device="cuda")
    _check(load().hqc_decrypt_host_keyed(level, cnt, ctypes.c_void_p(u_host.data_ptr()),
                                         ctypes.c_void_p(v_host.data_ptr()), keys.handle,
                                         ctypes.c_void_p(key_idx_host.data_ptr()), ctypes.c_void_p(m_host.data_ptr()),
                                         int(chunk), _dev_ptr(workspace, torch.uint8, None, "workspace"),
                                         workspace.numel(), _stream(stream)))
    return m_host


# ---------------------------------------------------------------------------
# SHAKE256 and the KEM (device tensors in, device tensors out)
# ---------------------------------------------------------------------------
def hqc_shake256_batch(msg, outlen: int, out=None, stream=None):
    """SHAKE256 of each row of msg (CUDA uint8 [count][len]) -> [count][outlen]."""
    torch = _torch()
    cnt, ln = msg.shape
    if out is None:
        out = torch.empty((cnt, outlen), dtype=torch.uint8, device=msg.device)
    _check(load().hqc_shake256_batch(cnt, _dev_ptr(msg, torch.uint8, None, "msg"), ln,
                                     _dev_ptr(out, torch.uint8, (cnt, outlen), "out"), outlen, _stream(stream)))
    return out


def hqc_kem_keygen(level, seed_sk, seed_pk, stream=None):
    """(h, x, y, s) from seeds (CUDA uint8 [nkeys][32] each)."""
    torch = _torch()
    P = hqc_get_params(level)
    nk = seed_sk.shape[0]
    dev = seed_sk.device
    h = torch.empty((nk, P.W_u_pitch), dtype=torch.int64, device=dev)
    s = torch.empty_like(h)
    x = torch.empty((nk, P.w), dtype=torch.int32, device=dev)
    y = torch.empty_like(x)
    _check(load().hqc_kem_keygen(level, nk, _dev_ptr(seed_sk, torch.uint8, (nk, 32), "seed_sk"),
                                 _dev_ptr(seed_pk, torch.uint8, (nk, 32), "seed_pk"), _dev_ptr(h, torch.int64),
                                 _dev_ptr(x, torch.int32), _dev_ptr(y, torch.int32), _dev_ptr(s, torch.int64),
                                 _stream(stream)))
    return h, x, y, s


def hqc_kem_workspace_bytes(level: int, count: int) -> int:
    return int(load().hqc_kem_workspace_bytes(level, count))


def _kem_ws(level, cnt, workspace, dev):
    torch = _torch()
    need = hqc_kem_workspace_bytes(level, cnt)
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
    return workspace


def hqc_kem_encaps(level, h, s, key_idx, m, salt, u_out=None, v_out=None, K_out=None, workspace=None, stream=None):
    """(u, v, K): encapsulation of m [count][k] with salt [count][16] under
    key key_idx[i] of (h, s) [nkeys][W_u_pitch]; all CUDA tensors."""
    torch = _torch()
    P = hqc_get_params(level)
    h, s = _as_u64(h), _as_u64(s)
    cnt = key_idx.shape[0]
    dev = key_idx.device
    u_out = torch.zeros((cnt, P.W_u_pitch), dtype=torch.int64, device=dev) if u_out is None else _as_u64(u_out)
    v_out = torch.zeros((cnt, P.W_v), dtype=torch.int64, device=dev) if v_out is None else _as_u64(v_out)
    K_out = torch.zeros((cnt, 32), dtype=torch.uint8, device=dev) if K_out is None else K_out
    ws = _kem_ws(level, cnt, workspace, dev)
    _check(load().hqc_kem_encaps(level, cnt, _dev_ptr(h, torch.int64), _dev_ptr(s, torch.int64), h.shape[0],
                                 _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"),
                                 _dev_ptr(m, torch.uint8, (cnt, P.k), "m"), _dev_ptr(salt, torch.uint8, (cnt, 16), "salt"),
                                 _dev_ptr(u_out, torch.int64, (cnt, P.W_u_pitch), "u_out"),
                                 _dev_ptr(v_out, torch.int64, (cnt, P.W_v), "v_out"),
                                 _dev_ptr(K_out, torch.uint8, (cnt, 32), "K_out"), _dev_ptr(ws, torch.uint8),
                                 ws.numel(), _stream(stream)))
    return u_out, v_out, K_out


def hqc_kem_decaps(level, keys: Keyset, h, s, sigma, key_idx, u, v, salt, K_out=None, ok_out=None, workspace=None,
                   stream=None):
    """(K, ok): decapsulation with implicit rejection; ok is int32 [count]
    (1 where the re-encryption matched)."""
    torch = _torch()
    P = hqc_get_params(level)
    h, s, u, v = _as_u64(h), _as_u64(s), _as_u64(u), _as_u64(v)
    cnt = key_idx.shape[0]
    dev = key_idx.device
    K_out = torch.zeros((cnt, 32), dtype=torch.uint8, device=dev) if K_out is None else K_out
    ok_out = torch.zeros((cnt,), dtype=torch.int32, device=dev) if ok_out is None else ok_out
    ws = _kem_ws(level, cnt, workspace, dev)
    _check(load().hqc_kem_decaps(level, cnt, keys.handle, _dev_ptr(h, torch.int64), _dev_ptr(s, torch.int64),
                                 _dev_ptr(sigma, torch.uint8, (keys.nkeys, P.k), "sigma"),
                                 _dev_ptr(key_idx, torch.int32, (cnt,), "key_idx"),
                                 _dev_ptr(u, torch.int64, (cnt, P.W_u_pitch), "u"),
                                 _dev_ptr(v, torch.int64, (cnt, P.W_v), "v"),
                                 _dev_ptr(salt, torch.uint8, (cnt, 16), "salt"),
                                 _dev_ptr(K_out, torch.uint8, (cnt, 32), "K_out"),
                                 _dev_ptr(ok_out, torch.int32, (cnt,), "ok_out"), _dev_ptr(ws, torch.uint8),
                                 ws.numel(), _stream(stream)))
    return K_out, ok_out


def hqc_kem_host_workspace_bytes(level: int, chunk: int) -> int:
    return int(load().hqc_kem_host_workspace_bytes(level, chunk))


def hqc_kem_decaps_host(level, keys: Keyset, h, s, sigma, key_idx_host, u_host, v_host, salt_host, K_host=None,
                        ok_host=None, chunk=0, workspace=None, stream=None):
    """Decapsulation from (pinned) HOST tensors with chunked copy/compute
    overlap; h, s, sigma are CUDA tensors.  Returns (K_host, ok_host), valid
    once the stream reaches the end of the call."""
    torch = _torch()
    P = hqc_get_params(level)
    h, s = _as_u64(h), _as_u64(s)
    u_host, v_host = _as_u64(u_host), _as_u64(v_host)
    cnt = u_host.shape[0]
    for t, name in ((u_host, "u_host"), (v_host, "v_host"), (key_idx_host, "key_idx_host"), (salt_host, "salt_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CPU tensor" % name)
    if tuple(u_host.shape) != (cnt, P.W_u_pitch) or tuple(v_host.shape) != (cnt, P.W_v):
        raise ValueError("u_host / v_host shapes")
    if key_idx_host.dtype != torch.int32 or tuple(key_idx_host.shape) != (cnt,):
        raise ValueError("key_idx_host must be int32 [count]")
    if salt_host.dtype != torch.uint8 or tuple(salt_host.shape) != (cnt, 16):
        raise ValueError("salt_host must be uint8 [count][16]")
    if K_host is None:
        K_host = torch.empty((cnt, 32), dtype=torch.uint8).pin_memory()
    if ok_host is None:
        ok_host = torch.empty((cnt,), dtype=torch.int32).pin_memory()
    if workspace is None:
        workspace = torch.empty(hqc_kem_host_workspace_bytes(level, chunk if chunk > 0 else max(1, min(cnt, 16384))),
                                dtype=torch.uint8, device="cuda")
    _check(load().hqc_kem_decaps_host(level, cnt, keys.handle, _dev_ptr(h, torch.int64), _dev_ptr(s, torch.int64),
                                      _dev_ptr(sigma, torch.uint8, (keys.nkeys, P.k), "sigma"),
                                      ctypes.c_void_p(key_idx_host.data_ptr()), ctypes.c_void_p(u_host.data_ptr()),
                                      ctypes.c_void_p(v_host.data_ptr()), ctypes.c_void_p(salt_host.data_ptr()),
                                      ctypes.c_void_p(K_host.data_ptr()), ctypes.c_void_p(ok_host.data_ptr()),
                                      int(chunk), _dev_ptr(workspace, torch.uint8, None, "workspace"),
                                      workspace.numel(), _stream(stream)))
    return K_host, ok_host


def _host_u8(t, name):
    torch = _torch()
    if t.is_cuda or not t.is_contiguous() or t.dtype != torch.uint8:
        raise ValueError("%s must be a contiguous CPU uint8 tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def hqc_mixed_host_workspace_bytes(items_host, chunk: int = 0) -> int:
    """Device workspace for hqc_decrypt_mixed_host over these (host) items."""
    cnt = items_host.numel() // ITEM_DTYPE.itemsize
    return int(load().hqc_mixed_host_workspace_bytes(cnt, _host_u8(items_host, "items_host"), int(chunk)))


def hqc_decrypt_mixed_host(items_host, arena_host, keys, m_host, chunk=0, workspace=None, stream=None):
    """Mixed-level decryption from (pinned) HOST tensors: items_host (uint8
    view of ITEM_DTYPE records, in arena order), arena_host (int64 words),
    m_host (uint8); workspace a CUDA uint8 tensor (allocated here when
    None).  m_host is valid once the stream reaches the end of the call."""
    torch = _torch()
    cnt = items_host.numel() // ITEM_DTYPE.itemsize
    arena_host = _as_u64(arena_host)
    if arena_host.is_cuda or not arena_host.is_contiguous():
        raise ValueError("arena_host must be a contiguous CPU tensor")
    if workspace is None:
        need = hqc_mixed_host_workspace_bytes(items_host, chunk)
        if need == 0:
            raise ValueError("items are not in arena order or reach past the arena")
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    karr = (ctypes.c_void_p * 3)(*[(k.handle if k is not None else None) for k in keys])
    _check(load().hqc_decrypt_mixed_host(cnt, _host_u8(items_host, "items_host"),
                                         ctypes.c_void_p(arena_host.data_ptr()), arena_host.numel(), karr,
                                         _host_u8(m_host, "m_host"), m_host.numel(), int(chunk),
                                         _dev_ptr(workspace, torch.uint8, None, "workspace"), workspace.numel(),
                                         _stream(stream)))
    return m_host
