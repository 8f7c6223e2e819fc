"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every entry point the public header declares, and
its host logic (parameters, argument checks, workspace sizes) is right."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2512_12904_gb300 as hqc
from conftest import ROOT, read_golden

HEADER = os.path.join(ROOT, "include", "hqc_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hqc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = hqc.load()
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("level", [1, 3, 5])
def test_params_match_table1_and_oracle(level):
    rows = {int(r[0].split("-")[1]): r for r in read_golden("table1_params.txt")}
    r = rows[level]
    p = hqc.hqc_get_params(level)
    assert (p.n, p.w, p.we, p.wr, p.n1, p.k) == tuple(int(x) for x in (r[1], r[2], r[3], r[3], r[4], r[5]))
    assert 2 * p.delta + 1 == int(r[6]) and p.n2 == int(r[7]) and 64 * p.mult == int(r[9])
    o = oracle.params(level)
    assert (p.W_u, p.W_u_pitch, p.W_v, p.delta, p.mult) == (o.W_u, o.W_u_pitch, o.W_v, o.delta, o.mult)


def test_argument_errors_are_reported_without_a_gpu():
    lib = hqc.load()
    p = hqc._Params()
    assert lib.hqc_get_params(2, ctypes.byref(p)) == -1
    assert b"level" in lib.hqc_last_error()
    assert lib.hqc_get_params(1, None) == -1
    # count 0 is a no-op; bad level and negative count are rejected first
    assert lib.hqc_decrypt_batch(1, 0, None, None, None, None, None) == 0
    assert lib.hqc_decrypt_batch(4, 1, None, None, None, None, None) == -1
    assert lib.hqc_decrypt_batch(1, -5, None, None, None, None, None) == -1
    assert lib.hqc_decrypt_batch(1, 3, None, None, None, None, None) == -1
    # misaligned u
    assert lib.hqc_decrypt_batch(1, 1, ctypes.c_void_p(8), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 ctypes.c_void_p(16), None) == -1
    assert b"aligned" in lib.hqc_last_error()
    cfg = hqc._LaunchCfg(99, 0)
    assert lib.hqc_set_launch_config(1, ctypes.byref(cfg)) == -1
    assert lib.hqc_set_launch_config(7, None) == -1
    assert lib.hqc_set_launch_config(1, None) == 0


def test_keyset_validation_rejects_bad_supports_before_any_copy():
    lib = hqc.load()
    P = hqc.hqc_get_params(1)
    h = ctypes.c_void_p()
    bad = np.arange(P.w, dtype=np.uint32).reshape(1, P.w).copy()
    bad[0, 3] = P.n
    assert lib.hqc_keys_register(1, 1, bad.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == -1
    assert b">= n" in lib.hqc_last_error()
    dup = np.arange(P.w, dtype=np.uint32).reshape(1, P.w).copy()
    dup[0, 7] = dup[0, 2]
    assert lib.hqc_keys_register(1, 1, dup.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == -1
    assert b"repeats" in lib.hqc_last_error()
    assert lib.hqc_keys_register(1, 0, bad.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == -1


@pytest.mark.parametrize("level", [1, 3, 5])
def test_workspace_sizes(level):
    p = hqc.hqc_get_params(level)
    for cnt in (1, 7, 4096):
        b = hqc.hqc_staged_workspace_bytes(level, cnt)
        assert b >= cnt * p.W_v * 8 + cnt * p.n1 and b % 16 == 0
    assert hqc.hqc_staged_workspace_bytes(level, 0) == 0
    assert hqc.hqc_mixed_workspace_bytes() >= 4


def test_item_record_layout():
    assert hqc.ITEM_DTYPE.itemsize == 32


@pytest.mark.parametrize("level", [1, 3, 5])
def test_host_pipeline_workspace_and_argument_checks(level):
    lib = hqc.load()
    p = hqc.hqc_get_params(level)
    for chunk in (1, 5, 8192):
        b = hqc.hqc_host_workspace_bytes(level, chunk)
        assert b >= 2 * chunk * ((p.W_u_pitch + p.W_v) * 8 + 4 + p.k) and b % 16 == 0
    assert hqc.hqc_host_workspace_bytes(level, 0) == 0
    assert hqc.hqc_host_workspace_bytes(2, 16) == 0
    N = None
    assert lib.hqc_decrypt_host_keyed(2, 1, N, N, N, N, N, 16, N, 0, N) == -1
    assert lib.hqc_decrypt_host_keyed(level, -1, N, N, N, N, N, 16, N, 0, N) == -1
    assert lib.hqc_decrypt_host_keyed(level, 0, N, N, N, N, N, 16, N, 0, N) == 0
    assert lib.hqc_decrypt_host_keyed(level, 3, N, N, N, N, N, 16, N, 0, N) == -1
    assert b"NULL" in lib.hqc_last_error()


def test_kem_argument_checks_without_a_gpu():
    lib = hqc.load()
    N = None
    assert lib.hqc_shake256_batch(0, N, 5, N, 32, N) == 0
    assert lib.hqc_shake256_batch(-1, N, 5, N, 32, N) == -1
    assert lib.hqc_shake256_batch(3, N, 5, N, 32, N) == -1
    assert lib.hqc_kem_keygen(2, 1, N, N, N, N, N, N, N) == -1
    assert lib.hqc_kem_keygen(1, 0, N, N, N, N, N, N, N) == 0
    assert lib.hqc_kem_keygen(1, 2, N, N, N, N, N, N, N) == -1
    assert b"seeds" in lib.hqc_last_error()
    for level in (1, 3, 5):
        p = hqc.hqc_get_params(level)
        b = hqc.hqc_kem_workspace_bytes(level, 1000)
        assert b >= 1000 * (p.k + 4 * (2 * p.wr + p.we) + 4) and b % 16 == 0
    assert hqc.hqc_kem_workspace_bytes(1, 0) == 0
    assert lib.hqc_kem_encaps(1, 0, N, N, 1, N, N, N, N, N, N, N, 0, N) == 0
    assert lib.hqc_kem_encaps(1, 5, N, N, 1, N, N, N, N, N, N, N, 0, N) == -1
    assert lib.hqc_kem_decaps(1, 0, N, N, N, N, N, N, N, N, N, N, N, 0, N) == 0
    assert lib.hqc_kem_decaps(1, 5, N, N, N, N, N, N, N, N, N, N, N, 0, N) == -1
    assert b"keys" in lib.hqc_last_error()


def test_kem_host_pipeline_argument_checks():
    lib = hqc.load()
    N = None
    for level in (1, 3, 5):
        p = hqc.hqc_get_params(level)
        b = hqc.hqc_kem_host_workspace_bytes(level, 100)
        assert b >= 2 * (100 * ((p.W_u_pitch + p.W_v) * 8 + 4 + 16 + 32 + 4) + hqc.hqc_kem_workspace_bytes(level, 100))
    assert hqc.hqc_kem_host_workspace_bytes(1, 0) == 0
    assert lib.hqc_kem_decaps_host(1, 0, N, N, N, N, N, N, N, N, N, N, 0, N, 0, N) == 0
    assert lib.hqc_kem_decaps_host(1, 4, N, N, N, N, N, N, N, N, N, N, 0, N, 0, N) == -1
    assert b"NULL" in lib.hqc_last_error()
    assert lib.hqc_kem_decaps_host(4, 4, N, N, N, N, N, N, N, N, N, N, 0, N, 0, N) == -1


def test_mixed_host_pipeline_order_checks_on_the_host():
    lib = hqc.load()
    items = np.zeros(4, dtype=hqc.ITEM_DTYPE)
    P1 = hqc.hqc_get_params(1)
    row = P1.W_u_pitch + P1.W_v
    for i in range(4):
        items[i] = (1, 0, i * row, i * row + P1.W_u_pitch, i * P1.k)
    import torch
    t = torch.from_numpy(items.view(np.uint8).copy())
    b = hqc.hqc_mixed_host_workspace_bytes(t, chunk=2)
    assert b >= 2 * (2 * row * 8 + 2 * 2 * 32 + 2 * P1.k)
    bad = items.copy()
    bad[[1, 2]] = bad[[2, 1]]
    assert hqc.hqc_mixed_host_workspace_bytes(torch.from_numpy(bad.view(np.uint8).copy()), chunk=2) == 0
    N = None
    assert lib.hqc_decrypt_mixed_host(0, N, N, 0, N, N, 0, 0, N, 0, N) == 0
    assert lib.hqc_decrypt_mixed_host(3, N, N, 0, N, N, 0, 0, N, 0, N) == -1


def test_serving_argument_checks_without_a_gpu():
    """hqc_serve_run rejects a bad configuration (including a negative stall
    limit) before it touches the device."""
    lib = hqc.load()
    one32 = np.zeros(2, np.int32)
    one64 = np.zeros(2, np.int64)
    ring = hqc._ServeRing(1, one32.ctypes.data_as(ctypes.c_void_p), one32.ctypes.data_as(ctypes.c_void_p),
                          one64.ctypes.data_as(ctypes.c_void_p), one64.ctypes.data_as(ctypes.c_void_p),
                          one64.ctypes.data_as(ctypes.c_void_p))
    karr = (ctypes.c_void_p * 3)(None, None, None)
    st, lat = np.zeros(1, np.int32), np.zeros(1, np.int64)

    def call(cfg):
        return lib.hqc_serve_run(ctypes.byref(cfg), karr, ctypes.byref(ring), 1,
                                 one64.ctypes.data_as(ctypes.c_void_p), st.ctypes.data_as(ctypes.c_void_p),
                                 lat.ctypes.data_as(ctypes.c_void_p), None, None)

    assert ctypes.sizeof(hqc._ServeCfg) == 40  # 7 fields, padded to 8 bytes
    assert call(hqc._ServeCfg(1, 1, 1 << 20, 1, 0, -1)) == hqc.HQC_EINVAL
    assert b"stall_ms" in lib.hqc_last_error()
    assert call(hqc._ServeCfg(0, 1, 1 << 20, 1, 0, 0)) == hqc.HQC_EINVAL
    assert call(hqc._ServeCfg(1, 1, 0, 1, 0, 0)) == hqc.HQC_EINVAL


@pytest.mark.parametrize("level,limit", [(1, 7443), (3, 3698), (5, 2301)])
def test_noalloc_limit_is_the_largest_count_whose_workspace_fits(level, limit):
    """The allocation-free entry point's count limit and the per-stage
    workspace formula agree: the limit's workspace fits the compiled-in
    array and one more ciphertext's does not.  Counts beyond the limit are
    refused on the host, before any launch."""
    lib = hqc.load()
    scratch = 16 << 20
    assert lib.hqc_staged_workspace_bytes(level, limit) <= scratch < lib.hqc_staged_workspace_bytes(level, limit + 1)
    p16 = ctypes.c_void_p(16)
    rc = lib.hqc_decrypt_batch_staged_noalloc(level, limit + 1, p16, p16, p16, None, None, p16, None)
    assert rc == -1
    msg = lib.hqc_last_error()
    assert b"exceeds the static scratch" in msg and str(limit).encode() in msg


def test_serving_rejects_rings_whose_offsets_decrease_without_a_gpu():
    """The serving loop checks the ring's offsets on the host before it
    touches the device: offsets must start at 0 and never decrease, and
    in-place reads (transfer 2) need even word offsets."""
    lib = hqc.load()
    level = np.array([1, 1], np.int32)
    key = np.zeros(2, np.int32)
    words = np.zeros(2000, np.uint64)
    arr = np.zeros(2, np.int64)
    st = np.zeros(2, np.int32)
    lat = np.zeros(2, np.int64)
    P = ctypes.c_void_p

    def call(woff, moff, transfer=0):
        cfg = hqc._ServeCfg(1, 8, 1 << 20, 16, 0, 0, transfer)
        ring = hqc._ServeRing(2, level.ctypes.data_as(P), key.ctypes.data_as(P), woff.ctypes.data_as(P),
                              words.ctypes.data_as(P), moff.ctypes.data_as(P))
        keys = (P * 3)(None, None, None)
        stats = hqc._ServeStats()
        return lib.hqc_serve_run(ctypes.byref(cfg), keys, ctypes.byref(ring), 2, arr.ctypes.data_as(P),
                                 st.ctypes.data_as(P), lat.ctypes.data_as(P), None, ctypes.byref(stats))

    assert call(np.array([0, 554, 500], np.int64), np.array([0, 16, 32], np.int64)) == -1
    assert b"non-decreasing" in lib.hqc_last_error()
    assert call(np.array([0, 554, 1108], np.int64), np.array([0, 16, 8], np.int64)) == -1
    assert call(np.array([1, 554, 1108], np.int64), np.array([0, 16, 32], np.int64)) == -1
    assert call(np.array([0, 555, 1109], np.int64), np.array([0, 16, 32], np.int64), transfer=2) == -1
    assert b"even word offsets" in lib.hqc_last_error()
    assert call(np.array([0, 554, 1108], np.int64), np.array([0, 16, 32], np.int64), transfer=3) == -1


def test_rm_decode_batch_argument_checks():
    """hqc_rm_decode_batch rejects a bad level, a negative count and a NULL
    or misaligned w before touching the device; an empty batch is a no-op;
    hqc_rm_tc_timeouts rejects a NULL output."""
    lib = hqc.load()
    buf = ctypes.create_string_buffer(64)
    p16 = ctypes.c_void_p((ctypes.addressof(buf) + 15) & ~15)
    odd = ctypes.c_void_p(p16.value + 8)
    assert lib.hqc_rm_decode_batch(2, 1, p16, p16, 0, None) == hqc.HQC_EINVAL
    assert lib.hqc_rm_decode_batch(1, -1, p16, p16, 1, None) == hqc.HQC_EINVAL
    assert lib.hqc_rm_decode_batch(3, 1, None, p16, 1, None) == hqc.HQC_EINVAL
    assert lib.hqc_rm_decode_batch(5, 1, odd, p16, 0, None) == hqc.HQC_EINVAL
    assert lib.hqc_rm_decode_batch(1, 1, p16, None, 1, None) == hqc.HQC_EINVAL
    assert lib.hqc_rm_decode_batch(1, 0, None, None, 1, None) == hqc.HQC_OK
    assert lib.hqc_rm_tc_timeouts(None) == hqc.HQC_EINVAL


def test_debug_team_argument_checks():
    """hqc_decrypt_debug_team accepts forms 0, 1 and 2 only and checks y and
    the dump before touching the device; an empty batch is a no-op."""
    lib = hqc.load()
    buf = ctypes.create_string_buffer(64)
    p16 = ctypes.c_void_p((ctypes.addressof(buf) + 15) & ~15)
    for form in (-1, 3):
        assert lib.hqc_decrypt_debug_team(1, form, 1, p16, p16, p16, p16, p16, None) == hqc.HQC_EINVAL
    assert lib.hqc_decrypt_debug_team(1, 2, 1, p16, p16, None, p16, p16, None) == hqc.HQC_EINVAL
    assert lib.hqc_decrypt_debug_team(5, 2, 1, p16, p16, p16, None, p16, None) == hqc.HQC_EINVAL
    assert lib.hqc_decrypt_debug_team(3, 2, 0, p16, p16, p16, p16, p16, None) == hqc.HQC_OK
