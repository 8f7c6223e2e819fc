"""The allocation-free per-stage entry point (hqc_decrypt_batch_staged_noalloc).

It exists for callers that cannot allocate device memory at decryption
time; its scratch is an array compiled into the library.  This file runs
last so that a failure here never hides the other GPU tests.  Each check
calls the new entry point through the C ABI twice in a row and compares its
output with the existing per-stage entry point (bit-exact: the arithmetic
is over GF(2) and GF(2^8)).
"""
import numpy as np
import pytest

from workloads import adversarial, honest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_COUNT = {1: 7443, 3: 3698, 5: 2301}


@pytest.fixture(scope="module")
def hqc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2512_12904_gb300 as lib
    lib.load()
    return lib


def u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint64).view(np.int64)).cuda()


def i32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("level", [1, 3, 5])
def test_noalloc_matches_staged_on_two_calls(hqc, level):
    first = honest(level, 6, 97, first_ct=40000, tag=21)
    P, au, av, ay = adversarial(level, tag=30 + level)
    second = honest(level, 3, 33, first_ct=50000, tag=22)
    calls = [
        (first.u, first.v, first.y_rows),
        (np.concatenate([au, second.u]), np.concatenate([av, second.v]), np.concatenate([ay, second.y_rows])),
    ]
    for u, v, y in calls:
        ud, vd, yd = u64(u), u64(v), i32(y)
        want = hqc.hqc_decrypt_batch_staged(level, ud, vd, y=yd).cpu().numpy()
        got = hqc.hqc_decrypt_batch_staged_noalloc(level, ud, vd, y=yd).cpu().numpy()
        assert (got == want).all()
    assert (got[-33:] == second.m).all()


def test_noalloc_keyed_two_calls(hqc):
    wl = honest(1, 16, 300, first_ct=60000, tag=23)
    keys = hqc.Keyset(1, wl.y)
    kidx = torch.from_numpy(wl.key_idx.astype(np.int32)).cuda()
    ud, vd = u64(wl.u), u64(wl.v)
    want = hqc.hqc_decrypt_batch_keyed(1, ud, vd, keys, kidx).cpu().numpy()
    out = torch.full((300, wl.P.k), 0x5A, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        got = hqc.hqc_decrypt_batch_staged_noalloc(1, ud, vd, keys=keys, key_idx=kidx, m_out=out).cpu().numpy()
        assert (got == want).all() and (got == wl.m).all()
    keys.free()


@pytest.mark.parametrize("level", [1, 5])
def test_noalloc_rejects_counts_beyond_the_static_scratch(hqc, level):
    P = hqc.hqc_get_params(level)
    cnt = MAX_COUNT[level] + 1
    u = torch.zeros((cnt, P.W_u_pitch), dtype=torch.int64, device="cuda")
    v = torch.zeros((cnt, P.W_v), dtype=torch.int64, device="cuda")
    y = torch.zeros((cnt, P.w), dtype=torch.int32, device="cuda")
    m = torch.full((cnt, P.k), 7, dtype=torch.uint8, device="cuda")
    with pytest.raises(hqc.HqcError) as err:
        hqc.hqc_decrypt_batch_staged_noalloc(level, u, v, y=y, m_out=m)
    assert "exceeds the static scratch" in str(err.value) and str(MAX_COUNT[level]) in str(err.value)
    torch.cuda.synchronize()
    assert (m == 7).all()          # nothing was launched
    # the largest allowed count still works
    ok = hqc.hqc_decrypt_batch_staged_noalloc(level, u[:-1], v[:-1], y=y[:-1], m_out=m[:-1])
    want = hqc.hqc_decrypt_batch_staged(level, u[:-1], v[:-1], y=y[:-1])
    assert (ok == want).all()
