"""Data-independent running time of the fused kernel (HQC needs decryption
in constant time: Sec. III-B and III-D ask for it on CPU).  The kernel's
control flow depends only on the level; here its wall time on batches
with no errors, honest noise and maximal garbage must agree."""
import numpy as np
import pytest

import synth
from workloads import honest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hqc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2512_12904_gb300 as lib
    lib.load()
    return lib


def _interleaved_medians(fns, rounds=9):
    """Median time of each call in fns (name -> callable), measured round
    robin: every round times each call once, in a fixed cyclic order, so a
    drift of the GPU clock or the cache state during the measurement falls
    on all of them alike instead of on whichever ran first."""
    for fn in fns.values():
        for _ in range(3):
            fn()
    ts = {name: [] for name in fns}
    for _ in range(rounds):
        for name, fn in fns.items():
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts[name].append(a.elapsed_time(b))
    return {name: float(np.median(t)) for name, t in ts.items()}


@pytest.mark.parametrize("level", [1, 5])
def test_fused_time_does_not_depend_on_the_data(hqc, level):
    cnt = 8192 if level == 1 else 4096
    wl = honest(level, 16, cnt, first_ct=80000, tag=41)
    keys = hqc.Keyset(level, wl.y)
    kidx = torch.from_numpy(wl.key_idx.astype(np.int32)).cuda()
    batches = {
        "honest": (wl.u, wl.v),
        "zero": (np.zeros_like(wl.u), np.zeros_like(wl.v)),
        "garbage": (synth.words(wl.u.size, tag=42).reshape(wl.u.shape),
                    synth.words(wl.v.size, tag=43).reshape(wl.v.shape)),
    }
    fns, outs = {}, {}
    for name, (u, v) in batches.items():
        ud = torch.from_numpy(np.ascontiguousarray(u).view(np.int64)).cuda()
        vd = torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).cuda()
        m = torch.empty((cnt, wl.P.k), dtype=torch.uint8, device="cuda")
        outs[name] = m
        fns[name] = (lambda ud=ud, vd=vd, m=m: hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx, m))
    times = _interleaved_medians(fns)
    assert (outs["honest"].cpu().numpy() == wl.m).all()
    keys.free()
    spread = max(times.values()) / min(times.values())
    assert spread < 1.05, times


@pytest.mark.parametrize("level", [1, 5])
def test_decapsulation_time_does_not_depend_on_acceptance(hqc, level):
    """Implicit rejection must not show in the running time: batches that
    are all accepted, all rejected (tampered v) and all garbage take the
    same time."""
    cnt, nkeys = (16384, 64) if level == 1 else (4096, 32)
    P = hqc.hqc_get_params(level)

    def rows(n, width, tag):
        nw = (n * width + 7) // 8 + 1
        a = synth.words(nw, tag=tag).view(np.uint8)[:n * width].reshape(n, width).copy()
        return torch.from_numpy(a).cuda()

    h, x, y, s = hqc.hqc_kem_keygen(level, rows(nkeys, 32, 51), rows(nkeys, 32, 52))
    sigma = rows(nkeys, P.k, 53)
    kidx = torch.from_numpy(synth.key_assignment(cnt, nkeys, tag=54)).cuda()
    m, salt = rows(cnt, P.k, 55), rows(cnt, 16, 56)
    u, v, K = hqc.hqc_kem_encaps(level, h, s, kidx, m, salt)
    keys = hqc.Keyset(level, y.cpu().numpy().view(np.uint32))
    v_bad = v.clone()
    v_bad[:, 0] ^= 1 << 13
    g_u = torch.from_numpy(synth.words(u.numel(), tag=57).view(np.int64).reshape(tuple(u.shape))).cuda()
    g_v = torch.from_numpy(synth.words(v.numel(), tag=58).view(np.int64).reshape(tuple(v.shape))).cuda()
    ws = torch.empty(hqc.hqc_kem_workspace_bytes(level, cnt), dtype=torch.uint8, device="cuda")
    Kd = torch.empty_like(K)
    fns, oks, accepted = {}, {}, {}
    for name, (uu, vv) in {"accept": (u, v), "reject": (u, v_bad), "garbage": (g_u, g_v)}.items():
        oks[name] = torch.empty((cnt,), dtype=torch.int32, device="cuda")
        fns[name] = (lambda uu=uu, vv=vv, o=oks[name]:
                     hqc.hqc_kem_decaps(level, keys, h, s, sigma, kidx, uu, vv, salt, Kd, o, workspace=ws))
    times = _interleaved_medians(fns)
    accepted = {name: int(o.sum().item()) for name, o in oks.items()}
    keys.free()
    assert accepted == {"accept": cnt, "reject": 0, "garbage": 0}, accepted
    spread = max(times.values()) / min(times.values())
    assert spread < 1.05, times
