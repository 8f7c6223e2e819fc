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


def _median_ms(fn, reps=9):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


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
    times = {}
    for name, (u, v) in batches.items():
        ud = torch.from_numpy(np.ascontiguousarray(u).view(np.int64)).cuda()
        vd = torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).cuda()
        m = torch.empty((cnt, wl.P.k), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx, m)
        times[name] = _median_ms(lambda: hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx, m))
        if name == "honest":
            assert (m.cpu().numpy() == wl.m).all()
    keys.free()
    spread = max(times.values()) / min(times.values())
    assert spread < 1.05, times
