"""GPU parity: every CUDA entry point against the CPU oracle, bit-exact.

Inputs come from the seeded generator and the oracle's own key generation
and encryption; expected values come only from the oracle.  Integer and
GF arithmetic, so the bar is exact equality of every word and byte.
"""
import numpy as np
import pytest

import oracle
import synth
from workloads import adversarial, honest, noisy_keyed, with_garbage_padding

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVELS = (1, 3, 5)


@pytest.fixture(scope="module")
def hqc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2512_12904_gb300 as lib
    lib.load()
    return lib


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.view(dtype)
    return t.cuda()


def u64(a):
    return dev(np.ascontiguousarray(a, np.uint64).view(np.int64))


def i32(a):
    return dev(np.ascontiguousarray(a).astype(np.uint32).view(np.int32))


def host(t):
    return t.cpu().numpy()


def oracle_dumps(level, u, v, y):
    keys = ["t", "w", "r", "S", "lam", "L", "errmask", "errval", "cw", "m", "flag"]
    out = {k: [] for k in keys}
    for i in range(u.shape[0]):
        d = oracle.decrypt_dump(level, u[i], v[i], y[i])
        for k in keys:
            out[k].append(d[k])
    return {k: np.array(vv) for k, vv in out.items()}


@pytest.mark.parametrize("level", LEVELS)
def test_debug_path_every_intermediate(hqc, level):
    P, u, v, y = adversarial(level, tag=level)
    wl = honest(level, 4, 20, first_ct=500, tag=3)
    u = np.concatenate([u, wl.u]); v = np.concatenate([v, wl.v]); y = np.concatenate([y, wl.y_rows])
    want = oracle_dumps(level, u, v, y)
    got = hqc.hqc_decrypt_debug(level, u64(u), u64(v), i32(y))
    torch.cuda.synchronize()
    assert (host(got["t"]).view(np.uint64) == want["t"]).all()
    assert (host(got["w"]).view(np.uint64) == want["w"]).all()
    for k in ("r", "S", "lam", "errmask", "errval", "cw", "m"):
        g = host(got[k])
        bad = np.argwhere(g != want[k])
        assert bad.size == 0, (k, bad[:5], g[tuple(bad[0])], want[k][tuple(bad[0])])
    assert (host(got["L"]) == want["L"]).all()
    assert (host(got["flag"]) == want["flag"]).all()
    # the honest tail decrypts to its messages
    assert (host(got["m"])[-20:] == wl.m).all()


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("form", (0, 1, 2))
def test_latency_forms_every_rs_intermediate(hqc, level, form):
    """The fused kernels' own intermediates (not only m): form 0 (four-warp
    team per ciphertext), form 1 (cluster of four blocks, whose RM bytes
    reach block 0 through distributed shared memory) and form 2 (the
    persistent throughput kernels' per-turn code: HQC-1's two words per warp
    with Horner syndromes, HQC-3's one, HQC-5's two-warp teams) dump each
    ciphertext's RM bytes, syndromes and Lambda as the warps that ran RS
    hold them; all equal the oracle's, on adversarial and honest
    ciphertexts."""
    P, u, v, y = adversarial(level, tag=70 + level)
    wl = honest(level, 3, 11, first_ct=22000, tag=31)
    u = np.concatenate([u, wl.u]); v = np.concatenate([v, wl.v]); y = np.concatenate([y, wl.y_rows])
    want = oracle_dumps(level, u, v, y)
    got = hqc.hqc_decrypt_debug_team(level, u64(u), u64(v), i32(y), form=form)
    torch.cuda.synchronize()
    for k in ("r", "S", "lam", "m"):
        g = host(got[k])
        bad = np.argwhere(g != want[k])
        assert bad.size == 0, (k, bad[:5])
    assert (host(got["m"])[-11:] == wl.m).all()


def test_throughput_turns_every_rs_intermediate(hqc):
    """Form 2 over 519 HQC-1 ciphertexts: 64 blocks of four warps take two
    words per warp per turn, so some warps run a second turn (reusing their
    shared memory and the block's syndrome table) and the last group holds
    one word.  Every ninth v is replaced by random words (far beyond delta
    errors).  RM bytes, syndromes, Lambda and m all equal the oracle's."""
    level, count = 1, 519
    P = oracle.params(level)
    wl = honest(level, 4, count, first_ct=31000, tag=33)
    v = wl.v.copy()
    v[::9] = synth.words(v[::9].size, tag=34).reshape(v[::9].shape)
    want = oracle_dumps(level, wl.u, v, wl.y_rows)
    got = hqc.hqc_decrypt_debug_team(level, u64(wl.u), u64(v), i32(wl.y_rows), form=2)
    torch.cuda.synchronize()
    for k in ("r", "S", "lam", "m"):
        g = host(got[k])
        bad = np.argwhere(g != want[k])
        assert bad.size == 0, (k, bad[:5])
    ok = np.ones(count, bool)
    ok[::9] = False
    assert (host(got["m"])[ok] == wl.m[ok]).all()


# launch shapes of the single-level path: the default picks the latency form
# (a four-warp team per ciphertext) for batches of at most 512; an explicit
# shape runs the persistent fused kernel
SHAPES = ((0, 0), (4, 0))


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_literal_matches_oracle(hqc, level, shape):
    P, u, v, y = adversarial(level, tag=10 + level)
    wl = honest(level, 5, 37, first_ct=900, tag=4)
    u = np.concatenate([u, with_garbage_padding(P, wl.u, tag=5)]); v = np.concatenate([v, wl.v])
    y = np.concatenate([y, wl.y_rows])
    want = oracle.decrypt(level, u, v, y)
    hqc.hqc_set_launch_config(level, *shape)
    try:
        got = host(hqc.hqc_decrypt_batch(level, u64(u), u64(v), i32(y)))
    finally:
        hqc.hqc_set_launch_config(level, 0, 0)
    assert (got == want).all()
    assert (got[-37:] == wl.m).all()


@pytest.mark.parametrize("level", LEVELS)
def test_fused_keyed_and_staged_match_oracle(hqc, level):
    wl = honest(level, 16, 256 if level == 1 else 96, tag=5)
    keys = hqc.Keyset(level, wl.y)
    kidx = dev(wl.key_idx.astype(np.int32))
    want = oracle.decrypt(level, wl.u, wl.v, wl.y_rows)
    assert (want == wl.m).all()
    got = host(hqc.hqc_decrypt_batch_keyed(level, u64(wl.u), u64(wl.v), keys, kidx))
    assert (got == want).all()
    got2 = host(hqc.hqc_decrypt_batch_staged(level, u64(wl.u), u64(wl.v), keys=keys, key_idx=kidx))
    assert (got2 == want).all()
    got3 = host(hqc.hqc_decrypt_batch_staged(level, u64(wl.u), u64(wl.v), y=i32(wl.y_rows)))
    assert (got3 == want).all()
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_counts(hqc, level, shape):
    wl = honest(level, 3, 41, first_ct=3000, tag=6)
    hqc.hqc_set_launch_config(level, *shape)
    try:
        for cnt in (1, 2, 31, 33, 41):
            got = host(hqc.hqc_decrypt_batch(level, u64(wl.u[:cnt]), u64(wl.v[:cnt]), i32(wl.y_rows[:cnt])))
            assert (got == wl.m[:cnt]).all(), cnt
        empty = hqc.hqc_decrypt_batch(level, u64(wl.u[:0]), u64(wl.v[:0]), i32(wl.y_rows[:0]))
        assert empty.shape == (0, wl.P.k)
    finally:
        hqc.hqc_set_launch_config(level, 0, 0)


@pytest.mark.parametrize("level", LEVELS)
def test_latency_form_at_its_limit_and_past_it(hqc, level):
    """Batches of 512 (the latency form's limit, one team per ciphertext)
    and 513 (the persistent fused kernel) both match the oracle's messages,
    keyed with an out-of-range key index in each (that item is skipped: its
    m row keeps what the caller put there)."""
    wl = honest(level, 4, 513, first_ct=12000, tag=13)
    keys = hqc.Keyset(level, wl.y)
    kidx = wl.key_idx.astype(np.int32).copy()
    want = wl.m.copy()
    kidx[7] = 10 ** 6
    want[7] = 0xA5
    for cnt in (512, 513):
        out = torch.full((cnt, wl.P.k), 0xA5, dtype=torch.uint8, device="cuda")
        got = host(hqc.hqc_decrypt_batch_keyed(level, u64(wl.u[:cnt]), u64(wl.v[:cnt]), keys, dev(kidx[:cnt]),
                                               m_out=out))
        assert (got == want[:cnt]).all(), cnt
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
def test_cluster_latency_form(hqc, level):
    """Batches of at most 8 run the cluster form (four blocks per ciphertext
    sharing the product and the RM blocks, block 0 decoding RS): literal
    adversarial rows (beyond-delta v, all-zero and all-one u, garbage
    padding, repeated and out-of-range supports) in batches of 1, 5 and 8,
    and keyed honest batches of 1, 8 (with an out-of-range key index,
    skipped) and 9 (the one-block team form), all against the oracle."""
    P, au, av, ay = adversarial(level, tag=40 + level)
    want = oracle_dumps(level, au, av, ay)["m"]
    for lo, hi in ((0, 1), (1, 6), (6, 14)):
        got = host(hqc.hqc_decrypt_batch(level, u64(au[lo:hi]), u64(av[lo:hi]), i32(ay[lo:hi])))
        assert (got == want[lo:hi]).all(), (lo, hi)
    wl = honest(level, 3, 9, first_ct=16000, tag=27)
    keys = hqc.Keyset(level, wl.y)
    kidx = wl.key_idx.astype(np.int32).copy()
    kidx[4] = 3  # == nkeys: skipped
    want_k = wl.m.copy()
    want_k[4] = 0xA5
    for cnt in (1, 8, 9):
        out = torch.full((cnt, wl.P.k), 0xA5, dtype=torch.uint8, device="cuda")
        got = host(hqc.hqc_decrypt_batch_keyed(level, u64(wl.u[:cnt]), u64(wl.v[:cnt]), keys, dev(kidx[:cnt]),
                                               m_out=out))
        assert (got == want_k[:cnt]).all(), cnt
    keys.free()


BAD_KEY_ROWS = (3, 40, 41, 69)


def with_bad_keys(kidx, nkeys):
    """Key indices with entries outside [0, nkeys): nkeys itself, -1, a
    large positive value and INT32_MIN."""
    k = kidx.astype(np.int32).copy()
    for r, val in zip(BAD_KEY_ROWS, (nkeys, -1, 10 ** 6, -2 ** 31)):
        k[r] = val
    return k


@pytest.mark.parametrize("level", LEVELS)
def test_bad_key_index_is_skipped_by_every_keyed_form(hqc, level):
    """One rule for a key index outside [0, nkeys): the item is skipped and
    its output row keeps the caller's bytes, in the keyed fused kernel (both
    the latency form and the persistent kernel), the per-stage form, the
    allocation-free form and a graph plan (the host-buffer pipeline returns
    zero rows for them); every other item matches the oracle, and
    hqc_count_bad_key_idx counts them."""
    wl = honest(level, 4, 70, first_ct=14000, tag=24)
    keys = hqc.Keyset(level, wl.y)
    kidx_np = with_bad_keys(wl.key_idx, 4)
    kidx = dev(kidx_np)
    ud, vd = u64(wl.u), u64(wl.v)
    want = wl.m.copy()
    want[list(BAD_KEY_ROWS)] = 0xA5
    assert hqc.hqc_count_bad_key_idx(kidx, 4) == len(BAD_KEY_ROWS)
    assert hqc.hqc_count_bad_key_idx(kidx, 2 ** 31 - 1) == 2  # only the negative ones
    assert hqc.hqc_count_bad_key_idx(kidx[:0], 4) == 0

    def fresh():
        return torch.full((70, wl.P.k), 0xA5, dtype=torch.uint8, device="cuda")

    outs = {}
    outs["latency"] = hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx, m_out=fresh())
    hqc.hqc_set_launch_config(level, 4, 0)
    try:
        outs["persistent"] = hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx, m_out=fresh())
    finally:
        hqc.hqc_set_launch_config(level, 0, 0)
    outs["staged"] = hqc.hqc_decrypt_batch_staged(level, ud, vd, keys=keys, key_idx=kidx, m_out=fresh())
    outs["noalloc"] = hqc.hqc_decrypt_batch_staged_noalloc(level, ud, vd, keys=keys, key_idx=kidx, m_out=fresh())
    m_plan = fresh()
    plan = hqc.hqc_plan_create_keyed(level, ud, vd, keys, kidx, m_plan, autotune=False)
    m_plan.fill_(0xA5)
    plan.launch()
    outs["plan"] = m_plan
    u_h = torch.from_numpy(wl.u.view(np.int64).copy()).pin_memory()
    v_h = torch.from_numpy(wl.v.view(np.int64).copy()).pin_memory()
    k_h = torch.from_numpy(kidx_np).pin_memory()
    m_h = torch.full((70, wl.P.k), 0xA5, dtype=torch.uint8).pin_memory()
    ws = torch.empty(hqc.hqc_host_workspace_bytes(level, 16), dtype=torch.uint8, device="cuda")
    hqc.hqc_decrypt_host_keyed(level, u_h, v_h, keys, k_h, m_h, chunk=16, workspace=ws)
    torch.cuda.synchronize()
    for name, got in outs.items():
        assert (got.cpu().numpy() == want).all(), name
    # the host-buffer form copies whole chunks back: skipped rows are zero
    want_h = want.copy()
    want_h[list(BAD_KEY_ROWS)] = 0
    assert (m_h.numpy() == want_h).all()
    plan.destroy()
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
def test_encrypt_skips_bad_key_index(hqc, level):
    """Encryption follows the same rule: an item whose key index is outside
    [0, nkeys) leaves its u and v rows as the caller left them."""
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, 4, first=60)
    s = oracle.keygen(level, h, x, y)
    m, r1, r2, e = synth.ciphertext_randomness(S, 70, first=70)
    kidx = synth.key_assignment(70, 4, tag=25)
    want_u, want_v = oracle.encrypt(level, h, s, kidx, m, r1, r2, e)
    bad = with_bad_keys(kidx, 4)
    u_out = torch.full((70, P.W_u_pitch), 0x0F0F, dtype=torch.int64, device="cuda")
    v_out = torch.full((70, P.W_v), 0x0F0F, dtype=torch.int64, device="cuda")
    gu, gv = hqc.hqc_encrypt_batch(level, u64(h), u64(s), dev(bad), dev(m), i32(r1), i32(r2), i32(e),
                                   u_out=u_out, v_out=v_out)
    gu, gv = host(gu).view(np.uint64), host(gv).view(np.uint64)
    good = np.setdiff1d(np.arange(70), BAD_KEY_ROWS)
    assert (gu[good] == want_u[good]).all() and (gv[good] == want_v[good]).all()
    assert (gu[list(BAD_KEY_ROWS)] == 0x0F0F).all() and (gv[list(BAD_KEY_ROWS)] == 0x0F0F).all()


@pytest.mark.parametrize("level", LEVELS)
def test_launch_shapes_agree(hqc, level):
    wl = honest(level, 4, 200, first_ct=7000, tag=7)
    keys = hqc.Keyset(level, wl.y)
    kidx = dev(wl.key_idx.astype(np.int32))
    ref = None
    for wpc, cps in ((0, 0), (1, 1), (3, 1), (8, 0), (16, 0)):
        try:
            hqc.hqc_set_launch_config(level, wpc, cps)
            got = host(hqc.hqc_decrypt_batch_keyed(level, u64(wl.u), u64(wl.v), keys, kidx))
        except hqc.HqcError:
            continue  # shape does not fit on this device
        finally:
            hqc.hqc_set_launch_config(level, 0, 0)
        ref = got if ref is None else ref
        assert (got == wl.m).all()
    assert ref is not None


@pytest.mark.parametrize("level", LEVELS)
def test_keygen_and_encrypt_match_oracle(hqc, level):
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, 6, first=40)
    want_s = oracle.keygen(level, h, x, y)
    got_s = host(hqc.hqc_keygen_batch(level, u64(h), i32(x), i32(y))).view(np.uint64)
    assert (got_s == want_s).all()
    m, r1, r2, e = synth.ciphertext_randomness(S, 50, first=50)
    kidx = synth.key_assignment(50, 6, tag=9)
    want_u, want_v = oracle.encrypt(level, h, want_s, kidx, m, r1, r2, e)
    gu, gv = hqc.hqc_encrypt_batch(level, u64(h), u64(want_s), dev(kidx.astype(np.int32)), dev(m), i32(r1), i32(r2),
                                   i32(e))
    assert (host(gu).view(np.uint64) == want_u).all()
    assert (host(gv).view(np.uint64) == want_v).all()


def test_mixed_levels_one_launch(hqc):
    parts = {}
    for lvl, cnt in ((1, 40), (3, 35), (5, 25)):
        parts[lvl] = honest(lvl, 8, cnt, first_ct=20000, tag=11)
    order = synth.shuffle(np.arange(100, dtype=np.int32), tag=12)
    seq = [(1, i) for i in range(40)] + [(3, i) for i in range(35)] + [(5, i) for i in range(25)]
    seq = [seq[j] for j in order]
    items = np.zeros(len(seq), dtype=__import__("paper_2512_12904_gb300").ITEM_DTYPE)
    arena, m_off, words = [], 0, 0
    for idx, (lvl, i) in enumerate(seq):
        wl = parts[lvl]
        items[idx] = (lvl, wl.key_idx[i], words, words + wl.P.W_u_pitch, m_off)
        arena.append(wl.u[i]); arena.append(wl.v[i])
        words += wl.P.W_u_pitch + wl.P.W_v
        m_off += wl.P.k
    arena = np.concatenate(arena)
    keys = [hqc.Keyset(l, parts[l].y) for l in (1, 3, 5)]
    # the default shape runs this 100-item batch in the latency form (a team
    # per item); an explicit shape runs the one-warp-per-item mixed kernel
    for shape in SHAPES:
        hqc.hqc_set_launch_config(0, *shape)
        try:
            m_arena = torch.full((m_off,), 0xAA, dtype=torch.uint8, device="cuda")
            hqc.hqc_decrypt_mixed(dev(items.view(np.uint8)), u64(arena), keys, m_arena)
            got = host(m_arena)
        finally:
            hqc.hqc_set_launch_config(0, 0, 0)
        pos = 0
        for lvl, i in seq:
            k = parts[lvl].P.k
            assert (got[pos: pos + k] == parts[lvl].m[i]).all(), shape
            pos += k
    # an item with an out-of-range key is skipped, the rest still decrypt
    items2 = items.copy()
    items2[0]["key"] = 10 ** 6
    m2 = torch.full((m_off,), 0x55, dtype=torch.uint8, device="cuda")
    hqc.hqc_decrypt_mixed(dev(items2.view(np.uint8)), u64(arena), keys, m2)
    g2 = host(m2)
    k0 = parts[seq[0][0]].P.k
    assert (g2[:k0] == 0x55).all() and (g2[k0:] == got[k0:]).all()


def test_full_size_hqc1_bulk_sampled(hqc):
    # 65,536 HQC-1 ciphertexts under 256 keys in one keyed launch: every m
    # must round-trip, and a sample is compared with the oracle's decryption
    wl = honest(1, 256, 65536, tag=13)
    keys = hqc.Keyset(1, wl.y)
    got = host(hqc.hqc_decrypt_batch_keyed(1, u64(wl.u), u64(wl.v), keys, dev(wl.key_idx.astype(np.int32))))
    assert (got == wl.m).all()
    sample = synth.below(65536, 128, tag=14)
    want = oracle.decrypt(1, wl.u[sample], wl.v[sample], wl.y_rows[sample])
    assert (got[sample] == want).all()


def _mixed_batch(hqc, counts=((1, 40), (3, 35), (5, 25)), first_ct=30000, tag=15):
    parts = {lvl: honest(lvl, 6, cnt, first_ct=first_ct, tag=tag) for lvl, cnt in counts}
    seq = [(lvl, i) for lvl, cnt in counts for i in range(cnt)]
    order = synth.shuffle(np.arange(len(seq), dtype=np.int32), tag=tag + 1)
    seq = [seq[j] for j in order]
    items = np.zeros(len(seq), dtype=hqc.ITEM_DTYPE)
    arena, m_off, words, want = [], 0, 0, []
    for idx, (lvl, i) in enumerate(seq):
        wl = parts[lvl]
        items[idx] = (lvl, wl.key_idx[i], words, words + wl.P.W_u_pitch, m_off)
        arena += [wl.u[i], wl.v[i]]
        words += wl.P.W_u_pitch + wl.P.W_v
        m_off += wl.P.k
        want.append(wl.m[i])
    keys = [hqc.Keyset(l, parts[l].y) if l in parts else None for l in (1, 3, 5)]
    return dev(items.view(np.uint8)), u64(np.concatenate(arena)), keys, m_off, np.concatenate(want)


def test_mixed_plan_graph_autotuned(hqc):
    items, arena, keys, nbytes, want = _mixed_batch(hqc)
    m = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    plan = hqc.hqc_plan_create_mixed(items, arena, keys, m, autotune=True)
    info = plan.info()
    assert info["form"] in hqc.PLAN_FORMS
    for _ in range(2):
        m.zero_()
        plan.launch()
        torch.cuda.synchronize()
        assert (host(m) == want).all()
    plan.destroy()
    # without tuning: the single-kernel form with the default shape
    plan2 = hqc.hqc_plan_create_mixed(items, arena, keys, m, autotune=False)
    m.zero_()
    plan2.launch()
    torch.cuda.synchronize()
    assert plan2.info()["form"] == "mixed-single-kernel" and (host(m) == want).all()
    plan2.destroy()


def test_mixed_plan_single_level_present(hqc):
    items, arena, keys, nbytes, want = _mixed_batch(hqc, counts=((3, 30),), first_ct=31000, tag=17)
    m = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    plan = hqc.hqc_plan_create_mixed(items, arena, keys, m, autotune=True)
    plan.launch()
    torch.cuda.synchronize()
    assert (host(m) == want).all()
    plan.destroy()


@pytest.mark.parametrize("level", LEVELS)
def test_keyed_plan_graph_replay(hqc, level):
    wl = honest(level, 8, 300 if level == 1 else 120, first_ct=32000, tag=18)
    keys = hqc.Keyset(level, wl.y)
    ud, vd = u64(wl.u), u64(wl.v)
    kidx = dev(wl.key_idx.astype(np.int32))
    m = torch.zeros((ud.shape[0], wl.P.k), dtype=torch.uint8, device="cuda")
    plan = hqc.hqc_plan_create_keyed(level, ud, vd, keys, kidx, m, autotune=True)
    direct = host(hqc.hqc_decrypt_batch_keyed(level, ud, vd, keys, kidx))
    for _ in range(3):
        m.zero_()
        plan.launch()
        torch.cuda.synchronize()
        assert (host(m) == direct).all() and (direct == wl.m).all()
    assert plan.info()["tuned_ms"] > 0
    plan.destroy()
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
def test_host_pipelined_matches_oracle(hqc, level):
    """Chunked host-buffer decryption: ragged last chunk, one-item chunks,
    a single chunk larger than the batch, the empty batch and a short
    workspace."""
    wl = honest(level, 5, 75, first_ct=9000, tag=8)
    keys = hqc.Keyset(level, wl.y)
    u_h = torch.from_numpy(wl.u.view(np.int64).copy()).pin_memory()
    v_h = torch.from_numpy(wl.v.view(np.int64).copy()).pin_memory()
    k_h = torch.from_numpy(wl.key_idx.astype(np.int32)).pin_memory()
    for chunk in (1, 16, 32, 200):
        ws = torch.empty(hqc.hqc_host_workspace_bytes(level, chunk), dtype=torch.uint8, device="cuda")
        m_h = hqc.hqc_decrypt_host_keyed(level, u_h, v_h, keys, k_h, chunk=chunk, workspace=ws)
        torch.cuda.current_stream().synchronize()
        assert (m_h.numpy() == wl.m).all(), chunk
    m0 = hqc.hqc_decrypt_host_keyed(level, u_h[:0], v_h[:0], keys, k_h[:0], chunk=8, workspace=ws)
    assert m0.shape == (0, wl.P.k)
    short = torch.empty(hqc.hqc_host_workspace_bytes(level, 64) - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(hqc.HqcError):
        hqc.hqc_decrypt_host_keyed(level, u_h, v_h, keys, k_h, chunk=64, workspace=short)
    keys.free()


def test_mixed_from_host_buffers(hqc):
    """Chunked mixed-level decryption from pinned host buffers: chunks that
    split levels unevenly, a ragged last chunk, an item skipped for its key
    (its m bytes come back zero), and a batch out of arena order refused."""
    parts = {}
    for lvl, cnt in ((1, 40), (3, 35), (5, 25)):
        parts[lvl] = honest(lvl, 8, cnt, first_ct=21000, tag=13)
    order = synth.shuffle(np.arange(100, dtype=np.int32), tag=14)
    seq = [(1, i) for i in range(40)] + [(3, i) for i in range(35)] + [(5, i) for i in range(25)]
    seq = [seq[j] for j in order]
    items = np.zeros(len(seq), dtype=hqc.ITEM_DTYPE)
    arena, m_off, words, want = [], 0, 0, []
    for idx, (lvl, i) in enumerate(seq):
        wl = parts[lvl]
        items[idx] = (lvl, wl.key_idx[i], words, words + wl.P.W_u_pitch, m_off)
        arena.append(wl.u[i]); arena.append(wl.v[i])
        words += wl.P.W_u_pitch + wl.P.W_v
        m_off += wl.P.k
        want.append(wl.m[i])
    want = np.concatenate(want)
    arena_h = torch.from_numpy(np.concatenate(arena).view(np.int64)).pin_memory()
    keys = [hqc.Keyset(l, parts[l].y) for l in (1, 3, 5)]
    items_h = torch.from_numpy(items.view(np.uint8).copy()).pin_memory()
    for chunk in (1, 7, 33, 100, 0):
        m_h = torch.full((m_off,), 0xAA, dtype=torch.uint8).pin_memory()
        hqc.hqc_decrypt_mixed_host(items_h, arena_h, keys, m_h, chunk=chunk)
        torch.cuda.current_stream().synchronize()
        assert (m_h.numpy() == want).all(), chunk
    items2 = items.copy()
    items2[5]["key"] = 10 ** 6
    m_h = torch.full((m_off,), 0xAA, dtype=torch.uint8).pin_memory()
    hqc.hqc_decrypt_mixed_host(torch.from_numpy(items2.view(np.uint8).copy()).pin_memory(), arena_h, keys, m_h,
                               chunk=16)
    torch.cuda.current_stream().synchronize()
    g = m_h.numpy()
    s5, k5 = int(items2[5]["m_off"]), parts[seq[5][0]].P.k
    assert (g[s5:s5 + k5] == 0).all()
    g[s5:s5 + k5] = want[s5:s5 + k5]
    assert (g == want).all()
    swapped = items.copy()
    swapped[[3, 4]] = swapped[[4, 3]]
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    with pytest.raises(hqc.HqcError):
        hqc.hqc_decrypt_mixed_host(torch.from_numpy(swapped.view(np.uint8).copy()), arena_h, keys,
                                   torch.zeros(m_off, dtype=torch.uint8), chunk=16, workspace=ws)
    for k in keys:
        k.free()



def test_host_pipelined_full_size_sampled(hqc):
    """65,536 HQC-1 ciphertexts from pinned host buffers with the library's
    own chunking (whole waves, two slots): every m equals the device path's,
    and sampled items equal the oracle."""
    level, count, nkeys = 1, 65536, 256
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, nkeys, first=300)
    s = oracle.keygen(level, h, x, y)
    m, r1, r2, e = synth.ciphertext_randomness(S, count, first=400000)
    kidx = synth.key_assignment(count, nkeys, tag=31)
    hd, sd = u64(h), u64(s)
    u_d, v_d = hqc.hqc_encrypt_batch(level, hd, sd, dev(kidx.astype(np.int32)), dev(m), i32(r1), i32(r2), i32(e))
    keys = hqc.Keyset(level, y)
    u_h, v_h = u_d.cpu().pin_memory(), v_d.cpu().pin_memory()
    k_h = torch.from_numpy(kidx.astype(np.int32)).pin_memory()
    m_h = hqc.hqc_decrypt_host_keyed(level, u_h, v_h, keys, k_h)
    torch.cuda.current_stream().synchronize()
    assert (m_h.numpy() == m).all()
    idx = [0, 9727, 9728, 40000, count - 1]
    want = oracle.decrypt(level, u_h.numpy()[idx].view(np.uint64), v_h.numpy()[idx].view(np.uint64), y[kidx[idx]])
    assert (m_h.numpy()[idx] == want).all()
    keys.free()


def test_large_batch_2_20_hqc1(hqc):
    """2^20 HQC-1 ciphertexts (4.6 GB of u and v) in one keyed launch: 64-bit
    row arithmetic and many waves of the persistent grid; every m checked on
    the device, sampled items against the oracle."""
    level, count, nkeys = 1, 1 << 20, 64
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, nkeys, first=500)
    s = oracle.keygen(level, h, x, y)
    chunk = 1 << 17
    keys = hqc.Keyset(level, y)
    hd, sd = u64(h), u64(s)
    u_d = torch.empty((count, P.W_u_pitch), dtype=torch.int64, device="cuda")
    v_d = torch.empty((count, P.W_v), dtype=torch.int64, device="cuda")
    m_d = torch.empty((count, P.k), dtype=torch.uint8, device="cuda")
    kidx = synth.key_assignment(count, nkeys, tag=41)
    k_d = dev(kidx.astype(np.int32))
    for c0 in range(0, count, chunk):
        m, r1, r2, e = synth.ciphertext_randomness(S, chunk, first=1_000_000 + c0)
        m_d[c0:c0 + chunk] = dev(m)
        hqc.hqc_encrypt_batch(level, hd, sd, k_d[c0:c0 + chunk], m_d[c0:c0 + chunk], i32(r1), i32(r2), i32(e),
                              u_out=u_d[c0:c0 + chunk], v_out=v_d[c0:c0 + chunk])
    got = hqc.hqc_decrypt_batch_keyed(level, u_d, v_d, keys, k_d)
    assert bool((got == m_d).all().item())
    idx = [0, 123457, count // 2, count - 1]
    want = oracle.decrypt(level, host(u_d[idx]).view(np.uint64), host(v_d[idx]).view(np.uint64), y[kidx[idx]])
    assert (host(got[idx]) == want).all()
    keys.free()


VARIANTS = ("default", "solo-G1", "solo-G2", "solo-G4", "team2")


@pytest.mark.parametrize("level", LEVELS)
def test_every_keyed_plan_variant_matches_oracle(hqc, level):
    """Every kernel variant the keyed plan's tuner chooses among -- solo
    warps with G = 1, 2, 4 ciphertexts per turn, two-warp teams and the
    library's default -- at a full-GPU shape and at a one-warp-per-SM shape
    (several turns per warp), decrypts exactly as the oracle does on a batch
    with hard ciphertexts mixed in; G = 4 does not exist at HQC-5.  The
    tuned plan reports its choice and the candidates it timed."""
    wl, u, v = noisy_keyed(level, 8, 700, first_ct=40000, tag=60 + level)
    want = oracle.decrypt(level, u, v, wl.y_rows)
    keys = hqc.Keyset(level, wl.y)
    ud, vd, kidx = u64(u), u64(v), dev(wl.key_idx.astype(np.int32))
    for var in VARIANTS:
        for w, c in ((0, 0), (2, 1)):
            m = torch.full((700, wl.P.k), 0xA5, dtype=torch.uint8, device="cuda")
            if var == "solo-G4" and level == 5:
                with pytest.raises(hqc.HqcError):
                    hqc.hqc_plan_create_keyed(level, ud, vd, keys, kidx, m, variant=var)
                continue
            plan = hqc.hqc_plan_create_keyed(level, ud, vd, keys, kidx, m, variant=var, warps_per_cta=w,
                                             ctas_per_sm=c)
            plan.launch()
            torch.cuda.synchronize()
            assert (host(m) == want).all(), (var, w, c)
            plan.destroy()
    m = torch.zeros((700, wl.P.k), dtype=torch.uint8, device="cuda")
    plan = hqc.hqc_plan_create_keyed(level, ud, vd, keys, kidx, m, autotune=True)
    d = plan.describe()
    assert d["form"] == "keyed" and d["variant"] in VARIANTS
    assert len(d["candidates"]) >= 40
    assert [x["ms"] for x in d["candidates"]] == sorted(x["ms"] for x in d["candidates"])
    assert abs(d["candidates"][0]["ms"] - d["tuned_ms"]) < 1e-6
    m.zero_()
    plan.launch()
    torch.cuda.synchronize()
    assert (host(m) == want).all()
    plan.destroy()
    keys.free()


def _noisy_mixed_batch(hqc, counts, tag):
    """A shuffled HQC-1/3/5 item list (noisy ciphertexts), its arena and the
    oracle's messages in arena order."""
    parts = {lvl: noisy_keyed(lvl, 8, cnt, first_ct=45000, tag=tag + lvl) for lvl, cnt in counts}
    seq = [(lvl, i) for lvl, cnt in counts for i in range(cnt)]
    order = synth.shuffle(np.arange(len(seq), dtype=np.int32), tag=tag)
    seq = [seq[j] for j in order]
    items = np.zeros(len(seq), dtype=hqc.ITEM_DTYPE)
    arena, want, words, m_off = [], [], 0, 0
    exp = {lvl: oracle.decrypt(lvl, u, v, wl.y_rows) for lvl, (wl, u, v) in parts.items()}
    for idx, (lvl, i) in enumerate(seq):
        wl, u, v = parts[lvl]
        items[idx] = (lvl, wl.key_idx[i], words, words + wl.P.W_u_pitch, m_off)
        arena += [u[i], v[i]]
        want.append(exp[lvl][i])
        words += wl.P.W_u_pitch + wl.P.W_v
        m_off += wl.P.k
    keys = [hqc.Keyset(l, parts[l][0].y) for l in (1, 3, 5)]
    return dev(items.view(np.uint8)), u64(np.concatenate(arena)), keys, np.concatenate(want), m_off


def test_every_mixed_plan_form_matches_oracle(hqc):
    """Every form of the mixed plan -- the single mixed kernel, the levels
    side by side as graph branches, one after another, and one launch by
    block ranges -- with every per-level kernel variant, matches the
    oracle; the tuned plan reports per-level variants and candidates."""
    items, arena, keys, want, m_bytes = _noisy_mixed_batch(hqc, ((1, 400), (3, 350), (5, 250)), tag=300)

    def check(**kw):
        m = torch.full((m_bytes,), 0xA5, dtype=torch.uint8, device="cuda")
        plan = hqc.hqc_plan_create_mixed(items, arena, keys, m, **kw)
        plan.launch()
        torch.cuda.synchronize()
        assert (host(m) == want).all(), kw
        return plan

    check(form=1).destroy()
    check(form=1, warps_per_cta=4, ctas_per_sm=1).destroy()
    for var in VARIANTS:
        vs = [var if (var != "solo-G4" or lvl != 5) else "default" for lvl in (1, 3, 5)]
        check(form=2, variants=vs, grids=(20, 40, 92)).destroy()
        check(form=3, variants=vs).destroy()
    check(form=4, grids=(30, 50, 72)).destroy()
    check(form=4, grids=(3, 2, 5)).destroy()
    with pytest.raises(hqc.HqcError):
        check(form=2, grids=(0, 40, 92))
    plan = check(autotune=True)
    d = plan.describe()
    assert d["form"] in hqc.PLAN_FORMS and len(d["level_variants"]) == 3
    whole = [c for c in d["candidates"] if c["whole_batch"]]
    forms = {c["form"] for c in whole}
    assert forms == set(hqc.PLAN_FORMS), forms
    assert abs(min(c["ms"] for c in whole) - d["tuned_ms"]) < 1e-6
    assert any(not c["whole_batch"] and len(c["levels"]) == 1 for c in d["candidates"])
    plan.destroy()
    for k in keys:
        k.free()
