"""GPU parity of SHAKE256 and the KEM kernels against the CPU oracle (and
SHAKE256 against hashlib): bit-exact bytes, keys, ciphertexts and shared
secrets, on accepted and implicitly rejected decapsulations."""
import hashlib

import numpy as np
import pytest

import oracle
import synth

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


def cu8(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint8)).cuda()


def cu64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint64).view(np.int64)).cuda()


def cu32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.uint32).view(np.int32)).cuda()


def host_u64(t):
    return t.cpu().numpy().view(np.uint64)


def rows(count, width, tag):
    nw = (count * width + 7) // 8 + 1
    return synth.words(nw, tag=tag).view(np.uint8)[:count * width].reshape(count, width).copy()


@pytest.mark.parametrize("length", [0, 1, 33, 135, 136, 137, 272, 500, 4450])
def test_shake256_batch_matches_hashlib(hqc, length):
    count = 131  # two blocks of 128 threads, the second ragged
    msg = rows(count, length, tag=500 + length)
    for outlen in (1, 32, 136, 300):
        got = hqc.hqc_shake256_batch(cu8(msg), outlen).cpu().numpy()
        for i in (0, 1, 77, 127, 128, 130):
            assert got[i].tobytes() == hashlib.shake_256(msg[i].tobytes()).digest(outlen), (length, outlen, i)
        if length == 0:
            continue
        # every row against the oracle's SHAKE256 for one output length
        if outlen == 32:
            for i in range(count):
                assert got[i].tobytes() == oracle.shake256(msg[i].tobytes(), 32)


def _keys(level, nkeys, tag):
    return rows(nkeys, 32, tag), rows(nkeys, 32, tag + 1)


@pytest.mark.parametrize("level", LEVELS)
def test_kem_keygen_matches_oracle(hqc, level):
    sk, pk = _keys(level, 133, tag=600 + level)
    h, x, y, s = hqc.hqc_kem_keygen(level, cu8(sk), cu8(pk))
    oh, ox, oy, os_ = oracle.kem_keygen(level, sk, pk)
    assert (host_u64(h) == oh).all()
    assert (x.cpu().numpy().view(np.uint32) == ox).all()
    assert (y.cpu().numpy().view(np.uint32) == oy).all()
    assert (host_u64(s) == os_).all()


def _kem_setup(hqc, level, nkeys, count, tag):
    P = oracle.params(level)
    sk, pk = _keys(level, nkeys, tag)
    h, x, y, s = oracle.kem_keygen(level, sk, pk)
    sigma = rows(nkeys, P.k, tag + 2)
    kidx = synth.key_assignment(count, nkeys, tag=tag + 3)
    m = rows(count, P.k, tag + 4)
    salt = rows(count, 16, tag + 5)
    return P, h, y, s, sigma, kidx, m, salt


@pytest.mark.parametrize("level", LEVELS)
def test_encaps_matches_oracle(hqc, level):
    P, h, y, s, sigma, kidx, m, salt = _kem_setup(hqc, level, 5, 150, tag=700 + 10 * level)
    u, v, K = hqc.hqc_kem_encaps(level, cu64(h), cu64(s), cu32(kidx), cu8(m), cu8(salt))
    ou, ov, oK = oracle.kem_encaps(level, h, s, kidx, m, salt)
    assert (host_u64(u) == ou).all()
    assert (host_u64(v) == ov).all()
    assert (K.cpu().numpy() == oK).all()


@pytest.mark.parametrize("level", LEVELS)
def test_decaps_accept_and_reject_match_oracle(hqc, level):
    P, h, y, s, sigma, kidx, m, salt = _kem_setup(hqc, level, 4, 140, tag=800 + 10 * level)
    u, v, K = oracle.kem_encaps(level, h, s, kidx, m, salt)
    keys = hqc.Keyset(level, y)
    # tamper with a third of the items: a v bit, the salt, or u's padding
    ut, vt, st = u.copy(), v.copy(), salt.copy()
    vt[0::6, 5] ^= np.uint64(1 << 9)           # rejected (decodes to m, re-encryption differs)
    st[1::6, 3] ^= 0x40                         # rejected (other randomness)
    ut[2::6, P.W_u:] = np.uint64(0xA5A5A5A5)    # accepted (padding ignored)
    ut[3::6, 7] ^= np.uint64(1 << 33)           # rejected
    Kg, okg = hqc.hqc_kem_decaps(level, keys, cu64(h), cu64(s), cu8(sigma), cu32(kidx), cu64(ut), cu64(vt), cu8(st))
    oK, ook = oracle.kem_decaps(level, h, s, y, sigma, kidx, ut, vt, st)
    okg = okg.cpu().numpy().astype(bool)
    assert (okg == ook).all()
    assert (Kg.cpu().numpy() == oK).all()
    assert ook[2::6].all() and (oK[2::6] == K[2::6]).all()
    assert not ook[0::6].any() and not ook[1::6].any() and not ook[3::6].any()
    assert ook[4::6].all() and ook[5::6].all()
    keys.free()


@pytest.mark.parametrize("level,count,nkeys", [(1, 65536, 256), (3, 32768, 128), (5, 32768, 128)])
def test_kem_full_size_roundtrip_sampled(hqc, level, count, nkeys):
    """The bench sizes (65,536 HQC-1 items under 256 keys, 32,768 HQC-3 and
    HQC-5 items under 128): every decapsulated K equals the encapsulated one
    (a property at any size), and sampled items match the oracle byte for
    byte."""
    P = oracle.params(level)
    sk, pk = _keys(level, nkeys, tag=900 + level)
    h, x, y, s = hqc.hqc_kem_keygen(level, cu8(sk), cu8(pk))
    sigma = cu8(rows(nkeys, P.k, 902))
    kidx = cu32(synth.key_assignment(count, nkeys, tag=903))
    m = cu8(rows(count, P.k, 904))
    salt = cu8(rows(count, 16, 905))
    u, v, K = hqc.hqc_kem_encaps(level, h, s, kidx, m, salt)
    keys = hqc.Keyset(level, y.cpu().numpy().view(np.uint32))
    Kd, ok = hqc.hqc_kem_decaps(level, keys, h, s, sigma, kidx, u, v, salt)
    assert bool(ok.all().item()) and bool((Kd == K).all().item())
    idx = [0, 1, 4095, count // 2 + 7, count - 1]
    hh, ss, yy = host_u64(h), host_u64(s), y.cpu().numpy().view(np.uint32)
    ki = kidx.cpu().numpy()[idx]
    ou, ov, oK = oracle.kem_encaps(level, hh, ss, ki, m.cpu().numpy()[idx], salt.cpu().numpy()[idx])
    assert (host_u64(u)[idx] == ou).all() and (host_u64(v)[idx] == ov).all()
    assert (K.cpu().numpy()[idx] == oK).all()
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
def test_decaps_from_host_buffers_matches_device_path(hqc, level):
    """Chunked host-buffer decapsulation (ragged last chunk, one-item chunks,
    one chunk larger than the batch, and the library's own choice with
    chunk = 0) against the oracle, with rejections."""
    P, h, y, s, sigma, kidx, m, salt = _kem_setup(hqc, level, 3, 70, tag=1000 + 10 * level)
    u, v, K = oracle.kem_encaps(level, h, s, kidx, m, salt)
    v[::4, 2] ^= np.uint64(1 << 3)  # a quarter rejected
    oK, ook = oracle.kem_decaps(level, h, s, y, sigma, kidx, u, v, salt)
    keys = hqc.Keyset(level, y)
    hd, sd, sig = cu64(h), cu64(s), cu8(sigma)
    u_h = torch.from_numpy(u.view(np.int64).copy()).pin_memory()
    v_h = torch.from_numpy(v.view(np.int64).copy()).pin_memory()
    k_h = torch.from_numpy(kidx.astype(np.int32)).pin_memory()
    s_h = torch.from_numpy(salt.copy()).pin_memory()
    for chunk in (1, 16, 32, 100, 0):
        ws = torch.empty(hqc.hqc_kem_host_workspace_bytes(level, chunk or 100), dtype=torch.uint8, device="cuda")
        K_h, ok_h = hqc.hqc_kem_decaps_host(level, keys, hd, sd, sig, k_h, u_h, v_h, s_h, chunk=chunk, workspace=ws)
        torch.cuda.current_stream().synchronize()
        assert (K_h.numpy() == oK).all(), chunk
        assert (ok_h.numpy().astype(bool) == ook).all(), chunk
    short = torch.empty(hqc.hqc_kem_host_workspace_bytes(level, 64) - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(hqc.HqcError):
        hqc.hqc_kem_decaps_host(level, keys, hd, sd, sig, k_h, u_h, v_h, s_h, chunk=64, workspace=short)
    keys.free()


@pytest.mark.parametrize("level", LEVELS)
def test_kem_skips_bad_key_index(hqc, level):
    """An item whose key index is outside [0, nkeys) is skipped by
    encapsulation (u, v and K rows untouched) and by decapsulation (K row
    and ok entry untouched; zero from host buffers); every other item
    matches the oracle."""
    P, h, y, s, sigma, kidx, m, salt = _kem_setup(hqc, level, 4, 60, tag=900 + 10 * level)
    bad_rows = [2, 17, 59]
    bad = kidx.astype(np.int32).copy()
    bad[bad_rows] = (4, -1, 10 ** 7)
    good = np.setdiff1d(np.arange(60), bad_rows)
    ou, ov, oK = oracle.kem_encaps(level, h, s, kidx, m, salt)
    u0 = torch.full((60, P.W_u_pitch), 77, dtype=torch.int64, device="cuda")
    v0 = torch.full((60, P.W_v), 77, dtype=torch.int64, device="cuda")
    K0 = torch.full((60, 32), 0x3C, dtype=torch.uint8, device="cuda")
    gu, gv, gK = hqc.hqc_kem_encaps(level, cu64(h), cu64(s), cu32(bad), cu8(m), cu8(salt), u_out=u0, v_out=v0,
                                    K_out=K0)
    gu, gv, gK = host_u64(gu), host_u64(gv), gK.cpu().numpy()
    assert (gu[good] == ou[good]).all() and (gv[good] == ov[good]).all() and (gK[good] == oK[good]).all()
    assert (gu[bad_rows] == 77).all() and (gv[bad_rows] == 77).all() and (gK[bad_rows] == 0x3C).all()
    keys = hqc.Keyset(level, y)
    K1 = torch.full((60, 32), 0x3C, dtype=torch.uint8, device="cuda")
    ok1 = torch.full((60,), 9, dtype=torch.int32, device="cuda")
    Kd, okd = hqc.hqc_kem_decaps(level, keys, cu64(h), cu64(s), cu8(sigma), cu32(bad), cu64(ou), cu64(ov), cu8(salt),
                                 K_out=K1, ok_out=ok1)
    Kd, okd = Kd.cpu().numpy(), okd.cpu().numpy()
    assert (Kd[good] == oK[good]).all() and (okd[good] == 1).all()
    assert (Kd[bad_rows] == 0x3C).all() and (okd[bad_rows] == 9).all()
    # from host buffers the chunks come back whole: skipped rows are zero
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ws = torch.empty(hqc.hqc_kem_host_workspace_bytes(level, 16), dtype=torch.uint8, device="cuda")
    K_h, ok_h = hqc.hqc_kem_decaps_host(level, keys, cu64(h), cu64(s), cu8(sigma), pin(bad), pin(ou.view(np.int64)),
                                        pin(ov.view(np.int64)), pin(salt), chunk=16, workspace=ws)
    torch.cuda.synchronize()
    K_h, ok_h = K_h.numpy(), ok_h.numpy()
    assert (K_h[good] == oK[good]).all() and (ok_h[good] == 1).all()
    assert (K_h[bad_rows] == 0).all() and (ok_h[bad_rows] == 0).all()
    keys.free()


def test_decaps_ragged_counts_tampered_and_skipped(hqc):
    """HQC-1 decapsulation at counts below, at and above one block's warp
    count, a ragged count over every SM and a batch of 240,011 items (more
    than three waves of the persistent kernels), with every 97th item
    tampered and every 389th skipped: every accepted K equals the
    encapsulated one, tampered items are rejected with K(sigma, c) equal to
    the oracle's on a sample, and skipped items keep their rows."""
    level = 1
    P = oracle.params(level)
    nkeys = 64
    sk, pk = _keys(level, nkeys, tag=1200)
    h, x, y, s = hqc.hqc_kem_keygen(level, cu8(sk), cu8(pk))
    sigma = cu8(rows(nkeys, P.k, 1201))
    keys = hqc.Keyset(level, y.cpu().numpy().view(np.uint32))
    hh, ss, yy, sg = host_u64(h), host_u64(s), y.cpu().numpy().view(np.uint32), sigma.cpu().numpy()
    for count in (1, 23, 24, 25, 3647, 240011):
        kidx = cu32(synth.key_assignment(count, nkeys, tag=1202 + count))
        m = cu8(rows(count, P.k, 1203 + count))
        salt = cu8(rows(count, 16, 1204 + count))
        u, v, K = hqc.hqc_kem_encaps(level, h, s, kidx, m, salt)
        # every 97th item tampered (a v bit: rejected), every 389th skipped
        vt = v.clone()
        vt[0::97, 3] ^= 1 << 11
        kt = kidx.clone()
        kt[5::389] = nkeys + 3
        K0 = torch.full((count, 32), 0x5A, dtype=torch.uint8, device="cuda")
        ok0 = torch.full((count,), 7, dtype=torch.int32, device="cuda")
        Kd, ok = hqc.hqc_kem_decaps(level, keys, h, s, sigma, kt, u, vt, salt, K_out=K0, ok_out=ok0)
        okh, Kdh, Kh = ok.cpu().numpy(), Kd.cpu().numpy(), K.cpu().numpy()
        tam = np.zeros(count, bool)
        tam[0::97] = True
        skip = np.zeros(count, bool)
        skip[5::389] = True
        acc = ~tam & ~skip
        assert (okh[acc] == 1).all() and (Kdh[acc] == Kh[acc]).all(), count
        assert (okh[tam & ~skip] == 0).all() and not (Kdh[tam & ~skip] == Kh[tam & ~skip]).all(axis=1).any(), count
        assert (okh[skip] == 7).all() and (Kdh[skip] == 0x5A).all(), count
        idx = np.unique(np.r_[np.flatnonzero(tam & ~skip)[:3], np.flatnonzero(acc)[-2:], [count - 1]])
        idx = idx[~skip[idx]]
        ti = torch.from_numpy(idx).cuda()
        oK, ook = oracle.kem_decaps(level, hh, ss, yy, sg, kt[ti].cpu().numpy(), host_u64(u[ti]), host_u64(vt[ti]),
                                    salt[ti].cpu().numpy())
        assert (Kdh[idx] == oK).all() and (okh[idx] == ook).all(), count
    keys.free()
