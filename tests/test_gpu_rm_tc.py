"""S5-S7 alone (hqc_rm_decode_batch): the register butterflies and the
tensor-core product (tcgen05, fp16 operands, fp32 accumulators in tensor
memory) against the oracle's RM decoder, bit-exact.

Inputs: the received words w of real decryptions (from the oracle's dump
of adversarial and honest ciphertexts), uniformly random words, and blocks
built to tie (two codewords mixed half and half, all-zero and all-one
blocks), at counts that span many 128-block tiles and end in a ragged
tile."""
import numpy as np
import pytest

import oracle
import synth
from workloads import adversarial, honest

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


def oracle_r(level, w):
    """The oracle's RM byte of every block of every row of w (uint64 words)."""
    P = oracle.params(level)
    bits = np.unpackbits(np.ascontiguousarray(w, np.uint64).view(np.uint8), axis=1, bitorder="little")
    out = np.zeros((w.shape[0], P.n1), np.uint8)
    for i in range(w.shape[0]):
        for j in range(P.n1):
            out[i, j] = oracle.rm_decode_block(P.mult, bits[i, j * P.n2:(j + 1) * P.n2])
    return out


def tie_rows(level, count, tag):
    """Rows whose blocks are two RM codewords mixed half and half (many
    equal |F| at two indices), with all-zero and all-one blocks among them."""
    P = oracle.params(level)
    rng = np.random.default_rng(tag)
    rows = np.zeros((count, P.W_v), np.uint64)
    for i in range(count):
        bits = np.zeros(P.W_v * 64, np.uint8)
        for j in range(P.n1):
            kind = (i * P.n1 + j) % 7
            if kind == 0:
                blk = np.zeros(P.n2, np.uint8)
            elif kind == 1:
                blk = np.ones(P.n2, np.uint8)
            else:
                c1 = oracle.rm_encode_byte(int(rng.integers(256)))
                c2 = oracle.rm_encode_byte(int(rng.integers(256)))
                sel = rng.permutation(128) < 64
                blk = np.tile(np.where(sel, c1, c2).astype(np.uint8), P.mult)
            bits[j * P.n2:(j + 1) * P.n2] = blk
        rows[i] = np.packbits(bits, bitorder="little").view(np.uint64)
    return rows


def decode(hqc, level, w, tc):
    wd = torch.from_numpy(np.ascontiguousarray(w, np.uint64).view(np.int64)).cuda()
    return hqc.hqc_rm_decode_batch(level, wd, tensor_cores=tc).cpu().numpy()


@pytest.mark.parametrize("level", LEVELS)
def test_rm_decode_both_forms_match_the_oracle(hqc, level):
    P, au, av, ay = adversarial(level, tag=60 + level)
    wl = honest(level, 3, 12, first_ct=20000, tag=29)
    u = np.concatenate([au, wl.u]); v = np.concatenate([av, wl.v]); y = np.concatenate([ay, wl.y_rows])
    dumps = [oracle.decrypt_dump(level, u[i], v[i], y[i]) for i in range(u.shape[0])]
    w_real = np.stack([d["w"] for d in dumps])
    r_real = np.stack([d["r"] for d in dumps])
    w_rand = synth.words(37 * P.W_v, tag=300 + level).reshape(37, P.W_v)
    w_tie = tie_rows(level, 9, tag=310 + level)
    for w, want in ((w_real, r_real), (w_rand, oracle_r(level, w_rand)), (w_tie, oracle_r(level, w_tie))):
        for tc in (False, True):
            got = decode(hqc, level, w, tc)
            bad = np.argwhere(got != want)
            assert bad.size == 0, (tc, bad[:5])
    assert hqc.hqc_rm_tc_timeouts() == 0


@pytest.mark.parametrize("level", LEVELS)
def test_rm_tensor_cores_equal_butterflies_on_many_tiles(hqc, level):
    """Thousands of tiles (every block of every persistent block's loop)
    and a ragged last tile: the two forms give the same bytes."""
    P = oracle.params(level)
    count = 4099
    w = torch.from_numpy(synth.words(count * P.W_v, tag=320 + level).view(np.int64).reshape(count, P.W_v)).cuda()
    a = hqc.hqc_rm_decode_batch(level, w, tensor_cores=False)
    b = hqc.hqc_rm_decode_batch(level, w, tensor_cores=True)
    assert torch.equal(a, b)
    assert hqc.hqc_rm_tc_timeouts() == 0
    # spot check against the oracle
    rows = np.array([0, 1, count // 2, count - 2, count - 1])
    want = oracle_r(level, w[rows].cpu().numpy().view(np.uint64))
    assert (b[rows].cpu().numpy() == want).all()


def test_rm_decode_empty_batch(hqc):
    w = torch.zeros((0, hqc.hqc_get_params(1).W_v), dtype=torch.int64, device="cuda")
    for tc in (False, True):
        assert hqc.hqc_rm_decode_batch(1, w, tensor_cores=tc).shape == (0, hqc.hqc_get_params(1).n1)
