"""Client <-> server messages (Sec. 2: the client sends encrypted segments and
evaluation keys, the server returns output ciphertexts) on the host: round
trips of every kind, the documented byte layout, and every rejection --
other parameters, a flipped payload byte, a residue not below its prime, a
truncated message, a nonzero reserved byte."""
import struct
import zlib

import numpy as np
import pytest

from paper_2402_01296_gb300 import bcn


@pytest.fixture(scope="module")
def ctx():
    return bcn.Context(10, 3, 1, 1, device=-1)


def _cts(ctx, n=3, level=None, seed=5):
    level = level or ctx.L
    rng = np.random.default_rng(seed)
    a = np.empty((n, 2, level, ctx.N), dtype=np.uint32)
    for i in range(level):
        a[:, :, i] = rng.integers(0, ctx.q[i], (n, 2, ctx.N), dtype=np.uint32)
    return a


def _fnv1a(b: bytes) -> int:
    h = 2166136261
    for x in b:
        h = ((h ^ x) * 16777619) & 0xFFFFFFFF
    return h


def test_round_trips(ctx):
    sk, evk = ctx.keygen(3)
    gk = ctx.galois_keygen(sk, 5, 7)
    cts = _cts(ctx, level=2)
    pts = cts[:, 0].copy()
    for kind, arr, lv, g in ((ctx.MSG_CIPHERTEXTS, cts, 2, 0), (ctx.MSG_PLAINTEXTS, pts, 2, 0),
                             (ctx.MSG_RELIN_KEY, evk, 0, 0), (ctx.MSG_GALOIS_KEY, gk, 0, ctx.galois_elt(5))):
        m = ctx.deserialize(ctx.serialize(kind, arr, lv, g))
        assert m["kind"] == kind and m["level"] == lv and m["galois"] == g
        assert np.array_equal(m["words"], arr)


def test_byte_layout(ctx):
    cts = _cts(ctx, n=2, level=3)
    msg = ctx.serialize(ctx.MSG_CIPHERTEXTS, cts, 3)
    assert len(msg) == 64 + cts.size * 4
    assert msg[:4] == b"BCN1"
    kind, log_n, n_data, n_special, alpha, level, count, g, nw = struct.unpack_from("<9I", msg, 4)[:8] + (
        struct.unpack_from("<Q", msg, 36)[0],)
    assert (kind, log_n, n_data, n_special, alpha, level, count, g, nw) == (1, 10, 3, 1, 1, 3, 2, 0, cts.size)
    assert msg[48:64] == bytes(16)
    payload = msg[64:]
    assert payload == cts.astype("<u4").tobytes()  # little-endian words in the array's own order
    assert struct.unpack_from("<I", msg, 44)[0] == _fnv1a(payload)
    assert _fnv1a(b"a") == 0xE40C292C  # the published FNV-1a test vector
    assert zlib.crc32(payload) != 0  # (the payload is not empty)


def test_rejections(ctx):
    cts = _cts(ctx, n=1, level=3)
    msg = bytearray(ctx.serialize(ctx.MSG_CIPHERTEXTS, cts, 3))
    other = bcn.Context(10, 4, 1, 1, device=-1)
    with pytest.raises(bcn.BcnError):
        other.deserialize(bytes(msg))  # other parameters
    flipped = bytearray(msg)
    flipped[64 + 100] ^= 1
    with pytest.raises(bcn.BcnError, match="checksum"):
        ctx.deserialize(bytes(flipped))
    big = cts.copy()
    big[0, 1, 2, 7] = ctx.q[2]  # a residue equal to its prime
    bad = ctx.serialize(ctx.MSG_CIPHERTEXTS, big, 3)
    with pytest.raises(bcn.BcnError, match="below its prime"):
        ctx.deserialize(bad)
    with pytest.raises(bcn.BcnError, match="truncated"):
        ctx.deserialize(bytes(msg[:-4]))
    res = bytearray(msg)
    res[50] = 1
    with pytest.raises(bcn.BcnError, match="reserved"):
        ctx.deserialize(bytes(res))
    with pytest.raises(bcn.BcnError):
        ctx.deserialize(b"XCN1" + bytes(msg[4:]))
    sk, evk = ctx.keygen(3)
    with pytest.raises(bcn.BcnError):
        ctx.serialize(ctx.MSG_RELIN_KEY, evk, 0, galois=5)  # a Galois element on a relinearisation key


def test_seeded_encryption_c0_equals_full(ctx):
    """c0 of a seeded encryption is the c0 of the full encryption with the same
    key, plaintexts and seed (the seed then stands for c1)."""
    sk, _ = ctx.keygen(3)
    pts = _cts(ctx, n=4, level=ctx.L)[:, 0].copy()
    assert np.array_equal(ctx.encrypt_seeded(sk, pts, ctx.L, 11), ctx.encrypt(sk, pts, ctx.L, 11)[:, 0])
    imgs = np.random.default_rng(2).integers(0, 256, (3, 8, 8, 2), dtype=np.uint8)
    seg = (1, 2, 4, 5)
    assert np.array_equal(ctx.encrypt_segment_seeded(sk, imgs, seg, 2.0**20, 12),
                          ctx.encrypt_segment(sk, imgs, seg, 2.0**20, 12)[:, 0])


def test_integer_encoding_reduces_to_the_residues(ctx):
    """bcn_encode_i64's coefficients, reduced mod each prime, are bcn_encode's
    residues, below and above 2^52 in magnitude; a coefficient at 2^63 or more
    is refused."""
    v = np.random.default_rng(4).uniform(-3, 3, (4, ctx.N // 2))
    for scale in (2.0**30, 2.0**58):
        co = ctx.encode_i64(v, scale)
        q = np.array(ctx.q, dtype=np.int64)[None, :, None]
        assert np.array_equal((co[:, None, :] % q).astype(np.uint32), ctx.encode(v, ctx.L, scale))
    assert np.abs(ctx.encode_i64(v, 2.0**58)).max() > 2**53
    with pytest.raises(bcn.BcnError, match="2\\^63"):
        ctx.encode_i64(v, 2.0**70)
