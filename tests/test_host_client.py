"""Host-side (client) calls of libbcn.so against the oracle, and the C-ABI
symbol table against include/bcn.h.  No GPU needed: the context is host-only.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "bcn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bcn_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = bcn.lib()
    declared = header_functions()
    assert len(declared) >= 30
    for name in declared:
        assert hasattr(L, name), name
    # and the binding covers exactly the declared surface
    assert sorted(bcn.exported_symbols()) == declared


@pytest.fixture(scope="module", params=[(6, 3, 1, 1), (12, 3, 1, 1), (13, 4, 2, 2)])
def pair(request):
    return bcn.Context(*request.param, device=-1), O.Params(*request.param)


def test_primes_match(pair):
    c, P = pair
    assert c.primes == P.primes
    assert c.dnum == P.dnum(P.L)


def test_keygen_bit_exact(pair):
    c, P = pair
    for seed in (3, 77):
        sk, evk = c.keygen(seed)
        sk2, evk2 = P.keygen(seed)
        assert np.array_equal(sk, sk2) and np.array_equal(evk, evk2)


def test_galois_keygen_bit_exact(pair):
    """Galois keys (rotation keys, App. A Rot) from the library's client call
    equal the oracle's, residue by residue, for rotations left and right."""
    c, P = pair
    sk, _ = P.keygen(3)
    for steps in (1, 5, -2):
        assert c.galois_elt(steps) == P.galois_elt(steps)
        assert np.array_equal(c.galois_keygen(sk, steps, 12), P.galois_keygen(sk, steps, 12))


def test_encrypt_bit_exact(pair):
    c, P = pair
    sk, _ = P.keygen(3)
    pts = workloads.random_residues(P.q, (5,), P.N, 9)
    for level in (P.L, 1):
        a = c.encrypt(sk, np.ascontiguousarray(pts[:, :level]), level, 4)
        b = P.encrypt(sk, np.ascontiguousarray(pts[:, :level]), level, 4)
        assert np.array_equal(a, b)


def test_encode_matches_direct_sum(pair):
    """FFT encode vs the oracle's direct canonical-embedding sum: fp64 rounding
    differs, so |delta m_j| <= 1 + 2^-40 * scale * max|z| (fp64 on both sides)."""
    c, P = pair
    rng = np.random.default_rng(1)
    # 2^80: coefficients beyond int64, taken as the exact integers of the fp64 products
    for B, scale in ((P.N // 2, 2.0**25), (P.N // 4 + 3, 2.0**40), (P.N // 8 + 1, 2.0**80)):
        z = rng.uniform(-1.5, 1.5, (3, B))
        a = c.encode(z, P.L, scale)
        m = O.encode_coeffs(z, P.N, scale)
        ref = O.to_residues(m, P.q)
        d = O.crt_centered(a, P.q) - m
        tol = 1 + 2.0**-40 * scale * 1.5
        assert np.abs(np.array(d, dtype=np.float64)).max() <= tol
        if scale <= 2.0**30:
            assert np.mean(a != ref) < 0.05  # nearly all coefficients identical


def test_decrypt_decode_matches_oracle(pair):
    c, P = pair
    sk, _ = P.keygen(3)
    B = P.N // 2
    z = np.random.default_rng(2).uniform(-1, 1, (2, B))
    scale = 2.0**30
    pts = O.encode(z, P.N, scale, P.q)
    ct = P.encrypt(sk, pts, P.L, 4)
    got = c.decrypt_decode(sk, ct, P.L, scale, B)
    ref = O.decrypt_decode(P, sk, ct, P.L, B, scale)
    assert np.abs(got - ref).max() < 1e-9
    assert np.abs(got - z).max() < 1e-6


def test_encrypt_segment_layout():
    cfg = workloads.with_batch(workloads.get_config("cnn3_small"), 16)
    c = bcn.Context.from_config(cfg, device=-1)
    P = O.Params.from_config(cfg)
    sk, _ = P.keygen(3)
    imgs = workloads.images(cfg)
    cts = c.encrypt_segment(sk, imgs, cfg["segment"], 2.0**25, 4)
    assert cts.shape == (144, 2, 3, 4096)
    dec = c.decrypt_decode(sk, cts, 3, 2.0**25, 16)
    assert np.abs(dec - O.segment_values(cfg, imgs)).max() < 1e-4


def test_quantize_bit_exact():
    for w in workloads.cipher_weights(workloads.get_config("cifar_cnn")):
        a, s = bcn.quantize(w)
        b, s2 = O.quantize(w)
        assert s == s2 and np.array_equal(a, b)


def test_bad_arguments_are_errors():
    with pytest.raises(bcn.BcnError):
        bcn.Context(3, 3, 1, 1, device=-1)
    with pytest.raises(bcn.BcnError):
        bcn.Context(12, 3, 1, 2, device=-1)  # alpha > K
    c = bcn.Context(12, 3, 1, 1, device=-1)
    with pytest.raises(bcn.BcnError):
        c.encode(np.zeros((1, 4096)), 3, 1.0)  # B > N/2
    with pytest.raises(bcn.BcnError):
        c.encode(np.full((1, 8), 1.0), 3, float("inf"))  # not finite
