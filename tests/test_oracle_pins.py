"""Pins of the CPU oracle against facts fixed by mathematics and published
definitions (not against the oracle itself).  CPU only.

Each test names what it pins; a plausible slip in the oracle (a dropped term,
a sign, a transposed index, a wrong root or slot order) fails one of them.
"""
import os

import numpy as np
import pytest
import sympy
import torch
import torch.nn.functional as F

import workloads
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def schoolbook(a, b, q):
    """negacyclic product in Z_q[x]/(x^N+1), Python integers"""
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += ai * int(b[j])
            else:
                out[k - N] -= ai * int(b[j])
    return np.array([x % q for x in out], dtype=np.uint64)


def centred(v, q):
    v = np.asarray(v, dtype=np.int64) % q
    return np.where(v > q // 2, v - q, v)


@pytest.fixture(scope="module")
def small():
    return O.Params(6, 3, 1, 1)  # N = 64


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log_n,L,K", [(4, 3, 1), (12, 3, 1), (13, 7, 1), (14, 11, 2)])
def test_prime_chain(log_n, L, K):
    P = O.Params(log_n, L, K, 1)
    two_n = 2 << log_n
    assert P.q == sorted(P.q, reverse=True) and len(set(P.primes)) == L + K
    for q in P.q:
        assert sympy.isprime(q) and q % two_n == 1 and q < 2**30 and q > 2**29
    for p in P.p:
        assert sympy.isprime(p) and p % two_n == 1 and p < 2**31 and p > 2**30
    # nothing skipped: no prime = 1 (mod 2N) between consecutive chain primes
    for bound, chain in ((2**30, P.q), (2**31, P.p)):
        c = (bound - 1) // two_n * two_n + 1
        for q in chain:
            while c > q:
                assert not sympy.isprime(c)
                c -= two_n
            c -= two_n


@pytest.mark.parametrize("log_n", [4, 12, 14])
def test_psi_is_primitive_2n_root(log_n):
    P = O.Params(log_n, 2, 1, 1)
    N = P.N
    for t, q in enumerate(P.primes):
        psi = P.psi(t)
        assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1


# --------------------------------------------------------------------------
# NTT
# --------------------------------------------------------------------------
def test_ntt_monomial_closed_form():
    """NTT(x^m)_k = psi^{(2k+1) m}: evaluation at the odd powers of psi."""
    P = O.Params(5, 2, 1, 1)
    N = P.N
    for t, q in enumerate(P.primes):
        psi = P.psi(t)
        for m in (0, 1, 7, N - 1):
            a = np.zeros(N, dtype=np.uint32)
            a[m] = 1
            A = P.ntt_fwd(t, a)
            want = [pow(psi, (2 * k + 1) * m, q) for k in range(N)]
            assert A.tolist() == want


@pytest.mark.parametrize("log_n", [4, 6, 8])
def test_poly_mul_matches_schoolbook(log_n):
    P = O.Params(log_n, 3, 2, 1)
    rng = np.random.default_rng(log_n)
    for t, q in enumerate(P.primes):
        a = rng.integers(0, q, P.N, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, q, P.N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(P.poly_mul(t, a, b).astype(np.uint64), schoolbook(a, b, q))
    # edge values 0, 1, q-1
    q = P.primes[0]
    a = np.array([0, 1, q - 1] * (P.N // 3) + [q - 1] * (P.N % 3), dtype=np.uint32)
    b = np.full(P.N, q - 1, dtype=np.uint32)
    assert np.array_equal(P.poly_mul(0, a, b).astype(np.uint64), schoolbook(a, b, q))


@pytest.mark.parametrize("log_n", [12, 14])
def test_ntt_roundtrip(log_n):
    P = O.Params(log_n, 2, 1, 1)
    rng = np.random.default_rng(1)
    for t, q in enumerate(P.primes):
        a = rng.integers(0, q, P.N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(P.ntt_inv(t, P.ntt_fwd(t, a)), a)


# --------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    blocks, cur = {}, None
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("state"):
            cur = int(line.split()[1])
            blocks[cur] = []
        else:
            blocks[cur].append(int(line))
    for state, outs in blocks.items():
        assert [O.splitmix_raw(state, k) for k in range(len(outs))] == outs
    # a stream starts at mix64(seed + GAMMA*((tag<<40)+idx+1)); mix64(y) is the first raw output from y - GAMMA
    G, M = 0x9E3779B97F4A7C15, (1 << 64) - 1
    for seed, tag, idx in ((3, 1, 0), (4, 4, 5 * 256 + 2)):
        start = O.splitmix_raw((seed + G * ((tag << 40) + idx + 1) - G) & M, 0)
        assert [O.rng_output(seed, tag, idx, k) for k in range(3)] == [O.splitmix_raw(start, k) for k in range(3)]


def test_keygen_secret_and_key_errors(small):
    """evk_j = (-a s + e_j + P g_j s^2, a): removing a*s and P*g_j*s^2 leaves
    the same small error e_j (|e| <= 21, centred binomial) on every prime."""
    P = small
    sk, evk = P.keygen(3)
    assert set(np.unique(sk).tolist()) <= {-1, 0, 1}
    Pprod = int(np.prod([int(p) for p in P.p], dtype=object))
    for j in range(P.dnum(P.L)):
        errs = []
        for t, q in enumerate(P.primes):
            s = (sk.astype(np.int64) % q).astype(np.uint32)
            b, a = evk[j, 0, t], evk[j, 1, t]
            v = (b.astype(np.uint64) + schoolbook(a, s, q)) % q
            if t < P.L and j * P.alpha <= t < (j + 1) * P.alpha:
                s2 = schoolbook(s, s, q)
                v = (v + q - (Pprod % q) * s2 % q) % q
            errs.append(centred(v, q))
        for e in errs:
            assert np.array_equal(e, errs[0])
        assert np.abs(errs[0]).max() <= 21 and np.abs(errs[0]).max() > 0


def test_encrypt_decrypt_error_is_small(small):
    P = small
    sk, _ = P.keygen(3)
    rng = np.random.default_rng(0)
    m = rng.integers(-(2**40), 2**40, size=(4, P.N))
    ct = P.encrypt(sk, O.to_residues(m, P.q), P.L, 4)
    d = O.crt_centered(P.decrypt(sk, ct, P.L), P.q)
    e = (d - m).astype(np.int64)
    assert np.abs(e).max() <= 21
    assert abs(e.mean()) < 0.5 and 6 < e.var() < 15  # centred binomial eta=21: variance 10.5
    # different ciphertexts use different randomness
    assert not np.array_equal(ct[0, 1], ct[1, 1])


# --------------------------------------------------------------------------
# encoding and CRT
# --------------------------------------------------------------------------
def test_round_half_away():
    x = np.array([0.5, -0.5, 1.5, 2.5, -2.5, 0.49999999999999994, 3.0, -0.0])
    assert O.round_half_away(x).tolist() == [1, -1, 2, 3, -3, 0, 3, 0]


def test_slot_exponents_are_the_odd_residues():
    """{5^k, -5^k mod 2N} covers every odd residue mod 2N exactly once."""
    for N in (16, 64, 4096):
        e = O.slot_exponents(N)
        allr = np.concatenate([e, (2 * N - e) % (2 * N)])
        assert sorted(allr.tolist()) == list(range(1, 2 * N, 2))


def test_encode_constant_closed_form():
    """A constant vector c in all N/2 slots encodes to m_0 = round(S c), m_j = 0."""
    N, S = 64, 2.0**20
    m = O.encode_coeffs(np.full((1, N // 2), 0.3), N, S)[0]
    assert m[0] == round(S * 0.3) and np.all(m[1:] == 0)


def test_encode_is_multiplicative():
    """decode(m1 * m2) ~ z1 * z2 slot-wise: the canonical embedding turns the
    negacyclic product into the slot-wise product (App. A, Mult)."""
    N, S = 64, 2.0**24
    rng = np.random.default_rng(2)
    z1, z2 = rng.uniform(-1, 1, (2, N // 2))
    m1 = O.encode_coeffs(z1[None], N, S)[0]
    m2 = O.encode_coeffs(z2[None], N, S)[0]
    q = (1 << 127) - 1  # a large modulus so the product is exact in centred form
    prod = centred_big(schoolbook_big(m1, m2), q)
    z = O.decode(np.array(prod, dtype=np.float64)[None], N, N // 2, S * S)[0]
    assert np.abs(z - z1 * z2).max() < 1e-5


def schoolbook_big(a, b):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            v = int(a[i]) * int(b[j])
            if k < N:
                out[k] += v
            else:
                out[k - N] -= v
    return out


def centred_big(v, q):
    return [((x % q) - q) if (x % q) > q // 2 else (x % q) for x in v]


def test_decode_inverts_encode():
    N, S, B = 4096, 2.0**40, 1000
    z = np.random.default_rng(3).uniform(-2, 2, (3, B))
    m = O.encode_coeffs(z, N, S)
    assert np.abs(O.decode(m, N, B, S) - z).max() < 1e-9


def test_crt_centered():
    P = O.Params(12, 5, 1, 1)
    Q = 1
    for q in P.q:
        Q *= q
    rng = np.random.default_rng(4)
    vals = [int(rng.integers(-(2**62), 2**62)) * int(rng.integers(0, 2**60)) for _ in range(64)]
    vals += [Q // 2, -(Q // 2) + 1, 0, 1, -1]
    res = np.array([[v % q for v in vals] for q in P.q], dtype=np.uint32)[None]
    back = O.crt_centered(res, P.q)[0]
    assert [int(x) for x in back] == vals


# --------------------------------------------------------------------------
# homomorphic operations
# --------------------------------------------------------------------------
def _rand_ct(P, n, level, seed):
    return workloads.random_residues(P.q[:level], (n, 2), P.N, seed)


def test_mac_decrypts_to_weighted_sum(small):
    """Dec(sum_t w c_t + (pt, 0)) = sum_t w Dec(c_t) + pt, exactly (Mult(c,u), Add)."""
    P = small
    sk, _ = P.keygen(3)
    level = 3
    x = _rand_ct(P, 7, level, 5)
    rng = np.random.default_rng(6)
    idx = rng.integers(-1, 7, size=(5, 9)).astype(np.int32)
    w = rng.integers(-127, 128, size=(5, 9)).astype(np.int8)
    pt = workloads.random_residues(P.q[:level], (5,), P.N, 8)
    out = P.mac(level, idx, w, x, pt)
    dx = P.decrypt(sk, x, level).astype(np.int64)
    dout = P.decrypt(sk, out, level).astype(np.int64)
    for o in range(5):
        for i, q in enumerate(P.q[:level]):
            acc = pt[o, i].astype(np.int64)
            for t in range(9):
                if idx[o, t] >= 0:
                    acc = acc + int(w[o, t]) * dx[idx[o, t], i]
            assert np.array_equal(acc % q, dout[o, i])
    # no pt: only the weighted sum; c1 of the output never sees pt
    out2 = P.mac(level, idx, w, x, None)
    assert np.array_equal(out2[:, 1], out[:, 1]) and not np.array_equal(out2[:, 0], out[:, 0])


def test_square_decrypts_to_square(small):
    """(c0 + c1 s)^2 = d0 + d1 s + d2 s^2 exactly (Mult(c1, c2) before relinearisation)."""
    P = small
    sk, _ = P.keygen(3)
    ct = _rand_ct(P, 2, 3, 9)
    d = P.square(3, ct)
    m = P.decrypt(sk, ct, 3)
    m3 = P.decrypt(sk, d, 3)
    for c in range(2):
        for i, q in enumerate(P.q):
            assert np.array_equal(m3[c, i].astype(np.uint64), schoolbook(m[c, i], m[c, i], q))


def _ks_bound(P, level, sk):
    D = max(P.q) ** P.alpha
    Pp = 1
    for p in P.p:
        Pp *= p
    s1 = int(np.abs(sk).sum())
    return P.dnum(level) * P.N * P.alpha * D / 2 * 21 / Pp + (P.K + 1) / 2 * (1 + s1) + 1


@pytest.mark.parametrize("cfg", [(6, 3, 1, 1), (6, 5, 2, 2), (6, 5, 2, 1)])
def test_keyswitch_noise_bound(cfg):
    """k0 + k1 s - x s^2 (mod Q_level) is the key-switching noise, bounded by
    dnum * N * alpha * D/2 * 21 / P + (K+1)/2 * (1 + ||s||_1) + 1 (digit value
    times key error over P, plus the ModDown rounding)."""
    P = O.Params(*cfg)
    sk, evk = P.keygen(3)
    for level in (P.L, P.L - 1):
        x = workloads.random_residues(P.q[:level], (3,), P.N, 10 + level)
        ks = P.keyswitch(level, evk, x)
        ssq = [schoolbook((sk.astype(np.int64) % q), (sk.astype(np.int64) % q), q) for q in P.q[:level]]
        m = P.decrypt(sk, ks, level).astype(np.uint64)
        diff = np.zeros((3, level, P.N), dtype=np.uint32)
        for c in range(3):
            for i, q in enumerate(P.q[:level]):
                xs2 = schoolbook(x[c, i], ssq[i], q)
                diff[c, i] = (m[c, i] + q - xs2) % q
        noise = np.array(O.crt_centered(diff, P.q[:level]), dtype=np.float64)
        bound = _ks_bound(P, level, sk)
        assert np.abs(noise).max() <= bound
        # and it is genuinely small compared with Q_level
        assert np.abs(noise).max() < 2.0**40


def _ks_by_definition(q_data, p_special, alpha, level, x, evk):
    """Hybrid key switching written out with Python integers (App. A Mult(c1, c2)
    relinearisation; the hybrid variant the library implements): for each digit j (primes
    q_{j alpha} .. q_{min((j+1) alpha, level) - 1}) the digit value is the
    integer v_j = sum_i [x_i Dhat_i^-1]_{q_i} Dhat_i with centred residues
    [.]_q in (-q/2, q/2] and Dhat_i the product of the digit's other primes;
    its residue on a target prime t outside the digit is v_j mod t, on the
    digit's own primes x_t itself.  acc_b = sum_j ext_j * evk_j,b (negacyclic
    products by schoolbook, per prime of Q_level u P).  ModDown: the integer
    u_b = sum_m [acc_b,m Phat_m^-1]_{p_m} Phat_m and
    out_b,i = (acc_b,i - u_b) P^-1 mod q_i.  No NTT anywhere."""
    N = x.shape[-1]
    L, K = len(q_data), len(p_special)
    targets = list(q_data[:level]) + list(p_special)
    limb_of = list(range(level)) + [L + m for m in range(K)]  # target -> key limb
    Pbig = 1
    for p in p_special:
        Pbig *= p

    def cen(v, m):
        v %= m
        return v - m if v > (m - 1) // 2 else v

    dnum = -(-level // alpha)
    acc = [[[0] * N for _ in targets] for _ in range(2)]
    for j in range(dnum):
        lo, hi = j * alpha, min((j + 1) * alpha, level)
        D = q_data[lo:hi]
        Dbig = 1
        for d in D:
            Dbig *= d
        v = [0] * N  # integer digit values
        for i, qi in zip(range(lo, hi), D):
            dhat = Dbig // qi
            inv = pow(dhat % qi, -1, qi)
            for k in range(N):
                v[k] += cen(int(x[i, k]) * inv, qi) * dhat
        for ti, t in enumerate(targets):
            ext = [int(x[ti, k]) for k in range(N)] if lo <= ti < hi else [vk % t for vk in v]
            for b in range(2):
                key = [int(evk[j, b, limb_of[ti], k]) for k in range(N)]
                prod = schoolbook(np.array(ext, dtype=object), np.array(key, dtype=object), t)
                acc[b][ti] = [(a + int(pv)) % t for a, pv in zip(acc[b][ti], prod)]
    out = np.zeros((2, level, N), dtype=np.int64)
    for b in range(2):
        u = [0] * N
        for m, pm in enumerate(p_special):
            phat = Pbig // pm
            inv = pow(phat % pm, -1, pm)
            for k in range(N):
                u[k] += cen(acc[b][level + m][k] * inv, pm) * phat
        for i in range(level):
            qi = q_data[i]
            pinv = pow(Pbig % qi, -1, qi)
            out[b, i] = [((acc[b][i][k] - u[k]) * pinv) % qi for k in range(N)]
    return out


@pytest.mark.parametrize("cfg", [(4, 3, 1, 1), (4, 3, 2, 1), (4, 3, 2, 2), (4, 4, 2, 2)])
def test_keyswitch_exact_by_definition(cfg):
    """oc_keyswitch equals hybrid key switching computed from its definition with
    Python big integers and schoolbook products (N = 16), residue for residue,
    at the top level and below it (truncated last digits with alpha = 2), on
    random inputs and a random key: pins the centred ModUp lift, the fast basis
    conversion into every target prime, the key inner product and the centred
    ModDown, which a noise bound alone cannot tell from their uncentred forms."""
    P = O.Params(*cfg)
    rng = np.random.default_rng(sum(cfg))
    evk = np.zeros(P.evk_shape(), dtype=np.uint32)
    for t, m in enumerate(P.primes):
        evk[:, :, t] = rng.integers(0, m, size=evk[:, :, t].shape, dtype=np.uint64).astype(np.uint32)
    for level in sorted({P.L, P.L - 1, 1}, reverse=True):
        x = np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in P.q[:level]]).astype(np.uint32)
        # edge residues in the first coefficients: 0, 1, (q-1)/2, (q+1)/2, q-1
        for i, q in enumerate(P.q[:level]):
            x[i, :5] = [0, 1, (q - 1) // 2, (q + 1) // 2, q - 1]
        got = P.keyswitch(level, evk, x[None])[0]
        want = _ks_by_definition(P.q, P.p, P.alpha, level, x, evk)
        assert np.array_equal(got.astype(np.int64), want), f"level {level}"


@pytest.mark.parametrize("level", [4, 3, 2])
def test_rescale_exact_by_definition(level):
    """oc_rescale equals the rescale of the CRT integer: with X the centred
    integer of a polynomial's limbs mod Q_level and r = [X]_{q_top} centred,
    (X - r) / q_top is an exact integer whose residues are the output limbs
    (at the top level and below it, with edge residues around q_top / 2)."""
    P = O.Params(4, 4, 1, 1)
    rng = np.random.default_rng(40 + level)
    q = P.q[:level]
    ct = np.stack([np.stack([rng.integers(0, m, P.N, dtype=np.uint64) for m in q]) for _ in range(2)])
    qt = q[-1]
    ct[:, -1, :4] = [(qt - 1) // 2, (qt + 1) // 2, 0, qt - 1]
    ct = ct.astype(np.uint32)
    got = P.rescale(level, ct[None])[0]
    Q = 1
    for m in q:
        Q *= m
    for b in range(2):
        X = O.crt_centered(ct[b][None], q)[0]
        for k in range(P.N):
            xk = int(X[k])
            r = xk % qt
            r = r - qt if r > (qt - 1) // 2 else r
            assert (xk - r) % qt == 0
            y = (xk - r) // qt
            assert [int(got[b, i, k]) for i in range(level - 1)] == [y % m for m in q[:-1]], (b, k)


def test_relin_keeps_the_message(small):
    P = small
    sk, evk = P.keygen(3)
    ct = _rand_ct(P, 2, 3, 11)
    d = P.square(3, ct)
    r = P.relin(3, evk, d)
    a = O.crt_centered(P.decrypt(sk, d, 3), P.q)
    b = O.crt_centered(P.decrypt(sk, r, 3), P.q)
    assert np.abs(np.array(b - a, dtype=np.float64)).max() <= _ks_bound(P, 3, sk)


def test_rescale_divides_by_the_dropped_prime(small):
    """Dec(rescale(c)) = Dec(c)/q_top + eps with |eps| <= (1 + ||s||_1)/2."""
    P = small
    sk, _ = P.keygen(3)
    rng = np.random.default_rng(12)
    m = rng.integers(-(2**55), 2**55, size=(3, P.N))
    ct = P.encrypt(sk, O.to_residues(m, P.q), 3, 13)
    before = O.crt_centered(P.decrypt(sk, ct, 3), P.q)
    r = P.rescale(3, ct)
    after = O.crt_centered(P.decrypt(sk, r, 2), P.q[:2])
    qt = P.q[2]
    err = np.array([[float(a) - float(b) / qt for a, b in zip(ra, rb)] for ra, rb in zip(after, before)])
    assert np.abs(err).max() <= (1 + np.abs(sk).sum()) / 2 + 1e-6


def test_square_relin_rescale_is_the_composition(small):
    P = small
    sk, evk = P.keygen(3)
    ct = _rand_ct(P, 2, 3, 14)
    a = P.square_relin_rescale(3, evk, ct)
    b = P.rescale(3, P.relin(3, evk, P.square(3, ct)))
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# network pieces
# --------------------------------------------------------------------------
def test_quantize():
    w = workloads.cipher_weights(workloads.get_config("cryptonets"))[1]
    wi, s = O.quantize(w)
    assert np.abs(wi).max() == 127 and s == pytest.approx(np.abs(w).max() / 127)
    assert np.abs(wi.astype(np.float64) * s - w).max() <= s / 2 + 1e-12


@pytest.mark.parametrize("name", ["cnn3_small", "cryptonets", "cifar_cnn"])
def test_conv_tables_match_torch_conv2d(name):
    """The gather tables compute exactly F.conv2d / F.linear (a library routine)."""
    cfg = workloads.get_config(name)
    rng = np.random.default_rng(15)
    for layer, wf in zip(cfg["cipher"], workloads.cipher_weights(cfg)):
        wi, s = O.quantize(wf)
        idx, wt = O.layer_table(layer, wi)
        n_in, n_out = workloads.cipher_layer_io(layer)
        x = rng.standard_normal((n_in, 3))
        y = O.fp64_network(dict(cipher=[dict(layer, add=False, square=False)]), x, [], [(idx, wt)], [s])
        wr = torch.from_numpy(wi.astype(np.float64) * s)
        if layer["type"] == "conv":
            xt = torch.from_numpy(x.T.reshape(3, layer["cin"], layer["h"], layer["w"]))
            ref = F.conv2d(xt, wr, stride=layer["stride"], padding=layer["pad"]).reshape(3, -1).numpy().T
        else:
            ref = F.linear(torch.from_numpy(x.T), wr).numpy().T
        assert y.shape == (n_out, 3)
        assert np.abs(y - ref).max() < 1e-12


@pytest.mark.parametrize("name", ["cnn3_small", "cryptonets", "cifar_cnn", "cryptonets_fi"])
def test_plain_branch_matches_torch(name):
    cfg = workloads.with_batch(workloads.get_config(name), 5)
    imgs, noise, pw = workloads.images(cfg), workloads.laplace_noise(cfg), workloads.plain_weights(cfg)
    feats = O.plain_branch(cfg, imgs, noise, pw)
    y0, x0, h, w = cfg["segment"]
    x = torch.from_numpy(imgs.astype(np.float64) / 255.0 + noise.astype(np.float64)).permute(0, 3, 1, 2).clone()
    x[:, :, y0:y0 + h, x0:x0 + w] = 0
    ref = []
    for st, wgt in zip(cfg["plain"], pw):
        if st["op"] == "conv":
            x = F.conv2d(x, torch.from_numpy(wgt.astype(np.float64)), stride=st["stride"], padding=st["pad"])
            x = F.relu(x) if st["relu"] else x
        elif st["op"] == "avgpool2":
            x = F.avg_pool2d(x, 2)
        elif st["op"] == "tap_crop_crot":
            H = x.shape[2]
            o = (H - st["hc"]) // 2
            y = x[:, :, o:o + st["hc"], o:o + st["wc"]]
            z = F.conv2d(y, torch.from_numpy(wgt.astype(np.float64))[:, :, None, None])  # 1x1 conv = CRot
            ref.append(z.permute(1, 2, 3, 0).reshape(-1, 5).numpy())
        elif st["op"] == "tap_fc":
            wm, b = wgt if isinstance(wgt, tuple) else (wgt, None)
            bt = None if b is None else torch.from_numpy(b.astype(np.float64))
            ref.append(F.linear(x.reshape(5, -1), torch.from_numpy(wm.astype(np.float64)), bt).numpy().T)
        else:  # tap_integrate: a Linear, the square activation, a Linear
            w1, b1, w2, b2 = (torch.from_numpy(a.astype(np.float64)) for a in wgt)
            ref.append(F.linear(F.linear(x.reshape(5, -1), w1, b1).pow(2), w2, b2).numpy().T)
    assert len(feats) == len(ref)
    for a, b in zip(feats, ref):
        assert np.abs(a - b).max() < 1e-12


def test_feature_integration_is_the_two_layer_head():
    """Sec. 3.3: with the ciphertext branch's output x_c and the plaintext
    branch's output x_p, the integration head computes
        x_c1 = sigma(W_c1 x_c + W_p1 x_p + b_1),  x_p1 = sigma(W'_p1 x_p + b'_1),
        x_out = W_c2 x_c1 + W_p2 x_p1 + b_2       (sigma: the square activation;
    the logits are left without a final activation).  The feature-integration
    config expresses it as two ciphertext dense layers fed by two plaintext
    taps; its fp64 network must equal the head written out with torch layers
    on the branch outputs built from the images (conv2d / avg_pool2d)."""
    cfg = workloads.with_batch(workloads.get_config("cryptonets_fi"), 6)
    imgs, noise, pw = workloads.images(cfg), workloads.laplace_noise(cfg), workloads.plain_weights(cfg)
    feats = O.plain_branch(cfg, imgs, noise, pw)
    wf = workloads.cipher_weights(cfg)
    q = [O.quantize(w) for w in wf]
    tables = [O.layer_table(l, a) for l, (a, _) in zip(cfg["cipher"], q)]
    seg = O.segment_values(cfg, imgs)
    got = O.fp64_network(cfg, seg, feats, tables, [s for _, s in q])
    t = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float64))  # noqa: E731
    # plaintext branch output x_p: perturbed image, segment zeroed, conv3x3, 2x2 average pool
    y0, x0, h, w = cfg["segment"]
    xp = t(imgs.astype(np.float64) / 255.0 + noise.astype(np.float64)).permute(0, 3, 1, 2).clone()
    xp[:, :, y0:y0 + h, x0:x0 + w] = 0
    xp = F.avg_pool2d(F.conv2d(xp, t(pw[0]), padding=1), 2)
    # ciphertext branch output x_c: conv5x5/2 on the segment, plus the crop/CRot feature, squared
    wc = [t(a.astype(np.float64) * s) for a, s in q]
    seg_img = t(seg.T.reshape(6, 1, 16, 16))
    z = F.conv2d(xp[:, :, 4:10, 4:10], t(pw[2])[:, :, None, None])  # centre crop 14 -> 6, CRot
    xc = (F.conv2d(seg_img, wc[0], stride=2) + z).pow(2).reshape(6, -1)
    W_p1, b_1 = pw[3]
    Wq1, bq1, W_p2, b_2 = pw[4]
    xp_flat = xp.reshape(6, -1)
    xc1 = (F.linear(xc, wc[1]) + F.linear(xp_flat, t(W_p1), t(b_1))).pow(2)
    xp1 = F.linear(xp_flat, t(Wq1), t(bq1)).pow(2)
    x_out = F.linear(xc1, wc[2]) + F.linear(xp1, t(W_p2), t(b_2))
    assert np.abs(got - x_out.numpy().T).max() < 1e-9 * max(1.0, float(x_out.abs().max()))


def test_encode_beyond_int64_roundtrips():
    """Scales past 2^63 (the feature added after the last MAC of the
    integration head sits near 2^90): the coefficients become Python ints, the
    residues reduce them exactly, and CRT + decode return the values."""
    P = O.Params(10, 4, 1, 1)
    z = np.random.default_rng(31).uniform(-1, 1, (2, 100))
    scale = 2.0**90
    m = O.encode_coeffs(z, P.N, scale)
    assert m.dtype == object and max(abs(int(v)) for v in m.flat) > 2**63
    res = O.to_residues(m, P.q)
    back = O.crt_centered(res, P.q)
    assert all(int(a) == int(b) for a, b in zip(back.flat, m.flat))
    assert np.abs(O.decode(back, P.N, 100, scale) - z).max() < 1e-9


def test_level_and_scale_schedule():
    cfg = workloads.get_config("cryptonets")
    lv, out = workloads.level_schedule(cfg)
    assert lv == [7, 6, 5] and out == 5
    q = O.Params.from_config(cfg).q
    adds, S = O.scale_schedule(cfg, q, [0.5, 0.25, 0.125])
    S0 = 2.0**30
    a1 = S0 / 0.5
    a2 = (a1 * a1 / q[6]) / 0.25
    assert adds == [a1, a2] and S == (a2 * a2 / q[5]) / 0.125


# --------------------------------------------------------------------------
# whole network
# --------------------------------------------------------------------------
def argmax_agrees(dec, ref, margin=2e-3):
    top2 = np.sort(ref, axis=0)[-2:]
    clear = (top2[1] - top2[0]) > margin
    return np.all(np.argmax(dec, 0)[clear] == np.argmax(ref, 0)[clear]), int((~clear).sum())


def test_whole_network_small_config():
    """decrypt(eval(encrypt(x))) within 1e-3 of the fp64 network, same argmax."""
    prob = O.Problem(workloads.get_config("cnn3_small"))
    out = prob.evaluate()
    assert out.shape == (10, 2, 2, 4096)
    dec = prob.decode_output(out)
    ref = prob.fp64_logits()
    assert np.abs(dec - ref).max() < 1e-3
    ok, ties = argmax_agrees(dec, ref)
    assert ok and ties < 50


def test_whole_network_catches_a_dropped_feature():
    """Planted mistake: evaluating without the unidirectional add moves the
    logits.  (With this shallow plaintext branch the centre crop of the small
    config lies inside the zero-filled segment, so its own features are zero;
    nonzero features are planted here.)"""
    prob = O.Problem(workloads.with_batch(workloads.get_config("cnn3_small"), 64))
    feats = [np.random.default_rng(20).normal(0, 0.3, f.shape) for f in prob.feats]
    P = prob.params
    pts = [O.encode(f, P.N, s, P.q[:lv]) for f, s, lv in zip(feats, prob.add_scales, prob.levels)]
    ref = O.fp64_network(prob.cfg, prob.seg, feats, prob.tables, prob.s_w)
    good = prob.decode_output(O.evaluate(P, prob.cfg, prob.tables, prob.evk, prob.cts, pts))
    assert np.abs(good - ref).max() < 1e-3
    zero = [np.zeros_like(p) for p in pts]
    bad = prob.decode_output(O.evaluate(P, prob.cfg, prob.tables, prob.evk, prob.cts, zero))
    assert np.abs(bad - ref).max() > 1e-2


# --------------------------------------------------------------------------
# rotations (App. A Rot(c, k); App. D builds conv and dense layers from them)
# --------------------------------------------------------------------------
def automorph_by_definition(a, g, q):
    """a(X^g) mod (X^N + 1, q) by expanding every monomial (brute force)."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        e = i * g
        sign = -1 if (e // N) % 2 else 1  # X^N = -1
        out[e % N] += sign * int(a[i])
    return np.array([v % q for v in out], dtype=np.uint32)


def test_automorphism_is_the_substitution_and_a_ring_map(small):
    P = small
    rng = np.random.default_rng(40)
    q = P.q[0]
    for steps in (1, 3, 17):
        g = P.galois_elt(steps)
        a = rng.integers(0, q, P.N).astype(np.uint32)
        b = rng.integers(0, q, P.N).astype(np.uint32)
        ga = P.automorphism(1, g, a[None, None, :])[0, 0]
        assert np.array_equal(ga, automorph_by_definition(a, g, q))
        gb = P.automorphism(1, g, b[None, None, :])[0, 0]
        ab = np.array(schoolbook(a, b, q), dtype=np.uint32)
        gab = P.automorphism(1, g, ab[None, None, :])[0, 0]
        assert np.array_equal(gab, np.array(schoolbook(ga, gb, q), dtype=np.uint32))
    # sigma_g o sigma_h = sigma_{gh mod 2N}
    a = rng.integers(0, q, P.N).astype(np.uint32)[None, None, :]
    g, h = P.galois_elt(3), P.galois_elt(5)
    assert np.array_equal(P.automorphism(1, g, P.automorphism(1, h, a)),
                          P.automorphism(1, g * h % (2 * P.N), a))


def test_automorphism_rotates_the_slots():
    """With slot k at zeta^{5^k}, sigma_{5^r} moves slot k + r to slot k
    (cyclically over the N/2 slots): checked through encode and decode alone."""
    P = O.Params(10, 3, 1, 1)
    z = np.random.default_rng(41).uniform(-1, 1, (2, P.N // 2))
    S = 2.0**40
    m = O.encode_coeffs(z, P.N, S)
    res = O.to_residues(m, P.q)
    for steps in (1, 7, P.N // 2 - 1):
        rot = P.automorphism(P.L, P.galois_elt(steps), res)
        back = O.decode(O.crt_centered(rot, P.q), P.N, P.N // 2, S)
        assert np.abs(back - np.roll(z, -steps, axis=1)).max() < 1e-9


def test_galois_key_errors(small):
    """gk_j = (-a s + e_j + P g_j sigma_g(s), a): removing a*s and
    P*g_j*sigma_g(s) leaves the same small error on every prime."""
    P = small
    sk, _ = P.keygen(3)
    steps = 5
    g = P.galois_elt(steps)
    gk = P.galois_keygen(sk, steps, 8)
    Pprod = int(np.prod([int(p) for p in P.p], dtype=object))
    for j in range(P.dnum(P.L)):
        errs = []
        for t, q in enumerate(P.primes):
            s = (sk.astype(np.int64) % q).astype(np.uint32)
            b, a = gk[j, 0, t], gk[j, 1, t]
            v = (b.astype(np.uint64) + schoolbook(a, s, q)) % q
            if t < P.L and j * P.alpha <= t < (j + 1) * P.alpha:
                sg = automorph_by_definition(s, g, q)
                v = (v + q - (Pprod % q) * sg.astype(np.uint64) % q) % q
            errs.append(centred(v, q))
        for e in errs:
            assert np.array_equal(e, errs[0])
        assert np.abs(errs[0]).max() <= 21 and np.abs(errs[0]).max() > 0


@pytest.mark.parametrize("cfg", [(10, 3, 1, 1), (10, 5, 2, 2)])
def test_rotation_of_an_encryption_decrypts_to_the_rotated_slots(cfg):
    P = O.Params(*cfg)
    sk, _ = P.keygen(3)
    z = np.random.default_rng(42).uniform(-1, 1, (2, P.N // 2))
    S = 2.0**30
    ct = P.encrypt(sk, O.encode(z, P.N, S, P.q), P.L, 4)
    for steps in (1, 33):
        gk = P.galois_keygen(sk, steps, 7)
        for level in (P.L, P.L - 1):
            c = ct[:, :, :level]
            r = P.rotate(level, gk, steps, c)
            dec = O.decode(O.crt_centered(P.decrypt(sk, r, level), P.q[:level]), P.N, P.N // 2, S)
            # noise: the key switch (well below 2^20 here) over the scale
            assert np.abs(dec - np.roll(z, -steps, axis=1)).max() < 2.0**20 / S


def test_bhw_conv_by_rotations_is_the_convolution():
    """App. D: with n images' h x w segments of a channel in one ciphertext, the
    sum of rotated copies weighted by the kernel computes the convolution in the
    valid slots; a 0/1 mask encoded at the top prime's scale, multiplied in and
    rescaled away, zeroes the other slots.  Against torch conv2d."""
    P = O.Params(10, 4, 1, 1)
    n, cin, cout, h, w, k = 4, 2, 3, 10, 10, 3
    rng = np.random.default_rng(50)
    x = rng.uniform(-1, 1, (n, cin, h, w))
    wi = rng.integers(-127, 128, (cout, cin, k, k)).astype(np.int8)
    sk, _ = P.keygen(3)
    S = 2.0**30
    cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), P.L, 4)
    steps = {i * w + j for i in range(k) for j in range(k)} - {0}
    gks = {r: P.galois_keygen(sk, r, 60 + r) for r in steps}
    out = O.conv_bhw(P, P.L, gks, wi, cts, w)
    ref = F.conv2d(torch.from_numpy(x), torch.from_numpy(wi.astype(np.float64))).numpy()  # valid, stride 1
    dec = O.decode(O.crt_centered(P.decrypt(sk, out, P.L), P.q), P.N, P.N // 2, S)
    got = O.unpack_bhw(dec, n, h, w)[:, :, :h - k + 1, :w - k + 1]
    assert np.abs(got - ref).max() < 1e-3
    # mask the invalid slots: multiply by the 0/1 mask at scale q_top, rescale
    m = np.zeros((n, 1, h, w))
    m[:, :, :h - k + 1, :w - k + 1] = 1
    mask = O.encode(O.pack_bhw(m, P.N), P.N, float(P.q[P.L - 1]), P.q)[0]
    masked = P.rescale(P.L, P.mul_plain(P.L, out, mask))
    dm = O.unpack_bhw(O.decode(O.crt_centered(P.decrypt(sk, masked, P.L - 1), P.q[:P.L - 1]), P.N, P.N // 2, S),
                      n, h, w)
    assert np.abs(dm[:, :, :h - k + 1, :w - k + 1] - ref).max() < 1e-3
    dm[:, :, :h - k + 1, :w - k + 1] = 0
    assert np.abs(dm).max() < 1e-3


@pytest.mark.parametrize("K", [1, 2])
def test_ntt_domain_moddown_rescale_identity(K):
    """ModDown by P followed by the rescale by the top prime, written in the NTT
    domain the way the evaluator computes it -- the top limb
    c_top = INTT(A_top P^-1 + D_top) - conv_top(a_P) P^-1 in coefficient form,
    then out_i = (A_i P^-1 + D_i - NTT(conv_i(a_P) P^-1 + [c_top])) q_top^-1 --
    equals the coefficient-form definition (centred fast basis conversion of the
    P limbs, c_i = (a_i - conv_i) P^-1 + d_i, out_i = (c_i - [c_top]) q_top^-1)
    residue for residue, on random limbs."""
    P = O.Params(5, 4, K, 1)  # N = 32
    N, n = P.N, 4
    rng = np.random.default_rng(17 + K)
    q, p = P.q[:n], P.p
    a = [rng.integers(0, m, N, dtype=np.int64) for m in q + p]  # extended-basis limbs, coefficient form
    d = [rng.integers(0, m, N, dtype=np.int64) for m in q]
    Pprod = int(np.prod([int(v) for v in p], dtype=object))

    def conv(i_mod):  # centred fast basis conversion of the P limbs into modulus i_mod
        out = np.zeros(N, dtype=object)
        cnt = np.zeros(N, dtype=np.int64)
        for m, pm in enumerate(p):
            phat = Pprod // pm
            r = (a[n + m].astype(object) * pow(phat % pm, -1, pm)) % pm
            cnt += (r > (pm - 1) // 2).astype(np.int64)
            out = out + r * (phat % i_mod)
        return np.array([(int(v) - int(c) * Pprod) % i_mod for v, c in zip(out, cnt)], dtype=np.int64)

    top = n - 1
    qt = q[top]
    # coefficient-form definition
    c = [((a[i] - conv(q[i])) % q[i] * pow(Pprod % q[i], -1, q[i]) + d[i]) % q[i] for i in range(n)]
    lift = np.where(c[top] > (qt - 1) // 2, c[top] - qt, c[top])
    ref = [((c[i] - lift) % q[i] * pow(qt, -1, q[i])) % q[i] for i in range(top)]
    # NTT-domain form (the oracle's transform; any NTT of the same ring works)
    A = [P.ntt_fwd(i, a[i].astype(np.uint32)).astype(np.int64) for i in range(n)]
    D = [P.ntt_fwd(i, d[i].astype(np.uint32)).astype(np.int64) for i in range(n)]
    pinv = [pow(Pprod % m, -1, m) for m in q]
    ctop = (P.ntt_inv(top, ((A[top] * pinv[top] + D[top]) % qt).astype(np.uint32)).astype(np.int64)
            - conv(qt) * pinv[top]) % qt
    lt = np.where(ctop > (qt - 1) // 2, ctop - qt, ctop)
    for i in range(top):
        f = P.ntt_fwd(i, ((conv(q[i]) * pinv[i] + lt) % q[i]).astype(np.uint32)).astype(np.int64)
        o = ((A[i] * pinv[i] + D[i] - f) % q[i] * pow(qt, -1, q[i])) % q[i]
        got = P.ntt_inv(i, o.astype(np.uint32)).astype(np.int64)
        assert np.array_equal(got, ref[i])


# --------------------------------------------------------------------------
# App. D: fully connected layer by the diagonal method, strided packed convolution
# --------------------------------------------------------------------------
def test_fc_diagonals_reproduce_the_matrix_product():
    """Slot arithmetic alone (no encryption): sum_r u_r * (x rotated left by r)
    equals W x in every image's block, exactly (integers), for tall, wide and
    square W and blocks wider than both sides."""
    N = 256
    rng = np.random.default_rng(80)
    for n2, n1, n_img, block in ((10, 20, 4, 32), (30, 7, 3, 40), (16, 16, 8, 16)):
        W = rng.integers(-127, 128, (n2, n1))
        x = np.zeros(N // 2, dtype=np.int64)
        xs = rng.integers(-1000, 1000, (n_img, n1))
        for b in range(n_img):
            x[b * block:b * block + n1] = xs[b]
        diags = O.fc_diagonals(W, n_img, block, N)
        assert set(diags) <= set(range(-(n2 - 1), n1))
        y = sum(u * np.roll(x, -r) for r, u in diags.items())
        for b in range(n_img):
            assert np.array_equal(y[b * block:b * block + n2], W @ xs[b])
            assert not np.any(y[b * block + n2:(b + 1) * block])


def test_fc_diag_decrypts_to_the_matrix_product():
    P = O.Params(10, 4, 1, 1)
    n2, n1, n_img, block = 10, 20, 4, 32
    rng = np.random.default_rng(81)
    W = rng.integers(-127, 128, (n2, n1))
    xs = rng.uniform(-1, 1, (n_img, n1))
    z = np.zeros((1, P.N // 2))
    for b in range(n_img):
        z[0, b * block:b * block + n1] = xs[b]
    sk, _ = P.keygen(3)
    S = 2.0**30
    ct = P.encrypt(sk, O.encode(z, P.N, S, P.q), P.L, 4)[0]
    half = P.N // 2
    gks = {r % half: P.galois_keygen(sk, r % half, 90 + r % half)
           for r in O.fc_diagonals(W, n_img, block, P.N) if r % half}
    out = O.fc_diag(P, P.L, gks, W, ct, n_img, block)
    dec = O.decode(O.crt_centered(P.decrypt(sk, out[None], P.L - 1), P.q[:P.L - 1]), P.N, half, S)[0]
    for b in range(n_img):
        assert np.abs(dec[b * block:b * block + n2] - W @ xs[b]).max() < 1e-3
        assert np.abs(dec[b * block + n2:(b + 1) * block]).max() < 1e-3


def test_strided_conv_then_gapped_conv_is_the_convolution_chain():
    """A stride-2 3x3 convolution of BHW-packed maps (rotations, integer
    weights, a mask keeping the strided outputs) leaves its outputs at gap 2;
    a 2x2 convolution on that gap-2 map (rotations scaled by the gap) puts its
    outputs in the same gap-2 slots.  Against torch conv2d: the stride-2 conv,
    then a stride-1 conv of its output (absolute error 1e-3 on the first, whose
    values are O(10^2); relative 1e-5 on the second, O(10^4) after two layers of
    weights up to 127)."""
    P = O.Params(10, 5, 1, 1)
    n, cin, c1, c2, h, w = 3, 2, 2, 2, 12, 12
    rng = np.random.default_rng(82)
    x = rng.uniform(-1, 1, (n, cin, h, w))
    w1 = rng.integers(-127, 128, (c1, cin, 3, 3)).astype(np.int8)
    w2 = rng.integers(-127, 128, (c2, c1, 2, 2)).astype(np.int8)
    sk, _ = P.keygen(3)
    S = 2.0**30
    cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), P.L, 4)
    steps1 = {(i * w + j) for i in range(3) for j in range(3)} - {0}
    steps2 = {2 * (i * w + j) for i in range(2) for j in range(2)} - {0}
    gks = {r: P.galois_keygen(sk, r, 100 + r) for r in steps1 | steps2}
    y1 = O.conv_bhw(P, P.L, gks, w1, cts, w)                       # stride 1 everywhere
    m1 = O.mask_bhw(n, h, w, 3, 2, 1, P.N)                         # keep (2y', 2x')
    mpt = O.encode(m1[None], P.N, float(P.q[P.L - 1]), P.q)[0]
    y1 = P.rescale(P.L, P.mul_plain(P.L, y1, mpt))
    lv = P.L - 1
    y2 = O.conv_bhw(P, lv, gks, w2, y1, w, gap=2)
    ref1 = F.conv2d(torch.from_numpy(x), torch.from_numpy(w1.astype(np.float64)), stride=2).numpy()
    ref2 = F.conv2d(torch.from_numpy(ref1), torch.from_numpy(w2.astype(np.float64))).numpy()
    S1 = S  # the mask at scale q_top and its rescale keep the scale
    d1 = O.unpack_bhw(O.decode(O.crt_centered(P.decrypt(sk, y1, lv), P.q[:lv]), P.N, P.N // 2, S1), n, h, w)
    d2 = O.unpack_bhw(O.decode(O.crt_centered(P.decrypt(sk, y2, lv), P.q[:lv]), P.N, P.N // 2, S1), n, h, w)
    assert np.abs(d1[:, :, 0:10:2, 0:10:2] - ref1).max() < 1e-3           # 5 x 5 strided outputs at gap 2
    keep = np.zeros((h, w), bool)
    keep[0:10:2, 0:10:2] = True
    assert np.abs(d1[:, :, ~keep]).max() < 1e-3                            # the mask zeroed the rest
    assert np.abs(d2[:, :, 0:8:2, 0:8:2] - ref2).max() < 1e-5 * np.abs(ref2).max()  # its 4 x 4 outputs


def test_fc_diagonals_at_reproduce_the_gathered_product():
    """The diagonal method with inputs at arbitrary slots (App. D, after a
    strided packed convolution): sum_r u_r * (x rotated by r) on plain slot
    vectors holds sum_p W[j][p] x[s_in[p]] in slot o_out[j] of every image
    block and zero in every other slot, whatever the other slots hold."""
    rng = np.random.default_rng(83)
    N, n_img, block = 128, 3, 20
    s_in, o_out = [0, 2, 4, 10, 12, 14, 19], [0, 1, 2, 5]
    W = rng.integers(-9, 10, (len(o_out), len(s_in))).astype(float)
    x = rng.integers(-50, 51, N // 2).astype(float)  # every slot nonzero, the unused ones too
    diags = O.fc_diagonals_at(W, n_img, block, s_in, o_out, N)
    y = sum(u * np.roll(x, -r) for r, u in diags.items())  # rotation by r: slot k takes slot k + r
    want = np.zeros(N // 2)
    for b in range(n_img):
        for j, o in enumerate(o_out):
            want[b * block + o] = sum(W[j][p] * x[b * block + s] for p, s in enumerate(s_in))
    assert np.array_equal(y, want)


def _bhw_net(x, w1, f1, W2, f2, W3, stride):
    """The branch in plain fp64 per image: conv, +f1, square, flatten, dense,
    +f2, square, dense."""
    y = F.conv2d(torch.from_numpy(x), torch.from_numpy(w1.astype(np.float64)), stride=stride).numpy() + f1
    y = (y * y).reshape(x.shape[0], -1)
    z = y @ W2.T + f2
    return (z * z) @ W3.T


def test_bhw_branch_decrypts_to_the_network():
    """A conv-square-dense-square-dense branch evaluated in BHW packing (two
    images' 16 x 16 segments per ciphertext, a 5 x 5 stride-2 convolution, the
    dense layers by diagonals over the strided outputs) decrypts to the same
    network in plain fp64 within 1e-5 of its largest output; the scales follow
    the rescales (q_{L-1} after the first square, q_{L-3} after the second)."""
    P = O.Params(10, 7, 1, 1)
    n, h, w, k, s, c1, n2, n3 = 2, 16, 16, 5, 2, 2, 12, 4
    ho = (h - k) // s + 1
    layers = [dict(type="conv", cin=1, h=h, w=w, cout=c1, k=k, stride=s, pad=0, add=True, square=True),
              dict(type="dense", n_in=c1 * ho * ho, n_out=n2, add=True, square=True),
              dict(type="dense", n_in=n2, n_out=n3, add=False, square=False)]
    rng = np.random.default_rng(84)
    x = rng.uniform(0, 1, (n, 1, h, w))
    w1 = rng.integers(-3, 4, (c1, 1, k, k))
    W2 = rng.integers(-3, 4, (n2, c1 * ho * ho))
    W3 = rng.integers(-3, 4, (n3, n2))
    f1 = rng.uniform(-1, 1, (n, c1, ho, ho))
    f2 = rng.uniform(-1, 1, (n, n2))
    sk, evk = P.keygen(3)
    L, half, S = P.L, P.N // 2, 2.0**30
    s1 = S * S / P.q[L - 1]
    s2 = s1 * s1 / P.q[L - 3]
    cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), L, 4)
    v1 = np.zeros((c1, half))
    for b in range(n):
        for yy in range(ho):
            for xx in range(ho):
                v1[:, b * h * w + s * (yy * w + xx)] = f1[b, :, yy, xx]
    v2 = np.zeros((1, half))
    for b in range(n):
        v2[0, b * h * w:b * h * w + n2] = f2[b]
    feats = [O.encode(v1, P.N, S, P.q[:L]), O.encode(v2, P.N, s1, P.q[:L - 2])[0]]
    pos = [s * (yy * w + xx) for yy in range(ho) for xx in range(ho)]
    steps = {i * w + j for i in range(k) for j in range(k)}
    steps |= {p - j for p in pos for j in range(n2)} | {p - j for p in range(n2) for j in range(n3)}
    gks = {r % half: P.galois_keygen(sk, r % half, 400 + r % half) for r in steps if r % half}
    out = O.bhw_branch(P, evk, gks, layers, [w1, W2, W3], feats, cts, n)
    assert out.shape == (2, L - 4, P.N)
    dec = O.decode(O.crt_centered(P.decrypt(sk, out[None], L - 4), P.q[:L - 4]), P.N, half, s2)[0]
    ref = _bhw_net(x, w1, f1, W2, f2, W3, s)
    got = np.stack([dec[b * h * w:b * h * w + n3] for b in range(n)])
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
