"""CPU oracle for the bi-CryptoNets ciphertext branch -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path
(``paper_2402_01296_gb300``); the only module both sides import is the seeded
input generator ``workloads``.

Layers of the oracle:
  * ``ckks_oracle.c`` (built here with gcc): modular arithmetic, the negacyclic
    NTT, SplitMix64 sampling, keygen, symmetric encryption, decryption to
    residues, and the homomorphic operations of the ciphertext branch.
  * this file (numpy, fp64): CKKS encode/decode through the canonical
    embedding, CRT with Python integers, weight quantisation, conv/dense
    gather tables, the plaintext branch, the fp64 plaintext network, the
    scale schedule and the layer-by-layer evaluation schedule.

Citations are to "Bi-CryptoNets: Leveraging Different-Level Privacy for
Encrypted Inference" (arXiv 2402.01296).
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess
import threading

import numpy as np

import workloads

HERE = pathlib.Path(__file__).resolve().parent
SRC = HERE / "ckks_oracle.c"
LIBDIR = HERE / "_build"
LIB = LIBDIR / "libckks_oracle.so"

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the C part of the oracle (gcc -O2, OpenMP over ciphertexts)."""
    LIBDIR.mkdir(exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(tmp), str(SRC)])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(str(LIB))
            P, I, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
            sig = {
                "oc_create": (P, [I, I, I, I]),
                "oc_destroy": (None, [P]),
                "oc_n": (I, [P]),
                "oc_primes": (None, [P, P]),
                "oc_psi": (U64, [P, I]),
                "oc_dnum": (I, [P, I]),
                "oc_set_threads": (None, [I]),
                "oc_max_threads": (I, []),
                "oc_ntt_fwd": (None, [P, I, P]),
                "oc_ntt_inv": (None, [P, I, P]),
                "oc_poly_mul": (None, [P, I, P, P, P]),
                "oc_rng_first": (U64, [U64, U64, U64, U64]),
                "oc_splitmix_raw": (U64, [U64, U64]),
                "oc_keygen": (I, [P, U64, P, P]),
                "oc_encrypt": (I, [P, P, P, I, I, U64, P]),
                "oc_decrypt": (I, [P, P, P, I, I, I, P]),
                "oc_mac": (I, [P, I, I, I, I, P, P, P, P, P]),
                "oc_square": (I, [P, I, P, I, P]),
                "oc_keyswitch": (I, [P, I, P, P, I, P]),
                "oc_relin": (I, [P, I, P, P, I, P]),
                "oc_rescale": (I, [P, I, P, I, P]),
                "oc_square_relin_rescale": (I, [P, I, P, P, I, P]),
                "oc_automorphism": (I, [P, I, U64, P, I, P]),
                "oc_galois_keygen": (I, [P, P, U64, U64, P]),
                "oc_rotate": (I, [P, I, P, U64, P, I, P]),
                "oc_mul_plain": (I, [P, I, P, I, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def set_threads(n: int) -> None:
    lib().oc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oc_max_threads())


def splitmix_raw(state: int, k: int) -> int:
    """k-th output of plain SplitMix64 started from `state`."""
    return int(lib().oc_splitmix_raw(state, k))


def rng_output(seed: int, tag: int, idx: int, k: int) -> int:
    """k-th SplitMix64 output of stream (seed, tag, idx)."""
    return int(lib().oc_rng_first(seed, tag, idx, k))


# ---------------------------------------------------------------------------
# parameters and homomorphic operations (C)
# ---------------------------------------------------------------------------
class Params:
    """RNS-CKKS parameter set: ring degree N = 2^log_n, `n_data` data primes
    below 2^30 and `n_special` special primes below 2^31 (all = 1 mod 2N),
    `alpha` primes per key-switching digit."""

    def __init__(self, log_n: int, n_data: int, n_special: int, alpha: int):
        self.log_n, self.L, self.K, self.alpha = log_n, n_data, n_special, alpha
        self.N = 1 << log_n
        self._c = lib().oc_create(log_n, n_data, n_special, alpha)
        if not self._c:
            raise ValueError("oracle: bad parameters")
        pr = np.zeros(n_data + n_special, dtype=np.uint64)
        lib().oc_primes(self._c, _p(pr))
        self.primes = [int(v) for v in pr]
        self.q = self.primes[:n_data]
        self.p = self.primes[n_data:]

    @classmethod
    def from_config(cls, cfg: dict) -> "Params":
        return cls(cfg["log_n"], cfg["n_data"], cfg["n_special"], cfg["alpha"])

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            lib().oc_destroy(c)
            self._c = None

    def dnum(self, level: int) -> int:
        return int(lib().oc_dnum(self._c, level))

    def psi(self, t: int) -> int:
        return int(lib().oc_psi(self._c, t))

    # -- NTT -------------------------------------------------------------
    def ntt_fwd(self, t: int, a: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint32).copy()
        lib().oc_ntt_fwd(self._c, t, _p(a))
        return a

    def ntt_inv(self, t: int, a: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint32).copy()
        lib().oc_ntt_inv(self._c, t, _p(a))
        return a

    def poly_mul(self, t: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint32)
        b = np.ascontiguousarray(b, dtype=np.uint32)
        o = np.zeros(self.N, dtype=np.uint32)
        lib().oc_poly_mul(self._c, t, _p(a), _p(b), _p(o))
        return o

    # -- keys, encryption ------------------------------------------------
    def evk_shape(self):
        return (self.dnum(self.L), 2, self.L + self.K, self.N)

    def keygen(self, seed: int):
        sk = np.zeros(self.N, dtype=np.int8)
        evk = np.zeros(self.evk_shape(), dtype=np.uint32)
        rc = lib().oc_keygen(self._c, seed, _p(sk), _p(evk))
        assert rc == 0
        return sk, evk

    def encrypt(self, sk: np.ndarray, pt: np.ndarray, level: int, seed: int) -> np.ndarray:
        pt = np.ascontiguousarray(pt, dtype=np.uint32)
        n_ct = pt.shape[0]
        assert pt.shape == (n_ct, level, self.N)
        ct = np.zeros((n_ct, 2, level, self.N), dtype=np.uint32)
        rc = lib().oc_encrypt(self._c, _p(np.ascontiguousarray(sk)), _p(pt), n_ct, level, seed, _p(ct))
        assert rc == 0
        return ct

    def decrypt(self, sk: np.ndarray, ct: np.ndarray, level: int) -> np.ndarray:
        """Residues of m = sum_p c_p s^p; ct [n][n_poly][level][N] -> [n][level][N]."""
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        n, n_poly = ct.shape[0], ct.shape[1]
        assert ct.shape[2:] == (level, self.N)
        m = np.zeros((n, level, self.N), dtype=np.uint32)
        rc = lib().oc_decrypt(self._c, _p(np.ascontiguousarray(sk)), _p(ct), n, n_poly, level, _p(m))
        assert rc == 0
        return m

    # -- homomorphic operations ------------------------------------------
    def mac(self, level: int, idx: np.ndarray, w: np.ndarray, x: np.ndarray, pt=None) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int8)
        x = np.ascontiguousarray(x, dtype=np.uint32)
        n_out, K = idx.shape
        n_in = x.shape[0]
        assert x.shape[1:] == (2, level, self.N)
        out = np.zeros((n_out, 2, level, self.N), dtype=np.uint32)
        ptp = None
        if pt is not None:
            pt = np.ascontiguousarray(pt, dtype=np.uint32)
            assert pt.shape == (n_out, level, self.N)
            ptp = _p(pt)
        rc = lib().oc_mac(self._c, level, n_in, n_out, K, _p(idx), _p(w), _p(x), ptp, _p(out))
        assert rc == 0
        return out

    def square(self, level: int, ct: np.ndarray) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        d = np.zeros((ct.shape[0], 3, level, self.N), dtype=np.uint32)
        assert lib().oc_square(self._c, level, _p(ct), ct.shape[0], _p(d)) == 0
        return d

    def keyswitch(self, level: int, evk: np.ndarray, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint32)
        out = np.zeros((x.shape[0], 2, level, self.N), dtype=np.uint32)
        assert lib().oc_keyswitch(self._c, level, _p(np.ascontiguousarray(evk)), _p(x), x.shape[0], _p(out)) == 0
        return out

    def relin(self, level: int, evk: np.ndarray, d: np.ndarray) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.uint32)
        out = np.zeros((d.shape[0], 2, level, self.N), dtype=np.uint32)
        assert lib().oc_relin(self._c, level, _p(np.ascontiguousarray(evk)), _p(d), d.shape[0], _p(out)) == 0
        return out

    def rescale(self, level: int, ct: np.ndarray) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        out = np.zeros((ct.shape[0], 2, level - 1, self.N), dtype=np.uint32)
        assert lib().oc_rescale(self._c, level, _p(ct), ct.shape[0], _p(out)) == 0
        return out

    # -- rotations (App. A Rot; App. D) ----------------------------------
    def galois_elt(self, steps: int) -> int:
        """g = 5^steps mod 2N: sigma_g rotates the N/2 slots by `steps`."""
        return pow(5, steps % (self.N // 2), 2 * self.N)

    def automorphism(self, level: int, g: int, a: np.ndarray) -> np.ndarray:
        """a [..][level][N] -> a(X^g), limb i mod q_i."""
        a = np.ascontiguousarray(a, dtype=np.uint32)
        out = np.zeros_like(a)
        n_poly = int(np.prod(a.shape[:-2])) if a.ndim > 2 else 1
        assert lib().oc_automorphism(self._c, level, g, _p(a), n_poly, _p(out)) == 0
        return out

    def galois_keygen(self, sk: np.ndarray, steps: int, seed: int) -> np.ndarray:
        gk = np.zeros(self.evk_shape(), dtype=np.uint32)
        rc = lib().oc_galois_keygen(self._c, _p(np.ascontiguousarray(sk)), self.galois_elt(steps), seed, _p(gk))
        assert rc == 0
        return gk

    def rotate(self, level: int, gk: np.ndarray, steps: int, ct: np.ndarray) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        out = np.zeros_like(ct)
        rc = lib().oc_rotate(self._c, level, _p(np.ascontiguousarray(gk)), self.galois_elt(steps), _p(ct),
                             ct.shape[0], _p(out))
        assert rc == 0
        return out

    def mul_plain(self, level: int, ct: np.ndarray, pt: np.ndarray) -> np.ndarray:
        """(c0 u, c1 u) mod Q_level for an encoded plaintext u [level][N]."""
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        pt = np.ascontiguousarray(pt, dtype=np.uint32)
        assert pt.shape == (level, self.N)
        out = np.zeros_like(ct)
        assert lib().oc_mul_plain(self._c, level, _p(ct), ct.shape[0], _p(pt), _p(out)) == 0
        return out

    def square_relin_rescale(self, level: int, evk: np.ndarray, ct: np.ndarray) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32)
        out = np.zeros((ct.shape[0], 2, level - 1, self.N), dtype=np.uint32)
        rc = lib().oc_square_relin_rescale(self._c, level, _p(np.ascontiguousarray(evk)), _p(ct), ct.shape[0],
                                           _p(out))
        assert rc == 0
        return out


# ---------------------------------------------------------------------------
# encoding (canonical embedding, App. A: N/2 complex slots)
# ---------------------------------------------------------------------------
def round_half_away(x: np.ndarray) -> np.ndarray:
    """Round to nearest, ties away from zero, exactly (no x + 0.5 rounding)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.trunc(x)
    frac = x - t  # exact
    return t + np.where(np.abs(frac) >= 0.5, np.sign(x), 0.0)


def slot_exponents(N: int) -> np.ndarray:
    """e_k = 5^k mod 2N for k < N/2: slot k is the evaluation at zeta^{e_k},
    zeta = exp(i pi / N)."""
    e = np.zeros(N // 2, dtype=np.int64)
    v = 1
    for k in range(N // 2):
        e[k] = v
        v = (v * 5) % (2 * N)
    return e


def _cos_block(N: int, j0: int, j1: int, B: int) -> np.ndarray:
    """cos(pi * ((j * e_k) mod 2N) / N) for j in [j0, j1), k < B."""
    e = slot_exponents(N)[:B]
    j = np.arange(j0, j1, dtype=np.int64)[:, None]
    r = (j * e[None, :]) % (2 * N)
    return np.cos(np.pi * r.astype(np.float64) / N)


def encode_coeffs(values: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Real slot values z [n_vec][B] (B <= N/2, other slots 0) -> integer
    coefficients m [n_vec][N] with
        m_j = round(scale * (2/N) * sum_k z_k cos(pi j e_k / N)),
    the inverse canonical embedding of a real vector, rounded half away from 0.
    int64 when every |m_j| < 2^63; otherwise an object array of Python ints,
    each the exact integer value of the fp64 product (beyond 2^52 an fp64
    number has no fractional part)."""
    values = np.atleast_2d(np.asarray(values, dtype=np.float64))
    n_vec, B = values.shape
    assert B <= N // 2
    out = np.zeros((n_vec, N), dtype=np.float64)
    step = 1024
    for j0 in range(0, N, step):
        j1 = min(N, j0 + step)
        M = _cos_block(N, j0, j1, B)  # [j][k]
        x = scale * (2.0 / N) * (values @ M.T)
        out[:, j0:j1] = round_half_away(x)
    if not np.all(np.isfinite(out)):
        raise OverflowError("encoded coefficient is not finite")
    if np.all(np.abs(out) < 2.0**63):
        return out.astype(np.int64)
    big = np.empty(out.shape, dtype=object)
    big.flat[:] = [int(v) for v in out.flat]
    return big


def to_residues(m: np.ndarray, primes) -> np.ndarray:
    """Integer coefficients [..][N] (int64, or Python ints in an object array)
    -> uint32 residues [..][len(primes)][N]."""
    if m.dtype == object:
        res = [np.mod(m, int(q)).astype(np.uint32) for q in primes]
    else:
        m = np.asarray(m, dtype=np.int64)
        res = [np.mod(m, np.int64(q)).astype(np.uint32) for q in primes]
    return np.stack(res, axis=-2)


def encode(values: np.ndarray, N: int, scale: float, primes) -> np.ndarray:
    return to_residues(encode_coeffs(values, N, scale), primes)


def crt_centered(res: np.ndarray, primes) -> np.ndarray:
    """Residues [..][level][N] -> centred integers (Python ints, object array
    [..][N]) in (-Q/2, Q/2], Q = prod primes: x = sum_i r_i * Qhat_i *
    [Qhat_i^{-1}]_{q_i} mod Q."""
    primes = [int(q) for q in primes]
    Q = 1
    for q in primes:
        Q *= q
    acc = np.zeros(res.shape[:-2] + (res.shape[-1],), dtype=object)
    for i, q in enumerate(primes):
        qhat = Q // q
        c = qhat * pow(qhat % q, -1, q)
        acc = acc + res[..., i, :].astype(np.int64).astype(object) * c
    acc = acc % Q
    return np.where(acc > Q // 2, acc - Q, acc)


def decode(m: np.ndarray, N: int, B: int, scale: float) -> np.ndarray:
    """Centred coefficients m [n][N] (ints or floats) -> real slot values
    [n][B]: z_k = Re sum_j m_j zeta^{j e_k} / scale."""
    m = np.atleast_2d(np.asarray(m).astype(np.float64))
    out = np.zeros((m.shape[0], B))
    step = 1024
    for j0 in range(0, N, step):
        j1 = min(N, j0 + step)
        out += m[:, j0:j1] @ _cos_block(N, j0, j1, B)
    return out / scale


def decrypt_decode(params: Params, sk, ct: np.ndarray, level: int, B: int, scale: float) -> np.ndarray:
    m = params.decrypt(sk, ct, level)
    return decode(crt_centered(m, params.q[:level]), params.N, B, scale)


# ---------------------------------------------------------------------------
# network: quantisation, gather tables, plaintext branch, fp64 network
# ---------------------------------------------------------------------------
def quantize(w: np.ndarray):
    """Per-tensor symmetric int8: s_w = max|w| / 127, w_int = round(w / s_w)
    (ties away from zero), so the ciphertext branch multiplies by integers."""
    w64 = np.asarray(w, dtype=np.float32).astype(np.float64)
    s_w = float(np.max(np.abs(w64))) / 127.0
    if s_w == 0.0:
        return np.zeros(w64.shape, dtype=np.int8), 1.0
    return round_half_away(w64 / s_w).astype(np.int8), s_w


def layer_table(layer: dict, w_int: np.ndarray):
    """Gather table of a cipher layer: out[o] = sum_t wt[o,t] * in[idx[o,t]],
    idx = -1 for zero-padding taps.  Inputs and outputs are flattened in
    (channel, row, column) order."""
    if layer["type"] == "dense":
        n_in, n_out = layer["n_in"], layer["n_out"]
        idx = np.tile(np.arange(n_in, dtype=np.int32), (n_out, 1))
        return idx, np.ascontiguousarray(w_int.reshape(n_out, n_in), dtype=np.int8)
    cin, h, w, cout, k, s, pad = (layer[x] for x in ("cin", "h", "w", "cout", "k", "stride", "pad"))
    ho, wo = workloads.conv_out_hw(h, w, k, s, pad)
    K = cin * k * k
    idx = np.full((cout * ho * wo, K), -1, dtype=np.int32)
    wt = np.zeros((cout * ho * wo, K), dtype=np.int8)
    for co in range(cout):
        for oy in range(ho):
            for ox in range(wo):
                o = (co * ho + oy) * wo + ox
                for ci in range(cin):
                    for ky in range(k):
                        for kx in range(k):
                            t = (ci * k + ky) * k + kx
                            iy, ix = oy * s - pad + ky, ox * s - pad + kx
                            if 0 <= iy < h and 0 <= ix < w:
                                idx[o, t] = (ci * h + iy) * w + ix
                                wt[o, t] = w_int[co, ci, ky, kx]
    return idx, wt


def segment_values(cfg: dict, imgs: np.ndarray) -> np.ndarray:
    """Sensitive segment (Sec. 3) as slot vectors [n_ct][B]: ciphertext
    (c, y, x) holds pixel (y0+y, x0+x, c) / 255 of every image, one image per
    slot (batch packing)."""
    y0, x0, h, w = cfg["segment"]
    seg = imgs[:, y0:y0 + h, x0:x0 + w, :].astype(np.float64) / 255.0  # [B][h][w][C]
    return np.ascontiguousarray(seg.transpose(3, 1, 2, 0).reshape(-1, imgs.shape[0]))


def _conv2d(x: np.ndarray, wgt: np.ndarray, stride: int, pad: int) -> np.ndarray:
    """x [B][C][H][W], wgt [cout][cin][k][k] -> [B][cout][Ho][Wo] (cross-correlation)."""
    B, C, H, W = x.shape
    cout, cin, k, _ = wgt.shape
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    Ho, Wo = (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1
    out = np.zeros((B, cout, Ho, Wo))
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("bchw,oc->bohw", patch, wgt[:, :, ky, kx], optimize=True)
    return out


def perturbed_input(cfg: dict, imgs: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """Plaintext-branch input (Sec. 3.1): pixels / 255 plus the perturbation
    noise on the insensitive segment, the sensitive segment set to zero.
    Returns [B][C][H][W] float64."""
    y0, x0, h, w = cfg["segment"]
    x = imgs.astype(np.float64) / 255.0 + noise.astype(np.float64)
    x[:, y0:y0 + h, x0:x0 + w, :] = 0.0
    return np.ascontiguousarray(x.transpose(0, 3, 1, 2))


def plain_branch(cfg: dict, imgs: np.ndarray, noise: np.ndarray, weights) -> list:
    """fp64 plaintext branch with its unidirectional-connection taps:
    Resize = centre crop (offset floor((h_p - h_c)/2)), then CRot
    z^i = sum_j W^{i,j} y^j (Sec. 3.2); a dense tap is a fully connected map of
    the flattened (c, y, x) trunk output (with an optional bias); an
    integration tap is the plaintext half of the two-layer feature integration
    (Sec. 3.3).  Returns features [n][B] per tap."""
    x = perturbed_input(cfg, imgs, noise)
    feats = []
    for st, wgt in zip(cfg["plain"], weights):
        if st["op"] == "conv":
            x = _conv2d(x, wgt.astype(np.float64), st["stride"], st["pad"])
            if st["relu"]:
                x = np.maximum(x, 0.0)
        elif st["op"] == "avgpool2":
            B, C, H, W = x.shape
            x = x[:, :, :H // 2 * 2, :W // 2 * 2].reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))
        elif st["op"] == "tap_crop_crot":
            B, C, H, W = x.shape
            hc, wc = st["hc"], st["wc"]
            oy, ox = (H - hc) // 2, (W - wc) // 2
            y = x[:, :, oy:oy + hc, ox:ox + wc]
            z = np.einsum("ij,bjyx->iyxb", wgt.astype(np.float64), y, optimize=True)
            feats.append(np.ascontiguousarray(z.reshape(-1, B)))
        elif st["op"] == "tap_fc":
            B = x.shape[0]
            wm, bias = wgt if isinstance(wgt, tuple) else (wgt, None)
            z = wm.astype(np.float64) @ x.reshape(B, -1).T
            if bias is not None:
                z = z + bias.astype(np.float64)[:, None]
            feats.append(np.ascontiguousarray(z))
        elif st["op"] == "tap_integrate":
            # Sec. 3.3: plaintext neurons x_p^<1> = sigma(W'_1 x_p + b'_1) of the
            # first integration layer (sigma: the square activation), and their
            # term W_2 x_p^<1> + b_2 of the second layer
            B = x.shape[0]
            w1, b1, w2, b2 = (a.astype(np.float64) for a in wgt)
            h = w1 @ x.reshape(B, -1).T + b1[:, None]
            h = h * h
            feats.append(np.ascontiguousarray(w2 @ h + b2[:, None]))
        else:
            raise ValueError(st["op"])
    return feats


def fp64_network(cfg: dict, seg_vals: np.ndarray, feats: list, tables: list, scales: list) -> np.ndarray:
    """The same quantised network in float64 (real weights w_int * s_w, the
    square activation, the unidirectional adds): [n_in][B] -> [n_out][B]."""
    B = seg_vals.shape[1]
    step = 256  # images are independent: evaluate them in groups to bound memory
    outs = []
    for b0 in range(0, B, step):
        x = seg_vals[:, b0:b0 + step]
        fi = 0
        for layer, (idx, wt), s_w in zip(cfg["cipher"], tables, scales):
            safe = np.where(idx < 0, 0, idx)
            wr = wt.astype(np.float64) * s_w * (idx >= 0)
            y = np.einsum("ot,otb->ob", wr, x[safe], optimize=True)
            if layer["add"]:
                y = y + feats[fi][:, b0:b0 + step]
                fi += 1
            if layer["square"]:
                y = y * y
            x = y
        outs.append(x)
    return np.concatenate(outs, axis=1)


def scale_schedule(cfg: dict, q, scales: list):
    """Scale bookkeeping: integer weights divide the scale by s_w, a square
    squares it, the rescale divides by the dropped prime.  Returns (the scale
    each added feature must be encoded at, the output scale)."""
    S = 2.0 ** cfg["log_scale"]
    level = cfg["n_data"]
    add_scales = []
    for layer, s_w in zip(cfg["cipher"], scales):
        S = S / s_w
        if layer["add"]:
            add_scales.append(S)
        if layer["square"]:
            S = S * S / q[level - 1]
            level -= 1
    return add_scales, S


def evaluate(params: Params, cfg: dict, tables: list, evk: np.ndarray, cts: np.ndarray, pts: list,
             trace: list | None = None) -> np.ndarray:
    """Ciphertext-branch evaluation (Sec. 3.2, App. B): per layer the integer
    weight MAC, the optional plaintext-feature add, the optional square
    (tensor square, relinearise, rescale).  Returns the output ciphertexts."""
    level = params.L
    x = cts
    pi = 0
    for layer, (idx, wt) in zip(cfg["cipher"], tables):
        pt = None
        if layer["add"]:
            pt = pts[pi]
            pi += 1
        x = params.mac(level, idx, wt, x, pt)
        if trace is not None:
            trace.append(("mac", level, x))
        if layer["square"]:
            x = params.square_relin_rescale(level, evk, x)
            level -= 1
            if trace is not None:
                trace.append(("square", level, x))
    return x


# ---------------------------------------------------------------------------
# a whole seeded problem
# ---------------------------------------------------------------------------
class Problem:
    """Every input of one ciphertext-branch evaluation, built by the oracle
    from the seeded workload: keys, encrypted segment, plaintext-branch
    features and their encodings, quantised weights and tables."""

    def __init__(self, cfg: dict, params: Params | None = None, key_seed=workloads.SEED_KEYS,
                 enc_seed=workloads.SEED_ENC):
        self.cfg = cfg
        self.params = params or Params.from_config(cfg)
        P = self.params
        self.B = cfg["batch"]
        self.imgs = workloads.images(cfg)
        self.noise = workloads.laplace_noise(cfg)
        self.wf = workloads.cipher_weights(cfg)
        q = [quantize(w) for w in self.wf]
        self.w_int = [a for a, _ in q]
        self.s_w = [s for _, s in q]
        self.tables = [layer_table(l, w) for l, w in zip(cfg["cipher"], self.w_int)]
        self.pw = workloads.plain_weights(cfg)
        self.feats = plain_branch(cfg, self.imgs, self.noise, self.pw)
        self.add_scales, self.out_scale = scale_schedule(cfg, P.q, self.s_w)
        self.levels, self.out_level = workloads.level_schedule(cfg)
        self.sk, self.evk = P.keygen(key_seed)
        self.seg = segment_values(cfg, self.imgs)
        scale0 = 2.0 ** cfg["log_scale"]
        self.pt_in = encode(self.seg, P.N, scale0, P.q)
        self.cts = P.encrypt(self.sk, self.pt_in, P.L, enc_seed)
        self.pts = []
        fi = 0
        for layer, lv in zip(cfg["cipher"], self.levels):
            if layer["add"]:
                self.pts.append(encode(self.feats[fi], P.N, self.add_scales[fi], P.q[:lv]))
                fi += 1

    def evaluate(self, trace=None) -> np.ndarray:
        return evaluate(self.params, self.cfg, self.tables, self.evk, self.cts, self.pts, trace)

    def decode_output(self, out_ct: np.ndarray) -> np.ndarray:
        return decrypt_decode(self.params, self.sk, out_ct, self.out_level, self.B, self.out_scale)

    def fp64_logits(self) -> np.ndarray:
        return fp64_network(self.cfg, self.seg, self.feats, self.tables, self.s_w)


# ---------------------------------------------------------------------------
# BHW packing (App. D): one channel of n images' h x w segments per ciphertext
# ---------------------------------------------------------------------------
def pack_bhw(x: np.ndarray, N: int) -> np.ndarray:
    """x [n_img][C][h][w] -> slot vectors [C][N/2]: image b's pixel (y, x) of
    channel c in slot b*h*w + y*w + x; unused slots zero."""
    n, C, h, w = x.shape
    assert n * h * w <= N // 2
    out = np.zeros((C, N // 2))
    for c in range(C):
        out[c, :n * h * w] = x[:, c].reshape(-1)
    return out


def unpack_bhw(z: np.ndarray, n: int, h: int, w: int) -> np.ndarray:
    """slot vectors [C][N/2] -> [n][C][h][w] (the inverse of pack_bhw)."""
    C = z.shape[0]
    return z[:, :n * h * w].reshape(C, n, h, w).transpose(1, 0, 2, 3)


def conv_bhw(P: "Params", level: int, gks: dict, w_int: np.ndarray, cts: np.ndarray, w_img: int,
             gap: int = 1) -> np.ndarray:
    """Convolution of BHW-packed ciphertexts by rotations (App. D, homomorphic
    convolutional layer): out[co] = sum_{ci,i,j} w[co][ci][i][j] Rot(ct[ci], gap (i w_img + j)),
    k x k kernel.  The input map's logical pixel (y, x) sits in slot
    gap (y w_img + x) of its image's block (gap 1: every pixel of the segment;
    gap s after a stride-s layer), so the rotation by gap (i w_img + j) brings
    pixel (y + i, x + j) to the slot of (y, x): output (y, x) of each image sits
    in the input's slot of (y, x).  A stride-s layer is this sum with the
    outputs at logical positions (s y', s x') kept by a mask (mask_bhw); slots
    past the valid outputs hold neighbours' values.
    gks: {steps: Galois key}; cts [cin][2][level][N] -> [cout][2][level][N]."""
    cout, cin, k, _ = w_int.shape
    rots = []
    for ci in range(cin):
        for i in range(k):
            for j in range(k):
                r = gap * (i * w_img + j)
                rots.append(cts[ci] if r == 0 else P.rotate(level, gks[r], r, cts[ci:ci + 1])[0])
    x = np.stack(rots)
    idx = np.tile(np.arange(cin * k * k, dtype=np.int32), (cout, 1))
    return P.mac(level, idx, w_int.reshape(cout, -1).astype(np.int8), x)


def mask_bhw(n: int, h: int, w: int, k: int, stride: int, gap: int, N: int) -> np.ndarray:
    """0/1 slot vector [N/2] of the outputs a valid k x k, stride-s convolution
    keeps, for n images' h x w segments (slot b h w + y w + x) whose input
    pixels sit at gap `gap`: output (y', x') of the logical (h/gap) x (w/gap)
    map is at logical input position (s y', s x'), i.e. at slot
    b h w + gap s (y' w + x'), for s y' + k <= h/gap and s x' + k <= w/gap."""
    hl, wl = h // gap, w // gap
    m = np.zeros((n, h, w))
    ys = [gap * stride * yy for yy in range((hl - k) // stride + 1)]
    xs = [gap * stride * xx for xx in range((wl - k) // stride + 1)]
    for y in ys:
        m[:, y, xs] = 1.0
    return m.reshape(-1) if n * h * w == N // 2 else np.concatenate([m.reshape(-1), np.zeros(N // 2 - n * h * w)])


def fc_diagonals(W: np.ndarray, n_img: int, block: int, N: int) -> dict:
    """Slot vectors of the diagonal method (App. D, homomorphic fully connected
    layer) for y = W x, W [n2][n1], with image b's input x in slots
    [b block, b block + n1) and its output y in slots [b block, b block + n2):
    {r: u_r} over the rotations r = i - j (-(n2-1) <= r <= n1-1) with
    u_r[b block + j] = W[j][j + r] wherever 0 <= j < n2 and 0 <= j + r < n1,
    zero elsewhere, so that y = sum_r u_r * Rot(x, r) slot by slot."""
    n2, n1 = W.shape
    assert block >= max(n1, n2) and n_img * block <= N // 2
    out = {}
    for r in range(-(n2 - 1), n1):
        u = np.zeros(N // 2)
        for j in range(n2):
            if 0 <= j + r < n1:
                for b in range(n_img):
                    u[b * block + j] = W[j][j + r]
        if np.any(u):
            out[r] = u
    return out


def fc_diag(P: "Params", level: int, gks: dict, W: np.ndarray, ct: np.ndarray, n_img: int, block: int) -> np.ndarray:
    """Homomorphic fully connected layer by the diagonal method (App. D): the
    input ciphertext rotated by every r of fc_diagonals, each rotation multiplied
    by its diagonal u_r (Mult(c, u), u encoded at the scale q_{level-1} so that
    the rescale by q_{level-1} keeps the ciphertext's scale), the products summed,
    then one rescale.  Integer weights W [n2][n1].  ct [2][level][N] ->
    [2][level-1][N].  gks: {r mod N/2: Galois key}."""
    half = P.N // 2
    diags = fc_diagonals(W, n_img, block, P.N)
    acc = None
    for r, u in diags.items():
        rc = ct[None] if r % half == 0 else P.rotate(level, gks[r % half], r % half, ct[None])
        pt = encode(u[None], P.N, float(P.q[level - 1]), P.q[:level])[0]
        prod = P.mul_plain(level, rc, pt)[0].astype(np.uint64)
        acc = prod if acc is None else acc + prod
        acc %= np.array(P.q[:level], dtype=np.uint64)[None, :, None]
    return P.rescale(level, acc.astype(np.uint32)[None])[0]


def fc_diagonals_at(W: np.ndarray, n_img: int, block: int, s_in, o_out, N: int) -> dict:
    """The diagonal method (App. D, homomorphic fully connected layer) for
    inputs and outputs at any slots of each image's block: input p of image b
    in slot b block + s_in[p], output j in slot b block + o_out[j] (a strided
    packed convolution leaves its outputs at every s-th position).  A rotation
    by r moves slot k + r to slot k, so the term W[j][p] x_p needs the rotation
    r = s_in[p] - o_out[j] and sits in slot b block + o_out[j] of u_r:
    {r: u_r [N/2]} with y = sum_r u_r * Rot(x, r) holding y_j in slot
    b block + o_out[j].  Slots that are no s_in[p] never meet a nonzero entry,
    so the product also drops what a strided convolution's mask would."""
    n2, n1 = W.shape
    assert len(s_in) == n1 and len(o_out) == n2 and n_img * block <= N // 2
    assert 0 <= min(s_in) and max(s_in) < block and 0 <= min(o_out) and max(o_out) < block
    out = {}
    for j in range(n2):
        for p in range(n1):
            r = int(s_in[p]) - int(o_out[j])
            u = out.setdefault(r, np.zeros(N // 2))
            for b in range(n_img):
                u[b * block + o_out[j]] = W[j][p]
    return out


def add_plain(P: "Params", level: int, ct: np.ndarray, pt: np.ndarray) -> np.ndarray:
    """Add(c, u) of App. A: (c0 + u, c1) mod Q_level; ct [2][level][N], pt [level][N]."""
    out = np.array(ct, dtype=np.uint32)
    q = np.array(P.q[:level], dtype=np.uint64)[:, None]
    out[0] = ((out[0].astype(np.uint64) + np.asarray(pt, dtype=np.uint64)) % q).astype(np.uint32)
    return out


def fc_diag_sum(P: "Params", level: int, gks: dict, diags: list, cts: np.ndarray, pt=None) -> np.ndarray:
    """The dense layer of App. D over several input ciphertexts (BHW packing: one
    channel each): sum over inputs k and rotations r of Mult(Rot(x_k, r), u_{k,r}),
    each u encoded at the scale q_{level-1}; one rescale; then Add(c, pt) when
    pt [level-1][N] is given.  diags[k] = {r: u_r [N/2]} (fc_diagonals_at);
    cts [n_in][2][level][N] -> [2][level-1][N].  gks: {r mod N/2: Galois key}."""
    half = P.N // 2
    q = np.array(P.q[:level], dtype=np.uint64)[None, :, None]
    acc = np.zeros((2, level, P.N), dtype=np.uint64)
    for k, dk in enumerate(diags):
        for r in sorted(dk):
            x = cts[k][None]
            rc = x if r % half == 0 else P.rotate(level, gks[r % half], r % half, x)
            u = encode(dk[r][None], P.N, float(P.q[level - 1]), P.q[:level])[0]
            acc = (acc + P.mul_plain(level, rc, u)[0].astype(np.uint64)) % q
    y = P.rescale(level, acc.astype(np.uint32)[None])[0]
    return y if pt is None else add_plain(P, level - 1, y, pt)


def bhw_branch(P: "Params", evk: np.ndarray, gks: dict, layers: list, weights: list, feats: list,
               cts: np.ndarray, n_img: int) -> np.ndarray:
    """A ciphertext branch of one valid convolution then dense layers evaluated
    in BHW packing (App. D): n_img images' h x w segments of each input channel
    in one ciphertext (cts [cin][2][L][N], slot b h w + y w + x), in the
    layers' order:
      * conv (k x k, stride s): the packed convolution by rotations (conv_bhw);
        output (y', x') of image b stays at slot b h w + s (y' w + x');
      * dense: the diagonal method over the previous layer's ciphertexts
        (fc_diag_sum), input p = (channel, y', x') in torch's flattening order,
        output j at slot b h w + j;
    each followed, as the layer says, by Add(c, feature) (the unidirectional
    connection, Sec. 3.2) and the square (Mult(c, c), relinearise, rescale).
    weights: integer weights per layer (conv [cout][cin][k][k], dense
    [n_out][n_in]); feats: the encoded features of the layers with add=True in
    order (conv [cout][level][N] at the layer's level, dense [level-1][N] at the
    level after its rescale).  Returns [2][level][N] at the final level (outputs
    of image b at slots b h w + j)."""
    level = P.L
    h, w = layers[0]["h"], layers[0]["w"]
    block = h * w
    fi = 0
    x = cts
    pos = None
    for li, (lay, wt) in enumerate(zip(layers, weights)):
        if lay["type"] == "conv":
            assert li == 0 and lay["pad"] == 0
            x = conv_bhw(P, level, gks, np.asarray(wt, dtype=np.int8), x, w)
            if lay["add"]:
                x = np.stack([add_plain(P, level, x[c], feats[fi][c]) for c in range(x.shape[0])])
                fi += 1
            ho = (h - lay["k"]) // lay["stride"] + 1
            wo = (w - lay["k"]) // lay["stride"] + 1
            pos = [lay["stride"] * (yy * w + xx) for yy in range(ho) for xx in range(wo)]
        else:
            C = x.shape[0]
            n_pos = len(pos)
            assert wt.shape == (lay["n_out"], C * n_pos)
            diags = [fc_diagonals_at(wt[:, c * n_pos:(c + 1) * n_pos], n_img, block, pos,
                                     list(range(lay["n_out"])), P.N) for c in range(C)]
            pt = None
            if lay["add"]:
                pt = feats[fi]
                fi += 1
            x = fc_diag_sum(P, level, gks, diags, x, pt)[None]
            level -= 1
            pos = list(range(lay["n_out"]))
        if lay["square"]:
            x = P.square_relin_rescale(level, evk, x)
            level -= 1
    assert x.shape[0] == 1
    return x[0]
