"""Thin ctypes binding of libbcn.so (include/bcn.h), same names as the C ABI.

Argument marshalling only: host arrays are numpy, device buffers are torch CUDA
tensors (int32 storage for the uint32 residues), and every computation runs in
the native library.  There is no fallback: if the library cannot be loaded the
import of this module raises.
"""
from __future__ import annotations

import ctypes
import pathlib
import threading

import numpy as np

from . import _build

_P = ctypes.c_void_p
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_D = ctypes.c_double


class BcnError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_data", ctypes.c_uint32), ("n_special", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32)]


class _CtxInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("K", ctypes.c_uint32), ("alpha", ctypes.c_uint32),
                ("dnum", ctypes.c_uint32), ("device", ctypes.c_int)]


class _Layer(ctypes.Structure):
    _fields_ = [("type", _I), ("cin", _I), ("h", _I), ("w", _I), ("cout", _I), ("k", _I), ("stride", _I),
                ("pad", _I), ("n_in", _I), ("n_out", _I), ("add", _I), ("square", _I), ("w_int", _P), ("s_w", _D)]


class _ModelInfo(ctypes.Structure):
    _fields_ = [("n_layers", _I), ("n_in", _I), ("n_out", _I), ("out_level", _I), ("n_add", _I), ("stack", _I)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("model", _P), ("evk_eval", _P), ("cts", _P), ("pts", _P), ("out", _P)]


class _PlainStage(ctypes.Structure):
    _fields_ = [("op", _I), ("cin", _I), ("cout", _I), ("k", _I), ("stride", _I), ("pad", _I), ("relu", _I),
                ("hc", _I), ("wc", _I), ("ch_c", _I), ("n_out", _I), ("n_hidden", _I), ("bias", _I),
                ("weights", _P)]


# name -> (restype, argtypes); restype _I means a bcn_status
_SIGS = {
    "bcn_last_error": (ctypes.c_char_p, []),
    "bcn_ctx_create": (_I, [ctypes.POINTER(_Params), _I, ctypes.POINTER(_P)]),
    "bcn_ctx_destroy": (_I, [_P]),
    "bcn_ctx_get_info": (_I, [_P, ctypes.POINTER(_CtxInfo)]),
    "bcn_ctx_primes": (_I, [_P, _P]),
    "bcn_evk_words": (_SZ, [_P]),
    "bcn_device_status": (_I, [_P, _P]),
    "bcn_ctx_set_debug": (_I, [_P, _I]),
    "bcn_ctx_set_ntt_shape": (_I, [_P, _I]),
    "bcn_ctx_get_ntt_shape": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "bcn_ctx_get_debug": (_I, [_P, ctypes.POINTER(_I)]),
    "bcn_keygen": (_I, [_P, _U64, _P, _P]),
    "bcn_quantize": (_I, [_P, _SZ, _P, ctypes.POINTER(_D)]),
    "bcn_encode": (_I, [_P, _P, _I, _I, _I, _D, _P]),
    "bcn_encrypt": (_I, [_P, _P, _P, _I, _I, _U64, _P]),
    "bcn_encrypt_segment": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _D, _U64, _P]),
    "bcn_encrypt_seeded": (_I, [_P, _P, _P, _I, _I, _U64, _P]),
    "bcn_encrypt_segment_seeded": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _D, _U64, _P]),
    "bcn_expand_seeded": (_I, [_P, _P, _I, _I, _U64, _I, _P, _P]),
    "bcn_encode_i64": (_I, [_P, _P, _I, _I, _D, _P]),
    "bcn_expand_i64": (_I, [_P, _P, _I, _I, _P, _P]),
    "bcn_decrypt_decode": (_I, [_P, _P, _P, _I, _I, _D, _I, _P]),
    "bcn_message_bytes": (_SZ, [_P, _I, _I, _I]),
    "bcn_serialize": (_I, [_P, _I, _I, _I, ctypes.c_uint32, _P, _P, _SZ]),
    "bcn_deserialize_header": (_I, [_P, _P, _SZ, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                    ctypes.POINTER(ctypes.c_uint32)]),
    "bcn_deserialize": (_I, [_P, _P, _SZ, _P, _SZ]),
    "bcn_plain_model_create": (_I, [_P, _P, _I, _I, _I, _I, _P, ctypes.POINTER(_P)]),
    "bcn_plain_model_destroy": (_I, [_P]),
    "bcn_plain_feature_count": (_I, [_P, ctypes.POINTER(_I)]),
    "bcn_plain_workspace_bytes": (_I, [_P, _I, ctypes.POINTER(_SZ)]),
    "bcn_plain_branch_forward": (_I, [_P, _P, _P, _I, _P, _P, _SZ, _P]),
    "bcn_model_create": (_I, [_P, _P, _I, ctypes.POINTER(_P)]),
    "bcn_model_create_stacked": (_I, [_P, _P, _I, _I, ctypes.POINTER(_P)]),
    "bcn_eval_stacked": (_I, [_P, _P, _I, _P, _P, _P, _P, _SZ, _P]),
    "bcn_model_destroy": (_I, [_P]),
    "bcn_model_set_chunk": (_I, [_P, _I]),
    "bcn_model_set_mac_impl": (_I, [_P, _I]),
    "bcn_model_set_overlap": (_I, [_P, _I]),
    "bcn_model_get_info": (_I, [_P, ctypes.POINTER(_ModelInfo)]),
    "bcn_model_layers": (_I, [_P, _P, _P]),
    "bcn_model_scales": (_I, [_P, _D, _P, ctypes.POINTER(_D)]),
    "bcn_evk_prepare": (_I, [_P, _P, _P, _P]),
    "bcn_eval_workspace_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "bcn_eval": (_I, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "bcn_eval_host_workspace_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "bcn_eval_host": (_I, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "bcn_eval_host_async": (_I, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "bcn_eval_host_seeded_async": (_I, [_P, _P, _P, _U64, _P, _P, _P, _SZ, _P]),
    "bcn_eval_host_compact_async": (_I, [_P, _P, _P, _U64, _P, _P, _P, _SZ, _P]),
    "bcn_batch_plan": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
    "bcn_batch_create": (_I, [_P, _I, _I, _P, _SZ, ctypes.POINTER(_P)]),
    "bcn_batch_launch": (_I, [_P, _P]),
    "bcn_batch_lanes": (_I, [_P, _P]),
    "bcn_batch_destroy": (_I, [_P]),
    "bcn_model_cost": (_I, [_P, ctypes.POINTER(_D)]),
    "bcn_profile_enable": (_I, [_P, _I]),
    "bcn_profile_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D)]),
    "bcn_op_ntt": (_I, [_P, _P, _I, _I, _I, _P]),
    "bcn_op_mac": (_I, [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "bcn_op_workspace_bytes": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
    "bcn_op_tensor_square": (_I, [_P, _I, _P, _I, _P, _P, _SZ, _P]),
    "bcn_op_square_relin_rescale": (_I, [_P, _I, _P, _P, _I, _P, _P, _SZ, _P]),
    "bcn_op_rescale": (_I, [_P, _I, _P, _I, _P, _P]),
    "bcn_galois_elt": (ctypes.c_uint32, [_P, _I]),
    "bcn_op_mul_plain_rescale": (_I, [_P, _I, _P, _I, _P, _P, _P, _SZ, _P]),
    "bcn_galois_keygen": (_I, [_P, _P, _I, _U64, _P]),
    "bcn_op_rotate": (_I, [_P, _I, _P, _I, _P, _I, _P, _P, _SZ, _P]),
    "bcn_op_square_relin_rescale_noalloc": (_I, [_P, _I, _P, _P, _I, _P, _P]),
    "bcn_op_rotate_many_workspace_bytes": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
    "bcn_op_rotate_many": (_I, [_P, _I, _P, _P, _I, _P, _I, _P, _P, _SZ, _P]),
    "bcn_op_fc_diag_workspace_bytes": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
    "bcn_op_fc_diag": (_I, [_P, _I, _P, _P, _I, _P, _P, _I, _P, _P, _SZ, _P]),
    "bcn_op_fc_diag_sum": (_I, [_P, _I, _P, _P, _I, _P, _P, _I, _I, _P, _P, _P, _SZ, _P]),
    "bcn_int_peak_grid": (_I, [_I, ctypes.POINTER(_I)]),
    "bcn_int_peak_launch": (_I, [_I, _I, _P, _SZ, _P, ctypes.POINTER(_D)]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> pathlib.Path:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libbcn.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(str(path))
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(st: int, where: str):
    if st != 0:
        raise BcnError(st, where, lib().bcn_last_error().decode())


def _np_ptr(a: np.ndarray, dtype) -> int:
    assert a.dtype == np.dtype(dtype) and a.flags["C_CONTIGUOUS"], (a.dtype, dtype)
    return a.ctypes.data


def _dev_ptr(t, nwords=None) -> int:
    """Device pointer of a contiguous CUDA tensor of 4-byte elements."""
    import torch

    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if nwords is not None and t.numel() * t.element_size() < nwords * 4:
        raise ValueError(f"device buffer too small: {t.numel() * t.element_size()} bytes < {nwords * 4}")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def to_device(a: np.ndarray, device="cuda"):
    """uint32 / int8 numpy array -> CUDA tensor with the same bytes."""
    import torch

    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(device)


def to_host_u32(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------------------
def quantize(w: np.ndarray):
    """bcn_quantize: per-tensor symmetric int8 quantisation (fp64)."""
    w = np.ascontiguousarray(w, dtype=np.float32)
    out = np.zeros(w.shape, dtype=np.int8)
    s = _D()
    _check(lib().bcn_quantize(_np_ptr(w, np.float32), w.size, _np_ptr(out, np.int8), ctypes.byref(s)), "bcn_quantize")
    return out, s.value


class Context:
    """bcn_ctx: parameters, prime chain and device tables (device < 0: host only)."""

    def __init__(self, log_n: int, n_data: int, n_special: int, alpha: int, device: int = 0):
        p = _Params(log_n, n_data, n_special, alpha)
        h = _P()
        _check(lib().bcn_ctx_create(ctypes.byref(p), device, ctypes.byref(h)), "bcn_ctx_create")
        self._h = h
        info = _CtxInfo()
        _check(lib().bcn_ctx_get_info(self._h, ctypes.byref(info)), "bcn_ctx_get_info")
        self.N, self.L, self.K, self.alpha, self.dnum, self.device = (info.N, info.L, info.K, info.alpha, info.dnum,
                                                                      info.device)
        pr = np.zeros(self.L + self.K, dtype=np.uint64)
        _check(lib().bcn_ctx_primes(self._h, _np_ptr(pr, np.uint64)), "bcn_ctx_primes")
        self.primes = [int(x) for x in pr]
        self.q, self.p = self.primes[:self.L], self.primes[self.L:]

    @classmethod
    def from_config(cls, cfg: dict, device: int = 0) -> "Context":
        return cls(cfg["log_n"], cfg["n_data"], cfg["n_special"], cfg["alpha"], device)

    def close(self):
        if getattr(self, "_h", None):
            lib().bcn_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def evk_words(self) -> int:
        return int(lib().bcn_evk_words(self._h))

    def evk_shape(self):
        return (self.dnum, 2, self.L + self.K, self.N)

    def set_ntt_shape(self, shape: int):
        """bcn_ctx_set_ntt_shape: 0 the default block shape of the NTT-based kernels, 1 the alternative."""
        _check(lib().bcn_ctx_set_ntt_shape(self._h, int(shape)), "bcn_ctx_set_ntt_shape")

    def ntt_shape(self):
        """(selected shape, residues per thread of the NTT kernels)."""
        a, r = _I(), _I()
        _check(lib().bcn_ctx_get_ntt_shape(self._h, ctypes.byref(a), ctypes.byref(r)), "bcn_ctx_get_ntt_shape")
        return a.value, r.value

    def set_debug(self, on: bool = True):
        """bcn_ctx_set_debug: device-side checks of every call's inputs (residues
        below their primes, table indices in range) before it launches."""
        _check(lib().bcn_ctx_set_debug(self._h, int(on)), "bcn_ctx_set_debug")

    def debug(self) -> bool:
        v = _I()
        _check(lib().bcn_ctx_get_debug(self._h, ctypes.byref(v)), "bcn_ctx_get_debug")
        return bool(v.value)

    def device_status(self) -> int:
        """Reads and clears the device status word (0: no bounded wait gave up)."""
        v = ctypes.c_uint32(0)
        _check(lib().bcn_device_status(self._h, ctypes.byref(v)), "bcn_device_status")
        return int(v.value)

    # -- client side (host) ---------------------------------------------
    def keygen(self, seed: int):
        sk = np.zeros(self.N, dtype=np.int8)
        evk = np.zeros(self.evk_shape(), dtype=np.uint32)
        _check(lib().bcn_keygen(self._h, seed, _np_ptr(sk, np.int8), _np_ptr(evk, np.uint32)), "bcn_keygen")
        return sk, evk

    def galois_elt(self, steps: int) -> int:
        return int(lib().bcn_galois_elt(self._h, int(steps)))

    def galois_keygen(self, sk: np.ndarray, steps: int, seed: int) -> np.ndarray:
        gk = np.zeros(self.evk_shape(), dtype=np.uint32)
        _check(lib().bcn_galois_keygen(self._h, _np_ptr(np.ascontiguousarray(sk, dtype=np.int8), np.int8),
                                       int(steps), seed, _np_ptr(gk, np.uint32)), "bcn_galois_keygen")
        return gk

    def encode(self, values: np.ndarray, level: int, scale: float) -> np.ndarray:
        v = np.ascontiguousarray(np.atleast_2d(values), dtype=np.float64)
        n_vec, B = v.shape
        out = np.zeros((n_vec, level, self.N), dtype=np.uint32)
        _check(lib().bcn_encode(self._h, _np_ptr(v, np.float64), n_vec, B, level, scale, _np_ptr(out, np.uint32)),
               "bcn_encode")
        return out

    def encode_i64(self, values: np.ndarray, scale: float) -> np.ndarray:
        """bcn_encode_i64: the encoding's integer coefficients [n_vec][N] (int64)."""
        v = np.ascontiguousarray(np.atleast_2d(values), dtype=np.float64)
        n_vec, B = v.shape
        out = np.zeros((n_vec, self.N), dtype=np.int64)
        _check(lib().bcn_encode_i64(self._h, _np_ptr(v, np.float64), n_vec, B, scale, _np_ptr(out, np.int64)),
               "bcn_encode_i64")
        return out

    def expand_i64(self, coeffs_dev, n: int, level: int, out_dev, stream=None):
        """bcn_expand_i64: integer coefficients [n][N] (device int64) -> residues [n][level][N]."""
        import torch

        assert coeffs_dev.dtype == torch.int64 and coeffs_dev.is_cuda and coeffs_dev.is_contiguous()
        assert coeffs_dev.numel() >= n * self.N
        _check(lib().bcn_expand_i64(self._h, coeffs_dev.data_ptr(), n, level, _dev_ptr(out_dev, n * level * self.N),
                                    _stream(stream)), "bcn_expand_i64")

    def encrypt(self, sk: np.ndarray, pts: np.ndarray, level: int, seed: int) -> np.ndarray:
        pts = np.ascontiguousarray(pts, dtype=np.uint32)
        n = pts.shape[0]
        assert pts.shape == (n, level, self.N)
        out = np.zeros((n, 2, level, self.N), dtype=np.uint32)
        _check(lib().bcn_encrypt(self._h, _np_ptr(np.ascontiguousarray(sk), np.int8), _np_ptr(pts, np.uint32), n,
                                 level, seed, _np_ptr(out, np.uint32)), "bcn_encrypt")
        return out

    def encrypt_segment(self, sk, images: np.ndarray, seg, scale: float, seed: int) -> np.ndarray:
        images = np.ascontiguousarray(images, dtype=np.uint8)
        B, H, W, C = images.shape
        seg_a = np.ascontiguousarray(seg, dtype=np.int32)
        n = C * int(seg[2]) * int(seg[3])
        out = np.zeros((n, 2, self.L, self.N), dtype=np.uint32)
        _check(lib().bcn_encrypt_segment(self._h, _np_ptr(np.ascontiguousarray(sk), np.int8),
                                         _np_ptr(images, np.uint8), B, H, W, C, _np_ptr(seg_a, np.int32), scale,
                                         seed, _np_ptr(out, np.uint32)), "bcn_encrypt_segment")
        return out

    def encrypt_seeded(self, sk: np.ndarray, pts: np.ndarray, level: int, seed: int) -> np.ndarray:
        """bcn_encrypt_seeded: c0 alone [n][level][N] (c1 follows from the seed)."""
        pts = np.ascontiguousarray(pts, dtype=np.uint32)
        n = pts.shape[0]
        assert pts.shape == (n, level, self.N)
        out = np.zeros((n, level, self.N), dtype=np.uint32)
        _check(lib().bcn_encrypt_seeded(self._h, _np_ptr(np.ascontiguousarray(sk), np.int8), _np_ptr(pts, np.uint32),
                                        n, level, seed, _np_ptr(out, np.uint32)), "bcn_encrypt_seeded")
        return out

    def encrypt_segment_seeded(self, sk, images: np.ndarray, seg, scale: float, seed: int) -> np.ndarray:
        """bcn_encrypt_segment_seeded: c0 alone [C*h*w][L][N]."""
        images = np.ascontiguousarray(images, dtype=np.uint8)
        B, H, W, C = images.shape
        seg_a = np.ascontiguousarray(seg, dtype=np.int32)
        n = C * int(seg[2]) * int(seg[3])
        out = np.zeros((n, self.L, self.N), dtype=np.uint32)
        _check(lib().bcn_encrypt_segment_seeded(self._h, _np_ptr(np.ascontiguousarray(sk), np.int8),
                                                _np_ptr(images, np.uint8), B, H, W, C, _np_ptr(seg_a, np.int32), scale,
                                                seed, _np_ptr(out, np.uint32)), "bcn_encrypt_segment_seeded")
        return out

    def expand_seeded(self, c0_dev, n_ct: int, level: int, seed: int, out_dev, ct_base: int = 0, stream=None):
        """bcn_expand_seeded: c0 [n][level][N] (device) -> full ciphertexts [n][2][level][N]."""
        _check(lib().bcn_expand_seeded(self._h, _dev_ptr(c0_dev, n_ct * level * self.N), n_ct, level, seed, ct_base,
                                       _dev_ptr(out_dev, 2 * n_ct * level * self.N), _stream(stream)),
               "bcn_expand_seeded")

    def decrypt_decode(self, sk, cts: np.ndarray, level: int, scale: float, B: int) -> np.ndarray:
        cts = np.ascontiguousarray(cts, dtype=np.uint32)
        n = cts.shape[0]
        assert cts.shape == (n, 2, level, self.N)
        out = np.zeros((n, B), dtype=np.float64)
        _check(lib().bcn_decrypt_decode(self._h, _np_ptr(np.ascontiguousarray(sk), np.int8),
                                        _np_ptr(cts, np.uint32), n, level, scale, B, _np_ptr(out, np.float64)),
               "bcn_decrypt_decode")
        return out

    # -- messages (client <-> server) -------------------------------------
    MSG_CIPHERTEXTS, MSG_RELIN_KEY, MSG_GALOIS_KEY, MSG_PLAINTEXTS = 1, 2, 3, 4

    def serialize(self, kind: int, words: np.ndarray, level: int = 0, galois: int = 0) -> bytes:
        """bcn_serialize: ciphertexts [n][2][level][N] or plaintexts [n][level][N]
        (count = n), or a raw key (level 0, count 1; galois = its element for a
        Galois key) -> the message bytes."""
        w = np.ascontiguousarray(words, dtype=np.uint32)
        count = 1 if kind in (self.MSG_RELIN_KEY, self.MSG_GALOIS_KEY) else int(w.shape[0])
        nb = int(lib().bcn_message_bytes(self._h, kind, level, count))
        if nb == 0:
            raise BcnError(-1, "bcn_message_bytes", "bad message shape")
        out = np.zeros(nb, dtype=np.uint8)
        _check(lib().bcn_serialize(self._h, kind, level, count, int(galois), _np_ptr(w, np.uint32),
                                   _np_ptr(out, np.uint8), nb), "bcn_serialize")
        return out.tobytes()

    def deserialize(self, msg: bytes) -> dict:
        """bcn_deserialize: the message -> {kind, level, count, galois, words}
        (words shaped as serialize took them)."""
        buf = np.frombuffer(msg, dtype=np.uint8)
        k, lv, ct, g = _I(), _I(), _I(), ctypes.c_uint32()
        _check(lib().bcn_deserialize_header(self._h, _np_ptr(buf, np.uint8), buf.size, ctypes.byref(k),
                                            ctypes.byref(lv), ctypes.byref(ct), ctypes.byref(g)),
               "bcn_deserialize_header")
        if k.value == self.MSG_CIPHERTEXTS:
            shape = (ct.value, 2, lv.value, self.N)
        elif k.value == self.MSG_PLAINTEXTS:
            shape = (ct.value, lv.value, self.N)
        else:
            shape = self.evk_shape()
        out = np.zeros(shape, dtype=np.uint32)
        _check(lib().bcn_deserialize(self._h, _np_ptr(buf, np.uint8), buf.size, _np_ptr(out, np.uint32), out.size),
               "bcn_deserialize")
        return {"kind": k.value, "level": lv.value, "count": ct.value, "galois": g.value, "words": out}

    # -- device ----------------------------------------------------------
    def evk_prepare(self, evk_dev, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty_like(evk_dev)
        _check(lib().bcn_evk_prepare(self._h, _dev_ptr(evk_dev, self.evk_words()), _dev_ptr(out, self.evk_words()),
                                     _stream(stream)), "bcn_evk_prepare")
        return out

    def op_ntt(self, data, n_poly: int, level: int, inverse: bool, stream=None):
        _check(lib().bcn_op_ntt(self._h, _dev_ptr(data, n_poly * level * self.N), n_poly, level, int(inverse),
                                _stream(stream)), "bcn_op_ntt")

    def op_mac(self, level, n_in, idx_dev, w_dev, in_dev, pt_dev, out_dev, stream=None):
        n_out, K = idx_dev.shape
        _check(lib().bcn_op_mac(self._h, level, n_in, n_out, K, idx_dev.data_ptr(), w_dev.data_ptr(),
                                _dev_ptr(in_dev, n_in * 2 * level * self.N),
                                _dev_ptr(pt_dev, n_out * level * self.N) if pt_dev is not None else None,
                                _dev_ptr(out_dev, n_out * 2 * level * self.N), _stream(stream)), "bcn_op_mac")

    def op_workspace_bytes(self, level: int, n_ct: int) -> int:
        b = _SZ()
        _check(lib().bcn_op_workspace_bytes(self._h, level, n_ct, ctypes.byref(b)), "bcn_op_workspace_bytes")
        return b.value

    def _ws(self, level, n_ct):
        import torch

        nb = self.op_workspace_bytes(level, n_ct)
        return torch.empty(max(1, (nb + 3) // 4), dtype=torch.int32, device=f"cuda:{self.device}"), nb

    def op_tensor_square(self, level, in_dev, n_ct, out_dev, stream=None):
        ws, nb = self._ws(level, n_ct)
        _check(lib().bcn_op_tensor_square(self._h, level, _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                          _dev_ptr(out_dev, n_ct * 3 * level * self.N), ws.data_ptr(), nb,
                                          _stream(stream)), "bcn_op_tensor_square")

    def op_square_relin_rescale(self, level, evk_eval, in_dev, n_ct, out_dev, stream=None):
        ws, nb = self._ws(level, n_ct)
        _check(lib().bcn_op_square_relin_rescale(self._h, level, _dev_ptr(evk_eval, self.evk_words()),
                                                 _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                                 _dev_ptr(out_dev, n_ct * 2 * (level - 1) * self.N), ws.data_ptr(),
                                                 nb, _stream(stream)), "bcn_op_square_relin_rescale")

    def op_square_relin_rescale_noalloc(self, level, evk_eval, in_dev, n_ct, out_dev, stream=None):
        """bcn_op_square_relin_rescale_noalloc: the same square activation for
        callers that may not allocate device memory; its intermediates live in the
        library's fixed 32 MiB device array, so no workspace is passed (or made)."""
        _check(lib().bcn_op_square_relin_rescale_noalloc(
            self._h, level, _dev_ptr(evk_eval, self.evk_words()), _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
            _dev_ptr(out_dev, n_ct * 2 * (level - 1) * self.N), _stream(stream)),
            "bcn_op_square_relin_rescale_noalloc")

    def op_rotate(self, level, gk_eval, steps, in_dev, n_ct, out_dev, stream=None):
        """Slot rotation by `steps` (automorphism + key switch with the prepared Galois key)."""
        ws, nb = self._ws(level, n_ct)
        _check(lib().bcn_op_rotate(self._h, level, _dev_ptr(gk_eval, self.evk_words()), int(steps),
                                   _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                   _dev_ptr(out_dev, n_ct * 2 * level * self.N), ws.data_ptr(), nb, _stream(stream)),
               "bcn_op_rotate")

    def op_rotate_many(self, level, gk_evals: dict, steps: list, in_dev, n_ct, out_dev, workspace=None,
                       stream=None):
        """bcn_op_rotate_many: every ciphertext of in_dev [n_ct][2][level][N] rotated
        by every entry of `steps`, one hoisted ModUp per ciphertext; out_dev
        [n_ct][len(steps)][2][level][N].  gk_evals: {steps: prepared Galois key}
        (steps taken mod N/2; 0 needs no key)."""
        n_rot = len(steps)
        ptrs, st = self._key_table(gk_evals, steps)
        nb = _SZ(0)
        _check(lib().bcn_op_rotate_many_workspace_bytes(self._h, level, n_ct, ctypes.byref(nb)),
               "bcn_op_rotate_many_workspace_bytes")
        if workspace is None:
            import torch
            workspace = torch.empty(max(1, (nb.value + 3) // 4), dtype=torch.int32, device=f"cuda:{self.device}")
        _check(lib().bcn_op_rotate_many(self._h, level, ptrs, st, n_rot, _dev_ptr(in_dev, n_ct * 2 * level * self.N),
                                        n_ct, _dev_ptr(out_dev, n_ct * n_rot * 2 * level * self.N),
                                        workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "bcn_op_rotate_many")

    def _key_table(self, gk_evals: dict, steps: list):
        half = self.N // 2
        ptrs = (ctypes.c_void_p * max(1, len(steps)))()
        st = (ctypes.c_int * max(1, len(steps)))()
        for i, r in enumerate(steps):
            st[i] = int(r)
            key = gk_evals.get(r, gk_evals.get(r % half)) if r % half else None
            ptrs[i] = _dev_ptr(key, self.evk_words()) if key is not None else None
        return ptrs, st

    def op_fc_diag(self, level, gk_evals: dict, steps: list, diag_ntt, in_dev, n_ct, out_dev, stream=None):
        """bcn_op_fc_diag: the diagonal-method dense layer; diag_ntt [len(steps)][level][N]
        (NTT domain), in [n_ct][2][level][N] -> out [n_ct][2][level-1][N]."""
        import torch

        n_rot = len(steps)
        ptrs, st = self._key_table(gk_evals, steps)
        nb = _SZ(0)
        _check(lib().bcn_op_fc_diag_workspace_bytes(self._h, level, n_rot, ctypes.byref(nb)),
               "bcn_op_fc_diag_workspace_bytes")
        ws = torch.empty(max(1, (nb.value + 3) // 4), dtype=torch.int32, device=f"cuda:{self.device}")
        _check(lib().bcn_op_fc_diag(self._h, level, ptrs, st, n_rot, _dev_ptr(diag_ntt, n_rot * level * self.N),
                                    _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                    _dev_ptr(out_dev, n_ct * 2 * (level - 1) * self.N), ws.data_ptr(), nb.value,
                                    _stream(stream)), "bcn_op_fc_diag")

    def op_fc_diag_sum(self, level, gk_evals: dict, steps: list, diag_ntt, in_dev, n_in, n_groups, out_dev,
                       pt_dev=None, workspace=None, stream=None):
        """bcn_op_fc_diag_sum: the diagonal-method dense layer over n_in inputs per
        group; diag_ntt [n_in][len(steps)][level][N] (NTT domain), in
        [n_groups][n_in][2][level][N] -> out [n_groups][2][level-1][N], plus
        pt_dev [n_groups][level-1][N] when given."""
        n_rot = len(steps)
        ptrs, st = self._key_table(gk_evals, steps)
        if workspace is None:
            workspace = self.fc_diag_workspace(level, n_rot)
        _check(lib().bcn_op_fc_diag_sum(self._h, level, ptrs, st, n_rot,
                                        _dev_ptr(diag_ntt, n_in * n_rot * level * self.N),
                                        _dev_ptr(in_dev, n_groups * n_in * 2 * level * self.N), n_in, n_groups,
                                        _dev_ptr(pt_dev, n_groups * (level - 1) * self.N) if pt_dev is not None
                                        else None,
                                        _dev_ptr(out_dev, n_groups * 2 * (level - 1) * self.N), workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_op_fc_diag_sum")

    def fc_diag_workspace(self, level: int, n_rot: int):
        """A device workspace for bcn_op_fc_diag / bcn_op_fc_diag_sum."""
        import torch

        nb = _SZ(0)
        _check(lib().bcn_op_fc_diag_workspace_bytes(self._h, level, n_rot, ctypes.byref(nb)),
               "bcn_op_fc_diag_workspace_bytes")
        return torch.empty(max(1, (nb.value + 3) // 4), dtype=torch.int32, device=f"cuda:{self.device}")

    def op_mul_plain_rescale(self, level, in_dev, n_ct, pt_dev, out_dev, stream=None):
        """(c0 u, c1 u), then rescale: in [n_ct][2][level][N], pt [level][N] -> out at level - 1."""
        ws, nb = self._ws(level, n_ct)
        _check(lib().bcn_op_mul_plain_rescale(self._h, level, _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                              _dev_ptr(pt_dev, level * self.N),
                                              _dev_ptr(out_dev, n_ct * 2 * (level - 1) * self.N), ws.data_ptr(), nb,
                                              _stream(stream)), "bcn_op_mul_plain_rescale")

    def op_rescale(self, level, in_dev, n_ct, out_dev, stream=None):
        _check(lib().bcn_op_rescale(self._h, level, _dev_ptr(in_dev, n_ct * 2 * level * self.N), n_ct,
                                    _dev_ptr(out_dev, n_ct * 2 * (level - 1) * self.N), _stream(stream)),
               "bcn_op_rescale")


LAYER_TYPES = {"conv": 0, "dense": 1}


class Model:
    """bcn_model: the ciphertext branch (integer weights, feature adds, squares)."""

    def __init__(self, ctx: Context, layers: list, w_int: list, s_w: list, stack: int = 1):
        """stack > 1: bcn_model_create_stacked (that many requests side by side)."""
        self.ctx = ctx
        self._spec = (list(layers), list(w_int), list(s_w))
        self._keep = [np.ascontiguousarray(w, dtype=np.int8) for w in w_int]
        arr = (_Layer * len(layers))()
        for i, (l, w, s) in enumerate(zip(layers, self._keep, s_w)):
            a = arr[i]
            a.type = LAYER_TYPES[l["type"]]
            for f in ("cin", "h", "w", "cout", "k", "stride", "pad", "n_in", "n_out"):
                setattr(a, f, int(l.get(f, 0)))
            a.add, a.square = int(bool(l["add"])), int(bool(l["square"]))
            a.w_int = w.ctypes.data
            a.s_w = float(s)
        h = _P()
        if stack == 1:
            _check(lib().bcn_model_create(ctx.handle, ctypes.cast(arr, _P), len(layers), ctypes.byref(h)),
                   "bcn_model_create")
        else:
            _check(lib().bcn_model_create_stacked(ctx.handle, ctypes.cast(arr, _P), len(layers), int(stack),
                                                  ctypes.byref(h)), "bcn_model_create_stacked")
        self._h = h
        info = _ModelInfo()
        _check(lib().bcn_model_get_info(self._h, ctypes.byref(info)), "bcn_model_get_info")
        self.n_layers, self.n_in, self.n_out, self.out_level, self.n_add = (info.n_layers, info.n_in, info.n_out,
                                                                            info.out_level, info.n_add)
        self.stack = info.stack
        lv = np.zeros(self.n_layers, dtype=np.int32)
        no = np.zeros(self.n_layers, dtype=np.int32)
        _check(lib().bcn_model_layers(self._h, _np_ptr(lv, np.int32), _np_ptr(no, np.int32)), "bcn_model_layers")
        self.levels, self.n_outs = lv.tolist(), no.tolist()
        self.add_layers = [i for i, l in enumerate(layers) if l["add"]]

    def close(self):
        if getattr(self, "_h", None):
            lib().bcn_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def scales(self, input_scale: float):
        adds = np.zeros(max(1, self.n_add), dtype=np.float64)
        out = _D()
        _check(lib().bcn_model_scales(self._h, input_scale, _np_ptr(adds, np.float64), ctypes.byref(out)),
               "bcn_model_scales")
        return adds[:self.n_add].tolist(), out.value

    def pt_shapes(self):
        return [(self.n_outs[i], self.levels[i], self.ctx.N) for i in self.add_layers]

    def out_shape(self):
        return (self.n_out, 2, self.out_level, self.ctx.N)

    def workspace_bytes(self) -> int:
        b = _SZ()
        _check(lib().bcn_eval_workspace_bytes(self._h, ctypes.byref(b)), "bcn_eval_workspace_bytes")
        return b.value

    def host_workspace_bytes(self) -> int:
        b = _SZ()
        _check(lib().bcn_eval_host_workspace_bytes(self._h, ctypes.byref(b)), "bcn_eval_host_workspace_bytes")
        return b.value

    def alloc_workspace(self, host: bool = False):
        import torch

        nb = self.host_workspace_bytes() if host else self.workspace_bytes()
        return torch.empty(max(1, (nb + 3) // 4), dtype=torch.int32, device=f"cuda:{self.ctx.device}")

    KERNELS = ["mac", "square", "keyswitch", "moddown_rescale"]

    def set_chunk(self, chunk: int):
        _check(lib().bcn_model_set_chunk(self._h, int(chunk)), "bcn_model_set_chunk")

    def set_overlap(self, on: bool):
        """bcn_model_set_overlap: False gives the plain path (every kernel in order on one stream)."""
        _check(lib().bcn_model_set_overlap(self._h, 1 if on else 0), "bcn_model_set_overlap")

    def set_mac_impl(self, impl: int):
        """0: tensor cores where eligible (default); 1: CUDA cores only."""
        _check(lib().bcn_model_set_mac_impl(self._h, int(impl)), "bcn_model_set_mac_impl")

    def profile_enable(self, on: bool = True):
        _check(lib().bcn_profile_enable(self._h, int(on)), "bcn_profile_enable")

    def profile_read(self) -> dict:
        """{kernel: (total_ms, launches, algorithmic_bytes)} since profile_enable."""
        out = {}
        for i, name in enumerate(self.KERNELS):
            ms, n, b = _D(), ctypes.c_longlong(), _D()
            _check(lib().bcn_profile_read(self._h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)),
                   "bcn_profile_read")
            out[name] = (ms.value, n.value, b.value)
        return out

    def eval(self, evk_eval, cts_dev, pts_dev: list, out_dev, workspace, stream=None):
        N = self.ctx.N
        arr = (_P * max(1, len(pts_dev)))(*[_dev_ptr(p, int(np.prod(s))) for p, s in zip(pts_dev, self.pt_shapes())])
        _check(lib().bcn_eval(self._h, _dev_ptr(evk_eval, self.ctx.evk_words()),
                              _dev_ptr(cts_dev, self.n_in * 2 * self.ctx.L * N), ctypes.cast(arr, _P),
                              _dev_ptr(out_dev, int(np.prod(self.out_shape()))), workspace.data_ptr(),
                              workspace.numel() * workspace.element_size(), _stream(stream)), "bcn_eval")

    def stacked(self, requests: int) -> "Model":
        """The same network for `requests` slot batches side by side."""
        layers, w_int, s_w = self._spec
        return Model(self.ctx, layers, w_int, s_w, stack=requests)

    def eval_stacked(self, evk_evals: list, cts_dev, pts_dev: list, out_dev, workspace, stream=None):
        """bcn_eval_stacked: one prepared key per request of a stacked model."""
        N = self.ctx.N
        keys = (_P * len(evk_evals))(*[_dev_ptr(k, self.ctx.evk_words()) for k in evk_evals])
        arr = (_P * max(1, len(pts_dev)))(*[_dev_ptr(p, int(np.prod(s))) for p, s in zip(pts_dev, self.pt_shapes())])
        _check(lib().bcn_eval_stacked(self._h, ctypes.cast(keys, _P), len(evk_evals),
                                      _dev_ptr(cts_dev, self.n_in * 2 * self.ctx.L * N), ctypes.cast(arr, _P),
                                      _dev_ptr(out_dev, int(np.prod(self.out_shape()))), workspace.data_ptr(),
                                      workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_eval_stacked")

    def eval_host(self, evk_eval, cts_host: np.ndarray, pts_host: list, out_host: np.ndarray, workspace,
                  stream=None):
        """Host inputs and outputs (numpy uint32, ideally page-locked); synchronous."""
        for a in [cts_host, out_host, *pts_host]:
            assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
        assert out_host.shape == self.out_shape()
        arr = (_P * max(1, len(pts_host)))(*[p.ctypes.data for p in pts_host])
        _check(lib().bcn_eval_host(self._h, _dev_ptr(evk_eval, self.ctx.evk_words()), cts_host.ctypes.data,
                                   ctypes.cast(arr, _P), out_host.ctypes.data, workspace.data_ptr(),
                                   workspace.numel() * workspace.element_size(), _stream(stream)), "bcn_eval_host")

    def eval_host_async(self, evk_eval, cts_host: np.ndarray, pts_host: list, out_host: np.ndarray, workspace,
                        stream=None):
        """eval_host without the final synchronisation: out_host is ready once
        `stream` has passed this call; the host buffers must stay alive until then."""
        for a in [cts_host, out_host, *pts_host]:
            assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
        assert out_host.shape == self.out_shape()
        arr = (_P * max(1, len(pts_host)))(*[p.ctypes.data for p in pts_host])
        _check(lib().bcn_eval_host_async(self._h, _dev_ptr(evk_eval, self.ctx.evk_words()), cts_host.ctypes.data,
                                         ctypes.cast(arr, _P), out_host.ctypes.data, workspace.data_ptr(),
                                         workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_eval_host_async")

    def eval_host_seeded_async(self, evk_eval, c0_host: np.ndarray, seed: int, pts_host: list, out_host: np.ndarray,
                               workspace, stream=None):
        """bcn_eval_host_seeded_async: eval_host_async from c0 alone [n_in][L][N]
        and the encryption seed (c1 drawn on the device)."""
        for a in [c0_host, out_host, *pts_host]:
            assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
        assert out_host.shape == self.out_shape()
        arr = (_P * max(1, len(pts_host)))(*[p.ctypes.data for p in pts_host])
        _check(lib().bcn_eval_host_seeded_async(self._h, _dev_ptr(evk_eval, self.ctx.evk_words()), c0_host.ctypes.data,
                                                seed, ctypes.cast(arr, _P), out_host.ctypes.data, workspace.data_ptr(),
                                                workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_eval_host_seeded_async")

    def eval_host_compact_async(self, evk_eval, c0_host: np.ndarray, seed: int, feats_i64: list, out_host: np.ndarray,
                                workspace, stream=None):
        """bcn_eval_host_compact_async: from c0, the encryption seed and the
        features' integer coefficients (bcn_encode_i64, [n_out][N] int64 each)."""
        for a in [c0_host, out_host]:
            assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
        for f in feats_i64:
            assert f.dtype == np.int64 and f.flags["C_CONTIGUOUS"]
        assert out_host.shape == self.out_shape()
        arr = (_P * max(1, len(feats_i64)))(*[f.ctypes.data for f in feats_i64])
        _check(lib().bcn_eval_host_compact_async(self._h, _dev_ptr(evk_eval, self.ctx.evk_words()), c0_host.ctypes.data,
                                                 seed, ctypes.cast(arr, _P), out_host.ctypes.data, workspace.data_ptr(),
                                                 workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_eval_host_compact_async")


class Batch:
    """bcn_batch: many evaluations replayed as one CUDA graph over `lanes` streams.

    items: list of (model, evk_eval, cts_dev, [pts_dev...], out_dev)."""

    def __init__(self, items, lanes: int, workspace=None):
        self._keep = items
        n = len(items)
        arr = (_BatchItem * n)()
        self._pts_arrays = []
        for a, (model, evk, cts, pts, out) in zip(arr, items):
            pa = (_P * max(1, len(pts)))(*[_dev_ptr(p) for p in pts])
            self._pts_arrays.append(pa)
            a.model = model._h
            a.evk_eval = _dev_ptr(evk, model.ctx.evk_words())
            a.cts = _dev_ptr(cts, model.n_in * 2 * model.ctx.L * model.ctx.N)
            a.pts = ctypes.cast(pa, _P)
            a.out = _dev_ptr(out, int(np.prod(model.out_shape())))
        self._arr = arr
        self.workspace_bytes = Batch.plan(arr, n, lanes)
        if workspace is None:
            import torch

            dev = items[0][0].ctx.device
            workspace = torch.empty(max(1, (self.workspace_bytes + 3) // 4), dtype=torch.int32, device=f"cuda:{dev}")
        self.workspace = workspace
        h = _P()
        _check(lib().bcn_batch_create(ctypes.cast(arr, _P), n, lanes, workspace.data_ptr(),
                                      workspace.numel() * workspace.element_size(), ctypes.byref(h)),
               "bcn_batch_create")
        self._h = h
        lanes_of = np.zeros(n, dtype=np.int32)
        _check(lib().bcn_batch_lanes(self._h, _np_ptr(lanes_of, np.int32)), "bcn_batch_lanes")
        self.lane_of_item = lanes_of.tolist()

    @staticmethod
    def plan(arr, n, lanes) -> int:
        b = _SZ()
        _check(lib().bcn_batch_plan(ctypes.cast(arr, _P), n, lanes, ctypes.byref(b)), "bcn_batch_plan")
        return b.value

    @staticmethod
    def plan_items(items, lanes: int) -> int:
        arr = (_BatchItem * len(items))()
        for a, (model, evk, cts, pts, out) in zip(arr, items):
            a.model = model._h
            a.evk_eval, a.cts, a.out = _dev_ptr(evk), _dev_ptr(cts), _dev_ptr(out)
        return Batch.plan(arr, len(items), lanes)

    def launch(self, stream=None):
        _check(lib().bcn_batch_launch(self._h, _stream(stream)), "bcn_batch_launch")

    def close(self):
        if getattr(self, "_h", None):
            lib().bcn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def model_cost(model: "Model") -> float:
    c = _D()
    _check(lib().bcn_model_cost(model._h, ctypes.byref(c)), "bcn_model_cost")
    return c.value


PLAIN_OPS = {"conv": 0, "avgpool2": 1, "tap_crop_crot": 2, "tap_fc": 3, "tap_integrate": 4}


class PlainModel:
    """bcn_plain_model: the fp32 plaintext branch with its feature taps."""

    def __init__(self, ctx: Context, stages: list, weights: list, image_hwc, seg):
        self.ctx = ctx
        # a stage's weights: one array, or a tuple of arrays laid out back to back
        self._keep = [None if w is None else np.ascontiguousarray(
            np.concatenate([np.ravel(a) for a in w]) if isinstance(w, tuple) else w, dtype=np.float32)
            for w in weights]
        arr = (_PlainStage * len(stages))()
        for i, (s, w) in enumerate(zip(stages, self._keep)):
            a = arr[i]
            a.op = PLAIN_OPS[s["op"]]
            for f in ("cin", "cout", "k", "stride", "pad", "hc", "wc", "ch_c", "n_out", "n_hidden"):
                setattr(a, f, int(s.get(f, 0)))
            a.bias = int(bool(s.get("bias", False)))
            a.relu = int(bool(s.get("relu", False)))
            a.weights = None if w is None else w.ctypes.data
        H, W, C = image_hwc
        seg_a = np.ascontiguousarray(seg, dtype=np.int32)
        h = _P()
        _check(lib().bcn_plain_model_create(ctx.handle, ctypes.cast(arr, _P), len(stages), H, W, C,
                                            _np_ptr(seg_a, np.int32), ctypes.byref(h)), "bcn_plain_model_create")
        self._h = h
        n = _I()
        _check(lib().bcn_plain_feature_count(self._h, ctypes.byref(n)), "bcn_plain_feature_count")
        self.n_feat = n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().bcn_plain_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, B: int) -> int:
        b = _SZ()
        _check(lib().bcn_plain_workspace_bytes(self._h, B, ctypes.byref(b)), "bcn_plain_workspace_bytes")
        return b.value

    def forward(self, images_dev, noise_dev, feats_dev, workspace, stream=None):
        B = images_dev.shape[0]
        _check(lib().bcn_plain_branch_forward(self._h, images_dev.data_ptr(), noise_dev.data_ptr(), B,
                                              feats_dev.data_ptr(), workspace.data_ptr(),
                                              workspace.numel() * workspace.element_size(), _stream(stream)),
               "bcn_plain_branch_forward")
