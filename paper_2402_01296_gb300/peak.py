"""Measured integer-issue rates of the GPU (bcn_int_peak_launch).

The NTT-based kernels (square, key switch, ModDown/rescale) keep their limbs
in registers and shared memory; what bounds them is integer instruction issue,
not HBM.  Their roofline is therefore the rate of their own arithmetic with the
data in registers: the NTT core's lazy forward and inverse butterflies and the
key switch's Montgomery multiply-add, each timed here with CUDA events over a
full-occupancy launch of the library's microbenchmark kernel, beside the Shoup
multiply-add by a constant of the basis conversions.  The raw multiply-add (low
and high half) and modular-addition rates are measured for context.

A kernel class whose work is f forward butterflies, i inverse butterflies, m
Montgomery and s Shoup multiply-adds would take at least
f / r_fwd + i / r_inv + m / r_mont + s / r_shoup seconds; its algorithmic
operations (10 per butterfly, 5 per multiply-add) over that time are its peak
(`mix_peak`).
"""
from __future__ import annotations

from . import bcn

KINDS = {
    0: "imad_lo",
    1: "imad_hi",
    2: "modadd",
    3: "butterfly_fwd",
    4: "butterfly_inv",
    5: "mont_muladd",
    6: "shoup_muladd",
    7: "imad_wide",
    8: "dp4a",
}
OPS_BUTTERFLY, OPS_MULADD = 10, 5


def _launch(kind, iters, sink, stream):
    import ctypes

    units = ctypes.c_double(0.0)
    bcn._check(bcn.lib().bcn_int_peak_launch(kind, iters, sink.data_ptr(), sink.numel(), stream.cuda_stream,
                                             ctypes.byref(units)), "bcn_int_peak_launch")
    return units.value


def measure(device: int = 0, target_ms: float = 30.0, reps: int = 5) -> dict:
    """Rates of every kind in units per second (the best of `reps` launches of
    about `target_ms` each, after a calibration launch), with the grid used."""
    import ctypes

    import torch

    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream()
    out = {}
    for kind, name in KINDS.items():
        blocks = ctypes.c_int(0)
        bcn._check(bcn.lib().bcn_int_peak_grid(kind, ctypes.byref(blocks)), "bcn_int_peak_grid")
        sink = torch.zeros(blocks.value, dtype=torch.int32, device=f"cuda:{device}")
        iters = 256
        best = None
        for rep in range(reps + 2):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s.record(stream)
            units = _launch(kind, iters, sink, stream)
            e.record(stream)
            torch.cuda.synchronize()
            ms = s.elapsed_time(e)
            if rep == 0:  # calibration: scale to about target_ms per launch
                iters = max(16, min(1 << 24, int(iters * target_ms / max(ms, 1e-3))))
                continue
            if rep == 1:  # warm-up at the final size
                continue
            rate = units / (ms / 1e3)
            if best is None or rate > best[0]:
                best = (rate, ms, iters)
        out[name] = {"units_per_s": best[0], "ms": best[1], "iters": best[2], "blocks": blocks.value,
                     "threads": 256}
    return out


def mix_peak(rates: dict, fwd: float, inv: float, mont: float, shoup: float) -> float:
    """Algorithmic integer operations per second of a kernel whose work is
    `fwd` forward and `inv` inverse butterflies, `mont` products of two
    variables (Montgomery) and `shoup` products by constants (Shoup), each a
    multiply-add, at the measured register-resident rates."""
    t = (fwd / rates["butterfly_fwd"]["units_per_s"] + inv / rates["butterfly_inv"]["units_per_s"]
         + mont / rates["mont_muladd"]["units_per_s"] + shoup / rates["shoup_muladd"]["units_per_s"])
    ops = OPS_BUTTERFLY * (fwd + inv) + OPS_MULADD * (mont + shoup)
    return ops / t if t > 0 else 0.0
