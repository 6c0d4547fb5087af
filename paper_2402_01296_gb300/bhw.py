"""BHW packing and packed convolutions (App. D of the paper).

BHW packing puts one channel of n images' h x w segments into one ciphertext:
image b's pixel (y, x) in slot b*h*w + y*w + x (c ciphertexts for c channels).
A k x k convolution (stride 1) is then a sum of rotated copies of the input
ciphertexts weighted by the kernel's integer weights:
    out[co] = sum_{ci, i, j} w[co][ci][i][j] * Rot(in[ci], i*w + j),
which puts output (y, x) of every image into the input's slot of (y, x); the
slots with y > h - k or x > w - k receive neighbouring values and are zeroed
by an optional mask (a 0/1 plaintext multiplied in, then a rescale).  Every
step runs in the library's kernels: the rotations (automorphism + key switch
with the Galois key of each offset), the integer-weight MAC and the mask
product; this module only lays out the slots and sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import bcn


def pack(x: np.ndarray, N: int) -> np.ndarray:
    """x [n_img][C][h][w] -> slot vectors [C][N/2] (zeros past n*h*w)."""
    n, C, h, w = x.shape
    if n * h * w > N // 2:
        raise ValueError("the segments do not fit the N/2 slots")
    out = np.zeros((C, N // 2))
    out[:, :n * h * w] = x.transpose(1, 0, 2, 3).reshape(C, -1)
    return out


def unpack(z: np.ndarray, n: int, h: int, w: int) -> np.ndarray:
    """slot vectors [C][N/2] -> [n][C][h][w]."""
    C = z.shape[0]
    return z[:, :n * h * w].reshape(C, n, h, w).transpose(1, 0, 2, 3)


def valid_mask(n: int, h: int, w: int, k: int, N: int) -> np.ndarray:
    """1 in the slots of outputs (y <= h - k, x <= w - k) of the n images, else 0."""
    m = np.zeros((n, 1, h, w))
    m[:, :, :h - k + 1, :w - k + 1] = 1.0
    return pack(m, N)[0]


def rotation_steps(k: int, w: int) -> list:
    """The rotation offsets a k x k kernel needs over rows of width w (0 excluded)."""
    return [i * w + j for i in range(k) for j in range(k) if i * w + j]


class ConvBHW:
    """One k x k, stride-1 convolution of BHW-packed ciphertexts on the device.

    w_int: int8 [cout][cin][k][k]; gks: {steps: prepared Galois key} for every
    offset of rotation_steps(k, w)."""

    def __init__(self, ctx: bcn.Context, w_int: np.ndarray, w: int, gks: dict):
        import torch

        self.ctx, self.w = ctx, w
        self.cout, self.cin, self.k, _ = w_int.shape
        self.gks = gks
        kk = self.cin * self.k * self.k
        dev = f"cuda:{ctx.device}"
        self.idx = torch.from_numpy(np.tile(np.arange(kk, dtype=np.int32), (self.cout, 1))).to(dev)
        self.wt = torch.from_numpy(np.ascontiguousarray(w_int.reshape(self.cout, kk), dtype=np.int8)).to(dev)
        missing = [r for r in rotation_steps(self.k, w) if r not in gks]
        if missing:
            raise ValueError(f"no Galois key for rotations {missing}")

    def __call__(self, level: int, cts, out, stream=None):
        """cts [cin][2][level][N] -> out [cout][2][level][N] (device tensors)."""
        import torch

        N, kk = self.ctx.N, self.k * self.k
        rot = torch.empty((self.cin * kk, 2, level, N), dtype=torch.int32, device=cts.device)
        for ci in range(self.cin):
            for i in range(self.k):
                for j in range(self.k):
                    r, slot = i * self.w + j, ci * kk + i * self.k + j
                    if r == 0:
                        rot[slot].copy_(cts[ci])
                    else:
                        self.ctx.op_rotate(level, self.gks[r], r, cts[ci:ci + 1], 1, rot[slot:slot + 1], stream)
        self.ctx.op_mac(level, self.cin * kk, self.idx, self.wt, rot, None, out, stream)
        return out
