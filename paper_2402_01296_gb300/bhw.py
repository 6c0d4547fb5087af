"""BHW packing and the rotation-based layers of App. D of the paper.

BHW packing puts one channel of n images' h x w segments into one ciphertext:
image b's pixel (y, x) in slot b*h*w + y*w + x (c ciphertexts for c channels).

* Convolution (App. D, homomorphic convolutional layer): a k x k convolution
  is a sum of rotated copies of the input ciphertexts weighted by the kernel's
  integer weights,
      out[co] = sum_{ci, i, j} w[co][ci][i][j] * Rot(in[ci], gap * (i*w + j)),
  which puts output (y, x) of every image into the input's slot of (y, x).
  `gap` is the slot distance of neighbouring pixels of the input map: 1 for
  the segment itself, s after a stride-s layer.  All rotations of one input
  ciphertext share one ModUp (bcn_op_rotate_many).
* Strided convolution: the same sum, then a 0/1 mask (a plaintext product and
  a rescale) keeps the outputs at every s-th position; they stay where they
  are, so the next layer reads them at gap g*s.
* Fully connected layer (App. D, homomorphic fully connected layer) by the
  diagonal method: with image b's input vector in slots [b B, b B + n1),
      y = sum_r u_r * Rot(x, r),   u_r[b B + j] = W[j][j + r],
  over the rotations r = i - j, then one rescale (the diagonals are encoded at
  the scale of the prime the rescale drops).  One ModUp for all rotations; the
  products are summed in the NTT domain (bcn_op_fc_diag).

Every homomorphic step runs in the library's kernels; this module only lays
out the slots (host arithmetic on plain vectors) and sequences the calls.
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


def valid_mask(n: int, h: int, w: int, k: int, N: int, stride: int = 1, gap: int = 1) -> np.ndarray:
    """1 in the slots of the outputs a valid k x k, stride-s convolution keeps
    (logical output (y', x') of each image at slot gap*s*(y'*w + x') of its
    block, s*y' + k <= h/gap, s*x' + k <= w/gap), else 0: [N/2]."""
    hl, wl = h // gap, w // gap
    m = np.zeros((n, 1, h, w))
    for yy in range((hl - k) // stride + 1):
        for xx in range((wl - k) // stride + 1):
            m[:, 0, gap * stride * yy, gap * stride * xx] = 1.0
    return pack(m, N)[0]


def rotation_steps(k: int, w: int, gap: int = 1) -> list:
    """The rotation offsets a k x k kernel needs over rows of width w at slot
    distance `gap` (0 excluded)."""
    return [gap * (i * w + j) for i in range(k) for j in range(k) if i * w + j]


class ConvBHW:
    """One k x k convolution of BHW-packed ciphertexts on the device.

    w_int: int8 [cout][cin][k][k]; gks: {steps: prepared Galois key} for every
    offset of rotation_steps(k, w, gap)."""

    def __init__(self, ctx: bcn.Context, w_int: np.ndarray, w: int, gks: dict, gap: int = 1):
        import torch

        self.ctx, self.w, self.gap = ctx, w, gap
        self.cout, self.cin, self.k, _ = w_int.shape
        self.gks = gks
        self.steps = [gap * (i * w + j) for i in range(self.k) for j in range(self.k)]
        kk = self.cin * self.k * self.k
        dev = f"cuda:{ctx.device}"
        self.idx = torch.from_numpy(np.tile(np.arange(kk, dtype=np.int32), (self.cout, 1))).to(dev)
        self.wt = torch.from_numpy(np.ascontiguousarray(w_int.reshape(self.cout, kk), dtype=np.int8)).to(dev)
        missing = [r for r in self.steps if r and r not in gks]
        if missing:
            raise ValueError(f"no Galois key for rotations {missing}")

    def __call__(self, level: int, cts, out, stream=None):
        """cts [cin][2][level][N] -> out [cout][2][level][N] (device tensors)."""
        import torch

        N, kk = self.ctx.N, self.k * self.k
        # [cin][k*k][2][level][N]: the rotated copies in (ci, i, j) order, the MAC's tap order
        rot = torch.empty((self.cin, kk, 2, level, N), dtype=torch.int32, device=cts.device)
        self.ctx.op_rotate_many(level, self.gks, self.steps, cts, self.cin, rot, stream=stream)
        self.ctx.op_mac(level, self.cin * kk, self.idx, self.wt, rot, None, out, stream)
        return out


def fc_layout(W: np.ndarray, n_img: int, block: int, N: int):
    """The diagonal method's slot vectors for y = W x (W [n2][n1], image b's
    x in slots [b*block, b*block + n1), its y in [b*block, b*block + n2)):
    (steps, diagonals [len(steps)][N/2]) over the rotations r = i - j that
    carry a nonzero weight."""
    n2, n1 = W.shape
    if block < max(n1, n2) or n_img * block > N // 2:
        raise ValueError("image blocks must hold the input and the output and fit the slots")
    steps, diags = [], []
    jj = np.arange(n2)
    for r in range(1 - n2, n1):
        ok = (jj + r >= 0) & (jj + r < n1)
        if not ok.any():
            continue
        row = np.zeros(block)
        row[jj[ok]] = W[jj[ok], jj[ok] + r]
        if not row.any():
            continue
        u = np.zeros(N // 2)
        u[:n_img * block] = np.tile(row, n_img)
        steps.append(r)
        diags.append(u)
    return steps, np.array(diags)


class FcDiag:
    """Dense layer y = W x by the diagonal method on the device.

    W: integer weights [n2][n1]; gks: {r mod N/2: prepared Galois key} for
    every nonzero step of fc_layout; level: the input ciphertexts' level (the
    diagonals are encoded at the scale q_{level-1} over its primes).  diag_pts,
    when given, are the encoded diagonals [len(steps)][level][N] (coefficient
    form) to use instead of the library's encoder."""

    def __init__(self, ctx: bcn.Context, W: np.ndarray, n_img: int, block: int, level: int, gks: dict,
                 diag_pts: np.ndarray | None = None):
        self.ctx, self.level, self.gks = ctx, level, gks
        self.steps, diags = fc_layout(np.asarray(W), n_img, block, ctx.N)
        if diag_pts is None:
            diag_pts = ctx.encode(diags, level, float(ctx.q[level - 1]))
        self.diag = bcn.to_device(np.ascontiguousarray(diag_pts, dtype=np.uint32), f"cuda:{ctx.device}")
        ctx.op_ntt(self.diag, len(self.steps), level, inverse=False)
        half = ctx.N // 2
        missing = [r for r in self.steps if r % half and r % half not in gks and r not in gks]
        if missing:
            raise ValueError(f"no Galois key for rotations {missing}")

    def __call__(self, cts, n_ct: int, out, stream=None):
        """cts [n_ct][2][level][N] -> out [n_ct][2][level-1][N] (device tensors)."""
        self.ctx.op_fc_diag(self.level, self.gks, self.steps, self.diag, cts, n_ct, out, stream)
        return out
