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


def fc_layout_at(W: np.ndarray, n_img: int, block: int, s_in, o_out, N: int):
    """The diagonal method's slot vectors for inputs at slots s_in and outputs
    at slots o_out of each image block (App. D's dense layer after a strided
    packed convolution, whose outputs sit at every s-th slot): the term
    W[j][p] needs the rotation r = s_in[p] - o_out[j] and sits in slot
    b*block + o_out[j] of u_r.  Returns (steps ascending, diagonals
    [len(steps)][N/2]); slots that are no s_in[p] meet only zeros, which drops
    what the convolution's mask would."""
    W = np.asarray(W)
    s_in, o_out = np.asarray(s_in, dtype=np.int64), np.asarray(o_out, dtype=np.int64)
    n2, n1 = W.shape
    if len(s_in) != n1 or len(o_out) != n2:
        raise ValueError("one slot per input and per output")
    if min(s_in.min(), o_out.min()) < 0 or max(s_in.max(), o_out.max()) >= block or n_img * block > N // 2:
        raise ValueError("slots must lie inside the image blocks, and the blocks inside the N/2 slots")
    r = s_in[None, :] - o_out[:, None]  # [n2][n1]
    steps = sorted(set(int(v) for v in r.ravel()))
    at = {v: i for i, v in enumerate(steps)}
    rows = np.zeros((len(steps), block))
    ri = np.vectorize(at.get)(r)
    rows[ri, np.broadcast_to(o_out[:, None], r.shape)] = W
    diags = np.zeros((len(steps), N // 2))
    diags[:, :n_img * block] = np.tile(rows, (1, n_img))
    return steps, diags


class BranchBHW:
    """A ciphertext branch of one valid convolution followed by dense layers
    (the CryptoNets-scale networks), evaluated in BHW packing (App. D) on the
    device, n_img images per ciphertext group.

    layers: the branch's layer dicts (conv: cin, h, w, cout, k, stride, pad = 0;
    dense: n_in, n_out; each with add and square); weights: integer weights
    per layer (conv [cout][cin][k][k] int8, dense [n_out][n_in]); gks:
    {steps mod N/2: prepared Galois key} for every step of
    rotation_steps_needed(); evk_eval: the prepared relinearisation key.
    diag_pts: optional per dense layer [C][n_rot][level][N] coefficient-form
    encodings of fc_layout_at's diagonals (default: the library's encoder at
    scale q_{level-1}).

    Per group: the conv's rotations with one hoisted ModUp (bcn_op_rotate_many)
    and the integer MAC with the feature added in its epilogue; the square
    (relinearise, rescale); each dense layer as bcn_op_fc_diag_sum over the
    previous layer's ciphertexts with its feature added; the squares."""

    def __init__(self, ctx: bcn.Context, layers: list, weights: list, n_img: int, gks: dict, evk_eval,
                 diag_pts: list | None = None):
        import torch

        conv = layers[0]
        if conv["type"] != "conv" or conv["pad"] != 0 or any(l["type"] != "dense" for l in layers[1:]):
            raise ValueError("one valid convolution, then dense layers")
        self.ctx, self.layers, self.n_img, self.gks, self.evk = ctx, layers, n_img, gks, evk_eval
        self.h, self.w = conv["h"], conv["w"]
        self.block = self.h * self.w
        if n_img * self.block > ctx.N // 2:
            raise ValueError("the segments do not fit the N/2 slots")
        dev = f"cuda:{ctx.device}"
        self.dev = dev
        k, s = conv["k"], conv["stride"]
        self.cin, self.cout, self.kk = conv["cin"], conv["cout"], k * k
        self.conv_steps = [i * self.w + j for i in range(k) for j in range(k)]
        self.conv_w = np.ascontiguousarray(np.asarray(weights[0]).reshape(self.cout, -1), dtype=np.int8)
        ho, wo = (self.h - k) // s + 1, (self.w - k) // s + 1
        pos = [s * (y * self.w + x) for y in range(ho) for x in range(wo)]
        level = ctx.L - (1 if conv["square"] else 0)
        self.levels = [ctx.L]
        self.dense = []
        C = self.cout
        for li, lay in enumerate(layers[1:]):
            W = np.asarray(weights[li + 1])
            n_pos = len(pos)
            if W.shape != (lay["n_out"], C * n_pos):
                raise ValueError(f"dense layer {li + 1}: weights {W.shape}, expected {(lay['n_out'], C * n_pos)}")
            lays = [fc_layout_at(W[:, c * n_pos:(c + 1) * n_pos], n_img, self.block, pos,
                                 list(range(lay["n_out"])), ctx.N) for c in range(C)]
            steps = lays[0][0]
            if any(st != steps for st, _ in lays):
                raise ValueError("every channel's positions must give the same rotations")
            if diag_pts is not None:
                pts = np.ascontiguousarray(diag_pts[li], dtype=np.uint32)
            else:
                d = np.concatenate([dg for _, dg in lays])
                pts = ctx.encode(d, level, float(ctx.q[level - 1]))
            pts = pts.reshape(C * len(steps), level, ctx.N)
            t = bcn.to_device(pts, dev)
            ctx.op_ntt(t, C * len(steps), level, inverse=False)
            self.dense.append(dict(steps=steps, diag=t, n_in=C, level=level, add=lay["add"], square=lay["square"],
                                   ws=ctx.fc_diag_workspace(level, len(steps))))
            self.levels.append(level)
            level -= 1 + (1 if lay["square"] else 0)
            C, pos = 1, list(range(lay["n_out"]))
        self.out_level = level
        half = ctx.N // 2
        missing = [r for r in self.rotation_steps_needed() if r % half not in gks and r not in gks]
        if missing:
            raise ValueError(f"no Galois key for rotations {missing[:8]}")
        self._mac_cache = {}

    def rotation_steps_needed(self) -> list:
        """Every nonzero rotation (mod N/2) the branch uses."""
        half = self.ctx.N // 2
        st = set(r % half for r in self.conv_steps)
        for d in self.dense:
            st |= set(r % half for r in d["steps"])
        return sorted(st - {0})

    @staticmethod
    def steps_for(layers: list, n_img: int, N: int) -> list:
        """rotation_steps_needed() of a branch with these layers, before its keys exist."""
        conv = layers[0]
        k, s, w = conv["k"], conv["stride"], conv["w"]
        half = N // 2
        st = {i * w + j for i in range(k) for j in range(k)}
        ho, wo = (conv["h"] - k) // s + 1, (w - k) // s + 1
        pos = [s * (y * w + x) for y in range(ho) for x in range(wo)]
        for lay in layers[1:]:
            st |= {p - j for p in pos for j in range(lay["n_out"])}
            pos = list(range(lay["n_out"]))
        return sorted(set(r % half for r in st) - {0})

    def feature_shapes(self, n_groups: int) -> list:
        """Shapes of the encoded features the layers with add=True take, in order."""
        out = []
        if self.layers[0]["add"]:
            out.append((n_groups, self.cout, self.ctx.L, self.ctx.N))
        for d in self.dense:
            if d["add"]:
                out.append((n_groups, d["level"] - 1, self.ctx.N))
        return out

    def _mac_tables(self, G: int):
        import torch

        if G not in self._mac_cache:
            kk = self.cin * self.kk
            idx = (np.arange(G)[:, None, None] * kk + np.arange(kk)[None, None, :]).repeat(self.cout, axis=1)
            self._mac_cache[G] = (torch.from_numpy(idx.reshape(G * self.cout, kk).astype(np.int32)).to(self.dev),
                                  torch.from_numpy(np.tile(self.conv_w, (G, 1))).to(self.dev))
        return self._mac_cache[G]

    def __call__(self, cts, n_groups: int, feats: list, out, stream=None):
        """cts [n_groups][cin][2][L][N] -> out [n_groups][2][out_level][N] (device
        tensors); feats: device tensors of feature_shapes(n_groups)."""
        import torch

        c, G, N, L = self.ctx, n_groups, self.ctx.N, self.ctx.L
        fi = 0
        kk = self.cin * self.kk
        rot = torch.empty((G * self.cin, self.kk, 2, L, N), dtype=torch.int32, device=self.dev)
        c.op_rotate_many(L, self.gks, self.conv_steps, cts, G * self.cin, rot, stream=stream)
        idx, wt = self._mac_tables(G)
        y = torch.empty((G * self.cout, 2, L, N), dtype=torch.int32, device=self.dev)
        pt = None
        if self.layers[0]["add"]:
            pt, fi = feats[0], 1
        c.op_mac(L, G * kk, idx, wt, rot, pt, y, stream)
        del rot
        level = L
        if self.layers[0]["square"]:
            z = torch.empty((G * self.cout, 2, level - 1, N), dtype=torch.int32, device=self.dev)
            c.op_square_relin_rescale(level, self.evk, y, G * self.cout, z, stream)
            y, level = z, level - 1
        for i, d in enumerate(self.dense):
            last = i == len(self.dense) - 1 and not d["square"]
            z = out if last else torch.empty((G, 2, level - 1, N), dtype=torch.int32, device=self.dev)
            pt = None
            if d["add"]:
                pt, fi = feats[fi], fi + 1
            c.op_fc_diag_sum(level, self.gks, d["steps"], d["diag"], y, d["n_in"], G, z, pt_dev=pt,
                             workspace=d["ws"], stream=stream)
            y, level = z, level - 1
            if d["square"]:
                last = i == len(self.dense) - 1
                z = out if last else torch.empty((G, 2, level - 1, N), dtype=torch.int32, device=self.dev)
                c.op_square_relin_rescale(level, self.evk, y, G, z, stream)
                y, level = z, level - 1
        return out
