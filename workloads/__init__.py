"""Seeded synthetic workloads shared by the CUDA path's tests/benchmark and the oracle.

This module holds only shapes, sizes and seeded random draws: no step of the
method's arithmetic lives here.  It stands in for MNIST (28x28x1) and CIFAR-10
(32x32x3), which the paper uses (Sec. 5, App. B) and which are not available:
images are uniform uint8 with those shapes, float weights are N(0, 0.1), and the
insensitive segment's perturbation noise is Laplace(b = 0.1) on [0,1]-scaled
pixels (the paper perturbs the insensitive segment with noise, Sec. 3 and
Sec. 5).  Seeds: images 1, weights 2, keys 3, encryption 4, noise 5.

Network shapes:
  * "cnn3_small"  -- the small MNIST-shaped case (N = 4096, 3 data primes).
  * "cryptonets"  -- the CryptoNets-scale MNIST case (N = 8192, 7 data primes).
  * "cifar_cnn"   -- the CIFAR-shaped case (N = 16384, 11 data primes).
The ciphertext branch of each is a sequence of linear layers (conv / dense with
integer weights), each optionally followed by the unidirectional add of a
plaintext-branch feature and a square activation (Sec. 3.2, App. B).
"""
from __future__ import annotations

import copy
import numpy as np

SEED_IMAGES, SEED_WEIGHTS, SEED_KEYS, SEED_ENC, SEED_NOISE = 1, 2, 3, 4, 5

# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------
# cipher layers:  conv: cin,h,w (input map), cout, k, stride, pad
#                 dense: n_in, n_out
#                 add: a plaintext-branch feature is added to the layer output
#                 square: square activation (then relinearise + rescale)
# plain branch:   list of stages; "tap" entries produce the features, in the
#                 order of the cipher layers that have add=True.
CONFIGS = {
    "cnn3_small": dict(
        name="cnn3_small",
        log_n=12, n_data=3, n_special=1, alpha=1, log_scale=25.0,
        image=(28, 28, 1), batch=2048, segment=(8, 8, 12, 12),
        cipher=[
            dict(type="conv", cin=1, h=12, w=12, cout=5, k=5, stride=2, pad=0, add=True, square=True),
            dict(type="dense", n_in=80, n_out=10, add=False, square=False),
        ],
        plain=[
            dict(op="conv", cin=1, cout=4, k=3, stride=1, pad=1, relu=False),
            dict(op="avgpool2"),
            dict(op="tap_crop_crot", hc=4, wc=4, ch_c=5),
        ],
    ),
    "cryptonets": dict(
        name="cryptonets",
        log_n=13, n_data=7, n_special=1, alpha=1, log_scale=30.0,
        image=(28, 28, 1), batch=4096, segment=(6, 6, 16, 16),
        cipher=[
            dict(type="conv", cin=1, h=16, w=16, cout=5, k=5, stride=2, pad=0, add=True, square=True),
            dict(type="dense", n_in=180, n_out=100, add=True, square=True),
            dict(type="dense", n_in=100, n_out=10, add=False, square=False),
        ],
        plain=[
            dict(op="conv", cin=1, cout=4, k=3, stride=1, pad=1, relu=False),
            dict(op="avgpool2"),
            dict(op="tap_crop_crot", hc=6, wc=6, ch_c=5),
            dict(op="tap_fc", n_out=100),
        ],
    ),
    # The CryptoNets-scale network with the two-layer feature integration of
    # Sec. 3.3 as its head: the ciphertext neurons of integration layer 1 are
    # a dense layer on the ciphertext branch plus W_p1 x_p + b_1 from the
    # plaintext branch (a tap), squared; integration layer 2 is a dense layer
    # on them plus W_p2 x_p^<1> + b_2, the plaintext neurons' contribution
    # (a tap).  n_1 = 100 (50 + 50 neurons), n_2 = 10.
    "cryptonets_fi": dict(
        name="cryptonets_fi",
        log_n=13, n_data=7, n_special=1, alpha=1, log_scale=30.0,
        image=(28, 28, 1), batch=4096, segment=(6, 6, 16, 16),
        cipher=[
            dict(type="conv", cin=1, h=16, w=16, cout=5, k=5, stride=2, pad=0, add=True, square=True),
            dict(type="dense", n_in=180, n_out=50, add=True, square=True),
            dict(type="dense", n_in=50, n_out=10, add=True, square=False),
        ],
        plain=[
            dict(op="conv", cin=1, cout=4, k=3, stride=1, pad=1, relu=False),
            dict(op="avgpool2"),
            dict(op="tap_crop_crot", hc=6, wc=6, ch_c=5),
            dict(op="tap_fc", n_out=50, bias=True),
            dict(op="tap_integrate", n_hidden=50, n_out=10),
        ],
    ),
    "cifar_cnn": dict(
        name="cifar_cnn",
        log_n=14, n_data=11, n_special=2, alpha=2, log_scale=30.0,
        image=(32, 32, 3), batch=8192, segment=(8, 8, 16, 16),
        cipher=[
            dict(type="conv", cin=3, h=16, w=16, cout=16, k=3, stride=1, pad=1, add=True, square=True),
            dict(type="conv", cin=16, h=16, w=16, cout=32, k=3, stride=2, pad=1, add=True, square=True),
            dict(type="dense", n_in=2048, n_out=10, add=False, square=False),
        ],
        plain=[
            dict(op="conv", cin=3, cout=16, k=3, stride=1, pad=1, relu=True),
            dict(op="tap_crop_crot", hc=16, wc=16, ch_c=16),
            dict(op="conv", cin=16, cout=32, k=3, stride=2, pad=1, relu=True),
            dict(op="tap_crop_crot", hc=8, wc=8, ch_c=32),
        ],
    ),
}


def get_config(name: str) -> dict:
    return copy.deepcopy(CONFIGS[name])


def reduced_cifar(cout1: int = 4, cout2: int = 4, seg: int = 8, batch: int = 64) -> dict:
    """CIFAR-shaped case with the full ring and prime chain (N = 16384, 11 data
    primes, 2 special primes) but a smaller segment and fewer maps, so the oracle
    finishes in seconds.  Still two adds, two squares and the dense output."""
    c = get_config("cifar_cnn")
    y0 = (32 - seg) // 2
    c["name"] = f"cifar_cnn_reduced_{cout1}_{cout2}_{seg}"
    c["batch"] = batch
    c["segment"] = (y0, y0, seg, seg)
    h2 = (seg + 2 - 3) // 2 + 1
    c["cipher"] = [
        dict(type="conv", cin=3, h=seg, w=seg, cout=cout1, k=3, stride=1, pad=1, add=True, square=True),
        dict(type="conv", cin=cout1, h=seg, w=seg, cout=cout2, k=3, stride=2, pad=1, add=True, square=True),
        dict(type="dense", n_in=cout2 * h2 * h2, n_out=10, add=False, square=False),
    ]
    c["plain"] = [
        dict(op="conv", cin=3, cout=16, k=3, stride=1, pad=1, relu=True),
        dict(op="tap_crop_crot", hc=seg, wc=seg, ch_c=cout1),
        dict(op="conv", cin=16, cout=32, k=3, stride=2, pad=1, relu=True),
        dict(op="tap_crop_crot", hc=h2, wc=h2, ch_c=cout2),
    ]
    return c


def with_batch(cfg: dict, batch: int) -> dict:
    c = copy.deepcopy(cfg)
    c["batch"] = batch
    return c


# ---------------------------------------------------------------------------
# shape helpers (pure bookkeeping)
# ---------------------------------------------------------------------------
def conv_out_hw(h: int, w: int, k: int, stride: int, pad: int):
    return (h + 2 * pad - k) // stride + 1, (w + 2 * pad - k) // stride + 1


def cipher_layer_io(layer: dict):
    """(n_in, n_out) ciphertext counts of a cipher layer."""
    if layer["type"] == "conv":
        ho, wo = conv_out_hw(layer["h"], layer["w"], layer["k"], layer["stride"], layer["pad"])
        return layer["cin"] * layer["h"] * layer["w"], layer["cout"] * ho * wo
    return layer["n_in"], layer["n_out"]


def cipher_weight_shape(layer: dict):
    if layer["type"] == "conv":
        return (layer["cout"], layer["cin"], layer["k"], layer["k"])
    return (layer["n_out"], layer["n_in"])


def n_input_cts(cfg: dict) -> int:
    y0, x0, h, w = cfg["segment"]
    return cfg["image"][2] * h * w


def plain_shapes(cfg: dict):
    """Walk the plain branch; return a list of (stage, (C, H, W) before the stage)."""
    H, W, C = cfg["image"]
    shapes = []
    for st in cfg["plain"]:
        shapes.append((st, (C, H, W)))
        if st["op"] == "conv":
            H, W = conv_out_hw(H, W, st["k"], st["stride"], st["pad"])
            C = st["cout"]
        elif st["op"] == "avgpool2":
            H, W = H // 2, W // 2
    return shapes


def level_schedule(cfg: dict):
    """Live data primes at each cipher layer (only squares consume a level)."""
    lv = cfg["n_data"]
    out = []
    for layer in cfg["cipher"]:
        out.append(lv)
        if layer["square"]:
            lv -= 1
    return out, lv


# ---------------------------------------------------------------------------
# seeded draws (the random numbers passed to the method as inputs)
# ---------------------------------------------------------------------------
def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def images(cfg: dict, seed: int = SEED_IMAGES) -> np.ndarray:
    """uint8 images [B][H][W][C], uniform."""
    H, W, C = cfg["image"]
    return _rng(seed, 0).integers(0, 256, size=(cfg["batch"], H, W, C), dtype=np.uint8)


def laplace_noise(cfg: dict, b: float = 0.1, seed: int = SEED_NOISE) -> np.ndarray:
    """float32 Laplace(b) noise [B][H][W][C] by inverse CDF from 53-bit uniforms."""
    H, W, C = cfg["image"]
    u = _rng(seed, 0).random(size=(cfg["batch"], H, W, C)) - 0.5  # [-0.5, 0.5)
    u = np.where(u == -0.5, 0.0, u)
    return (-b * np.sign(u) * np.log1p(-2.0 * np.abs(u))).astype(np.float32)


def cipher_weights(cfg: dict, seed: int = SEED_WEIGHTS):
    """float32 N(0, 0.1) weights for every cipher layer (PyTorch layouts)."""
    return [(_rng(seed, 1, i).standard_normal(cipher_weight_shape(l)) * 0.1).astype(np.float32)
            for i, l in enumerate(cfg["cipher"])]


def plain_weights(cfg: dict, seed: int = SEED_WEIGHTS):
    """float32 N(0, 0.1) weights (and biases) for every plain-branch stage that
    has any: conv [cout][cin][k][k]; tap_crop_crot CRot [ch_c][ch_p]; tap_fc
    [n_out][C*H*W], or the tuple (W, b) with bias; tap_integrate the tuple
    (W'_1 [n_hidden][C*H*W], b'_1 [n_hidden], W_2 [n_out][n_hidden], b_2 [n_out])."""
    out = []
    for i, (st, (C, H, W)) in enumerate(plain_shapes(cfg)):
        g = _rng(seed, 2, i)
        nrm = lambda *shape: (g.standard_normal(shape) * 0.1).astype(np.float32)  # noqa: E731
        if st["op"] == "conv":
            out.append(nrm(st["cout"], st["cin"], st["k"], st["k"]))
        elif st["op"] == "tap_crop_crot":
            out.append(nrm(st["ch_c"], C))
        elif st["op"] == "tap_fc":
            w = nrm(st["n_out"], C * H * W)
            out.append((w, nrm(st["n_out"])) if st.get("bias") else w)
        elif st["op"] == "tap_integrate":
            nh, no = st["n_hidden"], st["n_out"]
            out.append((nrm(nh, C * H * W), nrm(nh), nrm(no, nh), nrm(no)))
        else:
            out.append(None)
    return out


def random_residues(primes, shape_before_limb, n: int, seed: int):
    """Uniform residues [..., len(primes), n] (uint32), limb i below primes[i]."""
    g = _rng(seed, 7)
    q = np.asarray(primes, dtype=np.uint64).reshape((1,) * len(shape_before_limb) + (len(primes), 1))
    r = g.integers(0, 2**62, size=tuple(shape_before_limb) + (len(primes), n), dtype=np.uint64)
    return (r % q).astype(np.uint32)


# ---------------------------------------------------------------------------
# the batched uneven workload: many evaluations of different ring degrees,
# segment sizes and slot occupancies
# ---------------------------------------------------------------------------
_BY_N = {12: "cnn3_small", 13: "cryptonets", 14: "cifar_cnn"}


def segment_network(base: dict, h: int, w: int) -> dict:
    """The network of `base` on a centred h x w sensitive segment: the same
    layers, with the first conv reading h x w and every later layer sized to
    follow; plaintext-branch crops follow the ciphertext-branch maps."""
    cfg = copy.deepcopy(base)
    H, W, C = cfg["image"]
    cfg["segment"] = ((H - h) // 2, (W - w) // 2, h, w)
    ch, hh, ww = C, h, w
    cipher = []
    for layer in cfg["cipher"]:
        layer = dict(layer)
        if layer["type"] == "conv":
            layer.update(cin=ch, h=hh, w=ww)
            hh, ww = conv_out_hw(hh, ww, layer["k"], layer["stride"], layer["pad"])
            ch = layer["cout"]
        else:
            layer["n_in"] = ch * hh * ww
            ch, hh, ww = layer["n_out"], 1, 1
        cipher.append(layer)
    cfg["cipher"] = cipher
    return cfg


def uneven_batch(n_eval: int = 64, seed: int = 11, log_ns=(12, 13, 14)):
    """Seeded list of evaluations: ring degree uniform over `log_ns` (with the
    matching parameter set and network), sensitive fraction f uniform in
    [0.10, 0.60] of the pixels as a centred h x w block (h = round(sqrt(f H W)),
    w = round(f H W / h), at least the first kernel size), slot occupancy
    uniform in [0.25, 1.0] of the N/2 slots.  Returns a list of configs with
    "occupancy" (images counted) added."""
    g = _rng(seed, 3)
    out = []
    for i in range(n_eval):
        base = get_config(_BY_N[int(log_ns[g.integers(0, len(log_ns))])])
        H, W, C = base["image"]
        f = g.uniform(0.10, 0.60)
        k = base["cipher"][0]["k"]
        h = max(k, min(H, int(round(np.sqrt(f * H * W)))))
        w = max(k, min(W, int(round(f * H * W / h))))
        cfg = segment_network(base, h, w)
        cfg["name"] = f"{base['name']}_{h}x{w}_{i}"
        slots = 1 << (cfg["log_n"] - 1)
        cfg["batch"] = max(1, int(round(g.uniform(0.25, 1.0) * slots)))
        out.append(cfg)
    return out
