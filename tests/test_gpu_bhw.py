"""BHW packing (App. D) on the GPU: the packed convolution (rotations by the
kernel offsets, integer-weight MAC) and the mask product (plaintext multiply
then rescale) against the oracle, bit-exact, at the CryptoNets-scale ring with
16 images' 16 x 16 segments per ciphertext and its 5 x 5 kernel."""
import numpy as np
import pytest
import torch

import workloads
from oracle import oracle as O
from paper_2402_01296_gb300 import bcn, bhw

pytestmark = pytest.mark.gpu


def test_conv_bhw_and_mask_bit_exact():
    c, P = bcn.Context(13, 7, 1, 1, device=0), O.Params(13, 7, 1, 1)
    n, cin, cout, h, w, k = 16, 1, 5, 16, 16, 5
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (n, cin, h, w))
    wi = rng.integers(-127, 128, (cout, cin, k, k)).astype(np.int8)
    sk, _ = P.keygen(3)
    S = 2.0**30
    cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), P.L, 4)
    steps = bhw.rotation_steps(k, w)
    gks = {r: P.galois_keygen(sk, r, 100 + r) for r in steps}
    ref = O.conv_bhw(P, P.L, gks, wi, cts, w)
    conv = bhw.ConvBHW(c, wi, w, {r: c.evk_prepare(bcn.to_device(g)) for r, g in gks.items()})
    out = torch.empty((cout, 2, P.L, P.N), dtype=torch.int32, device="cuda")
    conv(P.L, bcn.to_device(cts), out)
    got = bcn.to_host_u32(out)
    assert np.array_equal(got, ref)
    # the layout matches the oracle's packing, and the library's mask multiply + rescale
    assert np.array_equal(bhw.pack(x, P.N), O.pack_bhw(x, P.N))
    mask = O.encode(bhw.valid_mask(n, h, w, k, P.N)[None], P.N, float(P.q[P.L - 1]), P.q)[0]
    masked = torch.empty((cout, 2, P.L - 1, P.N), dtype=torch.int32, device="cuda")
    c.op_mul_plain_rescale(P.L, out, cout, bcn.to_device(mask), masked)
    want = P.rescale(P.L, P.mul_plain(P.L, ref, mask))
    assert np.array_equal(bcn.to_host_u32(masked), want)
    # decrypted: the convolution in the valid slots, zero elsewhere
    dec = c.decrypt_decode(sk, bcn.to_host_u32(masked), P.L - 1, S, P.N // 2)
    img = bhw.unpack(dec, n, h, w)
    conv_ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(wi.astype(np.float64))).numpy()
    # key-switching noise of 24 rotations times weights up to 127, and the mask's
    # encoding error times the neighbours' values (up to ~10^3)
    assert np.abs(img[:, :, :h - k + 1, :w - k + 1] - conv_ref).max() < 0.05
    img[:, :, :h - k + 1, :w - k + 1] = 0
    assert np.abs(img).max() < 0.1


@pytest.mark.parametrize("params,n2,n1,n_img,block", [((12, 4, 1, 1), 10, 40, 32, 64), ((13, 5, 2, 2), 8, 24, 16, 32)])
def test_fc_diag_bit_exact(params, n2, n1, n_img, block):
    """Dense layer by the diagonal method (App. D) on the device, against the
    oracle's rotate / multiply / sum / rescale, bit-exact on the same encoded
    diagonals; the library's slot layout equals the oracle's; the result
    decrypts to W x in every image's block."""
    c, P = bcn.Context(*params, device=0), O.Params(*params)
    rng = np.random.default_rng(n1 + n2)
    W = rng.integers(-127, 128, (n2, n1))
    xs = rng.uniform(-1, 1, (n_img, n1))
    z = np.zeros((1, P.N // 2))
    for b in range(n_img):
        z[0, b * block:b * block + n1] = xs[b]
    sk, _ = P.keygen(3)
    S = 2.0**30
    level = P.L
    ct = P.encrypt(sk, O.encode(z, P.N, S, P.q), level, 4)
    diags = O.fc_diagonals(W, n_img, block, P.N)
    steps, lay = bhw.fc_layout(W, n_img, block, P.N)
    assert steps == sorted(diags) and np.array_equal(lay, np.array([diags[r] for r in steps]))
    half = P.N // 2
    keys = {r % half: P.galois_keygen(sk, r % half, 200 + r % half) for r in steps if r % half}
    want = O.fc_diag(P, level, keys, W, ct[0], n_img, block)
    pts = O.encode(lay, P.N, float(P.q[level - 1]), P.q[:level])
    gks = {r: c.evk_prepare(bcn.to_device(k)) for r, k in keys.items()}
    fc = bhw.FcDiag(c, W, n_img, block, level, gks, diag_pts=pts)
    out = torch.empty((1, 2, level - 1, P.N), dtype=torch.int32, device="cuda")
    fc(bcn.to_device(ct), 1, out)
    got = bcn.to_host_u32(out)
    assert np.array_equal(got[0], want)
    assert c.device_status() == 0
    dec = c.decrypt_decode(sk, got, level - 1, S, half)[0]
    ref = np.stack([W @ xs[b] for b in range(n_img)])
    got_y = np.stack([dec[b * block:b * block + n2] for b in range(n_img)])
    # rotation noise times weights up to 127 over n1 inputs: relative to the outputs' size
    assert np.abs(got_y - ref).max() < 1e-5 * np.abs(ref).max()


def test_strided_then_gapped_conv_bit_exact():
    """A stride-2 3x3 packed convolution (hoisted rotations, MAC, mask product
    and rescale) and a 2x2 convolution of its gap-2 output, on the device,
    against the oracle, bit-exact; decrypted, the torch convolution chain."""
    c, P = bcn.Context(12, 5, 1, 1, device=0), O.Params(12, 5, 1, 1)
    n, cin, c1, c2, h, w = 3, 2, 3, 2, 12, 12
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (n, cin, h, w))
    w1 = rng.integers(-127, 128, (c1, cin, 3, 3)).astype(np.int8)
    w2 = rng.integers(-127, 128, (c2, c1, 2, 2)).astype(np.int8)
    sk, _ = P.keygen(3)
    S = 2.0**30
    cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), P.L, 4)
    steps = set(bhw.rotation_steps(3, w)) | set(bhw.rotation_steps(2, w, gap=2))
    keys = {r: P.galois_keygen(sk, r, 300 + r) for r in steps}
    gks = {r: c.evk_prepare(bcn.to_device(k)) for r, k in keys.items()}
    # oracle
    m1 = O.mask_bhw(n, h, w, 3, 2, 1, P.N)
    assert np.array_equal(m1, bhw.valid_mask(n, h, w, 3, P.N, stride=2))
    mpt = O.encode(m1[None], P.N, float(P.q[P.L - 1]), P.q)[0]
    y1 = P.rescale(P.L, P.mul_plain(P.L, O.conv_bhw(P, P.L, keys, w1, cts, w), mpt))
    y2 = O.conv_bhw(P, P.L - 1, keys, w2, y1, w, gap=2)
    # device
    conv1 = bhw.ConvBHW(c, w1, w, gks)
    conv2 = bhw.ConvBHW(c, w2, w, gks, gap=2)
    t1 = torch.empty((c1, 2, P.L, P.N), dtype=torch.int32, device="cuda")
    conv1(P.L, bcn.to_device(cts), t1)
    m = torch.empty((c1, 2, P.L - 1, P.N), dtype=torch.int32, device="cuda")
    c.op_mul_plain_rescale(P.L, t1, c1, bcn.to_device(mpt), m)
    assert np.array_equal(bcn.to_host_u32(m), y1)
    t2 = torch.empty((c2, 2, P.L - 1, P.N), dtype=torch.int32, device="cuda")
    conv2(P.L - 1, m, t2)
    got = bcn.to_host_u32(t2)
    assert np.array_equal(got, y2)
    assert c.device_status() == 0
    ref1 = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w1.astype(np.float64)), stride=2)
    ref2 = torch.nn.functional.conv2d(ref1, torch.from_numpy(w2.astype(np.float64))).numpy()
    dec = bhw.unpack(c.decrypt_decode(sk, got, P.L - 1, S, P.N // 2), n, h, w)
    assert np.abs(dec[:, :, 0:8:2, 0:8:2] - ref2).max() < 1e-5 * np.abs(ref2).max()
