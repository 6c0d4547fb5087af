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


def _branch_case(P, n, h, w, k, s, c1, n2, n3, rng):
    ho = (h - k) // s + 1
    layers = [dict(type="conv", cin=1, h=h, w=w, cout=c1, k=k, stride=s, pad=0, add=True, square=True),
              dict(type="dense", n_in=c1 * ho * ho, n_out=n2, add=True, square=True),
              dict(type="dense", n_in=n2, n_out=n3, add=False, square=False)]
    x = rng.uniform(0, 1, (n, 1, h, w))
    wts = [rng.integers(-3, 4, (c1, 1, k, k)).astype(np.int8), rng.integers(-3, 4, (n2, c1 * ho * ho)),
           rng.integers(-3, 4, (n3, n2))]
    f1 = rng.uniform(-1, 1, (n, c1, ho, ho))
    f2 = rng.uniform(-1, 1, (n, n2))
    half = P.N // 2
    v1 = np.zeros((c1, half))
    for b in range(n):
        for yy in range(ho):
            for xx in range(ho):
                v1[:, b * h * w + s * (yy * w + xx)] = f1[b, :, yy, xx]
    v2 = np.zeros((1, half))
    for b in range(n):
        v2[0, b * h * w:b * h * w + n2] = f2[b]
    return layers, x, wts, f1, f2, v1, v2


def _net(x, wts, f1, f2, s):
    y = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(wts[0].astype(np.float64)),
                                   stride=s).numpy() + f1
    y = (y * y).reshape(x.shape[0], -1)
    z = y @ wts[1].T + f2
    return (z * z) @ wts[2].T


def test_bhw_branch_bit_exact():
    """A whole conv-square-dense-square-dense branch in BHW packing (App. D) on
    the device -- hoisted rotations + MAC with the feature add, square,
    bcn_op_fc_diag_sum over the strided outputs of two channels with the
    feature add, square, the output dense layer -- for two groups of two
    images, bit-exact against the oracle's branch on the same encodings; the
    library's diagonal layout equals the oracle's."""
    c, P = bcn.Context(10, 7, 1, 1, device=0), O.Params(10, 7, 1, 1)
    n, h, w, k, s, c1, n2, n3 = 2, 16, 16, 5, 2, 2, 12, 4
    rng = np.random.default_rng(85)
    L, half, S = P.L, P.N // 2, 2.0**30
    s1 = S * S / P.q[L - 1]
    sk, evk = P.keygen(3)
    layers, _, wts, _, _, _, _ = _branch_case(P, n, h, w, k, s, c1, n2, n3, rng)
    steps = bhw.BranchBHW.steps_for(layers, n, P.N)
    keys = {r: P.galois_keygen(sk, r, 500 + r) for r in steps}
    groups, want, feats = [], [], [[], []]
    for g in range(2):
        _, x, _, _, _, v1, v2 = _branch_case(P, n, h, w, k, s, c1, n2, n3, rng)
        cts = P.encrypt(sk, O.encode(O.pack_bhw(x, P.N), P.N, S, P.q), L, 4 + g)
        ft = [O.encode(v1, P.N, S, P.q[:L]), O.encode(v2, P.N, s1, P.q[:L - 2])[0]]
        want.append(O.bhw_branch(P, evk, keys, layers, wts, ft, cts, n))
        groups.append(cts)
        feats[0].append(ft[0])
        feats[1].append(ft[1])
    # the device's diagonals: its own layout, the oracle's encodings of it
    ho = (h - k) // s + 1
    pos = [s * (yy * w + xx) for yy in range(ho) for xx in range(ho)]
    diag_pts, lv = [], L - 1
    for W, s_in, C in ((wts[1], pos, c1), (wts[2], list(range(n2)), 1)):
        per = []
        for ch in range(C):
            part = W[:, ch * len(s_in):(ch + 1) * len(s_in)]
            st, lay = bhw.fc_layout_at(part, n, h * w, s_in, list(range(W.shape[0])), P.N)
            od = O.fc_diagonals_at(part, n, h * w, s_in, list(range(W.shape[0])), P.N)
            assert st == sorted(od) and np.array_equal(lay, np.array([od[r] for r in st]))
            per.append(O.encode(lay, P.N, float(P.q[lv - 1]), P.q[:lv]))
        diag_pts.append(np.stack(per))
        lv -= 2
    gks = {r: c.evk_prepare(bcn.to_device(kk)) for r, kk in keys.items()}
    ev = c.evk_prepare(bcn.to_device(evk))
    br = bhw.BranchBHW(c, layers, wts, n, gks, ev, diag_pts=diag_pts)
    assert br.rotation_steps_needed() == steps and br.out_level == L - 4
    out = torch.empty((2, 2, L - 4, P.N), dtype=torch.int32, device="cuda")
    br(bcn.to_device(np.stack(groups)), 2, [bcn.to_device(np.stack(feats[0])), bcn.to_device(np.stack(feats[1]))],
       out)
    got = bcn.to_host_u32(out)
    assert c.device_status() == 0
    for g in range(2):
        assert np.array_equal(got[g], want[g]), g


def test_bhw_cryptonets_branch_full_size_decrypts():
    """The CryptoNets-scale branch (5 x 5 stride-2 conv to 5 maps, 180 -> 100,
    100 -> 10, two feature adds and two squares) in BHW packing at its full
    ring, N = 8192 with 16 images' 16 x 16 segments per ciphertext, three
    groups, with the library's own encoder and keys: every image's outputs
    decrypt to the same network in fp64 within 1e-4 of the largest output."""
    cfg = workloads.get_config("cryptonets")
    c = bcn.Context.from_config(cfg)
    n, h, w, k, s, c1, n2, n3 = 16, 16, 16, 5, 2, 5, 100, 10
    rng = np.random.default_rng(86)
    L, half, S = c.L, c.N // 2, 2.0**30
    s1 = S * S / c.q[L - 1]
    s2 = s1 * s1 / c.q[L - 3]
    sk, evk = c.keygen(3)
    layers, _, wts, _, _, _, _ = _branch_case(c, n, h, w, k, s, c1, n2, n3, rng)
    assert [l["n_in"] for l in layers[1:]] == [l["n_in"] for l in cfg["cipher"][1:]]
    steps = bhw.BranchBHW.steps_for(layers, n, c.N)
    gks = {r: c.evk_prepare(bcn.to_device(c.galois_keygen(sk, r, 600 + r))) for r in steps}
    br = bhw.BranchBHW(c, layers, wts, n, gks, c.evk_prepare(bcn.to_device(evk)))
    G = 3
    xs, cts, f1s, f2s, ft0, ft1 = [], [], [], [], [], []
    for g in range(G):
        _, x, _, f1, f2, v1, v2 = _branch_case(c, n, h, w, k, s, c1, n2, n3, rng)
        xs.append(x), f1s.append(f1), f2s.append(f2)
        cts.append(c.encrypt(sk, c.encode(bhw.pack(x, c.N), L, S), L, 10 + g))
        ft0.append(c.encode(v1, L, S))
        ft1.append(c.encode(v2, L - 2, s1)[0])
    out = torch.empty((G, 2, br.out_level, c.N), dtype=torch.int32, device="cuda")
    br(bcn.to_device(np.stack(cts)), G, [bcn.to_device(np.stack(ft0)), bcn.to_device(np.stack(ft1))], out)
    assert c.device_status() == 0
    dec = c.decrypt_decode(sk, bcn.to_host_u32(out), br.out_level, s2, half)
    for g in range(G):
        ref = _net(xs[g], wts, f1s[g], f2s[g], s)
        got = np.stack([dec[g, b * h * w:b * h * w + n3] for b in range(n)])
        assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()
