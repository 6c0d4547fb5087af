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
