"""The integer-operation counts behind bench.py's roofline (`bench.alu_ops`)
against an independent enumeration of what each kernel transforms: per square
layer and ciphertext, the key switch's forward NTTs digit by digit and target
prime by target prime (the digit's own primes reuse the square kernel's NTT of
d2), its inverse NTTs (special primes and the top data prime), ModDown's
forward NTTs, and the square kernel's transforms (two forward on the first
square layer's coefficient-form input, one inverse always) plus the domain
changes (features that meet NTT-domain ciphertexts, the outputs)."""
import math

import pytest

import bench
import workloads


def enumerate_work(cfg):
    """{class: [forward NTTs, N-element multiply-add passes, inverse NTTs]} per evaluation."""
    N, logN, K, a = 1 << cfg["log_n"], cfg["log_n"], cfg["n_special"], cfg["alpha"]
    levels, _ = workloads.level_schedule(cfg)
    work = {"square": [0, 0, 0], "keyswitch": [0, 0, 0], "moddown_rescale": [0, 0, 0]}
    in_ntt = False
    for layer, n in zip(cfg["cipher"], levels):
        C = workloads.cipher_layer_io(layer)[1]
        if layer["add"] and in_ntt:
            work["square"][0] += C * n  # features transformed to meet NTT-domain ciphertexts
        if not layer["square"]:
            continue
        for _ in range(C):
            for _limb in range(n):
                work["square"][0] += 0 if in_ntt else 2  # c0, c1 to the NTT domain
                work["square"][2] += 1  # d2 back to coefficient form
                work["square"][1] += 4  # c0^2, 2 c0 c1, c1^2 and c1^2 / N
                if a > 1:
                    work["square"][1] += 1  # d2 * Dhat^-1 for the key switch's ModUp
            targets = list(range(n)) + [("p", m) for m in range(K)]
            digits = [list(range(j * a, min(n, j * a + a))) for j in range(math.ceil(n / a))]
            for d in digits:
                if a == 1:
                    work["keyswitch"][1] += len(d)  # x * Dhat^-1 on the digit's primes (else in the square)
                for t in targets:
                    if t not in d:
                        work["keyswitch"][0] += 1  # ModUp residue -> forward NTT
                        work["keyswitch"][1] += len(d)  # fast basis conversion into t
                    work["keyswitch"][1] += 2  # both key halves
            for t in targets:
                if isinstance(t, tuple) or t == n - 1:
                    work["keyswitch"][2] += 2  # inverse NTT of both sums
                    if t == n - 1:
                        work["keyswitch"][1] += 4  # the rescale's first step, both polys
                else:
                    work["keyswitch"][1] += 2  # sums times N, both polys
            for _poly in range(2):
                work["moddown_rescale"][1] += K + 1  # the top limb's correction, shared by every limb
                for _limb in range(n - 1):
                    work["moddown_rescale"][0] += 1
                    work["moddown_rescale"][1] += K + 3  # Phat_m^-1 rides in the prepared key
        in_ntt = True
    if in_ntt:
        last = cfg["cipher"][-1]
        lout = levels[-1] - (1 if last["square"] else 0)
        work["square"][2] += workloads.cipher_layer_io(last)[1] * 2 * lout
    return work, N, logN


@pytest.mark.parametrize("name", ["cnn3_small", "cryptonets", "cryptonets_fi", "cifar_cnn"])
def test_alu_ops_match_enumeration(name):
    cfg = workloads.get_config(name)
    work, N, logN = enumerate_work(cfg)
    ops = bench.alu_ops(cfg)
    bf = (N // 2) * logN * bench.OPS_BUTTERFLY
    split = bench.alu_work(cfg)
    for k, (n_fwd, passes, n_inv) in work.items():
        assert ops[k] == (n_fwd + n_inv) * bf + passes * N * bench.OPS_MULADD, k
        assert (split[k]["fwd"], split[k]["inv"], split[k]["mont"] + split[k]["shoup"]) == (n_fwd, n_inv, passes), k
    # products of two variables: the square's three, the key switch's two per digit and target
    sq_mont = sum(workloads.cipher_layer_io(l)[1] * 3 * n
                  for l, n in zip(cfg["cipher"], workloads.level_schedule(cfg)[0]) if l["square"])
    assert split["square"]["mont"] == sq_mont and split["moddown_rescale"]["mont"] == 0


def test_cryptonets_ntt_counts_by_hand():
    """CryptoNets-scale network (7 + 1 primes, alpha 1): layer 1 at n = 7 with
    180 ciphertexts, layer 2 at n = 6 with 100."""
    work, _, _ = enumerate_work(workloads.get_config("cryptonets"))
    # key switch: 7 digits x 7 foreign targets of 8, plus 4 inverses, per ciphertext
    assert work["keyswitch"][0] == 180 * 7 * 7 + 100 * 6 * 6
    assert work["keyswitch"][2] == 180 * 4 + 100 * 4
    assert work["moddown_rescale"][0] == 180 * 12 + 100 * 10
    # square: forward 2 per limb on layer 1 and the layer-2 features; inverse 1 per limb of both layers
    # and the outputs (10 x 2 x 5)
    assert work["square"][0] == 180 * 7 * 2 + 100 * 6
    assert work["square"][2] == 180 * 7 + 100 * 6 + 10 * 2 * 5
