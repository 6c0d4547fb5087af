"""The NTT core's register distributions, checked on the host against the
header itself: a small host program compiled with nvcc includes
`ntt_core.cuh` and writes out `elem_def` (the element each register holds in
each pass) and `warp_local` for every block shape the library instantiates.
For every pass: the map is a permutation of the limb; it is linear in the
thread (element and padded shared-memory address of register u of thread tid
are the thread's base plus register u's offset of thread 0), which lets a
thread address every register from one base; and `warp_local` holds exactly
when each warp's registers form one contiguous block of 32 R elements (the
condition for exchanging through shared memory with a warp barrier)."""
import pathlib
import shutil
import subprocess

import numpy as np
import pytest

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2402_01296_gb300" / "csrc"
INCLUDE = pathlib.Path(__file__).resolve().parents[1] / "include"
SHAPES = [(l, 4) for l in range(4, 12)] + [(12, 16), (12, 32), (13, 16), (13, 32), (14, 16), (14, 32)]

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "ntt_core.cuh"
using namespace bcn;

template <int LOGN, int R, int P>
void dump(FILE *f) {
    using C = NttCore<LOGN, R>;
    if constexpr (P < C::PASSES) {
        int hdr[6] = {LOGN, R, P, C::template warp_local<P>() ? 1 : 0, C::s0_of(P), C::s1_of(P)};
        std::fwrite(hdr, sizeof(int), 6, f);
        std::vector<int> e((size_t)C::T * R);
        for (int tid = 0; tid < C::T; tid++)
            for (int u = 0; u < R; u++) e[(size_t)tid * R + u] = C::template elem_def<P>(u, tid);
        std::fwrite(e.data(), sizeof(int), e.size(), f);
        dump<LOGN, R, P + 1>(f);
    }
}

int main(int argc, char **argv) {
    FILE *f = std::fopen(argv[1], "wb");
    if (!f) return 1;
%s
    std::fclose(f);
    return 0;
}
"""


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not pathlib.Path(nvcc).exists():
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("ntt_layout")
    src = d / "layout.cu"
    calls = "\n".join(f"    dump<{l}, {r}, 0>(f);" for l, r in SHAPES)
    src.write_text(HARNESS % calls)
    exe = d / "layout"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", str(CSRC), "-I", str(INCLUDE),
                        "-gencode", "arch=compute_103a,code=sm_103a", str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = d / "layout.bin"
    subprocess.run([str(exe), str(out)], check=True)
    raw = np.fromfile(out, dtype=np.int32)
    res, i = [], 0
    while i < raw.size:
        logn, R, P, wl, s0, s1 = (int(v) for v in raw[i:i + 6])
        i += 6
        N = 1 << logn
        e = raw[i:i + N].reshape(N // R, R)
        i += N
        res.append((logn, R, P, bool(wl), s0, s1, e))
    return res


def pad(e):
    return e + (e >> 5)


def test_every_shape_and_pass_is_written(tables):
    seen = {(t[0], t[1]) for t in tables}
    assert seen == set(SHAPES)
    for logn, R, _ in {(t[0], t[1], 0) for t in tables}:
        passes = [t for t in tables if t[0] == logn and t[1] == R]
        assert passes[0][4] == 0 and passes[-1][5] == logn  # the passes cover every stage


def test_each_pass_is_a_permutation(tables):
    for logn, R, P, _, _, _, e in tables:
        assert np.array_equal(np.sort(e.ravel()), np.arange(1 << logn)), (logn, R, P)


def test_each_pass_is_linear_in_the_thread(tables):
    for logn, R, P, _, _, _, e in tables:
        assert np.array_equal(e, e[:, :1] + e[:1, :]), (logn, R, P)
        assert np.array_equal(pad(e), pad(e[:, :1]) + pad(e[:1, :])), (logn, R, P)


def test_warp_local_exactly_when_warps_hold_contiguous_blocks(tables):
    for logn, R, P, wl, _, _, e in tables:
        T = e.shape[0]
        WS = min(32, T)
        contiguous = all(
            np.array_equal(np.sort(e[w * WS:(w + 1) * WS].ravel()), np.arange(w * WS * R, (w + 1) * WS * R))
            for w in range(T // WS))
        assert wl == (contiguous and T >= 32), (logn, R, P, wl, contiguous)
