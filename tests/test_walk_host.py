"""The library's peak search, compiled for the host, finds the same seed
clusters and maximum bins as the oracle on hand-built and random histograms:
the z-ordered walk (split_walk, Sec. 3.3, reading R5) and the x86 recursive
split (split_recursive, Sec. 3.3, reading R16).  CPU only."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = oracle.default_params()
P_REC = oracle.default_params(split_mode=1)
NB = oracle.num_bins(P)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_2412_14966_gb300 import build
    out = str(tmp_path_factory.mktemp("walk") / "walk_harness.so")
    subprocess.run([build._nvcc(), *build.ARCH, "-O2", "-std=c++17", "-shared", "-Xcompiler",
                    "-fPIC", "--expt-relaxed-constexpr", "-I", build.INCLUDE, "-I", build.CSRC,
                    os.path.join(ROOT, "tests", "walk_harness.cu"), "-o", out], check=True)
    lib = C.CDLL(out)
    ip = C.POINTER(C.c_int32)
    lib.harness_seeds.argtypes = [C.POINTER(C.c_uint32), C.c_int, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, ip,
                                  C.c_int]
    lib.harness_seeds.restype = C.c_int
    return lib


def _gpu_walk(lib, N, split_mode=0):
    N = np.ascontiguousarray(N, np.uint32)
    cap = 4096
    lo = np.zeros(cap, np.int32); hi = np.zeros(cap, np.int32); bn = np.zeros(cap, np.int32)
    t_pp = int(round(P.min_integral_pp * oracle.ONE))
    t_gas = int(round(P.min_integral_gas * oracle.ONE))
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    n = lib.harness_seeds(N.ctypes.data_as(C.POINTER(C.c_uint32)), NB, P.bin_threshold, t_pp,
                          t_gas, P.dip_num, P.dip_den, oracle.gas_bin(P), split_mode, ip(lo),
                          ip(hi), ip(bn), cap)
    assert n >= 0, "the recursive split with and without its scratch gives different pieces"
    return list(zip(lo[:n].tolist(), hi[:n].tolist(), bn[:n].tolist()))


def _oracle(N, p=P):
    s = oracle.seeds_from_hist(np.ascontiguousarray(N, np.uint32), p)
    return list(zip(s["lo"].tolist(), s["hi"].tolist(), s["bin"].tolist()))


def _hist(start, vals):
    h = np.zeros(NB, np.uint32)
    h[start:start + len(vals)] = vals
    return h


HAND = [
    (2000, [1000, 3000, 5000, 3000, 1000]),
    (2000, [1000, 4000, 8000, 4000, 1500, 4000, 8000, 4000, 1000]),
    (2000, [1000, 4000, 8000, 7000, 6400, 7000, 8000, 4000, 1000]),
    (2000, [1000, 4000, 8000, 7000, 6399, 7000, 8000, 4000, 1000]),
    (2000, [2000, 6000, 12000, 6000, 1000, 1500, 2500, 1500, 500]),
    (2500, [1000, 3000, 2192, 1000, 1000]),
    (500, [1000, 3000, 2192, 1000, 1000]),
    (2000, [4000, 12000, 2000, 12000, 4000]),
    (2000, [3000, 12000, 3000, 1000, 1000, 1000, 3000, 12000, 3000]),
    (2000, [3000, 12000, 3000, 300, 3000, 4000, 300, 3000, 12000, 3000]),
    (2000, [2000, 5000, 2240, 1000, 4000, 9000, 4000]),
    (2000, [3000, 6000, 3000, 1000, 8000, 20000, 12000, 20000, 8000, 3000]),
    (2000, [9000, 9000, 9000, 100, 9000, 9000]),
    (0, [9000, 12000, 300, 12000, 9000]),
    (NB - 5, [9000, 12000, 300, 12000, 9000]),
    (995, [3000, 9000, 3000, 500, 3000, 9000, 3000]),
]


@pytest.mark.parametrize("case", range(len(HAND)))
def test_walk_hand_built(harness, case):
    start, vals = HAND[case]
    h = _hist(start, vals)
    assert _gpu_walk(harness, h) == _oracle(h)


def test_walk_random_histograms(harness):
    rng = np.random.default_rng(31)
    for trial in range(2000):
        N = np.zeros(NB, np.int64)
        for _ in range(rng.integers(1, 10)):
            c = rng.integers(20, NB - 20)
            w = rng.integers(1, 6)
            amp = rng.integers(300, 25000)
            for j in range(c - 3 * w, c + 3 * w + 1):
                N[j] += int(amp * np.exp(-0.5 * ((j - c) / w) ** 2))
        noise = rng.integers(-400, 400, NB)
        N = np.maximum(N + np.where(N > 0, noise, 0), 0)
        for _ in range(rng.integers(0, 3)):          # plateaus
            k = rng.integers(0, NB - 6)
            N[k:k + rng.integers(2, 5)] = N[k]
        if trial % 7 == 0:                           # a gas-region cluster
            N[990:1010] = rng.integers(100, 6000, 20)
        N = N.astype(np.uint32)
        assert _gpu_walk(harness, N) == _oracle(N), trial


def test_walk_random_ties(harness):
    """Few distinct values: flat tops, equal maxima on both sides of a dip,
    plateaus at minima (ties of the lowest-index maximum and of the leftmost
    minimum)."""
    rng = np.random.default_rng(37)
    levels = np.array([0, 100, 300, 1200, 2500, 4000, 6000, 9000], np.uint32)
    for trial in range(2000):
        N = np.zeros(NB, np.uint32)
        for _ in range(rng.integers(1, 6)):
            c = int(rng.integers(10, NB - 40))
            n = int(rng.integers(3, 30))
            N[c:c + n] = levels[rng.integers(0, len(levels), n)]
            if rng.random() < 0.5:                   # smooth and quantise: flat tops
                v = np.convolve(N[c:c + n].astype(float), np.ones(3) / 3, mode="same")
                N[c:c + n] = (np.round(v / 1500) * 1500).astype(np.uint32)
        assert _gpu_walk(harness, N) == _oracle(N), trial


def _random_hist(rng, trial):
    N = np.zeros(NB, np.int64)
    for _ in range(rng.integers(1, 10)):
        c = rng.integers(20, NB - 20)
        w = rng.integers(1, 6)
        amp = rng.integers(300, 25000)
        for j in range(c - 3 * w, c + 3 * w + 1):
            N[j] += int(amp * np.exp(-0.5 * ((j - c) / w) ** 2))
    noise = rng.integers(-400, 400, NB)
    N = np.maximum(N + np.where(N > 0, noise, 0), 0)
    if trial % 7 == 0:
        N[990:1010] = rng.integers(100, 6000, 20)
    return N.astype(np.uint32)


@pytest.mark.parametrize("case", range(len(HAND)))
def test_recursive_split_hand_built(harness, case):
    start, vals = HAND[case]
    h = _hist(start, vals)
    assert _gpu_walk(harness, h, 1) == _oracle(h, P_REC)


def test_recursive_split_random_histograms(harness):
    rng = np.random.default_rng(41)
    differ = 0
    for trial in range(1500):
        N = _random_hist(rng, trial)
        rec = _gpu_walk(harness, N, 1)
        assert rec == _oracle(N, P_REC), trial
        differ += rec != _gpu_walk(harness, N, 0)
    # the two flavours are different algorithms: they must part somewhere
    assert differ > 0


def test_recursive_split_random_ties(harness):
    """Flat tops and equal maxima: the lower-position rule for equal maxima and
    the leftmost minimum."""
    rng = np.random.default_rng(43)
    levels = np.array([0, 100, 300, 1200, 2500, 4000, 6000, 9000], np.uint32)
    for trial in range(1500):
        N = np.zeros(NB, np.uint32)
        for _ in range(rng.integers(1, 6)):
            c = int(rng.integers(10, NB - 40))
            n = int(rng.integers(3, 30))
            N[c:c + n] = levels[rng.integers(0, len(levels), n)]
        assert _gpu_walk(harness, N, 1) == _oracle(N, P_REC), trial


def test_recursive_split_deep_comb(harness):
    """One proto-cluster of 40 deep, well-separated peaks rising to the right
    nests 39 pending right-hand sides; every peak becomes a seed."""
    vals = []
    for k in range(40):
        vals += [3000, 9000 + 10 * k, 3000, 300]
    h = _hist(100, vals[:-1])
    rec = _gpu_walk(harness, h, 1)
    assert rec == _oracle(h, P_REC)
    assert len(rec) == 40


def test_recursive_split_deeper_than_any_fixed_stack(harness):
    """A comb of 600 peaks rising to the right in one proto-cluster nests 599
    pending right-hand sides (the split keeps them at their split points, so
    no depth is too deep); every peak becomes a seed, as in the oracle."""
    vals = []
    for k in range(600):
        vals += [9000 + 10 * k, 3000, 300]
    h = _hist(20, vals[:-1])
    assert int(np.count_nonzero(h)) < NB
    rec = _gpu_walk(harness, h, 1)
    assert rec == _oracle(h, P_REC)
    assert len(rec) == 600
