"""Pins of the oracle's Philox4x32-10 and of the stream contract.

The oracle's generator is checked word for word against Triton's Philox
(a separate implementation of Salmon et al., SC'11), executed on the CPU by
Triton's interpreter in a child process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678, 2 ** 64 - 1])
def test_philox_matches_triton(orc, seed):
    pytest.importorskip("triton")
    n = 64
    res = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox_ref.py"),
                          str(seed), str(n), str(seed % 1000 + 7)],
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    ref = json.loads(res.stdout.strip().splitlines()[-1])
    key = [seed & 0xffffffff, seed >> 32]
    for ctr, want in zip(ref["ctr"], ref["out"]):
        assert orc.philox4x32_10(ctr, key) == [int(w) for w in want]


def test_stream_counter_layout(orc):
    """counter = (idx_lo, tag<<30 | point, path, idx_hi), key = (seed_lo, seed_hi)."""
    seed, tag, point, path, idx = 0x0123456789ABCDEF, 2, 12345, 777, (5 << 32) | 99
    got = orc.stream_words(seed, tag, point, path, idx)
    want = orc.philox4x32_10([99, (tag << 30) | point, path, 5],
                             [seed & 0xffffffff, seed >> 32])
    assert got == want


def test_philox_words_uniform(orc):
    """Chi-square of the top byte over 4096 counters x 4 words (sanity, not a pin)."""
    words = np.array([orc.stream_words(9, 1, 0, 3, i) for i in range(4096)], dtype=np.uint64)
    top = (words.ravel() >> 24).astype(np.int64)
    counts = np.bincount(top, minlength=256)
    exp = len(top) / 256.0
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert 180 < chi2 < 340     # 255 dof: mean 255, sd ~22.6


def test_batched_call_is_the_same_generator(orc):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(500, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x89ABCDEF, 0x01234567]
    got = orc.philox_many(ctr, key)
    for i in range(0, 500, 7):
        assert list(got[i]) == orc.philox4x32_10(list(ctr[i]), key)

