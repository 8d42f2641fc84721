"""Pins for oracle.philox (Philox4x32-10, Salmon et al. SC'11)."""
import os

import numpy as np

from oracle.philox import philox4x32_10, seed_key

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([int(x, 16) for x in line.split()])
    return rows


def test_known_answer_vectors():
    rows = load_kat()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:6])
        assert [int(x) for x in out] == r[6:]


def test_vectorised_equals_scalar():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2 ** 32, size=(4, 17), dtype=np.uint64)
    k = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64)
    vec = philox4x32_10(c[0], c[1], c[2], c[3], k[0], k[1])
    for i in range(17):
        one = philox4x32_10(int(c[0, i]), int(c[1, i]), int(c[2, i]), int(c[3, i]), int(k[0]), int(k[1]))
        assert [int(v[i]) for v in vec] == [int(x) for x in one]


def test_output_words_look_uniform():
    # 2^16 counters -> 2^18 words; each byte value should appear ~ 2^10 times.
    x = np.arange(1 << 16, dtype=np.uint64)
    words = np.concatenate(philox4x32_10(x, 7, 3, 1, 0x1234, 0x5678))
    assert words.max() < 2 ** 32
    bytes_ = np.concatenate([(words >> np.uint64(8 * s)) & np.uint64(255) for s in range(4)])
    counts = np.bincount(bytes_.astype(np.int64), minlength=256)
    expected = bytes_.size / 256
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 400.0          # 255 dof: mean 255, sd ~ 22.6
    # mean of u / 2^32 close to 1/2
    assert abs(float((words / 2.0 ** 32).mean()) - 0.5) < 5e-3


def test_seed_key_split():
    assert seed_key(0x0123456789ABCDEF) == (0x89ABCDEF, 0x01234567)
    assert seed_key(5) == (5, 0)
