"""Pins of the oracle's noise: Philox words, Box-Muller normals, increments."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _kat_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals = [int(x, 16) for x in line.split()]
            rows.append((vals[0:4], vals[4:6], vals[6:10]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat_rows(golden_dir)
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
        assert [int(x) for x in got] == want


def test_philox_batched_matches_single(golden_dir):
    rows = _kat_rows(golden_dir)
    ctr = np.array([r[0] for r in rows], dtype=np.uint64)
    key = np.array([r[1] for r in rows], dtype=np.uint64)
    got = philox.philox4x32_10(ctr, key)
    assert [[int(x) for x in g] for g in got] == [r[2] for r in rows]


def test_uniforms_open_interval():
    w = np.array([0, 1, 2**31, 2**32 - 1], dtype=np.uint64)
    u = philox.words_to_uniform(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 0.5 * 2.0 ** -32


def test_box_muller_is_standard_normal():
    ctr = np.zeros((50000, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(50000)
    ctr[:, 3] = 12345
    z = philox.box_muller(philox.philox4x32_10(ctr, np.array([7, 9], dtype=np.uint64)))
    for k in range(4):
        assert stats.kstest(z[:, k], "norm").pvalue > 1e-4
    # pairs from one (u1, u2) are uncorrelated, as are the two pairs of a block
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.02


def test_box_muller_closed_form_point():
    # u1 = exp(-1/2) -> radius 1; u2 = 1/8 -> angle pi/4.
    # Choose words whose uniforms are those values up to 2^-33.
    k1 = int(np.exp(-0.5) * 2**32)
    k2 = 2**29  # (k + 1/2) 2^-32 = 1/8 + 2^-33
    z = philox.box_muller(np.array([k1, k2, k1, k2], dtype=np.uint64))
    u1 = (k1 + 0.5) * 2.0 ** -32
    u2 = (k2 + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2 * np.log(u1))
    assert abs(rad - 1.0) < 1e-8
    assert abs(z[0] - rad * np.cos(2 * np.pi * u2)) < 1e-15
    assert abs(z[0] - np.sqrt(0.5)) < 1e-7 and abs(z[1] - np.sqrt(0.5)) < 1e-7


@pytest.mark.parametrize("D", [1, 4, 10, 13])
def test_increments_scale_and_independence(D):
    N, M, T = 4, 4000, 2.0
    dW = philox.brownian_increments(3, 5, M, N, D, T)
    assert dW.shape == (N, M, D)
    dt = T / N
    x = dW.reshape(-1) / np.sqrt(dt)
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # different iterations and seeds give different paths
    assert not np.allclose(dW, philox.brownian_increments(3, 6, M, N, D, T))
    assert not np.allclose(dW, philox.brownian_increments(4, 5, M, N, D, T))


def test_increment_counter_layout():
    # Delta W[n, m, 4q + j] comes from Philox block (q, n, m, iteration), slot j.
    N, M, D, T, seed, it = 3, 5, 7, 1.0, 0x1234567890, 9
    dW = philox.brownian_increments(seed, it, M, N, D, T)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)
    for (n, m, q) in [(0, 0, 0), (2, 4, 1), (1, 3, 0)]:
        w = philox.philox4x32_10(np.array([q, n, m, it], dtype=np.uint64), key)
        z = philox.box_muller(w) * np.sqrt(T / N)
        for j in range(4):
            if 4 * q + j < D:
                assert dW[n, m, 4 * q + j] == z[j]


def test_init_key_differs_from_noise_key():
    k = philox.init_key(5)
    assert int(k[0]) == 5 ^ 0x494E4954 and int(k[1]) == 0
    z = philox.init_normals(5, 4001)
    assert z.shape == (4001,)
    assert stats.kstest(z, "norm").pvalue > 1e-4
