"""Counter-based noise for the FP64 oracle (test infrastructure only).

This module is part of the oracle: plain, slow, obviously correct CPU code that
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import it; the library never does.

The paper draws Brownian increments Delta W_n ~ N(0, Delta t_n) (Section 2.2,
Eq. "disc equations", first line) without fixing a generator.  To make the GPU
and CPU consume the *same* increments, both sides implement one published
counter-based generator from its definition:

* Philox4x32-10 -- J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
  "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Section 4 (the Philox
  S-box: two 32x32->64 multiplies per round, Weyl key schedule, 10 rounds).
* Box--Muller (G. E. P. Box, M. E. Muller, Ann. Math. Statist. 29, 1958): a
  pair of uniforms (u1, u2) in (0, 1) gives two independent standard normals
  sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2).

Counter / key conventions shared with the GPU (they are the interface, not
arithmetic):

* noise key  = (seed mod 2^32, seed >> 32 mod 2^32)
* init key   = (key0 XOR 0x494E4954, key1)          ("INIT" in ASCII)
* a 32-bit word k maps to the uniform u = (k + 1/2) * 2^-32, never 0 or 1;
* the four words (w0, w1, w2, w3) of one Philox block give normals
  (z0, z1) from (w0, w1) and (z2, z3) from (w2, w3).
"""
from __future__ import annotations

import numpy as np

# Philox4x32 round multipliers and Weyl key increments (SC'11, Section 4.2).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)

INIT_KEY_XOR = 0x494E4954


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds on arrays of counters.

    counter: uint32-compatible array [..., 4]; key: [..., 2] (broadcastable).
    Returns uint32 array [..., 4].

    One round (SC'11, Section 4.2): with (hi0, lo0) = M0 * c0 and
    (hi1, lo1) = M1 * c2 as 64-bit products,
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0).  Between rounds the key is
    bumped by the Weyl constants (k0 += W0, k1 += W1 mod 2^32).
    """
    c = np.asarray(counter, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def noise_key(seed: int):
    """Philox key for the Brownian increments of a run with this seed."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)


def init_key(seed: int):
    """Philox key for the parameter initialisation of a run with this seed."""
    k = noise_key(seed)
    k[0] ^= np.uint64(INIT_KEY_XOR)
    return k


def words_to_uniform(words):
    """u = (k + 1/2) 2^-32, exactly representable in FP64, in (0, 1)."""
    return (np.asarray(words, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(words):
    """Four Philox words [..., 4] -> four standard normals [..., 4] (FP64)."""
    u = words_to_uniform(words)
    r01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    r23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    ang01 = 2.0 * np.pi * u[..., 1]
    ang23 = 2.0 * np.pi * u[..., 3]
    return np.stack([r01 * np.cos(ang01), r01 * np.sin(ang01),
                     r23 * np.cos(ang23), r23 * np.sin(ang23)], axis=-1)


def brownian_counters(iteration: int, M: int, N: int, D: int, paths=None):
    """Philox counters for the increments of one iteration.

    Counter of (step n, path m, dimension quad q) is (q, n, m, iteration);
    quad q covers dimensions 4q .. 4q+3.  Returns uint64 [N, M, Q, 4], or
    [N, len(paths), Q, 4] for the paths listed in `paths`.
    """
    Q = (D + 3) // 4
    ms = np.arange(M) if paths is None else np.asarray(paths)
    n, m, q = np.meshgrid(np.arange(N), ms, np.arange(Q), indexing="ij")
    it = np.full_like(n, int(iteration) & 0xFFFFFFFF)
    return np.stack([q, n, m, it], axis=-1).astype(np.uint64)


def brownian_words(seed: int, iteration: int, M: int, N: int, D: int):
    """Raw Philox words of one iteration's noise, uint32 [N, M, 4*ceil(D/4)]."""
    ctr = brownian_counters(iteration, M, N, D)
    w = philox4x32_10(ctr, noise_key(seed))
    return w.reshape(N, M, -1)


def brownian_increments(seed: int, iteration: int, M: int, N: int, D: int, T: float, paths=None):
    """Delta W_n^m ~ N(0, Delta t) with Delta t = T/N (Section 2.2, Eq. disc
    equations, first line).  Returns FP64 [N, M, D] (with `paths`: only the
    listed paths, [N, len(paths), D]; a path's noise depends on its own
    counters alone)."""
    ctr = brownian_counters(iteration, M, N, D, paths)
    z = box_muller(philox4x32_10(ctr, noise_key(seed)))
    z = z.reshape(N, ctr.shape[1], -1)[:, :, :D]
    return np.sqrt(T / N) * z


def init_normals(seed: int, count: int):
    """Standard normals for parameter initialisation: element i uses Philox
    counter (i >> 2, 0, 0, 0) under the init key and takes word-pair slot
    (i & 3) of the Box-Muller output.  Returns FP64 [count]."""
    nblk = (count + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    z = box_muller(philox4x32_10(ctr, init_key(seed)))
    return z.reshape(-1)[:count]
