"""Philox4x32-10 and the Gaussian noise draw of the Monte Carlo method.

Test infrastructure only (see the package docstring).

The paper draws xi ~ N(0,1) for every noisy gate (Sec. 2, Eq. 1) without
naming a generator.  This build uses the counter-based Philox4x32 with 10
rounds from Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
as 1, 2, 3" (SC'11), so that the noise of trajectory b at gate g is a pure
function of (seed, b, g) on both the CPU and the GPU:

  key     = (seed mod 2^32, seed >> 32)
  counter = (b mod 2^32, b >> 32, g mod 2^32, g >> 32)
  round   : (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
                                 hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
            with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is advanced by
            the Weyl increments (0x9E3779B9, 0xBB67AE85) before rounds 2..10.
  u1      = (((w0 << 32 | w1) >> 11) + 0.5) * 2^-53, u2 likewise from (w2, w3)
  xi_a    = sqrt(-2 ln u1) cos(2 pi u2),  xi_b = sqrt(-2 ln u1) sin(2 pi u2)
            (Box and Muller, 1958).

Pins: the uniform words and normals are checked statistically (moments,
Kolmogorov-Smirnov against N(0,1), independence across counters) and the whole
noise model is pinned end to end by the Monte Carlo mean matching the exact
density matrix (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PHILOX_ROUNDS = 10


def philox4x32_10(counter, key):
    """Philox4x32-10 on one 128-bit counter with a 64-bit key (Python ints)."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in counter)
    k0, k1 = (int(x) & MASK32 for x in key)
    for rnd in range(PHILOX_ROUNDS):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = (
            ((p1 >> 32) ^ c1 ^ k0) & MASK32,
            p1 & MASK32,
            ((p0 >> 32) ^ c3 ^ k1) & MASK32,
            p0 & MASK32,
        )
    return c0, c1, c2, c3


def philox4x32_10_array(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10: uint64 arrays holding 32-bit words."""
    m = np.uint64(MASK32)
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & m for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & m
    k1 = np.asarray(k1, dtype=np.uint64) & m
    for rnd in range(PHILOX_ROUNDS):
        if rnd:
            k0 = (k0 + np.uint64(PHILOX_W0)) & m
            k1 = (k1 + np.uint64(PHILOX_W1)) & m
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        c0, c1, c2, c3 = (
            ((p1 >> np.uint64(32)) ^ c1 ^ k0) & m,
            p1 & m,
            ((p0 >> np.uint64(32)) ^ c3 ^ k1) & m,
            p0 & m,
        )
    return c0, c1, c2, c3


def noise_words(seed: int, traj: int, gate_id: int):
    """The four 32-bit words drawn for trajectory `traj` at gate `gate_id`."""
    return philox4x32_10(
        (traj & MASK32, (traj >> 32) & MASK32, gate_id & MASK32, (gate_id >> 32) & MASK32),
        (seed & MASK32, (seed >> 32) & MASK32),
    )


def uniform53(hi: int, lo: int) -> float:
    """Open-interval uniform in (0, 1) from the top 53 bits of a 64-bit word."""
    return ((((hi << 32) | lo) >> 11) + 0.5) * 2.0 ** -53


def normal_pair(seed: int, traj: int, gate_id: int):
    """(xi_a, xi_b), two independent N(0,1) draws (Box-Muller)."""
    w0, w1, w2, w3 = noise_words(seed, traj, gate_id)
    u1 = uniform53(w0, w1)
    u2 = uniform53(w2, w3)
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


def normal_pairs_array(seed: int, trajs, gate_ids):
    """Vectorised `normal_pair` over broadcastable arrays of (traj, gate_id)."""
    trajs = np.asarray(trajs, dtype=np.uint64)
    gate_ids = np.asarray(gate_ids, dtype=np.uint64)
    trajs, gate_ids = np.broadcast_arrays(trajs, gate_ids)
    s32 = np.uint64(32)
    m = np.uint64(MASK32)
    w0, w1, w2, w3 = philox4x32_10_array(
        trajs & m, trajs >> s32, gate_ids & m, gate_ids >> s32,
        np.uint64(seed & MASK32), np.uint64((seed >> 32) & MASK32))
    u1 = (((w0 << s32) | w1) >> np.uint64(11)).astype(np.float64)
    u2 = (((w2 << s32) | w3) >> np.uint64(11)).astype(np.float64)
    u1 = (u1 + 0.5) * 2.0 ** -53
    u2 = (u2 + 0.5) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)
