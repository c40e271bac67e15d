"""Counter-based randomness for ADASAP's sampling steps (oracle side).

The solver draws three random objects per iteration t (Alg. 2): the row block
B (b distinct indices of [n], drawn uniformly -- Sec. 4.3 "uniform sampling"),
the Nystrom test matrix Omega (b x r, Gaussian) and the power-iteration start
vector v0 (b, Gaussian; Alg. 5).  Both the CUDA path and this oracle derive
them from ONE published counter-based generator, each side implementing it
independently from its definition:

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11).  State: a 128-bit counter (c0, c1, c2, c3) and a 64-bit
key (k0, k1).  One round maps
    (hi0, lo0) = M0 * c0,   (hi1, lo1) = M1 * c2        (32x32 -> 64-bit products)
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.

Conventions of this project (shared by both sides; they are definitions, not
arithmetic of the method):
  key       = (seed mod 2^32, seed >> 32)
  streams   : FEISTEL=1, OMEGA=2, V0=3, CHECK=4
  normals   : element e of a stream at iteration t comes from Philox counter
              (e // 4, t, 0, stream); words (w0, w1) give normals 0 and 1,
              words (w2, w3) give normals 2 and 3, by Box-Muller:
              u(w) = (w + 0.5) * 2^-32,  rad = sqrt(-2 ln u(w_even)),
              z_even = rad * cos(2 pi u(w_odd)),  z_odd = rad * sin(2 pi u(w_odd)).
  Omega     : Omega[i, c] = z(i * r + c) / sqrt(b)  (scaled so E[Omega^T Omega] = I)
  block B   : B[i] = pi_t(i) for i < b, where pi_t is a permutation of [n]
              made from a balanced 4-round Feistel network on 2h bits
              (2^(2h) >= n, h >= 1) with cycle walking (Black & Rogaway,
              "Ciphers with arbitrary finite domains", CT-RSA 2002).  Round j
              maps (L, R) -> (R, L ^ F_j(R)), F_j(R) = word0 of Philox counter
              (R, t, j, FEISTEL) masked to h bits; x = (L << h) | R.  The walk
              repeats the 4-round map until the value is < n.  pi_t(0..b-1)
              are distinct because pi_t is a bijection of [n].
"""

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

FEISTEL = 1
OMEGA = 2
V0 = 3
CHECK = 4


def philox4x32_10(ctr, key):
    """Philox4x32-10 on an array of counters.

    ctr: (..., 4) integers < 2^32; key: (k0, k1).  Returns (..., 4) uint32.
    """
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def _unit(w):
    return (np.asarray(w, dtype=np.float64) + 0.5) * 2.0 ** -32


def normals(count, seed, t, stream):
    """`count` standard normals of `stream` at iteration t (Box-Muller, FP64)."""
    nblk = (count + 3) // 4
    j = np.arange(nblk, dtype=np.uint64)
    ctr = np.stack([j, np.full_like(j, t), np.zeros_like(j),
                    np.full_like(j, stream)], axis=-1)
    w = philox4x32_10(ctr, seed_key(seed))
    rad01 = np.sqrt(-2.0 * np.log(_unit(w[:, 0])))
    ang01 = 2.0 * np.pi * _unit(w[:, 1])
    rad23 = np.sqrt(-2.0 * np.log(_unit(w[:, 2])))
    ang23 = 2.0 * np.pi * _unit(w[:, 3])
    z = np.stack([rad01 * np.cos(ang01), rad01 * np.sin(ang01),
                  rad23 * np.cos(ang23), rad23 * np.sin(ang23)], axis=-1)
    return z.reshape(-1)[:count]


def feistel_half_bits(n):
    """h such that 2^(2h) >= n, h >= 1."""
    k = max(2, int(n - 1).bit_length()) if n > 1 else 2
    return (k + 1) // 2


def feistel_permute(x, n, seed, t):
    """pi_t(x) for an array of x in [0, n) (4-round Feistel + cycle walking)."""
    h = feistel_half_bits(n)
    mask = np.uint64((1 << h) - 1)
    key = seed_key(seed)
    x = np.asarray(x, dtype=np.uint64).copy()
    todo = np.ones(x.shape, dtype=bool)
    first = True
    while first or todo.any():
        first = False
        y = x[todo]
        L = (y >> np.uint64(h)) & mask
        R = y & mask
        for j in range(4):
            ctr = np.stack([R, np.full_like(R, t), np.full_like(R, j),
                            np.full_like(R, FEISTEL)], axis=-1)
            F = philox4x32_10(ctr, key)[..., 0].astype(np.uint64) & mask
            L, R = R, L ^ F
        x[todo] = (L << np.uint64(h)) | R
        todo = x >= np.uint64(n)
    return x.astype(np.int64)


def sample_block(n, b, seed, t):
    """B_t = (pi_t(0), ..., pi_t(b-1)): b distinct indices of [n]."""
    if not (0 < b <= n):
        raise ValueError("need 0 < b <= n")
    return feistel_permute(np.arange(b), n, seed, t)


def sample_omega(b, r, seed, t):
    """Gaussian test matrix Omega (b x r), entries N(0, 1/b)."""
    return normals(b * r, seed, t, OMEGA).reshape(b, r) / np.sqrt(b)


def sample_v0(b, seed, t):
    """Power-iteration start vector v0 ~ N(0, I_b) (Alg. 5)."""
    return normals(b, seed, t, V0)


def philox_schedule(n, b, r, seed):
    """Schedule t -> (B_t, Omega_t, v0_t) drawn from the counter-based generator."""
    def sched(t):
        return sample_block(n, b, seed, t), sample_omega(b, r, seed, t), sample_v0(b, seed, t)
    return sched
