"""Philox4x32-10 and Box-Muller white noise for the Gaussian initial conditions.

Oracle (test infrastructure only).  The paper draws Gaussian initial conditions (Sec. 2,
2LPTic) without fixing a generator; this library fixes the counter-based Philox4x32-10 of
Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written
here from its published definition:

  round:  (hi0, lo0) = mulhilo(0xD2511F53, c0);  (hi1, lo1) = mulhilo(0xCD9E8D57, c2)
          c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
  key schedule: k0 += 0x9E3779B9, k1 += 0xBB67AE85 between rounds; 10 rounds.

White-noise convention of this library (both the oracle and the CUDA kernel implement it):
  cell m of the N^3 lattice (m = (iz N + iy) N + ix) belongs to counter block g = m >> 2, lane
  l = m & 3; counter = (g mod 2^32, g >> 32, 0, 0); key = (seed mod 2^32, seed >> 32).
  The block's outputs r0..r3 give uniforms u_i = ((r_i >> 8) + 1) 2^-24 in (0, 1], and
  Box-Muller pairs (r0, r1) -> lanes 0, 1 and (r2, r3) -> lanes 2, 3:
      rho = sqrt(-2 ln u_a),  lane even: rho cos(2 pi u_b),  lane odd: rho sin(2 pi u_b).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Vectorised Philox4x32-10.  counter: uint32 array (..., 4); key: uint32 array (..., 2)."""
    c = [np.asarray(counter[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0).astype(np.uint32)
            k1 = (k1 + W1).astype(np.uint32)
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0.astype(np.uint64), lo1, hi0 ^ c[3] ^ k1.astype(np.uint64), lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def uniforms_from_bits(r):
    """u = ((r >> 8) + 1) * 2^-24, in (0, 1]; exactly representable in float32."""
    return ((np.asarray(r, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0**-24


def white_noise(n, seed):
    """Unit-variance Gaussian white noise on the n^3 lattice, float64, shape (n, n, n) = [iz][iy][ix]."""
    total = n**3
    nblk = (total + 3) // 4
    g = np.arange(nblk, dtype=np.uint64)
    counter = np.zeros((nblk, 4), dtype=np.uint32)
    counter[:, 0] = (g & MASK32).astype(np.uint32)
    counter[:, 1] = (g >> np.uint64(32)).astype(np.uint32)
    key = np.zeros((nblk, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    r = philox4x32_10(counter, key)
    u = uniforms_from_bits(r)
    out = np.empty((nblk, 4), dtype=np.float64)
    for pair in (0, 1):
        ua, ub = u[:, 2 * pair], u[:, 2 * pair + 1]
        rho = np.sqrt(-2.0 * np.log(ua))
        out[:, 2 * pair] = rho * np.cos(2.0 * np.pi * ub)
        out[:, 2 * pair + 1] = rho * np.sin(2.0 * np.pi * ub)
    return out.reshape(-1)[:total].reshape(n, n, n)
