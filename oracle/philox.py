"""Philox4x32-10 counter-based generator and the white-noise mapping.

Test infrastructure (oracle): never imported by the library.

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
Shaw (SC'11): a 4 x 32-bit counter and a 2 x 32-bit key, ten rounds of two
32x32->64 multiplications whose high halves are mixed with the other two
counter words and the key, with a Weyl increment of the key between rounds.

The paper draws its white noise with TRNG (Sec. 6, implementation details)
and fixes no generator mapping; this sampler's convention is:
  key     = (seed mod 2^32, seed >> 32)
  counter = (p, tag, sample mod 2^32, sample >> 32), tag = 0 for noise,
            p = index of the pair of cells (2p, 2p+1)
  k1 = (w0 * 2^32 + w1) >> 11, k2 = (w2 * 2^32 + w3) >> 11   (53-bit ints)
  u1 = (k1 + 1) 2^-53 in (0, 1],  u2 = k2 2^-53 in [0, 1)
  xi_{2p} = r cos(2 pi u2), xi_{2p+1} = r sin(2 pi u2), r = sqrt(-2 ln u1)
The discrete right-hand side is f = W^{1/2} xi with xi ~ N(0, I) (Sec. 4.2).
"""
import numpy as np

MASK32 = 0xFFFFFFFF
MUL0 = 0xD2511F53
MUL1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9
WEYL1 = 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & np.uint64(MASK32) for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & np.uint64(MASK32)
    k1 = np.asarray(k1, dtype=np.uint64) & np.uint64(MASK32)
    m32 = np.uint64(MASK32)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(WEYL0)) & m32
            k1 = (k1 + np.uint64(WEYL1)) & m32
        p0 = np.uint64(MUL0) * c0  # < 2^64, exact in uint64
        p1 = np.uint64(MUL1) * c2
        c0, c1, c2, c3 = ((p1 >> s32) ^ c1 ^ k0, p1 & m32, (p0 >> s32) ^ c3 ^ k1, p0 & m32)
    return c0, c1, c2, c3


def philox4x32_10_int(ctr, key):
    """Second statement with Python integers, one counter at a time."""
    x = [int(v) & MASK32 for v in ctr]
    k = [int(v) & MASK32 for v in key]
    for rnd in range(10):
        if rnd:
            k = [(k[0] + WEYL0) & MASK32, (k[1] + WEYL1) & MASK32]
        prod_a = MUL0 * x[0]
        prod_b = MUL1 * x[2]
        x = [(prod_b >> 32) ^ x[1] ^ k[0], prod_b & MASK32,
             (prod_a >> 32) ^ x[3] ^ k[1], prod_a & MASK32]
    return tuple(x)


def noise_words(ncells, seed, sample, tag=0):
    """Raw Philox words [npairs, 4] for one sample (uint64 holding u32)."""
    npairs = (int(ncells) + 1) // 2
    p = np.arange(npairs, dtype=np.uint64)
    z = np.zeros_like(p)
    seed = int(seed)
    sample = int(sample)
    w = philox4x32_10(p, z + tag, z + (sample & MASK32), z + (sample >> 32),
                      seed & MASK32, seed >> 32)
    return np.stack(w, axis=1)


def uniforms(words):
    """53-bit uniforms (u1 in (0,1], u2 in [0,1)) from Philox words."""
    w = words.astype(np.uint64)
    k1 = ((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(11)
    k2 = ((w[:, 2] << np.uint64(32)) | w[:, 3]) >> np.uint64(11)
    u1 = (k1.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = k2.astype(np.float64) * 2.0 ** -53
    return u1, u2


def normals(ncells, seed, sample):
    """Standard normals xi[ncells] of one sample (Box-Muller on the pair)."""
    u1, u2 = uniforms(noise_words(ncells, seed, sample))
    r = np.sqrt(-2.0 * np.log(u1))
    xi = np.empty(2 * len(u1))
    xi[0::2] = r * np.cos(2.0 * np.pi * u2)
    xi[1::2] = r * np.sin(2.0 * np.pi * u2)
    return xi[:ncells]


def normals_batch(ncells, seed, first_sample, nsamples):
    return np.stack([normals(ncells, seed, first_sample + s) for s in range(nsamples)])
