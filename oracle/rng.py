"""Counter-based Rademacher noise from SplitMix64.

Sec. 1: the random noise vectors have a Rademacher distribution, +-1 with
probability 1/2 (Z2); for complex matrices Z4 vectors with values +-1, +-i,
each with probability 1/4.  The paper fixes the distribution only; the
generator is this implementation's choice:

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): with GAMMA = 0x9E3779B97F4A7C15, the n-th output
(n = 1, 2, ...) of a generator started at state S is mix64(S + n * GAMMA),
where mix64 is the published 64-bit finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
    z ^= z >> 27; z *= 0x94D049BB133111EB;
    z ^= z >> 31.
All arithmetic is modulo 2^64.

    key(seed, s)   = output s+1 of a generator started at `seed`
    h(seed, s, x)  = output x+1 of a generator started at key(seed, s)
    Z2: z = +1 if the top bit of h is 0, else -1
    Z4: z = i^(top two bits of h)       (0 -> 1, 1 -> i, 2 -> -1, 3 -> -i)

x is the storage index of the site; one value per site is shared by every
spin-colour component (the dilution of Sec. 4.2 is a Kronecker product with
the 12 x 12 identity).
"""
import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB


def mix64_int(z):
    """SplitMix64 finaliser on one Python int (exact, arbitrary precision)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def mix64(z):
    """SplitMix64 finaliser on a numpy uint64 array (wraps modulo 2^64)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(M2)
        z ^= z >> np.uint64(31)
    return z


def set_key(seed, s):
    return mix64_int((int(seed) + (int(s) + 1) * GAMMA) & MASK)


def site_hash(seed, s, N):
    """h(seed, s, x) for x = 0..N-1 as uint64."""
    key = np.uint64(set_key(seed, s))
    x = np.arange(N, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + (x + np.uint64(1)) * np.uint64(GAMMA)
    return mix64(state)


def z2(seed, s, N):
    h = site_hash(seed, s, N)
    return 1.0 - 2.0 * (h >> np.uint64(63)).astype(np.float64)


def z4(seed, s, N):
    h = site_hash(seed, s, N)
    q = (h >> np.uint64(62)).astype(np.int64)
    return np.array([1.0, 1.0j, -1.0, -1.0j], dtype=np.complex128)[q]


def noise(seed, s, N, kind):
    """kind 0 -> Z2 (real float64), kind 1 -> Z4 (complex128)."""
    if kind == 0:
        return z2(seed, s, N)
    if kind == 1:
        return z4(seed, s, N)
    raise ValueError("noise kind must be 0 (Z2) or 1 (Z4)")
