"""Counter-based splitmix64 streams, uniforms and Box-Muller normals (numpy, vectorised)."""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix64(z):
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _mix64_int(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def _fnv1a(s: str) -> int:
    h = 0xCBF29CE484222325
    for c in s.encode():
        h ^= c
        h = (h * 0x100000001B3) & _MASK
    return h


def derive_key(seed: int, *tags) -> int:
    """Key of an independent stream named by (seed, tag, tag, ...)."""
    k = _mix64_int(int(seed) + 0x9E3779B97F4A7C15)
    for t in tags:
        t = _fnv1a(t) if isinstance(t, str) else int(t)
        k = _mix64_int(k ^ t)
    return k


def raw64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the stream `key` as uint64."""
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + ctr * _GAMMA)


def uniform01(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    u = raw64(key, n, offset) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller: pair (u1, u2) -> sqrt(-2 ln u1) cos(2 pi u2)."""
    u = uniform01(key, 2 * n, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def randint(key: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on {lo, ..., hi} (inclusive), by scaling a uniform."""
    u = uniform01(key, n)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64).clip(lo, hi)


def permutation(key: int, n: int) -> np.ndarray:
    """Fisher-Yates shuffle of 0..n-1 driven by the stream `key`."""
    p = np.arange(n, dtype=np.int64)
    u = uniform01(key, n)
    for i in range(n - 1, 0, -1):
        j = int(u[i] * (i + 1))
        j = min(j, i)
        p[i], p[j] = p[j], p[i]
    return p
