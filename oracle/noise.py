"""Noise synthesis (K.5 of the draft).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per 256 x 256 group (6.2; smaller at the right and bottom edges): three
pseudorandom channels RR, RG, RB from eight XorShift128+ generators seeded by
SplitMix64 from the group origin (K.5.2), each convolved with the 5x5
Laplacian-like kernel (centre -4, 1 at distance 2 on the axes) with the
group's bounds mirrored (6.5), then the additive update of K.5.3 on the XYB
samples.

READING (the generator): the printed update keeps s0 constant, which is not
an XorShift128+ generator; the published generator rotates its two state
words at every step.  Here each step first exchanges s0 and s1, then applies
the printed operations (s1 ^= s1 << 23; batch = s1 + s0; s1 ^= s0 ^
(s1 >> 18) ^ (s0 >> 5)).  The draft prints no generator output, so the bit
stream is "parity unpinned" against any other decoder; SplitMix64 is pinned
to its published first output.

READING (the strength): in_frac is taken from the unclamped product and only
in_int is clamped to [0, 14], as printed (the strength is discontinuous at
integers outside [0, 15)).
"""
import numpy as np

M64 = (1 << 64) - 1
GROUP = 256
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(z):
    """The SplitMix64 mixing function of K.5.2 on a Python int."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def seed_state(x0, y0):
    """s0[i], s1[i] for the group whose top-left pixel is (x0, y0)."""
    seed = ((y0 << 32) + x0) & M64
    s0 = [0] * 8
    s1 = [0] * 8
    s0[0] = splitmix64(seed + GOLDEN_GAMMA)
    s1[0] = splitmix64(s0[0])
    for i in range(1, 8):
        s0[i] = splitmix64(s1[i - 1])
        s1[i] = splitmix64(s0[i])
    return np.array(s0, dtype=np.uint64), np.array(s1, dtype=np.uint64)


def step(s0, s1):
    """One step of the eight generators (READING above).  Returns the new
    state and batch[0..8)."""
    s0, s1 = s1.copy(), s0.copy()
    s1 ^= s1 << np.uint64(23)
    batch = s1 + s0                               # wraps modulo 2^64
    s1 ^= s0 ^ (s1 >> np.uint64(18)) ^ (s0 >> np.uint64(5))
    return s0, s1, batch


def random_channels(x0, y0, w, h):
    """RR, RG, RB of one group, (3, h, w) binary32 values in [0, 1)."""
    s0, s1 = seed_state(x0, y0)
    out = np.zeros((3, h, w), dtype=np.float32)
    for c in range(3):
        for y in range(h):
            for seg in range(0, w, 16):
                s0, s1, batch = step(s0, s1)
                lo = (batch & np.uint64(0xFFFFFFFF)).astype(np.uint32)
                hi = (batch >> np.uint64(32)).astype(np.uint32)
                bits = np.empty(16, dtype=np.uint32)
                bits[0::2] = lo
                bits[1::2] = hi
                n = min(16, w - seg)
                f = ((bits[:n] >> np.uint32(9)) | np.uint32(0x3F800000)).view(np.float32)
                out[c, y, seg:seg + n] = f - np.float32(1.0)
    return out


def _mirror(i, n):
    while i < 0 or i >= n:
        i = -i - 1 if i < 0 else 2 * n - 1 - i
    return i


def laplacian(ch):
    """The 5x5 kernel of K.5.2 on one group channel (FP64), 6.5 mirroring at
    the group's bounds."""
    h, w = ch.shape
    x = ch.astype(np.float64)
    ym = lambda d: np.array([_mirror(y + d, h) for y in range(h)])
    xm = lambda d: np.array([_mirror(i + d, w) for i in range(w)])
    return (x[ym(-2)] + x[ym(2)] + x[:, xm(-2)] + x[:, xm(2)] - 4.0 * x)


def strength(v, lut):
    """K.5.3 strength for In = v (READING above)."""
    s = v * 14.0
    i = np.floor(s)
    f = s - i
    i = np.clip(i, 0, 14).astype(np.int64)
    lut = np.asarray(lut, dtype=np.float64)
    return np.clip(lut[i] * (1.0 - f) + lut[i + 1] * f, 0.0, 1.0)


def add_noise(xyb, lut):
    """K.5 on a cropped XYB image (3, ys, xs), FP64; returns the new image."""
    _, ys, xs = xyb.shape
    out = xyb.astype(np.float64).copy()
    for y0 in range(0, ys, GROUP):
        for x0 in range(0, xs, GROUP):
            h, w = min(GROUP, ys - y0), min(GROUP, xs - x0)
            rnd = random_channels(x0, y0, w, h)
            a = [0.22 * laplacian(rnd[c]) for c in range(3)]
            X = out[0, y0:y0 + h, x0:x0 + w]
            Y = out[1, y0:y0 + h, x0:x0 + w]
            sr = strength(Y + X, lut)
            sg = strength(Y - X, lut)
            nr = 0.01 * a[0] * sr + 0.99 * a[2] * sr
            ng = 0.01 * a[1] * sg + 0.99 * a[2] * sg
            out[0, y0:y0 + h, x0:x0 + w] = X + (nr - ng)
            out[1, y0:y0 + h, x0:x0 + w] = Y + (nr + ng)
            out[2, y0:y0 + h, x0:x0 + w] += 0.935669 * (nr + ng)
    return out


def margins(xyb):
    """Distance of In x 14 from the integers where the strength jumps
    (outside [0, 15)), per pixel, min over R and G (for tests)."""
    X, Y = xyb[0].astype(np.float64), xyb[1].astype(np.float64)
    out = np.full(X.shape, np.inf)
    for v in (Y + X, Y - X):
        s = v * 14.0
        d = np.abs(s - np.round(s))
        jump = (np.round(s) <= 0) | (np.round(s) >= 15)
        out = np.minimum(out, np.where(jump, d, np.inf))
    return out
