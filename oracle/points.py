"""Dose calculation points of the analytic structures, restated from the sampling rule.  Test
infrastructure only.

Rule (the sampling half of step (i) of the planning flow, Sec. 2.2.1, on the workload's
analytic volumes): candidate k of structure s is lo + u w per axis in the structure's bounding
box, u = the top 24 bits of SplitMix64 output number s 2^40 + 4 k + axis, times 2^-24; point i
of structure s is its i-th accepted candidate in order of k.  Acceptance: prostate = inside the
ellipsoid and not in the urethra; urethra = inside its cylinder; rectum = inside its cylinder
and not in the prostate; bladder = inside its sphere and in neither the prostate nor the rectum.

The geometry is rounded to float32 and each step below is one float32 numpy operation (IEEE,
round to nearest), in the order the rule's membership tests are written, so the points come out
bit for bit as any IEEE float32 evaluation of the same steps gives them.  SplitMix64 follows its
published definition (Steele, Lea and Flood 2014): Weyl state seed + (n + 1) gamma, then the
variant-13 finaliser.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
KEYS = ("a", "b", "c", "urethra_r", "rectum_r", "rectum_y", "rectum_half_len", "bladder_r", "bladder_z")


def splitmix64(seed, n):
    """Outputs number n (uint64 array, 0-based) of SplitMix64 seeded with `seed`."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & (2**64 - 1)) + (n + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def _f32(geometry):
    get = (lambda k: geometry[k]) if isinstance(geometry, dict) else (lambda k: getattr(geometry, k))
    return {k: np.float32(get(k)) for k in KEYS}


def _in_prostate(g, x, y, z):
    s = (x / g["a"]) * (x / g["a"]) + (y / g["b"]) * (y / g["b"])
    return s + (z / g["c"]) * (z / g["c"]) <= np.float32(1.0)


def _in_urethra(g, x, y, z):
    return (x * x + y * y <= g["urethra_r"] * g["urethra_r"]) & (np.abs(z) <= g["c"])


def _in_rectum(g, x, y, z):
    dy = y - g["rectum_y"]
    return (x * x + dy * dy <= g["rectum_r"] * g["rectum_r"]) & (np.abs(z) <= g["rectum_half_len"])


def _in_bladder(g, x, y, z):
    dz = z - g["bladder_z"]
    return x * x + y * y + dz * dz <= g["bladder_r"] * g["bladder_r"]


def _box(g, s):
    """(lo, w): bounding box corner and widths of structure s, float32."""
    if s == 0:
        return (-g["a"], -g["b"], -g["c"]), (g["a"] + g["a"], g["b"] + g["b"], g["c"] + g["c"])
    if s == 1:
        r = g["urethra_r"]
        return (-r, -r, -g["c"]), (r + r, r + r, g["c"] + g["c"])
    if s == 2:
        r, h = g["rectum_r"], g["rectum_half_len"]
        return (-r, g["rectum_y"] - r, -h), (r + r, r + r, h + h)
    r = g["bladder_r"]
    return (-r, -r, g["bladder_z"] - r), (r + r, r + r, r + r)


def candidates(geometry, s, seed, K):
    """The first K candidates of structure s: (x, y, z float32 arrays, accepted flags)."""
    g = _f32(geometry)
    lo, w = _box(g, s)
    k = np.arange(K, dtype=np.uint64)
    p = []
    for a in range(3):
        n = (np.uint64(s) << np.uint64(40)) + np.uint64(4) * k + np.uint64(a)
        u = (splitmix64(seed, n) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
        p.append(lo[a] + u * w[a])
    x, y, z = p
    if s == 0:
        acc = _in_prostate(g, x, y, z) & ~_in_urethra(g, x, y, z)
    elif s == 1:
        acc = _in_urethra(g, x, y, z)
    elif s == 2:
        acc = _in_rectum(g, x, y, z) & ~_in_prostate(g, x, y, z)
    else:
        acc = _in_bladder(g, x, y, z) & ~_in_prostate(g, x, y, z) & ~_in_rectum(g, x, y, z)
    return x, y, z, acc


def sample_points(geometry, counts, seed):
    """(points (N x 3) float32, sid (N,) int32), structure-major, N = sum(counts)."""
    pts, sid = [], []
    for s, n in enumerate(counts):
        n = int(n)
        if n == 0:
            continue
        # the candidate budget starts at 3 n + 1024 and doubles while short, at most 7 times
        K = 3 * n + 1024
        for _ in range(8):
            x, y, z, acc = candidates(geometry, s, seed, K)
            idx = np.flatnonzero(acc)
            if idx.size >= n:
                break
            K *= 2
        else:
            raise ValueError(f"structure {s} accepts too few candidates")
        idx = idx[:n]
        pts.append(np.stack([x[idx], y[idx], z[idx]], axis=1))
        sid.append(np.full(n, s, np.int32))
    return np.concatenate(pts).astype(np.float32), np.concatenate(sid)
