"""Pins of the point-sampling oracle (oracle/points.py) against what the rule and the
mathematics fix: the generator's published definition, the counts, membership of every point in
its structure (in FP64), the prefix property of "the i-th accepted candidate", and the symmetry
and uniformity a uniform sample of these shapes must show."""
import numpy as np
import pytest

import oracle
from oracle import points as OP
from synth import Geometry

SEED = 20260514


def _geo(scale=1.0):
    g = Geometry().scaled(scale)
    return {k: getattr(g, k) for k in OP.KEYS}


def test_splitmix64_vectorised_equals_published_and_c():
    # published first outputs (seed 1234567) and the C oracle's generator at large counters
    assert OP.splitmix64(1234567, [0, 1]).tolist() == [6457827717110365317, 3203168211198807973]
    rng = np.random.default_rng(0)
    for seed in (0, 1, 2**63 + 5, 1904015670):
        n = np.concatenate([np.arange(5), rng.integers(0, 2**62, 20)]).astype(np.uint64)
        n[-1] = (3 << 40) + 4 * 123456 + 2
        assert [int(v) for v in OP.splitmix64(seed, n)] == [oracle.splitmix64(seed, int(k)) for k in n]


@pytest.mark.parametrize("scale", [0.8, 1.0, 1.3])
def test_counts_membership_and_exclusions(scale):
    g = _geo(scale)
    counts = (1500, 250, 500, 401)
    P, sid = OP.sample_points(g, counts, SEED)
    assert P.dtype == np.float32 and P.shape == (sum(counts), 3)
    assert np.bincount(sid, minlength=4).tolist() == list(counts)
    assert np.all(np.diff(sid) >= 0)                      # structure-major
    x, y, z = [P[:, a].astype(np.float64) for a in range(3)]
    e = 1e-5   # float32 decisions near a boundary
    ell = (x / g["a"]) ** 2 + (y / g["b"]) ** 2 + (z / g["c"]) ** 2
    ure = np.hypot(x, y) ** 2 / g["urethra_r"] ** 2
    rec = (x ** 2 + (y - g["rectum_y"]) ** 2) / g["rectum_r"] ** 2
    bla = (x ** 2 + y ** 2 + (z - g["bladder_z"]) ** 2) / g["bladder_r"] ** 2
    pro, uu, rr, bb = (sid == s for s in range(4))
    assert np.all(ell[pro] <= 1 + e) and np.all((ure[pro] >= 1 - e) | (np.abs(z[pro]) > g["c"] - e))
    assert np.all(ure[uu] <= 1 + e) and np.all(np.abs(z[uu]) <= g["c"] + e)
    assert np.all(rec[rr] <= 1 + e) and np.all(np.abs(z[rr]) <= g["rectum_half_len"] + e)
    assert np.all(ell[rr] >= 1 - e)
    out_rec = (rec >= 1 - e) | (np.abs(z) >= g["rectum_half_len"] - e)
    assert np.all(bla[bb] <= 1 + e) and np.all(ell[bb] >= 1 - e) and np.all(out_rec[bb])


def test_prefix_property_and_seed_dependence():
    """Point i is the i-th accepted candidate: more points extend the sample, never reorder it;
    another seed gives other points."""
    g = _geo()
    a, sa = OP.sample_points(g, (300, 40, 80, 60), SEED)
    b, sb = OP.sample_points(g, (337, 41, 95, 60), SEED)
    off_a, off_b = np.cumsum([0, 300, 40, 80]), np.cumsum([0, 337, 41, 95])
    for s, n in enumerate((300, 40, 80, 60)):
        assert np.array_equal(a[off_a[s]:off_a[s] + n], b[off_b[s]:off_b[s] + n])
    c, _ = OP.sample_points(g, (300, 40, 80, 60), SEED + 1)
    assert not np.any(np.all(a == c, axis=1))
    # a count of zero leaves the structure out
    d, sd = OP.sample_points(g, (0, 40, 0, 60), SEED)
    assert np.bincount(sd, minlength=4).tolist() == [0, 40, 0, 60]
    assert np.array_equal(d[:40], a[300:340])


def test_symmetry_and_uniformity():
    """Uniform samples of these shapes: octant balance where the structure is symmetric, the
    analytic centroids, and the radial law of a uniform ball (fraction within half the radius
    = 1/8) on the bladder, whose excluded parts are negligible."""
    g = _geo()
    counts = (16000, 4000, 8000, 8000)
    P, sid = OP.sample_points(g, counts, SEED)
    x, y, z = [P[:, a].astype(np.float64) for a in range(3)]

    def balanced(mask, v, n):
        k = np.sum(v[mask] > 0)
        return abs(k - n / 2) <= 4.0 * np.sqrt(n / 4)

    pro, uu, rr, bb = (sid == s for s in range(4))
    for v in (x, y, z):
        assert balanced(pro, v, counts[0]) and balanced(uu, v, counts[1])
    assert balanced(rr, x, counts[2]) and balanced(rr, z, counts[2])
    assert balanced(bb, x, counts[3]) and balanced(bb, y, counts[3])
    assert abs(np.mean(y[rr]) - g["rectum_y"]) < 0.05
    # uniform ball: P(r <= R/2) = 1/8; the prostate cuts off a sliver near the base (< 0.1 %)
    r = np.sqrt(x[bb] ** 2 + y[bb] ** 2 + (z[bb] - g["bladder_z"]) ** 2) / g["bladder_r"]
    f = np.mean(r <= 0.5)
    assert abs(f - 0.125) <= 4.0 * np.sqrt(0.125 * 0.875 / counts[3])
    # uniform cylinder (the urethra excludes nothing): E[(x^2 + y^2) / r^2] = 1/2, E[z^2 / c^2] = 1/3
    n_u = counts[1]
    q = (x[uu] ** 2 + y[uu] ** 2) / g["urethra_r"] ** 2
    assert abs(np.mean(q) - 0.5) <= 4.0 * np.sqrt(1.0 / 12.0 / n_u)
    w = z[uu] ** 2 / g["c"] ** 2
    assert abs(np.mean(w) - 1.0 / 3.0) <= 4.0 * np.sqrt(4.0 / 45.0 / n_u)


def test_degenerate_structure_is_refused():
    g = _geo()
    g["rectum_y"] = 0.0   # a rectum inside the prostate: every candidate is excluded
    g["rectum_r"] = 0.2
    g["rectum_half_len"] = 1.0
    with pytest.raises(ValueError):
        OP.sample_points(g, (10, 10, 2000, 10), SEED)
