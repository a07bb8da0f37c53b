"""Seeded synthetic prostate HDR geometry and the point-source dose-rate matrix.

The paper optimises clinical cases (562 patients, Sec. 2.1.1) that are not available here.
This module builds seeded stand-ins with the sizes of the paper's workloads (mean 171 dwell
positions, 2753-15998 optimisation points, Sec. 2.1.1) and the structure set of Table 1
(target = prostate, urethra, rectum, bladder).

Recipe (one deterministic function of the seed):
  * prostate: ellipsoid, semi-axes (a, b, c) = (2.0, 1.5, 1.75) cm along (x lateral,
    y anterior, z superior), centred at the origin;
  * urethra: cylinder of radius 0.3 cm on the z axis, |z| <= c;
  * rectum: cylinder of radius 1.5 cm parallel to z, with a 0.3 cm gap behind the
    prostate's posterior surface (axis at y = -(b + 0.3 + 1.5)), |z| <= 3 cm;
  * bladder: sphere of radius 2 cm tangent to the prostate base, centre (0, 0, c + 2);
  * dose points: uniform rejection sampling, one structure id per point (the "i-th point
    in the j-th organ" of Eq. (dose)); prostate points exclude the urethra, rectum and
    bladder points exclude the prostate, bladder points exclude the rectum;
  * catheters: parallel to z on a 0.5 cm template grid inside the prostate cross-section
    shrunk by 0.3 cm and at least 0.5 cm from the urethra axis; n of them are picked by
    deterministic farthest-point selection;
  * dwell positions: every `dwell_step` cm along each catheter over the prostate's
    cranio-caudal extent |z| <= c;
  * dose rate (an input of the solver, step (i) of Sec. 2.2.1):
    A_il = Lambda * S_K * g(r) / r^2, r = max(|p_i - q_l|, 0.1 cm),
    g(r) = 1 + 0.005 r - 0.002 r^2, Lambda = 1.109 cGy h^-1 U^-1, S_K = 40700 U,
    converted from cGy/h to Gy/s (divide by 360000) so that dwell times are seconds.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STRUCTURES = ("prostate", "urethra", "rectum", "bladder")
BASE_SEED = 1904015670

LAMBDA = 1.109            # dose-rate constant, cGy h^-1 U^-1
S_K = 40700.0             # air-kerma strength, U
CGYH_TO_GYS = 1.0 / 360000.0
R_MIN_CM = 0.1
RX_GY = 15.0              # prescription dose (Sec. 2.1.1)


@dataclass
class Geometry:
    a: float = 2.0
    b: float = 1.5
    c: float = 1.75
    urethra_r: float = 0.3
    rectum_r: float = 1.5
    rectum_gap: float = 0.3
    rectum_half_len: float = 3.0
    bladder_r: float = 2.0

    def scaled(self, f: float) -> "Geometry":
        return Geometry(a=self.a * f, b=self.b * f, c=self.c * f,
                        urethra_r=self.urethra_r, rectum_r=self.rectum_r,
                        rectum_gap=self.rectum_gap,
                        rectum_half_len=self.rectum_half_len * f,
                        bladder_r=self.bladder_r * f)

    @property
    def rectum_y(self) -> float:
        return -(self.b + self.rectum_gap + self.rectum_r)

    @property
    def bladder_z(self) -> float:
        return self.c + self.bladder_r

    def in_prostate(self, p):
        return (p[:, 0] / self.a) ** 2 + (p[:, 1] / self.b) ** 2 + (p[:, 2] / self.c) ** 2 <= 1.0

    def in_urethra(self, p):
        return (p[:, 0] ** 2 + p[:, 1] ** 2 <= self.urethra_r ** 2) & (np.abs(p[:, 2]) <= self.c)

    def in_rectum(self, p):
        return ((p[:, 0] ** 2 + (p[:, 1] - self.rectum_y) ** 2 <= self.rectum_r ** 2)
                & (np.abs(p[:, 2]) <= self.rectum_half_len))

    def in_bladder(self, p):
        return p[:, 0] ** 2 + p[:, 1] ** 2 + (p[:, 2] - self.bladder_z) ** 2 <= self.bladder_r ** 2

    def volumes_cc(self) -> np.ndarray:
        """Analytic structure volumes (cm^3), used to turn point fractions into cc."""
        v_pro = 4.0 / 3.0 * np.pi * self.a * self.b * self.c
        v_ure = np.pi * self.urethra_r ** 2 * 2.0 * self.c
        v_rec = np.pi * self.rectum_r ** 2 * 2.0 * self.rectum_half_len
        v_bla = 4.0 / 3.0 * np.pi * self.bladder_r ** 3
        return np.array([v_pro - v_ure, v_ure, v_rec, v_bla])


@dataclass
class Patient:
    geometry: Geometry
    points: np.ndarray        # (N_p, 3) cm
    sid: np.ndarray           # (N_p,) int32 structure id, 0..3 in STRUCTURES order
    dwells: np.ndarray        # (N_d, 3) cm
    catheter: np.ndarray      # (N_d,) int32 catheter index of each dwell position
    catheter_xy: np.ndarray   # (n_cat, 2) cm
    A: np.ndarray             # (N_p, N_d) float32 dose-rate matrix, Gy/s (the problem's A)
    params: np.ndarray        # (S, 4) float64 per structure (w_min, D_min, D_max, w_max)
    volumes_cc: np.ndarray    # (S,) analytic volumes

    @property
    def n_pnt(self) -> int:
        return int(self.A.shape[0])

    @property
    def n_dwell(self) -> int:
        return int(self.A.shape[1])

    @property
    def n_per_struct(self) -> np.ndarray:
        return np.bincount(self.sid, minlength=len(STRUCTURES)).astype(np.int64)


def radial_g(r):
    return 1.0 + 0.005 * r - 0.002 * r * r


def dose_rate_matrix(points: np.ndarray, dwells: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Isotropic point-source dose rate in Gy/s, float64, shape (N_p, N_d)."""
    out = np.empty((points.shape[0], dwells.shape[0]), dtype=np.float64)
    for i0 in range(0, points.shape[0], chunk):
        p = points[i0:i0 + chunk]
        diff = p[:, None, :] - dwells[None, :, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
        r = np.maximum(r, R_MIN_CM)
        g = radial_g(r)
        if not np.all(g > 0):
            raise ValueError("radial function g(r) <= 0: geometry too large for the model")
        out[i0:i0 + chunk] = LAMBDA * S_K * g / (r * r) * CGYH_TO_GYS
    return out


def class_penalty_params() -> np.ndarray:
    """One-sided thresholds per structure with unit w_min / w_max.

    prostate D >= 100 % Rx, urethra D <= 110 %, rectum and bladder D <= 75 %.
    Columns: (w_min, D_min, D_max, w_max); an infinite bound disables that side.
    """
    inf = np.inf
    return np.array([
        [1.0, 1.00 * RX_GY, inf, 1.0],
        [1.0, -inf, 1.10 * RX_GY, 1.0],
        [1.0, -inf, 0.75 * RX_GY, 1.0],
        [1.0, -inf, 0.75 * RX_GY, 1.0],
    ])


# The paper's class solution (Table 1) for a 15 Gy prostate boost: per organ, the quadratic
# objectives of Eq. (1) on its surface and on its volume dose calculation points,
# (w_min, D_min, D_max, w_max) with doses in Gy.
TABLE1 = {
    "prostate": ((200.0, 15.0, 22.5, 80.0), (200.0, 15.0, 22.5, 1.0)),
    "urethra": ((30.0, 14.0, 16.0, 160.0), (30.0, 14.0, 16.0, 160.0)),
    "bladder": ((0.0, 0.0, 7.5, 60.0), (0.0, 0.0, 7.5, 60.0)),
    "rectum": ((0.0, 0.0, 7.5, 15.0), (0.0, 0.0, 7.5, 15.0)),
}


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def surface_points(g: "Geometry", rng, n_per_organ) -> list:
    """Dose points on each organ's surface, in STRUCTURES order: the prostate ellipsoid, the
    urethra and rectum cylinders (side walls), the bladder sphere."""
    n_pro, n_ure, n_rec, n_bla = n_per_organ
    pro = _unit_vectors(rng, n_pro) * np.array([g.a, g.b, g.c])
    th = rng.uniform(0.0, 2.0 * np.pi, n_ure)
    ure = np.column_stack([g.urethra_r * np.cos(th), g.urethra_r * np.sin(th),
                           rng.uniform(-g.c, g.c, n_ure)])
    th = rng.uniform(0.0, 2.0 * np.pi, n_rec)
    rec = np.column_stack([g.rectum_r * np.cos(th), g.rectum_y + g.rectum_r * np.sin(th),
                           rng.uniform(-g.rectum_half_len, g.rectum_half_len, n_rec)])
    bla = _unit_vectors(rng, n_bla) * g.bladder_r + np.array([0.0, 0.0, g.bladder_z])
    return [pro, ure, rec, bla]


def make_class_solution_patient(seed: int, n_catheters: int = 12, dwell_step: float = 0.5,
                                n_volume=(1200, 200, 300, 300), n_surface=(300, 100, 200, 200),
                                scale: float = 1.0) -> Patient:
    """A patient with the paper's full class solution (Table 1): eight point groups, the
    surface (group 2 s) and volume (group 2 s + 1) points of organ s in STRUCTURES order, each
    with its own two-sided objective.  `organ` of the returned record maps groups to organs."""
    base = make_patient(seed, n_catheters, dwell_step, n_volume, scale)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    surf = surface_points(base.geometry, rng, n_surface)
    groups, sid, params = [], [], []
    for s, name in enumerate(STRUCTURES):
        groups += [surf[s], base.points[base.sid == s]]
        sid += [np.full(len(surf[s]), 2 * s, np.int32), np.full(int(np.sum(base.sid == s)), 2 * s + 1, np.int32)]
        params += [TABLE1[name][0], TABLE1[name][1]]
    points = np.concatenate(groups, axis=0)
    A64 = dose_rate_matrix(points, base.dwells)
    pat = Patient(geometry=base.geometry, points=points, sid=np.concatenate(sid), dwells=base.dwells,
                  catheter=base.catheter, catheter_xy=base.catheter_xy, A=A64.astype(np.float32),
                  params=np.array(params, dtype=np.float64), volumes_cc=base.volumes_cc)
    pat.organ = np.repeat(np.arange(len(STRUCTURES)), 2)
    return pat


def group_weights(organ_weights, sid, organ) -> np.ndarray:
    """Per-group hidden weights for the library (which normalises each group by its own point
    count) that reproduce Eq. (obj)'s per-organ normalisation: w_group = w_organ N_group / N_organ."""
    n_group = np.bincount(sid, minlength=len(organ)).astype(np.float64)
    n_organ = np.bincount(organ, weights=n_group)
    w = np.asarray(organ_weights, dtype=np.float64)
    return (w[..., organ] * (n_group / n_organ[organ])).astype(np.float32)


def _sample_points(rng, n, lo, hi, accept):
    out = np.empty((0, 3))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    while out.shape[0] < n:
        cand = lo + (hi - lo) * rng.random((max(2 * (n - out.shape[0]), 256), 3))
        out = np.concatenate([out, cand[accept(cand)]], axis=0)
    return out[:n]


def _catheter_xy(g: Geometry, n: int, margin: float = 0.3, urethra_clear: float = 0.5):
    spacing = 0.5
    while True:
        kx = int(np.floor(g.a / spacing))
        ky = int(np.floor(g.b / spacing))
        xs = np.arange(-kx, kx + 1) * spacing
        ys = np.arange(-ky, ky + 1) * spacing
        X, Y = np.meshgrid(xs, ys)           # row-major: y outer, x inner
        X = X.ravel()
        Y = Y.ravel()
        ok = ((X / (g.a - margin)) ** 2 + (Y / (g.b - margin)) ** 2 <= 1.0) & \
             (np.hypot(X, Y) >= urethra_clear - 1e-9)
        cand = np.stack([X[ok], Y[ok]], axis=1)
        if cand.shape[0] >= n:
            break
        spacing *= 0.5
    # deterministic farthest-point selection, seeded at the candidate farthest from the axis
    r = np.hypot(cand[:, 0], cand[:, 1])
    chosen = [int(np.argmax(r))]
    dmin = np.hypot(cand[:, 0] - cand[chosen[0], 0], cand[:, 1] - cand[chosen[0], 1])
    for _ in range(n - 1):
        j = int(np.argmax(dmin))
        chosen.append(j)
        dmin = np.minimum(dmin, np.hypot(cand[:, 0] - cand[j, 0], cand[:, 1] - cand[j, 1]))
    return cand[chosen]


def dwell_positions(g: Geometry, n_catheters: int, dwell_step: float):
    """(dwells (N_d, 3) cm, catheter index of each, catheter xy): n catheters parallel to z
    (template grid, farthest-point selection), dwell positions every `dwell_step` cm over the
    prostate's cranio-caudal extent |z| <= c."""
    cxy = _catheter_xy(g, n_catheters)
    n_z = int(np.floor(2.0 * g.c / dwell_step + 1e-9)) + 1
    zs = (np.arange(n_z) - 0.5 * (n_z - 1)) * dwell_step
    dwells = np.array([[x, y, z] for (x, y) in cxy for z in zs])
    catheter = np.repeat(np.arange(len(cxy), dtype=np.int32), n_z)
    return dwells, catheter, cxy


def make_patient(seed: int, n_catheters: int = 12, dwell_step: float = 0.5,
                 n_points=(1200, 200, 300, 300), scale: float = 1.0) -> Patient:
    geom = Geometry().scaled(scale)
    ss = np.random.SeedSequence(seed)
    rngs = [np.random.default_rng(s) for s in ss.spawn(len(STRUCTURES))]
    g = geom
    pro = _sample_points(rngs[0], n_points[0], (-g.a, -g.b, -g.c), (g.a, g.b, g.c),
                         lambda p: g.in_prostate(p) & ~g.in_urethra(p))
    ure = _sample_points(rngs[1], n_points[1], (-g.urethra_r, -g.urethra_r, -g.c),
                         (g.urethra_r, g.urethra_r, g.c), g.in_urethra)
    rec = _sample_points(rngs[2], n_points[2],
                         (-g.rectum_r, g.rectum_y - g.rectum_r, -g.rectum_half_len),
                         (g.rectum_r, g.rectum_y + g.rectum_r, g.rectum_half_len),
                         lambda p: g.in_rectum(p) & ~g.in_prostate(p))
    bla = _sample_points(rngs[3], n_points[3],
                         (-g.bladder_r, -g.bladder_r, g.bladder_z - g.bladder_r),
                         (g.bladder_r, g.bladder_r, g.bladder_z + g.bladder_r),
                         lambda p: g.in_bladder(p) & ~g.in_prostate(p) & ~g.in_rectum(p))
    points = np.concatenate([pro, ure, rec, bla], axis=0)
    sid = np.concatenate([np.full(len(x), s, dtype=np.int32)
                          for s, x in enumerate((pro, ure, rec, bla))])

    dwells, catheter, cxy = dwell_positions(g, n_catheters, dwell_step)

    A64 = dose_rate_matrix(points, dwells)
    return Patient(geometry=geom, points=points, sid=sid, dwells=dwells, catheter=catheter,
                   catheter_xy=cxy, A=A64.astype(np.float32), params=class_penalty_params(),
                   volumes_cc=geom.volumes_cc())


def weights_loguniform(seed: int, n_plans: int, n_struct: int = 4, lo: float = 0.1,
                       hi: float = 10.0) -> np.ndarray:
    """Hidden weights, each drawn log-uniformly in [lo, hi]; shape (P, S), float32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    e = rng.uniform(np.log10(lo), np.log10(hi), size=(n_plans, n_struct))
    return (10.0 ** e).astype(np.float32)


def weights_dirichlet(seed: int, n_plans: int, n_struct: int = 4, alpha: float = 1.0,
                      scale: float = 10.0) -> np.ndarray:
    """Hidden weights drawn Dirichlet(alpha) over the structures and scaled; (P, S) float32.

    Dirichlet(1) is drawn as normalised Exp(1) variates (alpha = 1) or Gamma(alpha).
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 2]))
    e = rng.gamma(alpha, 1.0, size=(n_plans, n_struct))
    return (scale * e / e.sum(axis=1, keepdims=True)).astype(np.float32)


# Named workloads.  Each is a dict of generator parameters and solver settings.
WORKLOADS = {
    # one prostate, 12 catheters, 0.5 cm step (96 dwells), 2000 points, 8 log-uniform plans
    "prostate-2k-8plans": dict(seed=BASE_SEED + 0, n_catheters=12, dwell_step=0.5,
                               n_points=(1200, 200, 300, 300), n_plans=8,
                               weights="loguniform", max_iters=200, tol=0.0, m=10),
    # paper-scale batch: 18 catheters, 0.2 cm step (324 dwells), 12000 points, 1000 plans
    "prostate-12k-1000plans": dict(seed=BASE_SEED + 1, n_catheters=18, dwell_step=0.2,
                                   n_points=(7000, 1000, 2000, 2000), n_plans=1000,
                                   weights="dirichlet", max_iters=500, tol=1e-6, m=10),
}


def workload(name: str, n_plans: int | None = None):
    """Return (patient, weights[P,S], settings) for a named workload."""
    w = dict(WORKLOADS[name])
    pat = make_patient(w["seed"], w["n_catheters"], w["dwell_step"], w["n_points"])
    P = w["n_plans"] if n_plans is None else n_plans
    if w["weights"] == "loguniform":
        W = weights_loguniform(w["seed"], P)
    else:
        W = weights_dirichlet(w["seed"], P)
    return pat, W, w


def multi_patient_specs(n_patients: int = 64, seed: int = BASE_SEED + 3):
    """Uneven patient specs: catheters U{12..20}, isotropic scale U[0.8, 1.3], points
    U[5000, 20000] split 7:1:2:2 over (prostate, urethra, rectum, bladder)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3]))
    specs = []
    for k in range(n_patients):
        n_cat = int(rng.integers(12, 21))
        f = float(rng.uniform(0.8, 1.3))
        n_tot = int(rng.integers(5000, 20001))
        n_u = n_tot // 12
        n_r = n_b = 2 * n_tot // 12
        n_p = n_tot - n_u - n_r - n_b
        specs.append(dict(seed=seed * 1000 + k, n_catheters=n_cat, dwell_step=0.2,
                          n_points=(n_p, n_u, n_r, n_b), scale=f))
    return specs


def dwell_features(pat: Patient) -> np.ndarray:
    """The 10 per-dwell input features of the warm-start network, (n_dwell, 10) float32:
    signed distances (cm, negative inside) to the prostate surface, the urethra, the rectum
    and the bladder; depth along the catheter (0 at its first dwell, 1 at its last); x, y, z
    (cm); the prostate's size (cube root of a b c, cm); and the dwell density (dwell
    positions per cm^3 of prostate).  The prostate distance is the radial one, exact for a
    sphere."""
    g = pat.geometry
    p = pat.dwells
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    s = np.sqrt((x / g.a) ** 2 + (y / g.b) ** 2 + (z / g.c) ** 2)
    d_pro = np.where(s > 1e-9, (s - 1.0) * r / np.maximum(s, 1e-9), -min(g.a, g.b, g.c))
    d_ure = np.sqrt(x * x + y * y) - g.urethra_r
    d_rec = np.sqrt(x * x + (y - g.rectum_y) ** 2) - g.rectum_r
    d_bla = np.sqrt(x * x + y * y + (z - g.bladder_z) ** 2) - g.bladder_r
    depth = np.zeros(len(p))
    for c in np.unique(pat.catheter):
        m = pat.catheter == c
        zc = z[m]
        span = zc.max() - zc.min()
        depth[m] = (zc - zc.min()) / span if span > 0 else 0.0
    size = np.full(len(p), (g.a * g.b * g.c) ** (1.0 / 3.0))
    density = np.full(len(p), len(p) / (4.0 / 3.0 * np.pi * g.a * g.b * g.c))
    return np.stack([d_pro, d_ure, d_rec, d_bla, depth, x, y, z, size, density], axis=1).astype(np.float32)


def mlp_init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters of the warm-start network in the C ABI's layout (W_1 [14][128],
    b_1, W_2 [128][128], b_2, W_3, b_3, w_4 [128], b_4): weights uniform in +-sqrt(6 / fan_in)
    / 2, hidden biases 0, output weights uniform in +-1 / sqrt(128), output bias such that
    softplus(b_4) = 1 s."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    parts = []
    for fan_in, fan_out in ((14, 128), (128, 128), (128, 128)):
        lim = 0.5 * np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    parts.append(rng.uniform(-1.0, 1.0, 128) / np.sqrt(128.0))
    parts.append(np.array([np.log(np.expm1(1.0))]))
    return np.concatenate(parts).astype(np.float32)
