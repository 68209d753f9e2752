"""Synthetic phantom, breathing DVF family, PCA motion model and scan geometry.

The paper's test object is the NCAT phantom with demons-registered training
DVFs (Section 3). Neither is available, so this module generates a seeded
stand-in with the same structure: a 10-phase breathing cycle of a chest
phantom (body, two lungs, a tumor in the right lower lung, a spine), a
reference phase at end of exhale with zero DVF, PCA of the other nine phase
DVFs keeping K modes (Sections 2.1 and 3), and cone-beam projections at 1
degree steps of a one-minute gantry rotation (Section 3).

Conventions (every consumer uses them):
  * A volume is a C-ordered array [nz][ny][nx] (x fastest). Voxel (i, j, k)
    sits at origin + (i, j, k) * spacing with origin = -((n - 1) / 2) * spacing,
    so the isocentre is the volume centre. x = lateral (patient right = -x),
    y = anterior-posterior (+y posterior), z = superior-inferior (+z cranial).
  * A vector field is planar: [3][nz][ny][nx] in mm, component 0 = x.
  * Eigenvectors U are [K][3][nz][ny][nx]; u_k . u_k = N (N voxels), so w_k
    is in mm of RMS per-voxel displacement.
  * DVFs are pull-back fields: the deformed image at v is the reference image
    at v + x(v) (Section 2.3).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


# ----------------------------------------------------------------------------
# Grids and geometry
# ----------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Volume:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def spacing(self):
        return np.array([self.dx, self.dy, self.dz], dtype=np.float64)

    @property
    def origin(self):
        dims = np.array([self.nx, self.ny, self.nz], dtype=np.float64)
        return -0.5 * (dims - 1.0) * self.spacing

    @property
    def half_extent(self):
        dims = np.array([self.nx, self.ny, self.nz], dtype=np.float64)
        return 0.5 * dims * self.spacing

    def axes(self):
        """Voxel-centre coordinates (mm) along x, y and z."""
        o = self.origin
        return (
            o[0] + self.dx * np.arange(self.nx),
            o[1] + self.dy * np.arange(self.ny),
            o[2] + self.dz * np.arange(self.nz),
        )


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Flat-panel cone-beam geometry (mm). ds = ray sample step."""

    sad: float
    sdd: float
    nu: int
    nv: int
    du: float
    dv: float
    ds: float

    @property
    def n_rays(self):
        return self.nu * self.nv


# ----------------------------------------------------------------------------
# Chest phantom
# ----------------------------------------------------------------------------

MU_BODY = 0.02
MU_LUNG = 0.004
MU_TUMOR = 0.02
MU_SPINE = 0.04
TUMOR_DIAMETER = 10.0


def _structures(vol: Volume):
    """Structures in drawing order; a later one overrides an earlier one.

    Each is (kind, centre, semi-axes or radius, z half-length, mu).
    """
    hx, hy, hz = vol.half_extent
    return [
        ("ellipsoid", (0.0, 0.0, 0.0), (0.85 * hx, 0.60 * hy, 0.95 * hz), MU_BODY),
        ("ellipsoid", (+0.38 * hx, -0.05 * hy, 0.10 * hz), (0.30 * hx, 0.40 * hy, 0.60 * hz), MU_LUNG),
        ("ellipsoid", (-0.38 * hx, -0.05 * hy, 0.10 * hz), (0.30 * hx, 0.40 * hy, 0.60 * hz), MU_LUNG),
        ("ellipsoid", tuple(tumor_centre(vol)), (TUMOR_DIAMETER / 2,) * 3, MU_TUMOR),
        ("cylinder", (0.0, 0.45 * hy, 0.0), (0.08 * hx, 0.95 * hz), MU_SPINE),
    ]


def tumor_centre(vol: Volume) -> np.ndarray:
    """Tumor centre (mm) in the reference (end-of-exhale) image: right lower lung."""
    hx, hy, hz = vol.half_extent
    return np.array([-0.38 * hx, 0.0, -0.30 * hz], dtype=np.float64)


def _inside(kind, c, a, x, y, z):
    if kind == "ellipsoid":
        return ((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 + ((z - c[2]) / a[2]) ** 2 < 1.0
    r, zh = a
    return ((x - c[0]) ** 2 + (y - c[1]) ** 2 < r * r) & (np.abs(z - c[2]) < zh)


def _classify(kind, c, a, x, y, z, delta):
    """+1 surely inside, -1 surely outside, 0 ambiguous for every point within delta mm."""
    if kind == "ellipsoid":
        rho = np.sqrt(((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 + ((z - c[2]) / a[2]) ** 2)
        lip = delta / min(a)
        out = np.zeros(rho.shape, dtype=np.int8)
        out[rho + lip < 1.0] = 1
        out[rho - lip > 1.0] = -1
        return out
    r, zh = a
    rho = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2) / r
    dz = np.abs(z - c[2])
    lip = delta / r
    out = np.zeros(rho.shape, dtype=np.int8)
    out[(rho + lip < 1.0) & (dz + delta < zh)] = 1
    out[(rho - lip > 1.0) | (dz - delta > zh)] = -1
    return out


def phantom_point_values(vol: Volume, x, y, z) -> np.ndarray:
    """Attenuation (1/mm) of the analytic phantom at arbitrary points (mm)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    val = np.zeros(np.broadcast(x, y, z).shape, dtype=np.float64)
    for kind, c, a, mu in _structures(vol):
        val = np.where(_inside(kind, c, a, x, y, z), mu, val)
    return val


def phantom_volume(vol: Volume, subsamples: int = 4) -> np.ndarray:
    """Voxelised phantom [nz][ny][nx] (float64): each voxel is the mean over
    subsamples^3 points on a regular sub-grid of the voxel. Voxels that no
    structure boundary can cross take their centre value directly (the mean of
    identical sub-samples)."""
    ax, ay, az = vol.axes()
    delta = 0.5 * math.sqrt(vol.dx ** 2 + vol.dy ** 2 + vol.dz ** 2)
    out = np.empty(vol.shape, dtype=np.float64)
    offs = (np.arange(subsamples) + 0.5) / subsamples - 0.5
    sx, sy, sz = np.meshgrid(offs * vol.dx, offs * vol.dy, offs * vol.dz, indexing="ij")
    sx, sy, sz = sx.ravel(), sy.ravel(), sz.ravel()
    structs = _structures(vol)
    for k in range(vol.nz):  # one z-slab at a time bounds the memory
        z = np.full((vol.ny, vol.nx), az[k])
        y, x = np.meshgrid(ay, ax, indexing="ij")
        val = phantom_point_values(vol, x, y, z)
        ambiguous = np.zeros(val.shape, dtype=bool)
        for kind, c, a, mu in structs:
            ambiguous |= _classify(kind, c, a, x, y, z, delta) == 0
        iy, ix = np.nonzero(ambiguous)
        if iy.size:
            px = x[iy, ix][:, None] + sx[None, :]
            py = y[iy, ix][:, None] + sy[None, :]
            pz = z[iy, ix][:, None] + sz[None, :]
            val[iy, ix] = phantom_point_values(vol, px, py, pz).mean(axis=1)
        out[k] = val
    return out


# ----------------------------------------------------------------------------
# Breathing motion
# ----------------------------------------------------------------------------

PERIOD = 4.0  # s (Section 3: 4 s breathing period)
AMP_SI = 10.0  # mm, diaphragm peak SI displacement of the training cycle
AMP_AP = 3.0  # mm
AP_LAG = 0.4  # s


def breathing_phase(t):
    """s(t) = sin^4(pi t / 4 s): 0 at end of exhale (t = 0), 1 at end of inhale."""
    return np.sin(np.pi * np.asarray(t, dtype=np.float64) / PERIOD) ** 4


def dvf_analytic(vol: Volume, t: float, scale: float = 1.0, amp_si: float = AMP_SI,
                 amp_ap: float = AMP_AP, x=None, y=None, z=None) -> np.ndarray:
    """Analytic pull-back DVF at time t (mm), planar [3][...].

    SI: amp_si * s(t) * e(z, L(t)) * m(x, y); AP: amp_ap * (s(t - lag) - s(-lag)) *
    e(z, L0) * m(x, y); LR: 0, where e(z, L) = exp(-max(z - z_d, 0) / L) decays
    cranially from the diaphragm z_d = -0.5 Hz, L0 = 0.4 Hz, L(t) = L0 (1 + s(t)/2)
    and m = exp(-x^2/(0.9 Hx)^2 - y^2/(0.9 Hy)^2). The lag and the L(t) term give
    the nine training DVFs rank >= 3. Evaluated on the voxel grid unless points
    (x, y, z) are given.
    """
    hx, hy, hz = vol.half_extent
    if x is None:
        ax, ay, az = vol.axes()
        z, y, x = np.meshgrid(az, ay, ax, indexing="ij")
    s = float(breathing_phase(t))
    s_lag = float(breathing_phase(t - AP_LAG) - breathing_phase(-AP_LAG))
    zd = -0.5 * hz
    l0 = 0.4 * hz
    lt = l0 * (1.0 + 0.5 * s)
    above = np.maximum(z - zd, 0.0)
    m = np.exp(-(x / (0.9 * hx)) ** 2 - (y / (0.9 * hy)) ** 2)
    out = np.zeros((3,) + np.shape(x), dtype=np.float64)
    out[2] = scale * amp_si * s * np.exp(-above / lt) * m
    out[1] = scale * amp_ap * s_lag * np.exp(-above / l0) * m
    return out


def training_times(n_phases: int = 10) -> np.ndarray:
    """Phase times t_i = i * period / n_phases; phase 0 is the EOE reference."""
    return np.arange(n_phases) * (PERIOD / n_phases)


def training_dvfs(vol: Volume, amp_si: float = AMP_SI, amp_ap: float = AMP_AP,
                  n_phases: int = 10) -> np.ndarray:
    """The n_phases - 1 non-reference training DVFs, [n_phases-1][3][nz][ny][nx]."""
    ts = training_times(n_phases)[1:]
    return np.stack([dvf_analytic(vol, t, amp_si=amp_si, amp_ap=amp_ap) for t in ts])


# ----------------------------------------------------------------------------
# PCA motion model (Section 2.1, Eq. 1; Section 3: PCA of the nine DVFs, K = 3)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class PCAModel:
    mean: np.ndarray  # [3][nz][ny][nx] float64, mm
    U: np.ndarray  # [K][3][nz][ny][nx] float64, u_k . u_k = N
    sigma: np.ndarray  # [K] std-dev of the training coefficients (mm)
    eigvals: np.ndarray  # all Gram eigenvalues, descending
    coeffs: np.ndarray  # [n_train][K] training coefficients

    @property
    def K(self):
        return self.U.shape[0]

    def project(self, field: np.ndarray) -> np.ndarray:
        """Least-squares PCA coefficients of a DVF: u_k . (field - mean) / N."""
        n = field[0].size
        d = (field - self.mean).reshape(-1)
        return np.array([self.U[k].reshape(-1) @ d / n for k in range(self.K)])


def build_pca(train: np.ndarray, K: int) -> PCAModel:
    """PCA of training DVFs by the snapshot (Gram-matrix) method, in float64.

    mean = average of the training DVFs; u_k = eigenvectors of the sample
    covariance for the K largest eigenvalues, scaled to u_k . u_k = N and signed
    so that the SI component sums to >= 0.
    """
    m = train.shape[0]
    n = train[0, 0].size
    flat = train.reshape(m, -1).astype(np.float64)
    mean = flat.mean(axis=0)
    xc = flat - mean
    gram = xc @ xc.T
    lam, vec = np.linalg.eigh(gram)
    order = np.argsort(lam)[::-1]
    lam, vec = lam[order], vec[:, order]
    us = []
    for k in range(K):
        u = xc.T @ vec[:, k]
        u *= math.sqrt(n) / np.linalg.norm(u)
        if u.reshape(3, -1)[2].sum() < 0:
            u = -u
        us.append(u)
    U = np.stack(us)
    coeffs = xc @ U.T / n
    sigma = np.sqrt((coeffs ** 2).sum(axis=0) / (m - 1))
    shape = train.shape[1:]
    return PCAModel(mean=mean.reshape(shape), U=U.reshape((K,) + shape), sigma=sigma,
                    eigvals=lam, coeffs=coeffs)


def tumor_truth(vol: Volume, t: float, scale: float, amp_si: float = AMP_SI,
                amp_ap: float = AMP_AP) -> np.ndarray:
    """True tumor position at time t: the point p with p + x(p) = c0 for the
    analytic (continuous) field x, solved by Newton's method with a numerical
    Jacobian."""
    c0 = tumor_centre(vol)

    def resid(p):
        d = dvf_analytic(vol, t, scale, amp_si, amp_ap, x=np.array(p[0]), y=np.array(p[1]),
                         z=np.array(p[2]))
        return p + d.reshape(3) - c0

    p = c0.copy()
    for _ in range(50):
        r = resid(p)
        if np.max(np.abs(r)) < 1e-12:
            break
        jac = np.empty((3, 3))
        h = 1e-5
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            jac[:, c] = (resid(p + e) - resid(p - e)) / (2 * h)
        p = p - np.linalg.solve(jac, r)
    return p


def standard_normal(seed: int, shape) -> np.ndarray:
    """Standard-normal draws from numpy's default_rng(seed), C order."""
    return np.random.default_rng(seed).standard_normal(shape)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------


def workload_small(K: int = 3):
    """64^3 at 4 mm, K modes, SAD 1000 / SDD 1500 mm, 128x128 detector at 1.6 mm,
    ray step 2 mm; one projection at 0 deg of the 1.5x-amplitude phantom at t = 1 s,
    1% noise from seed 0, 30 iterations."""
    vol = Volume(64, 64, 64, 4.0, 4.0, 4.0)
    geom = Geometry(1000.0, 1500.0, 128, 128, 1.6, 1.6, 2.0)
    return dict(name="phantom 64^3 @ 4 mm, K=%d, 128x128 detector" % K, vol=vol, geom=geom, K=K,
                angle_deg=0.0, t=1.0, scale=1.5, seed=0, max_iters=30)


# Detector variants of the 40x30 cm panel (Section 3 down-samples to 200x150 at
# 2 mm; Section 5 compares 1000x750 at 0.4 mm).
# Samplings of the paper's 40 x 30 cm panel (Section 3): the benchmark's 512x384,
# the paper's down-sampled 200x150 at 2 mm, the 1000x750 of its resolution
# study, and the coarse 40x30 at 10 mm and 20x15 at 20 mm at and below the
# sampling where the paper reports the localisation degrading (Section 5).
DETECTORS = {"512x384": (512, 384, 0.776), "200x150": (200, 150, 2.0), "1000x750": (1000, 750, 0.4),
             "40x30": (40, 30, 10.0), "20x15": (20, 15, 20.0)}


def workload_paper(K: int = 3, detector: str = "512x384"):
    """Paper scale (Section 3): 256x256x120 at 2x2x2.5 mm, K modes, the 40x30 cm
    panel at 512x384 (0.776 mm; or one of DETECTORS), ray step 1 mm. Projection
    j is at gantry angle j deg and breathing time j/6 s (one-minute rotation,
    360 projections, 6 Hz), noise seed j (2^31 + j for the frames before the
    rotation, j < 0), 10 iterations, warm start from j - 1."""
    vol = Volume(256, 256, 120, 2.0, 2.0, 2.5)
    nu, nv, pitch = DETECTORS[detector]
    geom = Geometry(1000.0, 1500.0, nu, nv, pitch, pitch, 1.0)
    return dict(name="phantom 256x256x120 @ 2x2x2.5 mm, K=%d, %s detector" % (K, detector), vol=vol,
                geom=geom, K=K, scale=1.5, max_iters=10,
                frame_angle_deg=lambda j: float(j % 360), frame_time=lambda j: j / 6.0,
                frame_seed=lambda j: int(j) if j >= 0 else int(2**31 + j))


MIXED_SHAPES = [
    (128, 128, 128),
    (160, 160, 96),
    (192, 192, 112),
    (256, 256, 120),
    (256, 256, 120),
    (256, 256, 160),
    (224, 224, 128),
    (128, 128, 200),
]


def workload_mixed(patient: int):
    """One of eight uneven patients: shape from MIXED_SHAPES, 2 mm in-plane and
    2.5 mm slices, K drawn from {3, 4, 5}, SI amplitude uniform in [8, 20] mm
    (seed = patient id), paper-scale detector."""
    rng = np.random.default_rng(1000 + patient)
    nx, ny, nz = MIXED_SHAPES[patient % len(MIXED_SHAPES)]
    K = int(rng.integers(3, 6))
    amp = float(rng.uniform(8.0, 20.0))
    vol = Volume(nx, ny, nz, 2.0, 2.0, 2.5)
    geom = Geometry(1000.0, 1500.0, 512, 384, 0.776, 0.776, 1.0)
    return dict(name="patient %d" % patient, vol=vol, geom=geom, K=K, amp_si=amp, scale=1.5,
                max_iters=10)
