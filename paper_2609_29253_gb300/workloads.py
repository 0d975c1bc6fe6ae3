"""Seeded synthetic workloads for the photoacoustic operator.

This module only builds inputs: voxel grids, transducer descriptors, the
electrical impulse response parameters, the time axis and the phantoms x.  It
holds none of the operator's arithmetic, so both the CUDA path and the FP64
oracle can consume its output without sharing any of the method's code.

Geometry conventions follow the paper's Sec. 4 (Eq. plane_param and
Eq. cylinder_param):

* a planar element is (c0, e1, e2, L1, L2): the rectangle
  c0 + x1 e1 + x2 e2, |x1| <= L1, |x2| <= L2;
* a cylindrical element is (c0, e1, e2, R, theta_max, Lz) with c0 on the focal
  line, e1 the cylinder axis and e2 pointing from the focal line to the element
  centre: c0 + R cos(t) e2 + R sin(t) (e1 x e2) + z e1, |t| <= theta_max,
  |z| <= Lz.

Descriptors are float64 rows of 16 numbers:
``[kind, c0(3), e1(3), e2(3), L1, L2, R, theta_max, Lz, 0]`` with kind 0 for a
plane and 1 for a cylinder.

The named presets reproduce the synthetic systems of the benchmark table:

* ``c1`` -- 16^3 voxels at 0.1 mm, 32 planar 1x1 mm elements on a 10 mm
  Fibonacci sphere, 256 samples at 40 MHz, x ~ U[0,1) (seed 0);
* ``c2`` -- 128^3 voxels at 0.1 mm, a 128-element cylindrically focused linear
  array (0.3 mm pitch, 10 mm elevation, 20 mm focus) rotated over 180 angles
  about its focal line (23,040 positions), 1024 samples at 40 MHz, x = 200
  Gaussian blobs (seed 0);
* ``c3`` -- 256^3 voxels at 0.08 mm, 512 planar 3x3 mm elements on a 40 mm
  hemisphere x 10 rotations, 2048 samples at 40 MHz;
* ``c5`` -- 512^3 voxels at 0.05 mm, the c2 array x 128 rotations, 4096
  samples at 50 MHz.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PLANE = 0
CYLINDER = 1
METHOD_SURFACE = 0
METHOD_POINT = 1
METHOD_TRAPEZOID = 2
METHOD_LUT = 3  # surface method, cylinder arc integral from the paper's E / F lookup tables (q1 x q2 nodes)
LUT_PAPER = (1000, 1000)  # the paper's table sizes N_s x N_nu
RBF_BUMP = 0  # (1 - r^2/k^2)^2
RBF_CONE = 1  # 1 - r/k
RBF_WENDLAND = 2  # (1 - r/k)^2
EIR_GAUSS_SINE = 0  # exp(-(t-tc)^2/(2 s^2)) sin(2 pi fc (t - tc)) on [0, Te]
EIR_BOX = 1  # constant on [0, Te]
TX_STRIDE = 16


@dataclass
class Workload:
    """Everything one operator application needs, in SI units."""

    name: str
    n: tuple  # (nx, ny, nz)
    origin: np.ndarray  # centre of voxel (0, 0, 0)
    pitch: float
    tx: np.ndarray  # (K, 16) float64 descriptors
    c: float
    fs: float
    t0: float
    L: int
    U: int
    dl: int
    rbf_kind: int
    kappa: float
    eir_kind: int
    eir_par: np.ndarray  # (4,) float64
    n_lo: int  # first tap index of the discrete system kernel
    T: int  # number of taps
    method: int = METHOD_SURFACE
    q1: int = 0
    q2: int = 0
    x: np.ndarray | None = None  # (N,) float32 phantom
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def K(self) -> int:
        return int(self.tx.shape[0])

    @property
    def UL(self) -> int:
        return int(self.U * self.L)

    def with_tx(self, tx: np.ndarray) -> "Workload":
        return replace(self, tx=np.ascontiguousarray(tx, dtype=np.float64))

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# --------------------------------------------------------------------------
# geometry builders
# --------------------------------------------------------------------------
def centred_origin(n, pitch):
    return np.array([-(k - 1) / 2.0 * pitch for k in n], dtype=np.float64)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def plane_row(c0, e1, e2, L1, L2):
    r = np.zeros(TX_STRIDE)
    r[0] = PLANE
    r[1:4] = c0
    r[4:7] = e1
    r[7:10] = e2
    r[10] = L1
    r[11] = L2
    return r


def cylinder_row(c0, e1, e2, R, theta_max, Lz):
    r = np.zeros(TX_STRIDE)
    r[0] = CYLINDER
    r[1:4] = c0
    r[4:7] = e1
    r[7:10] = e2
    r[12] = R
    r[13] = theta_max
    r[14] = Lz
    return r


def facing_frame(p):
    """Frame of a planar element at p facing the origin: the normal
    n = -p/|p|, e1 = z x n normalised (x if parallel), e2 = n x e1, so that
    e1 x e2 = n points towards the centre."""
    n = -_unit(p)
    e1 = np.cross([0.0, 0.0, 1.0], n)
    if np.linalg.norm(e1) < 1e-12:
        e1 = np.array([1.0, 0.0, 0.0])
    e1 = _unit(e1)
    e2 = np.cross(n, e1)
    return e1, e2


def fibonacci_points(K, hemisphere=False):
    """Spherical Fibonacci points z_k = 1 - (2k+1)/K, azimuth k pi (3 - sqrt 5);
    with hemisphere=True, z_k = -(k + 1/2)/K (lower half)."""
    k = np.arange(K, dtype=np.float64)
    z = -(k + 0.5) / K if hemisphere else 1.0 - (2.0 * k + 1.0) / K
    az = k * math.pi * (3.0 - math.sqrt(5.0))
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rr * np.cos(az), rr * np.sin(az), z], axis=1)


def fibonacci_planar(K, radius, L1, L2, hemisphere=False, rotations=1, rot_step=0.0):
    pts = fibonacci_points(K, hemisphere) * radius
    rows = []
    for j in range(rotations):
        a = j * rot_step
        Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
        for p in pts:
            q = Rz @ p
            e1, e2 = facing_frame(q)
            rows.append(plane_row(q, e1, e2, L1, L2))
    return np.ascontiguousarray(np.array(rows))


def rotated_linear_cylinder_array(n_el, el_pitch, R, theta_max, Lz, n_angles, angle_span=2 * math.pi,
                                  angles=None):
    """A linear array of cylindrically focused elements along the z axis, which
    is also every element's focal line, rotated about z over ``n_angles``
    uniform angles in [0, angle_span).  Element j sits at
    z_j = (j - (n_el-1)/2) el_pitch."""
    if angles is None:
        angles = np.arange(n_angles) * angle_span / n_angles
    rows = []
    e1 = np.array([0.0, 0.0, 1.0])
    for a in angles:
        e2 = np.array([math.cos(a), math.sin(a), 0.0])
        for j in range(n_el):
            zj = (j - (n_el - 1) / 2.0) * el_pitch
            rows.append(cylinder_row(np.array([0.0, 0.0, zj]), e1, e2, R, theta_max, Lz))
    return np.ascontiguousarray(np.array(rows))


# --------------------------------------------------------------------------
# electrical impulse response and discrete-kernel window
# --------------------------------------------------------------------------
def gauss_sine_eir(fc, frac_bw=0.8, n_sigma=4.0):
    """Gaussian-modulated sine with a -6 dB fractional bandwidth ``frac_bw``:
    the amplitude spectrum exp(-2 pi^2 s^2 (f - fc)^2) halves at
    f - fc = sqrt(ln 2 / 2) / (pi s), so s = sqrt(ln2/2) / (pi frac_bw fc / 2).
    Centre tc = n_sigma s, support [0, 2 n_sigma s]."""
    s = math.sqrt(math.log(2.0) / 2.0) / (math.pi * 0.5 * frac_bw * fc)
    return np.array([fc, s, n_sigma * s, 2.0 * n_sigma * s], dtype=np.float64)


def tap_window(kappa, c, fs, U, Te):
    """Index window [n_lo, n_lo + T) covering the support of the discrete
    system kernel stated in Sec. 2.6: [-kappa U Fs / c - 1,
    (kappa / c + Te) U Fs + 1]."""
    ufs = U * fs
    n_lo = -int(math.ceil(kappa * ufs / c)) - 1
    n_hi = int(math.ceil((kappa / c + Te) * ufs)) + 1
    return n_lo, n_hi - n_lo + 1


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------
def voxel_centres(n, origin, pitch, idx=None):
    n = tuple(int(v) for v in n)
    if idx is None:
        idx = np.arange(n[0] * n[1] * n[2], dtype=np.int64)
    ix = idx % n[0]
    iy = (idx // n[0]) % n[1]
    iz = idx // (n[0] * n[1])
    return np.stack([origin[0] + pitch * ix, origin[1] + pitch * iy, origin[2] + pitch * iz], axis=1)


def uniform_phantom(N, seed=0):
    return np.random.default_rng(seed).random(N).astype(np.float32)


def blob_phantom(n, origin, pitch, n_blobs=200, seed=0, sigma=(0.1e-3, 0.4e-3), amp=(0.5, 1.0), inner=0.8):
    """Sum of isotropic Gaussian blobs: centres uniform in the inner ``inner``
    fraction of the box, widths U[sigma], amplitudes U[amp]; each blob is
    truncated at 4 sigma."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    ext = np.array([(k - 1) * pitch for k in n])
    lo = origin + 0.5 * (1 - inner) * ext
    cen = lo + rng.random((n_blobs, 3)) * inner * ext
    sig = rng.uniform(sigma[0], sigma[1], n_blobs)
    am = rng.uniform(amp[0], amp[1], n_blobs)
    x = np.zeros((n[2], n[1], n[0]), dtype=np.float64)
    axes = [origin[d] + pitch * np.arange(n[d]) for d in range(3)]
    for b in range(n_blobs):
        sl = []
        for d in range(3):
            a = np.searchsorted(axes[d], cen[b, d] - 4 * sig[b])
            e = np.searchsorted(axes[d], cen[b, d] + 4 * sig[b], side="right")
            sl.append((a, e))
        gx = np.exp(-((axes[0][sl[0][0]:sl[0][1]] - cen[b, 0]) ** 2) / (2 * sig[b] ** 2))
        gy = np.exp(-((axes[1][sl[1][0]:sl[1][1]] - cen[b, 1]) ** 2) / (2 * sig[b] ** 2))
        gz = np.exp(-((axes[2][sl[2][0]:sl[2][1]] - cen[b, 2]) ** 2) / (2 * sig[b] ** 2))
        x[sl[2][0]:sl[2][1], sl[1][0]:sl[1][1], sl[0][0]:sl[0][1]] += am[b] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return x.reshape(-1).astype(np.float32)


def tube_phantom(n, origin, pitch, n_tubes, seed, r_vox=(1.0, 3.0), inner=0.8, samples=64):
    """Vessel-like tubes: cubic Bezier centre lines inside the inner box,
    radius U[r_vox] voxels, profile (1 - (d/r)^2)_+ (max over tubes)."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    ext = np.array([(k - 1) * pitch for k in n])
    lo = origin + 0.5 * (1 - inner) * ext
    pts = voxel_centres(n, origin, pitch)
    x = np.zeros(len(pts))
    t = np.linspace(0, 1, samples)[:, None]
    for _ in range(n_tubes):
        P = lo + rng.random((4, 3)) * inner * ext
        curve = ((1 - t) ** 3) * P[0] + 3 * ((1 - t) ** 2) * t * P[1] + 3 * (1 - t) * t * t * P[2] + (t ** 3) * P[3]
        r = rng.uniform(*r_vox) * pitch
        bb_lo = curve.min(0) - r
        bb_hi = curve.max(0) + r
        sel = np.all((pts >= bb_lo) & (pts <= bb_hi), axis=1)
        idx = np.nonzero(sel)[0]
        if idx.size == 0:
            continue
        d = np.full(idx.size, np.inf)
        for a in range(samples - 1):
            p0, p1 = curve[a], curve[a + 1]
            seg = p1 - p0
            L2 = float(seg @ seg) or 1e-30
            w = np.clip(((pts[idx] - p0) @ seg) / L2, 0, 1)
            d = np.minimum(d, np.linalg.norm(pts[idx] - (p0 + w[:, None] * seg), axis=1))
        x[idx] = np.maximum(x[idx], np.clip(1 - (d / r) ** 2, 0, None))
    return x.astype(np.float32)


def rod_phantom(n, origin, pitch, spacing=0.9e-3, n_rods=7, r_xy=0.1125e-3, r_z=0.2625e-3):
    """A n_rods x n_rods grid of rods centred on the z = 0 plane, spacing
    apart, each with the paraboloidal profile (1 - (dx^2 + dy^2)/r_xy^2 -
    dz^2/r_z^2)_+ (support 225 x 225 x 525 um with the defaults)."""
    pts = voxel_centres(n, origin, pitch)
    c = (np.arange(n_rods) - (n_rods - 1) / 2.0) * spacing
    x = np.zeros(len(pts))
    for cx in c:
        for cy in c:
            v = 1.0 - ((pts[:, 0] - cx) ** 2 + (pts[:, 1] - cy) ** 2) / r_xy ** 2 - pts[:, 2] ** 2 / r_z ** 2
            x = np.maximum(x, np.clip(v, 0.0, None))
    return x.astype(np.float32)


# --------------------------------------------------------------------------
# presets
# --------------------------------------------------------------------------
def _make(name, n, pitch, tx, c, fs, t0, L, U, kappa, eir, x=None, dl=None, rbf=RBF_BUMP, method=METHOD_SURFACE,
          q=(0, 0), meta=None):
    n = tuple(int(v) for v in n)
    n_lo, T = tap_window(kappa, c, fs, U, eir[3])
    return Workload(name=name, n=n, origin=centred_origin(n, pitch), pitch=float(pitch),
                    tx=np.ascontiguousarray(tx, dtype=np.float64), c=float(c), fs=float(fs), t0=float(t0), L=int(L),
                    U=int(U), dl=int(U if dl is None else dl), rbf_kind=int(rbf), kappa=float(kappa),
                    eir_kind=EIR_GAUSS_SINE, eir_par=np.asarray(eir, dtype=np.float64), n_lo=n_lo, T=T,
                    method=method, q1=int(q[0]), q2=int(q[1]), x=x, meta=dict(meta or {}))


def method_q(method, q, lut=LUT_PAPER):
    """(q1, q2) of a workload: the point method's quadrature, the LUT's table
    sizes, else (0, 0)."""
    return tuple(q) if method == METHOD_POINT else tuple(lut) if method == METHOD_LUT else (0, 0)


def c1(dl=None, method=METHOD_SURFACE, q=(64, 64), seed=0):
    """16^3 voxels, 32 planar 1x1 mm elements on a 10 mm Fibonacci sphere."""
    n = (16, 16, 16)
    pitch = 0.1e-3
    tx = fibonacci_planar(32, 10e-3, 0.5e-3, 0.5e-3)
    x = uniform_phantom(16 ** 3, seed)
    return _make("c1: 16^3 @ 0.1 mm, 32 planar 1x1 mm, L=256 @ 40 MHz", n, pitch, tx, 1500.0, 40e6, 5.0e-6, 256, 11,
                 1.5 * pitch, gauss_sine_eir(5e6), x=x, dl=dl, method=method, q=method_q(method, q))


C2_ARRAY = dict(n_el=128, el_pitch=0.3e-3, R=20e-3, theta_max=math.asin(0.25), Lz=0.15e-3)


def c2(n_angles=180, angles=None, n_vox=128, with_x=True, dl=None):
    """128^3 voxels at 0.1 mm; 128-element cylindrical array x 180 angles."""
    n = (n_vox, n_vox, n_vox)
    pitch = 0.1e-3
    if angles is None:
        angles = np.arange(n_angles) * 2 * math.pi / 180.0
    a = C2_ARRAY
    tx = rotated_linear_cylinder_array(a["n_el"], a["el_pitch"], a["R"], a["theta_max"], a["Lz"], len(angles),
                                       angles=angles)
    origin = centred_origin(n, pitch)
    x = blob_phantom(n, origin, pitch, 200, 0) if with_x else None
    return _make("c2: 128^3 @ 0.1 mm, 128-el cylindrical array x 180 angles, L=1024 @ 40 MHz", n, pitch, tx, 1500.0,
                 40e6, 6.0e-6, 1024, 11, 1.5 * pitch, gauss_sine_eir(5e6), x=x, dl=dl)


def c3(with_x=True, rotations=10):
    n = (256, 256, 256)
    pitch = 0.08e-3
    tx = fibonacci_planar(512, 40e-3, 1.5e-3, 1.5e-3, hemisphere=True, rotations=rotations,
                          rot_step=math.radians(3.6))
    origin = centred_origin(n, pitch)
    x = blob_phantom(n, origin, pitch, 200, 0) if with_x else None
    return _make("c3: 256^3 @ 0.08 mm, 512 planar 3x3 mm x 10 rotations, L=2048 @ 40 MHz", n, pitch, tx, 1500.0,
                 40e6, 12e-6, 2048, 11, 1.5 * pitch, gauss_sine_eir(5e6), x=x)


def c5(with_x=True, n_angles=128):
    n = (512, 512, 512)
    pitch = 0.05e-3
    a = C2_ARRAY
    tx = rotated_linear_cylinder_array(a["n_el"], a["el_pitch"], a["R"], a["theta_max"], a["Lz"], n_angles)
    origin = centred_origin(n, pitch)
    x = blob_phantom(n, origin, pitch, 200, 0) if with_x else None
    return _make("c5: 512^3 @ 0.05 mm, 128-el cylindrical array x 128 angles, L=4096 @ 50 MHz", n, pitch, tx, 1500.0,
                 50e6, 1.0e-6, 4096, 11, 1.5 * pitch, gauss_sine_eir(5e6), x=x)


def c4_problem(p, n_range=(48, 160), k_range=(1024, 8192), seed_base=1000):
    """Problem p of the batched-reconstruction set: a cubic grid of n ~ U{n_range}
    voxels per axis at 0.1 mm, K ~ U{k_range} positions (even p: planar 3x3 mm
    elements on a 40 mm Fibonacci hemisphere; odd p: the c2 cylindrical array
    with round(K / 128) >= 1 rotation angles), L in {1024, 2048} at 40 MHz,
    and 5-15 vessel-like tubes as x (seed seed_base + p)."""
    rng = np.random.default_rng(seed_base + p)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    K = int(rng.integers(k_range[0], k_range[1] + 1))
    L = int(rng.choice([1024, 2048]))
    pitch = 0.1e-3
    origin = centred_origin((n, n, n), pitch)
    if p % 2 == 0:
        tx = fibonacci_planar(K, 40e-3, 1.5e-3, 1.5e-3, hemisphere=True)
        t0, kind = 16e-6, "planar"
    else:
        a = C2_ARRAY
        n_ang = max(1, int(round(K / a["n_el"])))
        tx = rotated_linear_cylinder_array(a["n_el"], a["el_pitch"], a["R"], a["theta_max"], a["Lz"], n_ang)
        t0, kind = 5e-6, "cylindrical"
    x = tube_phantom((n, n, n), origin, pitch, int(rng.integers(5, 16)), seed_base + p)
    return _make(f"c4 problem {p}: {n}^3 @ 0.1 mm, {len(tx)} {kind} positions, L={L} @ 40 MHz", (n, n, n), pitch, tx,
                 1500.0, 40e6, t0, L, 11, 1.5 * pitch, gauss_sine_eir(5e6), x=x)


def exp1(grid="fine", method=METHOD_SURFACE, q=(25, 25), lut=LUT_PAPER):
    """The paper's controlled synthetic study (Sec. 5.2): 215 cylindrically
    focused elements (R 25 mm, 7.5 mm elevation aperture, 0.25 mm wide)
    rotated about their focal line at 43 azimuths, at 5 positions spanning
    36.7 mm along it; a 6 x 6 x 1.05 mm volume on the fine 81 x 81 x 15 grid
    (75 um) or the coarse 27 x 27 x 5 grid (225 um); 7 x 7 rods; 2688 samples
    at 62.5 MHz from t = 0, U 11, dl = U."""
    n, pitch = ((81, 81, 15), 75e-6) if grid == "fine" else ((27, 27, 5), 225e-6)
    rows = []
    for zj in np.linspace(-18.35e-3, 18.35e-3, 5):
        for m in range(43):
            a = 2 * math.pi * m / 43
            rows.append(cylinder_row(np.array([0.0, 0.0, zj]), np.array([0.0, 0.0, 1.0]),
                                     np.array([math.cos(a), math.sin(a), 0.0]), 25e-3, math.asin(3.75 / 25.0),
                                     0.125e-3))
    origin = centred_origin(n, pitch)
    x = rod_phantom(n, origin, pitch)
    return _make(f"exp1 ({grid}): {n[0]}x{n[1]}x{n[2]} @ {pitch * 1e6:.0f} um, 215 cylindrical elements, "
                 f"L=2688 @ 62.5 MHz", n, pitch, np.array(rows), 1500.0, 62.5e6, 0.0, 2688, 11, 1.5 * pitch,
                 gauss_sine_eir(5e6, frac_bw=1.6), x=x, method=method, q=method_q(method, q, lut))


def small_cylinder(n_vox=12, n_angles=4, n_el=4, seed=0, dl=None, L=None):
    """A reduced c2-like system (same element, fewer voxels and positions) for
    parity tests the oracle finishes in seconds."""
    pitch = 0.1e-3
    n = (n_vox, n_vox, n_vox)
    a = C2_ARRAY
    angles = np.arange(n_angles) * 2 * math.pi / n_angles + 0.1
    tx = rotated_linear_cylinder_array(n_el, 3e-3, a["R"], a["theta_max"], a["Lz"], n_angles, angles=angles)
    x = uniform_phantom(n_vox ** 3, seed)
    return _make(f"cylinder {n_vox}^3 x {len(tx)} positions", n, pitch, tx, 1500.0, 40e6, 6.0e-6,
                 L or 1024, 11, 1.5 * pitch, gauss_sine_eir(5e6), x=x, dl=dl)
