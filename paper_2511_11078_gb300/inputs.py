"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle side.

This module holds none of the projector's arithmetic: it only draws random
numbers and lays out plain arrays (ellipsoid phantoms, the B-spline
interpolation prefilter that turns samples into coefficients, band-limited
noise, and the pose arrays of parallel-, cone- and helical-beam geometries).
Both the CUDA path and the FP64 oracle consume what it returns.

The paper's data (a BrainWeb head volume, ASTRA-simulated cone-beam
projections; Sec. 3) is not available; random-ellipsoid phantoms with
normalised densities in [0, 1], several hundred views and square-ish
detectors stand in for it.

Conventions: world units are lattice units (Sec. 2.1 places the bases on a
unit lattice); coefficient k of a grid with dims (nx, ny, nz) sits at
origin + k with origin = -(dims - 1)/2, so the volume centre is the world
origin; arrays are C-order [z][y][x].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20251111


def rng_for(config_index: int) -> np.random.Generator:
    """The seeded generator of workload `config_index` (1-based)."""
    return np.random.default_rng(SEED_BASE + int(config_index))


def centred_origin(dims) -> np.ndarray:
    d = np.asarray(dims, dtype=np.float64)
    return -(d - 1.0) / 2.0


# --------------------------------------------------------------------------
# directions and rotations
# --------------------------------------------------------------------------
def random_directions(rng: np.random.Generator, count: int) -> np.ndarray:
    """`count` unit vectors uniform on the sphere (normalised Gaussians)."""
    v = rng.normal(size=(count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_rotations(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions."""
    q = rng.normal(size=(count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    a, b, c, d = q.T
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = a * a + b * b - c * c - d * d
    R[:, 0, 1] = 2 * (b * c - a * d)
    R[:, 0, 2] = 2 * (b * d + a * c)
    R[:, 1, 0] = 2 * (b * c + a * d)
    R[:, 1, 1] = a * a - b * b + c * c - d * d
    R[:, 1, 2] = 2 * (c * d - a * b)
    R[:, 2, 0] = 2 * (b * d - a * c)
    R[:, 2, 1] = 2 * (c * d + a * b)
    R[:, 2, 2] = a * a - b * b - c * c + d * d
    return R


def detector_frame(direction: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two unit vectors spanning the plane perpendicular to `direction`
    (a detector's u and v axes before scaling by the pixel pitch)."""
    w = np.asarray(direction, dtype=np.float64)
    w = w / np.linalg.norm(w)
    ref = np.array([0.0, 0.0, 1.0]) if abs(w[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(ref, w)
    u /= np.linalg.norm(u)
    v = np.cross(w, u)
    return u, v


# --------------------------------------------------------------------------
# geometries (plain pose arrays; Eq. 1 lines are built from them)
# --------------------------------------------------------------------------
@dataclass
class ViewGeometry:
    """Pose arrays of a view-based geometry.

    kind "parallel": `src` holds the ray direction of each view.
    kind "cone":     `src` holds the source position of each view.
    Pixel (iu, iv) of view k has centre
        det_center[k] + (iu - (nu-1)/2) det_u[k] + (iv - (nv-1)/2) det_v[k]
    (det_u, det_v include the pixel pitch).  Ray r = (k*nv + iv)*nu + iu.
    """

    kind: str
    src: np.ndarray
    det_center: np.ndarray
    det_u: np.ndarray
    det_v: np.ndarray
    nu: int
    nv: int

    @property
    def n_views(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_rays(self) -> int:
        return self.n_views * self.nu * self.nv

    def subset_views(self, views) -> "ViewGeometry":
        v = np.asarray(views)
        return ViewGeometry(self.kind, self.src[v].copy(), self.det_center[v].copy(), self.det_u[v].copy(),
                            self.det_v[v].copy(), self.nu, self.nv)


@dataclass
class RayGeometry:
    """Explicit rays: unit direction `omega` [R,3] and a point `s` [R,3]."""

    omega: np.ndarray
    s: np.ndarray
    kind: str = field(default="rays")

    @property
    def n_rays(self) -> int:
        return int(self.omega.shape[0])


def parallel_views(directions: np.ndarray, nu: int, nv: int, pitch: float = 1.0,
                   center=(0.0, 0.0, 0.0)) -> ViewGeometry:
    """Parallel-beam views: one flat detector through `center` per direction."""
    d = np.asarray(directions, dtype=np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    V = d.shape[0]
    du = np.zeros((V, 3))
    dv = np.zeros((V, 3))
    for k in range(V):
        u, v = detector_frame(d[k])
        du[k], dv[k] = pitch * u, pitch * v
    dc = np.tile(np.asarray(center, dtype=np.float64), (V, 1))
    return ViewGeometry("parallel", d, dc, du, dv, int(nu), int(nv))


def tilt_series(n_views: int, nu: int, nv: int, pitch: float = 1.0) -> ViewGeometry:
    """Single-axis tilt: directions (cos t, sin t, 0), t = pi*i/n_views in
    [0, pi); detector v axis along e3, u axis = e3 x direction."""
    t = np.pi * np.arange(n_views) / n_views
    d = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], axis=1)
    e3 = np.array([0.0, 0.0, 1.0])
    du = pitch * np.cross(e3, d)
    dv = pitch * np.tile(e3, (n_views, 1))
    return ViewGeometry("parallel", d, np.zeros((n_views, 3)), du, dv, int(nu), int(nv))


def circular_cone(n_views: int, sod: float, sdd: float, nu: int, nv: int, pitch: float) -> ViewGeometry:
    """Circular cone-beam orbit about e3 at angles 2*pi*i/n_views; flat
    detector perpendicular to the central ray at distance `sdd` from the
    source, source at distance `sod` from the rotation axis."""
    return helical_cone(n_views, sod, sdd, nu, nv, pitch, turns=1.0, table_feed=0.0)


def helical_cone(n_views: int, sod: float, sdd: float, nu: int, nv: int, pitch: float,
                 turns: float = 1.0, table_feed: float = 0.0) -> ViewGeometry:
    """Helical cone-beam: angle 2*pi*turns*i/n_views, source height rising by
    `table_feed` per turn, centred so the helix is symmetric about z = 0."""
    theta = 2.0 * np.pi * turns * np.arange(n_views) / n_views
    z = table_feed * theta / (2.0 * np.pi)
    if n_views > 0:
        z = z - 0.5 * (z[0] + z[-1])
    src = np.stack([sod * np.cos(theta), sod * np.sin(theta), z], axis=1)
    inward = -np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], axis=1)
    dc = src + sdd * inward
    du = pitch * np.stack([-np.sin(theta), np.cos(theta), np.zeros_like(theta)], axis=1)
    dv = pitch * np.tile(np.array([0.0, 0.0, 1.0]), (n_views, 1))
    return ViewGeometry("cone", src, dc, du, dv, int(nu), int(nv))


def random_rays(rng: np.random.Generator, count: int, radius: float) -> RayGeometry:
    """Rays with directions uniform on the sphere and offsets uniform in the
    disc of `radius` of the plane perpendicular to each direction, shifted
    along the direction by a random amount (the line is unchanged)."""
    w = random_directions(rng, count)
    s = np.zeros((count, 3))
    for i in range(count):
        u, v = detector_frame(w[i])
        r = radius * np.sqrt(rng.uniform())
        a = rng.uniform(0, 2 * np.pi)
        s[i] = r * np.cos(a) * u + r * np.sin(a) * v + rng.uniform(-50, 50) * w[i]
    return RayGeometry(w, s)


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------
@dataclass
class Ellipsoids:
    centers: np.ndarray  # [E,3] world
    semi_axes: np.ndarray  # [E,3]
    rotations: np.ndarray  # [E,3,3] columns = principal axes
    densities: np.ndarray  # [E]


def random_ellipsoids(rng: np.random.Generator, dims, count: int, semi_range, density_range=(0.2, 1.0),
                      inner: float = 0.6) -> Ellipsoids:
    ext = (np.asarray(dims, dtype=np.float64) - 1.0)
    c = rng.uniform(-0.5 * inner, 0.5 * inner, size=(count, 3)) * ext
    a = rng.uniform(semi_range[0], semi_range[1], size=(count, 3))
    R = random_rotations(rng, count)
    rho = rng.uniform(density_range[0], density_range[1], size=count)
    return Ellipsoids(c, a, R, rho)


def rasterize(ell: Ellipsoids, dims, dtype=np.float64) -> np.ndarray:
    """Additive ellipsoid indicators sampled at the lattice points -> [z][y][x]."""
    nx, ny, nz = (int(v) for v in dims)
    org = centred_origin(dims)
    out = np.zeros((nz, ny, nx), dtype=dtype)
    n = (nx, ny, nz)
    for e in range(ell.centers.shape[0]):
        R = ell.rotations[e]
        a = ell.semi_axes[e]
        c = ell.centers[e]
        rad = float(a.max())
        # lattice points within the bounding cube of the ellipsoid
        lo = [max(0, int(np.floor(c[d] - rad - org[d]))) for d in range(3)]
        hi = [min(n[d] - 1, int(np.ceil(c[d] + rad - org[d]))) for d in range(3)]
        if any(hi[d] < lo[d] for d in range(3)):
            continue
        xs = org[0] + np.arange(lo[0], hi[0] + 1)
        ys = org[1] + np.arange(lo[1], hi[1] + 1)
        X, Y = np.meshgrid(xs - c[0], ys - c[1], indexing="xy")
        for kz in range(lo[2], hi[2] + 1):
            Z = org[2] + kz - c[2]
            # body coordinates = R^T (x - c)
            bx = R[0, 0] * X + R[1, 0] * Y + R[2, 0] * Z
            by = R[0, 1] * X + R[1, 1] * Y + R[2, 1] * Z
            bz = R[0, 2] * X + R[1, 2] * Y + R[2, 2] * Z
            inside = (bx / a[0]) ** 2 + (by / a[1]) ** 2 + (bz / a[2]) ** 2 <= 1.0
            out[kz, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1][inside] += ell.densities[e]
    return out


def ellipsoid_line_integrals(ell: Ellipsoids, s: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Analytic line integrals of the (continuous) ellipsoid phantom: density
    times chord length, summed over ellipsoids.  s, w: [R,3]."""
    s = np.asarray(s, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(s.shape[0])
    for e in range(ell.centers.shape[0]):
        R = ell.rotations[e]
        a = ell.semi_axes[e]
        ps = (s - ell.centers[e]) @ R / a
        pw = (w @ R) / a
        A = np.sum(pw * pw, axis=1)
        B = 2.0 * np.sum(ps * pw, axis=1)
        Cq = np.sum(ps * ps, axis=1) - 1.0
        disc = B * B - 4.0 * A * Cq
        ok = disc > 0
        chord = np.zeros_like(A)
        chord[ok] = np.sqrt(disc[ok]) / A[ok]
        out += ell.densities[e] * chord
    return out


def bandlimited_noise(rng: np.random.Generator, dims, sigma: float, amplitude: float) -> np.ndarray:
    """White Gaussian noise low-passed by a Gaussian of std `sigma` voxels,
    scaled to standard deviation `amplitude`; float32 [z][y][x]."""
    import scipy.fft as sfft

    nx, ny, nz = (int(v) for v in dims)
    wn = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    F = sfft.rfftn(wn, workers=-1)
    fz = np.fft.fftfreq(nz)[:, None, None]
    fy = np.fft.fftfreq(ny)[None, :, None]
    fx = np.fft.rfftfreq(nx)[None, None, :]
    H = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fx * fx + fy * fy + fz * fz)).astype(np.float32)
    F *= H
    out = sfft.irfftn(F, s=(nz, ny, nx), axes=(0, 1, 2), workers=-1).astype(np.float32)
    out *= amplitude / max(float(out.std()), 1e-30)
    return out


# --------------------------------------------------------------------------
# B-spline interpolation prefilter (samples -> coefficients) on a finite grid
# --------------------------------------------------------------------------
# Values of the centred B-spline at 0 and +-1: the only nonzero entries of the
# 1-D interpolation matrix for degrees 2 and 3 (degrees 0 and 1 interpolate
# with the identity).
_INTERP_TAPS = {2: (3.0 / 4.0, 1.0 / 8.0), 3: (2.0 / 3.0, 1.0 / 6.0)}


def _solve_tridiagonal_axis(x: np.ndarray, diag: float, off: float, axis: int) -> np.ndarray:
    """Solve T c = x along `axis` with T = tridiag(off, diag, off) of the axis
    length (Thomas algorithm, vectorised over the other axes)."""
    # a contiguous copy with the solve axis first: each step of the sweeps
    # is then one contiguous slab operation, done in place
    x = np.ascontiguousarray(np.moveaxis(np.asarray(x, dtype=np.float64), axis, 0))
    if x.base is not None or not x.flags.writeable:
        x = x.copy()
    N = x.shape[0]
    cp = np.zeros(N)
    m = np.zeros(N)
    m[0] = diag
    cp[0] = off / diag
    for k in range(1, N):
        m[k] = diag - off * cp[k - 1]
        cp[k] = off / m[k]
    tmp = np.empty_like(x[0])
    x[0] /= m[0]
    for k in range(1, N):
        np.multiply(x[k - 1], off, out=tmp)
        x[k] -= tmp
        x[k] /= m[k]
    for k in range(N - 2, -1, -1):
        np.multiply(x[k + 1], cp[k], out=tmp)
        x[k] -= tmp
    return np.moveaxis(x, 0, axis)


def prefilter(samples: np.ndarray, degree: int) -> np.ndarray:
    """Coefficients c on the finite grid with
    sum_{l in grid} c_l beta^n(k - l) = samples_k for every grid point k
    (separable: one tridiagonal solve per axis); identity for n <= 1."""
    out = np.asarray(samples, dtype=np.float64)
    if int(degree) not in _INTERP_TAPS:
        return out.copy()
    diag, off = _INTERP_TAPS[int(degree)]
    for ax in range(out.ndim):
        out = _solve_tridiagonal_axis(out, diag, off, ax)
    return np.ascontiguousarray(out)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dims: tuple
    degree: int
    coeffs: np.ndarray  # [z][y][x]
    geometry: object
    ellipsoids: Ellipsoids | None = None
    extra: dict = field(default_factory=dict)

    @property
    def origin(self) -> np.ndarray:
        return centred_origin(self.dims)


def workload_small(degree: int = 3) -> Workload:
    """24^3 cubic coefficients of a 6-ellipsoid phantom (semi-axes U(2,8),
    densities U(0.2,1), centres within the inner 60%), B-spline interpolated;
    parallel beam, 32 directions uniform on the sphere, 32x32 detector,
    pitch 1."""
    rng = rng_for(1)
    dims = (24, 24, 24)
    ell = random_ellipsoids(rng, dims, 6, (2.0, 8.0))
    c = prefilter(rasterize(ell, dims), degree)
    g = parallel_views(random_directions(rng, 32), 32, 32, 1.0)
    return Workload("small-24^3-parallel-32x32^2", dims, degree, c, g, ell)


def workload_tilt(degree: int = 3, n: int = 128) -> Workload:
    """128^3 coefficients (6 ellipsoids, semi-axes U(10,45)); parallel beam:
    180 single-axis tilt views over [0, 180 deg) about e3 plus 64 directions
    uniform on the sphere; 192x192 detector, pitch 1."""
    rng = rng_for(2)
    dims = (n, n, n)
    s = n / 128.0
    ell = random_ellipsoids(rng, dims, 6, (10.0 * s, 45.0 * s))
    c = prefilter(rasterize(ell, dims, dtype=np.float32), degree).astype(np.float32)
    nd = int(round(192 * s))
    g1 = tilt_series(180, nd, nd, 1.0)
    g2 = parallel_views(random_directions(rng, 64), nd, nd, 1.0)
    g = ViewGeometry("parallel", np.concatenate([g1.src, g2.src]), np.concatenate([g1.det_center, g2.det_center]),
                     np.concatenate([g1.det_u, g2.det_u]), np.concatenate([g1.det_v, g2.det_v]), nd, nd)
    return Workload("tilt-%d^3-parallel-244x%d^2" % (n, nd), dims, degree, c, g, ell)


def workload_cone(n: int = 256, n_views: int = 360, nd: int = 384, pitch: float = 1.2) -> Workload:
    """256^3 cubic coefficients of a 12-ellipsoid phantom; circular cone beam,
    360 views, source-to-centre 1000, source-to-detector 1500, 384x384
    detector, pitch 1.2."""
    rng = rng_for(3)
    dims = (n, n, n)
    s = n / 128.0
    ell = random_ellipsoids(rng, dims, 12, (10.0 * s, 45.0 * s))
    c = prefilter(rasterize(ell, dims, dtype=np.float32), 3).astype(np.float32)
    g = helical_cone(n_views, 1000.0, 1500.0, nd, nd, pitch, turns=1.0, table_feed=0.0)
    return Workload("cone-%d^3-%dx%d^2" % (n, n_views, nd), dims, 3, c, g, ell)


def workload_helical(n: int = 512, n_views: int = 720, nd: int = 768, pitch: float = 0.8) -> Workload:
    """512^3 cubic coefficients (ellipsoids + band-limited Gaussian noise
    texture, sigma 4 voxels, amplitude 0.05); helical cone beam, 720 views
    over 2 turns, helical pitch 0.5 (table feed per turn = 0.5 x detector
    height at the isocentre), 768x768 detector, pitch 0.8, SOD 1000, SDD 1500."""
    rng = rng_for(5)
    dims = (n, n, n)
    s = n / 128.0
    ell = random_ellipsoids(rng, dims, 12, (10.0 * s, 45.0 * s))
    vol = rasterize(ell, dims, dtype=np.float32) + bandlimited_noise(rng, dims, 4.0, 0.05)
    c = prefilter(vol, 3).astype(np.float32)
    feed = 0.5 * nd * pitch * 1000.0 / 1500.0
    g = helical_cone(n_views, 1000.0, 1500.0, nd, nd, pitch, turns=2.0, table_feed=feed)
    return Workload("helical-%d^3-%dx%d^2" % (n, n_views, nd), dims, 3, c, g, ell)


def footprint_samples(rng: np.random.Generator, count: int, degree: int):
    """Algorithm 1's training distribution: directions uniform on the
    sphere, offsets uniform in the disc of radius sqrt(3) W of H_w
    (W = (degree+1)/2).  Returns (omega [count,3], p [count,3]) with p in H_w."""
    W = 0.5 * (degree + 1)
    w = random_directions(rng, count)
    ref = np.where(np.abs(w[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    u = np.cross(ref, w)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(w, u)
    r = np.sqrt(3.0) * W * np.sqrt(rng.uniform(size=count))
    a = rng.uniform(0.0, 2.0 * np.pi, size=count)
    p = (r * np.cos(a))[:, None] * u + (r * np.sin(a))[:, None] * v
    return w, p
