"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the bench.

This module holds only input generation: particle placement, media constants,
incidence angles, receiver lines and random coefficient blocks.  It contains none
of the method's arithmetic (no wavenumbers, special functions, translations or
Sommerfeld quadrature), so both the CPU oracle and the CUDA path may consume its
outputs without sharing method code.

Workloads follow the paper's setting (Sec. 2: particles buried in the lower
half-space of a welded two-layer elastic medium, well separated, Sec. 7: the
star/pear family r(t) = a1 + a2 cos(a3 t)).  Placement is random sequential
addition with rejection: enclosing discs keep |x_l - x_m| >= 1.1 (R_l + R_m)
(the "10 % of particle size" separation of Sec. 2) and y_m + 1.1 R_m <= 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEP = 1.1  # separation factor between enclosing discs (Sec. 2 well-separatedness)


@dataclasses.dataclass
class Media:
    """Lame constants of the upper (x2 > 0) and lower (x2 < 0) layers; rho = 1 (Sec. 2)."""
    lam_u: float
    mu_u: float
    lam_l: float
    mu_l: float


@dataclasses.dataclass
class Workload:
    name: str
    media: Media
    omega: float
    p: int
    centres: np.ndarray      # (M, 2) float64
    radius: np.ndarray       # (M,) enclosing radius
    bc: np.ndarray           # (M,) int32: 0 rigid, 1 traction-free
    shape: np.ndarray        # (M,) int32: 0 disc, 1 star
    rotation: np.ndarray     # (M,) float64 radians
    inc_kind: np.ndarray     # (nrhs,) int32: 0 P-wave, 1 S-wave
    inc_angle: np.ndarray    # (nrhs,) float64 radians, direction (cos t, -sin t)
    receivers: np.ndarray    # (R, 2) float64
    n_panels: int = 32
    nodes_per_panel: int = 16
    t_max: float = 20.0
    gmres_tol: float = 1e-12
    depth: float = 0.5       # contour depth d of xi(t) = t - i d tanh(t)
    grade: int = 0           # branch-point grading levels of the contour panels
    proto: np.ndarray | None = None        # (M,) int32: -1 disc, q >= 0 star prototype q
    proto_shape: np.ndarray | None = None  # (Q, 3) float64: a1, a2, a3 of r(t) = a1 + a2 cos(a3 t) (Sec. 7)
    proto_bc: np.ndarray | None = None     # (Q,) int32: boundary condition of prototype q

    @property
    def M(self) -> int:
        return int(self.centres.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.inc_angle.shape[0])

    @property
    def nc(self) -> int:
        return 2 * self.p + 1

    @property
    def n_proto(self) -> int:
        return 0 if self.proto_shape is None else int(self.proto_shape.shape[0])


MEDIA_STD = Media(lam_u=1.0, mu_u=0.5, lam_l=2.0, mu_l=1.0)


def place_particles(rng: np.random.Generator, M: int, box, rmin: float, rmax: float,
                    max_tries: int = 200000, radius_fn=None):
    """Random sequential addition of M enclosing discs inside box=(x0,x1,y0,y1).

    Radii are drawn U[rmin, rmax] (a constant when rmin == rmax), or by radius_fn(rng, n) for the
    n-th particle (values within [rmin, rmax]).  A candidate is rejected if it violates the
    separation rule against any accepted disc or if y + SEP*R > 0.  A uniform cell grid keeps the
    neighbour check O(1).
    """
    x0, x1, y0, y1 = box
    cell = 2.0 * SEP * rmax
    nx = max(1, int(math.ceil((x1 - x0) / cell)))
    ny = max(1, int(math.ceil((y1 - y0) / cell)))
    grid: dict[tuple[int, int], list[int]] = {}
    cx = np.empty(M)
    cy = np.empty(M)
    rr = np.empty(M)
    n = 0
    tries = 0
    while n < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"placement failed after {max_tries} tries ({n}/{M} placed)")
        if radius_fn is not None:
            r = radius_fn(rng, n)
        else:
            r = rng.uniform(rmin, rmax) if rmax > rmin else rmin
        x = rng.uniform(x0, x1)
        y = rng.uniform(y0, y1)
        if y + SEP * r > 0.0:
            continue
        gx = min(nx - 1, int((x - x0) / cell))
        gy = min(ny - 1, int((y - y0) / cell))
        ok = True
        for ix in range(gx - 1, gx + 2):
            for iy in range(gy - 1, gy + 2):
                for j in grid.get((ix, iy), ()):
                    if (x - cx[j]) ** 2 + (y - cy[j]) ** 2 < (SEP * (r + rr[j])) ** 2:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        cx[n], cy[n], rr[n] = x, y, r
        grid.setdefault((gx, gy), []).append(n)
        n += 1
    return np.stack([cx, cy], axis=1), rr


def perturb_centres(centres: np.ndarray, radius: np.ndarray, sigma: float, seed: int,
                    max_rounds: int = 1000) -> np.ndarray:
    """Centres moved by N(0, sigma^2) per coordinate; both particles of a pair whose moves violate
    the separation rule, and a particle whose move violates burial, are re-drawn until the moved
    configuration is admissible (the inverse-problem truth of the gradient workload)."""
    rng = np.random.default_rng(seed)
    c = centres + rng.normal(0.0, sigma, centres.shape)

    def bad_set(c):
        bad = set(np.where(c[:, 1] + SEP * radius > 0.0)[0].tolist())
        rmax = float(radius.max())
        cell = 2.0 * SEP * rmax
        grid: dict[tuple[int, int], list[int]] = {}
        keys = np.floor(c / cell).astype(int)
        for i, (gx, gy) in enumerate(keys):
            grid.setdefault((gx, gy), []).append(i)
        for i, (gx, gy) in enumerate(keys):
            for ix in range(gx - 1, gx + 2):
                for iy in range(gy - 1, gy + 2):
                    for j in grid.get((ix, iy), ()):
                        if j > i and np.sum((c[i] - c[j]) ** 2) < (SEP * (radius[i] + radius[j])) ** 2:
                            bad.add(i)
                            bad.add(j)
        return sorted(bad)

    for _ in range(max_rounds):
        bad = bad_set(c)
        if not bad:
            return c
        c[bad] = centres[bad] + rng.normal(0.0, sigma, (len(bad), 2))
    raise RuntimeError("perturbation could not be made admissible")


def receiver_line(R: int, x0: float, x1: float, y: float) -> np.ndarray:
    xs = np.linspace(x0, x1, R)
    return np.stack([xs, np.full(R, y)], axis=1)


def contour_for_width(width: float, t_max: float = 20.0):
    """Sommerfeld rule for a particle cloud of horizontal extent `width`: depth 3 / width (at most
    the paper's 1/2), uniform panels of width ~ 8 pi / width (so that e^{i t dx} is resolved for
    every pair) and 4 grading levels at the branch points.  Returns (n_panels, depth, grade)."""
    depth = min(0.5, 3.0 / width)
    panel = min(1.25, 8.0 * math.pi / width)
    return int(math.ceil(2.0 * t_max / panel)), depth, 4


def config1(seed: int = 1002) -> Workload:
    """16 rigid discs R=0.5 in [-10,10]x[-8,-1], omega=2, p=10, one P-wave at 30 degrees."""
    rng = np.random.default_rng(seed)
    c, r = place_particles(rng, 16, (-10, 10, -8, -1), 0.5, 0.5)
    M = 16
    return Workload("discs16_p10", MEDIA_STD, 2.0, 10, c, r,
                    np.zeros(M, np.int32), np.zeros(M, np.int32), np.zeros(M),
                    np.zeros(1, np.int32), np.array([math.radians(30.0)]),
                    receiver_line(256, -12, 12, -0.5))


STAR_A2 = 0.2      # r(t) = a (1 + 0.2 cos(5 t)): the star of the workloads, enclosing radius 1.2 a
STAR_A3 = 5


def star_levels(rmin: float, rmax: float, Q: int) -> np.ndarray:
    """Q quantised enclosing radii, the midpoints of Q equal bins of [rmin, rmax]."""
    return rmin + (np.arange(Q) + 0.5) * (rmax - rmin) / Q


def _star_prototypes(levels: np.ndarray):
    """Prototype table of the stars: q = level + Q bc, shape (a, 0.2 a, 5) with a = R / 1.2."""
    Q = levels.size
    a = np.concatenate([levels, levels]) / (1.0 + STAR_A2)
    shape = np.stack([a, STAR_A2 * a, np.full(2 * Q, float(STAR_A3))], 1)
    return shape, np.repeat(np.arange(2, dtype=np.int32), Q)


def config2(seed: int = 1003, nrhs: int = 1, Q: int = 16) -> Workload:
    """1000 stars r(t) = a (1 + 0.2 cos 5t), a ~ U[0.3, 0.6] quantised to Q sizes (the finitely many
    prototype shapes of Sec. 2; reading), enclosing radius 1.2 a, rigid and traction-free alternating,
    random rotation, omega=4, p=16, in [-40,40]x[-30,-1]."""
    rng = np.random.default_rng(seed)
    M = 1000
    levels = star_levels(1.2 * 0.3, 1.2 * 0.6, Q)
    lev = np.empty(M, np.int64)

    def rad(g, n):
        lev[n] = g.integers(Q)
        return levels[lev[n]]

    c, r = place_particles(rng, M, (-40, 40, -30, -1), levels[0], levels[-1], radius_fn=rad)
    bc = (np.arange(M) % 2).astype(np.int32)
    rot = rng.uniform(0, 2 * math.pi, M)
    irng = np.random.default_rng(2003)
    ang = np.full(nrhs, math.radians(30.0)) if nrhs == 1 else np.radians(irng.uniform(10, 170, nrhs))
    npan, depth, grade = contour_for_width(float(c[:, 0].max() - c[:, 0].min()))
    shape, pbc = _star_prototypes(levels)
    return Workload("stars1000_p16", MEDIA_STD, 4.0, 16, c, r, bc,
                    np.ones(M, np.int32), rot, np.zeros(nrhs, np.int32), ang,
                    receiver_line(256, -40, 40, -0.5), proto=(lev + Q * bc).astype(np.int32),
                    proto_shape=shape, proto_bc=pbc, n_panels=npan, depth=depth, grade=grade)


def config3(seed: int = 1004, M: int = 10000, nrhs: int = 64, Q: int = 16) -> Workload:
    """10^4 particles, enclosing radius U[0.2,0.5], packing fraction 0.2 by enclosing area, omega=6,
    p=20, 64 plane waves (half P, half S) at angles U[10,170] degrees.  Even-numbered particles are
    discs with continuous radii; odd-numbered ones are stars r(t) = a (1 + 0.2 cos 5t) whose enclosing
    radius 1.2 a is one of Q quantised sizes (Q sizes x 2 boundary conditions = 2Q prototypes, random
    rotation).  Boundary conditions alternate rigid / traction-free within each kind.  `M` may be
    lowered for parity sub-cases; the box then shrinks to keep the packing fraction."""
    rng = np.random.default_rng(seed)
    er2 = (0.5 ** 3 - 0.2 ** 3) / (3 * 0.3)       # E[R^2] for R ~ U[0.2,0.5]
    area = M * math.pi * er2 / 0.2
    side = math.sqrt(area)
    levels = star_levels(0.2, 0.5, Q)
    lev = np.full(M, -1, np.int64)

    def rad(g, n):
        if n % 2 == 0:
            return g.uniform(0.2, 0.5)
        lev[n] = g.integers(Q)
        return levels[lev[n]]

    c, r = place_particles(rng, M, (-side / 2, side / 2, -side - 1.0, -1.0), 0.2, 0.5, radius_fn=rad)
    bc = ((np.arange(M) // 2) % 2).astype(np.int32)
    shape_kind = (np.arange(M) % 2).astype(np.int32)
    proto = np.where(shape_kind == 1, lev + Q * bc, -1).astype(np.int32)
    rot = rng.uniform(0, 2 * math.pi, M)
    irng = np.random.default_rng(2004)
    ang = np.radians(irng.uniform(10, 170, nrhs))
    kind = (np.arange(nrhs) >= nrhs // 2).astype(np.int32)
    npan, depth, grade = contour_for_width(float(c[:, 0].max() - c[:, 0].min()))
    shape, pbc = _star_prototypes(levels)
    return Workload(f"discs_stars{M}_p20_rhs{nrhs}", MEDIA_STD, 6.0, 20, c, r, bc,
                    shape_kind, rot, kind, ang,
                    receiver_line(256, -side / 2, side / 2, -0.5), proto=proto, proto_shape=shape,
                    proto_bc=pbc, n_panels=npan, depth=depth, grade=grade)


def config3_discs(seed: int = 1004, M: int = 10000, nrhs: int = 64) -> Workload:
    """The 10^4-particle workload with every particle a disc of continuous radius U[0.2, 0.5] (the
    substitute earlier measurements were quoted on)."""
    rng = np.random.default_rng(seed)
    er2 = (0.5 ** 3 - 0.2 ** 3) / (3 * 0.3)
    side = math.sqrt(M * math.pi * er2 / 0.2)
    c, r = place_particles(rng, M, (-side / 2, side / 2, -side - 1.0, -1.0), 0.2, 0.5)
    bc = (np.arange(M) % 2).astype(np.int32)
    rot = rng.uniform(0, 2 * math.pi, M)
    irng = np.random.default_rng(2004)
    ang = np.radians(irng.uniform(10, 170, nrhs))
    kind = (np.arange(nrhs) >= nrhs // 2).astype(np.int32)
    npan, depth, grade = contour_for_width(float(c[:, 0].max() - c[:, 0].min()))
    return Workload(f"discs{M}_p20_rhs{nrhs}", MEDIA_STD, 6.0, 20, c, r, bc,
                    np.zeros(M, np.int32), rot, kind, ang,
                    receiver_line(256, -side / 2, side / 2, -0.5), n_panels=npan, depth=depth, grade=grade)


def surrogate_tables(seed: int, ratio: np.ndarray, p: int) -> np.ndarray:
    """Seeded dense stand-ins (Q, 2nc, 2nc) for prototype scattering matrices, for timing only:
    N(0,1) + iN(0,1) entries times the order profile rho^|n| / |n|! of row and column, rho = ratio[q, b]
    supplied by the caller (small-particle matrices fall off like (k R / 2)^(|n|+|n'|) / (|n|! |n'|!)).
    They hold no scattering physics."""
    rng = np.random.default_rng(seed)
    Q = ratio.shape[0]
    nc = 2 * p + 1
    n = np.abs(np.arange(-p, p + 1))
    fact = np.array([math.factorial(int(k)) for k in n], float)
    prof = np.concatenate([ratio[:, 0:1] ** n[None, :] / fact, ratio[:, 1:2] ** n[None, :] / fact], 1)   # (Q, 2nc)
    z = rng.standard_normal((Q, 2 * nc, 2 * nc)) + 1j * rng.standard_normal((Q, 2 * nc, 2 * nc))
    return 0.5 * z * prof[:, :, None] * prof[:, None, :]


def config4(seed: int = 1005, M: int = 2000, nrhs: int = 32) -> Workload:
    """2000 rigid discs R ~ U[0.2,0.5], packing 0.2, omega=4, p=16, 32 P-waves, 128 receivers."""
    rng = np.random.default_rng(seed)
    er2 = (0.5 ** 3 - 0.2 ** 3) / (3 * 0.3)
    side = math.sqrt(M * math.pi * er2 / 0.2)
    c, r = place_particles(rng, M, (-side / 2, side / 2, -side - 1.0, -1.0), 0.2, 0.5)
    irng = np.random.default_rng(2005)
    ang = np.radians(irng.uniform(10, 170, nrhs))
    npan, depth, grade = contour_for_width(float(c[:, 0].max() - c[:, 0].min()))
    return Workload(f"discs{M}_p16_rhs{nrhs}", MEDIA_STD, 4.0, 16, c, r,
                    np.zeros(M, np.int32), np.zeros(M, np.int32), np.zeros(M),
                    np.zeros(nrhs, np.int32), ang, receiver_line(128, -side / 2, side / 2, -0.5),
                    n_panels=npan, depth=depth, grade=grade)


def small_case(seed: int, M: int, p: int, omega: float = 2.0, nrhs: int = 1,
               media: Media = MEDIA_STD, box=(-6.0, 6.0, -5.0, -1.0), rmin=0.3, rmax=0.6,
               mixed_bc: bool = True, n_panels: int = 32, nodes_per_panel: int = 16,
               t_max: float = 20.0, depth: float = 0.5, grade: int = 0) -> Workload:
    """A few particles for parity tests that the oracle finishes in seconds."""
    rng = np.random.default_rng(seed)
    c, r = place_particles(rng, M, box, rmin, rmax)
    bc = (np.arange(M) % 2).astype(np.int32) if mixed_bc else np.zeros(M, np.int32)
    irng = np.random.default_rng(seed + 1000)
    ang = np.radians(irng.uniform(10, 170, nrhs))
    kind = (np.arange(nrhs) % 2).astype(np.int32)
    return Workload(f"small{M}_p{p}", media, omega, p, c, r, bc, np.zeros(M, np.int32),
                    rng.uniform(0, 2 * math.pi, M), kind, ang,
                    receiver_line(32, box[0], box[1], -0.5), n_panels, nodes_per_panel, t_max,
                    depth=depth, grade=grade)


def random_coeffs(seed: int, M: int, p: int, nrhs: int) -> np.ndarray:
    """Random complex coefficient block in the library layout (M, 2, 2p+1, nrhs).

    Entries are N(0,1)+iN(0,1) scaled by 2^-|n| so high orders carry the small
    magnitudes that outgoing coefficients of well-resolved particles have."""
    rng = np.random.default_rng(seed)
    nc = 2 * p + 1
    z = rng.standard_normal((M, 2, nc, nrhs)) + 1j * rng.standard_normal((M, 2, nc, nrhs))
    n = np.abs(np.arange(-p, p + 1))
    return z * (0.5 ** n)[None, None, :, None]


@dataclasses.dataclass
class Workload3:
    """3D workload (Sec. 6): spheres below the interface z = 0 and plane waves from the upper layer."""
    name: str
    media: Media
    omega: float
    p: int
    centres: np.ndarray          # (M, 3)
    radius: np.ndarray           # (M,)
    bc: np.ndarray               # (M,) 0 rigid, 1 traction-free
    inc_kind: np.ndarray         # (nrhs,) 0 P, 1 SV, 2 SH
    inc_theta: np.ndarray        # (nrhs,) angle from the downward vertical
    inc_phi: np.ndarray          # (nrhs,) azimuth

    @property
    def M(self) -> int:
        return int(self.radius.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.inc_kind.shape[0])


def place_spheres(rng: np.random.Generator, M: int, box, rmin: float, rmax: float, max_tries: int = 200000):
    """Random sequential addition of M spheres in box = (x0, x1, y0, y1, z0, z1): radii U[rmin, rmax],
    centres uniform, rejected when |c_l - c_m| < 1.1 (R_l + R_m) or z + 1.1 R > 0."""
    x0, x1, y0, y1, z0, z1 = box
    c = np.empty((M, 3))
    r = np.empty(M)
    n = tries = 0
    while n < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"placement failed after {max_tries} tries ({n}/{M} placed)")
        rad = rng.uniform(rmin, rmax)
        x = np.array([rng.uniform(x0, x1), rng.uniform(y0, y1), rng.uniform(z0, z1)])
        if x[2] + SEP * rad > 0.0:
            continue
        if n and (np.linalg.norm(c[:n] - x[None, :], axis=1) < SEP * (r[:n] + rad)).any():
            continue
        c[n], r[n] = x, rad
        n += 1
    return c, r


def spheres3d(seed: int = 1006, M: int = 500, nrhs: int = 16, box=None, bc: str = "rigid", p: int = 8) -> Workload3:
    """The 3D workload: upper lam = 1, mu = 0.5, lower lam' = 2, mu' = 1, omega = 2; M spheres of radius
    U[0.3, 0.5] in [-15, 15]^2 x [-12, -1] (or the given box); order p; nrhs plane waves from the upper
    layer with seeded kinds (P, SV, SH), angles from the vertical U[10, 60] degrees and azimuths
    U[0, 2 pi).  bc: "rigid" (every sphere), or "alternate" (rigid and traction-free by index parity)."""
    rng = np.random.default_rng(seed)
    box = box or (-15.0, 15.0, -15.0, 15.0, -12.0, -1.0)
    c, r = place_spheres(rng, M, box, 0.3, 0.5)
    b = np.zeros(M, dtype=np.int32) if bc == "rigid" else (np.arange(M) % 2).astype(np.int32)
    irng = np.random.default_rng(seed + 1000)
    kinds = irng.integers(0, 3, size=nrhs).astype(np.int32)
    th = np.deg2rad(irng.uniform(10.0, 60.0, size=nrhs))
    ph = irng.uniform(0.0, 2.0 * np.pi, size=nrhs)
    return Workload3(f"spheres{M}_p{p}_rhs{nrhs}", Media(1.0, 0.5, 2.0, 1.0), 2.0, p, c, r, b, kinds, th, ph)
