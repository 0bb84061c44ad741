"""Seeded synthetic inputs for the first-order (Blatter-Pattyn) Stokes assembly.

This module is the only code shared by the CUDA path's tests/bench and the CPU oracle.
It holds input generation only -- meshes, geometry fields, sliding coefficients and
velocity vectors -- and none of the method's arithmetic (no basis functions, no
quadrature, no viscosity, no residual).  Every random number is drawn here from
numpy's PCG64 with an explicit seed and handed to both sides as data.

Geometry follows the paper's "topologically extruded" setting (Sec. 2): a 2D base
triangulation extruded vertically by sigma layers, z = b + sigma * H, so the margins
are vertical.  The synthetic problem (dome, bed, beta) stands in for the paper's
Greenland / Antarctica datasets, which are not available:

* base mesh: an m x m grid on [-220, 220]^2 km whose interior points are jittered by
  up to +-0.2 h per coordinate (boundary points slide along their edge), every quad
  split along the diagonal chosen by the in-circle predicate, i.e. the Delaunay
  triangulation of the jittered points; triangles counter-clockwise;
* surface: the radially symmetric dome s(r) = H0 (1 - (r/R)^(4/3))^(3/7), R = 200 km,
  floored at H_min = 10 m so the whole square carries ice;
* bed: flat (H = s), or b = A_b sin(2 pi x / lam) sin(2 pi y / lam) with A_b = 500 m, lam = 20 km
  beneath the same surface (H = max(s - b, H_min));
* beta: lognormal with mean 1e3 Pa yr / m and log-sd 0.5, either iid per vertex or a
  Gaussian field with 10 km correlation length built from 512 random Fourier features;
* velocities: iid uniform in [-100, 100] m/yr per node and component.

Degrees of freedom are numbered column-major and interleaved:
dof(a, l, c) = 2 * (a * (L + 1) + l) + c for base vertex a, node level l, component c
(c = 0 for u, 1 for v).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RHO_ICE = 910.0       # kg m^-3
RHO_WATER = 1028.0    # kg m^-3 (sea water)
GRAVITY = 9.81        # m s^-2
GLEN_N = 3.0
RATE_FACTOR = 1e-16   # Pa^-3 yr^-1
DELTA = 1e-10         # yr^-2, regularises the effective strain rate at U = 0
HALF_WIDTH = 220e3    # m
DOME_RADIUS = 200e3   # m
H_MIN = 10.0          # m
BED_AMPLITUDE = 500.0  # m
BED_WAVELENGTH = 20e3  # m
BETA_MEAN = 1e3       # Pa yr m^-1
BETA_LOG_SD = 0.5
BETA_CORR_LEN = 10e3  # m
N_FOURIER = 512


@dataclasses.dataclass
class Params:
    """Physical constants (units m, yr, Pa)."""

    n: float = GLEN_N
    A: float = RATE_FACTOR
    rho: float = RHO_ICE
    g: float = GRAVITY
    delta: float = DELTA
    rho_w: float = RHO_WATER
    margin: int = 0       # 0: stress-free lateral margin; 1: cryostatic pressure against the ocean

    def as_array(self) -> np.ndarray:
        return np.array([self.n, self.A, self.rho, self.g, self.delta], dtype=np.float64)


@dataclasses.dataclass
class Mesh:
    """An extruded wedge mesh: base triangulation + per-vertex fields + sigma levels."""

    xy: np.ndarray      # [nv, 2] float64
    tri: np.ndarray     # [ntri, 3] int32, counter-clockwise
    bed: np.ndarray     # [nv] float64
    thick: np.ndarray   # [nv] float64
    beta: np.ndarray    # [nv] float64
    sigma: np.ndarray   # [nlayers + 1] float64, 0 = bed ... 1 = surface
    params: Params = dataclasses.field(default_factory=Params)
    name: str = ""
    rate_factor: np.ndarray | None = None  # [nv * (L + 1)] nodal A (Pa^-3 yr^-1), node a (L + 1) + l

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def ntri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nlayers(self) -> int:
        return int(self.sigma.shape[0] - 1)

    @property
    def nwedges(self) -> int:
        return self.ntri * self.nlayers

    @property
    def ndof(self) -> int:
        return 2 * self.nv * (self.nlayers + 1)

    def dof(self, a, l, c):
        return 2 * (np.asarray(a) * (self.nlayers + 1) + np.asarray(l)) + np.asarray(c)

    def edges(self) -> np.ndarray:
        """Unique undirected base edges [E, 2] (sorted pairs)."""
        t = self.tri.astype(np.int64)
        e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
        e.sort(axis=1)
        return np.unique(e, axis=0)

    def expected_nnz(self) -> int:
        """Size of the extruded pattern: 4 (V + 2E)(3L + 1).

        Each base vertex pair (a, b) with a == b or a ~ b couples node levels |l - l'| <= 1,
        i.e. (L + 1) + 2L = 3L + 1 level pairs, times 4 component pairs.
        """
        return 4 * (self.nv + 2 * len(self.edges())) * (3 * self.nlayers + 1)


def _incircle(ax, ay, bx, by, cx, cy, dx, dy):
    """Sign of the in-circle determinant: > 0 when d lies inside the circle abc (abc CCW)."""
    adx, ady = ax - dx, ay - dy
    bdx, bdy = bx - dx, by - dy
    cdx, cdy = cx - dx, cy - dy
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            - (bdx * bdx + bdy * bdy) * (adx * cdy - cdx * ady)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def jittered_grid(m: int, seed: int, half_width: float = HALF_WIDTH, jitter: float = 0.2):
    """Jittered m x m grid triangulated by the Delaunay (in-circle) diagonal choice.

    Returns (xy [nv,2], tri [2 m^2, 3] int32 CCW).  Vertex (i, j) has index j * (m+1) + i.
    """
    rng = np.random.default_rng(seed)
    n1 = m + 1
    h = 2.0 * half_width / m
    gx, gy = np.meshgrid(np.arange(n1), np.arange(n1), indexing="xy")  # gx varies along axis 1
    x = -half_width + gx * h
    y = -half_width + gy * h
    jx = rng.uniform(-jitter * h, jitter * h, size=x.shape)
    jy = rng.uniform(-jitter * h, jitter * h, size=y.shape)
    # boundary points slide only along their edge; corners stay fixed
    on_x_edge = (gx == 0) | (gx == m)
    on_y_edge = (gy == 0) | (gy == m)
    jx = np.where(on_x_edge, 0.0, jx)
    jy = np.where(on_y_edge, 0.0, jy)
    xy = np.stack([(x + jx).ravel(), (y + jy).ravel()], axis=1)

    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    v00 = j * n1 + i
    v10 = v00 + 1
    v01 = v00 + n1
    v11 = v01 + 1
    # quad v00 v10 v11 v01 (CCW).  Diagonal v00-v11 unless v01 lies inside circle(v00, v10, v11).
    P = xy
    inside = _incircle(P[v00, 0], P[v00, 1], P[v10, 0], P[v10, 1], P[v11, 0], P[v11, 1],
                       P[v01, 0], P[v01, 1]) > 0
    t_a = np.where(inside[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    t_b = np.where(inside[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    tri = np.empty((2 * m * m, 3), dtype=np.int32)
    tri[0::2] = t_a
    tri[1::2] = t_b
    return xy, tri


def dome_thickness(xy: np.ndarray, H0: float = 2000.0, R: float = DOME_RADIUS,
                   h_min: float = H_MIN) -> np.ndarray:
    r = np.hypot(xy[:, 0], xy[:, 1])
    core = np.clip(1.0 - (r / R) ** (4.0 / 3.0), 0.0, None)
    return np.maximum(H0 * core ** (3.0 / 7.0), h_min)


def sinusoidal_bed(xy: np.ndarray, amplitude: float = BED_AMPLITUDE,
                   wavelength: float = BED_WAVELENGTH) -> np.ndarray:
    k = 2.0 * math.pi / wavelength
    return amplitude * np.sin(k * xy[:, 0]) * np.sin(k * xy[:, 1])


def lognormal_beta_iid(nv: int, seed: int, mean: float = BETA_MEAN, log_sd: float = BETA_LOG_SD):
    rng = np.random.default_rng(seed)
    mu = math.log(mean) - 0.5 * log_sd ** 2
    return np.exp(rng.normal(mu, log_sd, size=nv))


def lognormal_beta_field(xy: np.ndarray, seed: int, mean: float = BETA_MEAN,
                         log_sd: float = BETA_LOG_SD, corr_len: float = BETA_CORR_LEN,
                         nfeat: int = N_FOURIER) -> np.ndarray:
    """Correlated lognormal field from random Fourier features (Gaussian covariance)."""
    rng = np.random.default_rng(seed)
    kvec = rng.normal(0.0, 1.0 / corr_len, size=(nfeat, 2))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=nfeat)
    field = np.zeros(xy.shape[0])
    chunk = 65536
    for s in range(0, xy.shape[0], chunk):
        arg = xy[s:s + chunk] @ kvec.T + phase[None, :]
        field[s:s + chunk] = np.cos(arg).sum(axis=1)
    field = (field - field.mean()) / field.std()
    mu = math.log(mean) - 0.5 * log_sd ** 2
    return np.exp(mu + log_sd * field)


def lognormal_beta_field_torch(xy: np.ndarray, seed: int, device, mean: float = BETA_MEAN,
                               log_sd: float = BETA_LOG_SD, corr_len: float = BETA_CORR_LEN,
                               nfeat: int = N_FOURIER):
    """The same field as `lognormal_beta_field` (same seeded draws, same formula), evaluated in FP64
    with torch on `device` -- for generating many fields quickly.  Returns a numpy array."""
    import torch
    rng = np.random.default_rng(seed)
    kvec = rng.normal(0.0, 1.0 / corr_len, size=(nfeat, 2))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=nfeat)
    P = torch.as_tensor(xy, dtype=torch.float64, device=device)
    arg = P @ torch.as_tensor(kvec.T, device=device) + torch.as_tensor(phase, device=device)[None, :]
    field = torch.cos(arg).sum(dim=1)
    field = (field - field.mean()) / field.std(correction=0)
    mu = math.log(mean) - 0.5 * log_sd ** 2
    return torch.exp(mu + log_sd * field).cpu().numpy()


def uniform_sigma(nlayers: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, nlayers + 1)


def random_velocity(mesh: Mesh, seed: int, amplitude: float = 100.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=mesh.ndof)


def dome_mesh(m: int, nlayers: int, mesh_seed: int, beta_seed: int, H0: float = 2000.0,
              bed: str = "flat", beta: str = "iid", name: str = "") -> Mesh:
    """Dome ice sheet on a jittered grid.  With the sinusoidal bed the ice surface keeps the dome
    shape s(r) and the bed undulates beneath it (H = max(s - b, H_min)), as in bumpy-bed benchmark
    set-ups; lifting the whole dome onto the bumps would give 15 % surface slopes."""
    xy, tri = jittered_grid(m, mesh_seed)
    surface = dome_thickness(xy, H0=H0)
    if bed == "flat":
        b = np.zeros(xy.shape[0])
        thick = surface
    else:
        b = sinusoidal_bed(xy)
        thick = np.maximum(surface - b, H_MIN)
    be = (lognormal_beta_iid(xy.shape[0], beta_seed) if beta == "iid"
          else lognormal_beta_field(xy, beta_seed))
    return Mesh(xy=xy, tri=tri, bed=b, thick=thick, beta=be, sigma=uniform_sigma(nlayers),
                name=name)


def marine_mesh(m: int, nlayers: int, mesh_seed: int, beta_seed: int, H0: float = 2000.0, front: float = 60.0,
                name: str = "") -> Mesh:
    """Marine-terminating ice cap for the ocean margin condition: the whole square is ice whose
    surface follows the dome profile from H0 at the centre down to `front` at the distance of the
    square's half width (and stays at `front` beyond it), on a bed that dips from +200 m at the
    centre to -300 m there.  The square's boundary is then a grounded calving front 360 m thick with
    its lower 300 m below sea level, just above flotation (rho_w / rho 300 m = 339 m): the ice and
    water pressures on the front nearly balance, as at real tidewater fronts."""
    xy, tri = jittered_grid(m, mesh_seed)
    r = np.minimum(np.hypot(xy[:, 0], xy[:, 1]) / HALF_WIDTH, 1.0)
    core = np.clip(1.0 - r ** (4.0 / 3.0), 0.0, None)
    surface = front + (H0 - front) * core ** (3.0 / 7.0)
    b = 200.0 - 500.0 * r
    return Mesh(xy=xy, tri=tri, bed=b, thick=surface - b, beta=lognormal_beta_field(xy, beta_seed),
                sigma=uniform_sigma(nlayers), params=Params(margin=1), name=name)


SECONDS_PER_YEAR = 365.25 * 86400.0
GAS_CONSTANT = 8.314         # J mol^-1 K^-1


def arrhenius_rate_factor(mesh: Mesh, T_centre: float = -30.0, T_margin: float = -15.0,
                          T_bed: float = -2.0) -> np.ndarray:
    """Nodal rate factor A [nv * (L + 1)] (Pa^-3 yr^-1) from a synthetic pressure-corrected
    temperature field by the Arrhenius relation A = A0 exp(-Q / (R T*)): the surface temperature
    rises linearly with the distance from the centre (T_centre to T_margin at the dome radius), the
    bed is at T_bed, and T* is linear in sigma between them.  Constants: the two-regime values of
    Cuffey and Paterson (2010), A(-10 C) = 3.5e-25 s^-1 Pa^-3, Q = 60 kJ/mol below -10 C and
    115 kJ/mol above, with A0 = A(-10 C) exp(Q / (R 263.15 K)) in each regime."""
    r = np.minimum(np.hypot(mesh.xy[:, 0], mesh.xy[:, 1]) / DOME_RADIUS, 1.0)
    Ts = T_centre + (T_margin - T_centre) * r
    L = mesh.nlayers
    T = np.empty((mesh.nv, L + 1))
    for l in range(L + 1):
        T[:, l] = T_bed + (Ts - T_bed) * mesh.sigma[l]
    Tk = 273.15 + T
    Q = np.where(Tk < 263.15, 6.0e4, 1.15e5)
    A0 = 3.5e-25 * np.exp(Q / (GAS_CONSTANT * 263.15))
    return (A0 * np.exp(-Q / (GAS_CONSTANT * Tk)) * SECONDS_PER_YEAR).reshape(-1)


# ---------------------------------------------------------------- named workloads

def config_small() -> Mesh:
    """Dome on a 32 x 32 jittered grid (2,048 triangles) x 5 layers = 10,240 wedges, flat bed."""
    return dome_mesh(32, 5, 101, 102, bed="flat", beta="iid", name="dome-2k-tri-x5")


def config_medium() -> Mesh:
    """224 x 224 grid (100,352 triangles) x 10 layers = 1,003,520 wedges, sinusoidal bed."""
    return dome_mesh(224, 10, 201, 202, bed="sinusoidal", beta="field", name="dome-100k-tri-x10")


def config_large() -> Mesh:
    """447 x 447 grid (399,618 triangles) x 10 layers = 3,996,180 wedges, sinusoidal bed."""
    return dome_mesh(447, 10, 301, 302, bed="sinusoidal", beta="field", name="dome-400k-tri-x10")


def config_marine() -> Mesh:
    """Marine ice cap with the ocean margin condition: 224 x 224 grid x 10 layers = 1,003,520 wedges."""
    return marine_mesh(224, 10, 501, 502, name="marine-100k-tri-x10")


def ensemble_members(count: int = 64, seed0: int = 4000, scale: float = 1.0):
    """Uneven ensemble: member i has T in [5k, 50k] triangles, L in [5, 20], H0 in [1, 3] km.

    `scale` shrinks the triangle counts (for small tests); the draw per member is seeded
    by seed0 + i so any subset of members is reproducible on its own.
    """
    members = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        T = rng.uniform(5e3, 50e3) * scale
        L = int(rng.integers(5, 21))
        H0 = float(rng.uniform(1000.0, 3000.0))
        m = max(2, int(round(math.sqrt(T / 2.0))))
        members.append(dome_mesh(m, L, seed0 + i, seed0 + 1000 + i, H0=H0, bed="sinusoidal",
                                 beta="field", name=f"member{i}"))
    return members


def slab_mesh(m: int, nlayers: int, slope: float, thickness: float, beta: float,
              half_width: float = 20e3, seed: int = 7, jitter: float = 0.0) -> Mesh:
    """Inclined slab: constant H, surface and bed both of slope `slope` in x."""
    xy, tri = jittered_grid(m, seed, half_width=half_width, jitter=jitter)
    b = slope * xy[:, 0]
    return Mesh(xy=xy, tri=tri, bed=b, thick=np.full(xy.shape[0], thickness),
                beta=np.full(xy.shape[0], beta), sigma=uniform_sigma(nlayers), name="slab")


# ---------------------------------------------------------------- warm-start network test inputs

MLP_SHAPES = [(128, 16), (128,), (128, 128), (128,), (128, 128), (128,), (32, 128), (32,)]  # W1 b1 ... W4 b4


def dyadic_mlp_case(seed: int, n: int, density: float = 0.125):
    """A network and a batch whose values are short dyadic fractions: inputs k/4 (|k| <= 8), first-layer
    weights in {0, +-1/4, +-1/2}, deeper weights +-1/4 on a random `density` fraction of entries,
    biases k / 2^(2 layer + 2).  Every value is exactly a BF16 number with few significant bits, so
    the sums a network evaluation forms stay exact in FP32 (the oracle checks that per input).

    Returns (params float32 [39328] in the parameter layout W1, b1, ..., W4, b4 (weights row-major,
    out x in), X float64 [n, 16], E float64 [n, 32] output errors k/8, |k| <= 8, from which a test
    builds targets T = Y - E)."""
    rng = np.random.default_rng(seed)
    parts = []
    for layer, (wshape, bshape) in enumerate(zip(MLP_SHAPES[0::2], MLP_SHAPES[1::2])):
        if layer == 0:
            W = rng.choice(np.array([-0.5, -0.25, 0.0, 0.0, 0.25, 0.5]), size=wshape)
        else:
            W = np.where(rng.random(wshape) < density, rng.choice(np.array([-0.25, 0.25]), size=wshape), 0.0)
        b = rng.integers(-16, 17, size=bshape) / float(2 ** (2 * layer + 4))
        parts += [W.ravel(), b]
    params = np.concatenate(parts).astype(np.float32)
    X = rng.integers(-8, 9, size=(n, 16)) / 4.0
    E = rng.integers(-8, 9, size=(n, 32)) / 8.0
    return params, X, E
