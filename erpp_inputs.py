"""Seeded synthetic inputs for the ERPP coupling step.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1405_6969_gb300``).  It holds no arithmetic of the method
itself: it draws particle clouds, particle properties and divergence-free
random velocity fields, and it defines the workloads by their sizes and
physical parameters.  Every array is float64 NumPy, structure-of-arrays:

* particle vectors are ``[3, n]`` (component-major),
* grid fields are ``[3, nz, ny, nx]`` with nodes at ``x_j = j * L / N``
  (the collocation points of a periodic pseudo-spectral grid, Sec. 3).

The workloads stand in for the paper's runs (Sec. 3 validation boxes and the
Sec. 4 homogeneous-shear run); no dataset is involved.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes and physical parameters of one synthetic coupling workload."""

    name: str
    n: tuple  # (nx, ny, nz)
    L: tuple  # (Lx, Ly, Lz)
    n_particles: int
    nu: float = 0.01
    rho_f: float = 1.0
    dt: float = 1e-3
    sigma_over_dx: float = 1.0  # Gaussian width sigma_R in grid spacings
    cutoff: float = 3.0  # stencil truncation radius in widths sigma_R
    kmax: float = 4.0  # random-field band limit |k| <= kmax
    field_seed: int = 0
    particle_seed: int = 0
    cloud: str = "uniform"  # "uniform" | "clusters"
    n_clusters: int = 50
    cluster_std: float = 0.05
    shear_rate: float = 0.0
    radius: float = 1e-3  # used when stokes_mix is None
    rho_ratio: float = 1000.0  # rho_p / rho_f when stokes_mix is None
    stokes_mix: tuple | None = None  # Stokes numbers in equal thirds
    mass_loading: float | None = None
    slip_std: float = 0.05
    gravity: tuple = (0.0, 0.0, 0.0)
    steps: int = 1

    @property
    def dx(self):
        return self.L[0] / self.n[0]

    @property
    def sigma_R(self):
        return self.sigma_over_dx * self.dx

    @property
    def eps_R(self):
        # Regularisation time for the requested Gaussian width, from the
        # definition sigma_R = sqrt(2 nu eps_R) (Sec. 2.3).
        return self.sigma_R ** 2 / (2.0 * self.nu)

    @property
    def n_nodes(self):
        return self.n[0] * self.n[1] * self.n[2]

    def params(self, **over):
        """Physical parameter dictionary understood by both the oracle and
        the CUDA binding."""
        d = dict(
            n=tuple(int(v) for v in self.n),
            L=tuple(float(v) for v in self.L),
            nu=self.nu,
            rho_f=self.rho_f,
            eps_R=self.eps_R,
            cutoff=self.cutoff,
            dt=self.dt,
            gravity=tuple(self.gravity),
            shear_rate=self.shear_rate,
        )
        d.update(over)
        return d

    def scaled(self, name, n, n_particles, L=None):
        """Same physics on another grid: keeps sigma_R / dx fixed."""
        return dataclasses.replace(self, name=name, n=tuple(n),
                                   n_particles=int(n_particles),
                                   L=tuple(L) if L is not None else self.L)


# --------------------------------------------------------------------------
# The workloads.  Sizes and parameters are the ones the coupling benchmark is
# defined on; quantities it leaves open take the values noted inline.
# --------------------------------------------------------------------------

CFG_SMALL = Workload(  # plain FP64 single step, 32^3, 1k particles
    name="box2pi_32cube_1k_sigma1dx", n=(32, 32, 32), L=(TWO_PI,) * 3,
    n_particles=1000, sigma_over_dx=1.0, kmax=4.0, field_seed=0,
    particle_seed=0, cloud="uniform", steps=1)

CFG_CLUSTERED = Workload(  # FP32 vs FP64, 128^3, 100k clustered particles
    name="box2pi_128cube_100k_clustered_sigma1.5dx", n=(128, 128, 128),
    L=(TWO_PI,) * 3, n_particles=100_000, sigma_over_dx=1.5, kmax=8.0,
    cloud="clusters", n_clusters=50, cluster_std=0.05, shear_rate=1.0,
    steps=10)

CFG_SHEAR = Workload(  # homogeneous-shear-like box, 1M particles
    name="shear_4pix2pix2pi_512x256x256_1M", n=(512, 256, 256),
    L=(2 * TWO_PI, TWO_PI, TWO_PI), n_particles=1_000_000,
    sigma_over_dx=1.0, kmax=8.0, cloud="uniform", shear_rate=1.0,
    stokes_mix=(0.1, 1.0, 10.0), mass_loading=0.4, steps=100)

CFG_CUBE256 = Workload(  # 256^3 with 1M particles
    name="box2pi_256cube_1M_sigma1dx", n=(256, 256, 256), L=(TWO_PI,) * 3,
    n_particles=1_000_000, sigma_over_dx=1.0, kmax=8.0, cloud="uniform",
    shear_rate=1.0, stokes_mix=(0.1, 1.0, 10.0), mass_loading=0.4)

CFG_ADJOINT = Workload(  # adjoint: 128^3, 100k uniform particles
    name="adjoint_128cube_100k_sigma1.5dx", n=(128, 128, 128),
    L=(TWO_PI,) * 3, n_particles=100_000, sigma_over_dx=1.5, kmax=4.0,
    cloud="uniform")

WORKLOADS = {w.name: w for w in (CFG_SMALL, CFG_CLUSTERED, CFG_SHEAR,
                                 CFG_CUBE256, CFG_ADJOINT)}


# --------------------------------------------------------------------------
# Random divergence-free band-limited field
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SpectralField:
    """u(x) = scale * sum_k Re(a_k exp(i k.x)), a_k perpendicular to k."""

    m: np.ndarray  # [K, 3] integer wave numbers (k = 2 pi m / L)
    k: np.ndarray  # [K, 3] physical wave vectors
    a: np.ndarray  # [K, 3] complex amplitudes (already scaled)

    def at_points(self, x: np.ndarray, chunk: int = 4096) -> np.ndarray:
        """Evaluate at points x [3, n] (float64, exact sum over modes)."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        for s in range(0, x.shape[1], chunk):
            xs = x[:, s:s + chunk]
            ph = np.exp(1j * (self.k @ xs))  # [K, c]
            out[:, s:s + chunk] = np.real(self.a.T @ ph)
        return out


def random_field(n, L, kmax, seed):
    """Draw a divergence-free random field with modes 0 < |k| <= kmax.

    For every integer wave-number triple m (k = 2 pi m / L) in lexicographic
    order with 0 < |k| <= kmax, each component gets N(0,1) + i N(0,1); the
    vector is then projected perpendicular to k.  Both k and -k are drawn,
    and u = sum Re(a_k exp(i k.x)).  The field is rescaled so that every
    component has unit rms over the grid nodes.

    Returns (grid [3, nz, ny, nx] float64, SpectralField for point values).
    """
    nx, ny, nz = (int(v) for v in n)
    Lx, Ly, Lz = (float(v) for v in L)
    rng = np.random.default_rng(seed)
    mmax = [int(math.floor(kmax * La / TWO_PI)) for La in (Lx, Ly, Lz)]
    ms, ks = [], []
    for mx in range(-mmax[0], mmax[0] + 1):
        for my in range(-mmax[1], mmax[1] + 1):
            for mz in range(-mmax[2], mmax[2] + 1):
                k = np.array([TWO_PI * mx / Lx, TWO_PI * my / Ly,
                              TWO_PI * mz / Lz])
                kk = float(k @ k)
                if kk == 0.0 or kk > kmax * kmax * (1 + 1e-12):
                    continue
                ms.append((mx, my, mz))
                ks.append(k)
    m = np.array(ms, dtype=np.int64).reshape(-1, 3)
    k = np.array(ks, dtype=np.float64).reshape(-1, 3)
    a = rng.standard_normal((len(m), 3)) + 1j * rng.standard_normal((len(m), 3))
    khat = k / np.linalg.norm(k, axis=1, keepdims=True)
    a = a - khat * np.sum(a * khat, axis=1, keepdims=True)
    for d, na in enumerate((nx, ny, nz)):
        assert 2 * mmax[d] < na, "band limit not resolved by the grid"
    # Grid values through one inverse FFT per component (exact for a
    # band-limited sum; numpy's ifftn carries the 1/N factor).
    ntot = nx * ny * nz
    grid = np.empty((3, nz, ny, nx), dtype=np.float64)
    try:
        import scipy.fft as sfft
        ifftn = lambda A: sfft.ifftn(A, workers=-1)  # noqa: E731
    except Exception:  # pragma: no cover
        ifftn = np.fft.ifftn
    for c in range(3):
        A = np.zeros((nz, ny, nx), dtype=np.complex128)
        np.add.at(A, (m[:, 2] % nz, m[:, 1] % ny, m[:, 0] % nx), a[:, c])
        grid[c] = np.real(ifftn(A)) * ntot
    rms = np.sqrt(np.mean(grid ** 2, axis=(1, 2, 3)))
    # a component with no admissible mode (boxes too thin for K_max on two
    # axes) stays identically zero
    rms = np.where(rms > 0.0, rms, 1.0)
    grid /= rms[:, None, None, None]
    a = a / rms[None, :]
    return grid, SpectralField(m=m, k=k, a=a)


# --------------------------------------------------------------------------
# Particle clouds and properties
# --------------------------------------------------------------------------

def uniform_positions(n_particles, L, seed):
    rng = np.random.default_rng(seed)
    L = np.asarray(L, dtype=np.float64)[:, None]
    return rng.random((3, n_particles)) * L


def wrap_into_box(x, L):
    """Map coordinates into [0, L) (periodic box)."""
    L = np.asarray(L, dtype=np.float64)[:, None]
    y = np.mod(x, L)
    y[y >= L] = 0.0
    return y


def clustered_positions(n_particles, L, n_clusters, std, seed):
    """Mixture of Gaussian clusters: centres uniform, each particle picks a
    centre uniformly and is offset by N(0, std^2) per axis, then wrapped."""
    rng = np.random.default_rng(seed)
    Lv = np.asarray(L, dtype=np.float64)[:, None]
    centres = rng.random((3, n_clusters)) * Lv
    which = rng.integers(0, n_clusters, size=n_particles)
    x = centres[:, which] + std * rng.standard_normal((3, n_particles))
    return wrap_into_box(x, L)


def particle_properties(w: Workload, n_particles=None, seed=None):
    """Per-particle radius and density (float64 arrays).

    Without a Stokes mix every particle has ``w.radius`` and density
    ``w.rho_ratio * rho_f``.  With a Stokes-number mix the particles are
    split in equal thirds with relaxation times tau_p = St * tau_eta, where
    tau_eta = sigma_R^2 / nu (the smallest flow scale is taken equal to
    sigma_R, as in the paper's shear run where the grid spacing is about
    one Kolmogorov length), and the common density is chosen so that the
    total particle mass divided by the fluid mass equals ``mass_loading``.
    """
    n = w.n_particles if n_particles is None else int(n_particles)
    rng = np.random.default_rng(w.particle_seed + 17 if seed is None else seed)
    if w.stokes_mix is None:
        radius = np.full(n, w.radius)
        rho_p = np.full(n, w.rho_ratio * w.rho_f)
        return radius, rho_p
    mu = w.rho_f * w.nu
    tau_eta = w.sigma_R ** 2 / w.nu
    cls = np.arange(n) % len(w.stokes_mix)
    rng.shuffle(cls)
    tau = np.asarray(w.stokes_mix, dtype=np.float64)[cls] * tau_eta
    V = float(np.prod(w.L))
    # mass loading Phi = sum_p rho_p (pi/6) d_p^3 / (rho_f V) with
    # d_p = sqrt(18 mu tau_p / rho_p): solve for the common rho_p.
    s = float(np.sum(tau ** 1.5))
    c = (math.pi / 6.0) * (18.0 * mu) ** 1.5 * s / (w.rho_f * V)
    rho_p_val = (c / w.mass_loading) ** 2
    d = np.sqrt(18.0 * mu * tau / rho_p_val)
    return 0.5 * d, np.full(n, rho_p_val)


@dataclasses.dataclass
class ParticleState:
    x: np.ndarray  # [3, n] positions in [0, L)
    v: np.ndarray  # [3, n]
    x_prev: np.ndarray  # [3, n]
    D: np.ndarray  # [3, n] force of the previous step
    radius: np.ndarray  # [n]
    rho_p: np.ndarray  # [n]

    @property
    def n(self):
        return self.x.shape[1]

    def copy(self):
        return ParticleState(*(np.array(a, copy=True) for a in
                               dataclasses.astuple(self)))


def make_particles(w: Workload, field: SpectralField | None = None,
                   n_particles=None, seed=None, prev_step=True):
    """Seeded particle state for a workload.

    Velocities: the fluid velocity at the particle (when ``field`` is given,
    evaluated exactly from its modes) plus the mean shear, plus N(0,
    slip_std^2) slip per component.  When ``prev_step`` is set, a previous
    position x_prev = x - dt v (wrapped) and a previous force D ~ N(0, s^2)
    with s the Stokes-drag scale of the slip are drawn as well, so that a
    step with the self-disturbance removal enabled has non-trivial inputs.
    """
    n = w.n_particles if n_particles is None else int(n_particles)
    seed = w.particle_seed if seed is None else seed
    if w.cloud == "uniform":
        x = uniform_positions(n, w.L, seed)
    elif w.cloud == "clusters":
        x = clustered_positions(n, w.L, w.n_clusters, w.cluster_std, seed)
    else:
        raise ValueError(w.cloud)
    rng = np.random.default_rng(seed + 1)
    v = w.slip_std * rng.standard_normal((3, n))
    if field is not None:
        v += field.at_points(x)
    v[0] += w.shear_rate * x[1]
    radius, rho_p = particle_properties(w, n, seed=seed + 17)
    x_prev = wrap_into_box(x - w.dt * v, w.L)
    mu = w.rho_f * w.nu
    D = (6.0 * math.pi * mu * radius)[None, :] * (
        w.slip_std * rng.standard_normal((3, n)))
    return ParticleState(x=x, v=v, x_prev=x_prev, D=D, radius=radius,
                         rho_p=rho_p)


def make_forces(n, scale, seed):
    """Independent N(0, scale^2) forces [3, n] (scatter-only inputs)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((3, n))


def make_grid(w: Workload, n=None, L=None, kmax=None, seed=None):
    """Random-field grid values for a workload (optionally on another grid)."""
    return random_field(n or w.n, L or w.L, w.kmax if kmax is None else kmax,
                        w.field_seed if seed is None else seed)


def batched_boxes(n_boxes=64, seed0=0):
    """The batched workload: independent periodic [0, 2 pi)^3 boxes, grid
    drawn from {64^3, 96^3, 128^3}, particle counts log-uniform in
    [1e3, 2e5], box i seeded with i.  sigma_R = dx, K_max = 4 field."""
    boxes = []
    for i in range(n_boxes):
        rng = np.random.default_rng(seed0 + i)
        g = int(rng.choice([64, 96, 128]))
        npart = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        boxes.append(Workload(name=f"box{i}", n=(g, g, g), L=(TWO_PI,) * 3,
                              n_particles=npart, sigma_over_dx=1.0, kmax=4.0,
                              field_seed=seed0 + i, particle_seed=seed0 + i,
                              cloud="uniform"))
    return boxes
