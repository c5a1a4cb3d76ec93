"""Seeded synthetic workloads for the QTT wave stepper.

This module only *generates inputs*: velocity grids, the Ricker source time
function, source and receiver positions, and random tensor-train cores for
timing.  It holds none of the method's arithmetic (no encoding, no operator,
no truncation), so both the FP64 oracle and the CUDA path can consume what it
produces without sharing any computational code.

Physical setup (Sec. 2, Eq. 1-2 and Sec. 5 of the paper): a square grid of
N = 2^n points per axis, spacing dh, time step dt, velocity c(x, z) > 0.  Grids
are stored row-major as c[x, z] with x horizontal and z depth (z = 0 at the
surface), i.e. flat index x * N + z.

The paper's own model (a 256x256 window of Marmousi, Sec. 5) is not available
here; the layered / folded / faulted generators below stand in for it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "CONFIGS",
    "config",
    "paper_run",
    "variant",
    "qtt3d_run",
    "layered_model_3d",
    "layered_model",
    "ricker",
    "random_tt_cores",
    "constant_model",
]


# ---------------------------------------------------------------------------
# velocity models
# ---------------------------------------------------------------------------
def constant_model(n: int, c: float) -> np.ndarray:
    """Homogeneous medium, c(x, z) = c on a 2^n x 2^n grid."""
    N = 1 << n
    return np.full((N, N), float(c), dtype=np.float64)


def layered_model(
    n: int,
    dh: float,
    seed: int,
    n_layers: int = 30,
    v_top: float = 1600.0,
    v_bottom: float = 4500.0,
    noise: float = 0.05,
    n_faults: int = 3,
    water_velocity: float = 1500.0,
    water_frac: float = 0.05,
    anticline: bool = False,
) -> np.ndarray:
    """Seeded layered, folded and faulted velocity section (m/s).

    * water (``water_velocity``) down to z_w = water_frac * N * dh;
    * ``n_layers`` interfaces at base depths evenly spaced in (z_w, N*dh),
      each displaced by A*sin(2*pi*x/Lambda + phi) with A ~ U[5, 40] m,
      Lambda ~ U[0.5, 2] km, phi ~ U[0, 2*pi);
    * optional anticline uplift -H*exp(-(x-x0)^2 / (2 W^2)) with
      H ~ U[100, 300] m, W ~ U[0.1, 0.2]*N*dh, x0 ~ U[0.3, 0.7]*N*dh;
    * layer velocity ramps linearly v_top -> v_bottom with layer index, times
      (1 + U[-noise, noise]) per layer;
    * ``n_faults`` normal faults: surface position ~ U[0, N*dh], dip
      U[55, 70] degrees, throw U[20, 80] m; the hanging wall takes
      c(x, z - throw).
    """
    rng = np.random.default_rng(seed)
    N = 1 << n
    L = N * dh
    x = (np.arange(N) + 0.5) * dh
    z = (np.arange(N) + 0.5) * dh
    X, Z = np.meshgrid(x, z, indexing="ij")  # [x, z]

    z_w = water_frac * L
    base = np.linspace(z_w, L, n_layers + 2)[1:-1]
    amp = rng.uniform(5.0, 40.0, n_layers)
    lam = rng.uniform(500.0, 2000.0, n_layers)
    phase = rng.uniform(0.0, 2.0 * np.pi, n_layers)
    lay_noise = 1.0 + rng.uniform(-noise, noise, n_layers + 1)
    if anticline:
        H = rng.uniform(100.0, 300.0)
        W = rng.uniform(0.1, 0.2) * L
        x0 = rng.uniform(0.3, 0.7) * L
        uplift = -H * np.exp(-((x - x0) ** 2) / (2.0 * W * W))
    else:
        uplift = np.zeros(N)
    f_x = rng.uniform(0.0, L, n_faults)
    f_dip = np.deg2rad(rng.uniform(55.0, 70.0, n_faults))
    f_throw = rng.uniform(20.0, 80.0, n_faults)

    # faults move the hanging wall down: the value at depth z comes from z - throw
    Zeff = Z.copy()
    for xf, dip, thr in zip(f_x, f_dip, f_throw):
        hanging = X > xf + Z / math.tan(dip)
        Zeff = np.where(hanging, Zeff - thr, Zeff)

    layer = np.zeros((N, N), dtype=np.int64)
    for i in range(n_layers):
        depth_i = base[i] + amp[i] * np.sin(2.0 * np.pi * x / lam[i] + phase[i]) + uplift
        layer += (Zeff >= depth_i[:, None]).astype(np.int64)
    ramp = v_top + (v_bottom - v_top) * layer / max(n_layers, 1)
    c = ramp * lay_noise[layer]
    c = np.where(Z < z_w, water_velocity, c)
    return c.astype(np.float64)


def layered_model_3d(n: int, dh: float, seed: int, n_layers: int = 20, v_top: float = 1600.0,
                     v_bottom: float = 4500.0, noise: float = 0.05, water_velocity: float = 1500.0,
                     water_frac: float = 0.05) -> np.ndarray:
    """Seeded layered and folded 3D velocity block c[x, y, z] (m/s): water
    down to z_w = water_frac * N * dh, then n_layers interfaces at base depths
    evenly spaced in (z_w, N*dh), each displaced by
    A sin(2 pi x / Lx + phi) + B sin(2 pi y / Ly + psi) with A, B ~ U[5, 40] m,
    Lx, Ly ~ U[0.5, 2] km, phases ~ U[0, 2 pi); velocity ramping
    v_top -> v_bottom with layer index, times (1 + U[-noise, noise]) per layer."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    L = N * dh
    x = (np.arange(N) + 0.5) * dh
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    z_w = water_frac * L
    base = np.linspace(z_w, L, n_layers + 2)[1:-1]
    A, B = rng.uniform(5.0, 40.0, n_layers), rng.uniform(5.0, 40.0, n_layers)
    Lx, Ly = rng.uniform(500.0, 2000.0, n_layers), rng.uniform(500.0, 2000.0, n_layers)
    px, py = rng.uniform(0.0, 2.0 * np.pi, n_layers), rng.uniform(0.0, 2.0 * np.pi, n_layers)
    lay_noise = 1.0 + rng.uniform(-noise, noise, n_layers + 1)
    layer = np.zeros((N, N, N), dtype=np.int64)
    for i in range(n_layers):
        depth = base[i] + A[i] * np.sin(2 * np.pi * X / Lx[i] + px[i]) + B[i] * np.sin(2 * np.pi * Y / Ly[i] + py[i])
        layer += (Z >= depth).astype(np.int64)
    c = (v_top + (v_bottom - v_top) * layer / max(n_layers, 1)) * lay_noise[layer]
    return np.where(Z < z_w, water_velocity, c).astype(np.float64)


# ---------------------------------------------------------------------------
# source time function
# ---------------------------------------------------------------------------
def ricker(t: np.ndarray | float, f: float) -> np.ndarray:
    """Ricker wavelet w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
    tau = t - 1.5/f (so w(0) is ~1e-8 of the peak)."""
    tau = np.asarray(t, dtype=np.float64) - 1.5 / f
    a = (np.pi * f * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


# ---------------------------------------------------------------------------
# random tensor-train cores (timing inputs only)
# ---------------------------------------------------------------------------
def tt_rank_profile(d: int, chi: int) -> list[int]:
    """Bond sizes r_0..r_d = min(2^k, 2^(d-k), chi), the largest ranks a
    d-site binary tensor train can have under the cap chi."""
    return [min(2 ** k, 2 ** (d - k), chi) for k in range(d + 1)]


def random_tt_cores(d: int, chi: int, seed: int, decay: float = 0.0) -> list[np.ndarray]:
    """Gaussian cores [r_{k-1}][2][r_k] with the saturated rank profile.
    ``decay`` > 0 scales bond index j by exp(-decay*j) so that spectra decay."""
    rng = np.random.default_rng(seed)
    r = tt_rank_profile(d, chi)
    cores = []
    for k in range(d):
        g = rng.standard_normal((r[k], 2, r[k + 1]))
        if decay > 0.0:
            g *= np.exp(-decay * np.arange(r[k + 1]))[None, None, :]
        cores.append(g / math.sqrt(2 * r[k]))
    return cores


# ---------------------------------------------------------------------------
# benchmark configurations
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    n: int
    dh: float
    f_peak: float
    steps: int
    chi: int
    eps: float
    order: str  # "interleaved" | "sequential"
    bc: str  # "periodic" | "zero"
    precision: str  # "fp64" | "tf32" | "bf16" | "fp32"
    model: str
    seed: int
    chi_c: int
    eps_c: float
    sources: list[tuple[int, int]]
    receivers: list[tuple[int, int]]
    dt_fixed: float | None = None  # a time step given by the run, else 0.5 dh / c_max
    dims: int = 2  # 3: the 3D extension, points (ix, iy, iz)

    @property
    def N(self) -> int:
        return 1 << self.n

    @property
    def d(self) -> int:
        return self.dims * self.n

    def velocity(self) -> np.ndarray:
        if self.model == "constant":
            return constant_model(self.n, 2000.0)
        if self.model == "layered":
            return layered_model(self.n, self.dh, self.seed)
        if self.model == "layered3d":
            return layered_model_3d(self.n, self.dh, self.seed)
        if self.model == "marmousi":
            return layered_model(
                self.n, self.dh, self.seed, n_layers=120, v_top=1500.0,
                v_bottom=5500.0, n_faults=8, anticline=True)
        raise ValueError(self.model)

    def dt(self, c: np.ndarray) -> float:
        """dt = 0.5 * dh / c_max (Courant number 0.5 < 1/sqrt(2)) in 2D,
        0.5 * dh / (c_max sqrt(3/2)) (Courant number 0.41 < 1/sqrt(3)) in 3D,
        unless the run fixes it."""
        if self.dt_fixed is not None:
            return self.dt_fixed
        return 0.5 * self.dh / float(np.max(c)) / (math.sqrt(1.5) if self.dims == 3 else 1.0)

    def lambda2(self, c: np.ndarray) -> float:
        """lambda^2 = (dt/dh)^2, the squared mesh ratio of Eq. 2."""
        return (self.dt(c) / self.dh) ** 2

    def source_amplitudes(self, c: np.ndarray, steps: int | None = None) -> np.ndarray:
        """s_k = lambda^2 * w(k dt): a point force of unit strength, i.e. the
        discrete delta(x - x_s)/dh^2 scaled by dt^2, added into u^{k+1}."""
        steps = self.steps if steps is None else steps
        dt = self.dt(c)
        return self.lambda2(c) * ricker(np.arange(steps) * dt, self.f_peak)


def _cfg(idx: int) -> Workload:
    if idx == 0:  # 64x64, constant c, centre source
        n = 6
        N = 1 << n
        return Workload("qtt64_const", n, 10.0, 15.0, 300, 32, 1e-10, "interleaved",
                        "periodic", "fp64", "constant", 1, 32, 1e-8,
                        [(N // 2, N // 2)], [(8 * i, 2) for i in range(N // 8)])
    if idx == 1:  # 256x256 layered model
        n = 8
        N = 1 << n
        return Workload("qtt256_layered", n, 12.5, 20.0, 1000, 64, 1e-7, "interleaved",
                        "periodic", "fp64", "layered", 2, 64, 1e-8,
                        [(N // 2, 2)], [(8 * i, 2) for i in range(N // 8)])
    if idx == 2:  # 1024x1024 Marmousi-shaped section (the headline workload)
        n = 10
        N = 1 << n
        return Workload("qtt1024_marmousi", n, 4.0, 25.0, 4000, 128, 1e-6, "interleaved",
                        "periodic", "bf16", "marmousi", 3, 128, 1e-8,
                        [(N // 2, 2)], [(8 * i, 2) for i in range(N // 8)])
    if idx == 3:  # 64 shots on 512x512 layered model
        n = 9
        N = 1 << n
        return Workload("qtt512_layered_64shots", n, 6.25, 20.0, 2000, 256, 1e-7,
                        "interleaved", "periodic", "fp32", "layered", 4, 64, 1e-8,
                        [(N // 128 + s * N // 64, 2) for s in range(64)],
                        [(8 * i, 2) for i in range(N // 8)])
    if idx == 4:  # 2048x2048 Marmousi-shaped, learned ranks
        n = 11
        N = 1 << n
        return Workload("qtt2048_marmousi", n, 2.0, 30.0, 8000, 256, 1e-5, "interleaved",
                        "periodic", "fp64", "marmousi", 5, 256, 1e-8,
                        [(N // 2, 2)], [(8 * i, 2) for i in range(N // 8)])
    raise IndexError(idx)


CONFIGS = [_cfg(i) for i in range(5)]


def config(idx: int) -> Workload:
    return _cfg(idx)


def paper_run() -> Workload:
    """The run of the paper's results section on a synthetic stand-in for its
    256 x 256 Marmousi window (the dataset is not available here): dh = 10 m,
    dt = 1 ms, an impulsive source of strength 1 at the centre (1280 m,
    1280 m) as the initial condition u^0 = e_src, u^-1 = 0, chi_max = 128,
    eps = 1e-7, 300 steps; the Marmousi-shaped generator (120 folded and
    faulted layers with an anticline, 1500-5500 m/s, +-5 % per layer) at
    seed 6.  Courant number c_max dt / dh = 0.574 < 1/sqrt(2)."""
    n = 8
    N = 1 << n
    return Workload("qtt256_paper_run", n, 10.0, 0.0, 300, 128, 1e-7, "interleaved", "periodic", "fp64",
                    "marmousi", 6, 128, 1e-8, [(N // 2, N // 2)], [(8 * i, 2) for i in range(N // 8)],
                    dt_fixed=1e-3)


def qtt3d_run(n: int = 6) -> Workload:
    """The 3D extension's workload: a 2^n-per-axis layered and folded block
    (20 interfaces, 1600 -> 4500 m/s under a water layer, seed 7), dh = 20 m,
    Ricker 8 Hz (about 12 points per wavelength at 2000 m/s) at (N/2, N/2, 2),
    chi_max = 64, eps = 1e-6, interleaved order, periodic boundaries, 600
    steps; receivers every 8 points along x at y = N/2, z = 2."""
    N = 1 << n
    return Workload(f"qtt{N}_3d_layered", n, 20.0, 8.0, 600, 64, 1e-6, "interleaved", "periodic", "fp64",
                    "layered3d", 7, 64, 1e-8, [(N // 2, N // 2, 2)], [(8 * i, N // 2, 2) for i in range(N // 8)],
                    dims=3)


def variant(idx: int, order: str, bc: str) -> Workload:
    """Configuration idx with another site order and boundary condition."""
    return dataclasses.replace(_cfg(idx), name=f"{_cfg(idx).name}_{order}_{bc}", order=order, bc=bc)


def chi_per_shot(seed: int = 4, shots: int = 64) -> np.ndarray:
    """Per-shot bond caps drawn uniformly from {32, 64, 128, 256}."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([32, 64, 128, 256]), size=shots)


def mlp_params(seed: int = 7, n_feat: int = 40, width: int = 128) -> np.ndarray:
    """Initial parameters of the rank-proposal MLP, flat float32 in the layout
    W1 (width x n_feat), b1, W2 (width x width), b2, W3 (1 x width), b3:
    weights uniform in +-sqrt(6 / fan_in) (He et al. 2015), biases zero,
    except b3 = 0.5 (the middle of the scaled-rank range)."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((width, n_feat), (width, width), (1, width)):
        lim = np.sqrt(6.0 / cols)
        parts.append(rng.uniform(-lim, lim, size=(rows, cols)).ravel())
        parts.append(np.zeros(rows))
    parts[-1][:] = 0.5
    return np.concatenate(parts).astype(np.float32)


def gaussian_sketch(seed: int = 11, rows: int = 1024, cols: int = 512) -> np.ndarray:
    """Fixed Gaussian test matrix (standard normal, float64, row-major) for the
    randomised range finder; bond k uses its top-left block."""
    return np.random.default_rng(seed).standard_normal((rows, cols))
