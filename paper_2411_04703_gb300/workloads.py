"""Seeded synthetic workloads shaped like the paper's runs.

This module holds the workload definitions (grid, boost, boundaries, beam, plasma and
undulator parameters in normalised units) and the seeded generators of the lab-frame
beam.  It contains none of the method's arithmetic (no Lorentz transform, no field
transform, no push, deposit or field update): both the CUDA path and the FP64 oracle
receive the same lab-frame arrays from here and transform them independently.

Normalised units (rule stated with Table I, Sec. "Electron propagation in vacuum"):
time in 1/w_n, length in c/w_n, momentum u = p/(m_e c), fields in m_e c w_n/e,
densities in n_n = eps0 m_e w_n^2/e^2.  w_n is the plasma frequency of the RRF
density gamma_R N_e with the rest mass, or 2 pi gamma_R c / lambda_u when the run has
no plasma.  The paper's datasets and input decks are not available; these seeded
inputs stand in for them with the shapes of Table I and of the beam described with
it (30 pC Gaussian electron beam).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

C_LIGHT = 2.99792458e8
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12

PERIODIC, PML, OPEN = 0, 1, 2


def omega_plasma(n_m3: float) -> float:
    """Electron plasma frequency (rad/s) of density n (m^-3) with the rest mass."""
    return math.sqrt(n_m3 * Q_E * Q_E / (EPS0 * M_E))


def density_unit(omega_n: float) -> float:
    """n_n = eps0 m_e w_n^2 / e^2 in m^-3."""
    return EPS0 * M_E * omega_n * omega_n / (Q_E * Q_E)


@dataclasses.dataclass
class Beam:
    n: int                      # macroparticles
    gamma: float                # mean lab Lorentz factor
    rel_spread: float           # rms relative energy spread (lab)
    emit_n: float               # normalised rms emittance (normalised length units)
    sigma_r: float              # rms transverse size (lab = RRF), normalised
    sigma_z: float              # rms lab length, normalised
    weight: float               # real electrons per macroparticle, normalised (N / (n_n L_n^3))
    origin: Tuple[float, float, float]  # grid coordinate (cells) of the beam reference point
    q: float = -1.0
    m: float = 1.0


@dataclasses.dataclass
class Undulator:
    K: float
    lambda_u: float             # lab period, normalised
    phase: float = 0.0
    z_start: float = -math.inf  # lab z of the entrance (normalised); -inf: field everywhere
    ramp: float = -1.0          # lab length of the linear entrance ramp; < 0: none
    match: bool = True          # load the beam with matched transverse canonical momentum
    kind: int = 1               # 1: ideal on-axis planar field; 2: with its cosh/sinh y-dependence


@dataclasses.dataclass
class Plasma:
    ppc: Tuple[int, int, int]
    xrange: Tuple[int, int, int, int]   # transverse cell range x0, x1, y0, y1
    z_nodes: Tuple[float, ...]          # lab z of the profile nodes (normalised)
    n_nodes: Tuple[float, ...]          # lab density at the nodes (units of n_n)


@dataclasses.dataclass
class Workload:
    name: str
    grid: Tuple[int, int, int]
    d: Tuple[float, float, float]
    dt: float
    gamma_R: float
    bc: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]]
    pml: int
    order: int
    moving_window: bool
    window_v: float
    beam: Optional[Beam]
    undulator: Optional[Undulator]
    plasma: Optional[Plasma]
    steps: int
    length_unit_m: float
    seed: int
    tile: Tuple[int, int, int] = (8, 8, 8)
    sort_every: int = 8

    @property
    def ncell(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    def plasma_count_estimate(self) -> int:
        if self.plasma is None:
            return 0
        p = self.plasma
        x0, x1, y0, y1 = p.xrange
        lo = 1 if self.order == 1 else 2
        hi = 2 if self.order == 1 else 3
        nz = self.grid[2] if self.bc[2][0] == PERIODIC else self.grid[2] - lo - hi
        return (x1 - x0) * (y1 - y0) * nz * p.ppc[0] * p.ppc[1] * p.ppc[2]


def courant_dt(d, cfl=0.5):
    return cfl / math.sqrt(sum(1.0 / (v * v) for v in d))


def beam_weight(charge_C: float, n_macro: int, omega_n: float) -> float:
    L = C_LIGHT / omega_n
    return (charge_C / Q_E) / (density_unit(omega_n) * L ** 3) / n_macro


# ----------------------------------------------------------------------------- workloads

def vacuum_undulator(grid=(32, 32, 64), n_beam=65536, steps=200, seed=1, order=1,
                     name="vacuum undulator 32x32x64, 65,536 beam, CIC") -> Workload:
    """Plain method: periodic 3D grid, boost 10, lab gamma 100 beam, planar undulator
    K = 1 (lambda_u = 2 cm, two RRF periods across 64 cells), first-order shape."""
    gR = 10.0
    lam_u_m = 0.02
    omega_n = 2 * math.pi * gR * C_LIGHT / lam_u_m
    L = C_LIGHT / omega_n
    dx = 2 * math.pi / 32            # lambda'_u = 2 pi in these units -> 32 cells per period
    d = (dx, dx, dx)
    dt = courant_dt(d, 0.5)
    sigma_r = 4 * dx
    # lab rms length that maps to ~8 RRF cells (elongation factor 19.754 at gamma 100 / 10)
    sigma_z = 2.531156754515905e-05 / L
    beam = Beam(n=n_beam, gamma=100.0, rel_spread=1e-3, emit_n=1e-6 / L, sigma_r=sigma_r,
                sigma_z=sigma_z, weight=beam_weight(30e-12, n_beam, omega_n),
                origin=(grid[0] / 2, grid[1] / 2, grid[2] / 2))
    und = Undulator(K=1.0, lambda_u=lam_u_m / L, match=True)
    return Workload(name=name, grid=grid, d=d, dt=dt, gamma_R=gR,
                    bc=((PERIODIC, PERIODIC),) * 3, pml=0, order=order, moving_window=False,
                    window_v=0.0, beam=beam, undulator=und, plasma=None, steps=steps,
                    length_unit_m=L, seed=seed)


def plasma_buncher(grid=(128, 128, 512), n_beam=4194304, steps=5000, seed=2, pml=10,
                   ppc=(2, 2, 2), dx_m=2.5e-6, dz_m=75e-6,
                   name="plasma buncher 128x128x512, 4M beam + 8 ppc plasma, TSC") -> Workload:
    """Plasma buncher: boost 20, lab gamma 400 beam (sigma_r 10 um, sigma_z 30 um lab),
    cold lab-static plasma of 1e15 cm^-3 with immobile (frozen) neutralising ions, 8
    particles per cell, transverse PML, longitudinal moving window, second-order shape."""
    gR = 20.0
    n_lab = 1e21
    omega_n = omega_plasma(gR * n_lab)
    L = C_LIGHT / omega_n
    d = (dx_m / L, dx_m / L, dz_m / L)
    dt = courant_dt(d, 0.5)
    lo, hi = 2, 3
    nz = grid[2]
    beam = Beam(n=n_beam, gamma=400.0, rel_spread=1e-3, emit_n=1e-6 / L, sigma_r=10e-6 / L,
                sigma_z=30e-6 / L, weight=beam_weight(30e-12, n_beam, omega_n),
                origin=(grid[0] / 2, grid[1] / 2, 0.75 * nz))
    plasma = Plasma(ppc=ppc, xrange=(lo, grid[0] - hi, lo, grid[1] - hi),
                    z_nodes=(-1e12, 1e12), n_nodes=(n_lab / density_unit(omega_n),) * 2)
    # window speed = mean RRF beam velocity (0.995019 for gamma 400 in a gamma 20 frame)
    return Workload(name=name, grid=grid, d=d, dt=dt, gamma_R=gR,
                    bc=((PML, PML), (PML, PML), (OPEN, OPEN)), pml=pml, order=2,
                    moving_window=True, window_v=0.995018674132024, beam=beam, undulator=None,
                    plasma=plasma, steps=steps, length_unit_m=L, seed=seed)


def long_undulator(grid=(256, 256, 1024), n_beam=33554432, steps=20000, seed=3, pml=10,
                   name="long undulator 256x256x1024, 32M beam, TSC", z_start=None) -> Workload:
    """Long undulator: lab gamma 2000, K = 1.5, lambda_u = 2 cm, boost gamma/sqrt(1+K^2/2)
    (beam at rest on average once inside), PML on all faces, static window, second-order shape,
    64 cells per RRF undulator period.  The beam starts in front of the undulator and enters it
    through a linear ramp of one lab period (the gentle slope that avoids a transverse kick):
    by default the entrance sits four RRF bunch lengths ahead of the bunch centre at t' = 0
    (lab z = gamma_R z' there), so it sweeps over the bunch from head to tail.  z_start = 0 puts
    the grid's origin at the entrance instead: the bunch then starts inside the field."""
    K = 1.5
    gB = 2000.0
    gR = gB / math.sqrt(1 + K * K / 2)
    lam_u_m = 0.02
    omega_n = 2 * math.pi * gR * C_LIGHT / lam_u_m
    L = C_LIGHT / omega_n
    dz = 2 * math.pi / 64
    dxy = 4 * dz
    d = (dxy, dxy, dz)
    dt = courant_dt(d, 0.5)
    beam = Beam(n=n_beam, gamma=gB, rel_spread=5e-4, emit_n=0.5e-6 / L, sigma_r=6 * dxy,
                sigma_z=grid[2] * dz / 12 / 1866.0, weight=beam_weight(30e-12, n_beam, omega_n),
                origin=(grid[0] / 2, grid[1] / 2, grid[2] / 2))
    if z_start is None:
        z_start = gR * grid[2] * dz * (0.5 + 4.0 / 12.0)
    und = Undulator(K=K, lambda_u=lam_u_m / L, match=False, z_start=z_start, ramp=lam_u_m / L)
    return Workload(name=name, grid=grid, d=d, dt=dt, gamma_R=gR,
                    bc=((PML, PML),) * 3, pml=pml, order=2, moving_window=False,
                    window_v=0.0, beam=beam, undulator=und, plasma=None, steps=steps,
                    length_unit_m=L, seed=seed)


# Workloads the oracle finishes in seconds, spanning several 8^3 tiles with ragged tails.
def mini_vacuum(order=1, seed=11):
    return vacuum_undulator(grid=(20, 18, 44), n_beam=6000, steps=20, seed=seed, order=order,
                            name=f"mini vacuum undulator 20x18x44 order {order}")


def mini_dense_bunch(order=2, seed=17, n_beam=150000):
    """The vacuum undulator's physics on an oracle-sized grid with a dense bunch: sigma_r 1.2
    cells, ~3 RRF cells long, ~2000 particles per cell at the peak, its core filling one 8^3 tile
    with a few hundred particles per cell on average (the dense-bunch path of the particle
    kernel)."""
    w = vacuum_undulator(grid=(24, 20, 48), n_beam=n_beam, steps=20, seed=seed, order=order,
                         name=f"mini dense bunch 24x20x48 order {order}")
    w.beam.sigma_r = 1.2 * w.d[0]
    w.beam.sigma_z *= 3.0 / 8.0
    w.beam.origin = (12.0, 12.0, 20.0)
    return w


def mini_plasma(seed=12, grid=(28, 26, 52), n_beam=4000, steps=20):
    """Plasma-buncher physics on a small grid: 5 um longitudinal cells (the window shifts
    every ~6 steps), 1x2x2 particles per cell, a short beam (1 um lab, ~8 cells in the RRF)."""
    w = plasma_buncher(grid=grid, n_beam=n_beam, steps=steps, seed=seed, pml=4, ppc=(1, 2, 2),
                       dz_m=5e-6, name=f"mini plasma buncher {grid[0]}x{grid[1]}x{grid[2]}")
    w.beam.sigma_z = 1e-6 / w.length_unit_m
    w.beam.origin = (grid[0] / 2, grid[1] / 2, 0.6 * grid[2])
    return w


def plasma_buncher_2d(grid=(1024, 1, 2048), n_beam=1048576, steps=5000, seed=6, pml=10, ppc=(2, 1, 2),
                      name="plasma buncher 2-D 1024x2048 (x-z), 1M beam + 4 ppc plasma, TSC") -> Workload:
    """The plasma buncher in the paper's 2-D geometry (x-z plane, uniform along y: ny = 1 with a
    periodic y), 4 particles per cell as in the paper's 2-D plasma runs (Table I), transverse
    PML in x, moving window along z."""
    w = plasma_buncher(grid=grid, n_beam=n_beam, steps=steps, seed=seed, pml=pml, ppc=ppc, name=name)
    w.bc = ((PML, PML), (PERIODIC, PERIODIC), (OPEN, OPEN))
    lo, hi = 2, 3
    w.plasma = dataclasses.replace(w.plasma, xrange=(lo, grid[0] - hi, 0, 1))
    w.beam.origin = (grid[0] / 2, 0.5, 0.75 * grid[2])
    w.tile = (8, 1, 8)
    return w


def mini_plasma_2d(seed=16, grid=(28, 1, 52), n_beam=3000, steps=20):
    """The oracle-sized 2-D plasma buncher (x-z, ny = 1): 5 um longitudinal cells (the window
    shifts every ~6 steps), 2x1x2 particles per cell, a short beam."""
    w = mini_plasma(seed=seed, grid=grid, n_beam=n_beam, steps=steps)
    w.name = f"mini plasma buncher 2-D {grid[0]}x{grid[2]}"
    w.bc = ((PML, PML), (PERIODIC, PERIODIC), (OPEN, OPEN))
    w.plasma = dataclasses.replace(w.plasma, ppc=(2, 1, 2), xrange=(2, grid[0] - 3, 0, 1))
    w.beam.origin = (grid[0] / 2, 0.5, 0.6 * grid[2])
    w.tile = (8, 1, 8)
    return w


def mini_long_undulator(seed=13):
    # the grid lies inside the entrance ramp at t' = 0 (the entrance at its origin)
    w = long_undulator(grid=(24, 20, 48), n_beam=4000, steps=20, seed=seed, pml=4,
                       name="mini long undulator 24x20x48", z_start=0.0)
    return w


@dataclasses.dataclass
class Ensemble:
    """Independent runs sharing grid, cell size, time step, boost, boundaries and shape (the
    base workload); run r has undulator K[r], plasma density scale dens_scale[r] (times the
    base plasma profile) and n_beam[r] beam macroparticles of the base beam's shape and charge,
    sampled with seed base.seed * 1000 + r."""
    base: Workload
    K: Tuple[float, ...]
    dens_scale: Tuple[float, ...]
    n_beam: Tuple[int, ...]

    @property
    def runs(self) -> int:
        return len(self.K)


def batched_ensemble(runs=64, grid=(64, 64, 128), steps=1000, seed=4, order=2, ppc=(1, 2, 2),
                     K_range=(0.5, 2.0), n_lab_cm3=(1e14, 1e16), n_beam_range=(1e5, 1e6),
                     name="batched ensemble 64 x (64x64x128), K and density sweep, TSC") -> Ensemble:
    """Batched sweep: periodic runs on a cubic grid of 64 cells per RRF undulator period
    (boost 10, lab gamma 100 beam of 30 pC, lambda_u = 2 cm; the undulator normalisation
    w_n = 2 pi gamma_R c / lambda_u is shared by every run), undulator K uniform in
    K_range, lab plasma density log-uniform in n_lab_cm3 (cold, lab-static, 4 per cell, frozen
    ions), beam macroparticles log-uniform in n_beam_range (uneven), second-order shape."""
    gR = 10.0
    lam_u_m = 0.02
    omega_n = 2 * math.pi * gR * C_LIGHT / lam_u_m
    L = C_LIGHT / omega_n
    dx = 2 * math.pi / 64
    d = (dx, dx, dx)
    dt = courant_dt(d, 0.5)
    # lab rms length mapping to 12 RRF cells (elongation 19.754 at gamma 100 in a boost of 10)
    sigma_z = 12 * dx / 19.754
    beam = Beam(n=0, gamma=100.0, rel_spread=1e-3, emit_n=1e-6 / L, sigma_r=6 * dx, sigma_z=sigma_z,
                weight=0.0, origin=(grid[0] / 2, grid[1] / 2, grid[2] / 2))
    und = Undulator(K=1.0, lambda_u=lam_u_m / L, match=True)
    nz = grid[2]
    plasma = Plasma(ppc=ppc, xrange=(0, grid[0], 0, grid[1]), z_nodes=(-1e12, 1e12), n_nodes=(1.0, 1.0))
    base = Workload(name=name, grid=grid, d=d, dt=dt, gamma_R=gR, bc=((PERIODIC, PERIODIC),) * 3, pml=0,
                    order=order, moving_window=False, window_v=0.0, beam=beam, undulator=und,
                    plasma=plasma, steps=steps, length_unit_m=L, seed=seed)
    rng = np.random.Generator(np.random.Philox(key=seed))
    K = tuple(float(v) for v in rng.uniform(K_range[0], K_range[1], runs))
    n_unit_cm3 = density_unit(omega_n) * 1e-6
    dens = tuple(float(10 ** v / n_unit_cm3) for v in rng.uniform(math.log10(n_lab_cm3[0]), math.log10(n_lab_cm3[1]), runs))
    nb = tuple(int(round(10 ** v)) for v in rng.uniform(math.log10(n_beam_range[0]), math.log10(n_beam_range[1]), runs))
    return Ensemble(base=base, K=K, dens_scale=dens, n_beam=nb)


def mini_ensemble(runs=3, seed=14):
    """Three runs of 16 x 16 x 32 cells (two 8^3 tiles in z each), uneven beams, for parity."""
    e = batched_ensemble(runs=runs, grid=(16, 16, 32), steps=20, seed=seed, n_lab_cm3=(3e13, 3e15),
                         n_beam_range=(300, 3000), name=f"mini ensemble {runs} x (16x16x32)")
    e.base.beam.sigma_r = 2 * e.base.d[0]
    e.base.beam.sigma_z = 4 * e.base.d[2] / 19.754
    return e


def ensemble_run(e: Ensemble, r: int) -> Workload:
    """Run r of an ensemble as a single-run workload (its K, scaled plasma and beam size)."""
    b = e.base
    w = dataclasses.replace(b, name=f"{b.name} run {r}", seed=b.seed * 1000 + r)
    w.undulator = dataclasses.replace(b.undulator, K=e.K[r])
    w.plasma = dataclasses.replace(b.plasma, n_nodes=tuple(v * e.dens_scale[r] for v in b.plasma.n_nodes))
    w.beam = dataclasses.replace(b.beam, n=e.n_beam[r], weight=beam_weight(30e-12, e.n_beam[r], C_LIGHT / b.length_unit_m))
    return w


def adjoint_workload(grid=(64, 64, 256), n_beam=2097152, steps=1000, seed=5, n_nodes=32, ppc=(1, 2, 2),
                     name="differentiated run 64x64x256, 2M beam + 4 ppc plasma, CIC") -> Workload:
    """Differentiated run: the vacuum-undulator physics (boost 10, lab gamma 100 beam of 30 pC,
    K = 1, lambda_u = 2 cm, 32 cells per RRF undulator period, first-order shape, periodic) with
    a cold lab-static plasma of 4 particles per cell whose lab density is a piecewise-linear
    profile of n_nodes nodes spread over the box's lab image (seeded values around n_n)."""
    w = vacuum_undulator(grid=grid, n_beam=n_beam, steps=steps, seed=seed, order=1, name=name)
    zl = w.gamma_R * grid[2] * w.d[2]
    rng = np.random.Generator(np.random.Philox(key=seed))
    zn = tuple(float(v) for v in np.linspace(0.0, zl, n_nodes))
    dn = tuple(float(v) for v in 1.0 * (1.0 + 0.3 * rng.uniform(-1.0, 1.0, n_nodes)))
    w.plasma = Plasma(ppc=ppc, xrange=(0, grid[0], 0, grid[1]), z_nodes=zn, n_nodes=dn)
    w.beam.weight = beam_weight(30e-12, n_beam, C_LIGHT / w.length_unit_m)
    return w


def mini_adjoint(seed=15, steps=30):
    """The oracle-sized reduction of the differentiated run: 16 x 16 x 32, 2000 beam electrons."""
    w = adjoint_workload(grid=(16, 16, 32), n_beam=2000, steps=steps, seed=seed,
                         name="mini adjoint 16x16x32")
    w.beam.sigma_r = 2 * w.d[0]
    w.beam.sigma_z = 4 * w.d[2] / 19.754
    return w


# ----------------------------------------------------------------------------- generators

def sample_beam(w: Workload, n: Optional[int] = None, seed: Optional[int] = None):
    """Seeded lab-frame Gaussian beam at lab time 0.

    Returns x (3, n) and u (3, n) in normalised lab units relative to the beam reference
    point (which the loaders place at grid coordinate ``w.beam.origin`` at t' = 0), and
    the weights w (n,).  Positions: Gaussian (sigma_r, sigma_r, sigma_z); gamma: Gaussian
    around the mean with the relative spread; transverse momenta: Gaussian with
    sigma_u = emit_n / sigma_r (uncorrelated, waist at t = 0; the small divergence the
    paper adds to every beam); u_z from gamma.
    """
    b = w.beam
    n = b.n if n is None else int(n)
    rng = np.random.Generator(np.random.Philox(key=(w.seed if seed is None else seed)))
    x = np.empty((3, n))
    x[0] = rng.normal(0.0, b.sigma_r, n)
    x[1] = rng.normal(0.0, b.sigma_r, n)
    x[2] = rng.normal(0.0, b.sigma_z, n)
    u = np.empty((3, n))
    su = b.emit_n / b.sigma_r
    u[0] = rng.normal(0.0, su, n)
    u[1] = rng.normal(0.0, su, n)
    gam = b.gamma * (1.0 + b.rel_spread * rng.normal(0.0, 1.0, n))
    u[2] = np.sqrt(gam * gam - 1.0 - u[0] ** 2 - u[1] ** 2)
    wts = np.full(n, b.weight)
    return x, u, wts


def sample_uniform_particles(grid, n, seed, umax=0.5):
    """Seeded particles uniformly spread over a grid (grid coordinates, cells) with
    momenta uniform in [-umax, umax]^3: generic states for unit-level parity cases."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    X = np.empty((n, 3))
    for dd in range(3):
        X[:, dd] = rng.uniform(0.0, grid[dd], n)
    U = rng.uniform(-umax, umax, (n, 3))
    W = rng.uniform(0.5, 1.5, n)
    return X, U, W


def sample_fields(grid, seed, amp=1e-2):
    """Seeded smooth-ish random E and B (nine components with J) for field-only cases."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    nx, ny, nz = grid
    return [amp * rng.standard_normal((nz, ny, nx)) for _ in range(6)]
