"""Seeded synthetic inputs for the cutoff non-bonded force path.

This module draws the inputs and nothing else: positions, LJ types, charges,
masses and velocities, plus the per-type-pair constants A and B that Eq. 1
(Section II.A) takes as given.  It holds none of the method's arithmetic (no
pair force, no cell list, no cutoff filter, no integrator), so the CUDA path
and the FP64 oracle can both read their inputs from it without sharing code.

Units (the paper states none): Angstrom, femtosecond, amu, elementary charge,
kcal/mol.  Lennard-Jones constants follow the usual 12-6 convention
A = 48*eps*sigma^12 and B = 24*eps*sigma^6, for which Eq. 1 is minus the
gradient of 4*eps*((sigma/r)^12 - (sigma/r)^6); per-pair sigma and eps use
Lorentz-Berthelot mixing.  A and B are formed in float64 and rounded once to
float32; both sides of every comparison get the rounded values.

Workloads (seeded, synthetic; the paper's ApoA1 input files are not available,
Section III names the benchmark and its ~100k atoms / ~700 cells):
  * ``random_gas``  - uniform random atoms in a periodic cube with a minimum
    pair distance enforced by rejection (3,000 atoms in a 31 A cube, 4 types).
  * ``lattice_box`` - jittered cubic lattice at ~0.1 atoms/A^3 in ApoA1's box
    shape (92,224 atoms in 108.86 x 108.86 x 77.76 A, 8 types), and the same
    density at other sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Coulomb constant in kcal*A/(mol*e^2), the value CHARMM and NAMD use.  The
# paper only says k is a constant (Eq. 2).
K_COULOMB = 332.0636
# Boltzmann constant in kcal/(mol*K).
K_BOLTZMANN = 0.0019872043
# (kcal/mol/A) / amu expressed in A/fs^2.
ACCEL_PER_FORCE_PER_MASS = 4.184e-4


@dataclass
class System:
    """One periodic system, as float32 device-ready arrays plus float64 box."""

    name: str
    pos: np.ndarray  # float32 [N, 3], every coordinate in [0, L_d)
    q: np.ndarray  # float32 [N], elementary charges
    type: np.ndarray  # int32 [N], LJ type in [0, ntypes)
    box: np.ndarray  # float64 [3], box edge lengths L_d
    rc: float  # cutoff radius (exactly representable in float32)
    sigma: np.ndarray  # float64 [T]
    eps: np.ndarray  # float64 [T]
    AB: np.ndarray  # float32 [T, T, 2]: (A_ij, B_ij) of Eq. 1
    mass: np.ndarray  # float32 [N], amu
    vel: np.ndarray  # float64 [N, 3], A/fs
    k_coulomb: float = K_COULOMB
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ntypes(self) -> int:
        return int(self.sigma.shape[0])

    @property
    def inv_mass(self) -> np.ndarray:
        return (1.0 / self.mass.astype(np.float64)).astype(np.float32)

    def pos_q(self) -> np.ndarray:
        """float32 [N, 4] rows (x, y, z, q): the layout the device path reads."""
        out = np.empty((self.n, 4), dtype=np.float32)
        out[:, :3] = self.pos
        out[:, 3] = self.q
        return out

    def with_forcefield(self, sigma_scale: float = 1.0, mass_range=None, seed: int = 0) -> "System":
        """Copy with sigma scaled and (optionally) masses redrawn; positions, charges
        and types unchanged.  Used for the mechanically gentle variant."""
        sigma = self.sigma * sigma_scale
        AB = lj_table(sigma, self.eps)
        mass = self.mass
        vel = self.vel
        if mass_range is not None:
            rng = np.random.default_rng(seed)
            mass = rng.uniform(mass_range[0], mass_range[1], size=self.n).astype(np.float32)
            vel = maxwell_velocities(rng, mass, 300.0)
        meta = dict(self.meta, sigma_scale=sigma_scale, mass_range=mass_range)
        return System(self.name + "-gentle", self.pos, self.q, self.type, self.box, self.rc,
                      sigma, self.eps, AB, mass, vel, self.k_coulomb, meta)


def lj_table(sigma: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """(A_ij, B_ij) for every type pair, Lorentz-Berthelot mixed, rounded once to float32."""
    s = 0.5 * (sigma[:, None] + sigma[None, :])
    e = np.sqrt(eps[:, None] * eps[None, :])
    AB = np.empty(s.shape + (2,), dtype=np.float64)
    AB[..., 0] = 48.0 * e * s**12
    AB[..., 1] = 24.0 * e * s**6
    return AB.astype(np.float32)


def maxwell_velocities(rng: np.random.Generator, mass: np.ndarray, temp_k: float) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/fs) with the centre-of-mass velocity removed."""
    m = mass.astype(np.float64)
    sd = np.sqrt(K_BOLTZMANN * temp_k / m * ACCEL_PER_FORCE_PER_MASS)
    v = rng.standard_normal((m.shape[0], 3)) * sd[:, None]
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return v


def to_f32_in_box(pos64: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Round positions to float32, keeping every coordinate inside [0, L_d)."""
    p = np.mod(pos64, box[None, :])
    p32 = p.astype(np.float32)
    for d in range(3):
        top = np.float32(box[d])
        while float(top) >= box[d]:
            top = np.nextafter(top, np.float32(0))
        col = p32[:, d]
        col[col.astype(np.float64) >= box[d]] = top
        col[col < 0] = np.float32(0)
    return p32


def _charges_pm(rng: np.random.Generator, n: int, levels) -> np.ndarray:
    """Charges from a discrete set with exactly zero net charge: draw n//2 values,
    append their negatives (plus one zero when n is odd), shuffle."""
    half = rng.choice(np.asarray(levels, dtype=np.float64), size=n // 2)
    q = np.concatenate([half, -half, np.zeros(n - 2 * (n // 2))])
    rng.shuffle(q)
    return q.astype(np.float32)


def _reject_close_pairs(rng, pos: np.ndarray, box: np.ndarray, min_dist: float, max_iter: int = 1000):
    """Redraw one atom of every pair closer than ``min_dist`` until none is left.
    Uses scipy's periodic k-d tree for the neighbour query."""
    from scipy.spatial import cKDTree

    for _ in range(max_iter):
        tree = cKDTree(pos, boxsize=box)
        pairs = tree.query_pairs(min_dist, output_type="ndarray")
        if pairs.shape[0] == 0:
            return pos
        redo = np.unique(pairs[:, 1])
        pos[redo] = rng.uniform(0.0, 1.0, size=(redo.shape[0], 3)) * box[None, :]
    raise RuntimeError("rejection sampling did not converge")


def random_gas(n: int = 3000, box=(31.0, 31.0, 31.0), ntypes: int = 4, rc: float = 12.0,
               min_dist: float = 1.0, seed: int = 1, sigma_range=(2.5, 3.8),
               eps_range=(0.05, 0.2), mass_range=(1.0, 16.0),
               charge_levels=(-0.8, -0.4, 0.4, 0.8), temp_k: float = 300.0,
               name: str = "random_gas") -> System:
    """Uniform random atoms, minimum distance by rejection, discrete zero-net charges."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * box[None, :]
    if min_dist > 0:
        pos = _reject_close_pairs(rng, pos, box, min_dist)
    sigma = rng.uniform(*sigma_range, size=ntypes)
    eps = rng.uniform(*eps_range, size=ntypes)
    types = rng.integers(0, ntypes, size=n).astype(np.int32)
    q = _charges_pm(rng, n, charge_levels)
    mass = rng.uniform(*mass_range, size=n).astype(np.float32)
    vel = maxwell_velocities(rng, mass, temp_k)
    return System(name, to_f32_in_box(pos, box), q, types, box, float(np.float32(rc)), sigma, eps,
                  lj_table(sigma, eps), mass, vel,
                  meta=dict(seed=seed, min_dist=min_dist, generator="random_gas"))


APOA1_BOX = (108.86, 108.86, 77.76)
APOA1_SITES = (51, 51, 36)
APOA1_N = 92224


def lattice_box(n: int = APOA1_N, seed: int = 2, ntypes: int = 8, rc: float = 12.0,
                jitter: float = 0.3, sigma_range=(2.5, 3.8), eps_range=(0.05, 0.2),
                mass_range=(1.0, 16.0), charge_sd: float = 0.4, temp_k: float = 300.0,
                name: str | None = None) -> System:
    """Jittered cubic lattice at ApoA1's density (~0.1 atoms/A^3) and box aspect.

    At n = 92,224 the box is 108.86 x 108.86 x 77.76 A with 51 x 51 x 36 sites of
    which 1,412 random ones are left empty.  Other n scale every edge by
    (n / 92,224)^(1/3) and regenerate the lattice at the same spacing."""
    rng = np.random.default_rng(seed)
    s = (n / APOA1_N) ** (1.0 / 3.0)
    box = np.asarray(APOA1_BOX, dtype=np.float64) * (1.0 if n == APOA1_N else s)
    if n == APOA1_N:
        sites = np.asarray(APOA1_SITES)
    else:
        sites = np.ceil(np.asarray(APOA1_SITES, dtype=np.float64) * s).astype(int)
        while int(np.prod(sites)) < n:
            sites += 1
    spacing = box / sites
    gx, gy, gz = np.meshgrid(np.arange(sites[0]), np.arange(sites[1]), np.arange(sites[2]),
                             indexing="ij")
    grid = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    keep = np.sort(rng.permutation(grid.shape[0])[:n])
    pos = (grid[keep] + 0.5) * spacing[None, :]
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    sigma = rng.uniform(*sigma_range, size=ntypes)
    eps = rng.uniform(*eps_range, size=ntypes)
    types = rng.integers(0, ntypes, size=n).astype(np.int32)
    q = rng.normal(0.0, charge_sd, size=n)
    q -= q.mean()
    mass = rng.uniform(*mass_range, size=n).astype(np.float32)
    vel = maxwell_velocities(rng, mass, temp_k)
    return System(name or f"lattice_{n}", to_f32_in_box(pos, box), q.astype(np.float32), types,
                  box, float(np.float32(rc)), sigma, eps, lj_table(sigma, eps), mass, vel,
                  meta=dict(seed=seed, sites=sites.tolist(), jitter=jitter, generator="lattice_box"))


def small_random(n: int, box, ntypes: int = 3, rc: float = 3.0, seed: int = 0,
                 min_dist: float = 0.0, sigma_range=(0.8, 1.2), eps_range=(0.5, 1.5),
                 charge_levels=(-1.0, -0.5, 0.5, 1.0), mass_range=(1.0, 16.0),
                 name: str = "small") -> System:
    """Small random systems for pins and edge cases (any box shape)."""
    return random_gas(n=n, box=box, ntypes=ntypes, rc=rc, min_dist=min_dist, seed=seed,
                      sigma_range=sigma_range, eps_range=eps_range, mass_range=mass_range,
                      charge_levels=charge_levels, name=name)


# The named workloads.  The first is small enough for whole-system parity with
# the oracle in seconds; the second is the single-GPU throughput workload.
def workload_random_3000(seed: int = 1) -> System:
    """3,000 atoms, 31 A periodic cube, 4 LJ types, min pair distance 1 A, rc 12 A."""
    return random_gas(seed=seed, name="random_gas_3000")


def workload_lattice_92k(seed: int = 2) -> System:
    """92,224 atoms in ApoA1's 108.86 x 108.86 x 77.76 A box, 8 LJ types, rc 12 A."""
    return lattice_box(seed=seed, name="lattice_92224")


def sweep_sizes():
    """Atom counts of the size sweep at ApoA1 density: 92,224 x {1/4, 1, 4, 16}."""
    return [APOA1_N // 4, APOA1_N, APOA1_N * 4, APOA1_N * 16]



def batch_of_systems(nsys: int = 256, seed: int = 4, n_range=(500, 20000), rho_range=(0.08, 0.11),
                     type_range=(4, 8), rc_range=(9.0, 12.0), sigma_range=(1.9, 2.3),
                     eps_range=(0.05, 0.2), mass_range=(12.0, 16.0), charge_sd: float = 0.2,
                     jitter: float = 0.3):
    """Independent periodic systems of uneven size for the batched path.

    Atom counts are log-uniform in n_range, densities uniform in rho_range, boxes cubic
    with L = (N / rho)^(1/3), 4-8 LJ types, cutoffs uniform in rc_range.  A cutoff at or
    above L/2 (the minimum image would be ambiguous) is lowered to 0.999 L/2; such
    systems are listed in meta['rc_clamped'].  Atoms sit on a jittered cubic lattice
    (no overlaps); LJ diameters of 1.9-2.3 A against charges ~N(0, 0.2) e keep opposite
    charges from collapsing through each other during the run, so the int64 fixed-point
    pair terms stay in range."""
    rng = np.random.default_rng(seed)
    systems = []
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    for k in range(nsys):
        n = int(round(np.exp(rng.uniform(lo, hi))))
        rho = rng.uniform(*rho_range)
        L = (n / rho) ** (1.0 / 3.0)
        box = np.array([L, L, L])
        m = int(np.ceil(n ** (1.0 / 3.0)))
        g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
        g = g.reshape(-1, 3).astype(np.float64)
        keep = np.sort(rng.permutation(g.shape[0])[:n])
        spacing = L / m
        pos = (g[keep] + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(n, 3))
        ntypes = int(rng.integers(type_range[0], type_range[1] + 1))
        rc_drawn = rng.uniform(*rc_range)
        rc = float(np.float32(min(rc_drawn, 0.999 * L / 2)))
        sigma = rng.uniform(*sigma_range, size=ntypes)
        eps = rng.uniform(*eps_range, size=ntypes)
        types = rng.integers(0, ntypes, size=n).astype(np.int32)
        q = rng.normal(0.0, charge_sd, size=n)
        q -= q.mean()
        mass = rng.uniform(*mass_range, size=n).astype(np.float32)
        vel = maxwell_velocities(rng, mass, 300.0)
        systems.append(System(f"batch_{k}", to_f32_in_box(pos, box), q.astype(np.float32), types,
                              box, rc, sigma, eps, lj_table(sigma, eps), mass, vel,
                              meta=dict(seed=seed, index=k, rho=rho, rc_drawn=rc_drawn,
                                        rc_clamped=rc < rc_drawn - 1e-6)))
    return systems


def serving_jobs(n_jobs: int = 2000, rate_per_s: float = 200.0, seed: int = 5,
                 n_range=(1000, 150000), steps_range=(10, 500), rho: float = 0.1,
                 rc: float = 12.0):
    """MD jobs arriving as a Poisson stream: (system, n_steps, arrival time in s).

    Atom counts log-uniform in n_range, steps uniform integers in steps_range, density
    0.1 atoms/A^3 in cubic boxes, cutoff 12 A (lowered to 0.999 L/2 in small boxes),
    force field as in batch_of_systems.  Systems are drawn lazily (a callable per job),
    so a long stream does not hold every system in host memory at once."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_jobs))
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    ns = np.round(np.exp(rng.uniform(lo, hi, size=n_jobs))).astype(int)
    steps = rng.integers(steps_range[0], steps_range[1] + 1, size=n_jobs)
    seeds = rng.integers(0, 2**31 - 1, size=n_jobs)
    jobs = []
    for k in range(n_jobs):
        n, sd = int(ns[k]), int(seeds[k])

        def make(n=n, sd=sd):
            s = batch_of_systems(nsys=1, seed=sd, n_range=(n, n), rho_range=(rho, rho),
                                 rc_range=(rc, rc))[0]
            s.name = f"job_{sd}"
            return s
        jobs.append((make, int(steps[k]), float(t[k]), n))
    return jobs
