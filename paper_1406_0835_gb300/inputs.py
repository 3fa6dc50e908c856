"""Seeded synthetic inputs (hydrogen cells, ion positions, velocities, grids).

This module holds no arithmetic of the OF-DFT method: it only draws the
workloads (Sec. VI of arXiv:1406.0835 runs hydrogen at 0.983 g/cm^3,
32-2744 atoms, up to 4 MK) that both the CUDA library and the test oracle
are fed.  Random numbers come from numpy's PCG64 with explicit seeds.
"""
import math

import numpy as np

BOHR_CM = 0.529177210903e-8        # bohr in cm (CODATA 2018)
AMU_G = 1.66053906660e-24          # atomic mass unit in g (CODATA 2018)
AMU_ME = 1822.888486209            # atomic mass unit in electron masses
M_H_AMU = 1.00794                  # hydrogen atomic mass
KB_HA_PER_K = 3.166811563e-6       # Boltzmann constant, hartree per kelvin


def cell_edge(n_atoms, rho_gcc, mass_amu=M_H_AMU):
    """Edge (bohr) of a cubic cell holding n_atoms at mass density rho (g/cm^3)."""
    vol_cm3 = n_atoms * mass_amu * AMU_G / rho_gcc
    return vol_cm3 ** (1.0 / 3.0) / BOHR_CM


def smooth235(n):
    """True if n has no prime factor other than 2, 3, 5."""
    for p in (2, 3, 5):
        while n % p == 0 and n > 1:
            n //= p
    return n == 1


def grid_edge(L, spacing=0.25, lo=32, hi=160):
    """Smallest even {2,3,5}-smooth edge >= L/spacing, clamped to [lo, hi]."""
    m = max(lo, int(math.ceil(L / spacing - 1e-9)))
    while not (m % 2 == 0 and smooth235(m)):
        m += 1
    return min(m, hi)


def random_positions(n_atoms, L, seed, min_dist=0.8, max_tries=1000000):
    """Uniform positions in [0,L)^3 with minimum periodic-image distance,
    by rejection in a fixed order (each accepted atom is final)."""
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    pos = np.zeros((n_atoms, 3))
    k = 0
    tries = 0
    while k < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d atoms" % n_atoms)
        p = rng.random(3) * L
        if k:
            d = pos[:k] - p
            d -= L * np.round(d / L)
            if np.min(np.sum(d * d, axis=1)) < min_dist * min_dist:
                continue
        pos[k] = p
        k += 1
    return pos


def maxwell_boltzmann(n_atoms, T_kelvin, seed, mass_amu=M_H_AMU):
    """Velocities (bohr per atomic time unit) from a Maxwell-Boltzmann
    distribution, centre-of-mass velocity removed."""
    rng = np.random.default_rng(seed)
    m = mass_amu * AMU_ME
    sig = math.sqrt(KB_HA_PER_K * T_kelvin / m)
    v = rng.standard_normal((n_atoms, 3)) * sig
    v -= v.mean(axis=0)
    return v


def andersen_draws(n_atoms, seed):
    """Random numbers of one round of Andersen collisions: u[n] uniform in
    [0, 1) and xi[n, 3] standard normal (PCG64, seeded)."""
    rng = np.random.default_rng(seed)
    return rng.random(n_atoms), rng.standard_normal((n_atoms, 3))


def hydrogen(n_atoms, rho_gcc, T_kelvin, grid, seed, functional,
             min_dist=0.8, vel_seed=None):
    """One synthetic hydrogen workload as a plain dict."""
    L = cell_edge(n_atoms, rho_gcc)
    g = (grid, grid, grid) if np.isscalar(grid) else tuple(grid)
    spacing = L / n_atoms ** (1.0 / 3.0)
    if min_dist > 0.6 * spacing:          # very dense cells: keep the rejection sampler feasible
        min_dist = 0.5 * spacing
    d = dict(L=(L, L, L), grid=g, ions=random_positions(n_atoms, L, seed, min_dist),
             Z=np.ones(n_atoms), T=float(T_kelvin), functional=functional,
             rho=rho_gcc, n_atoms=n_atoms, masses=np.full(n_atoms, M_H_AMU * AMU_ME))
    if vel_seed is not None:
        d["vel"] = maxwell_boltzmann(n_atoms, T_kelvin, vel_seed)
    return d


def config_single_point(grid=32):
    """8 H at 1 g/cm^3, 100 kK, ftTF + PZ, 32^3 (single-point minimisation)."""
    return hydrogen(8, 1.0, 1.0e5, grid, seed=1, functional="fttf")


def config_md(functional="vt84f", grid=96, n_atoms=128):
    """128 H at 1 g/cm^3, 31.25 kK, SGA or ftGGA (VT84F), 96^3, MB velocities."""
    return hydrogen(n_atoms, 1.0, 3.125e4, grid, seed=2, functional=functional,
                    vel_seed=3)


def config_mixed(T_kelvin, grid=128, n_atoms=256):
    """256 H at 4 g/cm^3, ftGGA, 128^3; T in {1e4, 2.5e5, 4e6} K."""
    return hydrogen(n_atoms, 4.0, T_kelvin, grid, seed=4, functional="vt84f")


def config_batch(count=64, seed=5, n_range=(8, 512), rho_range=(0.1, 10.0),
                 T_range=(2.0e3, 4.0e6), grid_hi=160,
                 functionals=("fttf", "sga", "vt84f")):
    """Uneven batch: N_atoms, rho, T log-uniform; grid by the 0.25-bohr rule."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        na = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        rho = math.exp(rng.uniform(math.log(rho_range[0]), math.log(rho_range[1])))
        T = math.exp(rng.uniform(math.log(T_range[0]), math.log(T_range[1])))
        fn = functionals[int(rng.integers(len(functionals)))]
        L = cell_edge(na, rho)
        g = grid_edge(L, 0.25, 32, grid_hi)
        out.append(hydrogen(na, rho, T, g, seed=1000 + i, functional=fn))
    return out


def config_serve(count=24, seed=6, rate=50.0, n_range=(16, 128), rho_range=(0.1, 20.0),
                 T_range=(2.0e3, 4.0e6), grid_hi=96, functional="vt84f"):
    """Equation-of-state request stream: Poisson arrivals at `rate` per second
    of (rho, T, N_atoms) points drawn log-uniform, grid by the 0.25-bohr rule
    (32 .. grid_hi per edge).  Returns [(arrival_s, system dict)]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        na = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        rho = math.exp(rng.uniform(math.log(rho_range[0]), math.log(rho_range[1])))
        T = math.exp(rng.uniform(math.log(T_range[0]), math.log(T_range[1])))
        L = cell_edge(na, rho)
        g = grid_edge(L, 0.25, 32, grid_hi)
        d = hydrogen(na, rho, T, g, seed=2000 + i, functional=functional, vel_seed=3000 + i)
        out.append((t, d))
    return out
