"""Velocity-Verlet NVE molecular dynamics of the FP64 oracle.

TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper runs its MD in RXMD with NVE/NVT integration and 0.5 fs steps (Methodology,
MD Simulations of C-S-H Nanoparticle Reaction); QMD uses an explicit reversible
integrator (Methodology, QMD).  The oracle integrates with the textbook velocity-Verlet
scheme in float64 (a reading of "explicit reversible integrator" for the NVE case):

    v <- v + dt/2 * F/m;   x <- x + dt * v;   F <- F(x);   v <- v + dt/2 * F/m

with F/m converted from eV/(A amu) to A/fs^2 (1 eV/(A amu) = 9.648533212e-3 A/fs^2).
Positions are not wrapped back into the box (periodic images are handled by the shifts).
"""
from __future__ import annotations

import numpy as np

ACC = 9.648533212e-3      # (eV / (A amu)) -> A / fs^2
K_B = 8.617333262e-5      # eV / K


def kinetic(v, m):
    """Kinetic energy in eV of velocities v (A/fs) and masses m (amu)."""
    return 0.5 * float(np.sum(m[:, None] * v * v)) / ACC


def run_nve(model, pos, vel, Z, box, pbc, masses, dt, n_steps):
    """Integrate n_steps; returns (x, v, E_pot per step, E_kin per step) after each step."""
    x = np.array(pos, dtype=np.float64)
    v = np.array(vel, dtype=np.float64)
    m = np.asarray(masses, dtype=np.float64)
    E, _, F = model.evaluate(x, Z, box, pbc)
    epot, ekin = [], []
    for _ in range(n_steps):
        v += 0.5 * dt * ACC * F / m[:, None]
        x += dt * v
        E, _, F = model.evaluate(x, Z, box, pbc)
        v += 0.5 * dt * ACC * F / m[:, None]
        epot.append(float(E.sum()))
        ekin.append(kinetic(v, m))
    return x, v, np.array(epot), np.array(ekin)


def _thermostat_half(v, m, xi, eta, dt, g, kT, Q):
    """Nose-Hoover half step (dt/2) of the time-reversible Trotter splitting:
    xi += dt/4 G; v *= exp(-xi dt/2); eta += dt/2 xi; xi += dt/4 G', with
    G = (2 KE - g kT) / Q evaluated before and after the velocity scaling."""
    ke = kinetic(v, m)
    xi += 0.25 * dt * (2.0 * ke - g * kT) / Q
    v *= np.exp(-0.5 * dt * xi)
    eta += 0.5 * dt * xi
    ke = kinetic(v, m)
    xi += 0.25 * dt * (2.0 * ke - g * kT) / Q
    return v, xi, eta


def run_nvt(model, pos, vel, Z, box, pbc, masses, dt, n_steps, T, tau, xi=0.0, eta=0.0):
    """Nose-Hoover NVT (the paper thermalises and heats its systems in the canonical
    ensemble; Methodology, MD Simulations): one thermostat with mass Q = g kB T tau^2,
    g = 3N degrees of freedom, around a velocity-Verlet step.  Returns
    (x, v, E_pot, E_kin, H, xi, eta) with H = E_pot + E_kin + Q xi^2 / 2 + g kB T eta the
    conserved extended energy (per step)."""
    x = np.array(pos, dtype=np.float64)
    v = np.array(vel, dtype=np.float64)
    m = np.asarray(masses, dtype=np.float64)
    g = 3 * x.shape[0]
    kT = K_B * T
    Q = g * kT * tau * tau
    E, _, F = model.evaluate(x, Z, box, pbc)
    epot, ekin, H = [], [], []
    for _ in range(n_steps):
        v, xi, eta = _thermostat_half(v, m, xi, eta, dt, g, kT, Q)
        v += 0.5 * dt * ACC * F / m[:, None]
        x += dt * v
        E, _, F = model.evaluate(x, Z, box, pbc)
        v += 0.5 * dt * ACC * F / m[:, None]
        v, xi, eta = _thermostat_half(v, m, xi, eta, dt, g, kT, Q)
        ke = kinetic(v, m)
        epot.append(float(E.sum()))
        ekin.append(ke)
        H.append(float(E.sum()) + ke + 0.5 * Q * xi * xi + g * kT * eta)
    return x, v, np.array(epot), np.array(ekin), np.array(H), xi, eta
