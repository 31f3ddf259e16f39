"""FP64 reference of one molecular-dynamics step at constant temperature: the
velocity-Verlet step wrapped in Nose-Hoover thermostat half steps (the NVT
protocol of Sec. VI-A: production MD at fixed temperature).

TEST INFRASTRUCTURE ONLY (part of the oracle).

Equations of motion (Nose-Hoover, one thermostat variable xi with time
integral eta, g = 3n degrees of freedom, thermostat mass Q = g kB T tau^2):

    dr/dt   = v
    dv/dt   = F(r) / m - xi v
    dxi/dt  = (2 KE - g kB T) / Q,       KE = sum_i m_i |v_i|^2 / 2
    deta/dt = xi

They conserve H' = KE + U(r) + Q xi^2 / 2 + g kB T eta.  One step of length
dt is the symmetric (time-reversible) splitting

    thermostat(dt/2) . kick(dt/2) . drift(dt) . kick(dt/2) . thermostat(dt/2)

where kick and drift are the velocity-Verlet flows of the Hamiltonian part
and thermostat(h) integrates the (xi, eta, v) subsystem at fixed r as
xi += (h/2) G, v *= exp(-xi h), eta += xi h, xi += (h/2) G, with G the
force on xi evaluated from the current kinetic energy.  Nothing here shares
code with the library; forces are supplied by the caller.

Metal units: A, ps, amu, eV; 1 amu A^2/ps^2 = 1.0364269e-4 eV.
"""
from __future__ import annotations

import numpy as np

EV_PER_AMU_A2_PS2 = 1.0364269e-4     # kinetic energy unit conversion
KB_EV_PER_K = 8.617333262e-5         # Boltzmann constant


def kinetic_energy(v, m):
    """sum_i m_i |v_i|^2 / 2 in eV (v: [n, 3] A/ps, m: [n] amu)."""
    v = np.asarray(v, np.float64)
    return 0.5 * float(np.sum(np.asarray(m, np.float64) * np.sum(v * v, axis=1))) * EV_PER_AMU_A2_PS2


def thermostat_mass(n_atoms, temperature, tau):
    """(g kB T, Q) for g = 3 n degrees of freedom and period tau (ps)."""
    gkT = 3.0 * n_atoms * KB_EV_PER_K * temperature
    return gkT, gkT * tau * tau


def thermostat_flow(v, m, xi, eta, h, gkT, Q):
    """Advance (xi, eta, v) by a time h at fixed positions (see the module
    docstring).  Returns (v, xi, eta)."""
    v = np.asarray(v, np.float64)
    xi = xi + 0.5 * h * (2.0 * kinetic_energy(v, m) - gkT) / Q
    v = v * np.exp(-xi * h)
    eta = eta + xi * h
    xi = xi + 0.5 * h * (2.0 * kinetic_energy(v, m) - gkT) / Q
    return v, xi, eta


def accel(f, m):
    """F / m in A/ps^2 for F in eV/A and m in amu."""
    return np.asarray(f, np.float64) / (np.asarray(m, np.float64)[:, None] * EV_PER_AMU_A2_PS2)


def nvt_step(x, v, m, force, dt, temperature, tau, xi, eta, f0=None):
    """One Nose-Hoover velocity-Verlet step.

    x, v: [n, 3] positions (A) and velocities (A/ps); m: [n] masses (amu);
    force: callable r -> F(r) [n, 3] (eV/A); f0: F(x) if already known.
    temperature <= 0 turns the thermostat off (plain velocity Verlet).
    Returns (x, v, xi, eta, f) with f = F at the new positions."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    f = force(x) if f0 is None else np.asarray(f0, np.float64)
    nvt = temperature > 0.0
    if nvt:
        gkT, Q = thermostat_mass(len(x), temperature, tau)
        v, xi, eta = thermostat_flow(v, m, xi, eta, 0.5 * dt, gkT, Q)
    v = v + 0.5 * dt * accel(f, m)
    x = x + dt * v
    f = force(x)
    v = v + 0.5 * dt * accel(f, m)
    if nvt:
        v, xi, eta = thermostat_flow(v, m, xi, eta, 0.5 * dt, gkT, Q)
    return x, v, xi, eta, f


def conserved(x, v, m, potential, temperature, tau, xi, eta):
    """H' = KE + U + Q xi^2 / 2 + g kB T eta (eV)."""
    gkT, Q = thermostat_mass(len(x), temperature, tau)
    return kinetic_energy(v, m) + float(potential(x)) + 0.5 * Q * xi * xi + gkT * eta
