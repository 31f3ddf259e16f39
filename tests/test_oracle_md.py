"""Pins of the oracle's Nose-Hoover velocity-Verlet step (oracle/md.py), on a
small anharmonic test system with analytic forces (CPU only):

- one step against a fine fourth-order Runge-Kutta integration of the
  Nose-Hoover equations of motion themselves (an independent method): the
  local error must fall like dt^3 (a symmetric splitting is second order);
- the conserved quantity H' = KE + U + Q xi^2/2 + g kB T eta: its excursion
  over a fixed time must be small and fall like dt^2;
- time reversibility: a step of -dt undoes a step of dt to rounding;
- without the thermostat (T = 0, or a very slow one) the step is textbook
  velocity Verlet.
A mistake in the force on xi, the sign of the friction, the order of the
half steps or the unit conversion fails at least one of these."""
import numpy as np

from oracle import md as M

RNG = np.random.default_rng(11)
N = 5
MASS = np.array([195.084, 1.008, 12.0, 40.0, 195.084])
K_SPRING, A_QUART, C_PAIR = 4.0, 3.0, 0.7      # eV/A^2, eV/A^4, eV/A^2
X0 = RNG.normal(scale=0.3, size=(N, 3))
V0 = RNG.normal(scale=1.0, size=(N, 3)) * np.sqrt(300.0 * M.KB_EV_PER_K / (MASS[:, None] * M.EV_PER_AMU_A2_PS2))


def potential(x):
    """sum_i (k |x_i|^2 / 2 + a |x_i|^4 / 4) + sum_{i<j} c |x_i - x_j|^2 / 2"""
    r2 = np.sum(x * x, axis=1)
    s = x.sum(0)
    return float(np.sum(0.5 * K_SPRING * r2 + 0.25 * A_QUART * r2 * r2) + 0.5 * C_PAIR * (N * r2.sum() - s @ s))


def force(x):
    r2 = np.sum(x * x, axis=1)[:, None]
    return -(K_SPRING + A_QUART * r2) * x - C_PAIR * (N * x - x.sum(0))


def test_forces_are_minus_the_gradient():
    h = 1e-6
    f = force(X0)
    for i, c in ((0, 0), (1, 2), (3, 1)):
        xp, xm = X0.copy(), X0.copy()
        xp[i, c] += h
        xm[i, c] -= h
        assert abs(-(potential(xp) - potential(xm)) / (2 * h) - f[i, c]) <= 1e-7


def _rk4_reference(x, v, xi, eta, t_total, temperature, tau, substeps=4000):
    """The Nose-Hoover equations of motion integrated by classical RK4."""
    gkT, Q = M.thermostat_mass(N, temperature, tau)
    conv = 1.0 / M.EV_PER_AMU_A2_PS2

    def rhs(y):
        xx, vv, z = y[0], y[1], y[2]
        ke = 0.5 * np.sum(MASS * np.sum(vv * vv, axis=1)) * M.EV_PER_AMU_A2_PS2
        return (vv, force(xx) * conv / MASS[:, None] - z[0] * vv, np.array([(2 * ke - gkT) / Q, z[0]]))

    y = (x.copy(), v.copy(), np.array([xi, eta]))
    h = t_total / substeps
    for _ in range(substeps):
        k1 = rhs(y)
        k2 = rhs(tuple(a + 0.5 * h * b for a, b in zip(y, k1)))
        k3 = rhs(tuple(a + 0.5 * h * b for a, b in zip(y, k2)))
        k4 = rhs(tuple(a + h * b for a, b in zip(y, k3)))
        y = tuple(a + h / 6.0 * (b1 + 2 * b2 + 2 * b3 + b4) for a, b1, b2, b3, b4 in zip(y, k1, k2, k3, k4))
    return y[0], y[1], y[2][0], y[2][1]


def _step_error(dt, temperature=450.0, tau=0.02, xi0=3.0, eta0=0.1):
    x1, v1, xi1, eta1, _ = M.nvt_step(X0, V0, MASS, force, dt, temperature, tau, xi0, eta0)
    xr, vr, xir, etar = _rk4_reference(X0, V0, xi0, eta0, dt, temperature, tau)
    return (np.abs(x1 - xr).max(), np.abs(v1 - vr).max(), abs(xi1 - xir), abs(eta1 - etar))


def test_local_error_is_third_order_against_the_equations_of_motion():
    # the lightest particle (1 amu, 4 eV/A^2) has omega ~ 200 / ps: omega dt ~ 0.08
    e1 = _step_error(0.0004)
    e2 = _step_error(0.0002)
    for a, b in zip(e1, e2):
        assert a > 1e-11, e1             # well above the reference's own error
        assert 6.0 <= a / b <= 12.0, (e1, e2)   # 8 for dt^3; 4 or 16 for the wrong order


def _max_excursion(dt, t_total=0.08, temperature=450.0, tau=0.05):
    x, v, xi, eta = X0.copy(), V0.copy(), 0.0, 0.0
    h0 = M.conserved(x, v, MASS, potential, temperature, tau, xi, eta)
    f = None
    dev = 0.0
    for _ in range(int(round(t_total / dt))):
        x, v, xi, eta, f = M.nvt_step(x, v, MASS, force, dt, temperature, tau, xi, eta, f0=f)
        dev = max(dev, abs(M.conserved(x, v, MASS, potential, temperature, tau, xi, eta) - h0))
    return dev, M.kinetic_energy(V0, MASS)


def test_conserved_quantity_error_is_second_order():
    d1, ke = _max_excursion(0.0004)
    d2, _ = _max_excursion(0.0002)
    assert d1 < 0.02 * ke, (d1, ke)
    assert 3.0 <= d1 / d2 <= 5.5, (d1, d2)


def test_equipartition_at_the_target_temperature():
    """The thermostat drives the kinetic energy to its equipartition value
    (3n/2) kB T: the time average over the second half of 12 ps of a coupled
    anharmonic system (which the single thermostat samples ergodically)
    must be within 6 % of it, from a start at 300 K."""
    x, v, xi, eta, f = X0.copy(), V0.copy(), 0.0, 0.0, None
    ke = []
    steps = 60000
    for k in range(steps):
        x, v, xi, eta, f = M.nvt_step(x, v, MASS, force, 0.0004, 450.0, 0.05, xi, eta, f0=f)
        if k >= steps // 2:
            ke.append(M.kinetic_energy(v, MASS))
    target = 1.5 * N * 8.617333262e-5 * 450.0
    assert abs(np.mean(ke) / target - 1.0) <= 0.06, np.mean(ke) / target


def test_step_is_time_reversible():
    x1, v1, xi1, eta1, _ = M.nvt_step(X0, V0, MASS, force, 0.003, 450.0, 0.02, 1.5, 0.2)
    x0, v0, xi0, eta0, _ = M.nvt_step(x1, v1, MASS, force, -0.003, 450.0, 0.02, xi1, eta1)
    assert np.abs(x0 - X0).max() <= 1e-12
    assert np.abs(v0 - V0).max() <= 1e-11
    assert abs(xi0 - 1.5) <= 1e-11 and abs(eta0 - 0.2) <= 1e-12


def test_without_thermostat_it_is_velocity_verlet():
    dt = 0.003
    a0 = force(X0) / (MASS[:, None] * M.EV_PER_AMU_A2_PS2)
    x_vv = X0 + dt * V0 + 0.5 * dt * dt * a0
    a1 = force(x_vv) / (MASS[:, None] * M.EV_PER_AMU_A2_PS2)
    v_vv = V0 + 0.5 * dt * (a0 + a1)
    x1, v1, xi, eta, _ = M.nvt_step(X0, V0, MASS, force, dt, 0.0, 0.1, 0.0, 0.0)
    assert np.abs(x1 - x_vv).max() <= 1e-13 and np.abs(v1 - v_vv).max() <= 1e-12
    assert xi == 0.0 and eta == 0.0
    # a very slow thermostat (Q -> infinity) barely couples
    x2, v2, xi2, _, _ = M.nvt_step(X0, V0, MASS, force, dt, 450.0, 1e6, 0.0, 0.0)
    assert np.abs(x2 - x_vv).max() <= 1e-12 and np.abs(v2 - v_vv).max() <= 1e-10 and abs(xi2) < 1e-12
