"""Pins of the oracle's fine/coarse stepper against what the mathematics fixes.

None of these tests re-types the oracle's update formulas: they check
 * exact discrete plane waves for constant c (closed form from the symbol of
   the 3/5/7-point Laplacian and the two-step form of velocity Verlet),
 * the modified energy that velocity Verlet conserves exactly for a linear
   system M u'' = -A u (M = c^-2, A = -L symmetric), written with forward
   differences rather than the oracle's Laplacian,
 * time reversibility of velocity Verlet,
 * slice independence of F over a sweep (Alg. 3, parFor),
and a set of planted mistakes shows that each pin has teeth.
"""
import math

import numpy as np
import pytest

from oracle import fine
from paper_1905_00473_gb300 import workloads


def _coords(dim, n):
    return workloads.node_coords(dim, n)


def plane_wave(dim, n, kvec, c, dt, steps):
    """Closed-form discrete plane wave of the scheme, constant c.

    With symbol lambda = sum_i 4 sin^2(k_i dx/2)/dx^2 of -L, velocity Verlet
    reduces to u_{n+1} - 2u_n + u_{n-1} = -(c dt)^2 lambda u_n, whose
    solutions are cos(k.x - n theta) with sin(theta/2) = c dt sqrt(lambda)/2;
    the velocity follows from u_{n+1} - u_{n-1} = 2 dt v_n.
    """
    dx = 1.0 / n
    xs = _coords(dim, n)
    phase = sum(kvec[i] * xs[i] for i in range(dim)) + np.zeros([n] * dim)
    lam = sum(4.0 * math.sin(kvec[i] * dx / 2) ** 2 for i in range(dim)) / dx ** 2
    theta = 2.0 * math.asin(c * dt * math.sqrt(lam) / 2.0)
    amp = math.sin(theta) / dt
    u0 = np.cos(phase)
    v0 = amp * np.sin(phase)
    ut = np.cos(phase - steps * theta)
    vt = amp * np.sin(phase - steps * theta)
    return u0, v0, ut, vt


def modified_energy(u, v, c, dt, dx):
    """H = dx^d [1/2 sum c^-2 v^2 + 1/2 sum_e sum_j ((u_{j+e}-u_j)/dx)^2
                 - dt^2/8 sum c^-2 a^2],  a = c^2 L u.

    L is rebuilt here as the divergence of forward differences, not taken
    from the oracle.
    """
    fwd = [(np.roll(u, -1, axis=ax) - u) / dx for ax in range(u.ndim)]
    lap = sum((g - np.roll(g, 1, axis=ax)) / dx for ax, g in enumerate(fwd))
    a = c * c * lap
    pot = 0.5 * sum(np.sum(g * g) for g in fwd)
    kin = 0.5 * np.sum(v * v / (c * c))
    corr = dt * dt / 8.0 * np.sum(a * a / (c * c))
    return (kin + pot - corr) * dx ** u.ndim


def smooth_state(dim, n, seed):
    rng = np.random.default_rng(seed)
    u = workloads.fourier_mode_field(dim, n, rng, modes=6, kmax=3)
    v = 5.0 * workloads.fourier_mode_field(dim, n, rng, modes=6, kmax=3)
    return u, v


def variable_speed(dim, n, seed):
    rng = np.random.default_rng(seed)
    return workloads.smooth_random_speed(dim, n, rng)


PLANE_CASES = [
    (1, 32, (2 * math.pi * 3,)),
    (1, 32, (2 * math.pi * 15,)),
    (2, 16, (2 * math.pi * 1, 2 * math.pi * 5)),
    (2, 16, (2 * math.pi * -3, 2 * math.pi * 7)),
    (3, 8, (2 * math.pi * 1, 2 * math.pi * -2, 2 * math.pi * 3)),
]


def check_plane_waves(verlet, tol=1e-11):
    for dim, n, k in PLANE_CASES:
        c = 1.3
        dt = 0.25 / (n * c)
        steps = 37
        u0, v0, ut, vt = plane_wave(dim, n, k, c, dt, steps)
        cf = np.full([n] * dim, c)
        u, v = verlet(u0, v0, cf, dt, steps, 1.0 / n)
        scale = np.max(np.abs(v0)) + 1e-300
        if not (np.max(np.abs(u - ut)) < tol and np.max(np.abs(v - vt)) / scale < tol):
            return False
    return True


def check_energy(verlet, tol=1e-12):
    for dim, n in [(1, 64), (2, 24), (3, 10)]:
        c = variable_speed(dim, n, 7 + dim)
        u, v = smooth_state(dim, n, 11 + dim)
        dx = 1.0 / n
        dt = 0.25 * dx / np.max(c)
        h0 = modified_energy(u, v, c, dt, dx)
        u1, v1 = verlet(u, v, c, dt, 50, dx)
        h1 = modified_energy(u1, v1, c, dt, dx)
        if not (np.isfinite(h1) and abs(h1 - h0) / abs(h0) < tol):
            return False
    return True


def check_reversible(verlet, tol=1e-11):
    for dim, n in [(1, 40), (2, 16)]:
        c = variable_speed(dim, n, 3)
        u, v = smooth_state(dim, n, 5)
        dx = 1.0 / n
        dt = 0.25 * dx / np.max(c)
        u1, v1 = verlet(u, v, c, dt, 25, dx)
        u2, v2 = verlet(u1, -v1, c, dt, 25, dx)
        if not (np.max(np.abs(u2 - u)) < tol * np.max(np.abs(u))
                and np.max(np.abs(v2 + v)) < tol * np.max(np.abs(v))):
            return False
    return True


def all_pins(verlet):
    return {
        "plane": check_plane_waves(verlet),
        "energy": check_energy(verlet),
        "reversible": check_reversible(verlet),
    }


def test_plane_wave_exact():
    assert check_plane_waves(fine.velocity_verlet)


def test_modified_energy_conserved_variable_c():
    assert check_energy(fine.velocity_verlet)


def test_time_reversible():
    assert check_reversible(fine.velocity_verlet)


def test_plane_wave_at_config_cfl_all_dims():
    # the configs' CFL 0.25 / max c on every axis, many steps, several modes
    for dim, n in [(1, 64), (2, 32), (3, 12)]:
        rng = np.random.default_rng(dim)
        k = tuple(2 * math.pi * int(m) for m in rng.integers(-n // 2 + 1, n // 2, size=dim))
        c, dt = 2.0, 0.25 / (n * 2.0)
        u0, v0, ut, vt = plane_wave(dim, n, k, c, dt, 200)
        u, v = fine.velocity_verlet(u0, v0, np.full([n] * dim, c), dt, 200, 1.0 / n)
        assert np.max(np.abs(u - ut)) < 1e-10
        assert np.max(np.abs(v - vt)) < 1e-10 * np.max(np.abs(v0))


def test_slices_are_independent():
    dim, n, N = 2, 16, 5
    c = variable_speed(dim, n, 1)
    dx = 1.0 / n
    dt = 0.25 * dx / np.max(c)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((N, n, n))
    v = rng.standard_normal((N, n, n))
    uo, vo = fine.fine_all_slices(u, v, c, dt, 9, dx)
    perm = rng.permutation(N)
    up, vp = fine.fine_all_slices(u[perm], v[perm], c, dt, 9, dx)
    np.testing.assert_array_equal(up, uo[perm])
    np.testing.assert_array_equal(vp, vo[perm])
    for s in range(N):
        us, vs = fine.velocity_verlet(u[s], v[s], c, dt, 9, dx)
        np.testing.assert_array_equal(us, uo[s])
        np.testing.assert_array_equal(vs, vo[s])


def test_zero_steps_and_zero_state():
    c = np.ones((8, 8))
    u, v = np.random.default_rng(1).standard_normal((2, 8, 8))
    u1, v1 = fine.velocity_verlet(u, v, c, 0.01, 0, 1 / 8)
    np.testing.assert_array_equal(u1, u)
    np.testing.assert_array_equal(v1, v)
    z = np.zeros((8, 8))
    u2, v2 = fine.velocity_verlet(z, z, c, 0.01, 10, 1 / 8)
    assert not np.any(u2) and not np.any(v2)


def test_step_counts_of_the_configs():
    # m_F = smallest multiple of 4 with dt_com/m_F <= 0.25 dx/max c
    assert workloads.config1().m_f == 96
    assert workloads.config2().m_f == 192
    assert workloads.config3().m_f == 384
    w5 = workloads.config5(n=32)
    assert w5.m_f % 4 == 0
    assert w5.dt_f <= 0.25 * w5.dx_f / w5.cmax * (1 + 1e-12)
    assert w5.dt_com / (w5.m_f - 4) > 0.25 * w5.dx_f / w5.cmax


# ---- planted mistakes: each mutant of the oracle must fail at least one pin ----

def _verlet_with_laplacian(lap):
    def verlet(u, v, c, dt, steps, dx):
        u = np.array(u, dtype=np.float64)
        v = np.array(v, dtype=np.float64)
        c2 = c * c
        a = c2 * lap(u, dx)
        for _ in range(steps):
            u = u + dt * v + 0.5 * dt * dt * a
            a_next = c2 * lap(u, dx)
            v = v + 0.5 * dt * (a + a_next)
            a = a_next
        return u, v
    return verlet


def _lap_wrong_sign(u, dx):
    return -fine.laplacian(u, dx)


def _lap_first_axis_only(u, dx):
    return (np.roll(u, -1, axis=0) - 2 * u + np.roll(u, 1, axis=0)) / dx ** 2


def _lap_missing_center_scale(u, dx):
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        out += (np.roll(u, -1, axis=ax) - u + np.roll(u, 1, axis=ax)) / dx ** 2
    return out


def _lap_shifted(u, dx):
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        out += (np.roll(u, -2, axis=ax) - 2 * u + np.roll(u, 1, axis=ax)) / dx ** 2
    return out


def _verlet_c_not_squared(u, v, c, dt, steps, dx):
    return fine.velocity_verlet(u, v, np.sqrt(c), dt, steps, dx)


def _verlet_no_half_drift(u, v, c, dt, steps, dx):
    u = np.array(u, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    a = c * c * fine.laplacian(u, dx)
    for _ in range(steps):
        u = u + dt * v + dt * dt * a
        a_next = c * c * fine.laplacian(u, dx)
        v = v + 0.5 * dt * (a + a_next)
        a = a_next
    return u, v


def _verlet_stale_kick(u, v, c, dt, steps, dx):
    u = np.array(u, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    for _ in range(steps):
        a = c * c * fine.laplacian(u, dx)
        u = u + dt * v + 0.5 * dt * dt * a
        v = v + dt * a
    return u, v


def _verlet_a_once(u, v, c, dt, steps, dx):
    # reuses the first acceleration for the whole slice
    u = np.array(u, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    a = c * c * fine.laplacian(u, dx)
    for _ in range(steps):
        u = u + dt * v + 0.5 * dt * dt * a
        v = v + dt * a
    return u, v


MUTANTS = {
    "laplacian sign": _verlet_with_laplacian(_lap_wrong_sign),
    "laplacian one axis": _verlet_with_laplacian(_lap_first_axis_only),
    "laplacian centre weight": _verlet_with_laplacian(_lap_missing_center_scale),
    "laplacian shifted stencil": _verlet_with_laplacian(_lap_shifted),
    "c not squared": _verlet_c_not_squared,
    "drift without 1/2": _verlet_no_half_drift,
    "symplectic-Euler kick": _verlet_stale_kick,
    "frozen acceleration": _verlet_a_once,
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    with np.errstate(all="ignore"):
        res = all_pins(MUTANTS[name])
    assert not all(res.values()), f"mutant '{name}' passed every pin: {res}"
