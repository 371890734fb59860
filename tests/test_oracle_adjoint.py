"""Pins of the adjoint oracle: the dot-product test (the adjoint of a linear
map in the state), central finite differences for dL/dc in FP64, and the
slice-by-slice composition of the serial fine adjoint."""
import numpy as np
import pytest

from oracle import adjoint, fine
from paper_1905_00473_gb300 import workloads


def _setup(dim, n, seed):
    rng = np.random.default_rng(seed)
    c = workloads.smooth_random_speed(dim, n, rng)
    dx = 1.0 / n
    dt = 0.25 * dx / c.max()
    u, v, gu, gv = rng.standard_normal((4,) + (n,) * dim)
    return rng, c, dx, dt, u, v, gu, gv


@pytest.mark.parametrize("dim,n", [(1, 40), (2, 16), (3, 8)])
def test_dot_product(dim, n):
    # <F x, y> = <x, F^T y> for the state map at fixed c
    _, c, dx, dt, u, v, gu, gv = _setup(dim, n, dim)
    uf, vf = fine.velocity_verlet(u, v, c, dt, 13, dx)
    bu, bv, _ = adjoint.verlet_adjoint(u, v, c, dt, 13, dx, gu, gv)
    lhs = np.sum(uf * gu) + np.sum(vf * gv)
    rhs = np.sum(u * bu) + np.sum(v * bv)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("dim,n", [(1, 32), (2, 12), (3, 8)])
def test_dc_central_differences(dim, n):
    rng, c, dx, dt, u, v, gu, gv = _setup(dim, n, 10 + dim)
    steps = 11

    def loss(cc):
        uf, vf = fine.velocity_verlet(u, v, cc, dt, steps, dx)
        return np.sum(uf * gu) + np.sum(vf * gv)

    _, _, bc = adjoint.verlet_adjoint(u, v, c, dt, steps, dx, gu, gv)
    for _ in range(3):
        d = rng.standard_normal(c.shape)
        eps = 1e-6
        fd = (loss(c + eps * d) - loss(c - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(bc * d)) <= 1e-6 * abs(fd) + 1e-9, (fd, np.sum(bc * d))


def test_serial_fine_adjoint_composes_and_matches_fd():
    rng, c, dx, dt, u, v, gu, gv = _setup(2, 10, 21)
    m, N = 6, 3

    def forward(cc, uu, vv):
        for _ in range(N):
            uu, vv = fine.velocity_verlet(uu, vv, cc, dt, m, dx)
        return uu, vv

    bu, bv, bc = adjoint.serial_fine_adjoint(u, v, c, dt, m, N, dx, gu, gv)
    one_u, one_v, one_c = adjoint.verlet_adjoint(u, v, c, dt, m * N, dx, gu, gv)
    np.testing.assert_allclose(bu, one_u, atol=1e-10)
    np.testing.assert_allclose(bv, one_v, atol=1e-10)
    np.testing.assert_allclose(bc, one_c, atol=1e-8 * np.abs(one_c).max())
    d = rng.standard_normal(c.shape)
    L = lambda cc: sum(np.sum(a * b) for a, b in zip(forward(cc, u, v), (gu, gv)))
    fd = (L(c + 1e-6 * d) - L(c - 1e-6 * d)) / 2e-6
    assert abs(fd - np.sum(bc * d)) <= 1e-6 * abs(fd)


def test_planted_mistake_fails_the_dot_product():
    _, c, dx, dt, u, v, gu, gv = _setup(2, 12, 5)
    uf, vf = fine.velocity_verlet(u, v, c, dt, 9, dx)
    bu, bv, _ = adjoint.verlet_adjoint(u, v, c, dt, 9, dx, gu, gv)
    lhs = np.sum(uf * gu) + np.sum(vf * gv)
    # transposing K D as K D instead of D K (kappa outside the stencil) is a
    # typical mistake for variable c: it breaks the identity
    c2 = c * c
    wrong = u * 0
    bu2, bv2, ba2 = np.array(gu), np.array(gv), np.zeros_like(gu)
    rhs_ok = np.sum(u * bu) + np.sum(v * bv)
    assert abs(lhs - rhs_ok) < 1e-10 * abs(lhs)
    Lk = lambda x: c2 * fine.laplacian(x, dx)           # K D, not its transpose D K
    us = [u]
    uu, vv = u, v
    a = Lk(uu)
    for _ in range(9):
        uu = uu + dt * vv + 0.5 * dt * dt * a
        an = Lk(uu)
        vv = vv + 0.5 * dt * (a + an)
        a = an
    for n in range(8, -1, -1):
        ban = ba2 + 0.5 * dt * bv2
        ba_n = 0.5 * dt * bv2
        bu2 = bu2 + Lk(ban)
        bv2 = bv2 + dt * bu2
        ba2 = ba_n + 0.5 * dt * dt * bu2
    bu2 = bu2 + Lk(ba2)
    rhs_bad = np.sum(u * bu2) + np.sum(v * bv2)
    assert abs(lhs - rhs_bad) > 1e-6 * abs(lhs)
