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


# ---------------------------------------------------------------------------
# Adjoint of the parareal solve with the phase correctors frozen (the
# differentiation reading of Alg. 3: Omega^k held at its forward value).
# ---------------------------------------------------------------------------
from oracle import parareal, transfer  # noqa: E402


def _rand(rng, shape):
    return rng.standard_normal(shape)


@pytest.mark.parametrize("shape,ratio", [((24,), 4), ((20,), 2), ((18,), 3), ((12, 8), 2),
                                         ((8, 8), 1), ((12, 12, 4), 2)])
def test_transfer_transposes(shape, ratio):
    rng = np.random.default_rng(len(shape) * 10 + ratio)
    cshape = tuple(s // ratio for s in shape)
    x, y = _rand(rng, cshape), _rand(rng, shape)
    # <I x, y> = <x, I^T y>, <R y, x> = <y, R^T x>
    lhs = np.sum(transfer.interpolate(x, ratio) * y)
    assert abs(lhs - np.sum(x * adjoint.interpolate_T(y, ratio))) <= 1e-12 * (1 + abs(lhs))
    lhs = np.sum(transfer.restrict(y, ratio) * x)
    assert abs(lhs - np.sum(y * adjoint.restrict_T(x, ratio, shape))) <= 1e-12 * (1 + abs(lhs))


@pytest.mark.parametrize("shape", [(16,), (15,), (8, 6), (6, 4, 5)])
@pytest.mark.parametrize("order", [2, 4, 0])
def test_energy_map_transposes(shape, order):
    rng = np.random.default_rng(sum(shape) + order)
    dim = len(shape)
    c = 1.0 + 0.5 * rng.uniform(size=shape)
    dx = 1.0 / shape[-1]
    w, wt = _rand(rng, shape), _rand(rng, shape)
    g = _rand(rng, (dim + 1,) * 0 + ((dim + 1) * int(np.prod(shape)),))
    # Lambda (linear in (w, w_t) at fixed c)
    lhs = np.sum(transfer.energy_map(w, wt, c, dx, order) * g)
    bw, bwt, _ = adjoint.energy_map_T(g, wt, c, dx, order)
    assert abs(lhs - np.sum(w * bw) - np.sum(wt * bwt)) <= 1e-11 * (1 + abs(lhs))
    # Lambda^dagger (linear in (vec, zero mode) at fixed c)
    z = float(rng.standard_normal())
    q1, ut = transfer.reconstruct(g, z, c)
    a, b = _rand(rng, shape), _rand(rng, shape)
    lhs = np.sum(q1 * a) + np.sum(ut * b)
    bvec, bz, _ = adjoint.reconstruct_T(a, b, g, c)
    assert abs(lhs - np.sum(g * bvec) - z * bz) <= 1e-11 * (1 + abs(lhs))


def _pr_problem(corrector, dim=1, n=16, N=4, ratio=2, seed=5, grad_order=4):
    rng = np.random.default_rng(seed)
    c = workloads.smooth_random_speed(dim, n, rng)
    dt_f = 0.25 / (n * c.max())
    P = parareal.Problem(c_fine=c, ratio=ratio, n_slices=N, dt_com=8 * dt_f, m_f=8, m_c=2,
                         grad_order=grad_order, tol=1e-12, corrector=corrector)
    u0 = workloads.periodic_gaussian(dim, n, [0.4] * dim, 0.15)
    p0 = 0.3 * workloads.periodic_gaussian(dim, n, [0.6] * dim, 0.2)
    return P, u0, p0, rng


def _omegas(P, u0, p0, K):
    return [(r.X, r.Y) for r in parareal.iterate(P, u0, p0, K)]


@pytest.mark.parametrize("corrector", ["procrustes", "omega1", "plain"])
def test_frozen_forward_reproduces_the_iteration(corrector):
    P, u0, p0, _ = _pr_problem(corrector)
    recs = parareal.iterate(P, u0, p0, 3)
    hist = adjoint.parareal_frozen(P, u0, p0, 3, [(r.X, r.Y) for r in recs])
    for k, rec in enumerate(recs):
        for a, b in zip(rec.states, hist[k + 1]):
            np.testing.assert_allclose(a[0], b[0], atol=1e-13)
            np.testing.assert_allclose(a[1], b[1], atol=1e-11)


@pytest.mark.parametrize("corrector", ["procrustes", "omega1", "plain"])
@pytest.mark.parametrize("dim,n,ratio", [(1, 16, 2), (2, 8, 2), (1, 12, 1)])
def test_parareal_adjoint_dot_product(corrector, dim, n, ratio):
    """<J x, y> = <x, J^T y> for J: (u0, p0) -> u^{K+1}_N at K = 2 < N = 4."""
    P, u0, p0, rng = _pr_problem(corrector, dim=dim, n=n, ratio=ratio)
    K = 2
    om = _omegas(P, u0, p0, K)
    x0, x1 = _rand(rng, u0.shape), _rand(rng, u0.shape)
    gu, gv = _rand(rng, u0.shape), _rand(rng, u0.shape)
    out = adjoint.parareal_frozen(P, x0, x1, K, om)[-1][-1]
    lhs = np.sum(out[0] * gu) + np.sum(out[1] * gv)
    bu, bp, _ = adjoint.parareal_adjoint(P, x0, x1, K, om, gu, gv)
    rhs = np.sum(x0 * bu) + np.sum(x1 * bp)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("corrector", ["procrustes", "omega1", "plain"])
@pytest.mark.parametrize("dim,n", [(1, 16), (2, 8)])
def test_parareal_adjoint_dc_central_differences(corrector, dim, n):
    """dL/dc of the frozen map against central differences in FP64, with
    L = <g_u, u^{K+1}_N> + <g_v, u_t^{K+1}_N> and c perturbed on the fine
    grid (the coarse c is R c; Lambda, Lambda^dagger and both propagators
    see the change)."""
    P, u0, p0, rng = _pr_problem(corrector, dim=dim, n=n)
    K = 2
    om = _omegas(P, u0, p0, K)
    gu, gv = _rand(rng, u0.shape), _rand(rng, u0.shape)
    _, _, bc = adjoint.parareal_adjoint(P, u0, p0, K, om, gu, gv)
    c0 = P.c_fine.copy()

    def loss(c):
        P.c_fine = c
        out = adjoint.parareal_frozen(P, u0, p0, K, om)[-1][-1]
        P.c_fine = c0
        return np.sum(out[0] * gu) + np.sum(out[1] * gv)

    for _ in range(2):
        d = rng.standard_normal(c0.shape)
        eps = 1e-6
        fd = (loss(c0 + eps * d) - loss(c0 - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(bc * d)) <= 1e-6 * abs(fd) + 1e-8, (fd, np.sum(bc * d))


@pytest.mark.parametrize("corrector", ["procrustes", "plain"])
def test_parareal_adjoint_at_k_equal_n_is_the_serial_fine_adjoint(corrector):
    """Finite termination makes u^{N+1}_N = F^N u_0 for every (u0, p0, c) with
    the correctors frozen, so its gradient is the serial fine adjoint."""
    P, u0, p0, rng = _pr_problem(corrector, N=3)
    K = P.n_slices
    om = _omegas(P, u0, p0, K)
    gu, gv = _rand(rng, u0.shape), _rand(rng, u0.shape)
    bu, bp, bc = adjoint.parareal_adjoint(P, u0, p0, K, om, gu, gv)
    ru, rp, rc = adjoint.serial_fine_adjoint(u0, p0, P.c_fine, P.dt_com / P.m_f, P.m_f,
                                             P.n_slices, P.dx_f, gu, gv)
    scale = max(np.abs(ru).max(), np.abs(rp).max())
    np.testing.assert_allclose(bu, ru, atol=1e-9 * scale)
    np.testing.assert_allclose(bp, rp, atol=1e-9 * scale)
    np.testing.assert_allclose(bc, rc, atol=1e-8 * np.abs(rc).max())


def test_parareal_adjoint_planted_mistake_is_caught(monkeypatch):
    """Omega applied untransposed in the reverse sweep breaks the dot product."""
    P, u0, p0, rng = _pr_problem("procrustes")
    K = 2
    om = _omegas(P, u0, p0, K)
    gu, gv = _rand(rng, u0.shape), _rand(rng, u0.shape)
    out = adjoint.parareal_frozen(P, u0, p0, K, om)[-1][-1]
    lhs = np.sum(out[0] * gu) + np.sum(out[1] * gv)
    bad = [(Y, X) for X, Y in om]     # the reverse sweep then applies X Y^T instead of Y X^T
    orig = adjoint.parareal_frozen
    monkeypatch.setattr(adjoint, "parareal_frozen", lambda P_, a, b, K_, o: orig(P_, a, b, K_, om))
    bu, bp, _ = adjoint.parareal_adjoint(P, u0, p0, K, bad, gu, gv)
    rhs = np.sum(u0 * bu) + np.sum(p0 * bp)
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)
