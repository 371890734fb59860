"""pr_serial_sweep, the serial corrected sweep of Alg. 3 on its own, against
the FP64 oracle's serial sweep (oracle.parareal.serial_sweep) on the same
inputs: the previous iteration's slice states u^k_n, their fine values
F u^k_{n-1} and coarse values C R u^k_{n-1} (computed by the oracle), and, for
the Procrustes corrector, the Omega = X Y^T that pr_procrustes_correct builds
from the oracle's data matrices F = [Lambda R F u^k_{n-1}], G = [Lambda U_n].

FP64 contexts agree to ~1e-9 (same arithmetic, other rounding order and FFT
library); FP32 contexts to the 1e-4 relative energy-norm bound of the FP32
parareal solution."""
import numpy as np
import pytest

from oracle import energy, parareal, procrustes
from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P
from tests.test_parareal_gpu import CORR, _case, _ctx, _problem

pytestmark = pytest.mark.gpu


def _inputs(w, Pb, seed):
    """u^k_n (n = 0..N) and the oracle's F u^k_{n-1}, C R u^k_{n-1}."""
    rng = np.random.default_rng(seed)
    base = W.periodic_gaussian(w.dim, w.n_fine, [0.35] * w.dim, 0.12)
    uk = []
    for n in range(w.n_slices + 1):
        shift = tuple(int(x) for x in rng.integers(0, w.n_fine, size=w.dim))
        uk.append((np.roll(base, shift, axis=tuple(range(w.dim))) * (1.0 + 0.1 * n),
                   0.05 * np.roll(base, shift[::-1], axis=tuple(range(w.dim)))))
    v = [parareal.F(Pb, *uk[n - 1]) for n in range(1, w.n_slices + 1)]
    Uc = [parareal.C(Pb, *parareal.R(Pb, *uk[n - 1])) for n in range(1, w.n_slices + 1)]
    return uk, v, Uc


@pytest.mark.parametrize("dim,n,N,m_f,dtype,corrector", [
    (1, 64, 4, 8, "f64", "procrustes"),
    (1, 64, 4, 8, "f64", "omega1"),
    (1, 64, 4, 8, "f64", "plain"),
    (2, 32, 3, 8, "f64", "procrustes"),
    (2, 128, 3, 16, "f32", "procrustes"),
])
def test_serial_sweep_matches_oracle(lib, dim, n, N, m_f, dtype, corrector):
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(dim, n, N, m_f, dtype, 4)
    Pb = _problem(w, corrector, tol=1e-13)
    uk, v, Uc = _inputs(w, Pb, seed=n + N)
    X = Y = None
    ctx = _ctx(w, 4, tol=1e-13)
    if corrector == "procrustes":
        Fm = np.stack([parareal.Lam(Pb, *parareal.R(Pb, *vn)) for vn in v], axis=1)
        Gm = np.stack([parareal.Lam(Pb, *Un) for Un in Uc], axis=1)
        X, _, Y = procrustes.update_svd(None, None, None, Fm, Gm, 1e-13)
        binding.pr_procrustes_correct(ctx, torch.tensor(Fm.T.copy(), device="cuda"),
                                      torch.tensor(Gm.T.copy(), device="cuda"))
    expect = parareal.serial_sweep(Pb, uk[0], v, Uc, X, Y)
    dt = torch.float32 if dtype == "f32" else torch.float64
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    Fu, Fv = t(np.stack([x[0] for x in v])), t(np.stack([x[1] for x in v]))
    Uu, Uv = t(np.stack([x[0] for x in Uc])), t(np.stack([x[1] for x in Uc]))
    us = torch.zeros((N + 1,) + w.shape, dtype=dt, device="cuda")
    vs = torch.zeros_like(us)
    us[0], vs[0] = t(uk[0][0]), t(uk[0][1])
    binding.pr_serial_sweep(ctx, CORR[corrector], Fu, Fv, Uu, Uv, us, vs)
    binding.pr_check(ctx)
    ug, vg = us.double().cpu().numpy(), vs.double().cpu().numpy()
    for k in range(1, N + 1):
        e = energy.relative_energy_error(ug[k], vg[k], expect[k][0], expect[k][1], w.c, w.dx_f)
        assert e <= (1e-9 if dtype == "f64" else 1e-4), (k, e)


def test_serial_sweep_rejects_overlap_and_missing_coarse_grid(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(1, 64, 4, 8, "f64", 4)
    ctx = _ctx(w, 4)
    F = torch.zeros((4, 64), dtype=torch.float64, device="cuda")
    U = torch.zeros((4, 16), dtype=torch.float64, device="cuda")
    us = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    vs = torch.zeros_like(us)
    with pytest.raises(binding.PrError):   # the fine values alias output slices 1..4
        binding.pr_serial_sweep(ctx, CORR["plain"], us[1:], F, U, U, us, vs)
    with pytest.raises(binding.PrError):
        binding.pr_serial_sweep(ctx, 7, F, F, U, U, us, vs)
