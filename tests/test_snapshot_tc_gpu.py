"""The tensor-core snapshot products of UpdateSVD (Alg. 1: U^T F and
F - U U_F) through the C ABI, against FP64 numpy on the same inputs.

The products are formed in split-TF32 with FP32 accumulation: the bound used
here, 1e-5 of |A_m| |B_n| per entry (Cauchy-Schwarz scale of the entry),
sits an order above the expected 2^-21 per product plus the FP32
accumulation error, and two orders below what one TF32 pass (2^-11) gives.
Sizes are ragged in every dimension: M and K not multiples of the 128-row
tile or the 32-element chunk, N across the 32/64 column tiles and above 64
(two launches)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx():
    import torch
    from paper_1905_00473_gb300 import binding
    c = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    return binding.pr_create(2, 64, 4, c, 0.25 / 64, 1.0 / 64, 2, 8.0 / 64)


@pytest.mark.parametrize("K,M,N", [(12345, 300, 32), (49152, 1024, 32), (777, 129, 17),
                                   (4099, 64, 64), (20000, 200, 70), (31, 5, 3)])
def test_project_matches_fp64(lib, K, M, N):
    import torch
    from paper_1905_00473_gb300 import binding
    rng = np.random.default_rng(K + M + N)
    A = rng.standard_normal((M, K)) * rng.uniform(0.1, 10.0, size=(M, 1))
    B = rng.standard_normal((N, K))
    ctx = _ctx()
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.full((N, M), float("nan"), dtype=torch.float64, device="cuda")
    binding.pr_snapshot_project(ctx, Ad, Bd, Cd)
    binding.pr_check(ctx)
    C = Cd.cpu().numpy()                         # C[n, m] = sum_k A[m, k] B[n, k]
    ref = B @ A.T
    scale = np.outer(np.linalg.norm(B, axis=1), np.linalg.norm(A, axis=1))
    err = np.max(np.abs(C - ref) / scale)
    assert err <= 1e-5, err


@pytest.mark.parametrize("M,K,N", [(49152, 1024, 32), (5000, 300, 17), (130, 33, 64),
                                   (3000, 100, 65), (128, 1, 1)])
def test_deflate_matches_fp64(lib, M, K, N):
    import torch
    from paper_1905_00473_gb300 import binding
    rng = np.random.default_rng(M + K + N)
    A = rng.standard_normal((K, M))               # columns of length M
    T = rng.standard_normal((N, K))
    F = rng.standard_normal((N, M))
    ctx = _ctx()
    Ad, Td, Fd = (torch.tensor(x, device="cuda") for x in (A, T, F))
    Od = torch.full_like(Fd, float("nan"))
    binding.pr_snapshot_deflate(ctx, Ad, Td, Fd, Od)
    binding.pr_check(ctx)
    ref = F - T @ A                                # O[n, r] = F[n, r] - sum_j A[j, r] T[n, j]
    scale = np.outer(np.linalg.norm(T, axis=1), np.linalg.norm(A, axis=0)) + 1e-300
    err = np.max(np.abs(Od.cpu().numpy() - ref) / scale)
    assert err <= 1e-5, err
    # in place: O == F
    binding.pr_snapshot_deflate(ctx, Ad, Td, Fd, Fd)
    binding.pr_check(ctx)
    assert np.max(np.abs(Fd.cpu().numpy() - ref) / scale) <= 1e-5


def test_gram_of_an_orthonormal_basis_is_the_identity(lib):
    """Q^T Q of a 49152 x 256 orthonormal basis (the shape of the stored
    bases of the 512^2 workload) is the identity to FP32-level accuracy.
    The diagonal, a sum of 49152 positive products, comes out low by about
    3e-6 on a GB300 (the FP32 accumulation inside the tensor core is not
    unbiased round-to-nearest); the off-diagonal entries stay near 1e-9."""
    import torch
    from paper_1905_00473_gb300 import binding
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((49152, 256)))
    Qd = torch.tensor(Q.T.copy(), device="cuda")    # (columns, rows)
    G = torch.zeros((256, 256), dtype=torch.float64, device="cuda")
    ctx = _ctx()
    binding.pr_snapshot_project(ctx, Qd, Qd[:64].contiguous(), G[:64])
    binding.pr_check(ctx)
    Gh = G[:64].cpu().numpy()
    np.testing.assert_allclose(Gh, np.eye(256)[:64], atol=1e-5)
    off = Gh - np.eye(256)[:64] * np.diag(Gh[:, :64])[:, None]
    assert np.max(np.abs(off)) < 1e-7


def test_invalid_arguments_are_rejected(lib):
    import ctypes

    import torch
    from paper_1905_00473_gb300 import binding
    ctx = _ctx()
    lib_ = binding.load()
    a = torch.zeros(1024, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(a.data_ptr())
    s = ctypes.c_void_p(0)
    assert lib_.pr_snapshot_project(ctx.handle, p, 10, p, 32, 32, 4, 2, p, 4, s) == 1    # lda < K
    assert lib_.pr_snapshot_project(ctx.handle, None, 32, p, 32, 32, 4, 2, p, 4, s) == 1
    assert lib_.pr_snapshot_project(ctx.handle, p, 32, p, 32, -1, 4, 2, p, 4, s) == 1
    assert lib_.pr_snapshot_deflate(ctx.handle, p, 3, p, 8, p, 4, 4, 8, 2, p, 4, s) == 1  # lda < M
    # O partly overlapping F, or overlapping A
    b = torch.zeros(1024, dtype=torch.float64, device="cuda")
    pb = ctypes.c_void_p(b.data_ptr())
    q = ctypes.c_void_p(b.data_ptr() + 8)
    assert lib_.pr_snapshot_deflate(ctx.handle, p, 16, p, 8, pb, 16, 16, 8, 2, q, 16, s) == 1
    assert lib_.pr_snapshot_deflate(ctx.handle, p, 16, pb, 8, pb, 16, 16, 8, 2, p, 16, s) == 1
    assert lib_.pr_snapshot_project(ctx.handle, p, 32, pb, 32, 32, 4, 2, p, 4, s) == 1   # C on A
    assert lib_.pr_snapshot_project(None, p, 32, p, 32, 32, 4, 2, p, 4, s) == 1
