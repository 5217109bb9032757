"""The Arnoldi process on the device (gsk_arnoldi: GMRES's basis kernels,
CGS2) against the oracle's, through the C ABI: the Hessenberg matrix
element by element, finite termination with the exact eigenvalues, the
argument checks, the Ritz values and the eigenvalue tables (1b) built on
them, and the 128^3 workload."""
import numpy as np
import pytest

import oracle
from gpu_util import gsk, random_csr, to_dev
from problems import cd, configs

pytestmark = pytest.mark.gpu


def _h_close(Hg, Ho, tol):
    scale = np.abs(Ho).max()
    return np.abs(Hg - Ho).max() <= tol * scale


@pytest.mark.parametrize("case,m", [("c1", 20), ("random", 64), ("c2_21", 30), ("tiny", 5)])
def test_arnoldi_matches_oracle(case, m):
    import torch

    g = gsk()
    if case == "c1":
        s = configs.c1()
    elif case == "c2_21":
        s = configs.c2(21)
    elif case == "tiny":
        s = configs.c1(3)
    else:
        rp, ci, va = random_csr(5000, 14, long_rows=(7, 4000), long_len=300)
        s = cd.System(5000, rp, ci, va, np.ones(5000))
    A, _ = to_dev(g, s)
    v0 = np.random.default_rng(3).normal(size=s.n)
    H, k = g.arnoldi(A, torch.as_tensor(v0, device="cuda"), m)
    _, Ho, ko = oracle.arnoldi(s.rowptr, s.colidx, s.val, v0, m)
    assert k == ko
    # the same recurrences; GPU sums in a different order, and the process
    # amplifies rounding differences by at most the growth seen here
    assert _h_close(H, Ho[: k + 1, :k], 1e-10), np.abs(H - Ho[: k + 1, :k]).max()
    assert np.all(np.tril(H, -2) == 0.0) and np.all(np.diag(H, -1) > 0)


@pytest.mark.parametrize("k", [1, 5])
def test_arnoldi_finite_termination(k):
    import torch

    g = gsk()
    n = 3000
    vals = np.array([0.5 + 1.3 * j for j in range(k)])
    d = vals[np.arange(n) % k]
    A = g.Csr.from_host(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    v0 = np.random.default_rng(4).uniform(1, 2, n)
    H, steps = g.arnoldi(A, torch.as_tensor(v0, device="cuda"), 12)
    assert steps == k
    assert np.allclose(np.sort(np.linalg.eigvals(H[:k, :k]).real), vals, rtol=1e-11)


def test_arnoldi_arguments():
    import torch

    g = gsk()
    s = configs.c1(8)
    A, _ = to_dev(g, s)
    H, k = g.arnoldi(A, torch.zeros(s.n, dtype=torch.float64, device="cuda"), 4)
    assert k == 0 and H.shape == (1, 0)
    v = torch.ones(s.n, dtype=torch.float64, device="cuda")
    for m in (0, 65):
        with pytest.raises(g.GskError) as e:
            g.arnoldi(A, v, m)
        assert e.value.status == g.ERR_ARG
    A32 = g.Csr.from_host(s.rowptr, s.colidx, s.val, dtype=torch.float32)
    with pytest.raises(g.GskError) as e:
        g.arnoldi(A32, v, 4)
    assert e.value.status == g.ERR_ARG
    bad = v.clone()
    bad[5] = float("nan")
    with pytest.raises(g.GskError) as e:
        g.arnoldi(A, bad, 4)
    assert e.value.status == g.ERR_NONFINITE


def test_ritz_values_find_the_extreme_eigenvalue():
    """Problem 1 at 40 x 40 after GS(2) on the device: the largest Ritz value
    of 64 steps matches the dense eigensolver's lambda_max (Table 1b: 1.78),
    and the Ritz values of the device and oracle Hessenberg matrices agree."""
    import torch

    from paper_0812_2769_gb300 import spectrum

    g = gsk()
    s = configs.p1(40)
    A, b = to_dev(g, s)
    g.gs_scale(A, b, p=2.0)
    ritz, H, k = spectrum.ritz_values(A, m=64, seed=9)
    assert k == 64
    lmax = spectrum.summary(spectrum.dense_eigenvalues(A))["lambda_max"]
    assert abs(np.abs(ritz).max() - lmax) <= 1e-3 * lmax, (np.abs(ritz).max(), lmax)
    assert abs(lmax - 1.78) <= 0.006 * 1.78
    val_or = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)[0]
    v0 = np.random.default_rng(9).normal(size=s.n)
    _, Ho, _ = oracle.arnoldi(s.rowptr, s.colidx, val_or, v0, 64)
    ro = np.linalg.eigvals(Ho[:64, :64])
    assert abs(np.abs(ro).max() - np.abs(ritz).max()) <= 1e-9 * lmax


def test_eigen_table_1b_on_the_device_scaling():
    """reproduce.run_eigen('1b'): GS(2) on the device, the dense summary on the
    host: Table 1b's counts and extremes."""
    from paper_0812_2769_gb300 import reproduce

    res = reproduce.run_eigen("1b", out=lambda *_: None)
    for label, (lo, hi, _, cnt) in reproduce.PAPER_EIGEN["1b"].items():
        d = res[label]
        assert d["first_interval"] == cnt, (label, d)
        assert abs(d["lambda_min"] - lo) <= 0.01 * lo and abs(d["lambda_max"] - hi) <= 0.006 * hi, (label, d)


def test_arnoldi_c2_full_size():
    """The 128^3 workload (2.1 M unknowns) after GS(2): 16 device steps
    against the oracle's (a few seconds of CPU)."""
    import torch

    g = gsk()
    s = configs.c2(128)
    A, b = to_dev(g, s)
    g.gs_scale(A, b, p=2.0)
    v0 = np.random.default_rng(10).normal(size=s.n)
    H, k = g.arnoldi(A, torch.as_tensor(v0, device="cuda"), 16)
    val_or = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)[0]
    _, Ho, ko = oracle.arnoldi(s.rowptr, s.colidx, val_or, v0, 16)
    assert k == ko == 16
    assert _h_close(H, Ho[:17, :16], 1e-10), np.abs(H - Ho[:17, :16]).max()
