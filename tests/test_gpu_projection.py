"""GPU capped-simplex projection (mcf_project_capped_simplex, Sec. 2.3) against the oracle's
sort-based projection (Sec. 2.6), column by column, on random and adversarial columns."""
import numpy as np
import pytest

from oracle import pdmcf as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run_gpu(lib, Q, c, ld=None, mu0=None, inplace=False, garbage_pads=False):
    m, n = Q.shape
    ld = ld or (n + 3) // 4 * 4
    Qt = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    Qt[:, :n] = torch.from_numpy(Q.astype(np.float32))
    if garbage_pads and ld > n:
        Qt[:, n:] = 1e6
    cap = torch.from_numpy(c.astype(np.float32)).cuda()
    mu = torch.zeros(m, dtype=torch.float32, device="cuda") if mu0 is None else \
        torch.from_numpy(mu0.astype(np.float32)).cuda()
    Ft = Qt if inplace else torch.full((m, ld), -7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    d2 = lib.mcf_project_capped_simplex(n, m, ld, Qt.data_ptr(), cap.data_ptr(), Ft.data_ptr(),
                                        mu.data_ptr(), torch.cuda.current_stream().cuda_stream)
    F = Ft.cpu().numpy()
    assert np.all(F[:, n:] == 0)
    return F[:, :n], mu.cpu().numpy(), d2


def reference(Q, c):
    q64 = Q.astype(np.float32).astype(np.float64)
    c64 = c.astype(np.float32).astype(np.float64)
    F, mu = O.project_capped_simplex(q64.T, c64)
    return F.T, mu, float(np.sum((F.T - q64) ** 2))


def check(lib, Q, c, **kw):
    Fg, mug, d2 = run_gpu(lib, Q, c, **kw)
    Fr, mur, d2r = reference(Q, c)
    scale = max(1.0, float(np.abs(Q).max()), float(c.max()))
    assert np.all(Fg >= 0)
    assert np.all(Fg.sum(axis=1) <= c * (1 + 1e-5) + 1e-6 * scale)
    assert np.abs(Fg - Fr).max() <= 2e-5 * scale
    assert np.abs(mug - mur).max() <= 2e-5 * scale
    assert d2 == pytest.approx(d2r, rel=1e-4, abs=1e-8 * scale * scale)
    return Fg, mug


@pytest.mark.parametrize("n", [1, 3, 7, 100, 1000, 4097, 10000])
def test_random_columns(lib, n):
    rng = np.random.default_rng(n)
    m = 300 if n < 5000 else 60
    Q = rng.normal(scale=rng.choice([0.1, 1.0, 10.0]), size=(m, n))
    c = rng.uniform(0.05, 3.0, size=m) * max(1.0, n ** 0.5 / 10)
    check(lib, Q, c)


@pytest.mark.parametrize("case", ["ties", "allneg", "just_above", "tiny_c", "one_big",
                                  "below_cap", "spread"])
def test_adversarial_columns(lib, case):
    rng = np.random.default_rng(7)
    m, n = 200, 517
    Q = rng.normal(size=(m, n))
    c = rng.uniform(0.1, 5.0, size=m)
    if case == "ties":
        Q = np.round(Q, 1)
    elif case == "allneg":
        Q = -np.abs(Q) - 1e-3
    elif case == "just_above":
        c = np.maximum(Q, 0).sum(axis=1) * (1 - 1e-4)
    elif case == "tiny_c":
        c = np.full(m, 1e-6)
    elif case == "one_big":
        Q = -np.abs(Q)
        Q[:, 5] = 50.0
    elif case == "below_cap":
        c = np.maximum(Q, 0).sum(axis=1) * 1.5
    elif case == "spread":
        Q = np.sign(Q) * np.exp(rng.uniform(-12, 4, size=(m, n)))
    check(lib, Q, c)


def test_warm_starts_give_the_same_projection(lib):
    rng = np.random.default_rng(11)
    m, n = 400, 250
    Q = rng.normal(size=(m, n))
    c = rng.uniform(0.2, 2.0, size=m)
    _, mur, _ = reference(Q, c)
    for mu0 in (mur, mur * 3 + 1, mur * 0.5, np.full(m, 100.0)):
        check(lib, Q, c, mu0=mu0)


def test_inplace_and_ragged_pads(lib):
    rng = np.random.default_rng(12)
    m, n = 100, 37
    Q = rng.normal(size=(m, n))
    c = rng.uniform(0.2, 2.0, size=m)
    check(lib, Q, c, ld=48, garbage_pads=True)
    check(lib, Q, c, inplace=True)


def test_empty_and_invalid(lib):
    assert lib.mcf_project_capped_simplex(10, 0, 12, 0, 0, 0, 0) == 0.0
    with pytest.raises(lib.MCFError):
        lib.mcf_project_capped_simplex(10, 5, 9, 16, 16, 16, 16)       # ld < n
    x = torch.zeros(64, device="cuda")
    with pytest.raises(lib.MCFError):
        lib.mcf_project_capped_simplex(4, 1, 4, x.data_ptr() + 4, x.data_ptr(),
                                       x.data_ptr(), x.data_ptr())    # misaligned


def test_full_size_sampled(lib):
    """n = 10^4 columns (the large workload's vector length), m = 10^5: sampled columns
    against the oracle one by one."""
    rng = np.random.default_rng(13)
    m, n = 100000, 10000
    Qd = torch.randn((m, n), device="cuda", generator=torch.Generator("cuda").manual_seed(5)) * 0.05
    cap = torch.rand(m, device="cuda") * 2 + 0.1
    mu = torch.zeros(m, device="cuda")
    Ft = torch.empty_like(Qd)
    d2 = lib.mcf_project_capped_simplex(n, m, n, Qd.data_ptr(), cap.data_ptr(), Ft.data_ptr(),
                                        mu.data_ptr(), torch.cuda.current_stream().cuda_stream)
    rows = rng.choice(m, size=40, replace=False)
    Q = Qd[rows].cpu().numpy()
    c = cap[rows].cpu().numpy()
    Fr, mur, _ = reference(Q, c)
    Fg = Ft[rows].cpu().numpy()
    assert np.abs(Fg - Fr).max() <= 2e-5 * max(1.0, np.abs(Q).max())
    assert np.abs(mu[rows].cpu().numpy() - mur).max() <= 2e-5
    assert d2 > 0 and np.isfinite(d2)
