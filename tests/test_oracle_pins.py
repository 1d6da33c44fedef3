"""Pins for the CPU oracle: each test checks it against something other than itself
(closed forms, brute force, an independent solver, library routines, invariants).

Paper: Zhang & Boyd, "Solving Large Multicommodity Network Flow Problems on GPUs".
"""
import inspect
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize as so

from oracle import barrier as B
from oracle import pdmcf as O
from paper_2501_17996_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def solve(inst, **kw):
    return O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma, **kw)


def offdiag(n):
    return ~np.eye(n, dtype=bool)


# ----------------------------------------------------------------- network (Sec. 1.1)

def test_incidence_products_match_definition():
    inst = I.random_small(7, 20, 0)
    n, m = inst.n, inst.m
    A = O.incidence(n, inst.tail, inst.head).toarray()
    for l in range(m):
        col = np.zeros(n)
        col[inst.head[l]] = 1.0
        col[inst.tail[l]] = -1.0
        assert np.array_equal(A[:, l], col)
    rng = np.random.default_rng(1)
    Y = rng.normal(size=(n, n))
    F = rng.normal(size=(n, m))
    ya = np.empty((n, m))
    for i in range(n):
        for l in range(m):
            ya[i, l] = Y[i, inst.head[l]] - Y[i, inst.tail[l]]
    assert np.allclose(Y @ A, ya, rtol=0, atol=1e-13)
    fat = np.zeros((n, n))
    for l in range(m):
        fat[:, inst.head[l]] += F[:, l]
        fat[:, inst.tail[l]] -= F[:, l]
    assert np.allclose(F @ A.T, fat, rtol=0, atol=1e-12)
    # T = -F A^T has zero row sums for any F (columns of A sum to zero), Sec. 1.1
    assert np.allclose((-F @ A.T).sum(axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("n,deg,seed", [(20, 3, 0), (60, 5, 1), (150, 10, 2)])
def test_eta_bounds_spectral_norm(n, deg, seed):
    """Eq. (e-eta) and Appendix A: lambda_max(A A^T) <= 2 d_max, so eta <= 1/||A||_2."""
    t, h = I.ring_plus_random(n, deg, np.random.default_rng(seed))
    A = O.incidence(n, t, h).toarray()
    smax = np.linalg.svd(A, compute_uv=False)[0]
    d = np.diag(A @ A.T)
    assert smax ** 2 <= 2 * d.max() + 1e-9
    eta = O.eta_bound(n, t, h)
    assert eta <= 1.0 / smax + 1e-15
    assert math.isclose(eta, 1.0 / math.sqrt(2 * d.max()), rel_tol=1e-15)


# ----------------------------------------------------------------- projection (Sec. 2.3, 2.6)

def brute_project(q, c):
    """Projection onto {f >= 0, sum f <= c} by enumerating supports: for every support S
    try the slack candidate f_S = q_S and the tight candidate f_S = q_S - mu_S; keep the
    feasible candidate closest to q (the projection is one of them)."""
    n = len(q)
    best, best_d = None, math.inf
    for mask in range(1 << n):
        S = [i for i in range(n) if (mask >> i) & 1]
        cands = []
        f = np.zeros(n)
        f[S] = q[S]
        cands.append(f)
        if S:
            mu = (q[S].sum() - c) / len(S)
            g = np.zeros(n)
            g[S] = q[S] - mu
            cands.append(g)
        for f in cands:
            if np.all(f >= -1e-15) and f.sum() <= c + 1e-12:
                dist = float(np.sum((f - q) ** 2))
                if dist < best_d - 1e-15:
                    best, best_d = f, dist
    return best


def test_projection_vs_brute_force():
    rng = np.random.default_rng(0)
    cols, caps = [], []
    for _ in range(120):
        n = int(rng.integers(1, 8))
        q = rng.normal(scale=rng.choice([0.1, 1.0, 5.0]), size=n)
        if rng.random() < 0.2:
            q[: n // 2] = q[0]                  # ties
        cols.append(q)
        caps.append(float(rng.choice([1e-3, 0.5, 1.0, 3.0, abs(q).sum() * 0.999])))
    for q, c in zip(cols, caps):
        F, mu = O.project_capped_simplex(q[:, None], np.array([c]))
        ref = brute_project(q, c)
        assert np.allclose(F[:, 0], ref, atol=1e-12), (q, c)


@pytest.mark.parametrize("case", ["random", "ties", "allneg", "just_above", "tiny_c", "n1"])
def test_projection_kkt(case):
    rng = np.random.default_rng(hash(case) % 2**31)
    n, m = (1, 50) if case == "n1" else (257, 60)
    Q = rng.normal(size=(n, m))
    if case == "ties":
        Q = np.round(Q, 1)
    if case == "allneg":
        Q = -np.abs(Q)
    c = rng.uniform(0.1, 5.0, size=m)
    if case == "just_above":
        c = np.maximum(Q, 0).sum(axis=0) * (1 - 1e-9)
    if case == "tiny_c":
        c = np.full(m, 1e-9)
    F, mu = O.project_capped_simplex(Q, c)
    assert np.all(F >= 0)
    assert np.all(F.sum(axis=0) <= c * (1 + 1e-12) + 1e-15)
    assert np.all(mu >= 0)
    assert np.allclose(mu * (c - F.sum(axis=0)), 0, atol=1e-10)
    assert np.allclose(F, np.maximum(Q - mu, 0), atol=1e-14)
    # variational inequality of the Euclidean projection: <q - f, z - f> <= 0
    for _ in range(20):
        Z = np.abs(rng.normal(size=(n, m)))
        Z *= np.minimum(1.0, c / Z.sum(axis=0))
        assert np.all(np.sum((Q - F) * (Z - F), axis=0) <= 1e-10)


# ----------------------------------------------------------------- proxes (Sec. 2.3)

def conj_log(y, w):
    return w * np.log(w / (-y)) - w


def conj_pow(y, w, g):
    return (1 / g - 1) * (w * g) ** (1 / (1 - g)) * (-y) ** (-g / (1 - g))


def numeric_conj(y, u):
    """(-u)^*(y) = sup_s (y s + u(s)), by bounded scalar maximisation."""
    res = so.minimize_scalar(lambda ls: -(y * math.exp(ls) + u(math.exp(ls))),
                             bounds=(-30, 30), method="bounded", options={"xatol": 1e-12})
    return -res.fun


def test_conjugates_match_definition():
    rng = np.random.default_rng(3)
    for _ in range(30):
        y = -float(rng.uniform(0.05, 5))
        w = float(rng.uniform(0.3, 3))
        g = float(rng.uniform(0.2, 0.8))
        assert math.isclose(numeric_conj(y, lambda s: w * math.log(s)), conj_log(y, w), rel_tol=1e-7, abs_tol=1e-8)
        assert math.isclose(numeric_conj(y, lambda s: w * s ** g), conj_pow(y, w, g), rel_tol=1e-7, abs_tol=1e-8)
    util = O.Utility("pow", np.full((3, 3), 1.3), 0.4)
    Y = -np.full((3, 3), 0.7)
    np.fill_diagonal(Y, 0)
    assert math.isclose(util.conj_neg(Y), 6 * conj_pow(-0.7, 1.3, 0.4), rel_tol=1e-13)


def primal_prox(v, beta, du):
    """prox_{(-u)/beta}(v): root of s - v - u'(s)/beta = 0 on s > 0 (brentq)."""
    f = lambda s: s - v - du(s) / beta
    lo, hi = 1e-300, max(1.0, abs(v)) * 4 + 10
    while f(hi) < 0:
        hi *= 4
    return so.brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)


def test_prox_log_moreau_and_minimiser():
    rng = np.random.default_rng(4)
    for _ in range(200):
        y = float(rng.uniform(-20, 20))
        beta = float(rng.uniform(0.01, 3))
        w = float(rng.uniform(0.3, 3))
        z = float(O.prox_log(np.array([y]), beta, w)[0])
        assert z < 0
        # Moreau: prox_{beta f*}(y) = y - beta prox_{f/beta}(y/beta), f = -u
        s = primal_prox(y / beta, beta, lambda s: w / s)
        assert math.isclose(z, y - beta * s, rel_tol=1e-9, abs_tol=1e-11)
        # direct minimiser of beta (-u)^*(x) + (x - y)^2 / 2 over x < 0
        res = so.minimize_scalar(lambda lx: beta * conj_log(-math.exp(lx), w) + 0.5 * (-math.exp(lx) - y) ** 2,
                                 bounds=(-40, 10), method="bounded", options={"xatol": 1e-12})
        assert math.isclose(z, -math.exp(res.x), rel_tol=1e-6, abs_tol=1e-8)


def test_prox_pow_cubic_roots_and_moreau():
    rng = np.random.default_rng(5)
    for _ in range(200):
        y = float(rng.uniform(-10, 10))
        beta = float(rng.uniform(0.01, 3))
        w = float(rng.uniform(0.3, 3))
        # gamma = 1/2: c1 = 1, c2 = beta w^2 / 4, the cubic t^3 + y t^2 - c2 = 0
        z = float(O.prox_pow(np.array([y]), beta, w, 0.5)[0])
        roots = np.roots([1.0, y, 0.0, -beta * w * w / 4.0])
        real = [r.real for r in roots if abs(r.imag) < 1e-9 and r.real > 0]
        assert len(real) == 1
        assert math.isclose(-z, real[0], rel_tol=1e-9)
        # general gamma through the Moreau identity with the primal prox
        g = float(rng.uniform(0.2, 0.8))
        z = float(O.prox_pow(np.array([y]), beta, w, g)[0])
        s = primal_prox(y / beta, beta, lambda s: w * g * s ** (g - 1))
        assert math.isclose(z, y - beta * s, rel_tol=1e-9, abs_tol=1e-11)


def test_traffic_from_dual_inverts_marginal_utility():
    rng = np.random.default_rng(6)
    n = 6
    W = rng.uniform(0.3, 3, size=(n, n))
    G = rng.uniform(0.2, 0.8, size=(n, n))
    Y = -rng.uniform(0.1, 4, size=(n, n))
    np.fill_diagonal(Y, 0)
    off = offdiag(n)
    for util in (O.Utility("log", W), O.Utility("pow", W, G)):
        T = util.traffic_from_dual(Y)
        assert np.allclose(util.grad(T)[off], -Y[off], rtol=1e-12)


# ----------------------------------------------------------------- residual (Eq. e-res)

def test_residual_is_min_over_gamma():
    rng = np.random.default_rng(7)
    for _ in range(40):
        G = rng.normal(size=(4, 6))
        D = rng.normal(size=(4, 6))
        Q = rng.normal(size=(4, 6))
        F = Q + D
        res = so.minimize_scalar(lambda g: np.sum((G - g * D) ** 2), bounds=(0, 1e3),
                                 method="bounded", options={"xatol": 1e-12})
        direct = min(res.fun, float(np.sum(G * G)))
        assert math.isclose(O.residual(G, F, Q, True), direct, rel_tol=1e-8, abs_tol=1e-10)
    G = rng.normal(size=(3, 3))
    assert O.residual(G, np.ones((3, 3)), np.ones((3, 3)), True) == pytest.approx(np.sum(G * G))
    assert O.residual(G, np.ones((3, 3)), np.ones((3, 3)), False) == math.inf


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("kind", ["log", "pow"])
def test_two_node_closed_form(kind):
    """Two nodes, edges 0->1 (c_a) and 1->0 (c_b): any increasing utility saturates both
    edges, so T_10 = c_a, T_01 = c_b and Y_10 = -u'(c_a)."""
    ca, cb = 1.7, 0.45
    inst = I.two_node(ca, cb, kind, w12=0.8, w21=1.3, gamma=0.35 if kind == "pow" else None)
    r = solve(inst, eps=1e-12, stop_mode="kkt", max_iters=20000)
    assert r.status == "converged"
    assert r.T[1, 0] == pytest.approx(ca, rel=1e-9)
    assert r.T[0, 1] == pytest.approx(cb, rel=1e-9)
    du = (lambda s, w: w / s) if kind == "log" else (lambda s, w: w * 0.35 * s ** (0.35 - 1))
    assert r.Yhat[1, 0] == pytest.approx(-du(ca, 1.3), rel=1e-7)
    assert r.Yhat[0, 1] == pytest.approx(-du(cb, 0.8), rel=1e-7)
    assert np.allclose(r.T.sum(axis=1), 0, atol=1e-12)


def ring_distance(n):
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return (i - j) % n          # hops from source j to destination i along i -> i+1


@pytest.mark.parametrize("n", [3, 5, 8])
def test_directed_ring_log_closed_form(n):
    """Uniform ring, log utility: unique routes, so KKT gives T_ij = c/(d_ij (n-1)),
    Y_ij = -w d_ij (n-1)/c (each edge carries d pairs at distance d)."""
    c, w = 2.5, 1.4
    r = solve(I.directed_ring(n, c, w), eps=1e-12, stop_mode="kkt", max_iters=50000)
    d = ring_distance(n)
    off = offdiag(n)
    T_ref = np.zeros((n, n))
    T_ref[off] = c / (d[off] * (n - 1))
    assert np.allclose(r.T[off], T_ref[off], rtol=1e-8)
    assert np.allclose(r.Yhat[off], (-w * d * (n - 1) / c)[off], rtol=1e-7)
    U_ref = n * w * sum(math.log(c / (k * (n - 1))) for k in range(1, n))
    assert r.utility == pytest.approx(U_ref, rel=1e-10, abs=1e-10)


def test_directed_ring_power_closed_form():
    """Uniform ring, power utility: x_d = (lambda d / (w gamma))^(1/(gamma-1)) with lambda
    chosen by scalar bisection so that sum_d d x_d = c."""
    n, c, w, g = 6, 3.0, 0.9, 0.5
    r = solve(I.directed_ring(n, c, w, "pow", g), eps=1e-12, stop_mode="kkt", max_iters=50000)
    ds = np.arange(1, n)
    load = lambda lam: float(np.sum(ds * (lam * ds / (w * g)) ** (1 / (g - 1))))
    lam = so.brentq(lambda l: load(l) - c, 1e-8, 1e8, xtol=1e-300, rtol=1e-15)
    x = (lam * ds / (w * g)) ** (1 / (g - 1))
    d = ring_distance(n)
    off = offdiag(n)
    assert np.allclose(r.T[off], x[d[off] - 1], rtol=1e-8)


@pytest.mark.parametrize("n,m,seed,kind", [(4, 8, 1, "log"), (5, 12, 2, "log"),
                                           (5, 10, 3, "pow"), (6, 14, 4, "log")])
def test_agrees_with_barrier_newton(n, m, seed, kind):
    inst = I.random_small(n, m, seed, kind)
    _, Tb, Ub = B.solve(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma)
    r = solve(inst, eps=1e-11, stop_mode="kkt", max_iters=400000)
    off = offdiag(n)
    assert r.status == "converged"
    assert np.max(np.abs(r.T[off] - Tb[off]) / Tb[off]) < 1e-6
    assert r.utility == pytest.approx(Ub, rel=1e-9, abs=1e-9)


# ----------------------------------------------------------------- certificates

def test_first_iteration_closed_form():
    """From F = 0, Y = I - 11^T: Y A has column l = e_head - e_tail, so Q = alpha (e_h - e_t)
    and, when alpha <= c_l, Pi(Q) = alpha e_head; hence F^{1/2} = rho alpha e_head."""
    inst = I.tiny(0)
    r = solve(inst, stop_mode="none", max_iters=1)
    alpha = O.eta_bound(inst.n, inst.tail, inst.head)
    assert np.all(alpha <= inst.cap)
    F_ref = np.zeros((inst.n, inst.m))
    F_ref[inst.head, np.arange(inst.m)] = 1.9 * alpha
    assert np.allclose(r.F, F_ref, rtol=1e-15, atol=0)


def test_certificates_along_run():
    inst = I.tiny(1)
    n = inst.n
    Fsp, a = O.shortest_path_flow(n, inst.tail, inst.head, inst.cap)
    A = O.incidence(n, inst.tail, inst.head)
    util = O.Utility(inst.kind, inst.w)
    U_sp = util.value(-(Fsp @ A.T.toarray()))
    off = offdiag(n)
    for iters in (50, 200, 800):
        r = solve(inst, stop_mode="none", max_iters=iters)
        assert np.all(r.Fhat >= 0)
        assert np.all(r.Fhat.sum(axis=0) <= inst.cap * (1 + 1e-12))
        assert np.allclose(r.T.sum(axis=1), 0, atol=1e-12)
        assert np.all(np.diag(r.Yhat) == 0) and np.all(r.Yhat[off] < 0)
        if r.metrics.feasible:
            assert r.metrics.P <= r.metrics.D + 1e-9 * abs(r.metrics.D)
    assert r.metrics.rel_gap < 1e-4
    assert r.utility >= U_sp


def test_paper_constants_are_the_defaults():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    sig = inspect.signature(O.pdmcf).parameters
    for key in ("rho", "theta", "k_adapt", "tau"):
        assert sig[key].default == gold[key]["value"], key
    assert sig["omega0"].default == gold["omega0"]["value"]


def test_knn_generator_matches_table1_edge_counts():
    """Sec. 3.1 recipe: the edge counts of our kNN graphs match Table 1's m to a few %."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    for n, q, m_paper, _ in gold["table1_knn"]["rows"][:3]:
        ms = [I.knn(n, q, s).m for s in range(3)]
        assert abs(np.mean(ms) - m_paper) / m_paper < 0.05, (n, q, ms, m_paper)


# ----------------------------------------------------------------- the pins catch mistakes

def _ring_error(mod):
    n, c, w = 5, 2.5, 1.4
    inst = I.directed_ring(n, c, w)
    r = mod.pdmcf(inst.n, inst.tail, inst.head, inst.cap, "log", inst.w, eps=1e-10,
                  stop_mode="none", max_iters=3000)
    d = ring_distance(n)
    off = offdiag(n)
    t_err = np.max(np.abs(r.T[off] - c / (d[off] * (n - 1))))
    y_err = np.max(np.abs(r.Yhat[off] + w * d[off] * (n - 1) / c))
    return float(max(t_err, y_err))


def test_ring_pin_detects_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle (on the CPU) and check a pin catches each."""
    assert _ring_error(O) < 1e-8
    orig_inc = O.incidence
    mutations = {
        "prox drops beta": ("prox_log", lambda y, b, w: (y - np.sqrt(y * y + 4.0 * w)) / 2.0),
        "projection ignores capacity": ("project_capped_simplex",
                                        lambda Q, c: (np.maximum(Q, 0), np.zeros(Q.shape[1]))),
        "incidence head/tail swapped": ("incidence", lambda n, t, h: orig_inc(n, h, t)),
    }
    for name, (attr, fn) in mutations.items():
        with monkeypatch.context() as mp:
            mp.setattr(O, attr, fn)
            try:
                err = _ring_error(O)
            except Exception:
                err = math.inf
            assert not (err < 1e-6), name


def test_adaptation_stop_keeps_omega_constant():
    """Sec. 2.4: omega may stop adapting from some iteration on and stays constant after.

    The trigger iterations below were read by hand off the stored record of the run that
    never stops adapting (tests/golden/adapt_history_mid_s0.json: omega and rel_kkt at every
    stop test, k_check = 50), under the rule's reading (stop from the check where omega leaves
    a factor g^2 of omega_ref, its value at the first finite measure; or, in the final phase
    that begins at the first check with rel_kkt below adapt_guard_below, where omega leaves a
    factor g of its value there or rel_kkt exceeds g x the smallest so far):
      g = 1.05: omega_ref = 2.12601 (k = 250), band [1.92836, 2.34392]; omega = 1.84946 at
                k = 450 leaves it -> stop at 450.
      g = 1.5:  band (i) [0.94489, 4.7835] never left before 1050; the final phase begins at
                k = 650 (rel_kkt 0.00819) with omega_arm = 1.89063, band [1.26042, 2.83595];
                omega = 1.16422 at k = 1050 leaves it -> stop at 1050.
      g = 2.5, adapt_guard_below = 1e-3: band (i) [0.34016, 13.2876]; the final phase begins
                at k = 1400 (rel_kkt 8.60e-4), omega_arm = 0.89045, band [0.35618, 2.22613],
                never left; the smallest rel_kkt is 9.2716e-5 at k = 1950 and rel_kkt =
                2.9316e-4 > 2.5 x 9.2716e-5 = 2.3179e-4 at k = 2050 -> stop at 2050.
    Before the stop the run equals the unstopped one; after it omega never changes."""
    import json

    inst = I.mid(0)
    args = (inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma)
    kw = dict(stop_mode="none", max_iters=2200, k_check=50, history=True)
    rec = json.load(open(os.path.join(GOLDEN, "adapt_history_mid_s0.json")))["rows"]
    free = O.pdmcf(*args, adapt_guard=0, **kw)
    assert free.omega_frozen_at == -1
    for h, (k, w, r) in zip(free.history, rec):   # the record is this run's
        assert h["k"] == k and h["omega"] == pytest.approx(w, rel=1e-12)
        assert (r is None and not math.isfinite(h["rel_kkt"])) or h["rel_kkt"] == pytest.approx(r, rel=1e-9)
    for guard, below, trigger in ((1.05, 1e-2, 450), (1.5, 1e-2, 1050), (2.5, 1e-3, 2050)):
        held = O.pdmcf(*args, adapt_guard=guard, adapt_guard_below=below, **kw)
        assert held.omega_frozen_at == trigger, (guard, held.omega_frozen_at)
        w_frozen = next(h["omega"] for h in held.history if h["k"] == trigger)
        for a, b in zip(free.history, held.history):
            if a["k"] <= trigger:
                assert a["omega"] == b["omega"] and a["rel_kkt"] == b["rel_kkt"]
            else:
                assert b["omega"] == w_frozen
        assert free.omega != held.omega


def test_golden_solutions_are_the_literal_algorithm():
    """Every stored solution is that of Algorithm 2.1 with omega adapting throughout
    (Eq. e-primal_weight, adapt_guard = 0): the acceptance references (stopped at relative
    KKT 1e-4) come from runs on which the adaptation stop never fired, and a converged
    reference on which it fired is reproduced exactly by the run without the stop (on mid_s0
    the stop fired at k = 2610, after the last change of omega)."""
    import glob

    files = sorted(glob.glob(os.path.join(GOLDEN, "oracle_*.npz")))
    assert files
    fired = []
    for f in files:
        g = np.load(f)
        assert "omega_frozen_at" in g, f
        if "kkt1e-4" in f:
            assert int(g["omega_frozen_at"]) == -1, f
        elif int(g["omega_frozen_at"]) != -1:
            fired.append(os.path.basename(f))
    assert fired == ["oracle_mid_s0.npz"]
    inst = I.mid(0)
    g = np.load(os.path.join(GOLDEN, "oracle_mid_s0.npz"))
    r = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                eps=1e-9, stop_mode="kkt", max_iters=100000, k_check=10, adapt_guard=0)
    assert r.omega_frozen_at == -1 and r.iters == int(g["iters"])
    assert np.array_equal(r.T, g["T"]) and r.utility == float(g["utility"])


def test_warm_start_continues_the_iteration():
    """Reading of Sec. 3.1's warm start: restarting from (F^{k-1/2}, Y^k, omega) with k reset to
    0 continues the iteration exactly when the restart falls on a multiple of k_adapt (the
    primal-weight updates then land on the same iterations)."""
    inst = I.mid(1)
    args = (inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma)
    kw = dict(stop_mode="none", k_check=50, adapt_guard=0)
    straight = O.pdmcf(*args, max_iters=500, **kw)
    first = O.pdmcf(*args, max_iters=300, **kw)
    second = O.pdmcf(*args, max_iters=200, F0=first.F, Y0=first.Y, omega0=first.omega, **kw)
    assert second.omega == straight.omega
    assert np.array_equal(second.T, straight.T)
    assert np.array_equal(second.Yhat, straight.Yhat)


def test_duality_gap_bounds_the_traffic_error():
    """Log utility: u = w log s is strongly concave with modulus >= w_min / T_max^2 on the
    segment between a feasible T and the optimum T*, and U(T*) <= D (weak duality), so
    |T_ij - T*_ij| <= T_max sqrt(2 (D - U(T)) / w_min). The oracle's dual bound and its T
    must satisfy this at every stopping point; a dual bound too low would violate it."""
    inst = I.tiny(0)
    n = inst.n
    off = offdiag(n)
    Tstar = np.load(os.path.join(GOLDEN, "oracle_tiny_s0.npz"))["T"]
    wmin = inst.w[off].min()
    checked = 0
    for iters in (100, 300, 1000, 3000):
        r = solve(inst, stop_mode="none", max_iters=iters)
        if not r.metrics.feasible:
            continue
        gap = r.metrics.D - r.metrics.P
        assert gap >= -1e-12 * abs(r.metrics.D)
        tmax = max(r.T[off].max(), Tstar[off].max())
        bound = tmax * math.sqrt(2.0 * max(gap, 0.0) / wmin)
        assert np.abs(r.T[off] - Tstar[off]).max() <= bound * (1 + 1e-9) + 1e-12
        checked += 1
    assert checked >= 3
