"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

  * trajectory parity: both run exactly K iterations of Algorithm 2.1 from the same cold
    start; T = -F^A^T, Y^ and F^ of iteration K are compared element by element (FP64 path:
    1e-8 of scale; FP32 path: 1e-4 of scale), for every kernel launch shape;
  * converged parity (the acceptance criterion): the FP32 solve stopped at relative KKT
    1e-4 against the oracle run to 1e-9: relative utility error <= 1e-4 and max relative
    error of the off-diagonal T <= 1e-3;
  * closed forms (two nodes, first iteration), warm-start continuation, determinism,
    graphs vs plain launches, async vs sync;
  * properties at full size (n = 10^4, m = 10^5, the benchmark's launch shape).
"""
import os

import numpy as np
import pytest

from oracle import pdmcf as O
from paper_2501_17996_gb300 import instances as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def off(n):
    return ~np.eye(n, dtype=bool)


def oracle_k(inst, K, k_check):
    """K oracle iterations with the stop tests (and so the adaptation stop) every k_check
    iterations, as in the GPU solve it is compared with."""
    return O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                   stop_mode="none", max_iters=K, k_check=k_check)


def rel_err(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


def rel_elem(a, b, mask, floor=1e-6):
    """Entry by entry: max |a - b| / max(|b|, floor * max|b|). Beside the of-scale measure it
    sees wrong small entries. For FP32 iterates an entry near the floor carries about
    (of-scale error) / floor of relative error from rounding alone (a T entry is a sum of F
    entries up to the capacities), so FP32 bounds on it are loose by construction."""
    a, b = a[mask], b[mask]
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor * np.abs(b).max())))


def shapes_for(lib, inst, precision):
    vw = {"fp32": 4, "fp64": 2, "bf16": 8}[precision]
    nchunks = ((inst.n + 7) // 8 * 8) // vw
    out = []
    rows = ((inst.n + 7) // 8 * 8) // 4     # kinds 1 and 2 use 4-entry chunks
    for s, (g, v, b, piped) in enumerate(lib.mcf_shape_info()):
        if g * v >= (rows if piped else nchunks) and not (precision == "fp64" and (s >= 10 or piped)):
            out.append(s)
    return out


# ------------------------------------------------------------------ trajectory parity

TRAJ_CASES = {
    "tiny": lambda: I.tiny(0),
    "mid": lambda: I.mid(0),
    "midpow": lambda: I.large(0, n=100),
    "two_node": lambda: I.two_node(1.7, 0.45),
    "pairgamma": lambda: _pair_gamma(),
}


def _pair_gamma():
    inst = I.random_small(9, 30, 5, kind="pow")
    rng = np.random.default_rng(3)
    inst.gamma = rng.uniform(0.3, 0.7, size=(inst.n, inst.n))
    return inst


@pytest.mark.parametrize("case", list(TRAJ_CASES))
def test_fp64_trajectory_matches_oracle(lib, case):
    inst = TRAJ_CASES[case]()
    K = 200
    ref = oracle_k(inst, K, 25)
    with lib.Problem(inst) as p:
        g = p.solve(precision="fp64", stop_mode="none", max_iters=K, k_check=25,
                    want_T=True, want_F=True, want_Y=True)
    m = off(inst.n)
    assert g["iters"] == K
    assert rel_err(g["T"], ref.T, m) < 1e-8
    assert rel_elem(g["T"], ref.T, m) < 1e-7        # measured <= 1.2e-9 (knn)
    assert rel_err(g["Y"], ref.Yhat, m) < 1e-8
    assert rel_err(g["F"], ref.Fhat) < 1e-8
    assert g["omega"] == pytest.approx(ref.omega, rel=1e-8)
    assert np.all(np.diag(g["Y"]) == 0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_renumbered_network_matches_oracle(lib, precision, tol):
    """A kNN network (Sec. 3.1) that the library renumbers internally: T, Y^ and F, mapped
    back to the caller's numbering, follow the oracle's trajectory."""
    inst = I.knn(400, 6, 0)
    K = 100
    ref = oracle_k(inst, K, 25)
    with lib.Problem(inst) as p:
        assert p.node_order()[0]
        g = p.solve(precision=precision, stop_mode="none", max_iters=K, k_check=25,
                    want_T=True, want_F=True, want_Y=True)
    m = off(inst.n)
    assert rel_err(g["T"], ref.T, m) < tol
    # measured: FP64 1.2e-9, FP32 2.1e-2 (entries near the floor, see rel_elem)
    assert rel_elem(g["T"], ref.T, m) < (1e-7 if precision == "fp64" else 0.1)
    assert rel_err(g["Y"], ref.Yhat, m) < tol
    assert rel_err(g["F"], ref.Fhat) < tol
    assert np.all(np.diag(g["Y"]) == 0)


def test_adaptation_stop_matches_oracle(lib):
    """The stop of the omega adaptation (Sec. 2.4) is taken on the device at the same check
    as in the oracle, and the FP64 trajectories agree past it."""
    inst = I.mid(0)
    K = 1500
    ref = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                  stop_mode="none", max_iters=K, k_check=50, adapt_guard=1.05)
    assert ref.omega_frozen_at > 0
    with lib.Problem(inst) as p:
        g = p.solve(precision="fp64", stop_mode="none", max_iters=K, k_check=50,
                    adapt_guard=1.05, want_T=True)
    m = off(inst.n)
    assert g["omega_frozen_at"] == ref.omega_frozen_at
    assert g["omega"] == pytest.approx(ref.omega, rel=1e-9)
    assert rel_err(g["T"], ref.T, m) < 1e-7


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_every_shape_matches_oracle(lib, precision):
    inst = I.mid(0) if precision == "fp32" else I.tiny(0)
    K = 30
    ref = oracle_k(inst, K, 10)
    m = off(inst.n)
    tol = 1e-4 if precision == "fp32" else 1e-9
    shapes = shapes_for(lib, inst, precision)
    assert len(shapes) >= 10
    with lib.Problem(inst) as p:
        for s in shapes:
            g = p.solve(precision=precision, stop_mode="none", max_iters=K, k_check=10,
                        shape=s, want_T=True, want_F=True, want_Y=True)
            assert rel_err(g["T"], ref.T, m) < tol, s
            # measured (automatic shape): FP32 1.1e-3, FP64 5e-14
            assert rel_elem(g["T"], ref.T, m) < (1e-2 if precision == "fp32" else 1e-7), s
            assert rel_err(g["Y"], ref.Yhat, m) < tol, s
            assert rel_err(g["F"], ref.Fhat) < tol, s


def test_slice_trajectory_fp32(lib):
    """The large recipe (power utility, gamma = 1/2, lognormal capacities) at n = 1000."""
    inst = I.large_slice(0)
    K = 12
    ref = oracle_k(inst, K, 4)
    with lib.Problem(inst) as p:
        g = p.solve(precision="fp32", stop_mode="none", max_iters=K, k_check=4,
                    want_T=True, want_Y=True)
    m = off(inst.n)
    assert rel_err(g["T"], ref.T, m) < 1e-4
    assert rel_elem(g["T"], ref.T, m) < 0.1   # measured 4.3e-2: early T has many tiny entries
    assert rel_err(g["Y"], ref.Yhat, m) < 1e-4


def test_slice_pipelined_shapes_fp32(lib):
    """Every bulk-copy pipelined and in-sum edge-phase shape on the n = 1000 slice: head
    groups of several edges, head-aligned CTA ranges, in-sums consumed by the node phase."""
    inst = I.large_slice(1)
    K = 6
    ref = oracle_k(inst, K, 3)
    m = off(inst.n)
    piped = [s for s, (g, v, b, t) in enumerate(lib.mcf_shape_info()) if t]
    assert piped
    with lib.Problem(inst) as p:
        for s in piped:
            g = p.solve(precision="fp32", stop_mode="none", max_iters=K, k_check=3, shape=s,
                        want_T=True, want_Y=True)
            assert rel_err(g["T"], ref.T, m) < 1e-4, s
            assert rel_err(g["Y"], ref.Yhat, m) < 1e-4, s


def _hub_network(n=2000, seed=0):
    """A ring in both directions plus edges from every other node to node 0 and back: node 0
    has in-degree n - 1, so the head-aligned CTA ranges of kinds 1 and 2 hold the hub's in-edges
    in one range and most CTAs get an empty range."""
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    j = np.arange(2, n - 1)              # ring neighbours of node 0 are linked already
    zero = np.zeros(j.size, dtype=np.int64)
    tail = np.concatenate([i, (i + 1) % n, j, zero])
    head = np.concatenate([(i + 1) % n, i, zero, j])
    cap = rng.lognormal(0.0, 0.5, size=tail.size)
    w = rng.uniform(0.5, 1.5, size=(n, n))
    np.fill_diagonal(w, 0.0)
    return I.Instance(n, tail.astype(np.int32), head.astype(np.int32), cap, "pow", w, 0.5, "hub")


def test_hub_network_pipelined_shapes_fp32(lib):
    """Every bulk-copy pipelined and in-sum shape on a network with one node of in-degree
    n + 1 (one long head group, empty CTA ranges) against the oracle."""
    inst = _hub_network()
    K = 6
    ref = oracle_k(inst, K, 3)
    m = off(inst.n)
    piped = [s for s, (g, v, b, t) in enumerate(lib.mcf_shape_info())
             if t and g * v >= ((inst.n + 7) // 8 * 8) // 4]
    assert piped
    with lib.Problem(inst) as p:
        for s in piped:
            g = p.solve(precision="fp32", stop_mode="none", max_iters=K, k_check=3, shape=s,
                        want_T=True, want_Y=True)
            assert rel_err(g["T"], ref.T, m) < 1e-4, s
            assert rel_err(g["Y"], ref.Yhat, m) < 1e-4, s


def test_bf16_storage_every_shape_short_trajectory(lib):
    """F stored as BF16 (8-bit mantissa) for every shape, 3 iterations: each stored F value
    is rounded, so the bound is 1e-2 of scale; indexing mistakes give O(1) errors."""
    inst = I.mid(0)
    K = 3
    ref = oracle_k(inst, K, K)
    m = off(inst.n)
    shapes = shapes_for(lib, inst, "bf16")
    with lib.Problem(inst) as p:
        for s in shapes:
            g = p.solve(precision="bf16", stop_mode="none", max_iters=K, k_check=K, shape=s,
                        want_T=True, want_Y=True)
            assert rel_err(g["T"], ref.T, m) < 1e-2, s
            assert rel_err(g["Y"], ref.Yhat, m) < 1e-2, s


# ------------------------------------------------------------------ converged parity

INSTANCES = {"tiny_s0": lambda: I.tiny(0), "mid_s0": lambda: I.mid(0),
             "midpow_s0": lambda: I.large(0, n=100)}


@pytest.mark.parametrize("name,precision,tol", [("tiny_s0", "fp64", 1e-6),
                                                ("mid_s0", "fp32", 1e-4),
                                                ("midpow_s0", "fp32", 1e-4)])
def test_converged_matches_oracle(lib, name, precision, tol):
    """The acceptance criterion: both sides stopped at relative KKT <= 1e-4 (stop test every
    50 iterations), utility within 1e-4 of the converged optimum and T within 1e-3
    max-relative of the oracle's T stopped the same way. (The oracle's own T at that stop is
    up to 8e-4 from T*, so T* itself is checked at a tighter stop below.)"""
    gold = np.load(os.path.join(GOLDEN, f"oracle_{name}.npz"))
    same = os.path.join(GOLDEN, f"oracle_{name}_kkt1e-4.npz")
    inst = INSTANCES[name]()
    with lib.Problem(inst) as p:
        g = p.solve(precision=precision, stop_mode="kkt", eps=tol, max_iters=200000,
                    k_check=50, want_T=True, want_Y=True)
    assert g["rc"] == lib.MCF_OK and g["rel_kkt"] < tol
    m = off(inst.n)
    Tstar = gold["T"]
    Tref = np.load(same)["T"] if tol == 1e-4 else Tstar
    assert abs(g["utility"] - float(gold["utility"])) <= 1e-4 * abs(float(gold["utility"]))
    assert np.max(np.abs(g["T"][m] - Tref[m]) / Tref[m]) <= 1e-3
    assert np.allclose(g["T"].sum(axis=1), 0, atol=1e-4 * np.abs(Tstar).max())
    assert g["feasible"] == 1 and g["rel_gap"] >= -1e-6
    assert g["utility"] <= g["dual_bound"] + 1e-6 * abs(g["dual_bound"])


@pytest.mark.parametrize("name", ["mid_s0", "midpow_s0"])
def test_fp32_tighter_stop_matches_optimum(lib, name):
    """FP32 iterates run to relative KKT 5e-5: T within 1e-3 max-relative of the converged
    optimum T* (the FP64 oracle at this stop is within 5.4e-4 of T* on these instances)."""
    gold = np.load(os.path.join(GOLDEN, f"oracle_{name}.npz"))
    inst = INSTANCES[name]()
    with lib.Problem(inst) as p:
        g = p.solve(stop_mode="kkt", eps=5e-5, max_iters=200000, k_check=50, want_T=True)
    assert g["rc"] == lib.MCF_OK and g["rel_kkt"] < 5e-5
    m = off(inst.n)
    assert np.max(np.abs(g["T"][m] - gold["T"][m]) / gold["T"][m]) <= 1e-3
    assert abs(g["utility"] - float(gold["utility"])) <= 1e-4 * abs(float(gold["utility"]))


@pytest.mark.parametrize("name", ["mid_s0", "midpow_s0"])
def test_bf16_with_fp32_polish_matches_oracle(lib, name):
    """BF16-stored F until close to the target, then FP32 polish: the same acceptance
    criterion as the FP32 path."""
    gold = np.load(os.path.join(GOLDEN, f"oracle_{name}.npz"))
    inst = {"mid_s0": lambda: I.mid(0), "midpow_s0": lambda: I.large(0, n=100)}[name]()
    with lib.Problem(inst) as p:
        g = p.solve(precision="bf16", polish_iters=100000, stop_mode="kkt", eps=1e-4,
                    max_iters=200000, k_check=50, want_T=True)
    assert g["rc"] == lib.MCF_OK and g["rel_kkt"] < 1e-4
    m = off(inst.n)
    Tref = np.load(os.path.join(GOLDEN, f"oracle_{name}_kkt1e-4.npz"))["T"]
    assert abs(g["utility"] - float(gold["utility"])) <= 1e-4 * abs(float(gold["utility"]))
    assert np.max(np.abs(g["T"][m] - Tref[m]) / Tref[m]) <= 1e-3


# ------------------------------------------------------------------ closed forms and edges

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_node_closed_form(lib, precision):
    ca, cb = 1.7, 0.45
    inst = I.two_node(ca, cb, "log", w12=0.8, w21=1.3)
    with lib.Problem(inst) as p:
        g = p.solve(precision=precision, stop_mode="kkt", eps=1e-6, max_iters=20000,
                    want_T=True, want_Y=True)
    tol = 1e-5 if precision == "fp32" else 1e-9
    assert g["T"][1, 0] == pytest.approx(ca, rel=tol)
    assert g["T"][0, 1] == pytest.approx(cb, rel=tol)
    assert g["Y"][1, 0] == pytest.approx(-1.3 / ca, rel=10 * tol)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_first_iteration_closed_form(lib, precision):
    """From the cold start, F^{1/2} = alpha e_head per edge (alpha <= c_l), hence
    T_ij = alpha if the edge j -> i exists, 0 otherwise, T_ii = -alpha indeg(i)."""
    inst = I.mid(1)
    alpha = O.eta_bound(inst.n, inst.tail, inst.head)
    assert np.all(alpha <= inst.cap)
    Tref = np.zeros((inst.n, inst.n))
    Tref[inst.head, inst.tail] = alpha
    np.fill_diagonal(Tref, -alpha * np.bincount(inst.head, minlength=inst.n))
    with lib.Problem(inst) as p:
        g = p.solve(precision=precision, stop_mode="none", max_iters=1, want_T=True)
    tol = 1e-6 if precision == "fp32" else 1e-14
    assert np.abs(g["T"] - Tref).max() <= tol * alpha * 20
    assert g["feasible"] == 0 and g["nonpos_frac"] > 0


def test_warm_start_continues_the_iteration(lib):
    """Solving 100 iterations and then 60 warm-started ones equals 160 cold iterations
    (k restarts at 0 on a warm start, and 100 is a multiple of k_adapt)."""
    inst = I.mid(0)
    with lib.Problem(inst) as p:
        a = p.solve(precision="fp64", stop_mode="none", max_iters=160, want_T=True, want_Y=True)
        p.solve(precision="fp64", stop_mode="none", max_iters=100)
        b = p.solve(precision="fp64", stop_mode="none", max_iters=60, warm_start=1,
                    want_T=True, want_Y=True)
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["Y"], b["Y"])


def test_deterministic_and_graphs_equal_plain_launches(lib):
    inst = I.mid(2)
    with lib.Problem(inst) as p:
        r1 = p.solve(stop_mode="none", max_iters=150, k_check=50, want_T=True, want_Y=True)
        r2 = p.solve(stop_mode="none", max_iters=150, k_check=50, want_T=True, want_Y=True)
        r3 = p.solve(stop_mode="none", max_iters=150, k_check=50, use_graphs=0,
                     want_T=True, want_Y=True)
    for key in ("T", "Y"):
        assert np.array_equal(r1[key], r2[key])
        assert np.array_equal(r1[key], r3[key])
    assert r1["rel_kkt"] == r2["rel_kkt"] == r3["rel_kkt"]


def test_async_matches_batched_and_sync(lib):
    """Submitted requests run in the continuous-batching engine: identical to the same
    problems solved by mcf_solve_batch, and within FP32 tolerance of mcf_solve."""
    insts = [I.mid(s) for s in range(3)] + [I.tiny(1)]
    probs = [lib.Problem(inst) for inst in insts]
    opts = dict(stop_mode="kkt", eps=1e-4)
    sync = [p.solve(want_T=True, **opts) for p in probs]
    _, batched = lib.mcf_solve_batch(probs, lib.mcf_options_default(**opts), want_T=True)
    tickets = [p.submit(**opts) for p in probs]
    for t, p, s, b in zip(tickets, probs, sync, batched):
        r = lib.mcf_wait(t, 120000, p.n, p.m, want_T=True)
        assert r is not None and r["status"] == lib.MCF_OK
        assert r["iters"] == b["iters"]
        assert np.array_equal(r["T"], b["T"])
        m = off(p.n)
        assert np.abs(r["T"][m] - s["T"][m]).max() <= 1e-3 * np.abs(s["T"][m]).max()
    for p in probs:
        p.close()


def test_capacity_update_warm_resolve(lib):
    inst = I.mid(3)
    rng = np.random.default_rng(0)
    pert = I.perturb(inst, 0.1, "cap", rng)
    ref = O.pdmcf(pert.n, pert.tail, pert.head, pert.cap, pert.kind, pert.w, eps=1e-8,
                  stop_mode="kkt", max_iters=100000, k_check=10)
    with lib.Problem(inst) as p:
        cold = p.solve(stop_mode="kkt", eps=1e-4)
        p.update_capacities(pert.cap)
        warm = p.solve(stop_mode="kkt", eps=1e-4, warm_start=1, want_T=True)
    assert warm["rc"] == lib.MCF_OK
    assert abs(warm["utility"] - ref.utility) <= 1e-4 * abs(ref.utility)
    assert cold["iters"] > 0


# ------------------------------------------------------------------ full size

def test_large_properties_at_full_size(lib):
    """n = 10^4, m = 10^5 (power utility, gamma = 1/2) in the benchmark's launch shape:
    the first-iteration closed form, then certificates after 300 iterations."""
    inst = I.large(0)
    n = inst.n
    alpha = O.eta_bound(n, inst.tail, inst.head)
    rows = np.random.default_rng(0).choice(n, size=64, replace=False)
    with lib.Problem(inst) as p:
        g = p.solve(stop_mode="none", max_iters=1, want_T=True)
        T = g["T"]
        for i in rows:
            ref = np.zeros(n)
            ref[inst.tail[inst.head == i]] = alpha
            ref[i] = -alpha * np.sum(inst.head == i)
            assert np.abs(T[i] - ref).max() <= 1e-6 * alpha * 40
        g = p.solve(stop_mode="none", max_iters=300, k_check=100, want_T=True, want_Y=True)
    T, Y = g["T"], g["Y"]
    assert np.all(np.diag(Y) == 0)
    assert np.all(Y[off(n)] < 0)
    assert np.abs(T[rows].sum(axis=1)).max() <= 1e-4 * np.abs(T[rows]).max()
    if g["feasible"]:
        assert g["utility"] <= g["dual_bound"] * (1 + 1e-6)
    assert np.isfinite(g["rel_cons"])


# ------------------------------------------------------------------ precision features

def test_compensated_duals_lower_the_fp32_floor(lib):
    """On a low-degree network FP32 duals stall near 1e-4 relative KKT; the FP32 head +
    BF16 tail representation reaches a lower floor and a more accurate T."""
    inst = sorted(I.batched(seed=3, count=8), key=lambda i: i.n * i.m)[0]
    ref = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                  eps=1e-10, stop_mode="kkt", max_iters=100000, k_check=100)
    m = off(inst.n)
    out = {}
    with lib.Problem(inst) as p:
        for comp in (0, 1):
            g = p.solve(stop_mode="none", max_iters=8000, k_check=500, compensated_duals=comp,
                        want_T=True)
            out[comp] = (g["rel_kkt"], np.max(np.abs(g["T"][m] - ref.T[m]) / ref.T[m]))
    assert out[1][0] < 0.6 * out[0][0]
    assert out[1][1] < out[0][1]
    assert out[1][0] < 1e-4 and out[1][1] < 1e-4


def test_autotune_picks_a_working_shape(lib):
    inst = I.mid(0)
    with lib.Problem(inst) as p:
        shape, ms = p.autotune(stop_mode="none")
        shapes = lib.mcf_shape_info()
        assert 0 <= shape < len(shapes) and ms > 0
        g = p.solve(stop_mode="none", max_iters=30, k_check=10, shape=shape, want_T=True)
    ref = oracle_k(inst, 30, 10)
    assert rel_err(g["T"], ref.T, off(inst.n)) < 1e-4
