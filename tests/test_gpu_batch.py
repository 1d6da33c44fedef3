"""Batched engine (mcf_solve_batch): many uneven instances advanced by one launch per phase.

  * a problem's iterates are bit-identical alone and inside any batch (per-item FP64
    partials summed in a fixed order by the problem's own scalar block);
  * short trajectories match the FP64 oracle to FP32 accuracy;
  * converged results inside a mixed batch meet the acceptance criterion against the oracle;
  * warm re-solves after a capacity change take fewer iterations than a cold solve.
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


def mixed_instances():
    return I.batched(seed=3, count=8)


def test_alone_equals_in_mix(lib):
    insts = mixed_instances()
    probs = [lib.Problem(i) for i in insts]
    opts = lib.mcf_options_default(stop_mode="none", max_iters=120, k_check=40)
    _, mix = lib.mcf_solve_batch(probs, opts, want_T=True, want_Y=True)
    for k in (0, 3, 7):
        _, alone = lib.mcf_solve_batch([probs[k]], opts, want_T=True, want_Y=True)
        assert np.array_equal(alone[0]["T"], mix[k]["T"])
        assert np.array_equal(alone[0]["Y"], mix[k]["Y"])
        assert alone[0]["omega"] == mix[k]["omega"]
    for p in probs:
        p.close()


def test_batch_trajectories_match_oracle(lib):
    insts = mixed_instances()[:5]
    K = 30
    probs = [lib.Problem(i) for i in insts]
    opts = lib.mcf_options_default(stop_mode="none", max_iters=K, k_check=10)
    _, res = lib.mcf_solve_batch(probs, opts, want_T=True, want_Y=True)
    for inst, r in zip(insts, res):
        ref = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                      stop_mode="none", max_iters=K, k_check=10)
        m = off(inst.n)
        assert r["iters"] == K
        scale = np.abs(ref.T[m]).max()
        assert np.abs(r["T"][m] - ref.T[m]).max() / scale < 1e-4
        assert np.abs(r["Y"][m] - ref.Yhat[m]).max() / np.abs(ref.Yhat[m]).max() < 1e-4
    for p in probs:
        p.close()


def test_batch_converged_matches_oracle(lib):
    gold = {n: np.load(os.path.join(GOLDEN, f"oracle_{n}.npz")) for n in ("mid_s0", "midpow_s0")}
    insts = [I.mid(0), I.large(0, n=100)] + mixed_instances()[:6]
    probs = [lib.Problem(i) for i in insts]
    opts = lib.mcf_options_default(stop_mode="kkt", eps=1e-4, max_iters=200000, k_check=50)
    rc, res = lib.mcf_solve_batch(probs, opts, want_T=True)
    # FP32 iterates either meet 1e-4 or end at their rounding floor (stall rule) close to it
    for r in res:
        assert (r["status"] == lib.MCF_OK and r["rel_kkt"] < 1e-4) or \
            (r["stalled"] == 1 and r["rel_kkt"] < 5e-4)
    # the acceptance criterion: utility within 1e-4 of the optimum, T within 1e-3 of the
    # oracle's T stopped the same way (relative KKT 1e-4, stop test every 50 iterations)
    for name, r, inst in (("mid_s0", res[0], insts[0]), ("midpow_s0", res[1], insts[1])):
        g = gold[name]
        Tref = np.load(os.path.join(GOLDEN, f"oracle_{name}_kkt1e-4.npz"))["T"]
        m = off(inst.n)
        assert abs(r["utility"] - float(g["utility"])) <= 1e-4 * abs(float(g["utility"]))
        assert np.max(np.abs(r["T"][m] - Tref[m]) / Tref[m]) <= 1e-3
    for p in probs:
        p.close()


def test_batch_warm_resolve_after_capacity_change(lib):
    insts = mixed_instances()[:4]
    probs = [lib.Problem(i) for i in insts]
    opts = lib.mcf_options_default(stop_mode="kkt", eps=1e-4, max_iters=200000, k_check=50)
    _, cold = lib.mcf_solve_batch(probs, opts)
    rng = np.random.default_rng(0)
    for p, inst in zip(probs, insts):
        p.update_capacities(I.perturb(inst, 0.1, "cap", rng).cap)
    wopts = lib.mcf_options_default(stop_mode="kkt", eps=1e-4, max_iters=200000, k_check=50,
                                    warm_start=1)
    rc, warm = lib.mcf_solve_batch(probs, wopts)
    assert all(w["status"] == lib.MCF_OK or w["stalled"] == 1 for w in warm)
    assert sum(w["iters"] for w in warm) < sum(c["iters"] for c in cold)
    for p in probs:
        p.close()


def test_served_requests_alone_equal_in_mix(lib):
    """Continuous batching: requests submitted together (they overlap on the device and
    join the running batch) give the same result as each request served alone."""
    insts = I.batched(seed=9, count=10)
    probs = [lib.Problem(i) for i in insts]
    opts = dict(stop_mode="kkt", eps=1e-4, k_check=50)
    alone = []
    for p in probs:
        t = p.submit(**opts)
        alone.append(lib.mcf_wait(t, 300000, p.n, p.m, want_T=True))
    # cold again, all in flight at once
    tickets = [p.submit(**opts) for p in probs]
    for t, p, a in zip(tickets, probs, alone):
        r = lib.mcf_wait(t, 300000, p.n, p.m, want_T=True)
        assert r["status"] == a["status"] and r["stalled"] == a["stalled"]
        assert r["iters"] == a["iters"]
        assert np.array_equal(r["T"], a["T"])
    for p in probs:
        p.close()


def test_served_budget_rejects_oversized_request(lib):
    inst = I.mid(0)
    with lib.Problem(inst) as p:
        lib.mcf_serving_config(1000, 16)
        try:
            with pytest.raises(lib.MCFError) as ei:
                p.submit(stop_mode="kkt", eps=1e-4)
            assert ei.value.code == lib.MCF_ERR_OOM_BUDGET
        finally:
            lib.mcf_serving_config(120 * 10**9, 256)


def test_batch_autotuned_classes_keep_alone_equal_in_mix(lib):
    """The autotuned shape of a size class is fixed once per process, so alone-vs-mix
    identity holds with autotuning on (and results match the untuned run within FP32)."""
    insts = I.batched(seed=11, count=6)
    probs = [lib.Problem(i) for i in insts]
    opts = lib.mcf_options_default(stop_mode="none", max_iters=100, k_check=50, autotune=1)
    _, mix = lib.mcf_solve_batch(probs, opts, want_T=True)
    _, alone = lib.mcf_solve_batch([probs[2]], opts, want_T=True)
    assert np.array_equal(alone[0]["T"], mix[2]["T"])
    plain = lib.mcf_options_default(stop_mode="none", max_iters=100, k_check=50, autotune=0)
    _, untuned = lib.mcf_solve_batch(probs, plain, want_T=True)
    for a, b, inst in zip(mix, untuned, insts):
        m = off(inst.n)
        assert np.abs(a["T"][m] - b["T"][m]).max() <= 1e-4 * np.abs(b["T"][m]).max()
    for p in probs:
        p.close()


def test_served_ticket_outputs_are_its_own(lib):
    """A finished ticket's T is read when it is collected; a second submission on the same
    problem is refused until then, so back-to-back requests each return their own solve."""
    inst = I.batched(seed=5, count=1)[0]
    opts = dict(stop_mode="none", k_check=50)
    with lib.Problem(inst) as p:
        _, (ref100,) = lib.mcf_solve_batch([p], lib.mcf_options_default(max_iters=100, **opts),
                                           want_T=True)
        _, (ref300,) = lib.mcf_solve_batch([p], lib.mcf_options_default(max_iters=300, **opts),
                                           want_T=True)
        t1 = p.submit(max_iters=100, **opts)
        with pytest.raises(lib.MCFError) as ei:
            p.submit(max_iters=300, **opts)
        assert ei.value.code == lib.MCF_ERR_BUSY
        r1 = lib.mcf_wait(t1, 120000, p.n, p.m, want_T=True)
        t2 = p.submit(max_iters=300, **opts)
        r2 = lib.mcf_wait(t2, 120000, p.n, p.m, want_T=True)
        assert r1["iters"] == 100 and r2["iters"] == 300
        m = off(inst.n)
        scale = np.abs(ref300["T"][m]).max()
        assert np.abs(ref300["T"][m] - ref100["T"][m]).max() > 1e-3 * scale   # distinct results
        assert np.abs(r1["T"][m] - ref100["T"][m]).max() <= 1e-6 * scale
        assert np.abs(r2["T"][m] - ref300["T"][m]).max() <= 1e-6 * scale


def test_served_cancel_stops_a_running_ticket(lib):
    """mcf_cancel on a started batched ticket releases its slot at the next chunk boundary
    instead of letting it run to max_iters; the problem then takes new work."""
    import time

    inst = I.served_network(1000, seed=1)
    with lib.Problem(inst) as p:
        t = p.submit(stop_mode="none", max_iters=10**7, k_check=50)
        time.sleep(0.5)
        lib.mcf_cancel(t)
        r = lib.mcf_wait(t, 30000)
        assert r is not None, "a cancelled running ticket did not finish"
        assert r["status"] == lib.MCF_ERR_CANCELLED
        t2 = p.submit(stop_mode="none", max_iters=20, k_check=10)
        r2 = lib.mcf_wait(t2, 60000)
        assert r2["status"] == lib.MCF_OK and r2["iters"] == 20


def test_serving_shutdown_with_running_and_queued_tickets(lib):
    """Shutdown ends every unfinished ticket with MCF_ERR_CANCELLED (running ones after the
    chunk in progress) and the scheduler restarts on the next submission."""
    insts = I.batched(seed=13, count=4)
    probs = [lib.Problem(i) for i in insts]
    tickets = [p.submit(stop_mode="none", max_iters=10**7, k_check=50) for p in probs]
    import time

    time.sleep(0.3)
    lib.mcf_serving_shutdown()
    for t in tickets:
        r = lib.mcf_wait(t, 30000)
        assert r is not None and r["status"] == lib.MCF_ERR_CANCELLED
    t = probs[0].submit(stop_mode="none", max_iters=20, k_check=10)
    assert lib.mcf_wait(t, 60000)["status"] == lib.MCF_OK
    for p in probs:
        p.close()
