"""Host-side rules of the serving scheduler (mcf_submit / mcf_poll / mcf_wait / mcf_cancel /
mcf_serving_config / mcf_serving_shutdown), checked without running a solve: admission is
paused (max_resident = 0), so every ticket stays queued until it is cancelled or the
scheduler shuts down. Runs with or without a GPU."""
import pytest

from paper_2501_17996_gb300 import instances as I


@pytest.fixture()
def paused(lib):
    lib.mcf_serving_config(120 * 10**9, 0)
    try:
        yield lib
    finally:
        lib.mcf_serving_shutdown()
        lib.mcf_serving_config(120 * 10**9, 256)


def _busy(lib, fn, *a, **k):
    with pytest.raises(lib.MCFError) as ei:
        fn(*a, **k)
    assert ei.value.code == lib.MCF_ERR_BUSY, ei.value
    assert "outstanding ticket" in lib.mcf_last_error()


def test_one_outstanding_ticket_per_problem(paused):
    lib = paused
    inst = I.tiny(0)
    p = lib.Problem(inst)
    t = p.submit(precision="fp32")
    assert lib.mcf_poll(t) is None                       # queued: admission is paused
    _busy(lib, p.submit, precision="fp32")               # a second ticket on the same problem
    _busy(lib, p.solve)                                  # and every call that touches its state
    _busy(lib, p.update_capacities, inst.cap)
    _busy(lib, p.update_weights, inst.w)
    _busy(lib, lib.mcf_destroy_problem, p.h)
    _busy(lib, lib.mcf_solve_batch, [p], lib.mcf_options_default())
    lib.mcf_cancel(t)                                    # queued: cancelled at once
    r = lib.mcf_wait(t, 1000)
    assert r is not None and r["status"] == lib.MCF_ERR_CANCELLED
    with pytest.raises(lib.MCFError):                    # collected: the id is gone
        lib.mcf_poll(t)
    t2 = p.submit(precision="fp32")                      # the problem takes work again
    lib.mcf_cancel(t2)
    lib.mcf_cancel(t2)                                   # finished, not collected: discarded
    with pytest.raises(lib.MCFError):
        lib.mcf_poll(t2)
    p.close()


def test_shutdown_finishes_every_queued_ticket(paused):
    lib = paused
    probs = [lib.Problem(I.tiny(s)) for s in range(3)]
    tickets = [probs[0].submit(precision="fp32"),        # batched queue
               probs[1].submit(precision="fp64"),        # one-at-a-time queue
               probs[2].submit(precision="fp32", shape=0)]
    assert all(lib.mcf_poll(t) is None for t in tickets)
    lib.mcf_serving_shutdown()
    for t in tickets:
        r = lib.mcf_wait(t, 2000)
        assert r is not None, "a queued ticket was left pending by the shutdown"
        assert r["status"] == lib.MCF_ERR_CANCELLED
    for p in probs:                                      # collected: destroy is allowed
        p.close()
    # the scheduler restarts on the next submission
    q = lib.Problem(I.tiny(0))
    t = q.submit(precision="fp32")
    assert lib.mcf_poll(t) is None
    lib.mcf_serving_shutdown()
    assert lib.mcf_wait(t, 2000)["status"] == lib.MCF_ERR_CANCELLED
    q.close()


def test_serving_config_validation(lib):
    for bad in [(0, 4), (10**9, -1)]:
        with pytest.raises(lib.MCFError) as ei:
            lib.mcf_serving_config(*bad)
        assert ei.value.code == lib.MCF_ERR_INVALID
