"""PDMCF iterations of the FP64 oracle spread over all host cores (timing baseline only).

Test infrastructure, like the rest of oracle/: only the CPU-baseline leg of bench.py and the
tests use it. It performs the iterations of Algorithm 2.1 exactly as oracle.pdmcf does
(same formulas, same sort-based projection per column, same prox), but each phase is split
over worker processes that share F, Y and the scratch arrays through shared memory:

  edge phase (Eq. e-pdhg-step, Sec. 2.3): a worker owns a block of edges (columns of F):
      Q = F + alpha (Y_{:,head} - Y_{:,tail}), F^ = Pi(Q) column by column (Sec. 2.6 sort),
      F+ = 2 F^ - F, F_new = rho F^ + (1 - rho) F, its part of ||F_new - F||^2;
  node phase: a worker owns a block of destinations (rows of Y):
      V = Y - beta F+ A^T, Y^ = prox(V) (0 on the diagonal), Y_new = rho Y^ + (1 - rho) Y,
      its part of ||Y_new - Y||^2;
  then the primal weight rule of Eq. (e-primal_weight) on the summed norms.

The per-entry arithmetic is the oracle's; only the order of the sums in F+ A^T and in the two
norms differs (blocks, then their total), so the iterates agree with oracle.pdmcf to rounding.
`ParallelPDMCF.step` has the signature of oracle.pdmcf's `step` argument, so
oracle.pdmcf(..., step=pp.step) runs Algorithm 2.1 (stop test, primal weight rule and its
adaptation stop, metrics) with the updates spread over the workers; `run` performs plain
iterations for timing, the "PDMCF (CPU)" configuration of the paper's Tables 1-2.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import pdmcf as O

_W = {}   # worker state: attached shared arrays and the instance


def _attach(spec):
    shm = shared_memory.SharedMemory(name=spec[0])
    return shm, np.ndarray(spec[1], dtype=np.float64, buffer=shm.buf)


def _init(specs, inst):
    _W["shm"] = {}
    for key, spec in specs.items():
        shm, arr = _attach(spec)
        _W["shm"][key] = shm
        _W[key] = arr
    n, tail, head, cap, kind, w, gamma = inst
    _W["inst"] = (n, np.asarray(tail), np.asarray(head), np.asarray(cap, dtype=np.float64))
    _W["util"] = O.Utility(kind, w, gamma)
    # in-edges and out-edges of every node, for the rows of F+ A^T
    m = len(tail)
    order_h = np.argsort(head, kind="stable")
    order_t = np.argsort(tail, kind="stable")
    _W["in"] = (order_h, np.searchsorted(np.asarray(head)[order_h], np.arange(n + 1)))
    _W["out"] = (order_t, np.searchsorted(np.asarray(tail)[order_t], np.arange(n + 1)))
    _W["m"] = m


def _edge_block(args):
    lo, hi, src, alpha, rho = args
    n, tail, head, cap = _W["inst"]
    F = _W["F%d" % src]
    Fn = _W["F%d" % (1 - src)]
    Y = _W["Y%d" % src]
    Fp = _W["Fplus"]
    Q = F[:, lo:hi] + alpha * (Y[:, head[lo:hi]] - Y[:, tail[lo:hi]])
    Fhat, mu = O.project_capped_simplex(Q, cap[lo:hi])
    _W["Q"][:, lo:hi] = Q
    _W["Fhat"][:, lo:hi] = Fhat
    _W["mu"][0, lo:hi] = mu
    Fp[:, lo:hi] = 2.0 * Fhat - F[:, lo:hi]
    Fn[:, lo:hi] = rho * Fhat + (1.0 - rho) * F[:, lo:hi]
    d = Fn[:, lo:hi] - F[:, lo:hi]
    return float(np.sum(d * d))


def _node_block(args):
    lo, hi, src, beta, rho = args
    n = _W["inst"][0]
    Y = _W["Y%d" % src]
    Yn = _W["Y%d" % (1 - src)]
    Fp = _W["Fplus"][lo:hi]
    oi, pi = _W["in"]
    oo, po = _W["out"]
    FAt = np.zeros((hi - lo, n))
    for j in range(n):   # (F+ A^T)_{:,j} = sum_{in(j)} F+ - sum_{out(j)} F+
        FAt[:, j] = Fp[:, oi[pi[j]:pi[j + 1]]].sum(axis=1) - Fp[:, oo[po[j]:po[j + 1]]].sum(axis=1)
    V = Y[lo:hi] - beta * FAt
    util = _W["util"]
    Yhat = np.zeros_like(V)
    rows = np.arange(lo, hi)
    off = np.ones(V.shape, dtype=bool)
    off[rows - lo, rows] = False
    w = util.w[lo:hi][off]
    if util.kind == "log":
        Yhat[off] = O.prox_log(V[off], beta, w)
    else:
        Yhat[off] = O.prox_pow(V[off], beta, w, util.gamma[lo:hi][off])
    _W["Yhat"][lo:hi] = Yhat
    Yn[lo:hi] = rho * Yhat + (1.0 - rho) * Y[lo:hi]
    d = Yn[lo:hi] - Y[lo:hi]
    return float(np.sum(d * d))


class ParallelPDMCF:
    """Worker pool holding one instance. `step` is oracle.pdmcf's update step; `run(iters)`
    performs PDMCF iterations from the cold start (F = 0, Y = I - 1 1^T, omega = 1) and
    returns (F, Y, omega) afterwards. Arrays that `step` returns are views of shared memory,
    valid until the next step or `close` (copy what must outlive them)."""

    def __init__(self, inst, workers: int | None = None, rho=1.9, theta=0.5, k_adapt=100,
                 tau=1e-5):
        self.n = int(inst.n)
        self.m = int(len(inst.tail))
        self.workers = int(workers or os.cpu_count() or 1)
        self.rho, self.theta, self.k_adapt, self.tau = rho, theta, k_adapt, tau
        self.eta = O.eta_bound(self.n, inst.tail, inst.head)
        n, m = self.n, self.m
        shapes = {"F0": (n, m), "F1": (n, m), "Fplus": (n, m), "Y0": (n, n), "Y1": (n, n),
                  "Q": (n, m), "Fhat": (n, m), "mu": (1, m), "Yhat": (n, n)}
        self.cur = 0
        self._shm = {}
        specs = {}
        for key, shape in shapes.items():
            shm = shared_memory.SharedMemory(create=True, size=max(8, 8 * shape[0] * shape[1]))
            self._shm[key] = shm
            specs[key] = (shm.name, shape)
        self._arr = {k: np.ndarray(s, dtype=np.float64, buffer=self._shm[k].buf)
                     for k, s in shapes.items()}
        ctx = mp.get_context("spawn")
        payload = (n, np.asarray(inst.tail), np.asarray(inst.head), np.asarray(inst.cap),
                   inst.kind, np.asarray(inst.w), inst.gamma)
        self._pool = ctx.Pool(self.workers, initializer=_init, initargs=(specs, payload))
        step_e = max(1, -(-m // (4 * self.workers)))
        step_n = max(1, -(-n // (4 * self.workers)))
        self._eblocks = [(lo, min(m, lo + step_e)) for lo in range(0, m, step_e)]
        self._nblocks = [(lo, min(n, lo + step_n)) for lo in range(0, n, step_n)]

    def step(self, F, Y, alpha, beta, rho):
        """One update of Algorithm 2.1 step 2 from (F, Y): returns
        (Q, F^, mu, Y^, F_new, Y_new, Delta_F, Delta_Y) as oracle.pdmcf computes them."""
        a = self._arr
        src = self.cur
        if F is not a["F%d" % src]:
            a["F%d" % src][:] = F
        if Y is not a["Y%d" % src]:
            a["Y%d" % src][:] = Y
        dF2 = sum(self._pool.map(_edge_block, [(lo, hi, src, alpha, rho)
                                               for lo, hi in self._eblocks]))
        dY2 = sum(self._pool.map(_node_block, [(lo, hi, src, beta, rho)
                                               for lo, hi in self._nblocks]))
        self.cur = 1 - src
        return (a["Q"], a["Fhat"], a["mu"][0].copy(), a["Yhat"], a["F%d" % (1 - src)],
                a["Y%d" % (1 - src)], math.sqrt(dF2), math.sqrt(dY2))

    def run(self, iters: int):
        F = np.zeros((self.n, self.m))
        Y = np.eye(self.n) - np.ones((self.n, self.n))
        omega = 1.0
        for k in range(iters):
            alpha, beta = self.eta / omega, self.eta * omega
            _, _, _, _, F, Y, dF, dY = self.step(F, Y, alpha, beta, self.rho)
            if k % self.k_adapt == 0 and dF > self.tau and dY > self.tau:
                omega = (dY / dF) ** self.theta * omega ** (1.0 - self.theta)
        return F.copy(), Y.copy(), omega

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        self._arr = {}
        for shm in self._shm.values():
            try:
                shm.close()
            except BufferError:   # a caller still holds a view; the mapping ends with it
                pass
            shm.unlink()
        self._shm = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
