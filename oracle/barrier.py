"""Independent log-barrier Newton solver for the compact MCF problem (test infrastructure).

Solves Eq. (e-compact-prob) of Zhang & Boyd,
    maximize U(-F A^T)  subject to  F >= 0,  F^T 1 <= c,
for tiny networks (n m up to a few hundred variables) by the textbook barrier method:
minimise  t (-U(-F A^T)) - sum log F_il - sum_l log(c_l - 1^T f_l)  for increasing t,
each by damped Newton with a dense Hessian. It shares no arithmetic with pdmcf.py (no
projection, no prox, no PDHG) and exists only to pin that file's fixed point.
"""
from __future__ import annotations

import math

import numpy as np

from .pdmcf import incidence, shortest_path_flow


def _util_derivs(kind, w, gamma, T, off):
    """u, u', u'' entrywise on off-diagonal entries (zero elsewhere)."""
    u = np.zeros_like(T)
    d1 = np.zeros_like(T)
    d2 = np.zeros_like(T)
    t = T[off]
    ww = w[off]
    if kind == "log":
        u[off] = ww * np.log(t)
        d1[off] = ww / t
        d2[off] = -ww / (t * t)
    else:
        g = gamma[off]
        u[off] = ww * t ** g
        d1[off] = ww * g * t ** (g - 1.0)
        d2[off] = ww * g * (g - 1.0) * t ** (g - 2.0)
    return u, d1, d2


def solve(n, tail, head, cap, kind, w, gamma=None, t_final=1e13, mu_factor=10.0,
          newton_tol=1e-14, max_newton=200):
    """Returns (F, T, U) at the end of the barrier path (t = t_final)."""
    tail = np.asarray(tail)
    head = np.asarray(head)
    c = np.asarray(cap, dtype=np.float64)
    m = tail.shape[0]
    A = incidence(n, tail, head).toarray()
    w = np.asarray(w, dtype=np.float64)
    off = ~np.eye(n, dtype=bool)
    if kind == "pow":
        g = np.asarray(gamma, dtype=np.float64)
        gamma = np.broadcast_to(g, (n, n)).copy() if g.ndim == 0 else g
    # strictly feasible start: half the shortest-path flow plus a small uniform flow
    Fsp, a_sp = shortest_path_flow(n, tail, head, c)
    imbalance = np.abs(A.sum(axis=1)).max()
    delta = min(0.25 * a_sp / (imbalance + 1.0), 0.25 * c.min() / n)
    F = 0.5 * Fsp + delta

    def parts(F):
        T = -F @ A.T
        s = c - F.sum(axis=0)
        return T, s

    def phi(F, t):
        T, s = parts(F)
        if np.any(F <= 0) or np.any(s <= 0) or np.any(T[off] <= 0):
            return math.inf
        u, _, _ = _util_derivs(kind, w, gamma, T, off)
        return -t * u.sum() - np.log(F).sum() - np.log(s).sum()

    t = 1.0
    N = n * m
    while True:
        for _ in range(max_newton):
            T, s = parts(F)
            _, d1, d2 = _util_derivs(kind, w, gamma, T, off)
            # gradient of t(-U) wrt F_il is t (U' A)_il; Hessian block i is t A^T diag(-u''_i) A
            grad = t * (d1 @ A) - 1.0 / F + (1.0 / s)[None, :]
            H = np.zeros((N, N))
            for i in range(n):
                blk = t * (A.T * (-d2[i])[None, :]) @ A
                H[i * m:(i + 1) * m, i * m:(i + 1) * m] += blk
            H[np.diag_indices(N)] += (1.0 / F ** 2).ravel()
            cs = 1.0 / s ** 2
            for l in range(m):
                idx = np.arange(n) * m + l
                H[np.ix_(idx, idx)] += cs[l]
            gvec = grad.ravel()
            dx = -np.linalg.solve(H, gvec)
            lam2 = -float(gvec @ dx)
            if lam2 / 2.0 <= newton_tol:
                break
            step = 1.0
            f0 = phi(F, t)
            D = dx.reshape(n, m)
            while step > 1e-20:
                Fn = F + step * D
                fn = phi(Fn, t)
                if fn <= f0 - 0.25 * step * lam2:
                    break
                step *= 0.5
            F = Fn
        if t >= t_final:
            break
        t = min(t * mu_factor, t_final)
    T, _ = parts(F)
    u, _, _ = _util_derivs(kind, w, gamma, T, off)
    return F, T, float(u.sum())
