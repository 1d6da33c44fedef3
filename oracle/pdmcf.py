"""PDMCF in float64 on the CPU, written from the paper (test infrastructure only).

Zhang & Boyd, "Solving Large Multicommodity Network Flow Problems on GPUs":
  Sec. 1.1  problem (Eq. e-prob), incidence A, traffic T = -F A^T, utilities
  Sec. 1.2  optimality residual r(Q) (Eq. e-res)
  Sec. 2.1  reduced Lagrangian (Eq. e-L)
  Sec. 2.2  PDHG with over-relaxation (Eq. e-pdhg-step)
  Sec. 2.3  projection onto the capped simplex, log and power proxes
  Sec. 2.4  adaptive primal weight (Eq. e-primal_weight), eta = 1/sqrt(2 d_max) (Eq. e-eta)
  Sec. 2.5  Algorithm 2.1 (PDMCF), initialisation and stopping criterion
  Sec. 2.6  sort-based projection (Held et al.)

Notation follows the paper: F is n x m (row i = destination, column l = edge), Y and T
are n x n with T[i, j] the traffic from source j to destination i.

Readings where the paper is silent (each also listed in the design notes):
  * "k is a multiple of k_adapt" includes k = 0.
  * the stopping test may be evaluated only every ``k_check`` iterations (k_check = 1 is
    the paper's every-iteration test); the residual is then computed at iteration k-1
    for the test at iteration k, as in Sec. 2.5.
  * the relative KKT measure (not defined in the paper) is
        rel_kkt = max(rel_gap, rel_cons, rel_stat) evaluated at (F^, Y^), with
        rel_gap  = (D - P) / (1 + |P| + |D|),  P = U(T^),
                   D = sum_{i!=j} (-u_ij)^*(Y^_ij) + sum_l c_l max(0, max_i (Y^ A)_il),
        rel_cons = ||T(Y^) - T^||_F / (1 + ||T^||_F) over off-diagonal entries, where
                   T(Y^)_ij = (u_ij')^{-1}(-Y^_ij),
        rel_stat = sqrt(r) / (1 + ||G||_F).
    D is the dual function of the reduced Lagrangian (Eq. e-L): weak duality gives
    P <= U* <= D, so rel_gap >= 0 whenever T^ is in the domain.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------- network

def incidence(n: int, tail, head) -> sp.csr_matrix:
    """Incidence matrix of Sec. 1.1: A[i, l] = +1 if edge l enters i, -1 if it leaves i."""
    tail = np.asarray(tail, dtype=np.int64)
    head = np.asarray(head, dtype=np.int64)
    m = tail.shape[0]
    rows = np.concatenate([head, tail])
    cols = np.concatenate([np.arange(m), np.arange(m)])
    vals = np.concatenate([np.ones(m), -np.ones(m)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, m))


def eta_bound(n: int, tail, head) -> float:
    """Eq. (e-eta): eta = 1/sqrt(2 d_max), d_i = (A A^T)_ii = in-degree + out-degree."""
    d = np.zeros(n, dtype=np.int64)
    np.add.at(d, np.asarray(tail, dtype=np.int64), 1)
    np.add.at(d, np.asarray(head, dtype=np.int64), 1)
    return 1.0 / math.sqrt(2.0 * float(d.max()))


# --------------------------------------------------------------------------- utilities

class Utility:
    """Weighted log (u = w log s) or power (u = w s^gamma) utilities, Sec. 1.1.

    ``w[i, j]`` weights traffic j -> i; the diagonal has u_ii = 0.
    """

    def __init__(self, kind: str, w, gamma=None):
        if kind not in ("log", "pow"):
            raise ValueError(kind)
        self.kind = kind
        self.w = np.asarray(w, dtype=np.float64)
        n = self.w.shape[0]
        self.n = n
        self.off = ~np.eye(n, dtype=bool)
        if kind == "pow":
            g = np.asarray(gamma, dtype=np.float64)
            self.gamma = np.broadcast_to(g, (n, n)).copy() if g.ndim == 0 else g.copy()
        else:
            self.gamma = None

    # u_ij(s) summed over i != j  (Sec. 1.1, U(T) = sum_{i,j} u_ij(T_ij) with u_ii = 0)
    def value(self, T) -> float:
        t = T[self.off]
        w = self.w[self.off]
        if self.kind == "log":
            return float(np.sum(w * np.log(t)))
        g = self.gamma[self.off]
        return float(np.sum(w * t ** g))

    # U'_ij = u_ij'(T_ij), zero on the diagonal (Sec. 1.2)
    def grad(self, T):
        out = np.zeros_like(T)
        t = T[self.off]
        w = self.w[self.off]
        if self.kind == "log":
            out[self.off] = w / t
        else:
            g = self.gamma[self.off]
            out[self.off] = w * g * t ** (g - 1.0)
        return out

    # sum_{i != j} (-u_ij)^*(Y_ij), the conjugate of Sec. 2.1 evaluated entrywise:
    #   log:   sup_s (y s + w log s)     = w log(w / (-y)) - w
    #   power: sup_s (y s + w s^gamma)   = (1/gamma - 1) (w gamma)^(1/(1-gamma)) (-y)^(-gamma/(1-gamma))
    def conj_neg(self, Y) -> float:
        y = Y[self.off]
        if np.any(y >= 0):
            return math.inf
        w = self.w[self.off]
        if self.kind == "log":
            return float(np.sum(w * np.log(w / (-y)) - w))
        g = self.gamma[self.off]
        return float(np.sum((1.0 / g - 1.0) * (w * g) ** (1.0 / (1.0 - g)) * (-y) ** (-g / (1.0 - g))))

    # T(Y)_ij = (u_ij')^{-1}(-Y_ij): the traffic at which the marginal utility equals -Y_ij
    def traffic_from_dual(self, Y):
        out = np.zeros_like(Y)
        y = Y[self.off]
        w = self.w[self.off]
        if self.kind == "log":
            out[self.off] = w / (-y)
        else:
            g = self.gamma[self.off]
            out[self.off] = (w * g / (-y)) ** (1.0 / (1.0 - g))
        return out

    def prox(self, V, beta: float):
        """Entrywise prox_{beta (-u_ij)^*}(V_ij) of Sec. 2.3; the diagonal maps to 0."""
        out = np.zeros_like(V)
        v = V[self.off]
        w = self.w[self.off]
        if self.kind == "log":
            out[self.off] = prox_log(v, beta, w)
        else:
            out[self.off] = prox_pow(v, beta, w, self.gamma[self.off])
        return out


def prox_log(y, beta, w):
    """Sec. 2.3: prox_{beta (-u)^*}(y) = (y - sqrt(y^2 + 4 beta w)) / 2 for u = w log s."""
    y = np.asarray(y, dtype=np.float64)
    return (y - np.sqrt(y * y + 4.0 * beta * w)) / 2.0


def prox_pow(y, beta, w, gamma, max_newton: int = 200):
    """Sec. 2.3: for u = w s^gamma the prox is z = -t, t > 0 the unique root of
        h(t) = t^(c1+2) + y t^(c1+1) - c1 c2 = 0,
        c1 = gamma/(1-gamma),  c2 = beta (1/gamma - 1) (w gamma)^(1/(1-gamma)).

    Root bracket (derived, the paper gives no solver): with t_lo = max(0, -y) one has
    h(t_lo) = -c1 c2 < 0, and with t_hi = t_lo + (c1 c2)^(1/(c1+2)) one has h(t_hi) >= 0.
    On [t_lo, inf) h is increasing and convex, so Newton started at t_hi decreases
    monotonically to the root; it stops when a step no longer decreases t.
    """
    shape = np.shape(y)
    y = np.asarray(y, dtype=np.float64).ravel()
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), shape).ravel()
    g = np.broadcast_to(np.asarray(gamma, dtype=np.float64), shape).ravel()
    c1 = g / (1.0 - g)
    c2 = beta * (1.0 / g - 1.0) * (w * g) ** (1.0 / (1.0 - g))
    k = c1 * c2
    t_lo = np.maximum(0.0, -y)
    t = t_lo + k ** (1.0 / (c1 + 2.0))
    active = np.ones(y.shape, dtype=bool)
    for _ in range(max_newton):
        if not active.any():
            break
        ta, ya, c1a, ka = t[active], y[active], c1[active], k[active]
        p = ta ** c1a                        # t^c1
        h = p * ta * (ta + ya) - ka          # t^(c1+1) (t + y) - c1 c2
        dh = p * ((c1a + 2.0) * ta + (c1a + 1.0) * ya)
        tn = ta - h / dh
        tn = np.maximum(tn, t_lo[active])
        moved = tn < ta
        t_new = np.where(moved, tn, ta)
        t[active] = t_new
        idx = np.flatnonzero(active)
        active[idx[~moved]] = False
    return (-t).reshape(shape)


# --------------------------------------------------------------------------- projection

def project_capped_simplex(Q, c):
    """Column-wise Euclidean projection onto S_l = {f >= 0, 1^T f <= c_l}, Sec. 2.3/2.6.

    Pi(q) = (q - mu)_+ with mu = 0 if sum (q)_+ <= c, else (Held et al., Sec. 2.6): sort q
    in decreasing order to q', take the largest t with q'_t - (sum_{i<=t} q'_i - c)/t > 0
    and mu = (sum_{i<=t} q'_i - c)/t. Returns (F, mu) with mu the m multipliers.
    """
    Q = np.asarray(Q, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    n, m = Q.shape
    F = np.maximum(Q, 0.0)
    mu = np.zeros(m)
    need = F.sum(axis=0) > c
    if need.any():
        Qn = Q[:, need]
        cn = c[need]
        qs = -np.sort(-Qn, axis=0)                      # decreasing
        cs = np.cumsum(qs, axis=0)
        t = np.arange(1, n + 1, dtype=np.float64)[:, None]
        cond = qs - (cs - cn) / t > 0
        tstar = n - np.argmax(cond[::-1, :], axis=0)    # largest 1-based t with cond
        cols = np.arange(qs.shape[1])
        mun = (cs[tstar - 1, cols] - cn) / tstar
        mu[need] = mun
        F[:, need] = np.maximum(Qn - mun, 0.0)
    return F, mu


# --------------------------------------------------------------------------- residual, gap

def residual(G, F, Q, feasible: bool) -> float:
    """Eq. (e-res): r(Q) = min_{gamma>=0} ||G - gamma (F - Q)||_F^2 with F = Pi(Q)."""
    if not feasible:
        return math.inf
    D = F - Q
    g2 = float(np.sum(G * G))
    d2 = float(np.sum(D * D))
    gd = float(np.sum(G * D))
    if d2 == 0.0 or gd < 0.0:
        return g2
    return g2 - gd * gd / d2


def dual_bound(Yhat, A, c, util: Utility) -> float:
    """D(Y) = (-U)^*(Y) + sum_l c_l max(0, max_i (Y A)_il): minus the dual function of the
    reduced Lagrangian (Eq. e-L), since sup over F in the feasible set of Tr Y^T F A^T is
    sum_l c_l max(0, max_i (Y A)_il). Weak duality: U(T) <= D(Y) for feasible T."""
    if np.any(np.diag(Yhat) != 0.0):
        return math.inf
    conj = util.conj_neg(Yhat)
    YA = np.asarray(Yhat @ A)
    lin = float(np.sum(np.asarray(c) * np.maximum(0.0, YA.max(axis=0))))
    return conj + lin


@dataclass
class Metrics:
    feasible: bool
    nonpos_frac: float
    P: float
    D: float
    r: float
    g_norm: float
    rel_gap: float
    rel_cons: float
    rel_stat: float
    rel_kkt: float


def metrics(Fhat, Yhat, Q, A, c, util: Utility) -> Metrics:
    """Residual, duality gap and relative KKT at (F^, Y^) with F^ = Pi(Q)."""
    n = Fhat.shape[0]
    That = -np.asarray(Fhat @ A.T)
    off = util.off
    nonpos = int(np.sum(That[off] <= 0.0))
    feasible = nonpos == 0
    if feasible:
        P = util.value(That)
        G = np.asarray(util.grad(That) @ A)
        r = residual(G, Fhat, Q, True)
        gn = float(np.sqrt(np.sum(G * G)))
    else:
        P, r, gn = -math.inf, math.inf, math.inf
    D = dual_bound(Yhat, A, c, util)
    if feasible and math.isfinite(D):
        rel_gap = (D - P) / (1.0 + abs(P) + abs(D))
        rel_stat = math.sqrt(max(r, 0.0)) / (1.0 + gn)
    else:
        rel_gap = math.inf
        rel_stat = math.inf
    if np.all(Yhat[off] < 0):
        Ty = util.traffic_from_dual(Yhat)
        num = float(np.sqrt(np.sum((Ty[off] - That[off]) ** 2)))
        rel_cons = num / (1.0 + float(np.sqrt(np.sum(That[off] ** 2))))
    else:
        rel_cons = math.inf
    return Metrics(feasible, nonpos / float(n * (n - 1)), P, D, r, gn, rel_gap,
                   rel_cons, rel_stat, max(rel_gap, rel_cons, rel_stat))


# --------------------------------------------------------------------------- algorithm

@dataclass
class Result:
    status: str                  # "converged" | "max_iters"
    iters: int                   # PDHG iterations performed
    Fhat: np.ndarray             # returned flow, n x m (Sec. 2.5 returns F^{k-1/2})
    T: np.ndarray                # -F^ A^T
    Yhat: np.ndarray             # prox output Y^ of the last iteration
    utility: float
    metrics: Metrics | None
    omega: float
    F: np.ndarray                # relaxed iterate F^{k-1/2} (warm-start state)
    Y: np.ndarray                # relaxed iterate Y^k (warm-start state)
    mu: np.ndarray               # projection multipliers of the last iteration
    history: list = field(default_factory=list)
    omega_frozen_at: int = -1    # iteration from which omega stayed constant (-1: never)


def pdmcf(n, tail, head, cap, kind, w, gamma=None, *, eps=1e-6, stop_mode="kkt",
          max_iters=100000, rho=1.9, theta=0.5, k_adapt=100, tau=1e-5,
          omega_freeze_iter=-1, k_check=1, F0=None, Y0=None, omega0=1.0,
          adapt_guard=10.0, adapt_guard_below=1e-2, history=False, on_check=None,
          step=None) -> Result:
    """Algorithm 2.1 (PDMCF), float64.

    stop_mode: "paper" stops when r^k < n m eps (Sec. 2.5), "kkt" when rel_kkt^k < eps,
    "none" runs exactly max_iters iterations. Initialisation F^{-1/2} = 0,
    Y^0 = I - 1 1^T, omega^0 = 1 (Sec. 2.5) unless a warm start is given.

    omega stops adapting from iteration omega_freeze_iter on, and (adapt_guard > 0, written
    g) from the iteration after a stop test where omega is more than a factor g^2 away from
    omega_ref (omega at the first stop test with a finite rel_kkt), or, in the final phase,
    which begins at the first stop test with rel_kkt below adapt_guard_below (omega_arm =
    omega then), where omega is more than a factor g away from omega_arm or a finite
    rel_kkt exceeds g times the smallest one so far. Sec. 2.4 allows ending the adaptation after some iterations, a constant omega
    keeping the convergence proof; the guard is the point it is applied at (the rule of
    Eq. e-primal_weight can run away: omega -> 0 or infinity). adapt_guard = 0 is the
    adaptation without that stop.

    on_check, if given, is called with the record of every stop test (the same dict that
    ``history`` collects); it observes the run and changes nothing in it.

    step, if given, performs the updates of step 2 in place of the formulas below:
    step(F, Y, alpha, beta, rho) -> (Q, F^, mu, Y^, F_new, Y_new, Delta_F, Delta_Y), the same
    quantities (oracle.parallel spreads them over processes); the rest of the algorithm
    (stop test, primal weight rule, metrics) is unchanged.
    """
    tail = np.asarray(tail, dtype=np.int64)
    head = np.asarray(head, dtype=np.int64)
    c = np.asarray(cap, dtype=np.float64)
    m = tail.shape[0]
    A = incidence(n, tail, head)
    AT = A.T.tocsr()
    util = Utility(kind, w, gamma)
    eta = eta_bound(n, tail, head)

    F = np.zeros((n, m)) if F0 is None else np.array(F0, dtype=np.float64)
    Y = (np.eye(n) - np.ones((n, n))) if Y0 is None else np.array(Y0, dtype=np.float64)
    omega = float(omega0)
    r = math.inf
    met = None
    Fhat = Yhat = mu = None
    hist = []
    best_kkt = math.inf
    omega_ref = 0.0
    omega_arm = 0.0
    status = "max_iters"
    k = 0
    while True:
        # 1. stopping criterion (r^k and rel_kkt^k were computed in iteration k-1)
        if k > 0 and k % k_check == 0 and met is not None:
            if stop_mode == "paper" and r < n * m * eps:
                status = "converged"
                break
            if stop_mode == "kkt" and met.rel_kkt < eps:
                status = "converged"
                break
        if k >= max_iters:
            break
        alpha = eta / omega
        beta = eta * omega
        # 2. PDHG updates (Eq. e-pdhg-step)
        if step is None:
            Q = F + alpha * np.asarray(Y @ A)
            Fhat, mu = project_capped_simplex(Q, c)
            Fplus = 2.0 * Fhat - F
            V = Y - beta * np.asarray(Fplus @ AT)
            Yhat = util.prox(V, beta)
            F_new = rho * Fhat + (1.0 - rho) * F
            Y_new = rho * Yhat + (1.0 - rho) * Y
            dF = float(np.sqrt(np.sum((F_new - F) ** 2)))
            dY = float(np.sqrt(np.sum((Y_new - Y) ** 2)))
        else:
            Q, Fhat, mu, Yhat, F_new, Y_new, dF, dY = step(F, Y, alpha, beta, rho)
        # 3. adaptive primal weight (Eq. e-primal_weight)
        if (k % k_adapt == 0 and dF > tau and dY > tau
                and (omega_freeze_iter < 0 or k < omega_freeze_iter)):
            omega = (dY / dF) ** theta * omega ** (1.0 - theta)
        # residual r^{k+1} = r(F^{k-1/2} + alpha^k Y^k A), evaluated when it will be tested
        if (k + 1) % k_check == 0 or k + 1 >= max_iters:
            met = metrics(Fhat, Yhat, Q, A, c, util)
            r = met.r
            if adapt_guard > 0:
                fin = math.isfinite(met.rel_kkt)
                g2 = adapt_guard * adapt_guard
                drift_ref = omega_ref > 0 and (omega > g2 * omega_ref or omega * g2 < omega_ref)
                final_phase = omega_arm > 0 and ((fin and met.rel_kkt > adapt_guard * best_kkt)
                                                 or omega > adapt_guard * omega_arm
                                                 or omega * adapt_guard < omega_arm)
                if (drift_ref or final_phase) and \
                        (omega_freeze_iter < 0 or omega_freeze_iter > k + 1):
                    omega_freeze_iter = k + 1
                if fin:
                    best_kkt = min(best_kkt, met.rel_kkt)
                    if omega_ref == 0:
                        omega_ref = omega
                    if omega_arm == 0 and best_kkt < adapt_guard_below:
                        omega_arm = omega
            if history or on_check is not None:
                rec = dict(k=k + 1, omega=omega, r=r, rel_kkt=met.rel_kkt,
                           rel_gap=met.rel_gap, rel_cons=met.rel_cons,
                           rel_stat=met.rel_stat, P=met.P, D=met.D,
                           nonpos_frac=met.nonpos_frac)
                if history:
                    hist.append(rec)
                if on_check is not None:
                    on_check(rec)
        F, Y = F_new, Y_new
        k += 1
    if Fhat is None:
        raise ValueError("no iteration performed")
    T = -np.asarray(Fhat @ AT)
    U = util.value(T) if (met is not None and met.feasible) else -math.inf
    return Result(status, k, Fhat, T, Yhat, U, met, omega, F, Y, mu, hist, omega_freeze_iter)


def shortest_path_flow(n, tail, head, cap):
    """Sec. 1.1 feasibility argument: unit flow per (source, destination) pair along a
    fewest-edge path, scaled by alpha = 1/max_l(load_l / c_l). Returns (F, alpha)."""
    tail = np.asarray(tail, dtype=np.int64)
    head = np.asarray(head, dtype=np.int64)
    m = tail.shape[0]
    # BFS backwards from every destination i over reversed edges: parent edge per node
    into = [[] for _ in range(n)]
    for l in range(m):
        into[head[l]].append(l)
    F = np.zeros((n, m))
    for i in range(n):
        nxt_edge = -np.ones(n, dtype=np.int64)
        seen = np.zeros(n, dtype=bool)
        seen[i] = True
        frontier = [i]
        while frontier:
            new = []
            for v in frontier:
                for l in into[v]:
                    u = tail[l]
                    if not seen[u]:
                        seen[u] = True
                        nxt_edge[u] = l
                        new.append(u)
            frontier = new
        if not seen.all():
            raise ValueError("network is not strongly connected")
        for j in range(n):
            if j == i:
                continue
            v = j
            while v != i:
                l = nxt_edge[v]
                F[i, l] += 1.0
                v = head[l]
    load = F.sum(axis=0)
    alpha = 1.0 / np.max(load / np.asarray(cap, dtype=np.float64))
    return alpha * F, alpha
