"""Brute-force exact soft expectimax over exact Bayesian beliefs (test-side, independent).

For a finite POMDP given as matrices T[a][s, s'], Z[s', o], R[s, a] and a prior b, the
Reference-Based value of Eq. 1-2 with one preference update from the reference policy is
    Q_d(b, a) = sum_s b(s) R(s, a) + gamma * sum_o p(o | b, a) V_{d-1}(b_{a,o})
    V_d(b)    = eta * log sum_a pibar(a) exp(Q_d(b, a) / eta),   V_0 = 0,
with b' = b T[a], p(o | b, a) = sum_s' b'(s') Z[s', o], b_{a,o} = b' * Z[:, o] / p.
Written with numpy matrices and exact belief vectors, sharing nothing with the oracle's
particle recursion.

``porpp_anytime`` is the anytime planning loop of Alg. 1 on the same exact tree: iteration
k = 1, 2, ... searches to depth k and applies the preference update of Eq. 3,
    Psi(h, .) <- Psi(h, .) - [L Psi](h) + Q(h, .),   V(h) = [L Psi](h),
to preferences kept per action-observation history h across iterations, a history's first
visit starting from Psi_0 = eta log pibar ([L Psi] = eta log sum_a exp(Psi / eta)).
"""
import numpy as np
from scipy.special import logsumexp

TOY2_T = [np.eye(2), np.array([[0.0, 1.0], [1.0, 0.0]])]
TOY2_Z = np.array([[0.85, 0.15], [0.15, 0.85]])
TOY2_R = np.array([[1.0, -0.1], [-1.0, -0.1]])


def soft_expectimax(b, depth, eta, gamma, log_pibar, T=TOY2_T, Z=TOY2_Z, R=TOY2_R, hard=False):
    b = np.asarray(b, dtype=np.float64)

    def value(bel, d):
        if d == 0:
            return 0.0
        q = qvalues(bel, d)
        if hard:
            return float(np.max(q[np.isfinite(log_pibar)]))
        return float(eta * logsumexp(log_pibar + q / eta))

    def qvalues(bel, d):
        q = np.zeros(len(T))
        for a in range(len(T)):
            pred = bel @ T[a]
            q[a] = bel @ R[:, a]
            for o in range(Z.shape[1]):
                p = pred @ Z[:, o]
                if p > 0:
                    q[a] += gamma * p * value(pred * Z[:, o] / p, d - 1)
        return q

    return value(b, depth), qvalues(b, depth) if depth > 0 else None


def porpp_anytime(b, K, eta, gamma, log_pibar, T=TOY2_T, Z=TOY2_Z, R=TOY2_R):
    """Returns (V(root), Psi(root), Q(root) of the last iteration, [Q(root) per iteration])."""
    b = np.asarray(b, dtype=np.float64)
    log_pibar = np.asarray(log_pibar, dtype=np.float64)
    psi = {}

    def lse(p):
        return float(eta * logsumexp(p / eta))

    def visit(bel, hist, d, q_out):
        if d == 0:
            return 0.0
        q = np.zeros(len(T))
        for a in range(len(T)):
            pred = bel @ T[a]
            q[a] = bel @ R[:, a]
            for o in range(Z.shape[1]):
                p = pred @ Z[:, o]
                if p > 0:
                    q[a] += gamma * p * visit(pred * Z[:, o] / p, hist + ((a, o),), d - 1, None)
        if hist not in psi:
            psi[hist] = eta * log_pibar.copy()
        psi[hist] = psi[hist] - lse(psi[hist]) + q
        if q_out is not None:
            q_out.append(q)
        return lse(psi[hist])

    qs, v = [], None
    for k in range(1, K + 1):
        v = visit(b, (), k, qs)
    return v, psi[()].copy(), qs[-1], qs
