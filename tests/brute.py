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


def episode_mode_reference(model, A, n_obs, root_states, root_w, M, K, eta, gamma, seed,
                           log_pibar, step, draw_obs, terminal, heuristic, philox_words):
    """Alg. 1-3 as printed, written independently of the oracle: a list of belief nodes in
    creation order, each a dict keyed by (action, observation) for its children; episodes
    sampled from the root weights, actions from softmax(Psi / eta), the tree grown on first
    visits (continuous observations, n_obs = 0, always grow it), terminal states ending an
    episode, leaf heuristics aggregated per leaf, and the visit-weighted backup applying
    Psi <- Psi - L Psi + Q (Q = 0 for an action without visits) to every belief above the
    leaves, deepest first.  ``philox_words(idx, purpose, level, node)`` returns the four
    Philox words of counter (level, idx | purpose << 24, node, 0)."""
    from oracle import uniform
    w = np.asarray(root_w, dtype=np.float64)
    w = np.where([terminal(s) for s in root_states], 0.0, w)
    cdf = np.cumsum(w / w.sum())

    def new_node(parent, depth):
        return dict(parent=parent, depth=depth, psi=eta * np.asarray(log_pibar, float).copy(),
                    V=0.0, C=np.zeros(A), N=np.zeros(A, dtype=np.int64), kids={}, Hs=0.0, Nl=0)

    nodes = [new_node(None, 0)]
    steps = 0
    for k in range(1, K + 1):
        ep = []
        for e in range(M):
            u = uniform(philox_words(e, 7, 0, k)[0])
            i = int(np.argmax(u < cdf)) if u < cdf[-1] else len(cdf) - 1
            ep.append([root_states[i], 0, True])
        for d in range(k):
            for e in range(M):
                s, b, alive = ep[e]
                if not alive:
                    continue
                z = nodes[b]["psi"] / eta
                p = np.exp(z - z.max())
                c = np.cumsum(p / p.sum())
                u = uniform(philox_words(e, 8, d, k)[0])
                a = int(np.argmax(u < c)) if u < c[-1] else A - 1
                w9 = philox_words(e, 9, d, k)
                s2, r = step(s, a, w9[0], w9[1])
                w10 = philox_words(e, 10, d, k)
                o = draw_obs(s2, a, w10[0], w10[1])
                nodes[b]["C"][a] += r
                nodes[b]["N"][a] += 1
                steps += 1
                if terminal(s2):
                    ep[e][2] = False
                    continue
                key = (a, o) if n_obs else None
                if key is not None and key in nodes[b]["kids"]:
                    nb = nodes[b]["kids"][key]
                else:
                    nb = len(nodes)
                    nodes.append(new_node((b, a), d + 1))
                    if key is not None:
                        nodes[b]["kids"][key] = nb
                ep[e] = [s2, nb, True]
        for s, b, alive in ep:
            if alive:
                nodes[b]["Hs"] += heuristic(s)
                nodes[b]["Nl"] += 1
        for n in nodes:
            if n["depth"] == k:
                n["V"] = n["Hs"] / n["Nl"] if n["Nl"] else 0.0
        for d in range(k, 0, -1):
            ws = {}
            for n in nodes:
                if n["depth"] == d:
                    visits = n["Nl"] if d == k else int(n["N"].sum())
                    ws[n["parent"]] = ws.get(n["parent"], 0.0) + visits * n["V"]
            for bi, n in enumerate(nodes):
                if n["depth"] != d - 1:
                    continue
                q = np.array([n["C"][a] / n["N"][a] + gamma * ws.get((bi, a), 0.0) / n["N"][a]
                              if n["N"][a] else 0.0 for a in range(A)])
                n["psi"] = n["psi"] - eta * logsumexp(n["psi"] / eta) + q
                n["V"] = float(eta * logsumexp(n["psi"] / eta))
    return nodes, steps
