"""Closed forms and master-equation solutions that pin the oracle to the mathematics.

TEST INFRASTRUCTURE ONLY.  Nothing here calls the C oracle: the rate functions are written out
again from the model definitions so that a mistake in the oracle's propensities cannot hide
behind a shared formula.

  * 1-D birth-death chains: stationary law by detailed balance and the mean first-passage time
    T(a -> b) = sum_{k=a}^{b-1} (sum_{j<=k} pi_j) / (lambda_k pi_k) (standard result for a chain
    reflected at 0), used for Eq. "mfpt" checks and for the Schloegl MFPT the paper quotes as
    about 5e4 s (Sec. III.B.3);
  * the immigration-death process 0 -> X (kb), X -> 0 (kd x): X(t) = Binomial(x0, e^{-kd t})
    + Poisson(kb/kd (1 - e^{-kd t})), independent, which tends to Poisson(kb/kd);
  * truncated chemical master equations (CME) solved with a matrix exponential (1-D transients,
    the Schloegl P(X >= 700, t=5) = 1.148e-9 of Sec. III.B.3) or a sparse linear solve (2-D
    mean first-passage times of the toggle switch);
  * the enzymatic futile cycle's CME (Eq. "futile", 400 states with one enzyme of each kind and
    100 substrate molecules) by uniformization, for its tail P(S1 > 90, t = 100) = 2.72e-18
    printed in Sec. III.A;
  * the maximum-likelihood transition time of brute-force runs (Eq. "mld", Sec. II.C).
"""
from __future__ import annotations

import numpy as np
from scipy import sparse
from scipy.linalg import expm
from scipy.sparse.linalg import expm_multiply, spsolve
from scipy.special import gammaln, logsumexp


# ----------------------------------------------------------------------------------------------
# model rate functions, written out from the paper's reaction schemes
# ----------------------------------------------------------------------------------------------
def birth_death_rates(kb=10.0, kd=0.1):
    return (lambda x: np.full(np.shape(x), kb, dtype=np.float64),
            lambda x: kd * np.asarray(x, dtype=np.float64))


def schlogl_rates(c1=3e-7, c2=1e-4, c3=1e-3, c4=3.5, A=1e5, B=2e5):
    """Schloegl model (Sec. III.B.1) with combinatorial mass action: A+2X->3X at c1 A X(X-1)/2,
    3X->A+2X at c2 X(X-1)(X-2)/6, B->X at c3 B, X->B at c4 X."""
    def birth(x):
        x = np.asarray(x, dtype=np.float64)
        return c1 * A * x * (x - 1) / 2.0 + c3 * B

    def death(x):
        x = np.asarray(x, dtype=np.float64)
        return c2 * x * (x - 1) * (x - 2) / 6.0 + c4 * x
    return birth, death


# ----------------------------------------------------------------------------------------------
# 1-D birth-death chains
# ----------------------------------------------------------------------------------------------
def bd_log_stationary(birth, death, N: int) -> np.ndarray:
    """log of the unnormalised stationary measure on {0..N}: pi_{x+1}/pi_x = birth(x)/death(x+1)."""
    x = np.arange(N)
    steps = np.log(birth(x)) - np.log(death(x + 1))
    return np.concatenate([[0.0], np.cumsum(steps)])


def bd_stationary(birth, death, N: int) -> np.ndarray:
    lp = bd_log_stationary(birth, death, N)
    return np.exp(lp - logsumexp(lp))


def bd_modes(birth, death, N: int):
    """Local maxima and minima (interior) of the stationary law."""
    lp = bd_log_stationary(birth, death, N)
    maxima = [x for x in range(1, N) if lp[x] >= lp[x - 1] and lp[x] >= lp[x + 1]]
    minima = [x for x in range(1, N) if lp[x] <= lp[x - 1] and lp[x] <= lp[x + 1]]
    return maxima, minima


def bd_mfpt(a: int, b: int, birth, death) -> float:
    """Mean first-passage time from a up to b > a of a chain on {0,1,...} reflected at 0."""
    assert b > a >= 0
    lp = bd_log_stationary(birth, death, b)
    total = 0.0
    for k in range(a, b):
        # expected time to go from k to k+1
        total += np.exp(logsumexp(lp[:k + 1]) - lp[k] - np.log(birth(np.array([k]))[0]))
    return float(total)


def bd_generator(birth, death, N: int) -> sparse.csr_matrix:
    """Generator Q (rows = from) of the chain truncated to {0..N} (no birth out of N)."""
    x = np.arange(N + 1)
    up = birth(x).astype(np.float64)
    up[-1] = 0.0
    down = death(x).astype(np.float64)
    down[0] = 0.0
    Q = sparse.diags([-(up + down), up[:-1], down[1:]], [0, 1, -1], shape=(N + 1, N + 1), format="csr")
    return Q


def bd_transient(birth, death, x0: int, t: float, N: int) -> np.ndarray:
    """P(X(t) = x | X(0) = x0) on {0..N} by the matrix exponential of the truncated CME."""
    p0 = np.zeros(N + 1)
    p0[x0] = 1.0
    Q = bd_generator(birth, death, N)
    return expm_multiply((Q.T * t).tocsr(), p0)


# ----------------------------------------------------------------------------------------------
# immigration-death closed form
# ----------------------------------------------------------------------------------------------
def log_poisson_pmf(x, mean: float) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return x * np.log(mean) - mean - gammaln(x + 1)


def immigration_death_pmf(x0: int, kb: float, kd: float, t: float, N: int) -> np.ndarray:
    """Law of X(t) on {0..N}: Binomial(x0, e^{-kd t}) convolved with Poisson(kb/kd (1-e^{-kd t}))."""
    p = np.exp(-kd * t)
    k = np.arange(x0 + 1)
    lb = (gammaln(x0 + 1) - gammaln(k + 1) - gammaln(x0 - k + 1) + k * np.log(p)
          + (x0 - k) * np.log1p(-p)) if 0 < p < 1 else np.where(k == x0, 0.0, -np.inf)
    mean = kb / kd * (1 - p)
    x = np.arange(N + 1)
    lpo = log_poisson_pmf(x, mean)
    out = np.full(N + 1, -np.inf)
    for xi in range(N + 1):
        kk = k[k <= xi]
        out[xi] = logsumexp(lb[kk] + lpo[xi - kk])
    return np.exp(out)


# ----------------------------------------------------------------------------------------------
# 2-D truncated CME: toggle switch mean first-passage time
# ----------------------------------------------------------------------------------------------
def toggle_mfpt(a_u: float, a_v: float, start, in_target, d=1.0, K=1.0, n=2, b0=0.0,
                Umax: int = 200, Vmax: int = 200) -> float:
    """MFPT from ``start`` into the set ``in_target(u, v)`` for the two-gene toggle
    0->U at a_u/(1+(V/K)^n), 0->V at a_v/(1+(U/K)^n), U->0 and V->0 at d per molecule, plus basal
    production b0.  Solves sum_y Q(x,y) T(y) = -1 off the target with T = 0 on it, on the grid
    truncated to [0,Umax] x [0,Vmax] (no production out of the box)."""
    nu, nv = Umax + 1, Vmax + 1
    idx = lambda u, v: u * nv + v
    rows, cols, vals = [], [], []
    rhs = np.zeros(nu * nv)
    for u in range(nu):
        for v in range(nv):
            i = idx(u, v)
            if in_target(u, v):
                rows.append(i); cols.append(i); vals.append(1.0)
                continue
            rhs[i] = -1.0
            out = 0.0
            moves = []
            if u < Umax:
                moves.append((idx(u + 1, v), a_u / (1.0 + (v / K) ** n) + b0))
            if v < Vmax:
                moves.append((idx(u, v + 1), a_v / (1.0 + (u / K) ** n) + b0))
            if u > 0:
                moves.append((idx(u - 1, v), d * u))
            if v > 0:
                moves.append((idx(u, v - 1), d * v))
            for j, r in moves:
                if r > 0:
                    rows.append(i); cols.append(j); vals.append(r)
                    out += r
            rows.append(i); cols.append(i); vals.append(-out)
    A = sparse.csr_matrix((vals, (rows, cols)), shape=(nu * nv, nu * nv))
    T = spsolve(A.tocsc(), rhs)
    return float(T[idx(*start)])


def epigenetic_mfpt(start, in_target, a1=156.0, a2=30.0, n=3, m=1, K1=1.0, K2=1.0, k0=1.0,
                    G1: int = 400, G2: int = 120) -> float:
    """MFPT of the epigenetic switch of Sec. III.C from ``start`` into ``in_target(g1, g2)``:
    0 -> g1 at a1/(1+(g2/K2)^n), 0 -> g2 at a2/(1+(g1/K1)^m), g1 -> 0 and g2 -> 0 at k0 per
    molecule, written out again from the model's equations.  Solves sum_y Q(x,y) T(y) = -1 off
    the target, T = 0 on it, on [0,G1] x [0,G2] (no production out of the box)."""
    n1, n2 = G1 + 1, G2 + 1
    idx = lambda u, v: u * n2 + v
    rows, cols, vals = [], [], []
    rhs = np.zeros(n1 * n2)
    for u in range(n1):
        for v in range(n2):
            i = idx(u, v)
            if in_target(u, v):
                rows.append(i); cols.append(i); vals.append(1.0)
                continue
            rhs[i] = -1.0
            out = 0.0
            moves = []
            if u < G1:
                moves.append((idx(u + 1, v), a1 / (1.0 + (v / K2) ** n)))
            if v < G2:
                moves.append((idx(u, v + 1), a2 / (1.0 + (u / K1) ** m)))
            if u > 0:
                moves.append((idx(u - 1, v), k0 * u))
            if v > 0:
                moves.append((idx(u, v - 1), k0 * v))
            for j, r in moves:
                rows.append(i); cols.append(j); vals.append(r)
                out += r
            rows.append(i); cols.append(i); vals.append(-out)
    A = sparse.csr_matrix((vals, (rows, cols)), shape=(n1 * n2, n1 * n2))
    T = spsolve(A.tocsc(), rhs)
    return float(T[idx(*start)])


# ----------------------------------------------------------------------------------------------
# enzymatic futile cycle (Eq. "futile", Sec. III.A): truncation-free CME by uniformization
# ----------------------------------------------------------------------------------------------
def futile_states(total=100):
    """States (b1, b2, s1) of the futile cycle with one enzyme of each kind and S1 + S2 + B1 + B2
    = total: b1, b2 in {0, 1} (enzyme bound), 0 <= s1 <= total - b1 - b2 (then S2 is fixed)."""
    return [(b1, b2, s1) for b1 in (0, 1) for b2 in (0, 1) for s1 in range(total - b1 - b2 + 1)]


def futile_generator(kf=1.0, ks=0.1, total=100):
    """Transition rates of the six reactions, written out from the scheme E1 + S1 <-> B1 -> E1 + S2,
    E2 + S2 <-> B2 -> E2 + S1 with combinatorial mass action (E = 1 - B for each enzyme).
    Returns (states, index, list of (from, to, rate))."""
    st = futile_states(total)
    idx = {x: k for k, x in enumerate(st)}
    tr = []
    for k, (b1, b2, s1) in enumerate(st):
        s2 = total - s1 - b1 - b2
        if b1 == 0 and s1 > 0:
            tr.append((k, idx[(1, b2, s1 - 1)], kf * s1))          # E1 + S1 -> B1
        if b1 == 1:
            tr.append((k, idx[(0, b2, s1 + 1)], kf))               # B1 -> E1 + S1
            tr.append((k, idx[(0, b2, s1)], ks))                   # B1 -> E1 + S2
        if b2 == 0 and s2 > 0:
            tr.append((k, idx[(b1, 1, s1)], kf * s2))              # E2 + S2 -> B2
        if b2 == 1:
            tr.append((k, idx[(b1, 0, s1)], kf))                   # B2 -> E2 + S2
            tr.append((k, idx[(b1, 0, s1 + 1)], ks))               # B2 -> E2 + S1
    return st, idx, tr


def uniformized_transient(n: int, transitions, p0: np.ndarray, t: float) -> np.ndarray:
    """p(t) = sum_k Poisson(k; L t) p0 (I + Q/L)^k with L the largest exit rate.  Every term is
    non-negative, so probabilities far below the largest keep their relative accuracy (a matrix
    exponential in floating point resolves only about 1e-16 of the largest entry)."""
    out_rate = np.zeros(n)
    rows, cols, vals = [], [], []
    for a, b, r in transitions:
        out_rate[a] += r
        rows.append(a); cols.append(b); vals.append(r)
    L = out_rate.max()
    Pm = sparse.csr_matrix((np.asarray(vals) / L, (rows, cols)), shape=(n, n)) + sparse.diags(1.0 - out_rate / L)
    PT = Pm.T.tocsr()
    lam = L * t
    kmax = int(lam + 12.0 * np.sqrt(lam) + 50)
    logw = -lam
    v = p0.astype(np.float64).copy()
    acc = np.exp(logw) * v
    for k in range(1, kmax + 1):
        v = PT @ v
        logw += np.log(lam) - np.log(k)
        acc += np.exp(logw) * v
    return acc


def futile_s1_law(t: float, s1_0=50, s2_0=50, kf=1.0, ks=0.1) -> np.ndarray:
    """P(S1 = x, t) for x = 0..S1+S2 from S1 = s1_0, S2 = s2_0, both enzymes free."""
    total = s1_0 + s2_0
    st, idx, tr = futile_generator(kf, ks, total)
    p0 = np.zeros(len(st))
    p0[idx[(0, 0, s1_0)]] = 1.0
    p = uniformized_transient(len(st), tr, p0, t)
    law = np.zeros(total + 1)
    for k, (b1, b2, s1) in enumerate(st):
        law[s1] += p[k]
    return law


# ----------------------------------------------------------------------------------------------
# brute-force estimator of a transition time (Eq. "mld", Sec. II.C)
# ----------------------------------------------------------------------------------------------
def mle_transition_time(T: float, N: int, times) -> tuple:
    """Mean transition time from N brute-force runs of length T, n of which saw the transition, at
    times t_i (Eq. "mld", Sec. II.C): the maximum-likelihood mean of exponential waiting times
    whose runs without a transition are censored at T,

        mu = (sum t_i + (N - n) T) / n = (1/n) sum t_i + (N/n - 1) T,   sigma = mu / sqrt(n).

    Reading: the equation as printed puts the factor (1 - n/N) on T.  The censored likelihood
    gives (N/n - 1), and so do the paper's own epigenetic-switch figures (Sec. III.C): 753 runs
    of 1e6 s giving 1.3e6 s with sigma 6.5e4 s mean n = (mu / sigma)^2 = 400 transitions, which
    an exponential of mean 1.3e6 s yields (753 (1 - e^(-1/1.3)) = 404) at a mean observed time of
    4.4e5 s; with (N/n - 1) that is 1.3e6 s again, with (1 - n/N) it would be 9.0e5 s."""
    times = np.asarray(times, dtype=np.float64)
    n = len(times)
    if n == 0:
        raise ValueError("no transition observed: the estimate is unbounded")
    if n > N or np.any(times < 0) or np.any(times > T):
        raise ValueError("need 0 <= t_i <= T and at most N transitions")
    mu = (times.sum() + (N - n) * T) / n
    return mu, mu / np.sqrt(n)


def small_generator_expm(Q: np.ndarray, p0: np.ndarray, t: float) -> np.ndarray:
    """Dense matrix exponential for tiny state spaces (reference for brute-force checks)."""
    return p0 @ expm(Q * t)
