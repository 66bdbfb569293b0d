"""External validation metrics for a detected partition against the planted
ground truth of a synthetic graph (Sec. 5, evaluation metrics): NMI, AMI and
the pairwise F1 score. They score results; neither the CUDA path nor the
oracle uses them.

Every metric works on the contingency table M of two labelings: M_ij is the
number of nodes in cluster i of the first and cluster j of the second, N the
number of nodes, a_i and b_j its row and column sums.
"""
from __future__ import annotations

import numpy as np
from scipy.special import gammaln


def contingency(a, b) -> np.ndarray:
    a = np.unique(np.asarray(a).ravel(), return_inverse=True)[1]
    b = np.unique(np.asarray(b).ravel(), return_inverse=True)[1]
    if a.size != b.size:
        raise ValueError("labelings differ in length")
    M = np.zeros((a.max() + 1, b.max() + 1), dtype=np.int64)
    np.add.at(M, (a, b), 1)
    return M


def _entropy(s: np.ndarray, N: int) -> float:
    s = s[s > 0].astype(np.float64)
    return float(-(s / N * np.log(s / N)).sum())


def _mutual_information(M: np.ndarray) -> float:
    N = int(M.sum())
    a = M.sum(1).astype(np.float64)
    b = M.sum(0).astype(np.float64)
    i, j = np.nonzero(M)
    nij = M[i, j].astype(np.float64)
    return float((nij / N * np.log(nij * N / (a[i] * b[j]))).sum())


def nmi(a, b) -> float:
    """NMI(C, C') = -2 sum_ij M_ij log(M_ij N / (a_i b_j)) divided by
    sum_i a_i log(a_i / N) + sum_j b_j log(b_j / N), i.e. the mutual
    information over the mean of the two entropies. Two one-cluster
    labelings agree perfectly (1)."""
    M = contingency(a, b)
    N = int(M.sum())
    den = _entropy(M.sum(1), N) + _entropy(M.sum(0), N)
    if den == 0.0:
        return 1.0
    return 2.0 * _mutual_information(M) / den


def expected_mutual_information(M: np.ndarray) -> float:
    """E[MI] under the hypergeometric model of random labelings with the
    cluster sizes of M (Vinh, Epps and Bailey, JMLR 2010, Eq. 24a): for each
    pair of sizes (a_i, b_j) the sum over n_ij from max(1, a_i + b_j - N) to
    min(a_i, b_j) of (n_ij / N) log(N n_ij / (a_i b_j)) times the
    hypergeometric probability of n_ij. Pairs of equal sizes are grouped."""
    N = int(M.sum())
    ua, ca = np.unique(M.sum(1), return_counts=True)
    ub, cb = np.unique(M.sum(0), return_counts=True)
    lgN = gammaln(N + 1)
    total = 0.0
    for ai, mult_a in zip(ua.tolist(), ca.tolist()):
        for bj, mult_b in zip(ub.tolist(), cb.tolist()):
            lo, hi = max(1, ai + bj - N), min(ai, bj)
            if lo > hi:
                continue
            k = np.arange(lo, hi + 1, dtype=np.float64)
            log_p = (gammaln(ai + 1) + gammaln(bj + 1) + gammaln(N - ai + 1) + gammaln(N - bj + 1)
                     - lgN - gammaln(k + 1) - gammaln(ai - k + 1) - gammaln(bj - k + 1)
                     - gammaln(N - ai - bj + k + 1))
            term = (k / N) * np.log(N * k / (ai * bj)) * np.exp(log_p)
            total += mult_a * mult_b * float(term.sum())
    return total


def ami(a, b) -> float:
    """AMI(U, V) = (MI - E[MI]) / (max(H(U), H(V)) - E[MI])."""
    M = contingency(a, b)
    N = int(M.sum())
    hu, hv = _entropy(M.sum(1), N), _entropy(M.sum(0), N)
    emi = expected_mutual_information(M)
    den = max(hu, hv) - emi
    if den == 0.0 or (hu == 0.0 and hv == 0.0):
        return 1.0
    return (_mutual_information(M) - emi) / den


def pairwise_f1(pred, truth) -> float:
    """Every unordered node pair is a binary decision (same community or not).
    Precision = pairs together in both / pairs together in pred, recall =
    pairs together in both / pairs together in truth, F1 their harmonic mean.
    With no positive pair on either side the two partitions are all
    singletons; F1 is then 1 if both are, else 0."""
    M = contingency(pred, truth)
    pairs = lambda x: int((x * (x - 1) // 2).sum())
    tp = pairs(M)
    pp, tt = pairs(M.sum(1)), pairs(M.sum(0))
    if pp == 0 or tt == 0:
        return 1.0 if pp == tt else 0.0
    prec, rec = tp / pp, tp / tt
    return 0.0 if tp == 0 else 2.0 * prec * rec / (prec + rec)
