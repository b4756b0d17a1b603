"""Error bounds from the paper, used by several tests.

paper_bound: eq. (cascerr) of Sec. "Forward error" per k-block, summed over
the k-blocks, plus the FP64x2 accumulation of the block results."""
import numpy as np

from oracle import cascade as cs

EPS_DD = 2.0 ** -106
EPS_CASC = 2.0 ** -117


def paper_bound(a_hi, b_hi, kc=cs.KC):
    """Eq. (cascerr) per k-block, summed over blocks, plus the FP64x2
    accumulation of the block results: sum_p [2 eps_dd |A_p||B_p| +
    2 * 40 k_p^2 eps_casc ||a_ip||_inf ||b_pj||_inf] + K_B eps_dd |A||B|.
    (The factor 2 covers the paper's "approximately".)"""
    m, k = a_hi.shape
    n = b_hi.shape[1]
    tot = np.zeros((m, n))
    kb = max(1, (k + kc - 1) // kc)
    for p in range(kb):
        sl = slice(p * kc, (p + 1) * kc)
        ap, bp = np.abs(a_hi[:, sl]), np.abs(b_hi[sl, :])
        kp = ap.shape[1]
        if kp == 0:
            continue
        tot += 2 * EPS_DD * (ap @ bp)
        tot += 2 * 40 * kp * kp * EPS_CASC * np.outer(ap.max(axis=1), bp.max(axis=0))
    tot += kb * EPS_DD * (np.abs(a_hi) @ np.abs(b_hi))
    return tot
