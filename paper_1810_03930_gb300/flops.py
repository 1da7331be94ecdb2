"""Algorithmic work of one PLAM/PCAL iteration (Table "cost", Section 3.3).

The table counts, per iteration: X^T X (n p^2, symmetric), grad f^T X (2 n p^2),
X Psi(grad f^T X) (2 n p^2, shared by the update and, through the Section 3.3
shortcut, by the KKT test) and X (X^T X - I) (2 n p^2): 7 n p^2 + O(n p) for both
PLAM and PCAL.  This implementation forms the same work as X M with
M = Lambda - beta (B - I) for the update and X Psi(C) for the KKT residual.
"""


def iteration_flops(n: int, p: int) -> dict:
    """Floating-point operations of the BLAS3 part of one iteration, by step."""
    npp = n * p * p
    d = {
        "gram_xx": npp,            # B = X^T X (upper triangle, multiply-add = 2 flops)
        "gram_xg": 2 * npp,        # C = X^T G
        "update": 2 * npp,         # X M
        "kkt_product": 2 * npp,    # X Psi(C)
    }
    d["total"] = sum(d.values())
    return d


def iteration_bytes(n: int, p: int, w: int, kkt: bool = True) -> dict:
    """Algorithmic DRAM bytes of the n x p passes of one iteration (w = bytes per element).

    gram: read X and G; update: read X, G, R_prev and write R; primal: read X, R and
    write X.  The objective's own traffic is accounted for separately.
    """
    np_ = n * p * w
    return {"gram": 2 * np_, "update": 4 * np_, "primal": 3 * np_, "total": 9 * np_}
