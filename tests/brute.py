"""Pure-Python brute force for the coherence, independent of the oracle's C.

mu(Phi) = max_{j != k} |<phi_j, phi_k>| over the columns of Phi
(arXiv 2207.06374, Sec. "Introduction").  Only for tiny inputs: every ordered
pair j != k is visited with Python complex arithmetic, so neither the
upper-triangle shortcut nor the |.|^2 reduction of the oracle is reused here.
"""


def inner(x, y):
    """<x, y> = sum_i conj(x_i) y_i."""
    s = 0j
    for a, b in zip(x, y):
        s += a.conjugate() * b
    return s


def coherence(cols):
    """cols: list of N lists of d Python complex numbers (unit columns)."""
    best = 0.0
    for j in range(len(cols)):
        for k in range(len(cols)):
            if j != k:
                v = abs(inner(cols[j], cols[k]))
                if v > best:
                    best = v
    return best


def columns(phi):
    """numpy (d, N) -> list of column lists of Python complex numbers."""
    d, N = phi.shape
    return [[complex(phi[i, j]) for i in range(d)] for j in range(N)]
