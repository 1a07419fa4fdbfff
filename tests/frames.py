"""Closed-form frames used as test inputs (no TRSTMI arithmetic here).

Each construction has a known coherence, which pins the oracle (and, on the
GPU, the CUDA path) to mathematics rather than to itself:

* equiangular tight frames meet the Welch bound sqrt((N-d)/(d(N-1)))
  (arXiv 2207.06374, Sec. "Welch bound and equiangular lines");
* the Naimark complement of an ETF(N, d) is an ETF(N, N-d) (same section);
* vectors from different mutually unbiased bases have |<x, y>| = 1/sqrt(d),
  so a full set of d+1 MUBs, or one with a few points removed, has
  mu = 1/sqrt(d) (Sec. "Conjectures from Numerics", orthoplex bound).

All frames are numpy complex128 arrays of shape (d, N) with unit columns.
"""
import numpy as np


def haar_unitary(d, rng):
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def random_frame(d, N, rng):
    z = rng.standard_normal((d, N)) + 1j * rng.standard_normal((d, N))
    return z / np.linalg.norm(z, axis=0, keepdims=True)


def tetrahedral_2_4():
    """SIC in C^2: e0 plus three vectors at 120 degree phases; mu = 1/sqrt(3)."""
    w = np.exp(2j * np.pi / 3)
    cols = [np.array([1.0, 0.0])]
    for k in range(3):
        cols.append(np.array([1 / np.sqrt(3), np.sqrt(2 / 3) * w ** k]))
    return np.stack(cols, axis=1).astype(np.complex128)


def harmonic_3_7():
    """Rows {1,2,4} (a (7,3,1) difference set) of the 7-point DFT; an ETF."""
    w = np.exp(2j * np.pi / 7)
    rows = [1, 2, 4]
    return np.array([[w ** (r * j) for j in range(7)] for r in rows]) / np.sqrt(3)


def hesse_sic_3_9():
    """Weyl-Heisenberg orbit of the fiducial (0, 1, -1)/sqrt(2): SIC in C^3."""
    w = np.exp(2j * np.pi / 3)
    v = np.array([0.0, 1.0, -1.0], dtype=np.complex128) / np.sqrt(2)
    X = np.roll(np.eye(3), 1, axis=0)          # |k> -> |k+1>
    Z = np.diag([w ** k for k in range(3)])
    cols = []
    for a in range(3):
        for b in range(3):
            cols.append(np.linalg.matrix_power(X, a) @ np.linalg.matrix_power(Z, b) @ v)
    return np.stack(cols, axis=1)


def naimark_complement(phi):
    """ETF(N, d) -> ETF(N, N-d): complete sqrt(d/N) Phi to a unitary."""
    d, N = phi.shape
    u0 = np.sqrt(d / N) * phi                     # orthonormal rows
    # orthonormal basis of the orthogonal complement of the row space
    q, _ = np.linalg.qr(np.concatenate([u0.conj().T, np.eye(N)], axis=1))
    psi = q[:, d:N].conj().T                      # (N-d) x N, rows orthonormal
    psi = psi * np.sqrt(N / (N - d))
    return psi / np.linalg.norm(psi, axis=0, keepdims=True)


def mubs(d):
    """The standard basis plus the d bases (w^{k m^2 + l m})_m / sqrt(d), d prime."""
    w = np.exp(2j * np.pi / d)
    cols = [np.eye(d)[:, m] for m in range(d)]
    for k in range(d):
        for l in range(d):
            if d == 2:
                # for d = 2 use the Pauli eigenbases: (1, +-1)/sqrt2, (1, +-i)/sqrt2
                v = np.array([1.0, (-1) ** l * (1j if k else 1.0)]) / np.sqrt(2)
            else:
                v = np.array([w ** (k * m * m + l * m) for m in range(d)]) / np.sqrt(d)
            cols.append(v)
    return np.stack(cols, axis=1).astype(np.complex128)


def welch(N, d):
    return float(np.sqrt((N - d) / (d * (N - 1)))) if N > d else 0.0
