"""Pins of the oracle's smooth maximum (CPU only).

The objective of arXiv 2207.06374 (Sec. "Optimization procedure") is the
shifted log-sum-exp F_{s,delta}(x) over x = |G_jk|^2, j < k, of the
column-normalised frame.  Each check below is fixed by mathematics, not by
the oracle's own formula:

* the Proposition's bounds s <= F <= s + delta log n;
* equal x_i (equiangular tight frames): F = s + delta log n exactly;
* one pair (N = 2): F = s;
* delta -> infinity: F - delta log n is the log-mean-exp of x/delta scaled by
  delta, between mean(x) (Jensen) and mean(x) + (max - min)^2 / (8 delta)
  (Hoeffding's lemma), with the x computed by a library matrix product;
* the gradient against central differences of F along random directions;
* invariances: scaling a column or its phase leaves F unchanged, so the
  gradient is orthogonal to v_k and to i v_k in every column; a unitary
  applied to the frame or a permutation of the columns leave F unchanged;
* critical points: at an equiangular tight frame all weights are equal and
  Phi Phi^* = (N/d) I, so the gradient vanishes for every delta.
"""
import numpy as np
import pytest

import frames as F
import oracle as O


def _x_by_matmul(v):
    phi = v / np.linalg.norm(v, axis=0, keepdims=True)
    G = phi.conj().T @ phi
    iu = np.triu_indices(G.shape[0], 1)
    return np.abs(G[iu]) ** 2


def _raw_frame(d, N, rng):
    # unnormalised columns of different lengths: the objective normalises them
    z = rng.standard_normal((d, N)) + 1j * rng.standard_normal((d, N))
    return z * rng.uniform(0.5, 2.0, size=(1, N))


@pytest.mark.parametrize("d,N", [(2, 5), (3, 9), (4, 20), (8, 40)])
@pytest.mark.parametrize("delta", [1e-3, 0.05, 1.0])
def test_proposition_bounds(d, N, delta):
    rng = np.random.default_rng(7 * d + N)
    v = _raw_frame(d, N, rng)
    f, s, _ = O.lse(v, delta, grad=False)
    n = N * (N - 1) // 2
    x = _x_by_matmul(v)
    assert s == pytest.approx(x.max(), rel=1e-13)
    assert s <= f <= s + delta * np.log(n) + 1e-15
    # strict on the left unless one term dominates: with n >= 10 distinct
    # values and delta >= 0.05 the other terms add visibly
    if delta >= 0.05:
        assert f > s


@pytest.mark.parametrize("make", [F.tetrahedral_2_4, F.harmonic_3_7, F.hesse_sic_3_9,
                                  lambda: F.naimark_complement(F.harmonic_3_7())])
@pytest.mark.parametrize("delta", [1e-4, 0.01, 0.3])
def test_equiangular_frames_reach_the_upper_bound(make, delta):
    phi = make()
    d, N = phi.shape
    n = N * (N - 1) // 2
    W2 = F.welch(N, d) ** 2
    f, s, _ = O.lse(phi, delta, grad=False)
    assert s == pytest.approx(W2, abs=1e-14)
    assert f == pytest.approx(W2 + delta * np.log(n), abs=1e-13)


def test_single_pair_is_the_max():
    rng = np.random.default_rng(3)
    v = _raw_frame(5, 2, rng)
    for delta in (1e-6, 0.1, 10.0):
        f, s, _ = O.lse(v, delta, grad=False)
        assert f == s == pytest.approx(_x_by_matmul(v)[0], rel=1e-13)


@pytest.mark.parametrize("delta", [1e2, 1e4])
def test_large_delta_tends_to_the_mean(delta):
    rng = np.random.default_rng(11)
    v = _raw_frame(4, 15, rng)
    n = 15 * 14 // 2
    x = _x_by_matmul(v)
    f, _, _ = O.lse(v, delta, grad=False)
    lme = f - delta * np.log(n)
    slack = 1e-12 * delta          # rounding of delta * log(sum), sum ~ n
    assert x.mean() - slack <= lme <= x.mean() + (x.max() - x.min()) ** 2 / (8 * delta) + slack


@pytest.mark.parametrize("d,N,delta", [(2, 4, 0.05), (3, 8, 0.02), (5, 12, 0.1), (4, 30, 0.01)])
def test_gradient_matches_central_differences(d, N, delta):
    rng = np.random.default_rng(100 + N)
    v = _raw_frame(d, N, rng)
    _, _, g = O.lse(v, delta)
    eps = 1e-6
    for _ in range(6):
        u = rng.standard_normal((d, N)) + 1j * rng.standard_normal((d, N))
        fp, _, _ = O.lse(v + eps * u, delta, grad=False)
        fm, _, _ = O.lse(v - eps * u, delta, grad=False)
        fd = (fp - fm) / (2 * eps)
        an = float(np.sum(g.real * u.real + g.imag * u.imag))
        assert an == pytest.approx(fd, rel=2e-5, abs=2e-8)


def test_gradient_orthogonal_to_scale_and_phase():
    rng = np.random.default_rng(5)
    v = _raw_frame(6, 25, rng)
    _, _, g = O.lse(v, 0.02)
    inner = np.sum(v.conj() * g, axis=0)            # v_k^* g_k per column
    scale = np.max(np.abs(g)) * np.max(np.abs(v))
    assert np.max(np.abs(inner.real)) < 1e-13 * scale
    assert np.max(np.abs(inner.imag)) < 1e-13 * scale


def test_invariant_under_unitary_phases_and_permutation():
    rng = np.random.default_rng(9)
    v = _raw_frame(4, 18, rng)
    U = F.haar_unitary(4, rng)
    ph = np.exp(2j * np.pi * rng.uniform(size=18))
    perm = rng.permutation(18)
    f0, s0, g0 = O.lse(v, 0.03)
    f1, s1, g1 = O.lse((U @ v) * ph[None, :], 0.03)
    f2, s2, g2 = O.lse(v[:, perm], 0.03)
    assert f1 == pytest.approx(f0, rel=1e-13) and f2 == pytest.approx(f0, rel=1e-13)
    assert s1 == pytest.approx(s0, rel=1e-13) and s2 == pytest.approx(s0, rel=1e-13)
    # the gradient transforms with the frame
    assert np.allclose(g1, (U @ g0) * ph[None, :], rtol=0, atol=1e-12 * np.abs(g0).max())
    assert np.allclose(g2, g0[:, perm], rtol=0, atol=1e-13 * np.abs(g0).max())


@pytest.mark.parametrize("make", [F.tetrahedral_2_4, F.harmonic_3_7, F.hesse_sic_3_9])
def test_gradient_vanishes_at_equiangular_tight_frames(make):
    phi = make()
    for delta in (0.001, 0.1, 3.0):
        _, _, g = O.lse(phi, delta)
        assert np.max(np.abs(g)) < 1e-13


def test_gradient_nonzero_away_from_optimum():
    rng = np.random.default_rng(1)
    _, _, g = O.lse(_raw_frame(3, 9, rng), 0.01)
    assert np.max(np.abs(g)) > 1e-3


def test_rejects_bad_arguments():
    rng = np.random.default_rng(2)
    v = _raw_frame(3, 4, rng)
    with pytest.raises(ValueError):
        O.lse(v, 0.0)
    with pytest.raises(ValueError):
        O.lse(v[:, :1], 0.1)
    z = v.copy()
    z[:, 2] = 0
    with pytest.raises(ValueError):
        O.lse(z, 0.1)
