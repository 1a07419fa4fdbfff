"""Pins of the oracle's coherence bounds and frame diagnostics (CPU only).

Sec. "Conjectures from Numerics" of arXiv 2207.06374 states the orthoplex
bound mu >= 1/sqrt(d) and the Levenshtein bound mu^2 >= (2N - d(d+1)) /
((N - d)(d+1)) for N > d^2, with equality in the latter only for tight
frames with angle set {0, mu^2}; the chordal distance is sqrt(1 - |<x,y>|^2)
(Sec. "Introduction").  The checks: a full set of d + 1 mutually unbiased
bases is tight with angles {0, 1/d}, so it meets both bounds with equality;
the bounds hold on random frames; their behaviour in N; the extremes of
|G_jk| against a library matrix product; the number of distinct distances
of frames whose angle sets are known.
"""
import numpy as np
import pytest

import frames as F
import oracle as O


def _abs_offdiag(phi):
    G = phi.conj().T @ phi
    iu = np.triu_indices(G.shape[0], 1)
    return np.abs(G[iu])


@pytest.mark.parametrize("d", [2, 3, 5])
def test_full_mubs_meet_both_bounds(d):
    phi = F.mubs(d)
    N = phi.shape[1]
    assert N == d * (d + 1)
    mu = np.sqrt(O.gram_extremes(phi)[0])
    assert mu == pytest.approx(1 / np.sqrt(d), abs=1e-14)
    assert O.orthoplex(N, d) == pytest.approx(1 / np.sqrt(d), abs=1e-15)
    assert O.levenshtein(N, d) == pytest.approx(1 / np.sqrt(d), abs=1e-15)


def test_mubs_with_points_removed_meet_the_orthoplex_bound():
    phi = F.mubs(3)
    for j in range(3):                  # N = 12 - j > d^2 = 9
        sub = phi[:, : 12 - j]
        N = sub.shape[1]
        mu = np.sqrt(O.gram_extremes(sub)[0])
        assert mu == pytest.approx(O.orthoplex(N, 3), abs=1e-14)
        assert O.levenshtein(N, 3) < O.orthoplex(N, 3)


def test_bounds_apply_only_above_d_squared():
    for d in (2, 3, 4):
        for N in (d, d + 1, d * d):
            assert O.orthoplex(N, d) == 0.0 and O.levenshtein(N, d) == 0.0
        assert O.orthoplex(d * d + 1, d) > 0 and O.levenshtein(d * d + 1, d) > 0
    assert O.orthoplex(5, 1) == 0.0 and O.levenshtein(5, 1) == 0.0


def test_levenshtein_grows_with_N_towards_its_limit():
    d = 3
    vals = [O.levenshtein(N, d) for N in range(d * d + 1, 400)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    assert vals[-1] < np.sqrt(2 / (d + 1))
    # above d(d+1) it is the stronger of the two
    assert O.levenshtein(d * (d + 1) + 1, d) > O.orthoplex(d * (d + 1) + 1, d)


@pytest.mark.parametrize("d,N", [(2, 5), (2, 9), (3, 10), (3, 20), (4, 17), (4, 40)])
def test_bounds_hold_on_random_frames(d, N):
    rng = np.random.default_rng(d * 100 + N)
    for _ in range(5):
        phi = F.random_frame(d, N, rng)
        mu = np.sqrt(O.gram_extremes(phi)[0])
        assert mu >= O.welch(N, d) - 1e-15
        assert mu >= O.orthoplex(N, d) - 1e-15
        assert mu >= O.levenshtein(N, d) - 1e-15


@pytest.mark.parametrize("d,N", [(2, 4), (3, 11), (6, 40)])
def test_extremes_against_matmul(d, N):
    phi = F.random_frame(d, N, np.random.default_rng(N))
    mx, mn = O.gram_extremes(phi)
    a = _abs_offdiag(phi) ** 2
    assert mx == pytest.approx(a.max(), rel=1e-13)
    assert mn == pytest.approx(a.min(), rel=1e-12, abs=1e-30)


def test_extremes_of_known_frames():
    onb = np.eye(4, dtype=np.complex128)
    assert O.gram_extremes(onb) == (0.0, 0.0)
    sic = F.hesse_sic_3_9()
    mx, mn = O.gram_extremes(sic)
    assert mx == pytest.approx(0.25, abs=1e-14) and mn == pytest.approx(0.25, abs=1e-14)
    mx, mn = O.gram_extremes(F.mubs(3))
    assert mx == pytest.approx(1 / 3, abs=1e-14) and mn == pytest.approx(0.0, abs=1e-14)


def test_distinct_distances_of_known_frames():
    assert O.distinct_distances(F.tetrahedral_2_4(), 1e-6) == 1
    assert O.distinct_distances(F.hesse_sic_3_9(), 1e-6) == 1
    assert O.distinct_distances(F.harmonic_3_7(), 1e-6) == 1
    assert O.distinct_distances(F.mubs(3), 1e-6) == 2      # {0, 1/sqrt 3}
    assert O.distinct_distances(np.eye(5, dtype=np.complex128), 1e-6) == 1
    # a coarse resolution merges them: 0 and 0.577 share bin 0 at tol = 0.6
    assert O.distinct_distances(F.mubs(3), 0.6) == 1


def test_distinct_distances_of_random_frames_match_sorted_gaps():
    """Values farther apart than 2 tol are different distances and values
    closer than tol the same one, so with every gap outside [tol, 2 tol] the
    count equals 1 + the number of gaps above tol."""
    rng = np.random.default_rng(4)
    checked = 0
    for tol in (1e-3, 3e-3, 1e-2, 0.05):
        for _ in range(20):
            phi = F.random_frame(3, 12, rng)
            v = np.sort(_abs_offdiag(phi))
            gaps = np.diff(v)
            if np.any((gaps >= tol) & (gaps <= 2 * tol)):
                continue
            assert O.distinct_distances(phi, tol) == 1 + int(np.sum(gaps > tol))
            checked += 1
    assert checked >= 5


def test_distinct_distances_rejects_bad_arguments():
    with pytest.raises(ValueError):
        O.distinct_distances(np.eye(3, dtype=np.complex128), 0.0)
    with pytest.raises(ValueError):
        O.distinct_distances(np.eye(3, dtype=np.complex128), 2.0)
