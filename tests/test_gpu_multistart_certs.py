"""Multi-start and frame certificates on the GPU against the oracle.

Multi-start (Algorithm "TRSTMI optimization steps", last step of arXiv
2207.06374): trial i is the search with seed seed0 + i, so in binary64 every
trial's mu equals the oracle's run with that seed, the minimum and its index
follow, and grouping the trials into batches changes nothing.

Certificates (Sec. "Conjectures from Numerics"; chordal distance of Sec.
"Introduction"): max and min of |G_jk| against the oracle's enumeration
(binary64, 1e-13), the bounds against the oracle's formulas, the number of
distinct distances against the oracle's binning.
"""
import numpy as np
import pytest

import frames as F
import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")


def test_multistart_fp64_matches_oracle_trials():
    N, d, seed0, L, iters, K = 7, 3, 40, 6, 30, 64
    res, mus, phi = T.multistart(N, d, seed0, L, iters, K=K, precision="fp64")
    assert res.trials == L
    ref = []
    for i in range(L):
        _, m2, _, _ = O.run(N, d, seed0 + i, O.make_opts(K=K, T=iters), nthreads=4)
        ref.append(np.sqrt(m2))
    assert np.allclose(mus, ref, rtol=1e-12, atol=0)
    best = int(np.argmin(mus))
    assert res.best == best and res.best_seed == seed0 + best
    assert res.mu == mus[best]
    assert np.sqrt(O.mu2(phi)) == pytest.approx(res.mu, rel=1e-12)


def test_multistart_default_trials_and_batch_grouping():
    N, d = 9, 3
    a, mus_a, phi_a = T.multistart(N, d, 5, 0, 15, K=32, precision="fp32")
    assert a.trials == 2 * d * d
    b, mus_b, phi_b = T.multistart(N, d, 5, 0, 15, batch_cap=4, K=32, precision="fp32")
    assert np.array_equal(mus_a, mus_b) and a.best == b.best
    assert np.array_equal(phi_a, phi_b)


def test_multistart_screen_mode_trials_match_solo_runs():
    N, d, seed0, L, iters = 40, 6, 3, 4, 8
    res, mus, _ = T.multistart(N, d, seed0, L, iters, want_phi=False, K=32,
                               precision="bf16", topk=4)
    for i in range(L):
        with T.Search(N, d, seed0 + i, K=32, precision="bf16", topk=4) as s:
            s.step(iters)
            assert s.step(0).mu == mus[i]


def test_multistart_rejects_bad_arguments():
    with pytest.raises(T.TrstmiError):
        T.multistart(1, 2, 0, 3, 5)
    with pytest.raises(T.TrstmiError):
        T.multistart(4, 2, 0, 3, -1)


def _check_against_oracle(phi, tol):
    """The GPU normalises the columns; the oracle's enumeration takes unit
    columns, so it gets them normalised by numpy."""
    d, N = phi.shape
    c = T.certificates(phi, tol)
    phi = phi / np.linalg.norm(phi, axis=0, keepdims=True)
    mx, mn = O.gram_extremes(phi)
    assert c["mu"] == pytest.approx(np.sqrt(mx), rel=1e-13, abs=1e-15)
    assert c["mu_min"] == pytest.approx(np.sqrt(mn), rel=1e-12, abs=1e-7)
    assert c["welch"] == pytest.approx(O.welch(N, d), rel=1e-15)
    assert c["orthoplex"] == pytest.approx(O.orthoplex(N, d), rel=1e-15)
    assert c["levenshtein"] == pytest.approx(O.levenshtein(N, d), rel=1e-15)
    lb = max(O.welch(N, d), O.orthoplex(N, d), O.levenshtein(N, d))
    assert c["lower_bound"] == pytest.approx(lb, rel=1e-15)
    assert c["gap"] == pytest.approx(c["mu"] - lb, abs=1e-14)
    assert c["min_chordal"] == pytest.approx(np.sqrt(1 - mx), abs=1e-13)
    assert c["distinct"] == O.distinct_distances(phi, tol)
    return c


@pytest.mark.parametrize("make,distinct", [(F.tetrahedral_2_4, 1), (F.harmonic_3_7, 1),
                                           (F.hesse_sic_3_9, 1), (lambda: F.mubs(3), 2),
                                           (lambda: F.mubs(5), 2),
                                           (lambda: np.eye(6, dtype=np.complex128), 1)])
def test_certificates_of_known_frames(make, distinct):
    phi = make()
    c = _check_against_oracle(phi, 1e-6)
    assert c["distinct"] == distinct
    d, N = phi.shape
    if N == d * (d + 1):            # full MUBs: both bounds met with equality
        assert c["gap"] == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("d,N,tol", [(2, 5, 1e-3), (3, 40, 1e-4), (8, 70, 1e-5),
                                     (16, 200, 1e-6), (32, 130, 1e-3), (5, 257, 1e-7)])
def test_certificates_of_random_frames(d, N, tol):
    rng = np.random.default_rng(d + N)
    z = rng.standard_normal((d, N)) + 1j * rng.standard_normal((d, N))
    phi = z * rng.uniform(0.5, 2.0, size=(1, N))      # normalised inside
    c = _check_against_oracle(phi, tol)
    assert c["mu"] >= c["lower_bound"] - 1e-15


def test_instance_certificates_track_the_search():
    with T.Search(12, 3, 2, K=128, precision="fp64") as s:
        s.step(200)
        c = s.certificates(1e-6)
        assert c["mu"] == pytest.approx(s.coherence()[0], rel=1e-13)
        assert c["orthoplex"] == pytest.approx(1 / np.sqrt(3))
        assert c["mu"] >= c["lower_bound"]


def test_certificates_reject_bad_arguments():
    phi = F.mubs(3)
    for tol in (0.0, 1e-9, 2.0):
        with pytest.raises(T.TrstmiError):
            T.certificates(phi, tol)
    z = phi.copy()
    z[:, 3] = 0
    with pytest.raises(T.TrstmiError):
        T.certificates(z, 1e-6)
