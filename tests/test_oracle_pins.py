"""Pins of the CPU oracle to mathematics and to printed values (CPU only).

Every function of the oracle is checked against something other than itself:
published known-answer vectors, closed forms, exact special cases, invariances,
distribution laws and an independent brute force.  References are to
arXiv 2207.06374 (the TRSTMI paper) unless stated otherwise.
"""
import os

import numpy as np
import pytest
from scipy import stats

import brute
import frames as F
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(x, 16) for x in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


# ---------------------------------------------------- Gaussian entries

def _draws(n_cols=4000, d=4, seed=12345, c=3, t=7, tag=0):
    z = np.array([[O.gauss_entry(seed, d, i, j, c, t, tag) for i in range(d)]
                  for j in range(n_cols)]).reshape(-1)
    return z


def test_gauss_is_standard_complex_normal():
    """Z ~ CN(0,1): Re, Im ~ N(0, 1/2) independent; |Z|^2 ~ Exp(1); arg uniform."""
    z = _draws()
    n = z.size
    for part in (z.real, z.imag):
        assert stats.kstest(part * np.sqrt(2), "norm").pvalue > 1e-3
        assert abs(part.mean()) < 5 / np.sqrt(2 * n)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 5 / np.sqrt(n)
    assert stats.kstest(np.abs(z) ** 2, "expon").pvalue > 1e-3
    assert stats.kstest((np.angle(z) + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 5 / np.sqrt(n)
    # neighbouring entries (same Philox call, and adjacent calls) uncorrelated
    assert abs(np.corrcoef(z.real[0::2], z.real[1::2])[0, 1]) < 5 / np.sqrt(n / 2)


def test_gauss_counter_fields_decorrelate():
    """Changing any counter field (c, t, tag) or the seed gives a fresh draw."""
    base = _draws(500, 2)
    for kw in ({"c": 4}, {"t": 8}, {"tag": 1}, {"seed": 12346}):
        other = _draws(500, 2, **kw)
        assert not np.allclose(base, other)
        assert abs(np.corrcoef(base.real, other.real)[0, 1]) < 0.15


def test_gauss_entry_uses_box_muller_of_the_philox_words():
    """Z for (i even) is sqrt(-ln U0) e^{2 pi i U1} of the call's first words."""
    seed, d, i, j, c, t = (7 << 32) | 99, 5, 2, 3, 11, 13
    u = O.philox4x32_10([j * 3 + 1, c, t, 0], [seed & 0xffffffff, seed >> 32])
    U = [(x + 0.5) / 2.0 ** 32 for x in u]
    z = O.gauss_entry(seed, d, i, j, c, t, 0)
    assert abs(z - np.sqrt(-np.log(U[0])) * np.exp(2j * np.pi * U[1])) < 1e-14
    z = O.gauss_entry(seed, d, i + 1, j, c, t, 0)
    assert abs(z - np.sqrt(-np.log(U[2])) * np.exp(2j * np.pi * U[3])) < 1e-14


# -------------------------------------------------------- coherence mu

@pytest.mark.parametrize("d,N", [(1, 2), (1, 5), (2, 2), (2, 3), (3, 5), (4, 4), (5, 3), (3, 8)])
def test_mu_matches_brute_force(d, N):
    rng = np.random.default_rng(d * 100 + N)
    for _ in range(3):
        phi = F.random_frame(d, N, rng)
        assert abs(O.mu(phi) - brute.coherence(brute.columns(phi))) < 1e-14


def test_mu_d1_is_one():
    """In C^1 all unit vectors are parallel lines: mu = 1 = Welch bound."""
    rng = np.random.default_rng(1)
    phi = F.random_frame(1, 6, rng)
    assert abs(O.mu(phi) - 1.0) < 1e-15
    assert abs(O.welch(6, 1) - 1.0) < 1e-15


def test_mu_zero_for_orthonormal_basis():
    rng = np.random.default_rng(2)
    for d in (2, 3, 8):
        assert O.mu(np.eye(d, dtype=np.complex128)) == 0.0
        assert O.mu(F.haar_unitary(d, rng)) < 1e-14


@pytest.mark.parametrize("name,make", [
    ("tetrahedral(2,4)", F.tetrahedral_2_4),
    ("harmonic(3,7)", F.harmonic_3_7),
    ("hesse(3,9)", F.hesse_sic_3_9),
    ("naimark(7,4)", lambda: F.naimark_complement(F.harmonic_3_7())),
    ("naimark(9,6)", lambda: F.naimark_complement(F.hesse_sic_3_9())),
])
def test_etf_meets_welch_bound(name, make):
    phi = make()
    d, N = phi.shape
    W = np.sqrt((N - d) / (d * (N - 1)))
    assert abs(O.mu(phi) - W) < 1e-12
    assert abs(O.welch(N, d) - W) < 1e-15


def test_welch_values_at_the_workload_shapes():
    # closed-form values at the workload shapes (Sec. "Welch bound ...")
    assert abs(O.welch(4, 2) - 1 / np.sqrt(3)) < 1e-15
    assert abs(O.welch(7, 3) - np.sqrt(2 / 9)) < 1e-15
    assert abs(O.welch(9, 3) - 0.5) < 1e-15
    assert abs(O.welch(64, 8) - 1 / 3) < 1e-15
    assert abs(O.welch(1024, 32) - 1 / np.sqrt(33)) < 1e-15


@pytest.mark.parametrize("d", [2, 3])
def test_mubs_meet_orthoplex_bound(d):
    """(d+1) MUBs, and those with j < d points removed, have mu = 1/sqrt(d)."""
    phi = F.mubs(d)
    assert phi.shape == (d, d * (d + 1))
    assert abs(O.mu(phi) - 1 / np.sqrt(d)) < 1e-12
    for j in range(d):
        assert abs(O.mu(phi[:, j:]) - 1 / np.sqrt(d)) < 1e-12


def test_mu_invariances():
    """mu is invariant under a global unitary, column phases, permutation, conj."""
    rng = np.random.default_rng(3)
    for d, N in ((2, 5), (4, 9), (6, 13)):
        phi = F.random_frame(d, N, rng)
        m = O.mu(phi)
        U = F.haar_unitary(d, rng)
        assert abs(O.mu(U @ phi) - m) < 1e-13
        ph = np.exp(2j * np.pi * rng.random(N))
        assert abs(O.mu(phi * ph[None, :]) - m) < 1e-13
        assert abs(O.mu(phi[:, rng.permutation(N)]) - m) < 1e-13
        assert abs(O.mu(phi.conj()) - m) < 1e-13


def test_mu_at_least_welch_on_random_frames():
    rng = np.random.default_rng(4)
    for d, N in ((2, 4), (3, 9), (4, 16), (5, 11)):
        for _ in range(5):
            assert O.mu(F.random_frame(d, N, rng)) >= O.welch(N, d) - 1e-15


def test_bloch_sphere_correspondence_d2():
    """For C^2, |<x,y>|^2 = (1 + cos angle of Bloch vectors)/2."""
    rng = np.random.default_rng(5)
    phi = F.random_frame(2, 7, rng)
    a, b = phi[0], phi[1]
    bloch = np.stack([2 * (a.conj() * b).real, 2 * (a.conj() * b).imag,
                      np.abs(a) ** 2 - np.abs(b) ** 2], axis=1)
    cosang = bloch @ bloch.T
    iu = np.triu_indices(7, 1)
    assert abs(O.mu2(phi) - ((1 + cosang[iu]) / 2).max()) < 1e-14


def test_gram_abs2_frame_potential_bound():
    """sum_{j,k} |G_jk|^2 >= N^2/d, with equality for tight frames."""
    import ctypes
    def fp(phi):
        d, N = phi.shape
        b = O._flat(phi)
        return sum(O.lib().oracle_gram_abs2(d, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), j, k)
                   for j in range(N) for k in range(N))
    rng = np.random.default_rng(6)
    phi = F.random_frame(3, 8, rng)
    assert fp(phi) >= 64 / 3 - 1e-12
    assert abs(fp(F.harmonic_3_7()) - 49 / 3) < 1e-12
    assert abs(fp(F.mubs(3)) - 144 / 3) < 1e-12


# ------------------------------------------------ init and candidates

def test_init_unit_columns_and_seeded():
    a = O.init(9, 3, 42)
    b = O.init(9, 3, 42)
    c = O.init(9, 3, 43)
    assert np.array_equal(a, b) and not np.allclose(a, c)
    assert np.abs(np.linalg.norm(a, axis=0) - 1).max() < 1e-15
    # init draws are the tag-1 stream with c = t = 0, columns normalised
    z = np.array([[O.gauss_entry(42, 3, i, j, 0, 0, 1) for j in range(9)] for i in range(3)])
    assert np.abs(a - z / np.linalg.norm(z, axis=0)).max() < 1e-15


def test_candidate_special_cases():
    rng = np.random.default_rng(7)
    phi = F.random_frame(4, 10, rng)
    # Delta = 0 leaves the frame unchanged
    assert np.abs(O.candidate(phi, 5, 0.0, 3, 2) - phi).max() < 1e-15
    # unit columns for any Delta; same counters -> same candidate
    for delta in (1e-9, 0.1, 10.0):
        cand = O.candidate(phi, 5, delta, 3, 2)
        assert np.abs(np.linalg.norm(cand, axis=0) - 1).max() < 1e-15
        assert np.array_equal(cand, O.candidate(phi, 5, delta, 3, 2))
    # Delta -> infinity: the candidate is the normalised noise itself
    big = O.candidate(phi, 5, 1e12, 3, 2)
    z = np.array([[O.gauss_entry(5, 4, i, j, 2, 3, 0) for j in range(10)] for i in range(4)])
    assert np.abs(big - z / np.linalg.norm(z, axis=0)).max() < 1e-10
    # first order: (cand*|phi+dZ| - phi)/delta = Z
    delta = 1e-3
    cand = O.candidate(phi, 5, delta, 3, 2)
    nrm = np.linalg.norm(phi + delta * z, axis=0)
    assert np.abs((cand * nrm - phi) / delta - z).max() < 1e-9


def test_score_matches_candidate_by_candidate_and_threads():
    phi = O.init(12, 3, 8)
    s1 = O.score(phi, 8, 0.05, 4, 10, 37, nthreads=1)
    s4 = O.score(phi, 8, 0.05, 4, 10, 37, nthreads=4)
    assert np.array_equal(s1, s4)
    for k in (0, 17, 36):
        cand = O.candidate(phi, 8, 0.05, 4, 10 + k)
        assert abs(s1[k] - brute.coherence(brute.columns(cand)) ** 2) < 1e-14


# ------------------------------------------------------------- search

def _check_trace(tr, opts, mu2_init, delta0):
    m, dl = mu2_init, delta0
    for row in tr:
        assert row["delta_used"] == dl
        acc = row["mu2_best"] < m
        assert bool(row["accepted"]) == acc
        if acc:
            m = row["mu2_best"]
            dl = min(opts.gamma_inc * dl, opts.delta_max)
        else:
            dl = max(opts.gamma_dec * dl, opts.delta_min)
        assert row["mu2_cur"] == m and row["delta_next"] == dl


def test_search_trace_follows_rule_and_final_mu_is_exact():
    N, d, seed = 7, 3, 3
    opts = O.make_opts(K=64, T=60)
    phi, m2, dl, tr = O.run(N, d, seed, opts, nthreads=2)
    phi0 = O.init(N, d, seed)
    _check_trace(tr, opts, O.mu2(phi0), opts.delta0)
    assert len(tr) == 60 and tr["accepted"].sum() > 0
    assert np.all(np.diff(tr["mu2_cur"]) <= 0)
    assert abs(m2 - brute.coherence(brute.columns(phi)) ** 2) < 1e-14
    assert np.sqrt(m2) >= O.welch(N, d)
    # the first iteration's choice is the argmin of its scores (lowest c on ties)
    s = O.score(phi0, seed, opts.delta0, 1, 0, 64)
    assert tr[0]["cstar"] == int(np.argmin(s)) and tr[0]["mu2_best"] == s.min()


def test_search_resume_is_bitwise():
    N, d, seed = 6, 2, 11
    a = O.run(N, d, seed, O.make_opts(K=32, T=40))
    b = O.run(N, d, seed, O.make_opts(K=32, T=25))
    c = O.search(b[0], seed, O.make_opts(K=32, T=15), b[2], b[1], 25)
    assert np.array_equal(a[0], c[0]) and a[1] == c[1] and a[2] == c[2]


def test_replay_of_own_choices_reproduces_run():
    N, d, seed = 5, 2, 4
    opts = O.make_opts(K=32, T=30)
    phi, m2, dl, tr = O.run(N, d, seed, opts)
    phi0 = O.init(N, d, seed)
    rp, rm2, rdl, rtr = O.replay(phi0, seed, opts, opts.delta0, O.mu2(phi0), 0, tr["cstar"])
    assert np.array_equal(rp, phi) and rm2 == m2 and rdl == dl
    assert np.array_equal(rtr, tr)


def test_target_stops_search():
    opts = O.make_opts(K=128, T=2000, target_mu=0.6)
    phi, m2, dl, tr = O.run(4, 2, 1, opts)
    assert np.sqrt(m2) <= 0.6 and len(tr) < 2000
    assert np.sqrt(tr["mu2_cur"][-2]) > 0.6


def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_table2_mu.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, N, m = line.split()
                rows[(int(d), int(N))] = float(m)
    return rows


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_search_reaches_tetrahedral_code(seed):
    """d=2, N=4, K=256, Delta0=0.1, T=2000 in double precision: mu -> 1/sqrt(3),
    the Welch bound met by the tetrahedral SIC; the paper's Table 2 value for
    (2,4) is 0.5774 (rounded up), which the run must not exceed."""
    phi, m2, dl, tr = O.run(4, 2, seed, O.make_opts(K=256, T=2000))
    mu = np.sqrt(m2)
    assert abs(mu - 1 / np.sqrt(3)) < 1e-5
    assert mu <= _table2()[(2, 4)]


# ------------------------------ the binary32 plain-loop variant (CPU baseline)

@pytest.mark.parametrize("d,N,K", [(2, 4, 16), (8, 64, 12), (32, 200, 3), (5, 33, 9), (1, 6, 4)])
def test_f32_variant_matches_the_binary64_oracle_to_f32_rounding(d, N, K):
    """Same candidates, single-precision arithmetic: mu agrees with the
    binary64 oracle to binary32 rounding (entries within ~8 ulp, a Gram entry
    within ~(2d + 2) ulp more, so |dmu| <= ~(2d + 20) 2^-24 < 1e-5 here)."""
    phi = O.init(N, d, 3)
    for t, c0, delta in ((1, 0, 0.1), (7, 40, 0.6)):
        ref = O.score(phi, 3, delta, t, c0, K)
        f32 = O.score_f32(phi, 3, delta, t, c0, K, nthreads=2)
        assert np.max(np.abs(np.sqrt(f32) - np.sqrt(ref))) < (2 * d + 20) * 2.0 ** -24 * 4
        # the binary32 values are not the binary64 ones (the variant is not a copy)
        assert d == 1 or np.any(f32 != ref)


def test_f32_variant_on_closed_forms_and_zero_radius():
    """Radius 0 leaves the frame unchanged: the variant's mu is the frame's
    own, e.g. the tetrahedral code's 1/sqrt(3) and 1 in C^1."""
    import frames as F
    phi = F.tetrahedral_2_4()
    m = O.score_f32(phi, 1, 0.0, 1, 0, 3)
    assert np.allclose(np.sqrt(m), 1 / np.sqrt(3), atol=1e-6)
    m1 = O.score_f32(np.ones((1, 5), dtype=complex), 1, 0.3, 2, 0, 4)
    assert np.allclose(m1, 1.0, atol=1e-6)
