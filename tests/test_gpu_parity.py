"""CUDA path vs the CPU oracle, element by element on identical seeded inputs.

Tolerances: binary64 paths agree with the oracle to 1e-12 (relative on mu^2,
i.e. rounding-order differences only); binary32 coherence agrees to 1e-6
absolute on mu.  Shapes span several Gram tiles with a ragged tail, odd d,
N = 2, d = 1 and N <= d.
"""
import numpy as np
import pytest

import frames as F
import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")


def _mu_err(a2, b2):
    return abs(np.sqrt(a2) - np.sqrt(b2))


# ---------------------------------------------------------- coherence of frames


def check_precision_form_rows(tr, rtr, d, mu2_0):
    """Rows of a precision-form trace against the oracle's binary64 replay of
    the same choices: a certified row (flags bit 1 clear) carries the binary64
    mu^2 of the chosen candidate to 1e-12; an uncertified row was rejected on
    its binary32 score, which lies within the fp32/fp64 bound 2 (2d + 18) 2^-24
    of the binary64 value and above the current mu^2 by twice that bound."""
    cert = (tr["flags"] & 2) == 0
    assert np.allclose(tr["mu2_best"][cert], rtr["mu2_best"][cert], rtol=1e-12, atol=0)
    bound = 2.0 * (2 * d + 18) * 2.0 ** -24
    unc = ~cert
    assert np.all(tr["accepted"][unc] == 0)
    assert np.all(np.abs(tr["mu2_best"][unc] - rtr["mu2_best"][unc]) <= bound)
    prev = np.concatenate([[mu2_0], rtr["mu2_cur"][:-1]])
    assert np.all(rtr["mu2_best"][unc] >= prev[unc])
    return int(unc.sum())


@pytest.mark.parametrize("name,make", [
    ("tetrahedral(2,4)", F.tetrahedral_2_4), ("harmonic(3,7)", F.harmonic_3_7),
    ("hesse(3,9)", F.hesse_sic_3_9), ("mubs(3)", lambda: F.mubs(3)),
    ("naimark(9,6)", lambda: F.naimark_complement(F.hesse_sic_3_9())),
])
def test_frame_mu_closed_forms(name, make):
    phi = make()
    ref = O.mu2(phi)
    assert abs(T.mu2_frame(phi, "fp64") - ref) <= 1e-12 * ref
    assert _mu_err(T.mu2_frame(phi, "fp32"), ref) < 1e-6


@pytest.mark.parametrize("d,N", [(1, 5), (2, 2), (3, 17), (7, 130), (8, 64), (5, 301), (32, 200),
                                 (16, 3), (64, 70)])
def test_frame_mu_random(d, N):
    rng = np.random.default_rng(100 * d + N)
    phi = F.random_frame(d, N, rng)
    ref = O.mu2(phi)
    assert abs(T.mu2_frame(phi, "fp64") - ref) <= 1e-12 * max(ref, 1e-300)
    assert _mu_err(T.mu2_frame(phi, "fp32"), ref) < 1e-6


def test_frame_mu_orthonormal_is_zero():
    rng = np.random.default_rng(9)
    U = F.haar_unitary(12, rng)
    assert T.mu2_frame(U, "fp64") < 1e-28
    assert T.mu2_frame(U, "fp32") < 1e-12


# ------------------------------------------------------- init and candidates

@pytest.mark.parametrize("d,N,seed", [(2, 4, 1), (3, 9, 5), (7, 45, 12345678901), (32, 150, 3)])
def test_init_matches_oracle(d, N, seed):
    with T.Search(N, d, seed) as s:
        phi = s.get_phi()
    assert np.abs(phi - O.init(N, d, seed)).max() < 1e-14


@pytest.mark.parametrize("d,N", [(2, 4), (5, 33), (8, 64)])
def test_candidates_match_oracle(d, N):
    seed = 77
    with T.Search(N, d, seed) as s:
        phi0 = s.get_phi()
        for (t, c, delta) in [(1, 0, 0.1), (5, 300, 0.7), (123456, 4095, 1e-6)]:
            ref = O.candidate(phi0, seed, delta, t, c)
            assert np.abs(s.candidate(t, c, delta, "fp64") - ref).max() < 1e-13
            assert np.abs(s.candidate(t, c, delta, "fp32") - ref).max() < 2e-6


# ----------------------------------------------------------------- scoring

@pytest.mark.parametrize("d,N,K", [(2, 4, 256), (3, 7, 64), (8, 64, 96), (5, 130, 12), (1, 3, 8),
                                   (6, 4, 16)])
def test_scores_match_oracle(d, N, K):
    seed = 2024
    with T.Search(N, d, seed) as s:
        phi0 = s.get_phi()
        for (t, c0, delta) in [(1, 0, 0.1), (17, 1000, 0.02)]:
            ref = O.score(phi0, seed, delta, t, c0, K, nthreads=4)
            g64 = s.score(t, c0, K, delta, "fp64")
            g32 = s.score(t, c0, K, delta, "fp32")
            assert np.all(np.abs(g64 - ref) <= 1e-12 * np.maximum(ref, 1e-300))
            assert np.max(np.abs(np.sqrt(g32) - np.sqrt(ref))) < 1e-6
            # the fp64 path's argmin is a valid argmin of the oracle's scores
            # (equal to rounding: several candidates can tie, e.g. d = 1)
            c = int(np.argmin(g64))
            assert ref[c] <= ref.min() * (1 + 1e-12)
            if np.sort(ref)[1] > ref.min() * (1 + 1e-9):   # unique minimum
                assert c == int(np.argmin(ref))


def test_scores_full_size_sampled():
    """d=8, N=64, K=4096 and d=32, N=1024: sampled candidates, fp32 vs oracle."""
    for d, N, c0, cnt in ((8, 64, 4000, 16), (32, 1024, 1020, 2)):
        with T.Search(N, d, 5, precision="fp32", K=cnt) as s:
            phi0 = s.get_phi()
            ref = O.score(phi0, 5, 0.1, 9, c0, cnt, nthreads=4)
            g32 = s.score(9, c0, cnt, 0.1, "fp32")
            assert np.max(np.abs(np.sqrt(g32) - np.sqrt(ref))) < 1e-6


# ------------------------------------------------------------- trajectories

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fp64_trajectory_matches_oracle_tetrahedral(seed):
    """Config d=2, N=4, K=256, Delta0=0.1, 2000 iterations, binary64: identical
    argmin and accept sequence, final mu equal to 1e-12 and within 1e-5 of
    1/sqrt(3)."""
    opts = O.make_opts(K=256, T=2000)
    ophi, om2, odl, otr = O.run(4, 2, seed, opts)
    with T.Search(4, 2, seed, K=256, precision="fp64", trace_cap=2000) as s:
        info = s.step(2000)
        tr = s.trace()
        mu_cert, welch = s.coherence()
    assert info.iters_done == 2000 and len(tr) == 2000
    assert np.array_equal(tr["cstar"], otr["cstar"])
    assert np.array_equal(tr["accepted"], otr["accepted"])
    assert np.allclose(tr["mu2_cur"], otr["mu2_cur"], rtol=1e-12, atol=0)
    assert np.allclose(tr["delta_next"], otr["delta_next"], rtol=1e-12, atol=0)
    assert abs(info.mu - np.sqrt(om2)) < 1e-12
    assert abs(mu_cert - 1 / np.sqrt(3)) < 1e-5 and abs(welch - 1 / np.sqrt(3)) < 1e-15


@pytest.mark.parametrize("d,N,K,iters", [(3, 7, 128, 150), (5, 17, 64, 100), (3, 2, 8, 20)])
def test_fp64_trajectory_matches_oracle_other_shapes(d, N, K, iters):
    seed = 31
    opts = O.make_opts(K=K, T=iters)
    ophi, om2, odl, otr = O.run(N, d, seed, opts, nthreads=4)
    with T.Search(N, d, seed, K=K, precision="fp64") as s:
        s.step(iters)
        tr = s.trace()
        phi = s.get_phi()
    assert np.array_equal(tr["cstar"], otr["cstar"])
    assert np.array_equal(tr["accepted"], otr["accepted"])
    assert np.abs(phi - ophi).max() < 1e-12


def test_fp32_run_decisions_replay_in_fp64():
    """The fp32 path's choices, replayed by the oracle in binary64, give the
    same accept decisions while the improvements exceed fp32 resolution."""
    d, N, K, iters, seed = 4, 12, 256, 40, 8
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        s.step(iters)
        tr = s.trace()
        mu_cert, _ = s.coherence()
        phi = s.get_phi()
    opts = O.make_opts(K=K, T=iters)
    rphi, rm2, rdl, rtr = O.replay(phi0, seed, opts, 0.1, O.mu2(phi0), 0, tr["cstar"])
    gaps = np.abs(np.sqrt(rtr["mu2_best"]) - np.sqrt(np.maximum(rtr["mu2_cur"], 0)))
    clear = gaps > 1e-5
    assert np.array_equal(tr["accepted"][clear], rtr["accepted"][clear])
    assert np.max(np.abs(np.sqrt(tr["mu2_best"]) - np.sqrt(rtr["mu2_best"]))) < 1e-6
    # coherence() certifies the frame after renormalising it in binary64
    assert abs(mu_cert - O.mu(phi / np.linalg.norm(phi, axis=0))) < 1e-12


def test_checkpoint_resume_is_bitwise():
    for prec in ("fp64", "fp32"):
        with T.Search(9, 3, 4, K=64, precision=prec) as a:
            a.step(30)
            blob = a.get_state()
            a.step(25)
            pa = a.get_phi()
            ta = a.trace(25)
        with T.Search(9, 3, 4, K=64, precision=prec) as b:
            b.set_state(blob)
            b.step(25)
            pb = b.get_phi()
            tb = b.trace(25)
        with T.Search(9, 3, 4, K=64, precision=prec) as c:
            c.step(55)
            pc = c.get_phi()
        assert np.array_equal(pa, pb) and np.array_equal(pa, pc)
        assert np.array_equal(ta, tb)


def test_set_phi_and_coherence():
    phi = F.hesse_sic_3_9()
    with T.Search(9, 3, 1) as s:
        s.set_phi(phi * 3.0)             # renormalised on the way in
        mu, w = s.coherence()
        assert abs(mu - 0.5) < 1e-12 and abs(w - 0.5) < 1e-15
        assert np.abs(s.get_phi() - phi).max() < 1e-14
        bad = phi.copy()
        bad[:, 4] = 0
        with pytest.raises(T.TrstmiError):
            s.set_phi(bad)


def test_target_stops_early():
    with T.Search(4, 2, 1, K=128, target_mu=0.6) as s:
        info = s.step(2000)
        assert info.done == 1 and info.iters_done < 2000 and info.mu <= 0.6
        more = s.step(10)
        assert more.iters_done == 0


def test_degenerate_shapes():
    with T.Search(5, 1, 3, K=16) as s:          # C^1: mu = 1 always
        s.step(5)
        assert abs(s.coherence()[0] - 1.0) < 1e-15
    with T.Search(3, 6, 3, K=64) as s:          # N <= d: optimum is 0
        s.step(300)
        assert s.coherence()[0] < 1e-3
    with pytest.raises(T.TrstmiError):
        T.Search(1, 3, 0)
    with pytest.raises(T.TrstmiError):
        T.Search(4, 0, 0)
    with pytest.raises(T.TrstmiError):
        T.Search(4, 2, 0, K=0)


# ------------------------------------------------- bf16 tensor-core screen

@pytest.mark.parametrize("d,N,K", [(32, 1024, 6), (32, 300, 16), (7, 129, 16), (2, 4, 64),
                                   (32, 128, 8), (16, 1536, 3), (1, 5, 8), (32, 2, 4)])
def test_screen_scores_match_oracle(d, N, K):
    """bf16 screen (before re-scoring) within 4e-3 of the oracle's mu on the
    same seeded candidates (the target tolerance; the worst-case bound for
    bf16 input rounding of unit columns is 2u + u^2, u = 2^-8, which only
    degenerate frames such as d = 1 approach)."""
    seed = 99
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        for (t, c0, delta) in [(1, 0, 0.1), (4, 77, 0.5)]:
            ref = O.score(phi0, seed, delta, t, c0, K, nthreads=4)
            gbf = s.score(t, c0, K, delta, "bf16")
            assert np.max(np.abs(np.sqrt(gbf) - np.sqrt(ref))) < 4e-3


@pytest.mark.parametrize("d,N,K", [(32, 768, 4), (32, 300, 16), (7, 129, 16), (2, 4, 64),
                                   (1, 5, 8), (32, 2, 4)])
def test_tf32_screen_scores_match_oracle(d, N, K):
    """tf32 screen (fp32 values rounded to 10 mantissa bits, kind::tf32 MMAs)
    within 1e-3 of the oracle's mu on the same seeded candidates."""
    seed = 97
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        for (t, c0, delta) in [(1, 0, 0.1), (3, 40, 0.4)]:
            ref = O.score(phi0, seed, delta, t, c0, K, nthreads=4)
            g = s.score(t, c0, K, delta, "tf32")
            assert np.max(np.abs(np.sqrt(g) - np.sqrt(ref))) < 1e-3


def test_tf32_screen_rejects_shapes_beyond_its_range():
    with T.Search(300, 33, 1, K=4, precision="fp32") as s:
        with pytest.raises(T.TrstmiError) as e:
            s.score(1, 0, 4, 0.1, "tf32")
        assert e.value.status == T.TRSTMI_EUNSUPPORTED


def test_tf32_mode_decisions_replay_exactly():
    """tf32 precision form: screened iterations, fp32 re-score, fp64
    certification; every decision reproduced by the oracle in binary64."""
    d, N, K, iters, seed = 12, 200, 96, 15, 13
    with T.Search(N, d, seed, K=K, precision="tf32", topk=6, screen_min_delta=0.0) as s:
        phi0 = s.get_phi()
        s.step(iters)
        tr = s.trace()
        phi = s.get_phi()
    assert np.all(tr["flags"] & 1 == 1)
    rphi, rm2, _, rtr = O.replay(phi0, seed, O.make_opts(K=K, T=iters), 0.1, O.mu2(phi0), 0,
                                 tr["cstar"])
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    check_precision_form_rows(tr, rtr, d, O.mu2(phi0))
    assert np.abs(phi - rphi).max() < 1e-12


def test_bf16_mode_decisions_replay_exactly():
    """Screen + fp32 top-k + fp64 certification: the certified mu of every
    chosen candidate equals the oracle's binary64 mu of that candidate, and the
    oracle's accept/radius rule reproduces every decision and the final frame."""
    d, N, K, iters, seed = 8, 40, 128, 25, 6
    with T.Search(N, d, seed, K=K, precision="bf16", topk=8) as s:
        phi0 = s.get_phi()
        s.step(iters)
        tr = s.trace()
        phi = s.get_phi()
    opts = O.make_opts(K=K, T=iters)
    rphi, rm2, rdl, rtr = O.replay(phi0, seed, opts, 0.1, O.mu2(phi0), 0, tr["cstar"])
    check_precision_form_rows(tr, rtr, d, O.mu2(phi0))
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    assert np.abs(phi - rphi).max() < 1e-12
    # the fp32 re-score of the winner is within fp32 tolerance of its fp64 mu
    assert np.max(np.abs(np.sqrt(tr["mu2_screen"]) - np.sqrt(rtr["mu2_best"]))) < 1e-6


def test_bf16_mode_full_size_iterations_replay():
    """d=32, N=1024, K=1024 (the precision-form workload): three iterations,
    every decision reproduced by the oracle in binary64."""
    d, N, K, seed = 32, 1024, 1024, 1
    with T.Search(N, d, seed, K=K, precision="bf16") as s:
        phi0 = s.get_phi()
        s.step(3)
        tr = s.trace()
        mu, _ = s.coherence()
    opts = O.make_opts(K=K, T=3)
    rphi, rm2, rdl, rtr = O.replay(phi0, seed, opts, 0.1, O.mu2(phi0), 0, tr["cstar"])
    check_precision_form_rows(tr, rtr, d, O.mu2(phi0))
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    assert abs(mu - np.sqrt(rm2)) < 1e-12


def test_bf16_mode_reaches_tetrahedral_code():
    """Precision form on the pinned case d=2, N=4: final certified mu within
    1e-5 of the oracle's fp64 run, i.e. of 1/sqrt(3)."""
    _, om2, _, _ = O.run(4, 2, 1, O.make_opts(K=256, T=2000))
    with T.Search(4, 2, 1, K=256, precision="bf16") as s:
        s.step(2000)
        mu, w = s.coherence()
        tr = s.trace()
    assert abs(mu - np.sqrt(om2)) < 1e-5 and abs(mu - w) < 1e-5
    # the screen ranked the iterations with delta >= screen_min_delta
    assert np.array_equal(tr["flags"] & 1, (tr["delta_used"] >= 0.01).astype(np.int32))


@pytest.mark.parametrize("d,N,K", [(32, 1024, 4), (7, 129, 16), (2, 4, 64), (16, 1536, 3)])
def test_fp16_screen_scores_match_oracle(d, N, K):
    """fp16 screen within 1e-3 of the oracle's mu (2^-11 input rounding)."""
    seed = 98
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        ref = O.score(phi0, seed, 0.1, 2, 5, K, nthreads=4)
        g16 = s.score(2, 5, K, 0.1, "fp16")
        assert np.max(np.abs(np.sqrt(g16) - np.sqrt(ref))) < 1e-3


# ----------------------------- wide bf16 / fp16 screen: 32 < d <= 64, N <= 768

@pytest.mark.parametrize("precision,tol", [("bf16", 4e-3), ("fp16", 1e-3)])
@pytest.mark.parametrize("d,N,K", [(64, 768, 4), (40, 300, 16), (33, 129, 16), (64, 2, 4),
                                   (48, 700, 6), (64, 130, 8), (63, 5, 32)])
def test_wide_screen_scores_match_oracle(d, N, K, precision, tol):
    """Two 128-byte operand atoms per column (Re 0..63, Im 0..63) and sixteen
    kind::f16 MMAs per tile: the same input-rounding bound as for d <= 32 (the
    error of |G_jk| is bounded by the rounding of unit vectors, whatever d)."""
    seed = 96
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        for (t, c0, delta) in [(1, 0, 0.1), (5, 31, 0.6)]:
            ref = O.score(phi0, seed, delta, t, c0, K, nthreads=4)
            g = s.score(t, c0, K, delta, precision)
            assert np.max(np.abs(np.sqrt(g) - np.sqrt(ref))) < tol


@pytest.mark.parametrize("d,N", [(65, 40), (80, 769), (128, 300)])
def test_wide_screen_rejects_shapes_beyond_its_range(d, N):
    with T.Search(N, d, 1, K=4, precision="fp32") as s:
        for precision in ("bf16", "fp16", "tf32"):
            with pytest.raises(T.TrstmiError) as e:
                s.score(1, 0, 4, 0.1, precision)
            assert e.value.status == T.TRSTMI_EUNSUPPORTED


# ------------------------------- large N: the candidate swept in bands
# Beyond 1536 columns (768 with two operand atoms per column: tf32 and the
# wide bf16 / fp16 formats) a candidate's blocks no longer fit the shared
# memory together: bands of 1280 (512) columns stay resident while the blocks
# to their right stream through, each band regenerating them.  Every tile of
# the upper triangle is still reduced once, with the same input rounding.

@pytest.mark.parametrize("precision,tol", [("bf16", 4e-3), ("fp16", 1e-3), ("tf32", 1e-3)])
@pytest.mark.parametrize("d,N,K", [(32, 2048, 3), (32, 4096, 2), (7, 1700, 4), (32, 1537, 2),
                                   (16, 3001, 2), (1, 2500, 4)])
def test_banded_screen_scores_match_oracle(d, N, K, precision, tol):
    """Screen tolerance as for N <= 1536.  At d = 1 every |G_jk| is the product
    of two rounded column norms, so the rounding errors add up instead of
    averaging out: there the bound itself applies, 2u + u^2 on mu with
    u = 2^-8 for bf16 (8 significand bits)."""
    if d == 1 and precision == "bf16":
        tol = 2 * 2.0 ** -8 + 2.0 ** -16
    seed = 95
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        for (t, c0, delta) in [(1, 0, 0.1), (2, 9, 0.5)]:
            ref = O.score(phi0, seed, delta, t, c0, K, nthreads=16)
            g = s.score(t, c0, K, delta, precision)
            assert np.max(np.abs(np.sqrt(g) - np.sqrt(ref))) < tol


@pytest.mark.parametrize("precision,tol", [("bf16", 4e-3), ("fp16", 1e-3)])
@pytest.mark.parametrize("d,N,K", [(64, 2048, 2), (64, 4096, 1), (40, 1000, 3), (48, 777, 4)])
def test_banded_wide_screen_scores_match_oracle(d, N, K, precision, tol):
    seed = 94
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        ref = O.score(phi0, seed, 0.2, 3, 5, K, nthreads=16)
        g = s.score(3, 5, K, 0.2, precision)
        assert np.max(np.abs(np.sqrt(g) - np.sqrt(ref))) < tol


@pytest.mark.parametrize("precision,d,N", [("bf16", 32, 2048), ("bf16", 64, 2048),
                                           ("tf32", 32, 4096)])
def test_banded_screen_choice_is_valid_among_the_oracle_scores(precision, d, N):
    """The precision form at N = 2048 / 4096: one screened iteration, checked
    against the oracle's scores of all K candidates as at N = 1024."""
    K, seed = 64, 5
    with T.Search(N, d, seed, K=K, precision=precision, topk=4, screen_min_delta=0.0) as s:
        phi0 = s.get_phi()
        s.step(1)
        row = s.trace()[-1]
        assert row["flags"] & 1 == 1
        check_ranking_against_oracle(s, phi0, seed, int(row["t"]), float(row["delta_used"]),
                                     SCREEN_TOL[precision], int(row["cstar"]))


def test_survivor_pair_pass_drawing_its_own_blocks_matches_the_oracle():
    """40 survivors of N = 4096 (32 column blocks each) need more room than the
    survivors' screen blocks may take, so every tile of the survivor pair pass
    draws its own two blocks instead of copying them; the ranking, the listed
    pairs' binary32 re-scores and the choice still match the oracle."""
    d, N, K, seed = 16, 4096, 48, 8
    with T.Search(N, d, seed, K=K, precision="bf16", topk=40, screen_min_delta=0.0) as s:
        phi0 = s.get_phi()
        s.step(1)
        row = s.trace()[-1]
        assert row["flags"] & 1 == 1
        check_ranking_against_oracle(s, phi0, seed, int(row["t"]), float(row["delta_used"]),
                                     SCREEN_TOL["bf16"], int(row["cstar"]))


def test_wide_bf16_mode_decisions_replay_exactly():
    """Precision form at d = 48 (wide screen every iteration, fp32 top-k,
    fp64 certification): every decision reproduced by the oracle in binary64."""
    d, N, K, iters, seed = 48, 300, 96, 12, 17
    with T.Search(N, d, seed, K=K, precision="bf16", topk=6, screen_min_delta=0.0) as s:
        phi0 = s.get_phi()
        s.step(iters)
        tr = s.trace()
        phi = s.get_phi()
    assert np.all(tr["flags"] & 1 == 1)
    rphi, rm2, _, rtr = O.replay(phi0, seed, O.make_opts(K=K, T=iters), 0.1, O.mu2(phi0), 0,
                                 tr["cstar"])
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    check_precision_form_rows(tr, rtr, d, O.mu2(phi0))
    assert np.abs(phi - rphi).max() < 1e-12


def test_overflowing_survivor_pair_lists_fall_back_to_the_full_passes():
    """Two directions, each repeated N/2 times, perturbed at radius 1e-3: every
    pair within a group stays within the screen's bound of the maximum, far
    more than a survivor's pair list holds, so every list overflows.  The
    survivors are then re-scored over all pairs and the winner certified by
    the full binary64 pass (every iteration screens, so there is no filter
    pass); the ranking and every decision still match the oracle."""
    d, N, K, iters, seed, delta0 = 8, 600, 64, 3, 21, 1e-3
    rng = np.random.default_rng(4)
    dirs = rng.standard_normal((d, 2)) + 1j * rng.standard_normal((d, 2))
    dirs /= np.linalg.norm(dirs, axis=0)
    phi0 = np.repeat(dirs, N // 2, axis=1)
    with T.Search(N, d, seed, K=K, precision="bf16", topk=8, screen_min_delta=0.0,
                  delta0=delta0) as s:
        s.set_phi(phi0)
        phi_start = s.get_phi()
        s.step(1)
        row = s.trace()[-1]
        # every pair near |G| = 1, so the screen's maximum collects the largest
        # rounding of many pairs: the bf16 bound 2u + u^2 (u = 2^-8) itself,
        # not the tolerance measured on random frames
        check_ranking_against_oracle(s, phi_start, seed, int(row["t"]), delta0,
                                     2.0 ** -7 + 2.0 ** -16, int(row["cstar"]))
        s.step(iters - 1)
        tr = s.trace()
        phi = s.get_phi()
    assert np.all(tr["flags"] & 1 == 1)
    opts = O.make_opts(K=K, T=iters, delta0=delta0)
    rphi, rm2, _, rtr = O.replay(phi_start, seed, opts, delta0, O.mu2(phi_start), 0,
                                 tr["cstar"])
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    check_precision_form_rows(tr, rtr, d, O.mu2(phi_start))
    assert np.abs(phi - rphi).max() < 1e-12


def test_screen_gate_by_radius():
    """screen_min_delta = 0: every iteration screened; huge: none screened
    (fp32 Gram of all candidates); decisions replay in binary64 either way."""
    d, N, K, iters, seed = 6, 50, 64, 12, 3
    for smd, expect in ((0.0, 1), (1e9, 0)):
        with T.Search(N, d, seed, K=K, precision="fp16", screen_min_delta=smd) as s:
            phi0 = s.get_phi()
            s.step(iters)
            tr = s.trace()
        assert np.all((tr["flags"] & 1) == expect)
        rphi, rm2, _, rtr = O.replay(phi0, seed, O.make_opts(K=K, T=iters), 0.1, O.mu2(phi0), 0,
                                     tr["cstar"])
        assert np.array_equal(tr["accepted"], rtr["accepted"])
        check_precision_form_rows(tr, rtr, d, O.mu2(phi0))


def test_precision_form_rejects_on_fp32_bound_late_in_a_run():
    """Late in a run most survivors are worse than the current frame: those
    are rejected on their binary32 score (no binary64 work), and every
    decision still matches the oracle's binary64 replay."""
    d, N, K, iters, seed = 4, 16, 64, 150, 8
    with T.Search(N, d, seed, K=K, precision="bf16", topk=4) as s:
        phi0 = s.get_phi()
        s.step(iters)
        tr = s.trace()
        phi = s.get_phi()
    rphi, rm2, _, rtr = O.replay(phi0, seed, O.make_opts(K=K, T=iters), 0.1, O.mu2(phi0), 0,
                                 tr["cstar"])
    assert np.array_equal(tr["accepted"], rtr["accepted"])
    assert check_precision_form_rows(tr, rtr, d, O.mu2(phi0)) > 0
    assert np.abs(phi - rphi).max() < 1e-12


# ------------------------- the screen modes' choice against the oracle's K scores

SCREEN_TOL = {"bf16": 4e-3, "fp16": 1e-3, "tf32": 1e-3}


def check_ranking_against_oracle(s, phi0, seed, t, delta, tol, cstar):
    """One screened iteration (candidates of iteration t, radius delta around
    phi0) against the oracle's binary64 scores of all K candidates:
    * every screen score within the screen tolerance of the oracle's mu;
    * the survivors are exactly the topk smallest screen scores (ties to the
      lowest index), in increasing order;
    * their binary32 re-scores within 1e-6 of the oracle's mu, and the chosen
      candidate is the best of them (ties to the lowest index);
    * the choice is a valid one among all K: its oracle mu is within twice
      the screen tolerance of the oracle's best, and every survivor's oracle
      mu within twice the tolerance of the oracle's topk-th best."""
    scores, surv, top = s.last_ranking()
    K, k = len(scores), len(surv)
    ref = O.score(phi0, seed, delta, t, 0, K, nthreads=16)
    mu, mu_ref = np.sqrt(scores), np.sqrt(ref)
    assert np.max(np.abs(mu - mu_ref)) < tol
    order = np.lexsort((np.arange(K), scores.astype(np.float32)))[:k]
    assert np.array_equal(surv, order)
    assert np.max(np.abs(np.sqrt(top) - mu_ref[surv])) < 1e-6
    best = min(range(k), key=lambda q: (np.float32(top[q]), int(surv[q])))
    assert int(surv[best]) == int(cstar)
    assert mu_ref[cstar] <= mu_ref.min() + 2 * tol
    kth = np.sort(mu_ref)[k - 1]
    assert np.all(mu_ref[surv] <= kth + 2 * tol)
    return mu_ref


@pytest.mark.parametrize("precision,d,N", [("bf16", 32, 1024), ("fp16", 32, 1024),
                                           ("tf32", 32, 768), ("bf16", 64, 768)])
def test_screen_choice_is_valid_among_the_oracle_scores_full_size(precision, d, N):
    """The precision-form workload's shape (K = 1024, top-8): two screened
    iterations, each checked against the oracle's scores of all K candidates."""
    K, seed = 1024, 3
    tol = SCREEN_TOL[precision]
    with T.Search(N, d, seed, K=K, precision=precision, topk=8, screen_min_delta=0.0) as s:
        for _ in range(2):
            phi0 = s.get_phi()
            s.step(1)
            row = s.trace()[-1]
            assert row["flags"] & 1 == 1
            check_ranking_against_oracle(s, phi0, seed, int(row["t"]), float(row["delta_used"]),
                                         tol, int(row["cstar"]))


@pytest.mark.parametrize("precision", ["bf16", "fp16", "tf32"])
def test_screen_choice_when_candidates_nearly_tie(precision):
    """A radius far below the screen's resolution: candidate coherences differ
    by ~1e-5, so the screen's order is mostly rounding and the oracle's best
    candidate usually lies outside the top-2.  The choice must still be one
    of the oracle's near-best (within twice the screen tolerance), and the
    survivors the screen's own two smallest scores."""
    d, N, K, seed = 8, 40, 256, 12
    tol = SCREEN_TOL[precision]
    with T.Search(N, d, seed, K=K, precision=precision, topk=2, screen_min_delta=0.0,
                  delta0=1e-5) as s:
        phi0 = s.get_phi()
        s.step(1)
        row = s.trace()[-1]
        mu_ref = check_ranking_against_oracle(s, phi0, seed, 1, 1e-5, tol, int(row["cstar"]))
    assert np.ptp(mu_ref) < 1e-3


def test_fp32_mode_choice_is_the_oracle_argmin():
    """Binary32 ranking of every candidate (no screen): the chosen candidate's
    oracle mu is within the binary32 tolerance of the oracle's best of K."""
    d, N, K, seed = 16, 300, 512, 4
    with T.Search(N, d, seed, K=K, precision="fp32") as s:
        phi0 = s.get_phi()
        s.step(1)
        row = s.trace()[-1]
        scores, _, _ = s.last_ranking()
    ref = np.sqrt(O.score(phi0, seed, 0.1, 1, 0, K, nthreads=16))
    assert np.max(np.abs(np.sqrt(scores) - ref)) < 1e-6
    c = int(row["cstar"])
    assert c == int(np.lexsort((np.arange(K), scores.astype(np.float32)))[0])
    assert ref[c] <= ref.min() + 2e-6
