"""The trust-region CG-Steihaug procedure on the GPU against the oracle.

Both sides run the same sequence (smoothing stages, trust-region loop,
CG-Steihaug steps) in binary64 with the model's B the exact Hessian of F
(the paper's B_k = grad^2 f_k; Algorithm "Trust-Region CG-Steihaug"): the
Hessian products are the chain rule through the normalisation, the Gram
entries and the softmax weights on both sides.  They differ only in the order
of their sums (a few units in the last place per operation), so rows are
compared while |grad F| > 1e-8: F, s and the radius to 1e-10 relative, the
discrete decisions (CG iterations and exit, accept) exactly, and |grad F| to
1e-7 relative plus 1e-9 absolute: the iterates agree to ~1e-12, and near a
stationary point of a small-delta stage the Hessian's norm (~1/delta, up to
1e4) carries that into the gradient, a difference of nearly equal sums.  The central-difference option (hessian="difference", step h = 1e-6)
is held to the oracle's central differences: their sums' rounding is
amplified by 1/h, so its rows are compared while |grad F| > 1e-5, F and s to
1e-8, |grad F| to 1e-4.  The end points are compared through their coherence.
"""
import numpy as np
import pytest

import frames as F
import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")

SCHEDULE = (0.1, 0.03, 0.01, 0.003, 0.001, 3e-4, 1e-4)
# (gradient floor of the compared rows, rel. tol. of F / s / radius, rel. and
# abs. tol. of |grad F|)
TOL = {"exact": (1e-8, 1e-10, 1e-7, 1e-9), "difference": (1e-5, 1e-8, 1e-4, 0.0)}


def _start(d, N, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((d, N)) + 1j * rng.standard_normal((d, N))
    return z / np.linalg.norm(z, axis=0, keepdims=True)


def _compare_rows(tr, otr, hessian):
    gfloor, rel, grel, gabs = TOL[hessian]
    k = 0
    while (k < min(len(tr), len(otr)) and otr["gnorm"][k] > gfloor
           and tr["stage"][k] == otr["stage"][k]):
        a, b = tr[k], otr[k]
        assert a["F"] == pytest.approx(b["F"], rel=rel), k
        assert a["s"] == pytest.approx(b["s"], rel=rel), k
        assert a["gnorm"] == pytest.approx(b["gnorm"], rel=grel, abs=gabs), k
        assert a["radius"] == pytest.approx(b["radius"], rel=rel), k
        assert (a["cg_iters"], a["cg_status"], a["accepted"]) == \
            (b["cg_iters"], b["cg_status"], b["accepted"]), k
        k += 1
    return k


@pytest.mark.parametrize("hessian", ["exact", "difference"])
@pytest.mark.parametrize("path", [1, 2])       # 1: stack driven from the host; 2: resident
@pytest.mark.parametrize("d,N,seed", [(2, 4, 1), (3, 7, 1), (3, 9, 2), (4, 8, 3), (2, 5, 4)])
def test_trace_matches_oracle(d, N, seed, path, hessian):
    v = _start(d, N, seed)
    phi, tr = T.tr_solve(v, deltas=SCHEDULE, max_outer=100, max_cg=200, path=path,
                         hessian=hessian)
    ophi, otr = O.tr_solve(v, O.tr_opts(deltas=SCHEDULE, max_outer=100, max_cg=200,
                                        hessian=hessian))
    assert _compare_rows(tr, otr, hessian) >= 5
    assert np.sqrt(O.mu2(phi)) == pytest.approx(np.sqrt(O.mu2(ophi)), abs=1e-6)


@pytest.mark.parametrize("path", [1, 2])
def test_hessian_products_on_a_larger_frame_match_the_oracle(path):
    """d = 6, N = 30 (several warps of pairs and columns): the first stage's
    rows, each with dozens of exact Hessian products, as the oracle takes them."""
    v = _start(6, 30, 5)
    kw = dict(deltas=(0.03, 0.01), max_outer=15, max_cg=80)
    _, tr = T.tr_solve(v, path=path, **kw)
    _, otr = O.tr_solve(v, O.tr_opts(**kw))
    assert _compare_rows(tr, otr, "exact") >= 10
    assert tr["cg_iters"][:10].sum() >= 20


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("d,N,seed", [(4, 16, 0), (5, 25, 1)])
def test_reaches_the_sics(d, N, seed, path):
    phi, tr = T.tr_solve(_start(d, N, seed), deltas=SCHEDULE, path=path)
    assert np.sqrt(O.mu2(phi)) == pytest.approx(F.welch(N, d), abs=1e-6)
    assert np.allclose(np.linalg.norm(phi, axis=0), 1.0, atol=1e-14)


@pytest.mark.parametrize("path", [1, 2])
def test_config_shape_d8_n64_descends_and_obeys_the_rules(path):
    v = _start(8, 64, 3)
    mu0 = np.sqrt(O.mu2(v))
    phi, tr = T.tr_solve(v, deltas=(0.03, 0.01, 0.003), max_outer=40, max_cg=60, path=path)
    mu1 = np.sqrt(O.mu2(phi))
    assert mu1 < mu0 - 0.2
    for a, b in zip(tr[:-1], tr[1:]):
        if a["stage"] != b["stage"]:
            continue
        if a["accepted"]:
            assert b["F"] <= a["F"] + 1e-14
        else:
            assert b["F"] == a["F"]
        assert a["step_norm"] <= a["radius"] * (1 + 1e-12)
    # the first rows as the oracle takes them
    otr = O.tr_solve(v, O.tr_opts(deltas=(0.03,), max_outer=3, max_cg=60))[1]
    for k in range(len(otr)):
        assert tr["F"][k] == pytest.approx(otr["F"][k], rel=1e-8)
        assert tr["cg_iters"][k] == otr["cg_iters"][k]


def test_polishing_a_search_result():
    with T.Search(9, 3, 11, K=64, precision="fp64") as s:
        s.step(20)
        mu_before = s.coherence()[0]
        tr = s.tr_solve(deltas=SCHEDULE)
        mu_after, welch = s.coherence()
        assert len(tr) > 0
        assert mu_after < mu_before
        assert mu_after == pytest.approx(0.5, abs=1e-6)       # the SIC of C^3
        assert np.sqrt(O.mu2(s.get_phi())) == pytest.approx(mu_after, rel=1e-12)


def test_rejects_bad_options():
    v = _start(2, 4, 0)
    for kw in [dict(deltas=()), dict(deltas=(0.1, 0.0)), dict(max_cg=0), dict(eta=0.3),
               dict(radius0=0.0), dict(fd_step=0.0), dict(radius0=2.0, radius_max=1.0),
               dict(path=3), dict(hessian=2)]:
        with pytest.raises(T.TrstmiError) as e:
            T.tr_solve(v, **kw)
        assert e.value.status == T.TRSTMI_EINVAL
    z = v.copy()
    z[:, 1] = 0
    with pytest.raises(T.TrstmiError):
        T.tr_solve(z)


# ----------------------------------------- the whole algorithm: L trials together

def _init(N, d, seed):
    with T.Search(N, d, seed, K=1) as s:
        return s.get_phi()


@pytest.mark.parametrize("path", [1, 2])
def test_trials_advance_together_exactly_as_alone(path):
    N, d, seed0, L = 9, 3, 20, 5
    kw = dict(deltas=(0.1, 0.01, 0.001), max_outer=40, max_cg=50, path=path)
    work = np.zeros((L, 2), dtype=np.int32)
    res, mus, phi, tr = T.tr_multistart(N, d, seed0, L, trace_cap=4096, work=work, **kw)
    assert res.trials == L
    # every CG iteration takes one Hessian product; the winner's rows are its iterations
    assert tuple(work[res.best]) == (len(tr), int(tr["cg_iters"].sum()))
    for i in range(L):
        solo_phi, solo_tr = T.tr_solve(_init(N, d, seed0 + i), **kw)
        assert np.sqrt(O.mu2(solo_phi)) == pytest.approx(mus[i], rel=1e-13)
        assert work[i, 0] == len(solo_tr) and work[i, 1] == solo_tr["cg_iters"].sum()
        if i == res.best:
            assert np.array_equal(solo_phi, phi)
            assert np.array_equal(solo_tr, tr)
    assert res.best == int(np.argmin(mus)) and res.mu == mus[res.best]


def test_trials_match_the_oracle_and_batches_change_nothing():
    N, d, seed0, L = 8, 4, 3, 6
    kw = dict(deltas=SCHEDULE, max_outer=100, max_cg=200)
    a = T.tr_multistart(N, d, seed0, L, **kw)
    b = T.tr_multistart(N, d, seed0, L, batch_cap=4, **kw)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for i in range(L):
        ophi, _ = O.tr_solve(O.init(N, d, seed0 + i), O.tr_opts(deltas=SCHEDULE, max_outer=100,
                                                                 max_cg=200))
        assert a[1][i] == pytest.approx(np.sqrt(O.mu2(ophi)), abs=1e-6)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_the_papers_table_2_shapes_with_2d2_trials(d):
    """Algorithm "TRSTMI optimization steps" with L = 2 d^2 at N = d^2: the
    minimum over the trials is no worse than Table 2 (values rounded up)."""
    table = {2: 0.5774, 3: 0.5001, 4: 0.4473}
    res, mus, phi, _ = T.tr_multistart(d * d, d, 1, 0, deltas=SCHEDULE)
    assert res.trials == 2 * d * d
    assert res.mu <= table[d]
    assert np.sqrt(O.mu2(phi)) == pytest.approx(res.mu, rel=1e-12)


def test_resident_path_refuses_frames_it_cannot_hold():
    with pytest.raises(T.TrstmiError) as e:
        T.tr_solve(_start(32, 300, 0), deltas=(0.1,), max_outer=1, path=2)
    assert e.value.status == T.TRSTMI_EUNSUPPORTED
