"""The paper's smooth maximum on the GPU against the oracle.

F_{s,delta} = s + delta log sum_{j<k} exp((|G_jk|^2 - s)/delta) over the
column-normalised frame of V, s = max |G_jk|^2, and the real gradient in V
(arXiv 2207.06374, Sec. "Optimization procedure"), through the C ABI.

Tolerances.  binary64: F and s to 1e-12 relative, the gradient to 1e-10 of
its largest entry (only the order of the sums differs).  binary32: the
variable is rounded to binary32 and the Gram of unit vectors accumulates 2d
products, so each x = |G|^2 is within dx = 2 (2d + 4) 2^-24 of its binary64
value.  F moves by at most max dx plus delta times the relative error of
S = sum exp((x - s)/delta), whose terms carry 2 dx / delta plus the rounding
of exp: |dF| <= 3 dx + 4 delta 2^-24.  The softmax weights carry a relative
error of 2 dx / delta; G, phi and the block products (sums of at most
2d and 64 terms) add (2d + 128) 2^-24, so the gradient is compared within
4 dx / delta + 4 (2d + 128) 2^-24 of its largest entry.  Each column's
gradient is a projection of 2 sum_j w_jk G_jk phi_j / r_k, of size up to
2 / r_k, so where the exact gradient vanishes (d = 1, equiangular frames)
only rounding noise on that scale is left: every comparison also allows
floor * 2 / r_k per column (floor 1e-14 in binary64, (2d + 128) 2^-24 in
binary32).
"""
import numpy as np
import pytest

import frames as FR
import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")

U = 2.0 ** -24


def _raw(d, N, rng, count=None):
    shape = (d, N) if count is None else (count, d, N)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return z * rng.uniform(0.5, 2.0, size=shape[:-2] + (1, N))


def _close(g, g_o, v, rel, floor):
    """|g - g_o| within rel * max|g_o| plus floor * 2 / r_k in column k."""
    r = np.linalg.norm(v, axis=0)
    lim = rel * np.max(np.abs(g_o)) + floor * 2.0 / r[None, :]
    return bool(np.all(np.abs(g - g_o) <= lim))


def _fp32_tols(d, delta):
    dx = 2 * (2 * d + 4) * U
    return 3 * dx + 4 * delta * U, 4 * dx / delta + 4 * (2 * d + 128) * U


# shapes spanning one to several tiles with ragged tails, d = 1, N = 2, N <= d
SHAPES = [(2, 4), (1, 5), (7, 2), (3, 9), (5, 37), (8, 70), (16, 200), (32, 130), (40, 33),
          (4, 257)]


@pytest.mark.parametrize("d,N", SHAPES)
def test_fp64_matches_oracle(d, N):
    rng = np.random.default_rng(1000 + 7 * d + N)
    v = _raw(d, N, rng, count=3)
    for delta in (0.05, 0.003):
        F, s, g = T.lse(v, delta, "fp64")
        for q in range(3):
            f_o, s_o, g_o = O.lse(v[q], delta)
            assert F[q] == pytest.approx(f_o, rel=1e-12, abs=0)
            assert s[q] == pytest.approx(s_o, rel=1e-13, abs=0)
            assert _close(g[q], g_o, v[q], 1e-10, 1e-14)


@pytest.mark.parametrize("d,N", SHAPES)
def test_fp32_matches_oracle_within_its_bound(d, N):
    rng = np.random.default_rng(2000 + 7 * d + N)
    v = _raw(d, N, rng, count=2)
    delta = 0.05
    tol_f, tol_g = _fp32_tols(d, delta)
    F, s, g = T.lse(v, delta, "fp32")
    for q in range(2):
        f_o, s_o, g_o = O.lse(v[q], delta)
        assert abs(F[q] - f_o) <= tol_f
        assert abs(s[q] - s_o) <= 2 * (2 * d + 4) * U
        assert _close(g[q], g_o, v[q], tol_g, (2 * d + 128) * U)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_frames_against_oracle(precision):
    """The bench's shape (d = 32, N = 1024, several frames per launch): the
    oracle evaluates two of them in full."""
    rng = np.random.default_rng(77)
    v = _raw(32, 1024, rng, count=4)
    delta = 0.01
    F, s, g = T.lse(v, delta, precision)
    n = 1024 * 1023 // 2
    assert np.all(s <= F) and np.all(F <= s + delta * np.log(n) + 1e-12)
    if precision == "fp32":
        tol_f, tol_g = _fp32_tols(32, delta)
        floor = (2 * 32 + 128) * U
    else:
        tol_f, tol_g, floor = 1e-12, 1e-10, 1e-14
    for q in (0, 3):
        f_o, s_o, g_o = O.lse(v[q], delta)
        rel = 1.0 if precision == "fp32" else abs(f_o)
        assert abs(F[q] - f_o) <= tol_f * rel
        assert _close(g[q], g_o, v[q], tol_g, floor)


@pytest.mark.parametrize("make", [FR.tetrahedral_2_4, FR.harmonic_3_7, FR.hesse_sic_3_9])
def test_equiangular_frames_closed_form(make):
    phi = make()
    d, N = phi.shape
    n = N * (N - 1) // 2
    W2 = FR.welch(N, d) ** 2
    for delta in (1e-3, 0.2):
        F, s, g = T.lse(phi, delta, "fp64")
        assert s == pytest.approx(W2, abs=1e-14)
        assert F == pytest.approx(W2 + delta * np.log(n), abs=1e-13)
        assert np.max(np.abs(g)) < 1e-13


def test_scaling_columns_by_powers_of_two_changes_nothing():
    rng = np.random.default_rng(5)
    v = _raw(6, 90, rng)
    c = 2.0 ** rng.integers(-3, 4, size=(1, 90))
    F0, s0, g0 = T.lse(v, 0.02, "fp64")
    F1, s1, g1 = T.lse(v * c, 0.02, "fp64")
    assert F0 == F1 and s0 == s1
    assert np.array_equal(g1 * c, g0)     # grad scales by 1/c exactly


def test_results_are_deterministic():
    rng = np.random.default_rng(6)
    v = _raw(16, 300, rng, count=5)
    a = T.lse(v, 0.01, "fp32")
    b = T.lse(v, 0.01, "fp32")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


def test_device_entry_point_matches_host_entry_point():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    count, d, N = 3, 12, 150
    v = _raw(d, N, rng, count=count)
    F_h, s_h, g_h = T.lse(v, 0.04, "fp32")
    flat = np.ascontiguousarray(np.transpose(v, (0, 2, 1))).view(np.float64).reshape(-1)
    dev = torch.device("cuda:0")
    v_t = torch.from_numpy(flat.copy()).to(dev)
    nbytes = T.lse_scratch_bytes(N, d, count, "fp32")
    scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = scratch.data_ptr()
    aligned = (base + 255) // 256 * 256
    out = torch.zeros(2 * count, dtype=torch.float64, device=dev)
    grad = torch.zeros_like(v_t)
    stream = torch.cuda.current_stream(dev)
    T.lse_device(N, d, count, v_t.data_ptr(), 0.04, "fp32", aligned, nbytes, out.data_ptr(),
                 grad.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    o = out.cpu().numpy().reshape(count, 2)
    g = grad.cpu().numpy().view(np.complex128).reshape(count, N, d).transpose(0, 2, 1)
    assert np.array_equal(o[:, 0], F_h) and np.array_equal(o[:, 1], s_h)
    assert np.array_equal(g, g_h)


def test_rejects_bad_arguments_and_zero_columns():
    rng = np.random.default_rng(9)
    v = _raw(3, 6, rng)
    for bad in [dict(delta=0.0), dict(delta=-1.0), dict(delta=float("inf")),
                dict(precision="bf16")]:
        kw = dict(delta=0.1, precision="fp64")
        kw.update(bad)
        with pytest.raises(T.TrstmiError) as e:
            T.lse(v, kw["delta"], kw["precision"])
        assert e.value.status == T.TRSTMI_EINVAL
    with pytest.raises(T.TrstmiError):
        T.lse(v[:, :1], 0.1)
    z = v.copy()
    z[:, 4] = 0
    with pytest.raises(T.TrstmiError) as e:
        T.lse(z, 0.1)
    assert e.value.status == T.TRSTMI_EINVAL
