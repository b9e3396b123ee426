"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, exact algebraic identities of Section 4, brute force, textbook
routines other than the ones the oracle calls, and stated properties of the
estimator.  A dropped term, a wrong sign, index or transposed operand anywhere
in ``oracle/mrq.py`` fails at least one of these."""
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import datagen
from oracle import mrq, index_file

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, rest = line.split("=", 1)
            vals[key.strip()] = np.array([float(t) for t in rest.split()])
    return vals


# ----------------------------------------------------------------- PCA (Alg. 1)

def test_pca_against_svd_and_closed_form():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3000, 12)) * np.linspace(3, 0.2, 12) + 7.0
    mu, lam, Pp = mrq.pca_train(X)
    Xc = X - X.mean(axis=0)
    # independent route: singular values of the centred data
    sv = np.linalg.svd(Xc, compute_uv=False)
    np.testing.assert_allclose(lam, sv ** 2 / X.shape[0], rtol=1e-10)
    np.testing.assert_allclose(Pp @ Pp.T, np.eye(12), atol=1e-12)
    cov = Xc.T @ Xc / X.shape[0]
    np.testing.assert_allclose(Pp.T @ np.diag(lam) @ Pp, cov, atol=1e-10 * np.abs(cov).max())
    # sign convention: largest-magnitude entry of each row is positive
    for row in Pp:
        assert row[np.argmax(np.abs(row))] > 0


def test_pca_exact_small_case():
    # four points +-a e1, +-b e2 (plus a mean offset): covariance diag(a^2/2, b^2/2)
    a, b = 3.0, 1.0
    X = np.array([[a, 0], [-a, 0], [0, b], [0, -b]]) + np.array([10.0, -4.0])
    mu, lam, Pp = mrq.pca_train(X)
    np.testing.assert_allclose(mu, [10.0, -4.0])
    np.testing.assert_allclose(lam, [a * a / 2, b * b / 2], rtol=1e-14)
    np.testing.assert_allclose(Pp, np.eye(2), atol=1e-14)


def test_orthogonal_from_gaussian():
    G = datagen.rotation_gaussian(32, 11)
    P = mrq.orthogonal_from_gaussian(G)
    np.testing.assert_allclose(P.T @ P, np.eye(32), atol=1e-12)
    R = P.T @ G                              # G = P R with R upper triangular, diag > 0
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-10)
    assert np.all(np.diag(R) > 0)


# ---------------------------------------------------------------------- k-means

def test_kmeans_hand_example():
    X = np.array([[0.0], [1.0], [10.0], [11.0], [12.0]])
    C, a = mrq.kmeans(X, np.array([[0.0], [5.0]]), iters=1)
    # assignment to (0, 5): {0, 1} -> 0, {10, 11, 12} -> 1; means 0.5 and 11
    np.testing.assert_allclose(C[:, 0], [0.5, 11.0])
    assert a.tolist() == [0, 0, 1, 1, 1]
    # tie goes to the lower id; an empty list keeps its centroid
    C2, a2 = mrq.kmeans(np.array([[1.0]]), np.array([[0.0], [2.0], [9.0]]), iters=1)
    assert a2.tolist() == [0]
    np.testing.assert_allclose(C2[:, 0], [1.0, 2.0, 9.0])


def test_kmeans_final_assignment_is_nearest():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, 4))
    C, a = mrq.kmeans(X, X[:7], iters=5)
    np.testing.assert_array_equal(a, np.argmin(cdist(X, C, "sqeuclidean"), axis=1))


# ----------------------------------------------------------------- quantization

def test_encode_golden():
    g = _load_golden("encode_examples.txt")
    u1, v1 = mrq.encode(g["o_1bit"][None, :], 1)
    np.testing.assert_array_equal(u1[0], g["u_1bit"])
    np.testing.assert_array_equal(v1[0], g["v_1bit"])
    u2, v2 = mrq.encode(g["o_2bit"][None, :], 2)
    np.testing.assert_array_equal(u2[0], g["u_2bit"])
    np.testing.assert_array_equal(v2[0], g["v_2bit"])
    u3, v3 = mrq.encode(g["o_3bit"][None, :], 3)
    np.testing.assert_array_equal(u3[0], g["u_3bit"])
    np.testing.assert_array_equal(v3[0], g["v_3bit"])


def test_factor_closed_form_one_hot():
    # o' = e_1 in d dims: <v, o'> = 1 and <v,o'>/|v| = 1/sqrt(d), so
    # f_rescale = -2 r and f_err = 2 r sqrt((1 - 1/d) d)/sqrt(d - 1) = 2 r.
    d, r = 64, 2.5
    o = np.zeros((1, d)); o[0, 0] = 1.0
    u, v = mrq.encode(o, 1)
    f_add, f_res, f_err, ip = mrq.factors(np.array([r]), np.array([0.75]), v, o, d)
    assert ip[0] == pytest.approx(1.0)
    assert f_add[0] == pytest.approx(r * r + 0.75)
    assert f_res[0] == pytest.approx(-2 * r)
    assert f_err[0] == pytest.approx(2 * r, rel=1e-12)


def test_quantize_query_golden_and_grid_identity():
    g = _load_golden("query_quant_examples.txt")
    qbar, lo, delta = mrq.quantize_query(g["qprime"], 2)
    np.testing.assert_array_equal(qbar, g["qbar_2bit"])
    assert lo == pytest.approx(g["vl"][0]) and delta == pytest.approx(g["delta"][0])
    # on-grid query: the quantized inner-product identity is exact
    rng = np.random.default_rng(1)
    for bits in (1, 2, 4):
        d = 64
        top = (1 << bits) - 1
        u = rng.integers(0, top + 1, size=(50, d))
        v = 2 * u - top
        qb = rng.integers(0, 16, size=d); qb[0], qb[1] = 0, 15
        vl, dl = -0.375, 0.0625                      # exact in binary
        qp = vl + dl * qb
        direct = v @ qp
        formula = dl * (2.0 * (u @ qb) - top * qb.sum()) + vl * (2.0 * u.sum(axis=1) - d * top)
        np.testing.assert_allclose(formula, direct, rtol=0, atol=1e-12)


def _tiny_list_index(u, bits, f_add, f_rescale, f_err, centroid):
    """A one-list OracleIndex holding just what Eq. 4 / Eq. 5 read (hand examples)."""
    u = np.asarray(u, dtype=np.uint8)
    n, d = u.shape
    top = (1 << bits) - 1
    z = np.zeros(n)
    return mrq.OracleIndex(
        D=d, d=d, bits=bits, nlist=1, mu=np.zeros(d), lam=np.zeros(d), Pp=np.eye(d),
        Pr=np.eye(d), W=np.eye(d), centroids=np.asarray(centroid, dtype=np.float64)[None, :],
        list_offsets=np.array([0, n]), ids=np.arange(n), xd=np.zeros((n, d)),
        xr=np.zeros((n, 0)), xnorm2=z, u=u, v=2.0 * u.astype(np.float64) - top,
        f_add=np.asarray(f_add, dtype=np.float64), f_rescale=np.asarray(f_rescale, dtype=np.float64),
        f_err=np.asarray(f_err, dtype=np.float64), ip_vo=z, resid_norm=z)


def test_quantized_estimate_hand_example():
    """Eq. 4 / Eq. 5 through a 2-bit quantized query, every value worked by hand
    (tests/golden/quantized_estimate_example.txt)."""
    g = _load_golden("quantized_estimate_example.txt")
    idx = _tiny_list_index(g["u"].reshape(2, 4), 2, g["f_add"], g["f_rescale"], g["f_err"],
                           np.zeros(4))
    args = (idx, 0, g["qd"], float(g["g"][0]), float(g["qr2"][0]), float(g["sigma"][0]),
            float(g["eps0"][0]), float(g["m"][0]))
    for qbits in (2, 0):                        # on the grid both branches agree exactly
        e = mrq.estimate_list(*args, qbits=qbits)
        np.testing.assert_allclose(e["ip"], g["ip"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(e["dis"], g["dis"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(e["lb"], g["lb"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(e["ub"], g["ub"], rtol=0, atol=1e-14)
        if qbits:
            np.testing.assert_array_equal(e["qbar"], g["qbar"])
            np.testing.assert_array_equal(e["int_dot"], g["int_dot"])
            assert e["vl"] == g["vl"][0] and e["delta"] == g["delta"][0]


@pytest.fixture(scope="module")
def multibit_indices():
    """One small workload encoded with 1, 2 and 4 bits per dimension (same rotation, IVF)."""
    w = datagen.workload("small", n=4000, n_comp=16, nlist=8, n_query=20)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 17)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 18)
    out = {b: mrq.build_index(base, w.d, b, w.nlist, G, init_idx=init, kmeans_iters=4)
           for b in (1, 2, 4)}
    return w, queries, out


@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("qbits", [2, 4])
def test_quantized_estimate_on_grid_is_exact(multibit_indices, bits, qbits):
    """When q' lies on the query grid (v_l and delta exact in binary), the quantized
    branch of Eq. 4 must give <v, q'> itself: the code values of the stored levels
    (v = 2u - (2^B - 1)) against q', summed directly here; the integer dot is <u, qbar>."""
    w, queries, idxs = multibit_indices
    idx = idxs[bits]
    top_q = (1 << qbits) - 1
    rng = np.random.default_rng(100 * bits + qbits)
    for j in range(idx.nlist):
        sl = idx.list_slice(j)
        if sl.stop == sl.start:
            continue
        qb = rng.integers(0, top_q + 1, size=idx.d)
        qb[rng.integers(idx.d)] = 0
        qb[(rng.integers(idx.d - 1) + 1 + int(np.argmin(qb))) % idx.d] = top_q
        vl, dl = -0.625, 2.0 ** -(qbits + 1)          # exact in binary
        qgrid = vl + dl * qb
        gj = 0.25                                     # sqrt(g) = 0.5, exact
        qd = idx.centroids[j] + 0.5 * qgrid
        e = mrq.estimate_list(idx, j, qd, gj, 0.3, 0.2, 1.9, 4.0, qbits=qbits)
        np.testing.assert_array_equal(e["qbar"], qb)
        assert e["vl"] == vl and e["delta"] == dl
        u = idx.u[sl].astype(np.int64)
        np.testing.assert_array_equal(e["int_dot"], u @ qb)
        top = (1 << bits) - 1
        v = 2 * u - top
        direct = np.array([sum(float(v[r, i]) * qgrid[i] for i in range(idx.d))
                           for r in range(u.shape[0])])
        np.testing.assert_allclose(e["ip"], direct, rtol=0, atol=1e-12)
        want = idx.f_add[sl] + gj + 0.3 + idx.f_rescale[sl] * 0.5 * direct
        np.testing.assert_allclose(e["dis"], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bits", [1, 4])
def test_quantized_estimate_off_grid_is_the_dequantized_query(multibit_indices, bits):
    """Off the grid, the quantized branch equals <v, q_hat'> for the dequantized query
    q_hat' = v_l + delta*qbar, and q_hat' is within delta/2 of q' in every coordinate
    (round to nearest on a min/max grid with 2^B_q levels)."""
    w, queries, idxs = multibit_indices
    idx = idxs[bits]
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, queries[:6])
    top = (1 << bits) - 1
    for i in range(6):
        lists, g = mrq.probe(idx, qd[i], 3)
        for j in lists:
            j = int(j)
            sl = idx.list_slice(j)
            e = mrq.estimate_list(idx, j, qd[i], float(g[j]), qr2[i], sigma[i], 1.9, 4.0, qbits=4)
            qprime = (qd[i] - idx.centroids[j]) / math.sqrt(g[j])
            qhat = e["vl"] + e["delta"] * e["qbar"].astype(np.float64)
            assert e["qbar"].min() == 0 and e["qbar"].max() == 15
            assert np.max(np.abs(qhat - qprime)) <= 0.5 * e["delta"] * (1 + 1e-5) + 1e-7
            v = 2.0 * idx.u[sl].astype(np.float64) - top
            np.testing.assert_allclose(e["ip"], v @ qhat, rtol=0,
                                       atol=1e-12 * (1 + np.abs(v).sum(axis=1).max()))


# ------------------------------------------- decision margin (which queries are strict)

def test_decision_margin_hand_example():
    """k = 2, four candidates with scale 10: tau = 2.0 (2nd smallest UB).
    |lb - tau|/10 = .15 .05 .09 .2; the 2nd/3rd UB gap is (3 - 2)/3 = 1/3, which
    protects the two candidates inside the k smallest UBs (lb <= ub <= tau), so their
    margins are 1/3, 1/3; the others keep .09 and .2."""
    lb = np.array([0.5, 1.5, 2.9, 4.0])
    ub = np.array([1.0, 2.0, 3.0, 5.0])
    sc = np.full(4, 10.0)
    allrel = np.ones(4, dtype=bool)
    assert mrq._decision_margin(lb, ub, sc, 2.0, 2, allrel) == pytest.approx(0.09, rel=1e-12)
    assert mrq._decision_margin(lb, ub, sc, 2.0, 2, np.array([1, 1, 0, 1], bool)) == \
        pytest.approx(0.2, rel=1e-12)
    assert mrq._decision_margin(lb, ub, sc, 2.0, 2, np.array([1, 1, 0, 0], bool)) == \
        pytest.approx(1.0 / 3.0, rel=1e-12)
    # per-candidate scales divide each candidate's own gap: (2.9 - 2)/... at scale 1
    sc2 = np.array([10.0, 10.0, 1.0, 10.0])
    assert mrq._decision_margin(lb, ub, sc2, 2.0, 2, allrel) == pytest.approx(0.2, rel=1e-12)


def test_decision_margin_zero_width_bounds():
    """d = D: lb = ub.  k = 1, bounds 1, 1.001, 4 and tau = 1: the first candidate sits
    exactly on tau (|lb - tau| = 0), yet it stays selected until the 1st/2nd upper-bound
    gap (0.001/1.001) closes, so the margin is that gap, not 0."""
    b = np.array([1.0, 1.001, 4.0])
    mg = mrq._decision_margin(b, b, np.ones(3), 1.0, 1, np.ones(3, dtype=bool))
    assert mg == pytest.approx(0.001 / 1.001, rel=1e-12)
    # fewer than k + 1 candidates: no (k+1)-th bound can displace them
    assert mrq._decision_margin(b[:1], b[:1], np.ones(1), 1.0, 1, np.ones(1, bool)) == math.inf


def test_margin_covers_bound_perturbations(small_workload, small_oracle_index, monkeypatch):
    """The margin is the promise the GPU parity tests rely on: moving every bound (and
    every estimate) of a query by less than a fraction of its margin must leave that
    query's answer unchanged.  Two kinds of move: random ones (estimates, bound widths,
    sigma), and an adversarial one that pushes every stage-1 lower bound toward
    tau_A (up when selected, capped at the candidate's own upper bound; down when not),
    the move that flips the closest stage-1 decision first."""
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:30]
    k, nprobe, kw = w.k, w.nprobe, dict(eps0=1.0, m=1.0, qbits=4)
    ref = mrq.search_contract(idx, Q, k, nprobe, **kw)
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, Q)
    orig_est = mrq.estimate_list
    orig_proj = mrq.project_queries
    rng = np.random.default_rng(7)
    st = {"a": 0.0, "tau": None}

    def noisy_est(*a, **kk):
        e = dict(orig_est(*a, **kk))
        n = e["dis"].shape[0]
        if st["tau"] is not None:                    # adversarial: toward tau_A
            up = e["lb"] <= st["tau"]
            e["lb"] = np.where(up, np.minimum(e["lb"] + st["a"], e["ub"]), e["lb"] - st["a"])
            return e
        shift = rng.uniform(-0.5, 0.5, n) * st["a"]
        widen = rng.uniform(-0.5, 0.5, n) * st["a"]
        e["dis"] = e["dis"] + shift
        e["lb"] = e["lb"] + shift - widen
        e["ub"] = e["ub"] + shift + widen
        return e

    def noisy_proj(idx_, Q_):
        qd_, qr_, qr2_, sig_, qp2_ = orig_proj(idx_, Q_)
        if st["tau"] is not None:
            return qd_, qr_, qr2_, sig_, qp2_
        # moves every stage-2 bound (and stage-1 eps_r) by m * d_sigma <= a/4
        return qd_, qr_, qr2_, sig_ + st["a"] * 0.25 * rng.uniform(-1, 1, sig_.shape), qp2_

    checked = 0
    for i in range(Q.shape[0]):
        if not math.isfinite(ref.margin[i]):
            continue
        lists, g = mrq.probe(idx, qd[i], nprobe)
        pos = np.concatenate([np.arange(*idx.list_slice(int(j)).indices(idx.n)) for j in lists])
        ub = np.concatenate([orig_est(idx, int(j), qd[i], float(g[j]), qr2[i], sigma[i], 1.0, 1.0,
                                      qbits=4)["ub"] for j in lists])
        tau_a = float(np.sort(ub)[k - 1])
        s_min = min(float(np.min(idx.f_add[pos])) + float(g[lists].min()) + qr2[i],
                    float(np.min(idx.xnorm2[pos])) + qp2[i], float(ref.dists[i, k - 1]))
        monkeypatch.setattr(mrq, "estimate_list", noisy_est)
        monkeypatch.setattr(mrq, "project_queries", noisy_proj)
        for trial in range(3):
            st["a"] = 0.1 * ref.margin[i] * s_min
            st["tau"] = tau_a if trial == 0 else None
            r = mrq.search_contract(idx, Q[i:i + 1], k, nprobe, **kw)
            assert r.ids[0].tolist() == ref.ids[i].tolist(), (i, trial, ref.margin[i])
        monkeypatch.undo()
        checked += 1
    assert checked >= 25

# --------------------------------------------- decomposition identities (Eq. 1-3)

def test_eq3_decomposition_exact(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, queries[:20])
    rng = np.random.default_rng(0)
    pos = rng.integers(0, idx.n, size=300)
    assign = np.searchsorted(idx.list_offsets, pos, side="right") - 1
    X = base[idx.ids[pos]].astype(np.float64)
    for i in range(20):
        c = idx.centroids[assign]
        xr = idx.xr[pos]
        xb = (idx.xd[pos] - c) / idx.resid_norm[pos][:, None]
        qdc = qd[i][None, :] - c
        qn = np.linalg.norm(qdc, axis=1)
        qb = qdc / qn[:, None]
        C1 = idx.resid_norm[pos] ** 2 + qn ** 2 + np.sum(xr * xr, axis=1) + qr2[i]
        C2 = -2 * idx.resid_norm[pos] * qn * np.sum(xb * qb, axis=1)
        C3 = -2 * (xr @ qr[i])
        true = np.sum((X - queries[i].astype(np.float64)) ** 2, axis=1)
        np.testing.assert_allclose(C1 + C2 + C3, true, rtol=1e-9)
        # Eq. 4 with the estimator replaced by the exact <x_b, q_b>, plus C3, is exact
        op = np.sum(xb * qb, axis=1)
        est = idx.f_add[pos] + qn ** 2 + qr2[i] + idx.f_rescale[pos] * qn * idx.ip_vo[pos] * op + C3
        np.testing.assert_allclose(est, true, rtol=1e-9)
        # Eq. 7 differs from the exact distance by the residual cross term only
        diso = idx.xnorm2[pos] + qp2[i] - 2 * (idx.xd[pos] @ qd[i])
        np.testing.assert_allclose(diso + C3, true, rtol=1e-9)


def test_residual_variance_identity_and_chebyshev(small_workload, small_oracle_index):
    # Eq. 6 over the centred base set holds exactly: Var_x <x_r, q_r> = sum q_i^2 lam_i
    w, base, queries = small_workload
    idx = small_oracle_index
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, queries[:10])
    xr_all = idx.xr
    for i in range(10):
        t = xr_all @ qr[i]
        assert abs(t.mean()) < 1e-9 * (np.abs(t).max() + 1)
        np.testing.assert_allclose(t.var(), sigma[i] ** 2, rtol=1e-9)
        for m in (1.5, 2.0, 4.0):                         # Chebyshev
            assert np.mean(np.abs(t) >= m * sigma[i]) <= 1.0 / m ** 2


def test_tail_vanishes_when_d_equals_D():
    w = datagen.workload("small", n=3000, D=64, n_comp=16)
    base, queries = datagen.base_and_queries(w, n_query=5)
    G = datagen.rotation_gaussian(64, 1)
    idx = mrq.build_index(base, 64, 1, 8, G, init_idx=np.arange(8), kmeans_iters=3)
    assert idx.xr.shape[1] == 0
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, queries)
    assert np.all(sigma == 0) and np.all(qr2 == 0)
    np.testing.assert_allclose(idx.f_add, idx.resid_norm ** 2)
    # the estimate is the pure RaBitQ estimate |x-c|^2 + |q-c|^2 - 2|x-c||q-c|<v,q'>/<v,o'>
    lists, g = mrq.probe(idx, qd[0], 1)
    j = int(lists[0])
    e = mrq.estimate_list(idx, j, qd[0], float(g[j]), 0.0, 0.0, 1.9, 4.0)
    sl = idx.list_slice(j)
    qprime = (qd[0] - idx.centroids[j]) / math.sqrt(g[j])
    rabitq = (idx.resid_norm[sl] ** 2 + g[j]
              - 2 * idx.resid_norm[sl] * math.sqrt(g[j]) * (idx.v[sl] @ qprime) / idx.ip_vo[sl])
    np.testing.assert_allclose(e["dis"], rabitq, rtol=1e-12)
    np.testing.assert_allclose(e["ub"] - e["dis"], 1.9 * math.sqrt(g[j]) * idx.f_err[sl], rtol=1e-12)


# ----------------------------------------------------- estimator (Section 4.2)

def test_estimator_unbiased_over_rotations():
    # <x_bar, q>/<x_bar, x> is unbiased for <x, q> over the random rotation
    rng = np.random.default_rng(7)
    d = 32
    x = rng.standard_normal(d); x /= np.linalg.norm(x)
    q = rng.standard_normal(d); q = 0.6 * x + 0.8 * q / np.linalg.norm(q); q /= np.linalg.norm(q)
    errs = []
    for s in range(3000):
        P = mrq.orthogonal_from_gaussian(datagen.rotation_gaussian(d, 10_000 + s))
        o = (x @ P)[None, :]                # o' = P^T x
        qq = q @ P
        _, v = mrq.encode(o, 1)
        errs.append((v[0] @ qq) / (v[0] @ o[0]) - x @ q)
    errs = np.array(errs)
    assert abs(errs.mean()) < 3 * errs.std() / math.sqrt(errs.size)


def test_eq5_interval_holds_for_most_rotations():
    # |est - <x,q>| <= sqrt((1 - a^2)/a^2) * eps0/sqrt(d - 1), a = <x_bar, x> (Eq. 5)
    rng = np.random.default_rng(8)
    d, eps0 = 64, 1.9
    x = rng.standard_normal(d); x /= np.linalg.norm(x)
    q = rng.standard_normal(d); q /= np.linalg.norm(q)
    z = []
    for s in range(1500):
        P = mrq.orthogonal_from_gaussian(datagen.rotation_gaussian(d, 20_000 + s))
        o, qq = x @ P, q @ P
        _, v = mrq.encode(o[None, :], 1)
        a = (v[0] @ o) / np.linalg.norm(v[0])
        err = (v[0] @ qq) / (v[0] @ o) - x @ q
        z.append(err / (math.sqrt((1 - a * a) / (a * a)) / math.sqrt(d - 1)))
    z = np.array(z)
    # RaBitQ's analysis: conditioned on a, the error is a (d-1)-sphere coordinate of
    # scale sqrt(1 - a^2)/a * sqrt(1 - <x,q>^2), i.e. z ~ N(0, 1 - <x,q>^2) for large d
    s_theory = math.sqrt(1 - (x @ q) ** 2)
    assert abs(z.std() - s_theory) < 0.06
    from scipy.stats import norm
    p_miss = 2 * norm.sf(eps0 / s_theory)
    assert abs(np.mean(np.abs(z) > eps0) - p_miss) < 0.025


def test_bound_rate_and_multibit_accuracy(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, queries[:30])
    viol = tot = 0
    for i in range(30):
        lists, g = mrq.probe(idx, qd[i], 2)
        for j in lists:
            sl = idx.list_slice(int(j))
            e = mrq.estimate_list(idx, int(j), qd[i], float(g[j]), qr2[i], 0.0, 1.9, 0.0)
            # exact projected distance |x_d - q_d|^2 + |x_r|^2 + |q_r|^2 (C3 excluded)
            ref = np.sum((idx.xd[sl] - qd[i]) ** 2, axis=1) + np.sum(idx.xr[sl] ** 2, axis=1) + qr2[i]
            viol += np.sum((ref < e["lb"]) | (ref > e["ub"]))
            tot += ref.size
    assert viol / tot < 0.08          # Eq. 5's interval with eps0 = 1.9 fails for a few %
    # more bits per dimension -> the estimate approaches the exact inner product
    rng = np.random.default_rng(2)
    o = rng.standard_normal((400, 64)); o /= np.linalg.norm(o, axis=1, keepdims=True)
    q = rng.standard_normal(64); q /= np.linalg.norm(q)
    errs = []
    for b in (1, 2, 4, 8):
        _, v = mrq.encode(o, b)
        est = (v @ q) / np.sum(v * o, axis=1)
        errs.append(np.sqrt(np.mean((est - o @ q) ** 2)))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 0.02 * errs[0]


# -------------------------------------------------------------- search (Alg. 2)

def test_exact_knn_against_cdist():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((700, 9)); Q = rng.standard_normal((13, 9))
    ids, dd = mrq.exact_knn(S, Q, 5)
    D = cdist(Q, S, "sqeuclidean")
    for i in range(13):
        o = np.lexsort((np.arange(700), D[i]))[:5]
        assert ids[i].tolist() == o.tolist()
        np.testing.assert_allclose(dd[i], D[i, o], rtol=1e-12)


def test_probe_ties_to_lower_id():
    idx = mrq.OracleIndex(D=2, d=2, bits=1, nlist=4, mu=None, lam=None, Pp=None, Pr=None, W=None,
                          centroids=np.array([[1.0, 0], [0, 1.0], [-1.0, 0], [5.0, 5.0]]),
                          list_offsets=np.zeros(5, dtype=np.int64), ids=np.zeros(0, dtype=np.int64),
                          xd=None, xr=None, xnorm2=None, u=None, v=None, f_add=None, f_rescale=None,
                          f_err=None, ip_vo=None, resid_norm=None)
    lists, g = mrq.probe(idx, np.zeros(2), 3)
    assert lists.tolist() == [0, 1, 2]


def test_no_pruning_full_probe_is_brute_force(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:12]
    ref_ids, ref_d = mrq.exact_knn(base, Q, w.k)
    for mode in (mrq.MODE_MRQ, mrq.MODE_MRQ_PLUS):
        for fn in (mrq.search_contract, mrq.search_literal):
            r = fn(idx, Q, w.k, idx.nlist, eps0=1e9, m=1e9, mode=mode)
            np.testing.assert_array_equal(r.ids, ref_ids)
            np.testing.assert_allclose(r.dists, ref_d, rtol=1e-9)


# m >= 12 covers the residual cross term of true neighbours on this clustered data
# (their 2<x_r, q_r> reaches about 2 m sigma at m = 4)
@pytest.mark.parametrize("eps0,m", [(4.0, 12.0), (1.9, 12.0), (1.0, 16.0)])
def test_contract_equals_literal_when_bounds_hold(small_workload, small_oracle_index, eps0, m):
    """Both threshold semantics return the exact top-k of the probed lists when the
    bounds that matter hold: the k smallest-UB1 candidates and the k smallest-UB2
    candidates of S1 satisfy exact <= UB (so tau >= the k-th exact distance), and
    every true top-k member satisfies LB <= exact (so it survives)."""
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:60]
    rc = mrq.search_contract(idx, Q, w.k, w.nprobe, eps0=eps0, m=m)
    rl = mrq.search_literal(idx, Q, w.k, w.nprobe, eps0=eps0, m=m)
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, Q)
    checked_c = checked_l = 0
    for i in range(Q.shape[0]):
        lists, g = mrq.probe(idx, qd[i], w.nprobe)
        pos, lb, ub = [], [], []
        for j in lists:
            sl = idx.list_slice(int(j))
            e = mrq.estimate_list(idx, int(j), qd[i], float(g[j]), qr2[i], sigma[i], eps0, m)
            pos.append(np.arange(sl.start, sl.stop)); lb.append(e["lb"]); ub.append(e["ub"])
        p, lb, ub = np.concatenate(pos), np.concatenate(lb), np.concatenate(ub)
        ex = np.sum((idx.xd[p] - qd[i]) ** 2, axis=1) + np.sum((idx.xr[p] - qr[i]) ** 2, axis=1)
        diso = idx.xnorm2[p] + qp2[i] - 2 * idx.xd[p] @ qd[i]
        lb2, ub2 = diso - m * sigma[i], diso + m * sigma[i]
        top = np.lexsort((idx.ids[p], ex))[:w.k]
        want = idx.ids[p][top].tolist()
        members_ok = bool(np.all(lb[top] < ex[top]) and np.all(lb2[top] < ex[top]))
        if members_ok:                                   # paper-literal loop
            checked_l += 1
            assert rl.ids[i].tolist() == want
        first = np.argsort(ub)[:w.k]
        s1 = lb <= np.partition(ub, w.k - 1)[w.k - 1]
        first2 = np.nonzero(s1)[0][np.argsort(ub2[s1])[:w.k]]
        if members_ok and np.all(ex[first] <= ub[first]) and np.all(ex[first2] <= ub2[first2]):
            checked_c += 1
            assert rc.ids[i].tolist() == want
    assert checked_c >= 30 and checked_l >= 30
    # the contract prunes: far fewer exact computations than candidates
    assert rc.n_s2.sum() < 0.25 * rc.n_cand.sum()


def test_recall_reasonable_and_quantized_query(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    truth, _ = mrq.exact_knn(base, queries, w.k)
    r = mrq.search_contract(idx, queries, w.k, 16)
    assert mrq.recall_at_k(r.ids, truth) > 0.9
    rq = mrq.search_contract(idx, queries, w.k, 16, qbits=4)
    assert mrq.recall_at_k(rq.ids, truth) > 0.85
    # stage 2 of MRQ+ removes most exact computations that MRQ performs (Exp-3)
    rm = mrq.search_contract(idx, queries, w.k, 16, mode=mrq.MODE_MRQ)
    assert r.n_s2.sum() < 0.5 * rm.n_s2.sum()


def test_index_file_round_trip(tmp_path, small_oracle_index):
    idx = small_oracle_index
    p = str(tmp_path / "i.mrq")
    index_file.write_index(idx, p)
    f = index_file.read_index(p)
    assert f["header"] == dict(n=idx.n, D=idx.D, d=idx.d, bits=idx.bits, nlist=idx.nlist)
    np.testing.assert_array_equal(f["CODE"].reshape(idx.n, idx.d), idx.u)
    np.testing.assert_array_equal(f["LOFF"], idx.list_offsets)
    np.testing.assert_array_equal(f["XD__"].reshape(idx.n, idx.d), idx.xd.astype(np.float32))


def test_contract_thresholds_by_definition(small_workload, small_oracle_index):
    """tau_A and S1 of the contract recomputed through a full sort: S1 counts equal
    #{LB1 <= k-th smallest UB1} (MRQ mode, where S2 = S1)."""
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:25]
    r = mrq.search_contract(idx, Q, w.k, w.nprobe, eps0=1.9, m=4.0, mode=mrq.MODE_MRQ)
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(idx, Q)
    for i in range(Q.shape[0]):
        lists, g = mrq.probe(idx, qd[i], w.nprobe)
        lb, ub = [], []
        for j in lists:
            e = mrq.estimate_list(idx, int(j), qd[i], float(g[j]), qr2[i], sigma[i], 1.9, 4.0)
            lb.append(e["lb"]); ub.append(e["ub"])
        lb, ub = np.concatenate(lb), np.concatenate(ub)
        tau = np.sort(ub)[w.k - 1]
        assert r.n_s1[i] == int(np.sum(lb <= tau)) == r.n_s2[i]


# ------------------------------------------------- 1 bit + refinement (stage 1a/1b)

@pytest.fixture(scope="module")
def refine_pair():
    """The same data, rotation and IVF encoded with 1 and with 3 bits."""
    w = datagen.workload("small", n=8000, n_comp=24, nlist=24, n_query=60)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 11)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 12)
    one = mrq.build_index(base, w.d, 1, w.nlist, G, init_idx=init, kmeans_iters=6)
    three = mrq.build_index(base, w.d, 3, w.nlist, G, init_idx=init, kmeans_iters=6)
    return w, base, queries, one, three


def test_sign_plane_is_the_one_bit_code(refine_pair):
    """Stage 1a of a B-bit code is the 1-bit method: its top plane equals the code a
    1-bit build writes for the same o', and its sign-plane estimate and bounds (with
    the 1-bit factors) equal that build's estimate and bounds, float and quantized."""
    w, base, queries, one, three = refine_pair
    assert one.f_rescale1 is None and three.f_rescale1 is not None
    np.testing.assert_array_equal(three.ids, one.ids)
    np.testing.assert_array_equal(three.u >> 2, one.u)
    np.testing.assert_allclose(three.f_rescale1, one.f_rescale, rtol=1e-12)
    np.testing.assert_allclose(three.f_err1, one.f_err, rtol=1e-12)
    assert not np.allclose(three.f_rescale1, three.f_rescale, rtol=1e-3)
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(three, queries[:8])
    for i in range(8):
        lists, g = mrq.probe(three, qd[i], 3)
        for j in lists:
            for qb in (0, 4):
                a = mrq.estimate_list(three, int(j), qd[i], float(g[j]), qr2[i], sigma[i],
                                      1.9, 4.0, qb, sign_plane=True)
                b = mrq.estimate_list(one, int(j), qd[i], float(g[j]), qr2[i], sigma[i],
                                      1.9, 4.0, qb)
                for key in ("dis", "lb", "ub"):
                    np.testing.assert_allclose(a[key], b[key], rtol=1e-10, atol=1e-9)


def test_refine_without_pruning_is_brute_force(refine_pair):
    w, base, queries, one, three = refine_pair
    Q = queries[:10]
    ref_ids, ref_d = mrq.exact_knn(base, Q, w.k)
    for qb in (0, 4):
        r = mrq.search_contract(three, Q, w.k, three.nlist, eps0=1e9, m=1e9, qbits=qb, refine=True)
        np.testing.assert_array_equal(r.ids, ref_ids)
        np.testing.assert_allclose(r.dists, ref_d, rtol=1e-9)
    # a 1-bit code has no refinement: the flag changes nothing
    a = mrq.search_contract(one, Q, w.k, 4, refine=True)
    b = mrq.search_contract(one, Q, w.k, 4)
    np.testing.assert_array_equal(a.ids, b.ids)
    np.testing.assert_array_equal(a.n_s1, b.n_s1)


def test_refine_equals_exact_when_bounds_hold(refine_pair):
    """When every probed candidate satisfies LB <= exact <= UB at both stage-1 levels and
    at stage 2, every threshold is at least the k-th exact distance and no true member is
    pruned, so the two-level contract returns the exact top-k of the probed lists."""
    w, base, queries, one, three = refine_pair
    eps0, m, nprobe = 4.0, 16.0, 4
    Q = queries[:60]
    r = mrq.search_contract(three, Q, w.k, nprobe, eps0=eps0, m=m, refine=True)
    plain = mrq.search_contract(three, Q, w.k, nprobe, eps0=eps0, m=m)
    qd, qr, qr2, sigma, qp2 = mrq.project_queries(three, Q)
    checked = 0
    for i in range(Q.shape[0]):
        lists, g = mrq.probe(three, qd[i], nprobe)
        p, lo, hi = [], [], []
        for j in lists:
            sl = three.list_slice(int(j))
            p.append(np.arange(sl.start, sl.stop))
            for sp in (True, False):
                e = mrq.estimate_list(three, int(j), qd[i], float(g[j]), qr2[i], sigma[i],
                                      eps0, m, sign_plane=sp)
                lo.append((sp, e["lb"])); hi.append((sp, e["ub"]))
        p = np.concatenate(p)
        lba = np.concatenate([a for sp, a in lo if sp]); uba = np.concatenate([a for sp, a in hi if sp])
        lbb = np.concatenate([a for sp, a in lo if not sp]); ubb = np.concatenate([a for sp, a in hi if not sp])
        ex = np.sum((three.xd[p] - qd[i]) ** 2, axis=1) + np.sum((three.xr[p] - qr[i]) ** 2, axis=1)
        diso = three.xnorm2[p] + qp2[i] - 2 * three.xd[p] @ qd[i]
        ok = all(np.all((lb_ <= ex) & (ex <= ub_)) for lb_, ub_ in
                 ((lba, uba), (lbb, ubb), (diso - m * sigma[i], diso + m * sigma[i])))
        if ok:
            checked += 1
            top = np.lexsort((three.ids[p], ex))[:w.k]
            assert r.ids[i].tolist() == three.ids[p][top].tolist()
            assert plain.ids[i].tolist() == r.ids[i].tolist()
    assert checked >= 30
    # the sign plane's wider interval lets more candidates through stage 1a than the
    # full code passes in one stage, and the refinement removes most of them again
    assert r.n_s1.sum() <= 1.5 * plain.n_s1.sum()


# ------------------------------------------------------ Eq. 8: automatic d selection

def test_choose_d_hand_examples():
    # one unit of variance on each of the first 200 coordinates, 0.1 on the other 824
    # (D = 1024): total 282.4; the first 128 hold 128 / 282.4 = 0.453, the first 256
    # hold (200 + 56 * 0.1) / 282.4 = 0.728, the first 512 (200 + 312 * 0.1) / 282.4 = 0.819
    lam = np.r_[np.ones(200), np.full(824, 0.1)]
    assert mrq.choose_d(lam, 1024) == 512
    assert mrq.choose_d(lam, 1024, target=0.7) == 256
    assert mrq.choose_d(lam, 1024, target=0.45) == 128      # at least 128 even when fewer do
    # the denominator is the whole spectrum: ten coordinates of variance 1 and 950 of
    # 0.001 (D = 960) leave 10 / 10.95 = 0.913 in the first 128
    assert mrq.choose_d(np.r_[np.ones(10), np.full(950, 1e-3)], 960) == 128
    # flat spectrum (D = 960): 512 / 960 = 0.53 < 0.8, the next power of two passes D, so
    # d = D, no tail (IVF-RaBitQ)
    assert mrq.choose_d(np.ones(960), 960) == 960
    # D below 128 (DEEP's 96): d = D; D not a multiple of 32: d rounds down
    assert mrq.choose_d(np.ones(96), 96) == 96
    assert mrq.choose_d(np.ones(100), 100) == 96
    # no power of two above the library's largest d: d = 1024 for a flat D = 1536
    assert mrq.choose_d(np.ones(1536), 1536) == 1024


def test_choose_d_on_a_closed_form_spectrum():
    """lam_i = i^-1 (i = 1..D, D = 960): the captured fraction at p is H_p / H_960 with
    H the harmonic number; H_128 / H_960 = 5.4384 / 7.4425 = 0.731, H_256 / H_960 = 6.1312 /
    7.4425 = 0.824, so Eq. 8 picks 256.  Also run through the oracle's own PCA on data with
    that spectrum (a random orthogonal basis times scaled Gaussians)."""
    D = 960
    lam = 1.0 / np.arange(1, D + 1)
    assert mrq.choose_d(lam, D) == 256
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((D, D)))
    X = (rng.standard_normal((20_000, D)) * np.sqrt(lam)) @ U.T
    _, lam_hat, _ = mrq.pca_train(X)
    assert mrq.choose_d(lam_hat, D) == 256


# ------------------------------------------------------------ MR-SQ (Exp-5), 8-bit SQ

def test_sq8_hand_example():
    # column 0: 0 .. 255 integers, so lo = 0, delta = 1 and the codes are the values;
    # column 1: -1, 1, 0.5, 0: lo = -1, delta = 2/255, (0.5 + 1) / (2/255) = 191.25 -> 191;
    # 0 sits exactly on a half level in exact arithmetic (127.5), but the decision is taken
    # in float32: delta = fl(2/255) = 0.0078431377 > 2/255, 1 / delta = 127.49999, and
    # floor(127.49999 + 0.5) = 127; column 2 is constant -> 0
    X = np.array([[0, -1, 3], [255, 1, 3], [17, 0.5, 3], [100, 0, 3]], dtype=np.float32)
    lo, delta, c = mrq.sq8_train(X)
    np.testing.assert_array_equal(lo, np.float32([0, -1, 3]))
    np.testing.assert_array_equal(delta, np.float32([1, 2 / 255, 0]))
    np.testing.assert_array_equal(c, np.array([[0, 0, 0], [255, 255, 0], [17, 191, 0],
                                               [100, 127, 0]], dtype=np.uint8))


def test_sq8_reconstruction_bound():
    """Round to nearest on a uniform grid: |x - x_hat| <= delta / 2 per coordinate (up to
    float32 rounding of the grid), and the extremes reconstruct exactly."""
    rng = np.random.default_rng(7)
    X = (rng.standard_normal((4000, 48)) * rng.uniform(0.1, 5, 48)).astype(np.float32)
    lo, delta, c = mrq.sq8_train(X)
    xhat = lo.astype(np.float64) + c.astype(np.float64) * delta.astype(np.float64)
    err = np.abs(xhat - X.astype(np.float64))
    assert np.all(err <= delta.astype(np.float64) / 2 * (1 + 1e-4) + 1e-6)
    assert np.all(c[np.argmin(X, axis=0), np.arange(48)] == 0)
    assert np.all(c[np.argmax(X, axis=0), np.arange(48)] == 255)


def test_mrsq8_estimate_within_its_bound(small_workload, small_oracle_index):
    """dis'' - |x_r|^2 - |q_r|^2 is |q_d' - x_hat|^2, within |x_hat - x_d'| of |q_d' - x_d'|
    (triangle inequality): | sqrt(dis'' - |x_r|^2 - |q_r|^2) - |q_d' - x_d'| | <= |delta|/2."""
    w, base, queries = small_workload
    idx = small_oracle_index
    sq = mrq.sq8_train(idx.xd)
    qd, qr, qr2, _, _ = mrq.project_queries(idx, queries[:20])
    bound = np.linalg.norm(sq[1].astype(np.float64)) / 2 * (1 + 1e-4) + 1e-9
    xr2 = np.linalg.norm(idx.xr, axis=1) ** 2
    for i in range(20):
        est = mrq.sq8_estimate(idx, sq, qd[i], qr2[i])
        lead = np.sqrt(np.maximum(est - xr2 - qr2[i], 0))
        true_lead = np.linalg.norm(idx.xd - qd[i], axis=1)
        assert np.all(np.abs(lead - true_lead) <= bound)
        # and the dropped term is exactly the residual cross term
        full = np.sum((idx.xd - qd[i]) ** 2, axis=1) + np.sum((idx.xr - qr[i]) ** 2, axis=1)
        assert np.allclose(full - (true_lead ** 2 + xr2 + qr2[i]), -2 * idx.xr @ qr[i], atol=1e-8)


def test_mrsq8_full_rerank_is_brute_force(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:12]
    ref_ids, ref_d = mrq.exact_knn(base, Q, w.k)
    r = mrq.search_mrsq8(idx, Q, w.k, idx.nlist, rerank=idx.xd.shape[0])
    np.testing.assert_array_equal(r.ids, ref_ids)
    np.testing.assert_allclose(r.dists, ref_d, rtol=1e-9)


def test_mrsq8_rerank_range(small_workload, small_oracle_index):
    """The answer is the exact top-k of the rerank range, and with enough range the
    recall matches the exact top-k of the probed lists (8-bit codes are fine-grained)."""
    w, base, queries = small_workload
    idx = small_oracle_index
    Q = queries[:40]
    r = mrq.search_mrsq8(idx, Q, w.k, w.nprobe, rerank=200)
    assert np.all(r.n_s1 == np.minimum(200, r.n_cand))
    full = mrq.search_contract(idx, Q, w.k, w.nprobe, eps0=1e9, m=1e9)   # exact over probed
    assert mrq.recall_at_k(r.ids, full.ids) > 0.99
    r10 = mrq.search_mrsq8(idx, Q, w.k, w.nprobe, rerank=w.k)
    assert mrq.recall_at_k(r10.ids, full.ids) < mrq.recall_at_k(r.ids, full.ids)


# -------------------------------------------------------- MR-PQ (Exp-5), OPQ codes

@pytest.fixture(scope="module")
def pq_setup(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    init = datagen.kmeans_init_indices(idx.xd.shape[0], 16, 21)
    pq = mrq.opq_train(idx.xd, M=16, K=16, init_idx=init, opq_iters=4, km_iters=4)
    return w, base, queries, idx, pq, init


def test_opq_rotation_is_orthogonal_and_procrustes_optimal(pq_setup):
    """R is orthogonal, and for the final codes no other orthogonal matrix (the identity,
    random rotations, R itself perturbed) brings X closer to their decoded rows."""
    w, base, queries, idx, pq, init = pq_setup
    R, C, codes = pq
    d = R.shape[0]
    np.testing.assert_allclose(R.T @ R, np.eye(d), atol=1e-10)
    X = idx.xd.astype(np.float64)
    Y = mrq.pq_decode(C, codes.astype(np.int64))
    # the Procrustes step for these codes (one more alternation) cannot do worse than R
    U, _, Vt = np.linalg.svd(X.T @ Y)
    best = np.linalg.norm(X @ (U @ Vt) - Y)
    rng = np.random.default_rng(3)
    for Q in [np.eye(d), R] + [np.linalg.qr(rng.standard_normal((d, d)))[0] for _ in range(5)]:
        assert best <= np.linalg.norm(X @ Q - Y) + 1e-9
    # one alternation from the identity: R is the orthogonal polar factor of X^T Y0 for the
    # codes Y0 of plain PQ, A (A^T A)^(-1/2) with A = X^T Y0 (computed by an eigensolver,
    # not an SVD)
    R1, _, _ = mrq.opq_train(X, M=16, K=16, init_idx=init, opq_iters=1, km_iters=4)
    _, C0, codes0 = mrq.opq_train(X, M=16, K=16, init_idx=init, opq_iters=0, km_iters=4)
    A = X.T @ mrq.pq_decode(C0, codes0.astype(np.int64))
    lam, V = np.linalg.eigh(A.T @ A)
    polar = A @ (V / np.sqrt(lam)[None, :]) @ V.T
    np.testing.assert_allclose(R1, polar, atol=1e-8)


def test_opq_lowers_distortion_against_plain_pq(pq_setup):
    """The learned rotation never raises the quantization distortion over the alternations
    (each step minimises it over its own variable), so it ends at most at plain PQ's."""
    w, base, queries, idx, pq, init = pq_setup
    X = idx.xd.astype(np.float64)
    dist = []
    for it in (0, 1, 2, 4):
        R, C, codes = mrq.opq_train(X, M=16, K=16, init_idx=init, opq_iters=it, km_iters=4)
        dist.append(np.sum((X @ R - mrq.pq_decode(C, codes.astype(np.int64))) ** 2))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(dist, dist[1:]))
    assert dist[-1] < dist[0]


def test_pq_estimate_is_the_rotated_decoded_distance(pq_setup):
    """The lookup-table sum equals |q_d' - y R^T|^2 for the decoded row y (R orthogonal:
    |q R - y| = |q - y R^T|), plus |x_r|^2 + |q_r|^2 -- a transposed R or a wrong
    subspace slice breaks it."""
    w, base, queries, idx, pq, init = pq_setup
    R, C, codes = pq
    Y = mrq.pq_decode(C, codes.astype(np.int64)) @ R.T      # back in the x_d' frame
    qd, qr, qr2, _, _ = mrq.project_queries(idx, queries[:10])
    xr2 = np.linalg.norm(idx.xr, axis=1) ** 2
    for i in range(10):
        est = mrq.pq_estimate(idx, pq, qd[i], qr2[i])
        want = np.linalg.norm(Y - qd[i], axis=1) ** 2 + xr2 + qr2[i]
        np.testing.assert_allclose(est, want, rtol=1e-9, atol=1e-9)


def test_pq_with_one_centroid_per_point_is_exact():
    """K = n: every point is its own centroid, the codes reconstruct X R exactly and the
    MR-PQ estimate is |q_d' - x_d'|^2 + |x_r|^2 + |q_r|^2."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((16, 8))
    R, C, codes = mrq.opq_train(X, M=2, K=16, init_idx=np.arange(16), opq_iters=2, km_iters=2)
    np.testing.assert_allclose(mrq.pq_decode(C, codes.astype(np.int64)), X @ R, atol=1e-10)


def test_mrpq_full_rerank_is_brute_force(pq_setup):
    w, base, queries, idx, pq, init = pq_setup
    Q = queries[:10]
    ref_ids, ref_d = mrq.exact_knn(base, Q, w.k)
    r = mrq.search_mrpq(idx, Q, w.k, idx.nlist, pq, rerank=idx.xd.shape[0])
    np.testing.assert_array_equal(r.ids, ref_ids)
    np.testing.assert_allclose(r.dists, ref_d, rtol=1e-9)
    r2 = mrq.search_mrpq(idx, queries[:40], w.k, w.nprobe, pq, rerank=300)
    full = mrq.search_contract(idx, queries[:40], w.k, w.nprobe, eps0=1e9, m=1e9)
    assert mrq.recall_at_k(r2.ids, full.ids) > 0.97


def test_index_file_optional_sign_plane_sections(tmp_path, refine_pair):
    """The writer adds FRE1/FER1 for a multi-bit index (and only then); the reader returns
    them unchanged (float32)."""
    w, base, queries, one, three = refine_pair
    p1, p3 = str(tmp_path / "b1.mrq"), str(tmp_path / "b3.mrq")
    index_file.write_index(one, p1)
    index_file.write_index(three, p3)
    f1, f3 = index_file.read_index(p1), index_file.read_index(p3)
    assert "FRE1" not in f1 and "FER1" not in f1
    np.testing.assert_array_equal(f3["FRE1"], three.f_rescale1.astype(np.float32))
    np.testing.assert_array_equal(f3["FER1"], three.f_err1.astype(np.float32))
