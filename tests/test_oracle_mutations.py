"""Planted mistakes in the CPU oracle must be caught by its pins.

Each case swaps one oracle function for a plausibly wrong variant (a dropped
term, a wrong sign, a wrong index, a missing step), reruns the pin that guards
it, and expects that pin to fail.  Mistakes are planted in the oracle only, on
the CPU."""
import math

import numpy as np
import pytest

import datagen
from oracle import mrq
import test_oracle_pins as pins


def _small():
    w = datagen.workload("small", n=6000, n_comp=24, nlist=24, n_query=60)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 3)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 4)
    idx = mrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=5)
    return (w, base, queries), idx


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_tail_variance_index_off_by_d(monkeypatch):
    orig = mrq.project_queries

    def wrong(idx, Q):
        qd, qr, qr2, sigma, qp2 = orig(idx, Q)
        lam = idx.lam[:idx.D - idx.d]                      # wrong slice of sigma_i^2
        return qd, qr, qr2, np.sqrt(np.sum(qr * qr * lam[None, :], axis=1)), qp2
    monkeypatch.setattr(mrq, "project_queries", wrong)
    wk, idx = _small()
    _fails(pins.test_residual_variance_identity_and_chebyshev, wk, idx)


def test_rescale_sign_flipped(monkeypatch):
    orig = mrq.factors

    def wrong(*a):
        f_add, f_res, f_err, ip = orig(*a)
        return f_add, -f_res, f_err, ip
    monkeypatch.setattr(mrq, "factors", wrong)
    wk, idx = _small()
    _fails(pins.test_eq3_decomposition_exact, wk, idx)


def test_error_factor_without_dimension_scaling(monkeypatch):
    orig = mrq.factors

    def wrong(resid_norm, xr2, v, o, d):
        f_add, f_res, f_err, ip = orig(resid_norm, xr2, v, o, d)
        return f_add, f_res, f_err * math.sqrt(d - 1), ip
    monkeypatch.setattr(mrq, "factors", wrong)
    _fails(pins.test_factor_closed_form_one_hot)


def test_code_sign_inverted(monkeypatch):
    orig = mrq.encode

    def wrong(o, bits):
        return orig(-np.asarray(o), bits)
    monkeypatch.setattr(mrq, "encode", wrong)
    _fails(pins.test_encode_golden)


def test_random_rotation_missing_from_projection(monkeypatch):
    orig = mrq.build_index

    def wrong(*a, **k):
        idx = orig(*a, **k)
        idx.W = idx.Pp.copy()                              # queries no longer rotated by P_r
        return idx
    monkeypatch.setattr(mrq, "build_index", wrong)
    wk, idx = _small()
    _fails(pins.test_eq3_decomposition_exact, wk, idx)


def test_kmeans_update_not_averaged(monkeypatch):
    def wrong(X, init, iters):
        C = np.array(init, dtype=np.float64, copy=True)
        for _ in range(iters):
            a = mrq._assign(X, C)
            sums = np.zeros_like(C)
            np.add.at(sums, a, X)
            C = sums                                       # forgot to divide by the count
        return C, mrq._assign(X, C)
    monkeypatch.setattr(mrq, "kmeans", wrong)
    _fails(pins.test_kmeans_hand_example)


def test_estimate_drops_query_tail_norm(monkeypatch):
    orig = mrq.estimate_list

    def wrong(idx, j, qd, g_j, qr2, sigma, eps0, m, qbits=0):
        return orig(idx, j, qd, g_j, 0.0, sigma, eps0, m, qbits)   # |q_r|^2 of Eq. 4 dropped
    monkeypatch.setattr(mrq, "estimate_list", wrong)
    wk, idx = _small()
    _fails(pins.test_bound_rate_and_multibit_accuracy, wk, idx)


def test_threshold_from_too_few_upper_bounds(monkeypatch):
    orig = mrq._kth

    def wrong(values, k):
        return orig(values, max(1, k // 4))                # tau_A from too few candidates
    monkeypatch.setattr(mrq, "_kth", wrong)
    wk, idx = _small()
    _fails(pins.test_contract_thresholds_by_definition, wk, idx)


def test_query_grid_offset_sign_flipped(monkeypatch):
    orig = mrq.quantize_query

    def wrong(qprime, qbits):
        qbar, lo, delta = orig(qprime, qbits)
        return qbar, -lo, delta                             # sign of v_l flipped
    monkeypatch.setattr(mrq, "quantize_query", wrong)
    _fails(pins.test_quantize_query_golden_and_grid_identity)


def _estimate_with_ip(orig, change):
    """estimate_list whose quantized inner product is replaced by change(e, top, d),
    with dis', LB and UB moved consistently (a mistake inside the Eq. 4 identity)."""
    def wrong(idx, j, qd, g_j, qr2, sigma, eps0, m, qbits=0, sign_plane=False):
        e = dict(orig(idx, j, qd, g_j, qr2, sigma, eps0, m, qbits, sign_plane=sign_plane))
        if qbits > 0:
            sl = idx.list_slice(j)
            top = 1 if sign_plane else (1 << idx.bits) - 1
            fres = idx.f_rescale1[sl] if sign_plane else idx.f_rescale[sl]
            ip = change(e, top, idx.d, idx.u[sl] >> (idx.bits - 1) if sign_plane else idx.u[sl])
            dd = fres * math.sqrt(g_j) * (ip - e["ip"])
            e.update(ip=ip, dis=e["dis"] + dd, lb=e["lb"] + dd, ub=e["ub"] + dd)
        return e
    return wrong


@pytest.mark.parametrize("pin", ["test_quantized_estimate_hand_example", "on_grid"])
def test_quantized_inner_product_drops_qbar_sum(monkeypatch, pin):
    # ip = delta*(2<u,qbar>) + v_l*(2 sum u - d*top): the -top*sum(qbar) term dropped
    wrong = _estimate_with_ip(mrq.estimate_list,
                              lambda e, top, d, u: e["ip"] + e["delta"] * top * float(e["qbar"].sum()))
    monkeypatch.setattr(mrq, "estimate_list", wrong)
    if pin == "on_grid":
        _fails(pins.test_quantized_estimate_on_grid_is_exact,
               pins.multibit_indices.__wrapped__(), 1, 4)
    else:
        _fails(pins.test_quantized_estimate_hand_example)


@pytest.mark.parametrize("pin", ["test_quantized_estimate_hand_example", "on_grid"])
def test_quantized_inner_product_offset_without_top(monkeypatch, pin):
    # the v_l term with d where d*(2^B - 1) belongs (invisible at B = 1)
    def change(e, top, d, u):
        return e["ip"] + e["vl"] * (d * top - d)
    monkeypatch.setattr(mrq, "estimate_list", _estimate_with_ip(mrq.estimate_list, change))
    if pin == "on_grid":
        _fails(pins.test_quantized_estimate_on_grid_is_exact,
               pins.multibit_indices.__wrapped__(), 4, 4)
    else:
        _fails(pins.test_quantized_estimate_hand_example)


def test_quantized_inner_product_offset_sign(monkeypatch):
    # v_l*(d*top - 2 sum u): the offset term with its sign flipped
    def change(e, top, d, u):
        su = u.astype(np.int64).sum(axis=1)
        return e["ip"] - 2.0 * e["vl"] * (2.0 * su - d * top)
    monkeypatch.setattr(mrq, "estimate_list", _estimate_with_ip(mrq.estimate_list, change))
    _fails(pins.test_quantized_estimate_hand_example)
    _fails(pins.test_quantized_estimate_off_grid_is_the_dequantized_query,
           pins.multibit_indices.__wrapped__(), 4)


def _margin_variant(kind):
    def wrong(lb, ub, sc, tau, k, rel):
        srt = np.sort(ub)
        if kind == "gap_ranks":                               # gap of ranks k-1, k-2
            gap_k = ((srt[k - 1] - srt[k - 2]) / max(abs(srt[k - 1]), 1e-30)
                     if srt.size > k and k >= 2 else math.inf)
        else:
            gap_k = (srt[k] - srt[k - 1]) / max(abs(srt[k]), 1e-30) if srt.size > k else math.inf
        m = np.abs(lb - tau) / sc
        if kind != "no_zero_width":
            m = np.where(ub <= tau, np.maximum(m, gap_k), m)
        return float(np.max(m[rel]) if kind == "max" else np.min(m[rel]))
    return wrong


@pytest.mark.parametrize("kind,pin", [("max", "test_decision_margin_hand_example"),
                                      ("gap_ranks", "test_decision_margin_hand_example"),
                                      ("no_zero_width", "test_decision_margin_zero_width_bounds")])
def test_decision_margin_mistakes(monkeypatch, kind, pin):
    monkeypatch.setattr(mrq, "_decision_margin", _margin_variant(kind))
    _fails(getattr(pins, pin))


def test_sign_plane_with_full_code_factors(monkeypatch):
    orig = mrq.build_index

    def wrong(*a, **k):
        idx = orig(*a, **k)
        if idx.f_rescale1 is not None:                     # stage 1a rescaled like the B-bit code
            idx.f_rescale1 = idx.f_rescale.copy()
        return idx
    monkeypatch.setattr(mrq, "build_index", wrong)
    _fails(pins.test_sign_plane_is_the_one_bit_code, pins.refine_pair.__wrapped__())


def test_sign_plane_from_lowest_plane(monkeypatch):
    orig = mrq.estimate_list

    def wrong(idx, j, *a, sign_plane=False, **k):
        if not sign_plane:
            return orig(idx, j, *a, **k)
        saved = idx.u
        idx.u = (saved & 1) << (idx.bits - 1)              # the least significant plane
        try:
            return orig(idx, j, *a, sign_plane=True, **k)
        finally:
            idx.u = saved
    monkeypatch.setattr(mrq, "estimate_list", wrong)
    _fails(pins.test_sign_plane_is_the_one_bit_code, pins.refine_pair.__wrapped__())


def test_eq8_denominator_over_the_lead_only(monkeypatch):
    def wrong(lam, D, target=0.8, max_d=1024):
        # the garbled formula taken literally: the denominator runs over the leading
        # coordinates only, so every candidate "captures" all of its own variance
        lam = np.maximum(np.asarray(lam, dtype=np.float64)[:D], 0.0)
        cap = min((D // 32) * 32, max_d)
        p = 128
        while p < cap:
            if lam[:p].sum() >= target * lam[:p].sum():
                return p
            p *= 2
        return cap
    monkeypatch.setattr(mrq, "choose_d", wrong)
    _fails(pins.test_choose_d_hand_examples)


def test_eq8_on_standard_deviations(monkeypatch):
    orig = mrq.choose_d

    def wrong(lam, D, target=0.8, max_d=1024):
        return orig(np.sqrt(np.maximum(np.asarray(lam, dtype=np.float64), 0.0)), D, target, max_d)
    monkeypatch.setattr(mrq, "choose_d", wrong)
    _fails(pins.test_choose_d_on_a_closed_form_spectrum)


def test_sq8_truncating_codes(monkeypatch):
    def wrong(xd):
        X = np.asarray(xd, dtype=np.float32)
        lo, hi = X.min(axis=0), X.max(axis=0)
        delta = ((hi - lo) / np.float32(255)).astype(np.float32)
        safe = np.where(delta > 0, delta, np.float32(1))
        c = np.floor((X - lo) / safe)                        # no rounding to nearest
        return lo, delta, np.where(delta > 0, np.clip(c, 0, 255), 0).astype(np.uint8)
    monkeypatch.setattr(mrq, "sq8_train", wrong)
    _fails(pins.test_sq8_reconstruction_bound)


def test_mrsq8_grid_off_by_one_level(monkeypatch):
    orig = mrq.sq8_train

    def shifted(xd):
        lo, delta, c = orig(xd)
        return lo + delta, delta, c                          # reconstruction one level up
    monkeypatch.setattr(mrq, "sq8_train", shifted)
    wk, idx = _small()
    _fails(pins.test_mrsq8_estimate_within_its_bound, wk, idx)


def test_mrsq8_dropped_tail_norm(monkeypatch):
    orig = mrq.sq8_estimate

    def wrong(idx, sq, qd, qr2, pos=None):
        sel = slice(None) if pos is None else pos
        return orig(idx, sq, qd, qr2, pos) - np.sum(idx.xr[sel] ** 2, axis=1)
    monkeypatch.setattr(mrq, "sq8_estimate", wrong)
    wk, idx = _small()
    _fails(pins.test_mrsq8_estimate_within_its_bound, wk, idx)


def test_pq_query_rotated_by_the_transpose(monkeypatch):
    orig = mrq.pq_estimate

    def wrong(idx, pq, qd, qr2, pos=None):
        R, C, codes = pq
        return orig(idx, (R.T, C, codes), qd, qr2, pos)
    monkeypatch.setattr(mrq, "pq_estimate", wrong)
    fx = pins.pq_setup.__wrapped__(*pins_small())
    _fails(pins.test_pq_estimate_is_the_rotated_decoded_distance, fx)


def test_procrustes_factors_swapped(monkeypatch):
    real_svd = np.linalg.svd

    def swapped(a, *args, **kw):
        U, S, Vt = real_svd(a, *args, **kw)
        return Vt.T, S, U.T                      # the rotation becomes V U^T, not U V^T
    wk, idx = _small()
    init = datagen.kmeans_init_indices(idx.xd.shape[0], 16, 21)
    pq = mrq.opq_train(idx.xd, M=16, K=16, init_idx=init, opq_iters=4, km_iters=4)
    monkeypatch.setattr(np.linalg, "svd", swapped)
    _fails(pins.test_opq_rotation_is_orthogonal_and_procrustes_optimal,
           (wk[0], wk[1], wk[2], idx, pq, init))


def pins_small():
    wk, idx = _small()
    return wk, idx


def _shard_fixture():
    import test_shard as ts
    wk, idx = _small()
    return ts.sharded.__wrapped__(wk, idx)


def test_merge_keeps_the_largest(monkeypatch):
    def wrong(parts, k):
        nq = parts[0][0].shape[0]
        ids = np.full((nq, k), -1, dtype=np.int64)
        dists = np.full((nq, k), np.inf)
        for q in range(nq):
            pairs = sorted(((float(d_), int(i_)) for pi, pd in parts
                            for i_, d_ in zip(pi[q], pd[q]) if i_ >= 0), reverse=True)[:k]
            for t, (d_, i_) in enumerate(sorted(pairs)):
                ids[q, t], dists[q, t] = i_, d_
        return ids, dists
    monkeypatch.setattr(mrq, "merge_answers", wrong)
    import test_shard as ts
    _fails(ts.test_sharded_without_pruning_is_exact_over_probed_lists, _shard_fixture())


def test_shard_rows_off_by_one(monkeypatch):
    orig = mrq.restrict_lists

    def wrong(idx, lists):
        sh = orig(idx, lists)
        sh.ids = np.roll(sh.ids, 1)                              # rows one slot off their lists
        return sh
    monkeypatch.setattr(mrq, "restrict_lists", wrong)
    import test_shard as ts
    _fails(ts.test_shards_partition_the_index, _shard_fixture())


def test_sampled_pca_ignores_the_sample(monkeypatch):
    orig = mrq.build_index

    def wrong(*a, pca_rows=None, **k):
        return orig(*a, **k)                                        # full-base PCA
    monkeypatch.setattr(mrq, "build_index", wrong)
    import test_shard as ts
    _fails(ts.test_sampled_pca_is_the_pca_of_the_sample)
