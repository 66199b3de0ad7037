"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test names the passage or mathematical fact it checks. Together they are
chosen so that a plausible slip anywhere in the oracle (a dropped term, a
wrong sign, a wrong constant, a transposed index, an off-by-one in the key
race) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 1e-3


def _uniform_draws(seed, shape):
    """Uniforms of the method's form (odd 24-bit integer * 2^-24) from numpy's Philox."""
    g = np.random.Generator(np.random.Philox(key=[seed, 7]))
    bits = g.integers(0, 2 ** 32, size=shape, dtype=np.uint32)
    return (((bits >> 8) | 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def _chi2_p(counts, probs, min_expected=5.0):
    """Chi-square p-value with cells of small expectation merged."""
    counts = np.asarray(counts, np.float64)
    probs = np.asarray(probs, np.float64)
    n = counts.sum()
    order = np.argsort(probs)
    obs, exp_ = [], []
    acc_o = acc_e = 0.0
    for i in order:
        acc_o += counts[i]
        acc_e += probs[i] * n
        if acc_e >= min_expected:
            obs.append(acc_o)
            exp_.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 or acc_o > 0:
        if obs:
            obs[-1] += acc_o
            exp_[-1] += acc_e
        else:
            obs.append(acc_o)
            exp_.append(acc_e)
    obs, exp_ = np.array(obs), np.array(exp_)
    exp_ *= obs.sum() / exp_.sum()
    if len(obs) < 2:
        return 1.0
    return stats.chisquare(obs, exp_).pvalue


def _effective_weights(w, bias):
    """Weights of the items as the race sees them at the end of the stream:
    w_i times every later bias factor f_s = 1 - w_s/(W_{s-1} + w_s) (FP64),
    Eq. (temporal-bias) applied before each combine."""
    w = np.asarray(w, np.float64)
    eff = w.copy()
    if not bias:
        return eff
    W = 0.0
    for s, ws in enumerate(w):
        if W > 0:
            f = 1.0 - ws / (W + ws)
            eff[:s] *= f
            W *= f
        W += ws
    return eff


def _successive_sampling_subsets(w, K):
    """Exact law of the K-subset drawn by successive sampling without
    replacement with probabilities proportional to w (brute force over
    ordered K-tuples)."""
    w = np.asarray(w, np.float64)
    T = w.sum()
    law = {}
    for tup in itertools.permutations(range(len(w)), K):
        p, rem = 1.0, T
        for i in tup:
            p *= w[i] / rem
            rem -= w[i]
        key = tuple(sorted(tup))
        law[key] = law.get(key, 0.0) + p
    return law


# ------------------------------------------------------------------ exp / log

def test_exp_matches_libm(orc):
    x = np.linspace(-87.0, 0.0, 400001).astype(np.float32)
    x = np.concatenate([x, np.float32([-0.0, -1e-30, -1e-8, -0.34657359, -0.34657360])])
    y = orc.exp32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 4.0


def test_log_matches_libm(orc):
    k = np.concatenate([np.arange(1, 2 ** 24, 97, dtype=np.int64), [1, 3, 2 ** 24 - 1, 2 ** 23 + 1]])
    u = ((k | 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    y = orc.log32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 4.0
    assert np.all(y < 0.0)  # E = -ln u > 0 for every u the method draws


# ------------------------------------------------------------------ Philox

def test_philox_uniforms_are_uniform_and_exact(orc):
    u = orc.uniforms(seed=12345, stream_id=3, t=7, p0=0, n=1 << 20).astype(np.float64)
    assert np.all((u > 0.0) & (u < 1.0))
    k = u * 2.0 ** 24
    assert np.all(k == np.round(k)) and np.all(np.round(k) % 2 == 1)
    counts, _ = np.histogram(u, bins=256, range=(0.0, 1.0))
    assert stats.chisquare(counts).pvalue > ALPHA
    # neighbouring pixels (same Philox block) are uncorrelated
    assert abs(np.corrcoef(u[0::4], u[1::4])[0, 1]) < 0.01


def test_philox_counter_and_key_change_output(orc):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for c in ([0, 2, 3, 4], [1, 3, 3, 4], [1, 2, 2, 4], [1, 2, 3, 5]):
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    assert not np.array_equal(orc.philox([1, 2, 3, 4], [5, 7]), base)
    # avalanche: one flipped counter bit flips about half the output bits
    flips = []
    for bit in range(32):
        o = orc.philox([1 ^ (1 << bit), 2, 3, 4], [5, 6])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(o, base)))
    assert 48 < np.mean(flips) < 80


def test_uniform_uses_one_block_per_four_pixels(orc):
    for p in (0, 5, 1023):
        out = orc.philox([p >> 2, 9, 4, 0], [0xDEADBEEF, 0x1234])
        x = int(out[p & 3])
        u = orc.uniforms(seed=(0x1234 << 32) | 0xDEADBEEF, stream_id=4, t=9, p0=p, n=1)[0]
        assert u == np.float32(((x >> 8) | 1) * 2.0 ** -24)


# ------------------------------------------------------------------ density / weight

def test_watson_parameters_match_paper(orc):
    g = json.load(open(os.path.join(GOLDEN, "watson_params.json")))
    # Eq. (cone_retinal_density) at e = 0: (1)^-1 [a (1)^-2 + (1 - a) e^0] = 1, so d(0) = 2 d_c(0).
    assert orc.density64([0.0])[0] == pytest.approx(2.0 * g["d_c0_per_deg2"], rel=1e-15)


def test_density_slope_at_zero(orc):
    # d/de ln d(e) at 0 = -1/r_m - 2 a / r_2 - (1 - a) / r_e (differentiating the closed form).
    g = json.load(open(os.path.join(GOLDEN, "watson_params.json")))
    a, r2, re_, rm = g["a_k"], g["r_2k_deg"], g["r_ek_deg"], g["r_m_deg"]
    h = 1e-5
    d = orc.density64(np.array([h, 2 * h]))
    d0 = orc.density64([0.0])[0]
    # second-order one-sided difference
    slope = (-3 * d0 + 4 * d[0] - d[1]) / (2 * h) / d0
    assert slope == pytest.approx(-1.0 / rm - 2.0 * a / r2 - (1.0 - a) / re_, rel=1e-6)


def test_density_power_law_tail(orc):
    # for e >> r_e the exponential term vanishes and d(e) e^3 -> 2 d_c(0) a r_m r_2^2
    g = json.load(open(os.path.join(GOLDEN, "watson_params.json")))
    e = 1.0e7
    lim = 2.0 * g["d_c0_per_deg2"] * g["a_k"] * g["r_m_deg"] * g["r_2k_deg"] ** 2
    assert orc.density64([e])[0] * e ** 3 == pytest.approx(lim, rel=1e-5)


def test_density_exponential_term(orc):
    # Where (1 + e/r_2)^-2 is negligible against the exponential term is not
    # reachable, so pin the exponential's scale by the log-slope at the point
    # where both terms are known: slope(e) = -1/(r_m+e) + [A' + B'] / [A + B]
    # with A = a(1+e/r_2)^-2, B = (1-a) exp(-e/r_e). A wrong r_e or a missing
    # minus sign in the exponent changes this by far more than 1e-6.
    g = json.load(open(os.path.join(GOLDEN, "watson_params.json")))
    a, r2, re_, rm = g["a_k"], g["r_2k_deg"], g["r_ek_deg"], g["r_m_deg"]
    for e in (20.0, 60.0, 120.0):
        A = a * (1 + e / r2) ** -2
        B = (1 - a) * math.exp(-e / re_)
        dA = -2.0 * a / r2 * (1 + e / r2) ** -3
        dB = -B / re_
        expect = -1.0 / (rm + e) + (dA + dB) / (A + B)
        h = 1e-4 * e
        dd = orc.density64(np.array([e - h, e, e + h]))
        slope = (dd[2] - dd[0]) / (2 * h) / dd[1]
        assert slope == pytest.approx(expect, rel=1e-6)


def test_density32_tracks_fp64(orc):
    e = np.linspace(0.0, 180.0, 20001).astype(np.float32)
    d32 = orc.density32(e).astype(np.float64)
    d64 = orc.density64(e.astype(np.float64)) / (2.0 * 14804.6)
    assert np.max(np.abs(d32 / d64 - 1.0)) < 2e-6


def test_weight_inside_fovea_is_one_and_bounded(orc):
    cfg = orc.make_config(257, 131, 4, r_f=20.0)
    gx, gy = 100.3, 60.7
    w = orc.weight_grid(cfg, gx, gy)
    yy, xx = np.mgrid[0:131, 0:257]
    d = np.sqrt(((xx + 0.5) - gx) ** 2 + ((yy + 0.5) - gy) ** 2)
    assert np.all(w[d <= 19.999] == 1.0)  # Eq. (phat), e <= r_f
    assert np.all(w > 0.0) and np.all(w <= 1.0)
    assert np.all(w[d > 20.001] < 1.0)


def test_weight_is_normalised_density_ratio(orc):
    # w(e) = d(e)/d(r_f) outside the fovea (Eq. phat); default scale puts r_f at 2.5 deg
    cfg = orc.make_config(4000, 1, 1, r_f=200.0)
    xs = np.arange(201, 4000, 7)
    w = np.array([orc.weight32(cfg, int(x), 0, 0.5, 0.5) for x in xs], np.float64)
    e = xs.astype(np.float64) * (2.5 / 200.0)
    ref = orc.density64(e) / orc.density64([2.5])[0]
    assert np.max(np.abs(w / ref - 1.0)) < 3e-6


def test_weight_continuous_and_monotone(orc):
    cfg = orc.make_config(4096, 1, 1, r_f=100.0)
    # pixel centres along a ray from the gaze: x + 0.5 - gx = x
    w = np.array([orc.weight32(cfg, x, 0, 0.5, 0.5) for x in range(0, 4096)], np.float64)
    assert np.all(w[:101] == 1.0)
    assert 1.0 - w[101] < 0.02          # continuity at r_f: one pixel past the edge
    assert np.all(np.diff(w) <= 2e-7)   # non-increasing up to FP32 rounding
    assert w[-1] < w[200] < w[101]


def test_weight_clamps_eccentricity(orc):
    cfg = orc.make_config(10, 10, 1, r_f=1.0, deg_per_px=50.0)
    w_far = orc.weight32(cfg, 9, 9, -1e6, -1e6)
    w_180 = orc.density32([180.0])[0] / orc.density32([50.0])[0]
    assert w_far == pytest.approx(float(w_180), rel=1e-6)
    assert w_far > 0.0


# ------------------------------------------------------------------ sampling laws

W6 = np.array([0.9, 0.15, 0.4, 1.0, 0.05, 0.6], np.float32)


@pytest.mark.parametrize("bias", [False, True])
def test_k1_selection_matches_chao(orc, bias):
    """K = 1: the last sample held is i with probability w_i / sum w
    (Eq. chao-selection-probability), with effective weights under the bias."""
    n_trials = 200_000
    u = _uniform_draws(11 + bias, (n_trials, len(W6)))
    idx, _ = orc.run_streams(1, bias, W6, u)
    counts = np.bincount(idx[:, 0].astype(np.int64), minlength=len(W6))
    eff = _effective_weights(W6, bias)
    assert _chi2_p(counts, eff / eff.sum()) > ALPHA


@pytest.mark.parametrize("bias", [False, True])
def test_literal_alg2_matches_same_law(orc, bias):
    """Alg. 2 applied literally (rand * (R1 + R2) <= R1 keeps R1), after
    Eq. (temporal-bias), follows the same law as the key race."""
    n_trials = 200_000
    u = _uniform_draws(21 + bias, (n_trials, len(W6)))
    idx = orc.chao_literal(bias, W6, u)
    counts = np.bincount(idx.astype(np.int64), minlength=len(W6))
    eff = _effective_weights(W6, bias)
    assert _chi2_p(counts, eff / eff.sum()) > ALPHA


def test_bias_favours_recent_samples(orc):
    # Sec. 4.2: the bias lets newer samples displace the history more easily
    w = np.ones(8, np.float32)
    u = _uniform_draws(5, (100_000, 8))
    idx_b, _ = orc.run_streams(1, True, w, u)
    idx_n, _ = orc.run_streams(1, False, w, u)
    assert np.mean(idx_b[:, 0] == 7) > np.mean(idx_n[:, 0] == 7) + 0.1


@pytest.mark.parametrize("K,bias", [(2, False), (3, False), (2, True), (3, True)])
def test_topk_subsets_match_successive_sampling(orc, K, bias):
    """K > 1: the K smallest exponential keys are a successive sample without
    replacement (A-ES); the subset law is enumerated by brute force."""
    w = W6[:5] if K == 3 else W6
    n_trials = 200_000
    u = _uniform_draws(31 + K + 10 * bias, (n_trials, len(w)))
    idx, _ = orc.run_streams(K, bias, w, u)
    law = _successive_sampling_subsets(_effective_weights(w, bias), K)
    keys = sorted(law)
    pos = {k: i for i, k in enumerate(keys)}
    subs = np.sort(idx.astype(np.int64), axis=1)
    counts = np.zeros(len(keys))
    for row, c in zip(*np.unique(subs, axis=0, return_counts=True)):
        counts[pos[tuple(int(v) for v in row)]] += c
    assert counts.sum() == n_trials
    assert _chi2_p(counts, [law[k] for k in keys]) > ALPHA


def test_equal_weights_give_uniform_subsets(orc):
    """Equal weights, no bias: classic reservoir sampling, every K-subset
    equally likely (Sec. 3.1)."""
    n, K, n_trials = 6, 3, 200_000
    u = _uniform_draws(77, (n_trials, n))
    idx, _ = orc.run_streams(K, False, np.full(n, 0.5, np.float32), u)
    subs = np.sort(idx.astype(np.int64), axis=1)
    _, counts = np.unique(subs, axis=0, return_counts=True)
    assert len(counts) == math.comb(n, K)
    assert stats.chisquare(counts).pvalue > ALPHA


def test_reservoir_size_never_exceeds_k(orc):
    rng = np.random.default_rng(3)
    for K in (1, 2, 5, 16):
        for n_items in (1, 3, K, K + 4):
            w = rng.uniform(0.01, 1.0, n_items).astype(np.float32)
            u = _uniform_draws(K * 100 + n_items, (50, n_items))
            idx, _ = orc.run_streams(K, True, w, u)
            occupied = (idx != orc.EMPTY).sum(axis=1)
            assert np.all(occupied == min(K, n_items))
            for row in idx:
                held = row[row != orc.EMPTY]
                assert len(set(held.tolist())) == len(held) and np.all(held < n_items)


def test_running_weight_sum_recursion(orc):
    """W follows Eq. (temporal-bias) then Alg. 2's sum, deterministically."""
    rng = np.random.default_rng(9)
    w = rng.uniform(0.001, 1.0, 400).astype(np.float32)
    u = _uniform_draws(1, (1, 400))
    for bias in (False, True):
        _, W = orc.run_streams(4, bias, w, u)
        ref = 0.0
        for ws in w.astype(np.float64):
            if bias and ref > 0:
                ref *= 1.0 - ws / (ref + ws)
            ref += ws
        if not bias:
            assert W[0] == pytest.approx(w.astype(np.float64).sum(), rel=1e-5)
        assert W[0] == pytest.approx(ref, rel=1e-5)


def test_bias_product_renormalisation_keeps_law(orc):
    """Weights growing 4x per item drive the bias product far below 2^-64;
    the exact power-of-two rescale must not change the sampling law."""
    n = 40
    w = (4.0 ** (np.arange(n) - n)).astype(np.float32)
    eff = _effective_weights(w, True)
    assert np.prod([1.0]) == 1.0 and eff[0] / w[0] < 2.0 ** -64  # the product does underflow 2^-64
    for K in (1, 2):
        u = _uniform_draws(500 + K, (200_000, n))
        idx, W = orc.run_streams(K, True, w, u)
        assert np.all(np.isfinite(W))
        law = _successive_sampling_subsets(eff[-8:] / eff.sum(), K) if K == 2 else None
        if K == 1:
            counts = np.bincount(idx[:, 0].astype(np.int64), minlength=n)
            assert _chi2_p(counts, eff / eff.sum()) > ALPHA
        else:
            # items before the last 8 carry < 1e-9 of the mass; test the rest
            held = np.sort(idx.astype(np.int64), axis=1)
            assert np.all(held >= n - 8)
            keys = sorted(law)
            pos = {k: i for i, k in enumerate(keys)}
            counts = np.zeros(len(keys))
            for row, c in zip(*np.unique(held - (n - 8), axis=0, return_counts=True)):
                counts[pos[tuple(int(v) for v in row)]] += c
            assert _chi2_p(counts, [law[k] for k in keys]) > ALPHA


def test_pixel_step_renormalises_bias_product(orc):
    """P is kept within [2^-64, 1] and the stored keys carry the same factor."""
    import ctypes as C
    K = 2
    W = np.zeros(1, np.float32)
    P = np.ones(1, np.float32)
    key = np.full(K, np.inf, np.float32)
    idx = np.full(K, orc.EMPTY, np.uint32)
    wt = np.zeros(K, np.float32)
    rgb = np.zeros(3 * K, np.float32)
    c = np.zeros(3, np.float32)
    lib = orc.load()
    seen_small = False
    for s in range(60):
        w = np.float32(4.0 ** (s - 60))
        before = P[0]
        lib.orc_pixel_step(K, 1, C.c_float(w), C.c_float(0.5), s, c.ctypes.data, 0, W.ctypes.data,
                           P.ctypes.data, key.ctypes.data, idx.ctypes.data, wt.ctypes.data,
                           rgb.ctypes.data)
        assert 2.0 ** -64 <= P[0] <= 1.0
        if P[0] > before:
            seen_small = True
    assert seen_small


# ------------------------------------------------------------------ resolve

def test_resolve_special_cases(orc):
    lib = orc.load()
    out = np.empty(3, np.float64)
    # K = 1: the resident sample itself (the paper's n = 1 output, Sec. 4.2)
    idx = np.array([4], np.uint32)
    wt = np.array([0.37], np.float32)
    rgb = np.array([0.1, 0.7, 0.3], np.float32)
    lib.orc_resolve_pixel(1, idx.ctypes.data, wt.ctypes.data, rgb.ctypes.data, out.ctypes.data)
    assert np.array_equal(out, rgb.astype(np.float64))
    # equal colours in every slot return that colour
    idx = np.array([1, 2, 3], np.uint32)
    wt = np.array([0.2, 0.9, 0.05], np.float32)
    rgb = np.tile(np.float32([0.25, 0.5, 0.75]), 3)
    lib.orc_resolve_pixel(3, idx.ctypes.data, wt.ctypes.data, rgb.ctypes.data, out.ctypes.data)
    assert np.allclose(out, [0.25, 0.5, 0.75], rtol=1e-15)
    # dyadic weights: exact weighted mean; empty slots ignored
    idx = np.array([0, orc.EMPTY, 5], np.uint32)
    wt = np.array([0.25, 0.5, 0.75], np.float32)
    rgb = np.array([1, 0, 0, 9, 9, 9, 0, 1, 0.5], np.float32)
    lib.orc_resolve_pixel(3, idx.ctypes.data, wt.ctypes.data, rgb.ctypes.data, out.ctypes.data)
    assert np.array_equal(out, [0.25, 0.75, 0.375])
    # no occupied slot: zero
    idx = np.full(2, orc.EMPTY, np.uint32)
    lib.orc_resolve_pixel(2, idx.ctypes.data, wt.ctypes.data, rgb.ctypes.data, out.ctypes.data)
    assert np.array_equal(out, [0.0, 0.0, 0.0])


# ------------------------------------------------------------------ frame streams

def _tiny_stream(orc, K=3, bias=True, pixels=None, w=37, h=23, frames=6, fov_flush_at=None):
    from synth import Foveator, gaze_path
    fv = Foveator(w, h, (6.0, 12.0), seed=4)
    gz = gaze_path(w, h, frames, seed=4, model="jitter", jitter_px=3.0)
    st = orc.OracleStream(w, h, K, r_f=6.0, seed=99, stream_id=2, temporal_bias=bias, pixels=pixels)
    for t in range(frames):
        fr, fm = fv.frame(*gz[t])
        fm = fm.numpy().copy()
        if fov_flush_at is not None and t == fov_flush_at:
            fm[:, : w // 2] = 0xFF
        st.push_frame(fr.numpy(), gz[t], fm)
    return st


def test_stream_state_invariants(orc):
    st = _tiny_stream(orc)
    s = st.state()
    occ = s["idx"] != orc.EMPTY
    assert np.all(occ.sum(axis=1) == min(3, 6))
    assert np.all(s["idx"][occ] < 6)
    assert np.all(np.isinf(s["key"][~occ])) and np.all(np.isfinite(s["key"][occ]))
    assert np.all(s["W"] > 0) and np.all((s["P"] > 0) & (s["P"] <= 1))
    assert np.all((s["wt"][occ] > 0) & (s["wt"][occ] <= 1))
    out = st.resolve()
    assert np.all((out >= 0) & (out <= 1))


def test_sampled_pixels_match_full_frame(orc):
    full = _tiny_stream(orc).state()
    pix = np.array([0, 5, 36, 37, 400, 850], np.int64)
    part = _tiny_stream(orc, pixels=pix).state()
    for k in full:
        assert np.array_equal(full[k][pix], part[k]), k


def test_flush_clears_history(orc):
    st = _tiny_stream(orc, fov_flush_at=5)
    s = st.state()
    w = 37
    flushed = (np.arange(37 * 23) % w) < w // 2
    # flushed pixels hold only the frame-5 sample in slot 0
    assert np.all(s["idx"][flushed, 0] == 5)
    assert np.all(s["idx"][flushed, 1:] == orc.EMPTY)
    assert np.all(s["P"][flushed] == 1.0)
    assert np.array_equal(s["W"][flushed], s["wt"][flushed, 0])
    assert np.all((s["idx"][~flushed] != orc.EMPTY).sum(axis=1) == 3)


def test_push_frame_rejects_bad_arguments(orc):
    st = orc.OracleStream(8, 4, 2, r_f=2.0)
    with pytest.raises(ValueError):
        st.push_frame(np.zeros((4, 8, 3), np.float32), (float("nan"), 1.0))
    with pytest.raises(ValueError):
        st.push_frame(np.zeros((4, 8, 3), np.float32), (1.0, 1.0), pitch=10)


def test_literal_rule_frame_path(orc):
    """The literal n = 1 rule through the frame path: the first frame always
    enters, W follows Eq. (temporal-bias) then Alg. 2's sum, a flush restarts
    the pixel, and the key and P planes are never touched."""
    st = _tiny_stream_rule(orc, rule=orc.RULE_LITERAL)
    s = st.state()
    assert np.all(s["idx"][:, 0] != orc.EMPTY) and np.all(s["idx"][:, 0] < 6)
    assert np.all(np.isinf(s["key"])) and np.all(s["P"] == 1.0)
    assert np.all((s["wt"][:, 0] > 0) & (s["wt"][:, 0] <= 1))
    first = _tiny_stream_rule(orc, rule=orc.RULE_LITERAL, frames=1).state()
    assert np.all(first["idx"][:, 0] == 0)
    assert np.array_equal(first["W"], first["wt"][:, 0])
    fl = _tiny_stream_rule(orc, rule=orc.RULE_LITERAL, flush_at=5).state()
    flushed = (np.arange(37 * 23) % 37) < 18
    assert np.all(fl["idx"][flushed, 0] == 5)
    assert np.array_equal(fl["W"][flushed], fl["wt"][flushed, 0])


def _tiny_stream_rule(orc, rule, frames=6, flush_at=None):
    from synth import Foveator, gaze_path
    w, h = 37, 23
    fv = Foveator(w, h, (6.0, 12.0), seed=4)
    gz = gaze_path(w, h, frames, seed=4, model="jitter", jitter_px=3.0)
    st = orc.OracleStream(w, h, 1, r_f=6.0, seed=99, stream_id=2, rule=rule)
    for t in range(frames):
        fr, fm = fv.frame(*gz[t])
        fm = fm.numpy().copy()
        if flush_at is not None and t == flush_at:
            fm[:, : w // 2] = 0xFF
        st.push_frame(fr.numpy(), gz[t], fm)
    return st


def test_literal_rule_rejects_k_above_one(orc):
    with pytest.raises(ValueError):
        st = orc.OracleStream(8, 4, 2, r_f=2.0, rule=orc.RULE_LITERAL)
        st.push_frame(np.zeros((4, 8, 3), np.float32), (1.0, 1.0))


# ------------------------------------------------------------------ full temporal bias

def test_lightness_special_values(orc):
    """CIE 1976 L*: 0 for black, 100 for white, 49.50 for 18% grey, continuous
    at the (6/29)^3 junction (both branches give 8), increasing in Y."""
    L = orc.lightness([[0, 0, 0], [1, 1, 1], [0.18, 0.18, 0.18]])
    assert L[0] == 0.0 and L[1] == pytest.approx(100.0, abs=1e-4)
    assert L[2] == pytest.approx(49.496, abs=2e-3)
    e = (6.0 / 29.0) ** 3
    lo, hi = orc.lightness([[e * 0.99999] * 3, [e * 1.00001] * 3])
    assert lo == pytest.approx(8.0, abs=1e-3) and hi == pytest.approx(8.0, abs=1e-3)
    y = np.linspace(0, 1, 2001)
    Ly = orc.lightness(np.repeat(y[:, None], 3, axis=1))
    assert np.all(np.diff(Ly) >= -1e-4)
    # luminance weights of sRGB primaries: pure green is lighter than pure red and blue
    r, g, b = orc.lightness(np.eye(3))
    assert g > r > b > 0


def _full_bias_pair(orc, colours, weights_inside=True, K=1, rule=0):
    """Two streams over the same 4x1 frames of uniform colour: Eq. (temporal-bias)
    and Eq. (full-temporal-bias)."""
    out = []
    for bias in (1, 2):
        st = orc.OracleStream(4, 1, K, r_f=100.0, seed=5, temporal_bias=bias, rule=rule)
        for c in colours:
            st.push_frame(np.tile(np.float32(c), (1, 4, 1)), (2.0, 0.5))
        out.append(st.state())
    return out


def test_full_bias_without_colour_change_is_temporal_bias(orc):
    for K, rule in ((1, 0), (4, 0), (1, 1)):
        a, b = _full_bias_pair(orc, [[0.3, 0.5, 0.2]] * 9, K=K, rule=rule)
        for k in a:
            assert np.array_equal(a[k], b[k]), (K, rule, k)


def test_full_bias_weight_recursion(orc):
    """Frame 0 black, frame 1 18% grey, w = 1 for both (inside the fovea):
    W1 = W0 (W0 / (W0 + w)) (1 - |Delta L|) + w with Delta L = (49.496 - 0)/100."""
    a, b = _full_bias_pair(orc, [[0, 0, 0], [0.18, 0.18, 0.18]])
    dl = 0.49496
    assert a["W"][0] == pytest.approx(1.0 * 0.5 + 1.0, rel=1e-6)
    assert b["W"][0] == pytest.approx(1.0 * 0.5 * (1 - dl) + 1.0, rel=1e-4)


def test_full_bias_total_change_flushes(orc):
    """Black to white is |Delta L| = 1: the history keeps no weight, as after a flush."""
    for K, rule in ((1, 0), (4, 0), (1, 1)):
        _, b = _full_bias_pair(orc, [[0, 0, 0]] * 5 + [[1, 1, 1]], K=K, rule=rule)
        assert np.all(b["idx"][:, 0] == 5)
        assert np.all(b["idx"][:, 1:] == orc.EMPTY)
        assert np.array_equal(b["W"], b["wt"][:, 0])


# ---------------------------------------------------------------- foveation (Sec. 4.3)

import oracle  # noqa: E402  (built on first use)

def test_foveation_constant_image_is_exact():
    # every block mean of a constant image is that constant, and both
    # reconstructions (convex combinations) return it exactly: 0.375 = 3/8
    # keeps every partial sum and quotient exact in FP32
    img = np.full((21, 37, 3), 0.375, np.float32)
    for L in range(1, 6):
        assert np.all(oracle.mip_means(img, L) == np.float32(0.375))
    for f in (oracle.FILTER_BOX, oracle.FILTER_BILINEAR):
        fr, ring = oracle.foveate(img, (3.0, 6.0, 10.0, 14.0, 20.0), 11.0, 9.0, f)
        assert np.all(fr == np.float32(0.375))
        assert ring.max() == 5 and ring.min() == 0


def _ramp(w, h):
    img = np.zeros((h, w, 3), np.float32)
    img[:, :, 0] = (np.arange(w) / 128.0)[None, :]
    img[:, :, 1] = (np.arange(h) / 64.0)[:, None]
    img[:, :, 2] = 0.25
    return img


def test_foveation_dyadic_ramp_closed_forms():
    # block means of a linear ramp are the ramp at the block centre, and
    # bilinear filtering of block means reproduces a linear ramp wherever no
    # clamp applies; dyadic values make both exact in FP32
    w, h = 64, 32
    img = _ramp(w, h)
    radii = (0.5, 0.75, 1.0)  # every pixel centre lies beyond all: level 3 everywhere
    for L in (1, 2, 3):
        b = 1 << L
        m = oracle.mip_means(img, L)
        cx = (np.arange(w // b) * b + (b - 1) / 2.0) / 128.0
        cy = (np.arange(h // b) * b + (b - 1) / 2.0) / 64.0
        assert np.array_equal(m[:, :, 0], np.broadcast_to(cx[None, :], m.shape[:2]).astype(np.float32))
        assert np.array_equal(m[:, :, 1], np.broadcast_to(cy[:, None], m.shape[:2]).astype(np.float32))
    fr, ring = oracle.foveate(img, radii, -100.0, -100.0, oracle.FILTER_BILINEAR)
    assert np.all(ring == 3)
    inner = (slice(4, h - 4), slice(4, w - 4))
    assert np.array_equal(fr[inner], img[inner])
    fb, _ = oracle.foveate(img, radii, -100.0, -100.0, oracle.FILTER_BOX)
    m3 = oracle.mip_means(img, 3)
    assert np.array_equal(fb, np.repeat(np.repeat(m3, 8, 0), 8, 1))


def test_foveation_bilinear_texel_centre_weights():
    # textbook bilinear magnification by 2 with texel-centre sampling and
    # clamp-to-edge: level-1 means [0, 1] give pixel colours [0, 1/4, 3/4, 1]
    img = np.zeros((2, 4, 3), np.float32)
    img[:, 2:] = 1.0
    fr, ring = oracle.foveate(img, (0.25,), -50.0, -50.0, oracle.FILTER_BILINEAR)
    assert np.all(ring == 1)
    assert np.array_equal(fr[0, :, 0], np.array([0.0, 0.25, 0.75, 1.0], np.float32))
    # and vertically: a [0; 1] column of level-1 means
    img = np.zeros((4, 2, 3), np.float32)
    img[2:] = 1.0
    fr, _ = oracle.foveate(img, (0.25,), -50.0, -50.0, oracle.FILTER_BILINEAR)
    assert np.array_equal(fr[:, 0, 1], np.array([0.0, 0.25, 0.75, 1.0], np.float32))


def test_foveation_ring_boundaries_exact():
    from fractions import Fraction as Fr
    w, h = 24, 18
    gx, gy = 10.25, 7.5
    radii = (2.5, 5.0, 7.75)
    img = np.zeros((h, w, 3), np.float32)
    _, ring = oracle.foveate(img, radii, gx, gy, oracle.FILTER_BOX)
    on_boundary = 0
    for y in range(h):
        for x in range(w):
            d2 = (Fr(2 * x + 1, 2) - Fr(gx)) ** 2 + (Fr(2 * y + 1, 2) - Fr(gy)) ** 2
            expect = sum(d2 > Fr(r) ** 2 for r in radii)
            on_boundary += any(d2 == Fr(r) ** 2 for r in radii)
            assert ring[y, x] == expect, (x, y)
    assert on_boundary > 0  # the inclusive boundary case is exercised


def test_foveation_mirror_symmetry():
    # mirroring the image and the gaze mirrors the output exactly (widths are
    # multiples of the largest block, so blocks map onto blocks; addition is
    # commutative and the bilinear weights swap): catches swapped weights or
    # a wrong neighbour index
    from synth import ground_truth
    w, h = 64, 40
    img = ground_truth(w, h, seed=8)
    radii = (5.0, 11.0, 17.0)
    gx, gy = 23.25, 14.5
    for f in (oracle.FILTER_BOX, oracle.FILTER_BILINEAR):
        a, ra = oracle.foveate(img, radii, gx, gy, f)
        b, rb = oracle.foveate(np.ascontiguousarray(img[:, ::-1]), radii, w - gx, gy, f)
        assert np.array_equal(ra, rb[:, ::-1])
        assert np.array_equal(a, b[:, ::-1])
        c, rc = oracle.foveate(np.ascontiguousarray(img[::-1]), radii, gx, h - gy, f)
        assert np.array_equal(ra, rc[::-1])
        assert np.array_equal(a, c[::-1])


def test_foveation_means_within_rounding_of_fp64():
    rng = np.random.default_rng(3)
    img = rng.random((45, 70, 3)).astype(np.float32)
    for L in range(1, 6):
        b = 1 << L
        m = oracle.mip_means(img, L)
        for by in range(m.shape[0]):
            for bx in range(m.shape[1]):
                ref = img[by * b:(by + 1) * b, bx * b:(bx + 1) * b].astype(np.float64).mean(axis=(0, 1))
                # 2L tree additions and one division, each within 2^-24 relative
                assert np.all(np.abs(m[by, bx] - ref) <= (2 * L + 1) * 2.0 ** -24 * ref + 1e-30)


def test_foveation_rejects_bad_arguments():
    img = np.zeros((4, 4, 3), np.float32)
    for radii in ((), (2.0, 1.0), (1.0,) * 6, (0.0,), (float("nan"),)):
        with pytest.raises(ValueError):
            oracle.foveate(img, radii, 1.0, 1.0)
    with pytest.raises(ValueError):
        oracle.foveate(img, (1.0,), 1.0, 1.0, filter=2)


def test_foveation_matches_the_input_generator():
    # the seeded input generator (numpy/torch) and the oracle (C loops) are
    # written separately from the same definition
    from synth import Foveator
    radii = (4.0, 9.0, 15.0)
    for name, f in (("box", oracle.FILTER_BOX), ("bilinear", oracle.FILTER_BILINEAR)):
        fv = Foveator(53, 29, radii, seed=6, filter=name)
        a, ra = oracle.foveate(fv.gt_numpy, radii, 20.3, 11.7, f)
        b, rb = fv.frame(20.3, 11.7)
        assert np.array_equal(ra, rb.numpy()) and np.array_equal(a, b.numpy())


# ---------------------------------------------------------------- reprojection (Sec. 4.3)

def _rp_frames(w, h, n, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, h, w, 3)).astype(np.float32), rng.uniform(0, [w, h], size=(n, 2))


@pytest.mark.parametrize("K,rule,bias", [(4, 0, 1), (3, 0, 2), (1, 1, 1), (2, 0, 0)])
def test_reproject_without_motion_is_the_plain_push(K, rule, bias):
    # zero motion and matching depth: every pixel keeps its own history, so
    # the reprojected push reduces to the plain one bit for bit
    w, h = 13, 9
    frames, gaze = _rp_frames(w, h, 7, seed=K)
    depth = np.full((h, w), 3.0, np.float32)
    a = oracle.OracleStream(w, h, K, 3.0, seed=5, temporal_bias=bias, rule=rule)
    b = oracle.OracleStream(w, h, K, 3.0, seed=5, temporal_bias=bias, rule=rule)
    for t in range(7):
        fm = None
        if t == 4:
            fm = np.zeros((h, w), np.uint8)
            fm[2:5, 3:9] = 0xFF
        a.push_frame(frames[t], gaze[t], fm)
        mv = np.zeros((h, w, 2), np.float32) if t % 2 else None
        b.push_frame_reproject(frames[t], gaze[t], mv, depth, depth, 0.01, fm)
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k].view(np.uint32) if sa[k].dtype == np.float32 else sa[k],
                              sb[k].view(np.uint32) if sb[k].dtype == np.float32 else sb[k]), k


@pytest.mark.parametrize("motion", [(2.0, -1.0), (2.3, -0.8), (1.7, -1.49)])
def test_reproject_pan_slot_provenance(motion):
    # with K above the frame count every candidate is inserted, so each slot's
    # provenance follows in closed form: at a pan of s pixels per frame the
    # history of p is the previous reservoir at p - s (nearest centre), and a
    # chain that starts outside the frame restarts empty
    w, h, K, T = 11, 8, 16, 6
    frames, gaze = _rp_frames(w, h, T, seed=3)
    st = oracle.OracleStream(w, h, K, 2.5, seed=9)
    mv = np.broadcast_to(np.array(motion, np.float32), (h, w, 2)).copy()
    sx, sy = int(np.floor(0.5 + motion[0])), int(np.floor(0.5 + motion[1]))  # integer source shift
    prov = {(x, y): [(0, x, y)] for x in range(w) for y in range(h)}
    st.push_frame_reproject(frames[0], gaze[0], mv)
    for t in range(1, T):
        st.push_frame_reproject(frames[t], gaze[t], mv)
        nxt = {}
        for x in range(w):
            for y in range(h):
                src = (x - sx, y - sy)
                hist = prov[src] if (0 <= src[0] < w and 0 <= src[1] < h) else []
                nxt[(x, y)] = hist + [(t, x, y)]
        prov = nxt
    s = st.state()
    for (x, y), lst in prov.items():
        p = y * w + x
        occ = [j for j in range(K) if s["idx"][p, j] != oracle.EMPTY]
        assert occ == list(range(len(lst))), (x, y)
        for j, (f, xs, ys) in enumerate(lst):
            assert s["idx"][p, j] == f
            assert np.array_equal(s["rgb"][p, j], frames[f][ys, xs])
            cfg = oracle.make_config(w, h, K, 2.5, seed=9)
            assert s["wt"][p, j] == np.float32(oracle.weight32(cfg, xs, ys, *gaze[f]))


def test_reproject_centre_rounding():
    # the source is the pixel containing the moved centre: a motion of +0.5
    # lands on the pixel's own left edge (kept), -0.5 on the right neighbour's
    # left edge; 2^-10 past either edge crosses it (dyadic: every step exact)
    w, h = 6, 3
    frames, gaze = _rp_frames(w, h, 2, seed=1)
    e = 2.0 ** -10
    for m, shift in ((0.5, 0), (-0.5, 1), (0.5 + e, -1), (0.5 - e, 0), (-0.5 - e, 1),
                     (-0.5 + e, 0)):
        st = oracle.OracleStream(w, h, 4, 2.0, seed=2)
        st.push_frame(frames[0], gaze[0])
        mv = np.zeros((h, w, 2), np.float32)
        mv[:, :, 0] = m
        st.push_frame_reproject(frames[1], gaze[1], mv)
        s = st.state()
        for x in range(w):
            src = x + shift
            n_occ = int(np.sum(s["idx"][x] != oracle.EMPTY))
            if 0 <= src < w:
                assert n_occ == 2 and np.array_equal(s["rgb"][x, 0], frames[0][0, src])
            else:
                assert n_occ == 1
    # vertically: -0.5 moves the bottom row's centres onto the frame's lower
    # edge, which lies outside (the frame is [0, h) x [0, w))
    st = oracle.OracleStream(w, h, 4, 2.0, seed=2)
    st.push_frame(frames[0], gaze[0])
    mv = np.zeros((h, w, 2), np.float32)
    mv[:, :, 1] = -0.5
    st.push_frame_reproject(frames[1], gaze[1], mv)
    occ = np.sum(st.state()["idx"] != oracle.EMPTY, axis=1).reshape(h, w)
    assert np.all(occ[:h - 1] == 2) and np.all(occ[h - 1] == 1)


def test_reproject_depth_test_flushes_occlusions():
    w, h = 8, 4
    frames, gaze = _rp_frames(w, h, 3, seed=4)
    cur = np.full((h, w), 4.0, np.float32)
    prev = cur.copy()
    prev[:, 2] = 5.0      # |5 - 4| = 1 = tol * 4: kept (strict test)
    prev[:, 3] = 5.5      # beyond the tolerance: flushed
    prev[:, 4] = 2.0      # a nearer surface moved away (disocclusion): flushed
    st = oracle.OracleStream(w, h, 4, 2.0, seed=2)
    st.push_frame(frames[0], gaze[0])
    st.push_frame(frames[1], gaze[1])
    st.push_frame_reproject(frames[2], gaze[2], None, cur, prev, 0.25)
    s = st.state()
    cfg = oracle.make_config(w, h, 4, 2.0, seed=2)
    for x in range(w):
        n_occ = int(np.sum(s["idx"][x] != oracle.EMPTY))
        if x in (3, 4):
            assert n_occ == 1 and s["idx"][x, 0] == 2
            assert s["W"][x] == np.float32(oracle.weight32(cfg, x, 0, *gaze[2]))
        else:
            assert n_occ == 3
    with pytest.raises(ValueError):
        st.push_frame_reproject(frames[2], gaze[2], None, cur, None, 0.25)
