"""Pins of the oracle's MLP surrogate (a spec addition; the paper has no surrogate):
gradients against fp64 finite differences, the fp32 same-order gradient against fp64, SGD in
closed form, bf16 rounding, and the surrogate run reducing to the plain run."""
import struct

import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W


def _batch(O, D, N, B, seed):
    rng = np.random.default_rng(seed)
    r = np.full(N, D // N)
    base = np.arange(N) * (D // N)
    feats = (base + (rng.random((B, N)) * r).astype(np.int64)).astype(np.int32)
    y = rng.normal(size=B).astype(np.float32)
    return feats, y


def test_gradient_finite_differences_fp64(oracle_mod):
    O = oracle_mod
    D, H, N, B = 12, 16, 4, 7
    p = O.mlp_init(D, H, seed=5).astype(np.float64)
    p += np.random.default_rng(1).normal(scale=0.05, size=len(p))      # break symmetry, non-zero biases
    feats, y = _batch(O, D, N, B, 2)
    loss, g = O.mlp_loss64(p, D, H, feats, y)
    rng = np.random.default_rng(3)
    for e in rng.choice(len(p), 60, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[e] += h
        pm[e] -= h
        num = (O.mlp_loss64(pp, D, H, feats, y, False)[0] - O.mlp_loss64(pm, D, H, feats, y, False)[0]) / (2 * h)
        assert abs(num - g[e]) <= 1e-6 * max(1.0, abs(g[e])) + 1e-8, e


def test_fp32_gradient_close_to_fp64(oracle_mod):
    O = oracle_mod
    D, H, N, B = 53, 256, 10, 64
    p = O.mlp_init(D, H, seed=7)
    p_bf = np.array([O.bf16_round(float(x)) for x in p], np.float32)   # weights as the forward sees them
    n_w1 = H * D
    feats, y = _batch(O, D, N, B, 4)
    g32 = O.mlp_grad(p, D, H, feats, y)
    # fp64 reference at the bf16-rounded weights (biases are used unrounded by both)
    p64 = p_bf.astype(np.float64)
    vb = O.mlp_param_count(D, H)
    # biases: positions of b1, b2, b3, b4 keep their fp32 values
    offs = [n_w1, n_w1 + H + H * H, n_w1 + 2 * (H + H * H), vb - 1]
    for o, ln in zip(offs, [H, H, H, 1]):
        p64[o:o + ln] = p[o:o + ln]
    _, g64 = O.mlp_loss64(p64, D, H, feats, y)
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    assert rel < 1e-5
    pr = O.mlp_forward(p, D, H, feats)
    assert pr.shape == (B,) and np.isfinite(pr).all()


def test_sgd_closed_form(oracle_mod):
    O = oracle_mod
    p = np.array([1.0, -2.0, 0.5], np.float32)
    m = np.array([0.1, 0.0, -0.3], np.float32)
    g = np.array([0.5, 1.0, 0.0], np.float32)
    O.mlp_sgd(p, m, g, lr=0.5, mu=0.9)
    assert np.allclose(m, [0.59, 1.0, -0.27], atol=1e-7)
    assert np.allclose(p, [1.0 - 0.295, -2.5, 0.5 + 0.135], atol=1e-7)


def test_bf16_round_nearest_even():
    from oracle import oracle as O
    O.build()
    f = lambda u: struct.unpack("<f", struct.pack("<I", u))[0]
    assert O.bf16_round(f(0x3F808000)) == f(0x3F800000)      # tie, even stays
    assert O.bf16_round(f(0x3F818000)) == f(0x3F820000)      # tie, odd rounds up
    assert O.bf16_round(f(0x3F80C000)) == f(0x3F810000)      # above half
    assert O.bf16_round(1.0) == 1.0


@pytest.mark.parametrize("kind", ["de", "ga"])
def test_pool_of_one_equals_plain(oracle_mod, kind):
    """A pool of one proposal leaves nothing to screen: the run equals the plain run."""
    O = oracle_mod
    sd = W.tiny_space()
    sp = O.from_def(sd)
    keys = O.valid_keys(sp)
    t = W.lognormal_table(len(keys), seed=0)
    E = O.run(kind, sp, keys, t, pop=20, gens=12, seed=2)
    S = O.run(kind, sp, keys, t, pop=20, gens=12, seed=2, surrogate=dict(pool=1, H=32, batch=32, steps=2),
              log_table=np.log(t.astype(np.float64)).astype(np.float32))
    for f in ("cand", "rep", "evalk", "fit", "popk", "popf", "best_key", "n_unique"):
        assert np.array_equal(E[f], S[f]), f
    assert S["s_ne"][-1] == E["n_unique"][-1]


def test_screening_picks_lowest_prediction(oracle_mod):
    """With screening on (low warm-up), evaluated configurations differ from the plain run and the
    evaluated set grows by exactly the new unique evaluations."""
    O = oracle_mod
    sd = W.medium_space()
    sp = O.from_def(sd)
    keys = O.valid_keys(sp)
    t = W.smooth_table(sd, O.unpack(sp, keys), seed=0)
    logt = np.log(t.astype(np.float64)).astype(np.float32)
    cfg = dict(pool=4, H=32, batch=64, steps=4, warm_mult=1, mae_ratio=10.0)
    S = O.run("de", sp, keys, t, pop=32, gens=6, seed=1, surrogate=cfg, log_table=logt)
    assert S["s_used"][0] == 0 and S["s_used"][2:].all()
    assert np.array_equal(S["s_ne"], S["n_unique"].astype(np.int64))
    E = O.run("de", sp, keys, t, pop=32, gens=6, seed=1)
    assert not np.array_equal(S["evalk"][2:], E["evalk"][2:])
