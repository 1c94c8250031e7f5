"""Learned early termination: traces, training kernels, fused inference.

* Trace change flags equal what the oracle's pool trace (Alg. 1, pool after
  every expansion) implies: step t changed the first k ids or not.
* Training kernels: Adam's first step moves every parameter by -lr*sign(g);
  the signs must match the gradient of the mean binary cross-entropy
  computed with numpy from the same traces (the plain definition).
* Inference: a model that never stops reproduces the fixed-L search exactly;
  one that always stops ends after `stop_min_steps` expansions.
* A trained model trades expansions for a bounded recall loss (the fixed-L
  search is the yardstick)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu
KS = 10


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def setup(nsg):
    base, q = datagen.workload("tiny", n=8000, nq=200)
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    gt, _ = oracle.knn_query(base, q, 10)
    return base, q, ref, idx, gt


def test_trace_flags_match_oracle_pool_trace(nsg, setup):
    base, q, ref, idx, _ = setup
    L, cap = 60, 400
    tr = idx.search_trace(T(q[:20]), 10, L, cap, params=nsg.SearchParams(0, 16384, 0, 0, -1, None, 0.5, KS))
    flags, steps, feat = H(tr["flag"]), H(tr["steps"]), H(tr["feat"])
    for i in range(20):
        pools = oracle.search_trace(ref["adj"], base, ref["nav"], q[i], L, max_steps=cap, deg=ref["deg"])
        assert steps[i] == len(pools)
        prev = {ref["nav"]}
        for t, pool in enumerate(pools):
            cur = set(int(x) for x in pool[:KS] if x >= 0)
            assert flags[i, t] == (1 if cur != prev else 0), (i, t)
            prev = cur
        f = feat[i, :steps[i]]
        assert np.isfinite(f).all()
        assert np.allclose(f[:, 0], np.minimum(np.arange(steps[i]) / L, 4.0) * 0.25, atol=1e-6)
        assert (f[:, 5] >= 0).all() and (f[:, 5] < 1).all()
        assert (f[:, 1] >= 0).all() and (f[:, 1] <= 1).all() and (f[:, 3] <= 1).all()


def _numpy_grad(w, feat, flag, steps):
    W1 = w[:512].reshape(64, 8)
    b1, w2, b2 = w[512:576], w[576:640], w[640]
    X, Y = [], []
    for i in range(len(steps)):
        Tq = int(steps[i])
        fl = flag[i, :Tq]
        last = int(np.nonzero(fl)[0].max()) if fl.any() else -1
        X.append(feat[i, :Tq])
        Y.append((np.arange(Tq) > last).astype(np.float64))
    X = np.concatenate(X).astype(np.float64)
    Y = np.concatenate(Y)
    A = X @ W1.T + b1
    Hh = np.maximum(A, 0)
    z = Hh @ w2 + b2
    p = 1 / (1 + np.exp(-z))
    dz = (p - Y) / len(Y)
    gw2 = Hh.T @ dz
    gb2 = dz.sum()
    dA = np.outer(dz, w2) * (A > 0)
    gW1 = dA.T @ X
    gb1 = dA.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])


def test_training_gradient_sign_matches_numpy(nsg, setup):
    base, q, ref, idx, _ = setup
    tr = idx.search_trace(T(q), 10, 80, 400)
    rng = np.random.default_rng(0)
    w0 = (rng.standard_normal(641) * 0.3).astype(np.float32)
    master = T(w0.copy())
    lr = 1e-3
    model, master, loss = nsg.nsg_stop_train(tr, iters=1, lr=lr, seed=0, master=master)
    step = w0.astype(np.float64) - H(master).astype(np.float64)
    g = _numpy_grad(w0.astype(np.float64), H(tr["feat"]), H(tr["flag"]), H(tr["steps"]))
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    assert big.sum() > 100
    assert np.array_equal(np.sign(step[big]), np.sign(g[big]))
    assert np.allclose(np.abs(step[big]), lr, rtol=1e-3)
    assert np.allclose(H(model).astype(np.float32), H(master), rtol=1e-3, atol=1e-3)


def _const_model(nsg, b2):
    w = np.zeros(641, np.float16)
    w[640] = b2
    return T(w)


def test_never_stop_is_the_fixed_search(nsg, setup):
    base, q, ref, idx, _ = setup
    never = _const_model(nsg, -30.0)
    a = idx.search_ex(T(q), 10, 60)
    b = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, 0, 0, -1, never, 0.5, KS))
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["n_expand"], b["n_expand"])


def test_always_stop_respects_min_steps(nsg, setup):
    base, q, ref, idx, _ = setup
    always = _const_model(nsg, 30.0)
    out = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, 0, 0, -1, always, 0.5, KS, 7))
    assert (H(out["n_expand"]) == 7).all()


def test_trained_model_saves_steps_with_bounded_recall_loss(nsg, setup):
    base, q, ref, idx, gt = setup
    train_q = datagen.workload("tiny", n=8000, nq=2000, seed_query=77)[1]
    tr = idx.search_trace(T(train_q), 10, 100, 600)
    model, master, loss = nsg.nsg_stop_train(tr, iters=300, lr=1e-2, seed=3)
    loss = H(loss)
    assert loss[-1] < loss[0]
    plain = idx.search_ex(T(q), 10, 100)
    lrn = idx.search_ex(T(q), 10, 100, params=nsg.SearchParams(0, 0, 0, 0, -1, model, 0.9, KS))
    r_plain = oracle.recall(H(plain["ids"]), gt, 10)
    r_lrn = oracle.recall(H(lrn["ids"]), gt, 10)
    assert H(lrn["n_expand"]).mean() < H(plain["n_expand"]).mean()
    assert r_lrn >= r_plain - 0.05
