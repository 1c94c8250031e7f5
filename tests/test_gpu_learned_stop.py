"""Learned early termination: traces, training kernels, fused inference.

* Trace change flags equal what the oracle's pool trace (Alg. 1, pool after
  every expansion) implies: step t changed the first k ids or not.
* Training kernels: Adam's first step moves every parameter by -lr*sign(g);
  the signs must match the gradient of the mean binary cross-entropy
  computed with numpy from the same traces (the plain definition).
* Features: all 8, before every expansion, equal the values rebuilt from the
  oracle's pool trace (exact divisions bit for bit, the logarithm to 2e-7).
* Inference: a model that never stops reproduces the fixed-L search exactly;
  one that always stops ends after `stop_min_steps` expansions; a random
  non-zero model stops every query at the step, and with the pool, that the
  MLP evaluated in numpy on the traced features predicts.
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


def _exact_d2(base, q, ids):
    # integer data: exact squared distances, float32 holds them exactly
    diff = base[ids].astype(np.int64) - q.astype(np.int64)
    return (diff * diff).sum(-1).astype(np.float32)


def _oracle_features(adj, deg, base, nav, q, L, k, cap):
    """The 8 stop features before every expansion of Alg. 1, rebuilt from the
    oracle's pool after each step: the expanded node is the first pool entry
    not yet expanded, its fresh neighbours are those never measured before,
    and a step changes the first k when their id set differs."""
    pools = oracle.search_trace(adj, base, nav, q, L, max_steps=cap, deg=deg)
    width = adj.shape[1]
    f32 = np.float32
    feats = []
    expanded, visited = set(), {nav}
    since, last_changed, last_m = 0, True, 0
    prev = [nav]
    for t in range(len(pools)):
        ids = [int(x) for x in prev if x >= 0]
        dd = _exact_d2(base, q, np.array(ids))
        size = len(ids)
        i = next(j for j in range(size) if ids[j] not in expanded)
        kk = min(k, size)
        d0, dk, dn, dl = dd[0], dd[kk - 1], dd[i], dd[size - 1]
        f = np.zeros(8, np.float32)
        f[0] = min(f32(t) / f32(L), f32(4.0)) * f32(0.25)
        f[1] = d0 / dk if dk > 0 else 1.0
        f[2] = min(dk / dn, f32(4.0)) if dn > 0 else 1.0
        f[3] = dk / dl if dl > 0 else 1.0
        f[4] = np.log2(f32(1.0) + f32(since)) * f32(0.125)
        f[5] = f32(i) / f32(L)
        f[6] = f32(last_m) / f32(width)
        f[7] = 1.0 if last_changed else 0.0
        feats.append(f)
        u = ids[i]
        expanded.add(u)
        fresh = [int(v) for v in adj[u, :deg[u]] if v >= 0 and int(v) not in visited]
        visited.update(fresh)
        last_m = len(fresh)
        cur = [int(x) for x in pools[t] if x >= 0]
        last_changed = set(cur[:k]) != set(ids[:k])
        since = 0 if last_changed else since + 1
        prev = pools[t]
    return np.array(feats), pools


def test_every_trace_feature_matches_the_oracle(nsg, setup):
    base, q, ref, idx, _ = setup
    L, cap = 60, 400
    tr = idx.search_trace(T(q[:30]), 10, L, cap, params=nsg.SearchParams(0, 16384, 0, 0, -1, None, 0.5, KS))
    feat, steps = H(tr["feat"]), H(tr["steps"])
    for i in range(30):
        want, pools = _oracle_features(ref["adj"], ref["deg"], base, ref["nav"], q[i], L, KS, cap)
        assert steps[i] == len(pools) == len(want)
        got = feat[i, :steps[i]]
        exact = [0, 1, 2, 3, 5, 6, 7]  # correctly rounded divisions of exact values
        assert np.array_equal(got[:, exact], want[:, exact]), i
        assert np.allclose(got[:, 4], want[:, 4], rtol=2e-7, atol=0), i


def _logits(w, feat):
    # the MLP 8 -> 64 (ReLU) -> 1 in float64 from the FP16 parameters
    w = w.astype(np.float64)
    W1, b1, w2, b2 = w[:512].reshape(64, 8), w[512:576], w[576:640], w[640]
    return np.maximum(feat.astype(np.float64) @ W1.T + b1, 0.0) @ w2 + b2


def test_fused_mlp_stops_where_numpy_predicts(nsg, setup):
    # random non-zero weights: the stop step and result of every query follow
    # from the traced features, the threshold and the evaluation schedule
    # (from min_steps on, every 4th expansion)
    base, q, ref, idx, _ = setup
    L, cap, min_steps, thr = 80, 600, 3, 0.7
    tr = idx.search_trace(T(q), 10, L, cap, params=nsg.SearchParams(0, 16384, 0, 0, -1, None, 0.5, KS))
    feat, steps = H(tr["feat"]), H(tr["steps"])
    assert steps.max() < cap
    rng = np.random.default_rng(11)
    w = np.zeros(641, np.float64)
    w[:512] = rng.standard_normal(512) * 2.0
    w[512:576] = rng.standard_normal(64) * 0.5
    w[576:640] = rng.standard_normal(64) / 8.0
    elig = [np.arange(min_steps, steps[i], 4) for i in range(len(q))]
    zt = np.log(thr / (1 - thr))
    # the output bias that makes about half of the queries stop early
    zmax = [_logits(np.r_[w[:640], 0.0].astype(np.float16), feat[i, e]).max() for i, e in enumerate(elig)]
    w[640] = zt - np.median(zmax)
    w16 = w.astype(np.float16)
    assert (w16[:640] != 0).sum() > 600
    model = T(w16)
    out = idx.search_ex(T(q), 10, L, params=nsg.SearchParams(0, 16384, 0, 0, -1, model, thr, KS, min_steps))
    ne, ids = H(out["n_expand"]), H(out["ids"])
    checked = stopped = 0
    for i in range(len(q)):
        zi = _logits(w16, feat[i, elig[i]])
        fire = np.nonzero(zi > zt)[0]
        stop_at = int(elig[i][fire[0]]) if len(fire) else int(steps[i])
        upto = zi[:fire[0] + 1] if len(fire) else zi
        if len(upto) and np.abs(upto - zt).min() < 1e-3:
            continue  # too close to the threshold for float32 vs float64 to agree
        checked += 1
        stopped += len(fire) > 0
        assert ne[i] == stop_at, i
        pools = oracle.search_trace(ref["adj"], base, ref["nav"], q[i], L, max_steps=cap, deg=ref["deg"])
        pool = np.array([ref["nav"]] + [-1] * 9) if stop_at == 0 else pools[stop_at - 1][:10]
        assert np.array_equal(ids[i], pool), i
    assert checked >= 0.9 * len(q)
    assert 0.2 * checked < stopped < checked  # some stop early, some run to the end
