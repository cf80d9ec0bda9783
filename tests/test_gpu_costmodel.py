"""The cost model's CUDA kernels against the fp64 oracle, and its training."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _problem(seed, B, D, H):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.5, size=H * D + 2 * H + 1).astype(np.float32)
    X = rng.normal(size=(B, D)).astype(np.float32)
    T = rng.normal(size=B).astype(np.float32)
    return p, X, T


def _call(name, *args):
    from paper_2201_10473_gb300 import costmodel
    st = getattr(costmodel._lib(), name)(*args)
    assert st == 0, (name, st)


@pytest.mark.parametrize("B,D,H", [(1, 1, 1), (7, 5, 6), (300, 16, 64), (1000, 16, 64), (33, 64, 128)])
def test_forward_and_gradient_match_oracle(B, D, H):
    from paper_2201_10473_gb300 import costmodel
    p, X, T = _problem(B + D + H, B, D, H)
    dp, dX, dT = (torch.from_numpy(v).cuda() for v in (p, X, T))
    Y = torch.empty(B, dtype=torch.float32, device="cuda")
    G = torch.empty(costmodel.param_count(D, H), dtype=torch.float32, device="cuda")
    L = torch.empty(1, dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _call("gf2x_mlp_forward", dp.data_ptr(), dX.data_ptr(), Y.data_ptr(), B, D, H, s)
    _call("gf2x_mlp_grad", dp.data_ptr(), dX.data_ptr(), dT.data_ptr(), G.data_ptr(), L.data_ptr(), B, D, H, s)
    torch.cuda.synchronize()
    y_ref = omlp.forward(p, X, D, H)
    L_ref, g_ref = omlp.loss_and_grad(p, X, T, D, H)
    # fp32 sums of D or H terms of O(1) magnitude: relative error well below 1e-4
    assert np.allclose(Y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4)
    assert np.isclose(L.item(), L_ref, rtol=1e-4, atol=1e-5)
    scale = np.abs(g_ref).max() + 1e-6
    assert np.abs(G.cpu().numpy() - g_ref).max() / scale < 1e-4


def test_adam_step_matches_oracle():
    from paper_2201_10473_gb300 import costmodel  # noqa: F401
    rng = np.random.default_rng(5)
    n = 1000
    p, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = rng.normal(size=n).astype(np.float32) * 0.1, np.abs(rng.normal(size=n)).astype(np.float32) * 0.1
    dp, dg, dm, dv = (torch.from_numpy(x.copy()).cuda() for x in (p, g, m, v))
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _call("gf2x_mlp_adam", dp.data_ptr(), dg.data_ptr(), dm.data_ptr(), dv.data_ptr(), n, ctypes.c_float(1e-2),
          ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), 3, s)
    q, m2, v2 = omlp.adam_step(p.astype(np.float64), g, m, v, 1e-2, 0.9, 0.999, 1e-8, 3)
    assert np.allclose(dp.cpu().numpy(), q, rtol=1e-5, atol=1e-6)
    assert np.allclose(dm.cpu().numpy(), m2, rtol=1e-5, atol=1e-7)
    assert np.allclose(dv.cpu().numpy(), v2, rtol=1e-5, atol=1e-7)


def test_training_fits_a_known_function():
    """The GPU-trained network learns y = sum of features on synthetic data."""
    from paper_2201_10473_gb300 import costmodel
    m = costmodel.CostModel(seed=3)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(2000, costmodel.IN_DIM)).astype(np.float32)
    T = X[:, :4].sum(axis=1) + 0.5 * np.maximum(X[:, 4], 0)
    m.mu, m.sd = np.zeros(costmodel.IN_DIM, np.float32), np.ones(costmodel.IN_DIM, np.float32)
    m.t_mu, m.t_sd = 0.0, 1.0
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    G = torch.zeros(m.np, device="cuda")
    M = torch.zeros_like(G)
    V = torch.zeros_like(G)
    L = torch.zeros(1, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    first = None
    for step in range(1, 1501):
        _call("gf2x_mlp_grad", m.params.data_ptr(), Xd.data_ptr(), Td.data_ptr(), G.data_ptr(), L.data_ptr(), 2000,
              costmodel.IN_DIM, m.hidden, s)
        if first is None:
            first = L.item()
        _call("gf2x_mlp_adam", m.params.data_ptr(), G.data_ptr(), M.data_ptr(), V.data_ptr(), m.np,
              ctypes.c_float(3e-3), ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), step, s)
    assert L.item() < 0.02 * first


@pytest.mark.parametrize("holdout", [17669, 57637])
def test_learned_model_beats_unguided_search(holdout):
    """Trained by the CUDA kernels on the GB300 timing log of the other sizes,
    the network orders the held-out size's candidates so that a plan within 5%
    of the exhaustive best comes far earlier than in random order, and its top
    10 are within 10% of the best (exhaustive search gives the best)."""
    from paper_2201_10473_gb300 import autotune, costmodel
    r = costmodel.evaluate_gain(costmodel.training_records(autotune.packaged_log()), holdout, 2048, k=10, steps=3000)
    assert r["model_measurements_to_5pct"] * 4 <= r["random_expected_measurements_to_5pct"], r
    assert r["regret_top_k"] <= 0.10, r


def test_guided_search_on_an_unseen_size():
    """Live on the GPU, at a size the timing log never saw: the network
    (trained on the log) picks 10 candidates to measure, and the best of them
    is within 10% of the best of an exhaustive measured search over all of
    them (several thousand) -- the regret check of the learned part."""
    from paper_2201_10473_gb300 import Context, autotune, costmodel
    n, batch = 30011, 2048
    model = costmodel.CostModel(seed=1)
    model.fit(costmodel.training_records(autotune.packaged_log()), steps=3000)
    tuner = autotune.Autotuner(Context(0, plan_db=None), None, reps=3, warmup=1)
    try:
        cands = autotune.candidate_specs(n)
        guided = tuner.search(n, batch, model.rank(n, batch, cands)[:10])
        full = tuner.search(n, batch, cands)
        assert guided and len(full) > 100 * len(guided) // 10
        best = full[0].ms
        assert guided[0].ms <= 1.10 * best, (guided[0].spec, guided[0].ms, full[0].spec, best)
    finally:
        tuner.ctx.close()
