"""What the learned estimator gains over the method without it.

Samples come from the reduced design-study variants (greedy ROMs after 1..5
expansion points, true output errors from full-order sweeps).  Trained on the
first variants by the GPU kernels, the network predicts the log10 output error
of held-out variants more accurately than the residual estimate does (as-is, or
calibrated by a least-squares line on the training set)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


def test_estimator_beats_the_residual_as_error_predictor():
    need_cuda()
    from paper_2310_04734_gb300 import api, design_study as ds
    variants = W.config5_reduced_variants(20)
    rounds, q, kmax = 5, 4, 40
    data = [ds.variant_samples(w, rounds, q, kmax) for w in variants]
    train, held = data[:14], data[14:]
    ntrain = sum(len(d.T) for d in train)
    order = W.mlp_order(ntrain, 2000, 256)
    st, losses = ds.train_estimator(train, W.mlp_init(), order, lr=1e-3)
    assert np.mean(losses[-100:]) < 0.5 * np.mean(losses[:20])
    Xh = np.concatenate([d.X for d in held])
    Th = np.concatenate([d.T for d in held])
    pred = api.mlp_predict(st.params, Xh).cpu().numpy()
    a, c = ds.linear_baseline(train)
    r_mlp = ds.rmse(pred, Th)
    r_raw = ds.rmse(Xh[:, 4], Th)
    r_lin = ds.rmse(a * Xh[:, 4] + c, Th)
    print("held-out RMSE of log10(error)/4: network %.4f, residual %.4f, calibrated residual %.4f"
          % (r_mlp, r_raw, r_lin))
    assert r_mlp < r_lin and r_mlp < r_raw


def test_estimator_driven_greedy_runs_and_is_confirmed_by_the_residual():
    need_cuda()
    from paper_2310_04734_gb300 import api, design_study as ds
    variants = W.config5_reduced_variants(10)
    data = [ds.variant_samples(w, 4, 4, 40) for w in variants[:6]]
    order = W.mlp_order(sum(len(d.T) for d in data), 800, 256)
    st, _ = ds.train_estimator(data, W.mlp_init(), order, lr=1e-3)
    for w in variants[6:]:
        e_res, s_res = ds.greedy_error(w, 5, 4, 40)
        e_mlp, s_mlp = ds.greedy_error(w, 5, 4, 40, mlp_params=st.params)
        print("%s: max output error after 5 points: residual-driven %.3e, estimator-driven %.3e"
              % (w.name, e_res, e_mlp))
        assert len(s_mlp) == 5 and len(set(s_mlp.tolist())) == 5
        assert np.isfinite(e_mlp)
