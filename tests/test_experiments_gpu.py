"""The paper's 2D experiments on the library's kernels: the learnable filter
fitted from the frequency-sampled ramp reconstructs better than its start
and than Ram-Lak (filter learning), and
TV beats Ram-Lak FBP on 30 noisy parallel views (sparse-view iterative
reconstruction)."""
import numpy as np
import pytest
import torch

from paper_1904_13342_gb300 import experiments as E

pytestmark = pytest.mark.gpu


def test_learned_filter_beats_its_ramp_start_and_ramlak():
    res = E.learn_filter(n=128, views=180, iters=60)
    k0, k, kr = (t[:8].cpu().numpy() for t in (res.K0, res.K, res.K_ramlak))
    print("\nK0", np.round(k0, 5), "\nK ", np.round(k, 5), "\nKr", np.round(kr, 5))
    print("loss ramp", res.losses[0], "learned", res.losses[-1], "ram-lak", res.loss_ramlak,
          "low-band distance to ram-lak", res.dist_to_ramlak[0], res.dist_to_ramlak[-2])
    assert res.losses[-1] < 0.95 * res.losses[0]
    assert res.losses[-1] <= res.loss_ramlak


def test_sparse_view_tv_beats_fbp():
    res = E.sparse_view_tv(n=128, iters=100, tune_seeds=range(1000, 1002), test_seeds=range(4))
    print("lambda", res.lam, "FBP", np.mean(res.psnr_fbp), "TV", np.mean(res.psnr_tv))
    assert np.mean(res.psnr_tv) > np.mean(res.psnr_fbp) + 3.0
