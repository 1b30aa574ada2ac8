"""The learned initialiser end to end on a small sparse-view problem: trained
on library-made pairs, the network improves on its FDK input, and TV started
from its output beats TV from zero at the same budget and reaches the long
plain run's PSNR in fewer steps."""
import numpy as np
import pytest
import torch

from paper_1904_13342_gb300 import learned_init as LI

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_trained_initializer_gains_over_fdk_and_plain_tv():
    setup = LI.SparseViewSetup(n=64, spacing=2.0, views=30, detector=(100, 128), detector_spacing=2.0)
    maker = LI.PairMaker(setup, DEV)
    net, losses = LI.train_initializer(maker, list(range(1000, 1016)), steps=200, batch=2)
    assert np.mean(losses[-20:]) < 0.5 * losses[0]
    L_est = LI.lipschitz(maker)
    res = LI.ab_test(maker, net, list(range(4)), lam=3.0, eps=1e-3, L_est=L_est, short_iter=10, long_iter=60)
    sm = res.summary()
    assert sm["psnr_cnn"] > sm["psnr_fdk"] + 1.0
    assert sm["psnr_learned"] > sm["psnr_short_tv"] + 1.0
    assert sm["iters_to_target"] is not None and sm["iters_to_target"] < 60
    assert sm["psnr_to_target"] >= sm["psnr_plain"] - 1e-6
    # the curves start at the inputs: zero and the network's output
    assert abs(res.curve_learned[0] - sm["psnr_cnn"]) < 1e-9
