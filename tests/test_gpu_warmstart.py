"""The trained warm-start network against the method without it.

On held-out 128 x 128 systems (seed 6, the first 8) the unaided FP64
minimiser converges within 5000 iterations for some systems only; for every
one of those the warm-started relaxation (network, FP32, FP64) must end in
the same minimum (energy to 1e-8 relative) in fewer iterations, and every
warm-started relaxation must reach max torque < 1e-6 meV.  Against the
trivial guess -- the +z ferromagnet with 0.05 rad noise, relaxed the same
way -- the network must need fewer iterations too: its gain over that guess
is small (the relaxed textures of random starts are not predictable, and
the network learnt a near-uniform state), but it is there.
"""
import os

import pytest

pytestmark = pytest.mark.gpu

W = pytest.importorskip("paper_1901_11350_gb300.warmstart")
UN = pytest.importorskip("paper_1901_11350_gb300.unet")
PARAMS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1901_11350_gb300",
                      "weights", "warmstart_hex128.npz")


def test_warm_start_gains_over_the_unaided_minimiser():
    net = UN.UNet(128, 8, W.load_params(PARAMS))
    rep = W.evaluate(net, seed=6, n=8, L=128, max_iter=5000, polish_max_iter=2000, chunk=8, per_system=1,
                     log=lambda m: None)
    una, warm = rep["unaided"], rep["warm"]
    assert warm["converged"] == 8
    assert una["converged"] >= 1
    assert warm["matched"] == una["converged"]
    assert warm["matched_iterations"] < warm["unaided_matched_iterations"]
    uni = rep["uniform"]
    assert uni["converged"] == 8
    print("warm start: mean iterations network %.1f, trivial +z %.1f, unaided %.1f"
          % (warm["mean_iterations"], uni["mean_iterations"], una["mean_iterations"]))
    assert warm["mean_iterations"] < uni["mean_iterations"]
