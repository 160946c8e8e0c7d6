"""Learned plan selection end to end on the GPU: the autotuner times every
candidate plan of a set of training shapes, the library's MLP kernels fit the
relative log run time, and on held-out shapes the model's choice is compared
with exhaustive timing (regret = t(chosen) / t(best) - 1) and with the method
without it (the fixed default plan)."""
import numpy as np
import pytest

from paper_1904_10119_gb300 import plansel

pytestmark = pytest.mark.gpu


def test_learned_choice_gains_over_the_fixed_default():
    res = plansel.run(train_shapes=30, test_shapes=30, seed=3, max_volume=1 << 21, reps=2, epochs=300)
    print({k: res[k] for k in ("train_plans", "loss_first", "loss_last")})
    print("regret mlp", res["regret_mlp"], "fixed", res["regret_fixed_default"], "analytic", res["regret_analytic"])
    assert res["train_plans"] >= 300
    assert res["loss_last"] < 0.5 * res["loss_first"]
    assert np.isfinite(res["regret_mlp"]["mean"]) and res["regret_mlp"]["mean"] >= 0.0
    assert res["regret_mlp"]["mean"] < res["regret_fixed_default"]["mean"]
