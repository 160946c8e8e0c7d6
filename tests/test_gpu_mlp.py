"""The plan-cost perceptron's forward, backward and Adam kernels against the
FP64 oracle (which is itself pinned by finite differences), and a training
run that must fit a smooth target."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3

pytestmark = pytest.mark.gpu


def _split(p, F, H):
    o = 0
    out = []
    for shape in [(H, F), (H,), (H, H), (H,), (1, H), (1,)]:
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape).astype(np.float64))
        o += k
    return out


@pytest.mark.parametrize("F,H,B", [(16, 64, 300), (7, 9, 11), (3, 64, 1)])
def test_forward_and_gradients_match_fp64_oracle(F, H, B):
    m = fft3.Mlp(F, H, seed=F + H)
    p = m.get_params()
    rng = np.random.default_rng(B)
    p[:] = rng.normal(0, 0.3, p.size).astype(np.float32)
    m.set_params(p)
    X = rng.normal(size=(B, F)).astype(np.float32)
    y = rng.normal(size=B).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    pred = torch.empty(B, device="cuda")
    grad = torch.empty(p.size, device="cuda")
    loss = torch.empty(1, device="cuda")
    L = fft3.load()
    assert L.fft3_mlp_forward(m.handle, Xd.data_ptr(), B, pred.data_ptr(), None) == 0
    assert L.fft3_mlp_grad(m.handle, Xd.data_ptr(), yd.data_ptr(), B, grad.data_ptr(), loss.data_ptr(), None) == 0
    torch.cuda.synchronize()
    params = _split(p, F, H)
    ref_pred, cache = oracle.mlp_forward(params, X)
    ref_loss = oracle.mse_loss(ref_pred, y)
    ref_grads = oracle.mlp_backward(params, cache, ref_pred, y)
    assert np.max(np.abs(pred.cpu().numpy() - ref_pred)) <= 1e-4 * max(1.0, np.max(np.abs(ref_pred)))
    assert abs(loss.item() - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    g = grad.cpu().numpy().astype(np.float64)
    flat_ref = np.concatenate([r.ravel() for r in ref_grads])
    assert np.linalg.norm(g - flat_ref) <= 1e-4 * max(1e-6, np.linalg.norm(flat_ref))
    m.close()


def test_adam_step_matches_oracle():
    F, H = 5, 8
    m = fft3.Mlp(F, H, seed=1)
    p = m.get_params().astype(np.float64)
    rng = np.random.default_rng(2)
    g = rng.normal(size=p.size).astype(np.float32)
    gd = torch.from_numpy(g).cuda()
    L = fft3.load()
    mom = [np.zeros(p.size)]
    vel = [np.zeros(p.size)]
    ref = [p]
    for t in (1, 2, 3):
        assert L.fft3_mlp_adam_step(m.handle, gd.data_ptr(), 1e-2, None) == 0
        ref, mom, vel = oracle.adam_step(ref, [g.astype(np.float64)], mom, vel, t, lr=1e-2)
    torch.cuda.synchronize()
    got = m.get_params().astype(np.float64)
    assert np.max(np.abs(got - ref[0])) <= 1e-5
    m.close()


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(1500, 6)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 3] ** 2).astype(np.float32)
    m = fft3.Mlp(6, 64, seed=3)
    curve = m.train(X, y, epochs=150, batch=128, lr=3e-3, seed=4)
    assert curve[-1] < 0.1 * curve[0]
    pred = m.predict(X)
    assert np.mean((pred - y) ** 2) == pytest.approx(float(curve[-1]), rel=1e-3, abs=1e-6)
    m.close()
