"""Learned gate on the GPU: the library's BF16 tensor-core forward/backward
against the FP64 oracle, a short training run, and checkpoint/resume.

Tolerances: the GPU rounds weights, features and layer-1 activations to
BF16 (8-bit mantissa) and accumulates in FP32, so its gradient is compared
with the exact FP64 gradient by direction (cosine >= 0.995) and size
(relative L2 error <= 6 %); its probabilities with the oracle run with the
same BF16 roundings, within 2e-3.
"""
import numpy as np
import pytest
import torch

from oracle import gate as ogate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_15121_gb300 import gate
    return gate


def batch(rng, B):
    base = rng.integers(2000, 30000, (B, 1, 1))
    D = (base * (1 + 0.01 * rng.normal(size=(B, 6, 6)))).astype(np.int32)
    jump = rng.random(B) < 0.5
    D[jump, :, 3:] = (D[jump, :, 3:] * rng.uniform(1.05, 2.0, (jump.sum(), 1, 1))).astype(np.int32)
    D[rng.random((B, 6, 6)) < 0.05] = 0
    y = (~jump).astype(np.float32)
    return D.reshape(B, 36), y


def test_gradient_against_fp64_oracle(G):
    rng = np.random.default_rng(0)
    X, y = batch(rng, 512)
    theta = G.init_params(3) + (0.05 * rng.normal(size=G.N_PARAMS)).astype(np.float32)
    tr = G.Trainer(512, theta)
    loss, grad, q = tr.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    tr.check_device()  # no bounded tensor-core wait gave up
    tr.close()
    g = grad.cpu().numpy().astype(np.float64)
    ref_loss, ref = ogate.loss_and_grad(X.reshape(-1, 6, 6), y.astype(np.float64), theta.astype(np.float64))
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert cos >= 0.995 and rel <= 0.06, (cos, rel)
    assert abs(float(loss) - ref_loss) <= 0.02 * ref_loss
    q_ref = ogate.forward_patches(X.reshape(-1, 6, 6), theta.astype(np.float64), round_bf16=True)
    assert np.abs(q.cpu().numpy() - q_ref).max() <= 2e-3


def test_training_reduces_loss_and_checkpoint_resumes(G, tmp_path):
    X, y = G.make_training_set(n_scenes=48, per_class=128, seed=5, workers=4)
    assert len(y) > 5000 and 0.2 < y.mean() < 0.8
    theta0 = G.init_params(0)
    theta, hist = G.train(X, y, epochs=6, batch=512, lr=3e-3, seed=0, log=lambda *_: None,
                          checkpoint=str(tmp_path / "ck.npz"))
    assert hist[-1] < 0.8 * hist[0]
    ck = np.load(tmp_path / "ck.npz")
    assert np.array_equal(ck["theta"], theta) and int(ck["version"]) == G.VERSION
    # resuming from the checkpoint continues exactly where the run stopped
    Xd, yd = torch.from_numpy(X[:1024]).cuda(), torch.from_numpy(y[:1024]).cuda()
    a = G.Trainer(1024, theta0)
    a.resume(ck["theta"], ck["m"], ck["v"], int(ck["step"]))
    b = G.Trainer(1024, theta0)
    b.resume(ck["theta"], ck["m"], ck["v"], int(ck["step"]))
    la = float(a.step(Xd, yd, 1e-3))
    lb = float(b.step(Xd, yd, 1e-3))
    # the loss and gradients are summed with atomics (order varies): equal
    # to FP32 rounding
    assert abs(la - lb) <= 1e-5 * abs(la)
    assert np.allclose(a.state()[0], b.state()[0], rtol=0, atol=1e-6)
    a.close()
    b.close()
    path = tmp_path / "w.bin"
    G.save_weights(str(path), theta, {"note": "test"})
    assert np.array_equal(G.load_weights(str(path)), theta)
