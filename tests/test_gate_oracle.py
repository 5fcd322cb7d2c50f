"""Pins of the learned-gate oracle (oracle/gate.py): analytic gradient vs
central finite differences, patch and image forms agree, the convolution vs
scipy, BF16 rounding vs torch's bfloat16 conversion, hand-computed features
and labels."""
import numpy as np
import pytest

from oracle import gate


def random_patches(rng, B):
    base = rng.integers(3000, 9000, (B, 1, 1))
    D = (base * (1 + 0.02 * rng.normal(size=(B, 6, 6)))).astype(np.int64)
    jump = rng.random(B) < 0.5
    D[jump, :, 3:] = (D[jump, :, 3:] * 1.5).astype(np.int64)
    D[rng.random((B, 6, 6)) < 0.05] = 0
    y = (rng.random(B) < 0.5).astype(np.float64)
    return D, y


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    D, y = random_patches(rng, 64)
    theta = gate.init_params(1)
    theta = theta + 0.05 * rng.normal(size=theta.shape)   # biases away from 0
    _, g = gate.loss_and_grad(D, y, theta)
    idx = rng.choice(theta.size, 120, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        num = (gate.bce(gate.forward_patches(D, tp), y) - gate.bce(gate.forward_patches(D, tm), y)) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)) + 1e-8, (i, num, g[i])


def test_patch_and_image_forms_agree():
    rng = np.random.default_rng(1)
    H, W = 23, 31
    D = rng.integers(4000, 4400, (H, W))
    D[:, 15:] *= 2
    D[rng.random((H, W)) < 0.1] = 0
    theta = gate.init_params(2) + 0.1 * rng.normal(size=gate.N_PARAMS)
    q_img = gate.forward_image(D, theta, round_bf16=False)
    Dp = np.pad(D, 3)
    for (v, u) in [(0, 0), (5, 7), (11, 15), (22, 30), (3, 29)]:
        patch = Dp[v + 1:v + 7, u + 1:u + 7][None]
        q = gate.forward_patches(patch, theta)[0]
        assert abs(q - q_img[v, u]) < 1e-12


def test_conv_is_scipy_correlation():
    from scipy.signal import correlate
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, 9, 3))
    Wt = rng.normal(size=(4, 9, 3))
    out = gate._conv3x3(x, Wt, np.zeros(4))
    for o in range(4):
        k = Wt[o].reshape(3, 3, 3)
        ref = correlate(x, k, mode="valid")[:, :, 0]
        assert np.allclose(out[..., o], ref, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 65504.0, 3.0e38]]).astype(np.float32)
    ours = gate.bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_features_by_hand():
    D = np.array([[1024, 1024, 2048, 0],
                  [1024, 512, 2048, 2048]])
    f = gate.features(D)
    # f0 = log2 of the ratio to the right neighbour (0 where either is invalid)
    assert f[0, 0, 0] == 0.0 and f[0, 1, 0] == 1.0 and f[0, 2, 0] == 0.0 and f[0, 3, 0] == 0.0
    assert f[1, 0, 0] == -1.0 and f[1, 1, 0] == 2.0 and f[1, 3, 0] == 0.0
    # f1 = log2 of the ratio to the pixel below; the last row has none
    assert f[0, 0, 1] == 0.0 and f[0, 1, 1] == -1.0 and f[0, 3, 1] == 0.0 and (f[1, :, 1] == 0).all()
    assert f[..., 2].tolist() == [[1, 1, 1, 0], [1, 1, 1, 1]]
    assert (f[..., 3:] == 0).all()


def test_patch_labels_by_hand():
    prim = np.zeros((8, 8), int)
    prim[:, 5:] = 1
    valid = np.ones((8, 8), bool)
    valid[:, 4] = False             # an invalid column just left of the boundary
    valid[7, :] = False
    lab = gate.patch_labels(prim, valid)
    want = np.zeros((8, 8), bool)
    # one primitive and >= 13 valid pixels: centres in columns 0..2 need rows
    # covering enough valid pixels; column 2 sees columns 0..4 (4 valid)
    for v in range(8):
        for u in range(8):
            rows = [r for r in range(v - 2, v + 3) if 0 <= r < 8]
            cols = [c for c in range(u - 2, u + 3) if 0 <= c < 8]
            vals = [prim[r, c] for r in rows for c in cols if valid[r, c]]
            want[v, u] = len(vals) >= 13 and len(set(vals)) == 1
    assert np.array_equal(lab, want)
    assert lab[2, 1] and lab[3, 2] and not lab[3, 3] and not lab[3, 5]
