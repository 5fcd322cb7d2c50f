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
    # a ramp (smooth) with a depth jump between columns 5 and 6, a hole
    d = np.tile(10.0 + 0.2 * np.arange(10), (9, 1))
    d[:, 6:] += 5.0                         # jump of 5 px >> max(3 %, 0.25)
    valid = np.ones((9, 10), bool)
    valid[4, 1:4] = False
    lab = gate.patch_labels(d, valid)
    assert lab[4, 3] and lab[2, 2]          # smooth, enough valid pixels
    assert not lab[4, 4] and not lab[4, 7]  # the patch straddles the jump
    assert lab[4, 8] and not lab[0, 0]      # right of the jump; corner patch has 9 pixels
    # only 4-adjacent valid pairs count: with column 6 invalid the jump
    # between columns 5 and 7 is not a pair of neighbours
    valid2 = valid.copy()
    valid2[:, 6] = False
    lab2 = gate.patch_labels(d, valid2)
    assert lab2[4, 4] and lab2[4, 5]


@pytest.mark.parametrize("radius", [3, 6])
def test_gate_image_is_min_of_patch_q(radius):
    # the image form's gate equals, pixel by pixel, the minimum of the patch
    # form's q over the lattice points (even coordinates) within radius - 1 of
    # the pixel in the zero-padded image
    rng = np.random.default_rng(4)
    H, W = 11, 13
    D = rng.integers(4000, 4300, (H, W))
    D[:, 7:] *= 2
    D[rng.random((H, W)) < 0.1] = 0
    theta = gate.init_params(5) + 0.1 * rng.normal(size=gate.N_PARAMS)
    _, _, qmin0 = gate.gate_image(D, theta, 0.5, radius, round_bf16=False)
    qs = np.unique(qmin0[D > 0])
    k = len(qs) // 2
    tau = float(0.5 * (qs[k - 1] + qs[k]))     # splits the image, far from every qmin
    g, q, qmin = gate.gate_image(D, theta, tau, radius, round_bf16=False)
    m, P = radius - 1, radius + 2
    Dp = np.pad(D, P)
    for v in range(H):
        for u in range(W):
            patches = np.stack([Dp[v + oy + P - 2:v + oy + P + 4, u + ox + P - 2:u + ox + P + 4]
                                for oy in range(-m, m + 1) for ox in range(-m, m + 1)
                                if (v + oy) % 2 == 0 and (u + ox) % 2 == 0])
            qm = gate.forward_patches(patches, theta).min()
            assert abs(qm - qmin[v, u]) < 1e-12
            assert g[v, u] == ((qm >= tau) and D[v, u] > 0)
    assert 0 < g.sum() < (D > 0).sum()


def test_lattice_patches_cover_the_window():
    # the 5x5 patches centred at the lattice points (even coordinates) within
    # r - 1 of a pixel cover its (2r + 1)^2 window for either parity
    for r in (3, 6):
        for px in (0, 1):
            covered = set()
            for c in range(px - (r - 1), px + r):
                if c % 2 == 0:
                    covered.update(range(c - 2, c + 3))
            assert set(range(px - r, px + r + 1)) <= covered, (r, px)


def _fp32_network(D, theta, rng, margin):
    """The network as a kernel computes it: exact FP32 features, BF16 weights,
    features and layer-1 activations, every sum accumulated in FP32 in a
    random order (each addition rounded to nearest), sigmoid in FP32."""
    w = gate.unflatten(theta)
    w = {k: (gate.bf16(v) if k.startswith("W") else v) for k, v in w.items()}
    H, W = D.shape
    P = max(4, margin + 2)
    Dp = np.zeros((H + 2 * P + 1, W + 2 * P + 1), D.dtype)
    Dp[P:P + H, P:P + W] = D
    f = gate.bf16(gate.features(Dp)[:-1, :-1]).astype(np.float32)

    def conv(x, Wt, b):
        Ho, Wo = x.shape[0] - 2, x.shape[1] - 2
        terms = []
        for oy in range(3):
            for ox in range(3):
                for c in range(x.shape[2]):
                    terms.append(x[oy:oy + Ho, ox:ox + Wo, c, None] * Wt[None, None, :, oy * 3 + ox, c].astype(np.float32))
        terms.append(np.broadcast_to(np.asarray(b, np.float32), (Ho, Wo, Wt.shape[0])))
        order = rng.permutation(len(terms))
        acc = np.zeros((Ho, Wo, Wt.shape[0]), np.float32)
        for k in order:
            acc = (acc + terms[k]).astype(np.float32)
        return acc
    h1 = gate.bf16(np.maximum(conv(f, w["W1"], w["b1"]), 0)).astype(np.float32)
    z = np.maximum(conv(h1, w["W2"], w["b2"]), 0)
    logit = np.float32(w["b3"][0])
    for c in rng.permutation(16):
        logit = (logit + z[..., c] * np.float32(w["W3"][c])).astype(np.float32)
    q = (1.0 / (1.0 + np.exp(-logit.astype(np.float64)))).astype(np.float32)
    m = P - 2 - margin
    return q[m:m + H + 2 * margin, m:m + W + 2 * margin].astype(np.float64)


def test_q_bounds_contain_fp32_evaluations():
    # the bounds of q (oracle.gate.q_bounds) contain the FP64 network and
    # FP32 evaluations in random accumulation orders, and they are tight:
    # most widths are at the FP32 noise level, a few are wider where a
    # layer-1 activation sits at a BF16 rounding boundary
    from paper_2504_15121_gb300 import gate as G
    theta = G.load_weights().astype(np.float64)
    rng = np.random.default_rng(11)
    H, W = 28, 36
    base = rng.integers(6000, 9000, (H, W))
    blocks = rng.integers(0, 2, (H // 7 + 1, W // 7 + 1)).repeat(7, 0).repeat(7, 1)[:H, :W]
    D = (base * (1 + 0.4 * blocks) + rng.integers(-40, 40, (H, W))).astype(np.int32)
    D[rng.random((H, W)) < 0.06] = 0
    lo, hi = gate.q_bounds(D, theta, margin=2)
    q64 = gate.forward_image(D, theta, margin=2)
    assert ((lo <= q64) & (q64 <= hi)).all()
    for _ in range(3):
        q32 = _fp32_network(D, theta, rng, margin=2)
        assert ((lo <= q32) & (q32 <= hi)).all(), np.abs(np.clip(q32, lo, hi) - q32).max()
    width = hi - lo
    assert np.median(width) < 1e-4 and (width < 1e-3).mean() > 0.9, (np.median(width), (width < 1e-3).mean())
