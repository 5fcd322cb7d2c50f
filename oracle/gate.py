"""FP64 oracle of the learned boundary gate (test infrastructure only).

Only the test suite, the package's smoke check, the benchmark's CPU leg and
the committed training-label script may import this module; the product
never does.

Network (frozen definition; the paper has no learned part -- it notes that
the method is differentiable apart from the adaptive support, Sec. I-C):

  features f(p), 8 channels, from the integer disparity codes D (0 = invalid,
  pixels outside the image invalid), L = log2 D rounded to FP32:
      f0 = L(p + e_u) - L(p)   if p and p + e_u are valid, else 0
      f1 = L(p + e_v) - L(p)   if p and p + e_v are valid, else 0
      (both differences in FP32 arithmetic)
      f2 = 1 if p is valid, else 0
      f3..f7 = 0
  h1 = relu(conv3x3(f) W1 + b1)          16 channels
  z  = relu(conv3x3(h1) W2 + b2)         16 channels
  q  = sigmoid(z . W3 + b3)              P(the 5x5 patch at p is one valid surface)
  conv3x3: out(p) = sum over o in {-1,0,1}^2 of W[(o_v+1)*3 + (o_u+1)] in(p + o).
  gate(p) = (min of q(c) over the lattice points c (both coordinates even)
  with |c - p|_inf <= r - 1 is >= tau) and p is valid, r the radius of the
  full window a certified pixel fits: the 5x5 patches centred at those
  lattice points cover p's (2r + 1)^2 window whatever the parity of p
  (pixels outside the image count, as invalid pixels).
  Label of a patch: at least 13 of its 25 pixels are valid (pixels outside
  the image are invalid) and all its valid pixels show one primitive.

Weight layout: W1[16][9][8], W2[16][9][16], W3[16], b1[16], b2[16], b3.
The GPU runs features, weights and layer-1 activations in BF16 with FP32
accumulation; `bf16` reproduces that rounding (round to nearest even).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 16
SHAPES = {"W1": (N_HID, 9, N_IN), "b1": (N_HID,), "W2": (N_HID, 9, N_HID), "b2": (N_HID,),
          "W3": (N_HID,), "b3": (1,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out = np.where(nan, np.nan, out)
    return out


def unflatten(theta):
    theta = np.asarray(theta, np.float64)
    out, k = {}, 0
    for name in ORDER:
        n = int(np.prod(SHAPES[name]))
        out[name] = theta[k:k + n].reshape(SHAPES[name])
        k += n
    return out


def flatten(w):
    return np.concatenate([np.asarray(w[n], np.float64).ravel() for n in ORDER])


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    w = {"W1": rng.normal(0, np.sqrt(2.0 / 27), SHAPES["W1"]), "b1": np.zeros(N_HID),
         "W2": rng.normal(0, np.sqrt(2.0 / 144), SHAPES["W2"]), "b2": np.zeros(N_HID),
         "W3": rng.normal(0, np.sqrt(1.0 / 16), SHAPES["W3"]), "b3": np.zeros(1)}
    return flatten(w)


# ---------------------------------------------------------------- features
def features(D):
    """f for every pixel of an integer-code image (any shape [..., H, W])."""
    D = np.asarray(D)
    valid = D > 0
    # L = log2 D rounded to FP32, and the steps are FP32 differences of
    # those values (the definition the kernel computes exactly)
    L = np.where(valid, np.log2(np.where(valid, D, 1).astype(np.float64)), 0.0).astype(np.float32)
    f = np.zeros(D.shape + (N_IN,))
    vr = np.zeros_like(valid)
    vr[..., :, :-1] = valid[..., :, :-1] & valid[..., :, 1:]
    vd = np.zeros_like(valid)
    vd[..., :-1, :] = valid[..., :-1, :] & valid[..., 1:, :]
    dr = np.zeros(D.shape)
    dr[..., :, :-1] = (L[..., :, 1:] - L[..., :, :-1]).astype(np.float64)
    dd = np.zeros(D.shape)
    dd[..., :-1, :] = (L[..., 1:, :] - L[..., :-1, :]).astype(np.float64)
    f[..., 0] = np.where(vr, dr, 0.0)
    f[..., 1] = np.where(vd, dd, 0.0)
    f[..., 2] = valid.astype(np.float64)
    return f


def _conv3x3(x, W, b):
    """x [..., H, W, Cin], W [Cout, 9, Cin]: valid 3x3 cross-correlation."""
    H, Wd = x.shape[-3] - 2, x.shape[-2] - 2
    out = np.zeros(x.shape[:-3] + (H, Wd, W.shape[0]))
    for oy in range(3):
        for ox in range(3):
            patch = x[..., oy:oy + H, ox:ox + Wd, :]
            out += patch @ W[:, oy * 3 + ox, :].T
    return out + b


def forward_image(D, theta, round_bf16=True, margin=0):
    """q for every pixel of an image and `margin` pixels around it (outside
    the image: invalid pixels)."""
    w = unflatten(theta)
    if round_bf16:
        w = {k: (bf16(v) if k.startswith("W") else v) for k, v in w.items()}
    H, W = D.shape
    P = max(4, margin + 2)
    Dp = np.zeros((H + 2 * P + 1, W + 2 * P + 1), D.dtype)
    Dp[P:P + H, P:P + W] = D
    f = features(Dp)[:-1, :-1]                  # (H + 2P) x (W + 2P)
    if round_bf16:
        f = bf16(f)
    h1 = np.maximum(_conv3x3(f, w["W1"], w["b1"]), 0.0)   # margin P - 1
    if round_bf16:
        h1 = bf16(h1)
    z = np.maximum(_conv3x3(h1, w["W2"], w["b2"]), 0.0)   # margin P - 2
    logit = z @ w["W3"] + w["b3"][0]
    q = 1.0 / (1.0 + np.exp(-logit))
    m = P - 2 - margin                 # q covers the image + (P - 2) on each side
    return q[m:m + H + 2 * margin, m:m + W + 2 * margin] if m > 0 else q


def _lattice_min(qe, H, W, m):
    """Minimum over the lattice points (even coordinates) within m of every
    pixel; qe covers the image and m pixels around it (origin at -m)."""
    ys, xs = np.mgrid[-m:H + m, -m:W + m]
    qlat = np.where((ys % 2 == 0) & (xs % 2 == 0), qe, np.inf)
    out = np.full((H, W), np.inf)
    for oy in range(2 * m + 1):
        for ox in range(2 * m + 1):
            out = np.minimum(out, qlat[oy:oy + H, ox:ox + W])
    return out


def gate_image(D, theta, tau, radius, round_bf16=True):
    """(gate bits, q, minimum of q over each pixel's lattice points) of an
    image for a full window of the given radius; the minimum includes the q
    of lattice points outside the image (which are invalid pixels)."""
    H, W = D.shape
    m = radius - 1
    qe = forward_image(D, theta, round_bf16, margin=m)
    qmin = _lattice_min(qe, H, W, m)
    return (qmin >= tau) & (D > 0), qe[m:m + H, m:m + W], qmin


# ---------------------------------------------------------------- bounds of a kernel's q
U_ACC = 2.0 ** -23       # unit error of one FP32 addition, rounding to nearest or towards zero
SIGMOID_ABS = 2e-6       # absolute error allowed to the kernel's FP32 sigmoid


def _gamma(n):
    return n * U_ACC / (1.0 - n * U_ACC)


def _conv3x3_pos_neg(lo, hi, W):
    """Range of a valid 3x3 cross-correlation (no bias) over inputs known to
    lie in [lo, hi] elementwise: each weight takes the end of the interval
    that minimises (maximises) its product."""
    Wp, Wn = np.maximum(W, 0.0), np.minimum(W, 0.0)
    return (_conv3x3(lo, Wp, 0.0) + _conv3x3(hi, Wn, 0.0),
            _conv3x3(hi, Wp, 0.0) + _conv3x3(lo, Wn, 0.0))


def q_bounds(D, theta, margin=0):
    """[q_lo, q_hi] for every pixel of an image and `margin` pixels around it:
    the values a kernel may produce that computes the features exactly as
    defined above, rounds weights, features and layer-1 activations to BF16
    (nearest even), accumulates each convolution and the head in FP32 in any
    order (each addition rounding to nearest or towards zero), and evaluates
    the sigmoid within SIGMOID_ABS.  Bound per sum of n terms t_i (the bias
    counted as a term): |fl(sum) - sum| <= gamma_n sum |t_i|,
    gamma_n = n u / (1 - n u), u = 2^-23.  Where a layer-1 activation lies
    within that bound of a BF16 rounding boundary both roundings are allowed;
    the ranges then pass through layer 2, the ReLUs, the head and the sigmoid
    by interval arithmetic (every step is monotone or linear)."""
    w = unflatten(theta)
    w = {k: (bf16(v) if k.startswith("W") else v) for k, v in w.items()}
    H, W = D.shape
    P = max(4, margin + 2)
    Dp = np.zeros((H + 2 * P + 1, W + 2 * P + 1), D.dtype)
    Dp[P:P + H, P:P + W] = D
    f = bf16(features(Dp)[:-1, :-1])
    # layer 1: 72 products (9 taps x 8 channels) and the bias
    a1 = _conv3x3(f, w["W1"], w["b1"])
    mag1 = _conv3x3(np.abs(f), np.abs(w["W1"]), np.abs(w["b1"]))
    e1 = _gamma(9 * N_IN + 1) * mag1
    h1_lo = bf16(np.maximum(a1 - e1, 0.0))
    h1_hi = bf16(np.maximum(a1 + e1, 0.0))
    # layer 2: 144 products and the bias
    a2_lo, a2_hi = _conv3x3_pos_neg(h1_lo, h1_hi, w["W2"])
    mag2 = _conv3x3(np.maximum(np.abs(h1_lo), np.abs(h1_hi)), np.abs(w["W2"]), np.abs(w["b2"]))
    e2 = _gamma(9 * N_HID + 1) * mag2
    a2_lo, a2_hi = a2_lo + w["b2"] - e2, a2_hi + w["b2"] + e2
    z_lo, z_hi = np.maximum(a2_lo, 0.0), np.maximum(a2_hi, 0.0)
    # head: 16 products and the bias, allowing the bias of layer 2 to be
    # folded into it (sums over |W3| (|a2| + |b2|))
    W3p, W3n = np.maximum(w["W3"], 0.0), np.minimum(w["W3"], 0.0)
    l_lo = z_lo @ W3p + z_hi @ W3n + w["b3"][0]
    l_hi = z_hi @ W3p + z_lo @ W3n + w["b3"][0]
    mag3 = (np.maximum(np.abs(a2_lo), np.abs(a2_hi)) + np.abs(w["b2"])) @ np.abs(w["W3"]) + abs(w["b3"][0])
    e3 = _gamma(2 * N_HID + 2) * mag3
    q_lo = 1.0 / (1.0 + np.exp(-(l_lo - e3))) - SIGMOID_ABS
    q_hi = 1.0 / (1.0 + np.exp(-(l_hi + e3))) + SIGMOID_ABS
    m = P - 2 - margin
    if m > 0:
        q_lo = q_lo[m:m + H + 2 * margin, m:m + W + 2 * margin]
        q_hi = q_hi[m:m + H + 2 * margin, m:m + W + 2 * margin]
    return q_lo, q_hi


def gate_bounds(D, theta, tau, radius):
    """(surely certified, surely not certified, q_lo, q_hi) of every pixel:
    the minimum of q over the pixel's lattice points (pixels outside the
    image included) is >= tau for every q in the bounds, or < tau for every q
    in them.  Pixels in neither set are undecided by the bounds."""
    H, W = D.shape
    m = radius - 1
    lo, hi = q_bounds(D, theta, margin=m)
    mlo = _lattice_min(lo, H, W, m)
    mhi = _lattice_min(hi, H, W, m)
    valid = D > 0
    return (mlo >= tau) & valid, (mhi < tau) | ~valid, lo[m:m + H, m:m + W], hi[m:m + H, m:m + W]


# ---------------------------------------------------------------- patches (training)
def forward_patches(Dp, theta, round_bf16=False, keep=False):
    """Dp [B, 6, 6] integer codes around each centre (centre at [2, 2]);
    returns q [B] (and the intermediates when keep=True)."""
    w = unflatten(theta)
    if round_bf16:
        w = {k: (bf16(v) if k.startswith("W") else v) for k, v in w.items()}
    f = features(Dp)[:, :5, :5, :]
    if round_bf16:
        f = bf16(f)
    a1 = _conv3x3(f, w["W1"], w["b1"])          # [B, 3, 3, 16]
    h1 = np.maximum(a1, 0.0)
    if round_bf16:
        h1 = bf16(h1)
    a2 = _conv3x3(h1, w["W2"], w["b2"])[:, 0, 0, :]   # [B, 16]
    z = np.maximum(a2, 0.0)
    logit = z @ w["W3"] + w["b3"][0]
    q = 1.0 / (1.0 + np.exp(-logit))
    if keep:
        return q, dict(f=f, a1=a1, h1=h1, a2=a2, z=z, logit=logit, w=w)
    return q


def bce(q, y):
    q = np.clip(q, 1e-12, 1 - 1e-12)
    return float(np.mean(-(y * np.log(q) + (1 - y) * np.log(1 - q))))


def loss_and_grad(Dp, y, theta):
    """Mean binary cross-entropy of the batch and its gradient (FP64,
    written out layer by layer)."""
    q, c = forward_patches(Dp, theta, keep=True)
    w = c["w"]
    B = len(y)
    dlogit = (q - y) / B                                  # d loss / d logit
    g = {"W3": c["z"].T @ dlogit, "b3": np.array([dlogit.sum()])}
    dz = np.outer(dlogit, w["W3"]) * (c["a2"] > 0)        # [B, 16]
    g["b2"] = dz.sum(0)
    gW2 = np.zeros(SHAPES["W2"])
    dh1 = np.zeros(c["h1"].shape)                         # [B, 3, 3, 16]
    for oy in range(3):
        for ox in range(3):
            hpos = c["h1"][:, oy, ox, :]                  # [B, 16]
            gW2[:, oy * 3 + ox, :] = dz.T @ hpos
            dh1[:, oy, ox, :] = dz @ w["W2"][:, oy * 3 + ox, :]
    g["W2"] = gW2
    da1 = dh1 * (c["a1"] > 0)
    g["b1"] = da1.sum((0, 1, 2))
    gW1 = np.zeros(SHAPES["W1"])
    f = c["f"]
    for oy in range(3):
        for ox in range(3):
            fp = f[:, oy:oy + 3, ox:ox + 3, :]            # [B, 3, 3, 8]
            gW1[:, oy * 3 + ox, :] = np.einsum("bijo,bijc->oc", da1, fp)
    g["W1"] = gW1
    return bce(q, y), flatten(g)


def patch_labels(d_true, valid):
    """Training label of every pixel: 1 where the 5x5 patch centred at it has
    at least 13 valid pixels (outside the image: invalid) and no depth
    discontinuity -- every two 4-adjacent valid pixels of the patch differ in
    noise-free disparity d_true by at most max(0.03 min(d1, d2), 0.25 px)."""
    H, W = d_true.shape
    lab = np.zeros((H, W), bool)

    def ok(a, b):
        return abs(a - b) <= max(0.03 * min(a, b), 0.25)
    for v in range(H):
        for u in range(W):
            cells = [(r, c) for r in range(v - 2, v + 3) for c in range(u - 2, u + 3)
                     if 0 <= r < H and 0 <= c < W and valid[r, c]]
            if len(cells) < 13:
                continue
            s = set(cells)
            lab[v, u] = all(ok(d_true[r, c], d_true[r2, c2])
                            for (r, c) in cells for (r2, c2) in ((r, c + 1), (r + 1, c))
                            if (r2, c2) in s)
    return lab
