"""Integer and control-flow identities the CUDA kernels rely on, checked
exhaustively or on random inputs on the CPU (no GPU, no oracle):

* the pair test of the component passes from per-pixel thresholds:
  2^16 |a - b| <= K min(a, b)  <=>  |a - b| <= min(floor(K a / 2^16),
  floor(K b / 2^16)) for positive integer codes (Sec. III-D relative depth
  test, exact form);
* the star walk's frozen extremes: stopping the running min/max at the first
  step that is not taken leaves the spread of that step, so the result
  (steps taken, data sum, spread that decides the exact tail) equals that of
  the walk that keeps the spread of the first failing step separately.
"""
import numpy as np


def test_pair_threshold_identity():
    rng = np.random.default_rng(7)
    for K in (0, 1, 655, 3277, 6554, 65536, 131072, 1 << 20):
        a = rng.integers(1, 131072, 200_000, dtype=np.int64)
        b = np.clip(a + rng.integers(-4000, 4000, a.size), 1, 131071)
        b[::7] = rng.integers(1, 131072, b[::7].size)
        direct = (np.abs(a - b) << 16) <= K * np.minimum(a, b)
        thr = np.abs(a - b) <= np.minimum((K * a) >> 16, (K * b) >> 16)
        assert np.array_equal(direct, thr), K
    # every code pair near one threshold, exhaustively
    K = 6554
    a = np.arange(1, 4096, dtype=np.int64)[:, None]
    b = np.arange(1, 4096, dtype=np.int64)[None, :]
    direct = (np.abs(a - b) << 16) <= K * np.minimum(a, b)
    thr = np.abs(a - b) <= np.minimum((K * a) >> 16, (K * b) >> 16)
    assert np.array_equal(direct, thr)


def walk_separate(w, D, wc, lo):
    """Running extremes always updated; the spread of the first failing step
    kept in its own variable."""
    wlo = whi = wc
    fdiff = 0.0
    alive = True
    A = n = 0
    for t, (wt, dt) in enumerate(zip(w, D), 1):
        wlo, whi = min(wlo, wt), max(whi, wt)
        diff = whi - wlo
        if alive:
            fdiff = diff
        alive = alive and diff < lo
        if alive:
            A += t * dt
            n += 1
    return n, A, fdiff


def walk_frozen(w, D, wc, lo):
    """Running extremes frozen after the first step that is not taken."""
    wlo = whi = wc
    alive = True
    A = n = 0
    for t, (wt, dt) in enumerate(zip(w, D), 1):
        if alive:
            wlo, whi = min(wlo, wt), max(whi, wt)
        alive = whi - wlo < lo
        if alive:
            A += t * dt
            n += 1
    return n, A, whi - wlo


def test_frozen_extremes_walk():
    rng = np.random.default_rng(3)
    for _ in range(20_000):
        L = int(rng.integers(1, 11))
        D = rng.integers(1, 131072, L)
        D[rng.random(L) < 0.1] = 0
        w = np.where(D > 0, 1.0 / np.maximum(D, 1), np.inf).astype(np.float32).tolist()
        Dc = int(rng.integers(1, 131072))
        wc = float(np.float32(1.0 / Dc))
        lo = float(np.float32(rng.choice([0.0, 1e-6, 1e-5, 1e-4, 1.0]) / Dc))
        n1, A1, f1 = walk_separate(w, D.tolist(), wc, lo)
        n2, A2, f2 = walk_frozen(w, D.tolist(), wc, lo)
        assert (n1, A1) == (n2, A2)
        if n1 < L:  # the exact tail only ever looks at the failing step's spread
            assert f1 == f2


def test_denoise_5x5_cofactors_fit_32_bits():
    # every subset of the 5x5 window (the centre always passes its own range
    # gate): the 3x3 cofactors and the determinant of the denoise solve stay
    # far inside 32 bits and below 2^24 (exact in FP32), as the kernels assume
    ou = np.array([u for v in range(-2, 3) for u in range(-2, 3) if (u, v) != (0, 0)], np.int64)
    ov = np.array([v for v in range(-2, 3) for u in range(-2, 3) if (u, v) != (0, 0)], np.int64)
    worst = np.zeros(4, np.int64)
    for lo in range(0, 1 << 24, 1 << 20):
        m = np.arange(lo, lo + (1 << 20), dtype=np.int64)
        bits = ((m[:, None] >> np.arange(24)) & 1).astype(np.int64)
        n = bits.sum(1) + 1
        Su, Sv = bits @ ou, bits @ ov
        Suu, Svv, Suv = bits @ (ou * ou), bits @ (ov * ov), bits @ (ou * ov)
        M00 = Suu * Svv - Suv * Suv
        M10 = Su * Svv - Sv * Suv
        M20 = Su * Suv - Sv * Suu
        det = n * M00 - Su * M10 + Sv * M20
        worst = np.maximum(worst, [np.abs(a).max() for a in (M00, M10, M20, det)])
    assert worst[:3].max() <= 2580 and worst[3] <= 217_300 < 1 << 24, worst


def test_star8_moments_fit_32_bits():
    # the compile-time M = 8, s = 10 star: distinct offsets of each ray
    # (rounding half away from zero); the largest support bounds every sum
    import math
    pts = set()
    for j in range(8):
        th = 2 * math.pi * j / 8
        for k in range(1, 11):
            u, v = math.cos(th) * k, math.sin(th) * k
            pts.add((int(math.copysign(math.floor(abs(u) + 0.5), u)), int(math.copysign(math.floor(abs(v) + 0.5), v))))
    pts.discard((0, 0))
    Su = sum(abs(u) for u, v in pts)
    Suu = sum(u * u for u, v in pts)
    Suv = sum(abs(u * v) for u, v in pts)
    assert len(pts) == 68 and Su == 222 and Suu == 1330 and Suv == 560
    assert 1024 * Suu * Suu < 1 << 31  # 1024 det <= 1024 Suu Svv
