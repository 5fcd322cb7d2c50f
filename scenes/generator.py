"""Seeded scene generator for rectified stereo disparity maps.

Geometry (paper §II, "Rectified stereo images"): two pinhole cameras with
the same intrinsics (fx, fy, cx, cy), the right one shifted by the baseline B
along +x.  A world point X = (x, y, z) projects to the left image at
u = fx x / z + cx, v = fy y / z + cy, and the disparity used throughout this
code base is the positive quantity d = u_left - u_right = fx B / z.

Every pixel ray of the left camera is intersected with analytic primitives
(planes, spheres, vertical cylinders, axis-aligned boxes).  The nearest hit
inside [z_near, z_far] wins (z-buffer at pixel centres); no hit means
background, which is encoded as disparity 0 (invalid) and excluded from
every error statistic.  Ground-truth normals come from the primitive that was
hit, turned to face the camera.

Order of corruption, for every scene: Gaussian noise on d, then quantisation
or encoding, then invalidation (occlusion bands and/or iid pixels) which
writes 0.

Nothing here estimates normals from disparities.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    baseline: float


@dataclass
class Scene:
    name: str
    camera: Camera
    disp: np.ndarray            # float32 [H, W]; 0 = invalid / background
    gt_normal: np.ndarray       # float32 [H, W, 3]; camera-facing unit normals, 0 on background
    prim: np.ndarray            # int32 [H, W]; primitive id, -1 on background
    background: np.ndarray      # bool [H, W]; no primitive hit
    disp_u16: np.ndarray | None = None   # uint16 rint(d * 256), 0 = invalid
    disp_f16: np.ndarray | None = None   # float16 d, 0 = invalid
    disp_true: np.ndarray | None = None  # float32 noise-free disparity, 0 on background
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return self.disp.shape[0]

    @property
    def W(self) -> int:
        return self.disp.shape[1]


# ---------------------------------------------------------------------------
# workload recipes (sizes, cameras and corruption of the benchmark scenes)
# ---------------------------------------------------------------------------
CONFIGS = {
    # 6 random planes, 320x240, f = 300, B = 0.1, sigma 0.25 px, 5 % iid invalid
    "planes_320x240": dict(kind="planes", W=320, H=240, f=300.0, B=0.1,
                           n_planes=6, sigma=0.25, invalid=0.05, cfg=1),
    # same recipe at 640x480 (f = 600) for the mixed-resolution batches
    "planes_640x480": dict(kind="planes", W=640, H=480, f=600.0, B=0.1,
                           n_planes=6, sigma=0.25, invalid=0.05, cfg=6),
    # 12 planes + 4 spheres + 2 cylinders, 1482x994, f = 1500, B = 0.18,
    # d in [30, 280] px, sigma 0.5 px, quantised to 1/16 px, 3 % invalid in
    # occlusion bands beside depth edges
    "mixed_1482x994": dict(kind="mixed", W=1482, H=994, f=1500.0, B=0.18,
                           sigma=0.5, quant=16, invalid=0.03, cfg=2),
    # driving-like: ground 1.5 m below the camera, facades at x = +-8 m,
    # 20 boxes on the ground; 2048x1024, f = 2260, B = 0.21, sigma 0.3 px,
    # uint16 (d * 256) and fp16 encodings, 8 % invalid
    "driving_2048x1024": dict(kind="driving", W=2048, H=1024, f=2260.0, B=0.21,
                              sigma=0.3, invalid=0.08, cfg=3),
    # the paper's sphere experiment (Fig. "figures"): radius 1.4 at 3 units,
    # baseline 0.3, 1024x1024; the focal length is not stated, f = 1024 here
    "sphere_1024": dict(kind="sphere", W=1024, H=1024, f=1024.0, B=0.3,
                        sigma=0.2, invalid=0.0, cfg=7),
}


def _rays(cam: Camera, W: int, H: int):
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    rx = ((u - cam.cx) / cam.fx)[None, :].repeat(H, 0)
    ry = ((v - cam.cy) / cam.fy)[:, None].repeat(W, 1)
    rz = np.ones((H, W))
    return rx, ry, rz


class _ZBuffer:
    def __init__(self, H, W, z_near, z_far):
        self.t = np.full((H, W), np.inf)
        self.n = np.zeros((H, W, 3))
        self.prim = np.full((H, W), -1, dtype=np.int32)
        self.z_near, self.z_far = z_near, z_far
        self.count = 0

    def offer(self, t, normal_fn, hit):
        """t: candidate hit depth (z, since the ray has unit z); hit: bool mask."""
        if not hit.any():
            self.count += 1
            return self.count - 1
        ok = hit & np.isfinite(t) & (t >= self.z_near) & (t <= self.z_far) & (t < self.t)
        pid = self.count
        self.count += 1
        if not ok.any():
            return pid
        nrm = normal_fn(ok)
        self.t[ok] = t[ok]
        self.n[ok] = nrm
        self.prim[ok] = pid
        return pid


def _face_camera(n, rx, ry, rz, ok):
    # camera-facing: n . ray < 0 at the hit (the camera sits at the origin)
    dot = n[..., 0] * rx[ok] + n[..., 1] * ry[ok] + n[..., 2] * rz[ok]
    s = np.where(dot > 0, -1.0, 1.0)
    return n * s[:, None]


def _add_plane(zb, rays, n, rho):
    rx, ry, rz = rays
    den = n[0] * rx + n[1] * ry + n[2] * rz
    with np.errstate(divide="ignore", invalid="ignore"):
        t = rho / den
    hit = (np.abs(den) > 1e-12) & (t > 0)

    def nf(ok):
        nn = np.broadcast_to(np.asarray(n, float), (int(ok.sum()), 3)).copy()
        return _face_camera(nn, rx, ry, rz, ok)
    return zb.offer(t, nf, hit)


def _add_sphere(zb, rays, c, r):
    rx, ry, rz = rays
    a = rx * rx + ry * ry + rz * rz
    b = -2.0 * (rx * c[0] + ry * c[1] + rz * c[2])
    cc = c[0] ** 2 + c[1] ** 2 + c[2] ** 2 - r * r
    disc = b * b - 4 * a * cc
    hit = disc >= 0
    sq = np.sqrt(np.where(hit, disc, 0.0))
    t = (-b - sq) / (2 * a)
    hit &= t > 0

    def nf(ok):
        X = np.stack([rx[ok] * t[ok], ry[ok] * t[ok], rz[ok] * t[ok]], -1)
        nn = (X - np.asarray(c)) / r
        return _face_camera(nn, rx, ry, rz, ok)
    return zb.offer(t, nf, hit)


def _add_vcylinder(zb, rays, c, r, y0, y1):
    """Open cylinder with its axis along camera y, centre (c[0], ., c[2])."""
    rx, ry, rz = rays
    a = rx * rx + rz * rz
    b = -2.0 * (rx * c[0] + rz * c[2])
    cc = c[0] ** 2 + c[2] ** 2 - r * r
    disc = b * b - 4 * a * cc
    hit = (disc >= 0) & (a > 1e-12)
    sq = np.sqrt(np.where(hit, disc, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (-b - sq) / (2 * a)
    y = ry * t
    hit &= (t > 0) & (y >= y0) & (y <= y1)

    def nf(ok):
        X = np.stack([rx[ok] * t[ok], np.zeros(int(ok.sum())), rz[ok] * t[ok]], -1)
        nn = X - np.array([c[0], 0.0, c[2]])
        nn /= np.linalg.norm(nn, axis=-1, keepdims=True)
        return _face_camera(nn, rx, ry, rz, ok)
    return zb.offer(t, nf, hit)


def _add_box(zb, rays, lo, hi, cam=None):
    """Axis-aligned box [lo, hi] (slab method), evaluated only inside the
    image rectangle that bounds the projection of its corners."""
    rx, ry, rz = rays
    H, W = rx.shape
    v0, v1, u0, u1 = 0, H, 0, W
    if cam is not None and lo[2] > 1e-3:
        cs = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                       for z in (lo[2], hi[2])])
        pu = cam.fx * cs[:, 0] / cs[:, 2] + cam.cx
        pv = cam.fy * cs[:, 1] / cs[:, 2] + cam.cy
        u0 = max(int(np.floor(pu.min())) - 1, 0)
        u1 = min(int(np.ceil(pu.max())) + 2, W)
        v0 = max(int(np.floor(pv.min())) - 1, 0)
        v1 = min(int(np.ceil(pv.max())) + 2, H)
        if u0 >= u1 or v0 >= v1:
            return zb.offer(np.full((H, W), np.inf), None, np.zeros((H, W), bool))
    sl = (slice(v0, v1), slice(u0, u1))
    tn_max = np.full((v1 - v0, u1 - u0), -np.inf)
    tf_min = np.full((v1 - v0, u1 - u0), np.inf)
    axis = np.zeros((v1 - v0, u1 - u0), dtype=np.int64)
    for k, rk in enumerate((rx[sl], ry[sl], rz[sl])):
        rk = np.where(np.abs(rk) < 1e-12, 1e-12, rk)
        t1 = lo[k] / rk
        t2 = hi[k] / rk
        tn = np.minimum(t1, t2)
        tf = np.maximum(t1, t2)
        upd = tn > tn_max
        axis = np.where(upd, k, axis)
        tn_max = np.maximum(tn_max, tn)
        tf_min = np.minimum(tf_min, tf)
    t = np.full((H, W), np.inf)
    hit = np.zeros((H, W), bool)
    hit[sl] = (tn_max <= tf_min) & (tn_max > 0)
    t[sl] = tn_max
    ax_full = np.zeros((H, W), dtype=np.int64)
    ax_full[sl] = axis

    def nf(ok):
        ax = ax_full[ok]
        nn = np.zeros((int(ok.sum()), 3))
        nn[np.arange(nn.shape[0]), ax] = 1.0
        return _face_camera(nn, rx, ry, rz, ok)
    return zb.offer(t, nf, hit)


def _random_pixel_ray(rng, cam, W, H):
    u = rng.uniform(0, W - 1)
    v = rng.uniform(0, H - 1)
    return np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])


def _random_facing_normal(rng, nz_min=0.2):
    while True:
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        if n[2] > 0:
            n[2] = -n[2]
        if abs(n[2]) >= nz_min:
            return n


def _right_view_occlusion(d, hit):
    """Left pixels that the right camera cannot see.

    Pixel u of a row lands at x = u - d(u) in the right image.  It is hidden
    when a pixel further right in the same row lands at or left of x with a
    larger disparity (it is nearer and covers it).
    """
    H, W = d.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    x = np.where(hit, u - d, np.inf)
    # running minimum of x over u' > u
    rev = np.minimum.accumulate(x[:, ::-1], axis=1)[:, ::-1]
    right_min = np.concatenate([rev[:, 1:], np.full((H, 1), np.inf)], axis=1)
    return hit & (right_min < x - 0.5)


def _grow_bands(mask, hit, target, max_iter=64):
    """Dilate occlusion bands horizontally into hit pixels until `target`."""
    n_hit = max(int(hit.sum()), 1)
    m = mask.copy()
    for _ in range(max_iter):
        if m.sum() >= target * n_hit:
            break
        grown = m.copy()
        grown[:, 1:] |= m[:, :-1]
        grown[:, :-1] |= m[:, 1:]
        grown &= hit
        if grown.sum() == m.sum():
            break
        m = grown
    return m


def _depth_edges(d, hit, rel=0.05):
    e = np.zeros_like(hit)
    dd = np.abs(d[:, 1:] - d[:, :-1]) > rel * np.maximum(d[:, 1:], d[:, :-1])
    both = hit[:, 1:] & hit[:, :-1]
    e[:, 1:] |= dd & both
    e[:, :-1] |= dd & both
    e |= hit & ~np.roll(hit, 1, 1)
    return e & hit


def _iid_top_up(rng, mask, hit, target):
    n_hit = int(hit.sum())
    need = int(round(target * n_hit)) - int(mask.sum())
    if need <= 0:
        return mask
    cand = np.flatnonzero(hit & ~mask)
    pick = rng.choice(cand, size=min(need, cand.size), replace=False)
    m = mask.copy().ravel()
    m[pick] = True
    return m.reshape(mask.shape)


def _finish(name, cam, zb, rng, sigma, quant, invalid_mode, target, encode16):
    hit = zb.prim >= 0
    z = np.where(hit, zb.t, np.inf)
    d_true = np.where(hit, cam.fx * cam.baseline / z, 0.0)
    noise = rng.normal(0.0, sigma, size=d_true.shape) if sigma > 0 else 0.0
    d = np.where(hit, d_true + noise, 0.0)
    d = np.where(hit & (d <= 0), 0.0, d)
    if quant:
        d = np.round(d * quant) / quant
    if invalid_mode == "iid":
        inv = _iid_top_up(rng, np.zeros_like(hit), hit, target)
    elif invalid_mode == "bands":
        occ = _right_view_occlusion(d_true, hit)
        occ = _grow_bands(occ | (_depth_edges(d_true, hit) & occ), hit, target)
        if occ.sum() < target * hit.sum():
            occ = _grow_bands(occ | _depth_edges(d_true, hit), hit, target)
        # scenes without depth jumps have no bands to grow: top up iid
        inv = _iid_top_up(rng, occ, hit, target)
    elif invalid_mode == "bands+iid":
        occ = _right_view_occlusion(d_true, hit)
        inv = _iid_top_up(rng, occ, hit, target)
    else:
        inv = np.zeros_like(hit)
    d = np.where(inv | ~hit, 0.0, d).astype(np.float32)
    u16 = f16 = None
    if encode16:
        q = np.rint(d.astype(np.float64) * 256.0)
        u16 = np.clip(q, 0, 65535).astype(np.uint16)
        u16[q > 65535] = 0
        f16 = d.astype(np.float16)
        d = (u16.astype(np.float64) / 256.0).astype(np.float32)
        f16 = np.where(u16 == 0, np.float16(0), f16).astype(np.float16)
    gt = np.where(hit[..., None], zb.n, 0.0).astype(np.float32)
    return Scene(name=name, camera=cam, disp=d, gt_normal=gt,
                 prim=zb.prim.astype(np.int32), background=~hit,
                 disp_u16=u16, disp_f16=f16, disp_true=d_true.astype(np.float32),
                 meta=dict(invalid_fraction=float((inv & hit).sum()) / max(int(hit.sum()), 1),
                           n_primitives=zb.count))


def make_scene(name: str, seed=0, frame: int = 0, sigma: float | None = None,
               W: int | None = None, H: int | None = None, scale: float = 1.0) -> Scene:
    """Render the scene recipe `name` (a key of CONFIGS) for `frame`.

    The random stream is np.random.default_rng([cfg, frame, seed]).  `scale`
    shrinks width, height and focal length together (same field of view).
    """
    cfg = dict(CONFIGS[name])
    if scale != 1.0:
        cfg["W"] = max(8, int(round(cfg["W"] * scale)))
        cfg["H"] = max(8, int(round(cfg["H"] * scale)))
        cfg["f"] = cfg["f"] * scale
    if W is not None:
        cfg["W"] = W
    if H is not None:
        cfg["H"] = H
    if sigma is not None:
        cfg["sigma"] = sigma
    W_, H_ = cfg["W"], cfg["H"]
    rng = np.random.default_rng([cfg["cfg"], frame, seed])
    cam = Camera(cfg["f"], cfg["f"], W_ / 2.0, H_ / 2.0, cfg["B"])
    rays = _rays(cam, W_, H_)
    kind = cfg["kind"]
    if kind == "planes":
        zb = _ZBuffer(H_, W_, 0.05, 1e4)
        for _ in range(cfg["n_planes"]):
            n = _random_facing_normal(rng)
            P = _random_pixel_ray(rng, cam, W_, H_) * rng.uniform(1.0, 10.0)
            _add_plane(zb, rays, n, float(n @ P))
        return _finish(name, cam, zb, rng, cfg["sigma"], 0, "iid", cfg["invalid"], False)
    if kind == "mixed":
        z_near = cam.fx * cam.baseline / 280.0
        z_far = cam.fx * cam.baseline / 30.0
        zb = _ZBuffer(H_, W_, z_near, z_far)
        for _ in range(12):
            n = _random_facing_normal(rng)
            P = _random_pixel_ray(rng, cam, W_, H_) * rng.uniform(1.5, 8.5)
            _add_plane(zb, rays, n, float(n @ P))
        for _ in range(4):
            c = _random_pixel_ray(rng, cam, W_, H_) * rng.uniform(2.0, 7.0)
            _add_sphere(zb, rays, c, rng.uniform(0.3, 1.0))
        for _ in range(2):
            c = _random_pixel_ray(rng, cam, W_, H_) * rng.uniform(2.0, 7.0)
            h = rng.uniform(1.0, 3.0)
            _add_vcylinder(zb, rays, c, rng.uniform(0.2, 0.6), c[1] - h / 2, c[1] + h / 2)
        return _finish(name, cam, zb, rng, cfg["sigma"], cfg["quant"], "bands",
                       cfg["invalid"], False)
    if kind == "driving":
        zb = _ZBuffer(H_, W_, 0.5, 150.0)
        cam_h = 1.5
        _add_plane(zb, rays, np.array([0.0, -1.0, 0.0]), -cam_h)       # ground y = +1.5
        for sx in (-1.0, 1.0):                                          # facades x = -+8
            rx, ry, rz = rays
            den = -sx * rx
            ok_den = np.abs(den) > 1e-12
            t = np.where(ok_den, -8.0 / np.where(ok_den, den, 1.0), np.inf)
            y = np.where(ok_den, ry * np.where(ok_den, t, 0.0), 0.0)
            hit = ok_den & (t > 0) & (y >= cam_h - 12.0) & (y <= cam_h)
            n = np.array([-sx, 0.0, 0.0])

            def nf(ok, n=n):
                nn = np.broadcast_to(n, (int(ok.sum()), 3)).copy()
                return _face_camera(nn, rx, ry, rz, ok)
            zb.offer(t, nf, hit)
        for _ in range(20):
            x = rng.uniform(-7.0, 7.0)
            zc = rng.uniform(4.0, 60.0)
            w, h, l = rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0), rng.uniform(0.5, 5.0)
            _add_box(zb, rays, np.array([x - w / 2, cam_h - h, zc - l / 2]),
                     np.array([x + w / 2, cam_h, zc + l / 2]), cam)
        return _finish(name, cam, zb, rng, cfg["sigma"], 0, "bands+iid", cfg["invalid"], True)
    if kind == "sphere":
        zb = _ZBuffer(H_, W_, 0.05, 1e4)
        _add_sphere(zb, rays, np.array([0.0, 0.0, 3.0]), 1.4)
        return _finish(name, cam, zb, rng, cfg["sigma"], 0, "none", 0.0, False)
    raise ValueError(kind)


def config_scene(cfg: int, frame: int = 0, seed: int = 0) -> Scene:
    """Scene for workload recipe number `cfg` (1: 320x240 planes, 2: 1482x994
    mixed, 3: 2048x1024 driving, 6: 640x480 planes, 7: sphere)."""
    for name, c in CONFIGS.items():
        if c["cfg"] == cfg:
            return make_scene(name, seed=seed, frame=frame)
    raise KeyError(cfg)


def plane_disparity(cam: Camera, n, rho, W: int, H: int) -> np.ndarray:
    """Exact (float64) disparity of the plane n . X = rho seen by `cam`.

    Pixels whose ray misses the plane in front of the camera get 0.
    """
    rx, ry, rz = _rays(cam, W, H)
    den = n[0] * rx + n[1] * ry + n[2] * rz
    with np.errstate(divide="ignore", invalid="ignore"):
        z = rho / den
    ok = (np.abs(den) > 1e-12) & (z > 0)
    return np.where(ok, cam.fx * cam.baseline / np.where(ok, z, 1.0), 0.0)
