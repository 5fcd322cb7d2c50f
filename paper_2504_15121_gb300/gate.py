"""Learned boundary gate: ctypes binding of the trainer (include/sn_gate.h),
the weights file format, the training set and the training loop.

Training runs on the GPU through the library's own forward/backward/Adam
kernels; this module only builds the data (patches of integer disparity
codes and their labels from the scene generator's ground truth) and drives
the loop.

Weights file (version 1): b"SNGW", uint32 version, uint32 n_params, then
n_params little-endian float32 in the order W1 [16][9][8], b1 [16],
W2 [16][9][16], b2 [16], W3 [16], b3; a JSON sidecar records how they were
trained.  sn_load_gate_weights takes the same bytes.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import struct
import time

import numpy as np
import torch

from .sn import SnError, SN_OK, lib

MAGIC = b"SNGW"
VERSION = 1
WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_WEIGHTS = os.path.join(WEIGHTS_DIR, "gate_v1.bin")

_vp, _i, _f = C.c_void_p, C.c_int, C.c_float
for _name, _args, _res in [
        ("sn_gate_param_count", [], _i),
        ("sn_gate_trainer_create", [_i, _vp, C.POINTER(_vp)], _i),
        ("sn_gate_trainer_destroy", [_vp], _i),
        ("sn_gate_trainer_grad", [_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp], _i),
        ("sn_gate_trainer_step", [_vp, _vp, _vp, _i, _f, _vp, _vp], _i),
        ("sn_gate_trainer_state", [_vp, _vp, _vp, _vp, C.POINTER(C.c_longlong)], _i),
        ("sn_gate_trainer_resume", [_vp, _vp, _vp, _vp, C.c_longlong], _i),
        ("sn_gate_trainer_check_device", [_vp, _vp], _i)]:
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

EXPORTS = ("sn_gate_param_count", "sn_gate_trainer_create", "sn_gate_trainer_destroy",
           "sn_gate_trainer_grad", "sn_gate_trainer_step", "sn_gate_trainer_state",
           "sn_gate_trainer_resume", "sn_gate_trainer_check_device")
N_PARAMS = lib.sn_gate_param_count()


def _check(st, what):
    if st != SN_OK:
        raise SnError(st, what)


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------- weights
def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights; the unused feature channels 3..7 start at 0."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / 27), (16, 9, 8))
    W1[:, :, 3:] = 0.0
    W2 = rng.normal(0, np.sqrt(2.0 / 144), (16, 9, 16))
    W3 = rng.normal(0, np.sqrt(1.0 / 16), 16)
    theta = np.concatenate([W1.ravel(), np.zeros(16), W2.ravel(), np.zeros(16), W3, [0.0]])
    assert theta.size == N_PARAMS
    return theta.astype(np.float32)


def weights_blob(theta) -> bytes:
    theta = np.asarray(theta, "<f4")
    return MAGIC + struct.pack("<II", VERSION, theta.size) + theta.tobytes()


def parse_blob(blob: bytes) -> np.ndarray:
    if blob[:4] != MAGIC:
        raise ValueError("not a gate weights file")
    ver, n = struct.unpack("<II", blob[4:12])
    if ver != VERSION or n != N_PARAMS:
        raise ValueError(f"weights version {ver} with {n} parameters; expected {VERSION}, {N_PARAMS}")
    return np.frombuffer(blob[12:12 + 4 * n], "<f4").copy()


def save_weights(path, theta, meta=None):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "wb") as f:
        f.write(weights_blob(theta))
    if meta is not None:
        with open(path[:-4] + ".json", "w") as f:
            json.dump(meta, f, indent=1, sort_keys=True)


def load_weights(path=DEFAULT_WEIGHTS) -> np.ndarray:
    with open(path, "rb") as f:
        return parse_blob(f.read())


# ---------------------------------------------------------------- trainer
class Trainer:
    def __init__(self, max_batch: int, theta0):
        self.max_batch = max_batch
        self.h = _vp()
        t0 = np.ascontiguousarray(theta0, np.float32)
        _check(lib.sn_gate_trainer_create(max_batch, t0.ctypes.data_as(_vp), C.byref(self.h)),
               "sn_gate_trainer_create")
        self.grad_buf = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if self.h:
            lib.sn_gate_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def grad(self, patches, y=None):
        """(loss, grad, q) on device tensors patches int32 [B, 36], y float [B]."""
        B = patches.shape[0]
        q = torch.empty(B, dtype=torch.float32, device="cuda")
        _check(lib.sn_gate_trainer_grad(self.h, _ptr(patches), _ptr(y), B, _ptr(self.grad_buf), _ptr(q),
                                        _ptr(self.loss_buf), _stream()), "sn_gate_trainer_grad")
        return self.loss_buf.clone(), self.grad_buf.clone(), q

    def step(self, patches, y, lr: float):
        B = patches.shape[0]
        _check(lib.sn_gate_trainer_step(self.h, _ptr(patches), _ptr(y), B, float(lr), _ptr(self.loss_buf),
                                        _stream()), "sn_gate_trainer_step")
        return self.loss_buf

    def check_device(self):
        """Raises SnError (SN_ETIMEOUT) if a bounded tensor-core wait of the
        trainer's GEMMs gave up since the last check (waits for the stream)."""
        _check(lib.sn_gate_trainer_check_device(self.h, _stream()), "sn_gate_trainer_check_device")

    def state(self):
        th, m, v = (np.zeros(N_PARAMS, np.float32) for _ in range(3))
        step = C.c_longlong()
        _check(lib.sn_gate_trainer_state(self.h, th.ctypes.data_as(_vp), m.ctypes.data_as(_vp),
                                         v.ctypes.data_as(_vp), C.byref(step)), "sn_gate_trainer_state")
        return th, m, v, step.value

    def resume(self, theta, m, v, step):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (theta, m, v)]
        _check(lib.sn_gate_trainer_resume(self.h, *[a.ctypes.data_as(_vp) for a in arrs], int(step)),
               "sn_gate_trainer_resume")


# ---------------------------------------------------------------- data
TRAIN_RECIPES = (("planes_320x240", 1.0), ("planes_640x480", 0.5), ("mixed_1482x994", 0.3),
                 ("driving_2048x1024", 0.25))


def codes(disp: np.ndarray) -> np.ndarray:
    """Integer disparity codes of a float map, as the library defines them
    (rint(256 d) with ties to even; valid iff 1 <= code <= 131071)."""
    x = disp.astype(np.float64) * 256.0
    r = np.rint(np.where(np.isfinite(x), x, 0.0))
    return np.where((disp > 0) & (r >= 1) & (r <= 131071), r, 0).astype(np.int32)


def one_surface_labels(d_true: np.ndarray, D: np.ndarray) -> np.ndarray:
    """True where the 5x5 patch centred at a pixel has at least 13 valid
    pixels (outside the image: invalid) and no depth discontinuity: every two
    4-adjacent valid pixels of the patch differ in noise-free disparity by at
    most max(0.03 min(d1, d2), 0.25 px)."""
    H, W = D.shape
    v = np.pad(D > 0, 3)
    t = np.pad(d_true.astype(np.float64), 3)
    # smooth[i] of a pair of neighbours: both valid and within the bound, or not both valid
    okr = np.ones_like(v)
    a, b = t[:, :-1], t[:, 1:]
    both = v[:, :-1] & v[:, 1:]
    okr[:, :-1] = ~both | (np.abs(a - b) <= np.maximum(0.03 * np.minimum(a, b), 0.25))
    okd = np.ones_like(v)
    a, b = t[:-1, :], t[1:, :]
    both = v[:-1, :] & v[1:, :]
    okd[:-1, :] = ~both | (np.abs(a - b) <= np.maximum(0.03 * np.minimum(a, b), 0.25))
    cnt = np.zeros((H, W), np.int64)
    smooth = np.ones((H, W), bool)
    for dy in range(5):
        for dx in range(5):
            cnt += v[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            if dx < 4:
                smooth &= okr[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            if dy < 4:
                smooth &= okd[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    return (cnt >= 13) & smooth


def _scene_samples(args):
    name, scale, frame, per_class, seed, pos_ratio = args
    from scenes import make_scene
    s = make_scene(name, frame=frame, scale=scale, seed=seed)
    D = codes(s.disp)
    lab = one_surface_labels(s.disp_true, D)
    rng = np.random.default_rng([seed, frame, 7])
    H, W = D.shape
    Dp = np.pad(D, 3)
    pos = np.flatnonzero(lab.ravel())
    neg = np.flatnonzero((~lab).ravel())
    take = []
    for idx, n in ((pos, int(round(per_class * pos_ratio))), (neg, per_class)):
        if idx.size:
            take.append(rng.choice(idx, size=min(n, idx.size), replace=False))
    sel = np.concatenate(take) if take else np.zeros(0, int)
    vv, uu = np.divmod(sel, W)
    patches = np.stack([Dp[v + 1:v + 7, u + 1:u + 7].ravel() for v, u in zip(vv, uu)]) if sel.size else \
        np.zeros((0, 36), np.int32)
    return patches.astype(np.int32), lab.ravel()[sel].astype(np.float32)


def make_training_set(n_scenes=2000, per_class=256, seed=0, workers=None, pos_ratio=1.0):
    """Patches from n_scenes seeded scenes (all recipes, reduced sizes):
    per scene `per_class` negatives and `pos_ratio` times as many positives.
    Uses a spawn-started process pool (safe after CUDA init)."""
    import multiprocessing as mp
    jobs = []
    for i in range(n_scenes):
        name, scale = TRAIN_RECIPES[i % len(TRAIN_RECIPES)]
        jobs.append((name, scale, 1000 + i, per_class, seed, pos_ratio))
    workers = workers or max(1, min(16, (os.cpu_count() or 2)))
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_scene_samples, jobs, chunksize=8)
    X = np.concatenate([p for p, _ in parts])
    y = np.concatenate([l for _, l in parts])
    return X, y


def train(X, y, epochs=4, batch=4096, lr=3e-3, seed=0, theta0=None, log=print, checkpoint=None):
    """Adam on the GPU; returns (theta, history)."""
    dev = "cuda"
    Xd = torch.from_numpy(X).to(dev)
    yd = torch.from_numpy(y).to(dev)
    n = Xd.shape[0]
    trainer = Trainer(batch, theta0 if theta0 is not None else init_params(seed))
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    k = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        losses = []
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            rate = lr * 0.5 * (1 + np.cos(np.pi * k / total))
            losses.append(trainer.step(Xd[idx].contiguous(), yd[idx].contiguous(), rate).clone())
            k += 1
        ep_loss = float(torch.stack(losses).mean())
        trainer.check_device()
        hist.append(ep_loss)
        log(f"epoch {ep} loss {ep_loss:.4f} ({time.time() - t0:.1f} s)")
        if checkpoint:
            th, m, v, step = trainer.state()
            np.savez(checkpoint, theta=th, m=m, v=v, step=step, epoch=ep, version=VERSION)
    theta, *_ = trainer.state()
    trainer.close()
    return theta, hist


def accuracy(theta, X, y, tau=0.5, batch=65536):
    """Fraction of correct decisions at threshold tau (GPU forward)."""
    tr = Trainer(batch, theta)
    correct = 0
    prec_num = prec_den = 0
    for i in range(0, len(y), batch):
        xb = torch.from_numpy(X[i:i + batch]).cuda()
        _, _, q = tr.grad(xb)
        qh = q.cpu().numpy()
        yb = y[i:i + batch]
        correct += int(((qh >= tau) == (yb > 0.5)).sum())
        prec_den += int((qh >= tau).sum())
        prec_num += int(((qh >= tau) & (yb > 0.5)).sum())
    tr.close()
    return correct / len(y), (prec_num / prec_den if prec_den else float("nan"))


def main():
    import argparse
    ap = argparse.ArgumentParser(description="Train the boundary gate on the GPU")
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--per-class", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--pos-ratio", type=float, default=1.0, help="positives per negative in the training set")
    a = ap.parse_args()
    t0 = time.time()
    X, y = make_training_set(a.scenes, a.per_class, a.seed, pos_ratio=a.pos_ratio)
    print(f"{len(y)} samples, {y.mean():.3f} positive, built in {time.time() - t0:.1f} s", flush=True)
    Xv, yv = make_training_set(64, 256, a.seed + 1)
    theta, hist = train(X, y, a.epochs, a.batch, a.lr, a.seed, checkpoint=a.checkpoint)
    acc, prec = accuracy(theta, Xv, yv, 0.5)
    acc9, prec9 = accuracy(theta, Xv, yv, 0.9)
    meta = dict(version=VERSION, scenes=a.scenes, per_class=a.per_class, epochs=a.epochs, batch=a.batch,
                lr=a.lr, seed=a.seed, samples=int(len(y)), loss=hist, recipes=TRAIN_RECIPES, pos_ratio=a.pos_ratio,
                val_scenes=64, val_seed=a.seed + 1, val_accuracy_tau05=acc, val_precision_tau05=prec,
                val_accuracy_tau09=acc9, val_precision_tau09=prec9)
    save_weights(a.out, theta, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
