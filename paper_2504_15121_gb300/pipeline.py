"""Frame-level conveniences over the C ABI: pitched output buffers and a
context holder.  All work is done by libsn.so through `sn`."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import sn


@dataclass
class FrameBuffers:
    """Device outputs of one frame, laid out as include/sn.h requires."""
    den: torch.Tensor          # [H, W] float32
    normals: torch.Tensor      # [3, H, W] float32, or [H, W, 4] int16 (snorm16)
    points: torch.Tensor       # [3, H, W] float32
    labels: torch.Tensor       # [H, W] int32
    mask: torch.Tensor         # [H, W] uint8
    num_components: torch.Tensor  # [1] int32

    @staticmethod
    def allocate(W: int, H: int, normal_fmt: int = sn.SN_NORMALS_F32X3, device="cuda"):
        nrm = (sn.empty_planes(3, H, W, torch.float32, device) if normal_fmt == sn.SN_NORMALS_F32X3
               else sn.empty_snorm(H, W, device))
        return FrameBuffers(
            den=sn.empty_image(H, W, torch.float32, device),
            normals=nrm,
            points=sn.empty_planes(3, H, W, torch.float32, device),
            labels=sn.empty_image(H, W, torch.int32, device),
            mask=sn.empty_image(H, W, torch.uint8, device),
            num_components=torch.zeros(1, dtype=torch.int32, device=device),
        )


def host_buffers(W: int, H: int, normal_fmt: int = sn.SN_NORMALS_F32X3, pin: bool = True) -> FrameBuffers:
    """Host outputs of one frame for sn_run_frame_host (contiguous; pinned by
    default, so that the copies are asynchronous); den is not used."""
    def host(shape, dtype):
        t = torch.empty(shape, dtype=dtype)
        return t.pin_memory() if pin else t
    nrm = host((3, H, W), torch.float32) if normal_fmt == sn.SN_NORMALS_F32X3 else host((H, W, 4), torch.int16)
    return FrameBuffers(den=None, normals=nrm, points=host((3, H, W), torch.float32),
                        labels=host((H, W), torch.int32), mask=host((H, W), torch.uint8),
                        num_components=host((1,), torch.int32))


_IN_DTYPE = {torch.float32: sn.SN_IN_F32, torch.float16: sn.SN_IN_F16, torch.int16: sn.SN_IN_U16X256,
             torch.uint16: sn.SN_IN_U16X256}


class Pipeline:
    """One sn_ctx for W x H frames with fixed camera and parameters."""

    def __init__(self, cam, W: int, H: int, gate_weights=None, **params):
        """params: fields of sn_params.  learned=1 loads the gate weights
        (gate_weights: path or bytes; default: the packaged trained weights)."""
        self.W, self.H = W, H
        self.params = sn.default_params(**params)
        self.ctx = sn.sn_create(cam, W, H, self.params)
        if self.params.learned:
            from . import gate
            blob = gate_weights if isinstance(gate_weights, (bytes, bytearray)) else \
                open(gate_weights or gate.DEFAULT_WEIGHTS, "rb").read()
            sn.sn_load_gate_weights(self.ctx, bytes(blob))

    def close(self):
        if self.ctx:
            sn.sn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def buffers(self, device="cuda") -> FrameBuffers:
        return FrameBuffers.allocate(self.W, self.H, self.params.normal_fmt, device)

    def host_buffers(self, pin: bool = True) -> FrameBuffers:
        return host_buffers(self.W, self.H, self.params.normal_fmt, pin)

    def run_frame_host(self, disp: torch.Tensor, out: FrameBuffers, stream=None):
        """sn_run_frame_host: host disparity in, host outputs (see host_buffers)."""
        sn.sn_run_frame_host(self.ctx, disp, out.normals, out.points, out.labels, out.mask,
                             num_components=out.num_components, stream=stream)
        return out

    def upload(self, disp_np, device="cuda") -> torch.Tensor:
        """Copy a host disparity map into a pitched device image."""
        import numpy as np
        a = np.ascontiguousarray(disp_np)
        if a.dtype == np.uint16:
            t = torch.from_numpy(a.view(np.int16))
        else:
            t = torch.from_numpy(a)
        img = sn.empty_image(self.H, self.W, t.dtype, device)
        img.copy_(t)
        return img

    def run_frame(self, disp: torch.Tensor, out: FrameBuffers, stream=None, write_den: bool = True):
        sn.sn_run_frame(self.ctx, disp, out.normals, out.points, out.labels, out.mask,
                        den=out.den if write_den else None, num_components=out.num_components,
                        stream=stream)
        return out
