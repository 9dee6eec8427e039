"""torch.autograd binding of the rasterizer: forward through gs_render, backward through
gs_render_backward (argument marshalling only; both run in the library's CUDA kernels).

Parameters are the raw ones of training: means [P,3], log-scales [P,3], quaternions [P,4],
opacity logits [P], SH [P,16,3].  A batch of cameras is rendered with one device frame per
camera, so every camera's forward state is alive until the backward."""
from __future__ import annotations

import torch

from . import Frame, Scene, gs_opts


class GaussianRasterizer:
    """Owns a device scene of P Gaussians and one frame per camera slot of a batch."""

    def __init__(self, ctx, P: int, width: int, height: int, batch: int = 1, max_pairs: int = 1 << 24,
                 opts=None, sh_degree: int = 3):
        self.ctx = ctx
        self.P = int(P)
        self.width, self.height = int(width), int(height)
        self.opts = opts or gs_opts()
        self.sh_degree = sh_degree
        self.scene = None
        self.frames = [Frame(ctx, P, max_pairs, width, height) for _ in range(batch)]

    def _update(self, means, log_scales, quats, logits, sh):
        args = [t.detach().contiguous() for t in (means, log_scales, quats, logits, sh)]
        if self.scene is None:
            self.scene = Scene(self.ctx, *args, sh_degree=self.sh_degree, activated=False)
        else:
            self.scene.gs_scene_update(*args, sh_degree=self.sh_degree, activated=False)
        self._keep = args

    def __call__(self, means, log_scales, quats, logits, sh, cams):
        return _RasterizeBatch.apply(means, log_scales, quats, logits, sh, self, list(cams))


class _RasterizeBatch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, logits, sh, rast: GaussianRasterizer, cams):
        if len(cams) > len(rast.frames):
            raise ValueError(f"{len(cams)} cameras but {len(rast.frames)} frames")
        rast._update(means, log_scales, quats, logits, sh)
        outs, saved = [], []
        for fr, cam in zip(rast.frames, cams):
            rgb, T, last = fr.render(rast.scene, cam, rast.opts)
            outs.append(rgb)
            saved.append((fr, T, last))
        ctx.rast = rast
        ctx.saved = saved
        return torch.stack(outs)

    @staticmethod
    def backward(ctx, grad_out):
        rast = ctx.rast
        grads = None
        for i, (fr, T, last) in enumerate(ctx.saved):
            grads = fr.gs_render_backward(rast.scene, grad_out[i].contiguous(), T, last, grads=grads,
                                          accumulate=i > 0)
        return grads["means"], grads["scales"], grads["quats"], grads["opacity"], grads["sh"], None, None
