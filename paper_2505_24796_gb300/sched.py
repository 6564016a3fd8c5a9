"""Learned scheduling of the batched multi-view renderer (host-side driver).

Every computation runs in the library's kernels (features, MLP forward/backward, Adam, ordering,
rendering); this module only sequences the calls and owns the buffers.

  views = MultiView(scene, cameras)          # per-view projection + sort, resident on the GPU
  data  = views.training_data()               # per-tile features and recorded tile costs
  model = TileCostModel(); model.fit(*data)   # trained on the GPU by tcgs_mlp_bwd + tcgs_adam_step
  q     = views.queue("mlp", model)           # (view << 16 | tile) items, longest predicted first
  views.render(q)                             # persistent batched render (tcgs_render_fwd_batched)
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Renderer, _lib, scene_to_device, tcgs_adam_step, tcgs_feature_norm, tcgs_mlp_bwd, tcgs_mlp_fwd,
               tcgs_project, tcgs_render_fwd_batched, tcgs_sched_order, tcgs_tile_features)

STAT_WALKED, STAT_CYCLES = 4, 5


class TileCostModel:
    """MLP 8 -> 32 -> 32 -> 1 predicting log(1 + list entries walked) of a tile."""

    def __init__(self, device="cuda", seed=0):
        rng = np.random.default_rng(seed)
        blocks = []
        for fan_in, shape in [(8, (32, 8)), (None, (32,)), (32, (32, 32)), (None, (32,)), (32, (32,)), (None, (1,))]:
            if fan_in is None:
                blocks.append(np.zeros(shape))
            else:
                blocks.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), shape))
        flat = np.concatenate([b.reshape(-1) for b in blocks]).astype(np.float32)
        assert flat.size == _lib.TCGS_MLP_PARAMS
        self.device = torch.device(device)
        self.params = torch.from_numpy(flat).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.norm = torch.cat([torch.zeros(8), torch.ones(8)]).to(self.device)
        self.step = 0

    def fit(self, X: torch.Tensor, y: torch.Tensor, steps=600, lr=3e-3):
        """Full-batch Adam on the mean squared error of log cost; returns the final loss."""
        self.norm = tcgs_feature_norm(X)
        for _ in range(steps):
            self.step += 1
            tcgs_mlp_bwd(self.params, self.norm, X, y, grad=self.grad)
            tcgs_adam_step(self.params, self.m, self.v, self.grad, lr, step=self.step)
        return self.loss(X, y)

    def loss(self, X, y) -> float:
        acc = torch.zeros(1, device=self.device)
        scratch = torch.zeros_like(self.params)
        tcgs_mlp_bwd(self.params, self.norm, X, y, grad=scratch, loss=acc)
        return float(acc.item())

    def predict(self, X) -> torch.Tensor:
        return tcgs_mlp_fwd(self.params, self.norm, X)


class MultiView:
    """One scene seen from several cameras: per-view projection, sort and output buffers."""

    def __init__(self, scene: dict, cameras, precision="tc_fp16_split", device="cuda"):
        self.device = torch.device(device)
        self.scene = scene_to_device(scene, self.device) if isinstance(scene["means3"], np.ndarray) else scene
        self.precision = precision
        P = self.scene["means3"].shape[0]
        self.views = []
        for cam in cameras:
            pr = tcgs_project(cam, self.scene["means3"], self.scene["scales"], self.scene["quats"], self.scene["sh"],
                              self.scene["sh_degree"])
            n = int(pr["tiles_touched"].to(torch.int64).sum().item())
            r = Renderer(cam, P, n + 1024, device=self.device, stats=True)
            r.proj = pr
            r.bin_sort(opacity=self.scene["opacity"])
            self.views.append(r)
        torch.cuda.synchronize(self.device)

    def render_each(self, stats=True):
        """One tcgs_render_fwd per view (tile stats recorded when asked)."""
        for r in self.views:
            if r.stats is not None:
                r.stats.zero_()
            saved = r.stats
            if not stats:
                r.stats = None
            r.render(self.scene["opacity"], self.precision)
            r.stats = saved

    def features(self) -> torch.Tensor:
        feats = [tcgs_tile_features(r.cam, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"],
                                    r.proj["conic"], self.scene["opacity"], r.proj["depth"], r.proj["radius"])
                 for r in self.views]
        return torch.cat(feats)

    def items(self) -> torch.Tensor:
        its = [(v << 16) + np.arange(r.num_tiles) for v, r in enumerate(self.views)]
        return torch.from_numpy(np.concatenate(its).astype(np.int32)).to(self.device)

    def tile_costs(self):
        """(walked entries, CTA cycles) per (view, tile), recorded by the last render_each()."""
        st = torch.cat([r.stats for r in self.views]).to(torch.int64)
        return st[:, STAT_WALKED], st[:, STAT_CYCLES] * 64

    def training_data(self):
        self.render_each(stats=True)
        torch.cuda.synchronize(self.device)
        walked, _ = self.tile_costs()
        X = self.features().contiguous()
        y = torch.log1p(walked.to(torch.float32)).contiguous()
        return X, y

    def queue(self, policy: str, model: TileCostModel | None = None) -> torch.Tensor:
        items = self.items()
        if policy == "natural":
            return items
        if policy == "length":
            cost = torch.cat([(r.bins["tile_ranges"][:, 1] - r.bins["tile_ranges"][:, 0]).to(torch.float32)
                              for r in self.views]).contiguous()
        elif policy == "mlp":
            cost = model.predict(self.features().contiguous())
        else:
            raise ValueError(policy)
        return tcgs_sched_order(cost, items)

    def batched_views(self, stats=False):
        out = []
        for r in self.views:
            if stats and r.stats is not None:
                r.stats.zero_()
            out.append(dict(cam=r.cam, tile_ranges=r.bins["tile_ranges"], ids_sorted=r.bins["ids_sorted"],
                            mean2d=r.proj["mean2d"], conic=r.proj["conic"], rgb=r.proj["rgb"], img=r.out["img"],
                            T_final=r.out["T_final"], n_contrib=r.out["n_contrib"],
                            tile_stats=r.stats if stats else None))
        return out

    def render(self, queue: torch.Tensor, max_ctas=0, stats=False):
        from . import render_opts
        opts = render_opts(self.precision)
        tcgs_render_fwd_batched(self.batched_views(stats), opts, self.scene["opacity"], queue, max_ctas=max_ctas)

    def time_render(self, queue, reps=10, warmup=3):
        for _ in range(warmup):
            self.render(queue)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            self.render(queue)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))
