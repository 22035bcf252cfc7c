"""The largest cloud a context accepts: 2^32 - 1 FP32 points (51.5 GB), so
point ids, group counts and the grid reach their largest values and the last
group is ragged (three points).  The oracle cannot replay four billion
points here, so the checks are ones that hold at any size, on samples:
- sampled points (random, the first, and the last eight) are displaced bit
  for bit as the oracle displaces them;
- at each sampled point's pixel the key is at most the point's own key (the
  frame holds a per-pixel minimum);
- every sampled winner's id is a point that projects, under the oracle's
  projection of its displaced position, to that pixel with that depth."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300.api import Context

from ._harness import CENTRE, UP

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(2**64 - 1)


def test_largest_cloud():
    n = (1 << 32) - 1
    W, H = 1920, 1080
    eye = (0.5, 0.5, 2.5)
    with Context(W, H) as ctx:
        pts = ctx.alloc_points(n, "f32")
        gen = torch.Generator(device="cuda")
        gen.manual_seed(91)
        pts.uniform_(0.0, 1.0, generator=gen)
        rng = np.random.default_rng(92)
        ids = np.unique(np.concatenate([rng.integers(0, n, 8192), [0, 1, 2, 3], np.arange(n - 8, n)]))
        idx = torch.from_numpy(ids.astype(np.int64)).cuda()
        want = pts[idx].cpu().numpy()
        ctx.set_sim(93, 0, 1e-3, 0)
        ctx.set_camera(eye, CENTRE, UP, 60.0, 0.1, 100.0)
        ctx.step_and_render()
        got = pts[idx].cpu().numpy()
        oracle.displace_ids_f32(want, ids.astype(np.uint32), 93, 0, 0, np.float32(1e-3))
        assert np.array_equal(got, want)

        M = oracle.camera_f32(eye, CENTRE, UP, 60.0, W / H, 0.1, 100.0)
        px, w = oracle.project_f32(M, want, W, H, np.float32(0.1), np.float32(100.0))
        vis = px != 0xFFFFFFFF
        assert vis.sum() > len(ids) // 2
        keys = ctx.frame_keys().view(-1)
        at = keys[torch.from_numpy(px[vis].astype(np.int64)).cuda()].cpu().numpy().view(np.uint64)
        mine = (w[vis].view(np.uint32).astype(np.uint64) << np.uint64(32)) | ids[vis].astype(np.uint64)
        assert (at <= mine).all()

        winners = (at & np.uint64(0xFFFFFFFF)).astype(np.int64)
        assert (winners < n).all()
        wpos = pts[torch.from_numpy(winners).cuda()].cpu().numpy()
        wpx, ww = oracle.project_f32(M, wpos, W, H, np.float32(0.1), np.float32(100.0))
        assert np.array_equal(wpx, px[vis])
        assert np.array_equal(ww.view(np.uint32).astype(np.uint64), at >> np.uint64(32))
        assert int((keys != -1).sum()) > 0
