"""The largest frames a context accepts: 32768 x 32768 (2^30 pixels, 8 GiB
per depth-id buffer) and 32767 x 32767 (a ragged last quad and a partial last
chunk).  Pixel indices, quad and chunk counts and the resolve's grid are at
their largest here.  The oracle projects every point and takes the per-pixel
minimum of the keys on the host, so only the covered pixels are compared key
by key; everywhere else the frame must be empty, counted on the device.  Three
frames from different cameras check that earlier frames' pixels are cleared
(the third frame splats into the first frame's buffer) and repainted."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context

from ._harness import CENTRE, UP, upload

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(2**64 - 1)


def _expected(pos, W, H, eye):
    """Covered pixel indices and their minimum keys (the oracle's projection,
    reduced on the host)."""
    M = oracle.camera_f32(eye, CENTRE, UP, 60.0, W / H, 0.1, 100.0)
    px, w = oracle.project_f32(M, pos, W, H, np.float32(0.1), np.float32(100.0))
    keep = px != 0xFFFFFFFF
    ids = np.nonzero(keep)[0].astype(np.uint64)
    keys = (w[keep].view(np.uint32).astype(np.uint64) << np.uint64(32)) | ids
    pix = px[keep].astype(np.int64)
    order = np.lexsort((keys, pix))
    pix, keys = pix[order], keys[order]
    first = np.ones(pix.size, bool)
    first[1:] = pix[1:] != pix[:-1]
    return pix[first], keys[first]


@pytest.mark.parametrize("W,H", [(32768, 32768), (32767, 32767)])
def test_largest_frames(W, H):
    n = 200_003
    stored = inputs.encode(inputs.uniform_cloud(n, 81), "f32")
    pos = np.array(stored, copy=True)
    color, bg = 0xFF00FF00, 0x01020304
    eyes = [(0.5, 0.5, 2.5), (2.0, 1.0, 1.5), (0.5, 0.5, 2.0)]
    with Context(W, H) as ctx:
        ctx.alloc_points(n, "f32")
        upload(ctx, stored)
        ctx.set_sim(8, 0, 1e-3, 0)
        ctx.set_style(color, bg)
        for f, eye in enumerate(eyes):
            ctx.set_camera(eye, CENTRE, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            oracle.displace(pos, "f32", 8, 0, f, np.float32(1e-3))
            pix, want = _expected(pos, W, H, eye)
            keys = ctx.frame_keys().view(-1)
            rgba = ctx.frame_rgba().view(-1)
            idx = torch.from_numpy(pix).cuda()
            got = keys[idx].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want), f"keys of frame {f}"
            assert int((keys != -1).sum()) == pix.size, f"non-empty pixels of frame {f}"
            assert (rgba[idx].cpu().numpy().view(np.uint32) == color).all(), f"covered colours of frame {f}"
            assert int((rgba != bg).sum()) == pix.size, f"background, frame {f}"
        got_pos = ctx.points.cpu().numpy()
    assert np.array_equal(got_pos, pos)
