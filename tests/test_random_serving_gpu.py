"""A sweep of seeded random serving scenarios against the oracle, bit for
bit: the shared cloud's size, and for each viewer its private cloud, frame
size, colours, camera orbit, join tick and number of frames are drawn
independently, so viewers join and leave mid-run and later joins reuse the
buffers of earlier ones (of other frame sizes).  Every frame of every viewer
is compared with the oracle's render of the shared and private clouds at that
viewer's tick and frame index; ticks alternate between the zero-copy tick and
the host round trip at random."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Server

pytestmark = pytest.mark.gpu

COUNT = 12
CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)
AMP = np.float32(1e-3)


def _scenario(k):
    rng = np.random.default_rng(70_000 + k)
    shared_n = int(rng.integers(1, 30_000))
    viewers = []
    for v in range(int(rng.integers(1, 7))):
        viewers.append(dict(n=int(rng.integers(1, 8_000)), W=int(rng.integers(1, 140)), H=int(rng.integers(1, 100)),
                            join=int(rng.integers(0, 6)), frames=int(rng.integers(1, 6)),
                            seed=int(rng.integers(0, 2**31)), cloud=v + 1, color=int(rng.integers(0, 2**32)),
                            background=int(rng.integers(0, 2**32)), radius=float(rng.uniform(0.4, 4.0)),
                            start=float(rng.uniform(0, 360)), elev=float(rng.uniform(-1.0, 1.0)),
                            step=float(rng.uniform(-25, 25))))
    roundtrips = rng.random(16) < 0.3
    return shared_n, viewers, roundtrips


@pytest.mark.parametrize("k", range(COUNT))
def test_random_serving(k):
    shared_n, viewers, roundtrips = _scenario(k)
    shared0 = inputs.encode(inputs.uniform_cloud(shared_n, 71_000 + k), "f32")
    priv0 = [inputs.encode(inputs.uniform_cloud(v["n"], 72_000 + 10 * k + i), "f32") for i, v in enumerate(viewers)]
    shared_color = 0xFF123456
    got = {}
    with Server(shared_n, "f32", 77, 0, float(AMP)) as srv:
        srv.shared_points().copy_(torch.from_numpy(shared0))
        srv.set_shared_color(shared_color)
        ids, done = {}, {}
        last = max(v["join"] + v["frames"] for v in viewers)
        for tick in range(last):
            for i, v in enumerate(viewers):
                if v["join"] == tick:
                    ids[i] = srv.add_viewer(v["n"], v["W"], v["H"], seed=v["seed"], cloud=v["cloud"],
                                            amplitude=float(AMP), color=v["color"], background=v["background"])
                    srv.viewer_points(ids[i]).copy_(torch.from_numpy(priv0[i]))
                    done[i] = 0
            for i, vid in ids.items():
                v = viewers[i]
                eye = inputs.orbit_eye(done[i], v["step"], v["radius"], CEN, v["elev"], v["start"])
                srv.set_camera(vid, eye, CEN, UP, 60.0, 0.1, 100.0)
            srv.tick(roundtrip=bool(roundtrips[tick % len(roundtrips)]))
            torch.cuda.synchronize()
            for i in list(ids):
                rgba, keys, f = srv.frame(ids[i])
                got[(i, done[i])] = (keys.cpu().numpy().reshape(-1).view(np.uint64).copy(),
                                     rgba.cpu().numpy().reshape(-1).view(np.uint32).copy())
                done[i] += 1
                assert f == done[i]
                if done[i] == viewers[i]["frames"]:
                    srv.remove_viewer(ids.pop(i))
    # the oracle: viewer i's frame j is rendered at tick join + j, after shared steps 0..join+j and private
    # steps 0..j
    for (i, j), (keys, rgba) in sorted(got.items()):
        v = viewers[i]
        shared = shared0.copy()
        for t in range(v["join"] + j + 1):
            oracle.displace_f32(shared, 77, 0, t, AMP)
        priv = priv0[i].copy()
        for s in range(j + 1):
            oracle.displace_f32(priv, v["seed"], v["cloud"], s, AMP)
        both = np.concatenate([shared, priv])
        colors = np.concatenate([np.full(shared_n, shared_color, np.uint32), np.full(v["n"], v["color"], np.uint32)])
        eye = inputs.orbit_eye(j, v["step"], v["radius"], CEN, v["elev"], v["start"])
        M = oracle.camera_f32(eye, CEN, UP, 60.0, v["W"] / v["H"], 0.1, 100.0)
        wk, wr = oracle.render(both, "f32", M, v["W"], v["H"], np.float32(0.1), np.float32(100.0), colors, 0,
                               v["background"])
        assert np.array_equal(keys, wk), f"keys of viewer {i} frame {j} (scenario {k})"
        assert np.array_equal(rgba, wr), f"rgba of viewer {i} frame {j} (scenario {k})"
