"""Failure paths on the GPU, none of which faults, traps or hangs it: a
bounded device wait that runs out, injected allocation failures, budget
refusals, out-of-order calls and invalid arguments.  After each, the
library keeps working and its frames still match the oracle."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context, MmrError

from ._harness import fixed_eye, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounded_wait_times_out_and_context_stays_usable():
    with Context(32, 32) as ctx:
        ctx.alloc_points(100, "f32")
        ctx.check_device()                               # clean to start with
        ctx.selftest_bounded_wait(max_cycles=1_000_000)  # ~0.5 ms, nothing ever arrives
        with pytest.raises(MmrError, match="TIMEOUT"):
            ctx.check_device()
        ctx.check_device()                               # the flag was cleared
        ctx.set_camera((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
        ctx.step_and_render()
        ctx.check_device()
    # and a full frame afterwards still matches the oracle
    stored = inputs.encode(inputs.uniform_cloud(5000, 31), "f32")
    args = (stored, "f32", 48, 40, 3, 1e-3, 2, fixed_eye)
    g, o = gpu_run(*args), oracle_run(*args)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1]) and np.array_equal(g[2], o[2])


def _run_child(code, env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "-c", textwrap.dedent(code)], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_batch_bounded_wait_times_out_and_batch_stays_usable():
    """The batch's pixel items wait for their cloud's point items with a
    bounded poll; run that wait on a count that never reaches zero."""
    from paper_2504_20937_b300.api import Batch
    stored = inputs.encode(inputs.uniform_cloud(3000, 32), "f32")
    desc = dict(n=3000, width=40, height=30, seed=3, cloud=0, amplitude=1e-3)
    with Batch([desc], "f32") as b:
        b.check_device()                                 # clean to start with
        b.selftest_bounded_wait(max_polls=1000)          # ~0.1 ms of polling, the count never reaches zero
        with pytest.raises(MmrError, match="TIMEOUT"):
            b.check_device()
        b.check_device()                                 # the flag was cleared
        b.points(0).copy_(torch.from_numpy(stored))
        b.set_camera(0, 0, (0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
        for _ in range(2):
            b.step_and_render()
        b.check_device()
        keys = b.frame_keys(0).cpu().numpy().reshape(-1).view(np.uint64)
    o = oracle_run(stored, "f32", 40, 30, 3, 1e-3, 2, fixed_eye)
    assert np.array_equal(keys, o[1])


def test_injected_allocation_failures():
    code = """
        import sys; sys.path.insert(0, '.')
        from paper_2504_20937_b300.api import Context, MmrError
        try:
            Context(64, 64)
            print("created")
        except MmrError as e:
            print("refused", e.status, "injected" in str(e))
    """
    r = _run_child(code, {"MMR_FAIL_ALLOC_AFTER": "0"})
    assert r.returncode == 0, r.stderr
    assert "refused -2 True" in r.stdout
    # the context's four set-up allocations pass; the point buffer is refused
    code2 = """
        import sys; sys.path.insert(0, '.')
        from paper_2504_20937_b300.api import Context, MmrError
        ctx = Context(64, 64)
        try:
            ctx.alloc_points(1000, "f32")
            print("allocated")
        except MmrError as e:
            print("refused", e.status, ctx.device_bytes)
        ctx.close()
    """
    r = _run_child(code2, {"MMR_FAIL_ALLOC_AFTER": "4"})
    assert r.returncode == 0, r.stderr
    assert "refused -2" in r.stdout


def test_budget_state_and_argument_errors():
    with Context(64, 64, budget_bytes=64 * 64 * 20 + 4 + 1000) as ctx:
        with pytest.raises(MmrError, match="BUDGET"):
            ctx.alloc_points(1_000_000, "f32")
        with pytest.raises(MmrError, match="STATE"):
            ctx.step_and_render()                         # no points yet
        with pytest.raises(MmrError, match="INVALID"):
            ctx.alloc_points(0, "f32")                    # an empty cloud is refused, nothing allocated
        with pytest.raises(MmrError, match="INVALID"):
            ctx.alloc_points(1 << 32, "f32")              # ids are 32-bit
        ctx.alloc_points(10, "f32")
        with pytest.raises(MmrError, match="STATE"):
            ctx.alloc_points(10, "f32")                   # one point buffer per context
        with pytest.raises(MmrError, match="STATE"):
            ctx.render()                                  # no camera yet
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_camera((0.5, 0.5, 0.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_camera((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 2.0, 1.0)
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_sim(1, 0, 2.0)
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_matrix([float("nan")] * 16, 0.1, 100.0)
        ctx.set_camera((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
        ctx.step_and_render()
        ctx.check_device()
    with pytest.raises(MmrError, match="INVALID"):
        Context(0, 10)


def test_calls_after_close_are_rejected():
    ctx = Context(16, 16)
    ctx.alloc_points(10, "f32")
    ctx.close()
    with pytest.raises(MmrError, match="INVALID"):
        ctx.step_and_render()
    with pytest.raises(MmrError, match="INVALID"):
        ctx.frame_ptrs()
    ctx.close()                                            # closing twice is harmless
