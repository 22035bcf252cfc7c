"""Pins of the CPU oracle against NVIDIA's own device code, run on the GPU:
cuRAND's Philox4x32-10 on a million random counters and keys, and CUDA's
round-to-nearest binary16 / bfloat16 conversions on every binary32 value.
The CUDA side is a test-only library (tests/cuda/nvidia_refs.cu)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def refs():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libnvrefs.so")
    src = os.path.join(HERE, "cuda", "nvidia_refs.cu")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        "-Xcompiler", "-fPIC", "-shared", src, "-o", lib], check=True)
    L = C.CDLL(lib)
    L.nvref_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.nvref_narrow.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]
    return L


def test_philox_matches_curand(refs):
    n = 1 << 20
    rng = np.random.default_rng(123)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 2, 0], [2**32 - 1] * 4]
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    do = torch.empty_like(dc)
    torch.cuda.synchronize()
    assert refs.nvref_philox(dc.data_ptr(), dk.data_ptr(), do.data_ptr(), n) == 0
    got = do.cpu().numpy().view(np.uint32)
    want = oracle.philox4x32_10_many(ctr, key)
    assert np.array_equal(got, want)


def test_narrowing_matches_cuda_on_every_float(refs):
    chunk = 1 << 28
    f16 = torch.empty(chunk, dtype=torch.int16, device="cuda")
    bf16 = torch.empty(chunk, dtype=torch.int16, device="cuda")
    for start in range(0, 1 << 32, chunk):
        assert refs.nvref_narrow(start, chunk, f16.data_ptr(), bf16.data_ptr()) == 0
        x = (np.arange(chunk, dtype=np.uint32) + np.uint32(start)).view(np.float32)
        nan = np.isnan(x)
        for dev, to in ((f16, oracle.f32_to_f16), (bf16, oracle.f32_to_bf16)):
            got = dev.cpu().numpy().view(np.uint16)
            want = to(x)
            bad = (got != want) & ~nan
            assert not bad.any(), f"mismatch at {np.nonzero(bad)[0][:3] + start}"
