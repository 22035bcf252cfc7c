"""The perspective divide of the point kernels (one shared reciprocal and
Markstein's FMA correction) against CUDA's IEEE division __fdiv_rn on the
GPU.  The kernel's own helper is compiled into a test-only library
(tests/cuda/division_check.cu) with the product's floating-point flags.

Scope of the checks:
- every divisor significand in [1, 2) against 4096 dividend significands
  each (2^35 pairs), both signs; with MMR_DIVISION_EXHAUSTIVE=1 all 2^46
  significand pairs (about five minutes on one B300);
- the hardware reciprocal estimate scales exactly by powers of two over
  divisor exponents -64..64, so the significand result holds over the
  whole allowed clip w range;
- random pairs with divisors over the whole allowed clip w range
  [2^-64, 2^64]: IEEE bit for bit inside the exact band, and giving the same
  pixel outside it.

Camera validation (2^-64 <= znear < zfar <= 2^64) is checked in
tests/test_parity_gpu.py."""
import ctypes as C
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def div():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libdivcheck.so")
    src = os.path.join(HERE, "cuda", "division_check.cu")
    hdr = os.path.join(ROOT, "paper_2504_20937_b300", "csrc", "mmr_device.cuh")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
                        "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", src, "-o", lib], check=True)
    L = C.CDLL(lib)
    L.div_significands.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p]
    L.div_rcp_scaling.argtypes = [C.c_void_p, C.c_void_p]
    L.div_random.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def _first(first):
    return f"a=0x{first[1]:08x} b=0x{first[2]:08x}"


def test_every_divisor_significand(div):
    exhaustive = os.environ.get("MMR_DIVISION_EXHAUSTIVE") == "1"
    count = 1 << 23 if exhaustive else 1 << 12
    bad = C.c_ulonglong(0)
    first = (C.c_uint32 * 3)()
    assert div.div_significands(count, C.byref(bad), first) == 0
    assert bad.value == 0, f"{bad.value} of {count << 23} pairs differ from __fdiv_rn, e.g. {_first(first)}"


def test_reciprocal_estimate_scales_exactly(div):
    bad = C.c_ulonglong(0)
    first = (C.c_uint32 * 3)()
    assert div.div_rcp_scaling(C.byref(bad), first) == 0
    assert bad.value == 0, f"{bad.value} divisors break scaling, e.g. {_first(first)}"


@pytest.mark.parametrize("seed", [1, 2])
def test_random_pairs_over_exponents(div, seed):
    bad = C.c_ulonglong(0)
    exact = C.c_ulonglong(0)
    first = (C.c_uint32 * 3)()
    assert div.div_random(seed, 4096, C.byref(bad), first, C.byref(exact)) == 0
    assert bad.value == 0, f"{bad.value} pairs fail, e.g. {_first(first)}"
    assert exact.value > 100_000_000          # most samples land in the exact band
