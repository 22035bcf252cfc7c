"""Host logic of the batched frame: the work list the persistent CTAs take
their items from (paper_2504_20937_b300/csrc/mmr_worklist.h), compiled with the
host C++ compiler and checked on 3,000 random batches.  Its ordering is what
makes a pixel item's bounded wait always end: every cloud's pixel items come
after all of its point items."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_batch_work_list_invariants():
    out_dir = os.path.join(HERE, "_build")            # git-ignored, beside the tests
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, f"worklist_check_{os.getpid()}")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2504_20937_b300", "csrc"),
                    os.path.join(HERE, "cpp", "worklist_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    finally:
        os.remove(exe)
    assert r.returncode == 0 and r.stdout.startswith("ok 3000"), r.stdout + r.stderr
