"""GPU tests of the bounds-checked debug build (libgaussianpile_check.so,
-DGP_CHECK), the stand-in for a memory sanitizer: its check machinery reports
a failed check (one failed on purpose in a kernel that touches no memory), and
the parity tests of the slice, voxelizer, view and batch paths, including the
random sweep of ragged sizes, pass through it with no index out of range."""
import os
import subprocess
import sys

import pytest

from paper_2603_20611_b300 import binding as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _env():
    return dict(os.environ, GP_LIBRARY="check", PYTHONPATH=ROOT)


def test_default_build_has_no_checks():
    ctx = B.Context(0)
    assert B.lib.gp_check_enabled() == 0
    assert B.lib.gp_check_selftest(ctx.h, None) == B.GP_ERR_STATE
    assert b"not a bounds-checked build" in B.lib.gp_last_error(ctx.h)


def test_checked_build_reports_a_failed_check():
    code = ("from paper_2603_20611_b300 import binding as B\n"
            "ctx = B.Context(0)\n"
            "assert B.lib.gp_check_enabled() == 1\n"
            "st = B.lib.gp_check_selftest(ctx.h, None)\n"
            "msg = B.lib.gp_last_error(ctx.h).decode()\n"
            "assert st == B.GP_ERR_STATE and 'site 99, index 5' in msg, (st, msg)\n"
            "assert B.lib.gp_check_selftest(ctx.h, None) == B.GP_ERR_STATE  # the word was cleared and set again\n"
            "print('ok')\n")
    p = subprocess.run([sys.executable, "-c", code], env=_env(), cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout + p.stderr


def test_parity_suites_pass_under_bounds_checks():
    files = ["tests/test_gpu_slice.py", "tests/test_gpu_sweep.py", "tests/test_gpu_voxel.py", "tests/test_gpu_view.py",
             "tests/test_gpu_batch.py", "tests/test_gpu_rowfact.py"]
    p = subprocess.run([sys.executable, "-m", "pytest", *files, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       env=_env(), cwd=ROOT, capture_output=True, text=True, timeout=3000)
    assert p.returncode == 0, p.stdout[-4000:] + p.stderr[-2000:]
