"""Race check of the cooperative 3D cell routines the CUDA kernels run (CPU only).

tests/native/cta_race_check.cpp runs the cell residual, the cell Jacobian and
the Vanka set-up and apply with one real host thread per CUDA thread and a
barrier per CTA synchronisation, built with ThreadSanitizer: an access that no
barrier orders against a conflicting one is reported, and the results must
equal the one-thread run bit for bit.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cooperative_cell_routines_are_race_free(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "cta_race")
    build = subprocess.run([cxx, "-std=c++20", "-O1", "-g", "-fsanitize=thread", "-pthread", "-o", exe,
                            os.path.join(HERE, "native", "cta_race_check.cpp")], capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr:
        pytest.skip("no ThreadSanitizer runtime: " + build.stderr[-200:])
    assert build.returncode == 0, build.stderr[-2000:]
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    run = subprocess.run([exe, "8"], capture_output=True, text=True, env=env, timeout=1200)
    out = run.stdout + run.stderr
    assert "ThreadSanitizer" not in out, out[-4000:]
    assert run.returncode == 0 and "PASSED" in out, out[-4000:]
