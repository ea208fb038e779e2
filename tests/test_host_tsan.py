"""ThreadSanitizer run of the host finite-element build (csrc/fem.cpp).

The device setup builds the coarsest level on a host thread of its own while
the main thread drives the shared worker pool through level 0, and both
threads call the per-level callbacks.  tests/host_build_tsan.cpp builds
2D Taylor-Hood P4, Scott-Vogelius P4 on the Alfeld split and 3D Taylor-Hood
P3 hierarchies with those options and with the host-only ones; the test
compiles it with -fsanitize=thread and requires a run without a report, and
the same digests with 1 and 8 worker threads."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tsan_binary(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("tsan") / "host_build_tsan")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-pthread",
           os.path.join(ROOT, "tests", "host_build_tsan.cpp"),
           os.path.join(ROOT, "paper_2407_07253_gb300", "csrc", "fem.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    if r.returncode != 0 and "sanitize" in r.stderr and "tsan" in r.stderr.lower():
        pytest.skip("ThreadSanitizer runtime not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-3000:]
    return out


def _run(binary, threads):
    env = dict(os.environ, STOKES_HOST_THREADS=str(threads),
               TSAN_OPTIONS="halt_on_error=1 exitcode=66 report_signal_unsafe=0")
    r = subprocess.run([binary], env=env, capture_output=True, text=True, timeout=900)
    assert "ThreadSanitizer" not in r.stderr, r.stderr[-4000:]
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    return r.stdout.split("\n")


def test_host_build_has_no_data_race(tsan_binary):
    many = _run(tsan_binary, 8)
    one = _run(tsan_binary, 1)
    assert len([x for x in many if x]) == 6
    assert many == one
