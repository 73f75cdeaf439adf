"""Host check of the Jacobi eigensolver's pair schedules: the schedule header
of the GPU library, compiled with g++, must give rounds that cover every
index once and sweeps that rotate every pair once (round-robin order, n up
to 300)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_jacobi_schedules_cover_every_pair_once(tmp_path):
    exe = tmp_path / "sched_check"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I" + os.path.join(ROOT, "paper_1408_5092_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "cpp", "sched_check.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
    assert int(out.stdout.split()[1]) == 47
