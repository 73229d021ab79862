"""The benchmark and the build entry compile (a syntax error there would only
show on the GPU machine, where they run)."""
import os
import py_compile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_and_entry_compile(tmp_path):
    for f in ("bench.py", "__graft_entry__.py"):
        py_compile.compile(os.path.join(ROOT, f), cfile=str(tmp_path / (f + "c")), doraise=True)


def test_bench_arguments_parse():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "--steps" in r.stdout and "--impl" in r.stdout
