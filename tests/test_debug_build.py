"""The debug build (-DSTENCIL_DEBUG): every store of a sweep's result checks
that it lands on an interior point of the padded array and records (never
traps on) the first one that does not.  CPU: it compiles, links and exports
every function the header declares.  GPU (test_gpu_debug_build.py): a set of
sweeps of every kernel family records no bad store."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_compiles_and_exports_every_symbol():
    from paper_1410_3060_gb300 import build, stencil
    path = build.build(debug=True)
    assert path != build.LIB and os.path.exists(path)
    code = ("import test_abi, paper_1410_3060_gb300.stencil as st; L = st.lib(); "
            "assert st.library_path().endswith('_build_debug/libstencil.so'); "
            "missing = [n for n in test_abi.declared_functions() if not hasattr(L, n)]; "
            "assert not missing, missing; print('ok')")
    env = dict(os.environ, STENCIL_LIBRARY=path, PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]
    assert stencil.EXPORTED.count("stencil_debug_bad_store") == 1
