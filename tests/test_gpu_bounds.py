"""Memory safety without compute-sanitizer: the bounds-checked build.

The library built with -DLBM_BOUNDS_CHECK checks every global access to a
state buffer (single elements against the lattice's nodes, bulk row copies
against the buffer's slot of the allocation) and reports an access out of
range as LBM_ECUDA instead of making it. tests/bounds_cases.py drives every
kernel variant over ragged and degenerate sizes with that build (a child
process, since a process loads one build of the library).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_kernel_stays_inside_its_buffers():
    from paper_1904_02471_gb300 import build
    lib = build.build(bounds=True)
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "bounds-checked runs ok" in r.stdout
