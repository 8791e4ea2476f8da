"""The trailing updates one panel at a time (GF2_PAIRS=0) give the same
decomposition as the oracle, with both table sizes of that update (8-bit
tables while more than 4096 rows remain below the panel, 4-bit after).  The library reads the switch when it loads, so
the cases run in a child process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import f2gen, oracle
from tests.gpu_util import assert_same_decomposition, gpu_decompose
cases = [(f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
         (f2gen.uniform(777, 2111, 4), 2111),
         (f2gen.uniform(3000, 500, 5), 500),
         (f2gen.sparse_rows(1000, 1000, 10, 14), 1000)]
X, Y = f2gen.fixed_rank_factors(1024, 1024, 512, 20)
cases.append((oracle.mmm(X, Y, 512, 1024), 1024))
# more than 4096 rows below the panels: the 8-bit-table update of one panel
# (the 4-bit one takes over once fewer rows remain)
cases.append((f2gen.uniform(8192, 8192, f2gen.BASE_SEED, 3), 8192))
cases.append((f2gen.uniform(12000, 1000, 6), 1000))
for A, m in cases:
    assert_same_decomposition(A, m, gpu_decompose(A, m))
print("single-panel updates ok")
"""


def test_single_panel_updates_match_oracle():
    env = dict(os.environ, GF2_PAIRS="0")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "single-panel updates ok" in r.stdout
