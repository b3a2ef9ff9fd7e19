"""The bounds-checked build of the library (lib/libiblbm_checked.so, the same
sources compiled with -DIBLBM_BOUNDS_CHECK: every computed index of the
time-step kernels range-checked, a violation counted and its access skipped,
never a trap) run on tiny lattices through every kernel path of a time step:
lattice-only steps on 4..16 cells per side (vectorised, two-cell and
one-cell collides, three precisions), a capsule with each stencil and with
records, deterministic spreading and the staged collide, a dense pair of
capsules (four nodes per warp, per-cell velocity pass), a batch and a slab
group.  Every case must count no fault and match the FP64 oracle.  The cases
run in a child process that loads the checked build (tests/bounds_cases.py)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_faults_and_oracle_parity():
    env = dict(os.environ, IBLBM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env, cwd=HERE,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    rows = [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]
    assert len(rows) >= 25, r.stdout
    for row in rows:
        assert row["faults"] == 0, row
        assert row["err"] < row["tol"], row
