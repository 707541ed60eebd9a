"""The bounds-checked build (-DFMT_CHECKED) on the GPU.

Every kernel of the checked build tests the indices it reads from device
memory (work items, nodes, problems, rows, scratch slots) against the sizes of
the buffers they address before it accesses memory through them; a failed
test skips the guarded work and the ABI call returns FMT_EINTERNAL naming the
site.  Nothing here faults the GPU: every planted index stays inside the
arrays it addresses, so an access that a test did not guard would still land
in bounds.

* The mechanism: fmt_check_probe writes inside a 64-element array in both
  builds; the checked build reports i >= n and clears its record.
* A real kernel's test: a work item's rows moved across the boundary of its
  node (still inside the point arrays) are reported by the first kernels of
  the fit that read them -- the tile QR on the FP64 path, the mixed path's
  per-item kernels on the mixed one -- and the next fit is correct.
* No false reports: the parity, mixed-precision, forest, metamorphic and
  allocation-free tests pass against the checked library.

The checked library is built here and loaded in a child process
(FMT_LIBRARY names it); the tests marked `inner` run only there.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = os.environ.get("FMT_CHECKED_CHILD") == "1"
inner = pytest.mark.skipif(not CHILD, reason="runs in the child process that loads the checked library")
outer = pytest.mark.skipif(CHILD, reason="runs in the parent process")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _child(*args, timeout=1500):
    from paper_1511_01353_gb300 import build as B
    lib = B.build_checked()
    env = dict(os.environ, FMT_LIBRARY=lib, FMT_CHECKED_CHILD="1")
    cmd = [sys.executable, "-m", "pytest", *args, "-m", "gpu", "-q", "-p", "no:cacheprovider"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    return p.returncode, (p.stdout + p.stderr)[-6000:]


@outer
def test_default_build_compiles_the_checks_out():
    from paper_1511_01353_gb300 import fmt as F
    assert not F.fmt_checked_build()
    F.fmt_check_probe(40, 32)  # nothing tests i against n; the write lands inside the array
    for i, n in ((64, 8), (-1, 8), (3, 33), (3, -1)):
        with pytest.raises(F.FmtError) as e:
            F.fmt_check_probe(i, n)
        assert e.value.status == F.FMT_EINVAL


@outer
def test_checked_build_reports_planted_indices():
    rc, out = _child(os.path.join("tests", "test_gpu_checked.py"))
    assert rc == 0, out
    assert "4 passed" in out, out  # every inner test ran


@outer
def test_checked_build_reports_nothing_on_valid_work():
    tests = ["test_gpu_parity.py", "test_gpu_mixed.py", "test_gpu_batch.py", "test_gpu_metamorphic.py",
             "test_zz_no_alloc.py"]
    rc, out = _child(*[os.path.join("tests", t) for t in tests])
    assert rc == 0, out
    assert " passed" in out and "failed" not in out, out


@inner
def test_inner_library_is_the_checked_build():
    from paper_1511_01353_gb300 import fmt as F
    assert F.fmt_checked_build()


@inner
def test_inner_probe_reports_and_clears():
    from paper_1511_01353_gb300 import fmt as F
    F.fmt_check_probe(3, 8)
    for i, n in ((40, 32), (0, 0), (8, 8)):
        with pytest.raises(F.FmtError) as e:
            F.fmt_check_probe(i, n)
        assert e.value.status == F.FMT_EINTERNAL
        assert "fmt_check_probe" in str(e.value)
        F.fmt_check_probe(7, 8)  # the record was cleared


@inner
@pytest.mark.parametrize("precision,site", [(0, "tile QR (k_tile_qr)"), (1, "mixed path per item")])
def test_inner_rows_across_a_node_are_reported(precision, site):
    # Two problems of 3000 points: the roots cover rows [0, 3000) and
    # [3000, 6000).  Item 0 (the first problem's) gets rows [2999, 3001):
    # inside the point arrays, outside its node.
    from paper_1511_01353_gb300 import fmt as F
    n0 = 3000
    w0, w1 = W.small(n=n0), W.small(n=n0, seed=W.SEED_BASE + 77)
    x, y, z, f = (np.concatenate([getattr(w0, k), getattr(w1, k)]) for k in "xyzf")
    p = F.make_params(4, 3, 64, 1e-4, precision=precision)
    tree = F.oct_build_batch(p, [0, n0, 2 * n0], dev(x), dev(y), dev(z), dev(f))
    F.fmt_debug_item_rows(tree, 0, 0, n0 - 1, n0 + 1)
    with pytest.raises(F.FmtError) as e:
        F.fit_level(tree, 0)
    assert e.value.status == F.FMT_EINTERNAL
    assert site in str(e.value), str(e.value)
    tree.close()
    # the records were read and cleared: the next fit reports nothing and is right
    T = O.fit(w0.x, w0.y, w0.z, w0.f, 4, 3, 64, 1e-4)
    t2 = F.fit(F.make_params(4, 3, 64, 1e-4, precision=precision), dev(w0.x), dev(w0.y), dev(w0.z), dev(w0.f))
    ex = F.parse_export(F.fmt_tree_export(t2))
    tol = (1e-10 if precision == 0 else 1e-6) * T.maxabs
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    t2.close()
