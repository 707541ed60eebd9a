"""Failure paths on the GPU, without faulting it: a bounded device wait that
runs out reports FMT_ETIMEOUT and leaves the context usable; every device
allocation of a fit, made to fail in turn, surfaces as FMT_ENOMEM from the
call that needed it, and the next fit is correct."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def small_fit_matches_oracle(precision):
    from paper_1511_01353_gb300 import fmt as F
    w = W.small()
    T = O.fit(w.x, w.y, w.z, w.f, 4, 3, 64, 1e-4)
    tree = F.fit(F.make_params(4, 3, 64, 1e-4, precision=precision), dev(w.x), dev(w.y), dev(w.z), dev(w.f))
    ex = F.parse_export(F.fmt_tree_export(tree))
    tol = (1e-10 if precision == F.FMT_FP64 else 1e-6) * T.maxabs
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    tree.close()


def test_bounded_wait_times_out_and_the_context_survives():
    from paper_1511_01353_gb300 import fmt as F
    t0 = time.perf_counter()
    with pytest.raises(F.FmtError) as e:
        F.fmt_wait_probe(50_000_000)  # 50 ms on an mbarrier that nothing arrives on
    dt = time.perf_counter() - t0
    assert e.value.status == F.FMT_ETIMEOUT
    assert 0.05 <= dt < 10.0
    small_fit_matches_oracle(F.FMT_FP64)
    small_fit_matches_oracle(F.FMT_MIXED)


@pytest.mark.parametrize("precision", [0, 1])
def test_every_device_allocation_failure_is_reported(precision):
    from paper_1511_01353_gb300 import fmt as F
    w = W.small()
    p = F.make_params(4, 3, 64, 1e-4, precision=precision)
    X = [dev(a) for a in (w.x, w.y, w.z, w.f)]
    failed = 0
    for k in range(1, 200):
        F.fmt_debug_fail_alloc(k)
        try:
            F.fit(p, *X).close()
            done = True
        except F.FmtError as err:
            assert err.status == F.FMT_ENOMEM, err
            done = False
            failed += 1
        finally:
            F.fmt_debug_fail_alloc(0)
        if done:
            break
    assert done and failed >= 5  # every allocation of the fit failed once, then the fit succeeded
    small_fit_matches_oracle(precision)
