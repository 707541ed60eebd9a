"""Several host threads driving the library at once, each on its own stream.

The kernels whose dynamic shared memory depends on the degree (tile QR,
merges, back substitution; the mixed path's Gram, factor and updates) are
launched from every thread.  The limit a launch needs belongs to the kernel,
not to the launch, so no thread may lower it between another thread's
setting and its launch (the serving engine's worker slots do exactly this).
Two threads fit trees of a low and a high degree a dozen times each: every
call succeeds, and every tree is bitwise the tree the same inputs give when
fitted alone.
"""
import threading

import numpy as np
import pytest

from paper_1511_01353_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROUNDS = 12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("precision,degrees", [(0, (4, 10)), (1, (5, 10))])
def test_two_threads_fitting_different_degrees(precision, degrees):
    from paper_1511_01353_gb300 import fmt as F
    F.load()
    cases = []
    for i, p in enumerate(degrees):
        w = W.small(n=12000, seed=W.SEED_BASE + 300 + i)
        params = F.make_params(p, 4, 0, 1e-6, precision=precision)
        cases.append((params, [dev(getattr(w, k)) for k in "xyzf"]))
    torch.cuda.synchronize()
    alone = []
    for params, arrs in cases:
        t = F.fit(params, *arrs)
        alone.append(F.fmt_tree_export(t))
        t.close()
    results = [[] for _ in cases]
    errors = []

    def worker(i):
        params, arrs = cases[i]
        s = torch.cuda.Stream()
        try:
            for _ in range(ROUNDS):
                t = F.fit(params, *arrs, stream=s)
                results[i].append(F.fmt_tree_export(t))
                t.close()
        except Exception as e:  # reported below, in the test's thread
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for i in range(len(cases)):
        assert len(results[i]) == ROUNDS
        assert all(r == alone[i] for r in results[i])
