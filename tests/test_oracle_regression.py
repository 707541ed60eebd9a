"""The oracle reproduces its committed regression record bitwise
(tests/golden/oracle_regression_small.txt, written by the script beside it).
A change to the oracle's arithmetic fails here until the record is rewritten
in a commit that names the passage of the paper, or the reading, behind it."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SCRIPT = os.path.join(HERE, "golden", "make_oracle_regression.py")


def test_oracle_matches_its_regression_record():
    spec = importlib.util.spec_from_file_location("make_oracle_regression", SCRIPT)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(mod.OUT) as fh:
        want = fh.read()
    got = mod.record()
    assert got == want, "the oracle's output changed; see " + os.path.relpath(SCRIPT, os.path.dirname(HERE))
