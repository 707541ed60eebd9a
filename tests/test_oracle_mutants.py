"""Mutation test of the oracle's pins (CPU only).

Each mutant plants one plausible mistake in a temporary copy of
oracle/fmt_oracle.c: a dropped term, a wrong sign or index, a transposed
operand, a wrong frame, a wrong refinement decision.  The copy is compiled
into a temporary library.  tests/test_oracle_pins.py then runs against it in
a child process (FMT_ORACLE_LIB), and at least one pin must fail.  An
unmutated copy must pass the same pins, so the harness itself is checked.
The committed oracle is never modified.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fmt_oracle.c")

# name -> (mistake, [(text, replacement, occurrences)])
MUTANTS = {
    "nmono_count": ("rank of the basis off (Sec. 2 stride l3_{p+1})",
                    [("(p + 1) * (p + 2) * (p + 3) / 6", "(p + 1) * (p + 2) * (p + 4) / 6", 1)]),
    "dropped_factorial": ("1/n! dropped from the geometric moments (Alg. 2)",
                          [("(ora_factorial(l) * ora_factorial(m) * ora_factorial(n))",
                            "(ora_factorial(l) * ora_factorial(m))", 1)]),
    "transposed_exponents": ("exponents of u and w exchanged",
                             [("ora_ipow(u, l) * ora_ipow(v, m) * ora_ipow(w, n)",
                               "ora_ipow(u, n) * ora_ipow(v, m) * ora_ipow(w, l)", 1)]),
    "quantise_rounds": ("quantisation rounds instead of truncating",
                        [("return (uint32_t)floor(t);", "return (uint32_t)floor(t + 0.5);", 1)]),
    "quantise_upper_face": ("upper face of the root cube not clamped into the last cell",
                            [("if (t >= 2097152.0) return ORA_QMAX;", "if (t > 2097152.0) return ORA_QMAX;", 1)]),
    "frame_corner": ("node frame centred on the box corner, not its centre (Sec. 4)",
                     [("(double)(2u * i + 1u) * h", "(double)(2u * i) * h", 1)]),
    "frame_scale": ("node frame maps the box onto [-1/2,1/2]^3, not [-1,1]^3 (Sec. 4)",
                    [("*s = 1.0 / h;", "*s = 0.5 / h;", 1)]),
    "norm_drops_term": ("first entry below the diagonal dropped from the column norm",
                        [("for (int64_t i = j + 1; i < n; ++i) xn2 += aj[i] * aj[i];",
                          "for (int64_t i = j + 2; i < n; ++i) xn2 += aj[i] * aj[i];", 1)]),
    "reflector_beta_sign": ("beta = +sign(alpha)*||x||: the cancelling Householder sign",
                            [("double beta = (alpha >= 0.0) ? -h : h;", "double beta = (alpha >= 0.0) ? h : -h;", 1)]),
    "reflector_tau_sign": ("wrong sign of the reflector scalar tau",
                           [("tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;", 1)]),
    "update_without_tau": ("tau dropped from the trailing-column update",
                           [("      w *= tau[j];\n      ak[j] -= w;", "      ak[j] -= w;", 1)]),
    "qt_skips_last": ("last reflector not applied to the right-hand side",
                      [("double *y) {\n  for (int j = 0; j < L; ++j) {",
                        "double *y) {\n  for (int j = 0; j < L - 1; ++j) {", 1)]),
    "q_instead_of_qt": ("reflectors applied in reverse order (Q y instead of Q^T y)",
                        [("for (int j = 0; j < L; ++j) {\n    if (tau[j] == 0.0) continue;",
                          "for (int j = L - 1; j >= 0; --j) {\n    if (tau[j] == 0.0) continue;", 1)]),
    "backsub_transposed": ("back substitution reads R transposed",
                           [("s -= A[(int64_t)k * ld + j] * F[k];", "s -= A[(int64_t)j * ld + k] * F[k];", 1)]),
    "rank_rule_off": ("no rank truncation: near-zero pivots divided through",
                      [("double thresh = 64.0 * (double)L * DBL_EPSILON * rmax;", "double thresh = 0.0;", 1)]),
    "rank_keep_index": ("kept coefficients written to the wrong columns",
                        [("F[keep[i]] = Fk[i];", "F[i] = Fk[i];", 1)]),
    "residual_sign": ("residual update adds Lambda F (Alg. 2 residual sign)",
                      [("    r[i] -= s;", "    r[i] += s;", 1)]),
    "octant_bits_yz": ("y and z bits exchanged in every octant code",
                       [("(((C->qy[g] >> shift) & 1u) << 1) |\n                    (((C->qz[g] >> shift) & 1u) << 2)",
                         "(((C->qz[g] >> shift) & 1u) << 1) |\n                    (((C->qy[g] >> shift) & 1u) << 2)", 2),
                        ("(((qy >> shift) & 1u) << 1) | (((qz >> shift) & 1u) << 2)",
                         "(((qz >> shift) & 1u) << 1) | (((qy >> shift) & 1u) << 2)", 1)]),
    "child_box_index": ("child box index takes the z bit of the octant for y",
                        [("ch.iy = 2u * nd.iy + (uint32_t)((o >> 1) & 1);",
                          "ch.iy = 2u * nd.iy + (uint32_t)((o >> 2) & 1);", 2)]),
    "rms_without_mean": ("E_RMS without the division by the octant's point count (Alg. 1)",
                         [("sqrt(S[o] / (double)child_count[o])", "sqrt(S[o])", 1)]),
    "refine_ge_tau": ("child refined when E = tau, not only when E > tau",
                      [("E > T->tau) nd->refine_mask", "E >= T->tau) nd->refine_mask", 1)]),
    "min_pts_ignores_rank": ("a child with fewer points than monomials is refined",
                             [("int64_t nmin = T->min_pts > T->nmono ? T->min_pts : T->nmono;",
                               "int64_t nmin = T->min_pts;", 1)]),
    "depth_limit_off_by_one": ("the deepest level D_max is never created",
                               [("(nd->depth + 1 <= T->max_depth)", "(nd->depth + 1 < T->max_depth)", 1)]),
    "root_clamp_off_by_one": ("root degree clamped one lower than the points allow",
                              [("while (ora_nmono(q + 1) <= n) ++q;", "while (ora_nmono(q + 1) < n) ++q;", 1)]),
    "tau_without_abs": ("tau from max f instead of max |f|",
                        [("double a = fabs(f[i]);", "double a = f[i];", 1)]),
    "eval_root_only": ("evaluation stops after the root",
                       [("      node = nd->child[o];", "      node = -1;", 1)]),
    "eval_frame_swapped": ("evaluation puts y and z of the target in each other's frame",
                           [("(x - cx) * sx, (y - cy) * sy, (z - cz) * sz", "(x - cx) * sx, (z - cz) * sz, (y - cy) * sy",
                             1)]),
}


def _mutate(text, edits):
    for old, new, count in edits:
        assert text.count(old) == count, (old, text.count(old))
        text = text.replace(old, new)
    return text


def _run_pins(lib_path):
    env = dict(os.environ, FMT_ORACLE_LIB=lib_path, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
           "-p", "no:cacheprovider"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    return p.returncode, p.stdout[-2000:]


def _build_and_run(tmp, name, text):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, "lib" + name + ".so")
    with open(src, "w") as fh:
        fh.write(text)
    O.compile_library(src, lib)
    return _run_pins(lib)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(SRC) as fh:
        original = fh.read()
    jobs = {"unmutated": original}
    for name, (_, edits) in MUTANTS.items():
        jobs[name] = _mutate(original, edits)
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {name: ex.submit(_build_and_run, str(tmp_path), name, text) for name, text in jobs.items()}
        res = {name: f.result() for name, f in futs.items()}
    rc, out = res.pop("unmutated")
    assert rc == 0, "the pins fail on an unmutated copy:\n" + out
    # pytest exit code 1: some test failed (an assertion or an exception in the
    # oracle binding), not a harness error (2-4) or a crash (negative)
    survivors = {name: (MUTANTS[name][0], rc) for name, (rc, _) in res.items() if rc != 1}
    assert not survivors, survivors


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_text_is_present(name):
    # each planted edit still matches the oracle source (guards against drift)
    with open(SRC) as fh:
        _mutate(fh.read(), MUTANTS[name][1])
