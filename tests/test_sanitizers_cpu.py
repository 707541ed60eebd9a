"""Host-side sanitizer runs (CPU only): AddressSanitizer and
UndefinedBehaviorSanitizer builds of the oracle and of libfmt's host code.

* The oracle's pins run against an ASan/UBSan build of oracle/fmt_oracle.c.
* A C driver runs the oracle through its entry points in all three modes and
  down its error paths (rank truncation, root degree clamp, NaN input), with
  LeakSanitizer on: every allocation must be freed.
* The host-side ABI tests (argument validation, layouts, the tree importer
  on truncated and corrupt blobs, the serving engine's checks) run against
  an ASan/UBSan build of libfmt (device code unchanged).

Each sanitized library is loaded in a child process with the ASan runtime
preloaded (FMT_ORACLE_LIB, FMT_LIBRARY); any report aborts the child.
"""
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=all"]


def _asan_runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True, check=True)
    except (OSError, subprocess.CalledProcessError):
        return None
    path = p.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


ASAN = _asan_runtime()
pytestmark = pytest.mark.skipif(ASAN is None, reason="no AddressSanitizer runtime for gcc")


def _pytest_child(env_extra, *tests):
    env = dict(os.environ, LD_PRELOAD=ASAN, ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0",
               UBSAN_OPTIONS="print_stacktrace=1", OMP_NUM_THREADS="2", **env_extra)
    cmd = [sys.executable, "-m", "pytest", *[os.path.join(ROOT, "tests", t) for t in tests], "-q",
           "-p", "no:cacheprovider"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, (p.stdout + p.stderr)[-4000:]


def test_oracle_pins_under_asan_ubsan(tmp_path):
    lib = str(tmp_path / "liboracle_san.so")
    O.compile_library(os.path.join(ROOT, "oracle", "fmt_oracle.c"), lib, extra=["-g", *SAN])
    rc, out = _pytest_child({"FMT_ORACLE_LIB": lib}, "test_oracle_pins.py")
    assert rc == 0, out


DRIVER = r"""
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
typedef struct ora_tree ora_tree;
int ora_fit(int, int, int, double, const double *, double, int64_t, const double *, const double *,
            const double *, const double *, int, ora_tree **);
int ora_eval(const ora_tree *, int64_t, const double *, const double *, const double *, double *, int64_t *);
void ora_free(ora_tree *);
static uint64_t s = 88172645463325252ull;
static double rnd(void) { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return (double)(s >> 11) * 0x1.0p-53; }
static int run(int64_t n, int deg, int mode, int plane, int expect) {
  double *x = malloc(8 * n), *y = malloc(8 * n), *z = malloc(8 * n), *f = malloc(8 * n), out[64];
  for (int64_t i = 0; i < n; ++i) {
    x[i] = rnd(); y[i] = rnd(); z[i] = plane ? 0.25 : rnd();
    f[i] = sin(3 * x[i]) * y[i] + z[i] * z[i];
  }
  if (expect) f[n / 2] = NAN;
  const double lo[3] = {0, 0, 0};
  ora_tree *T = 0;
  int rc = ora_fit(deg, 3, 10, 1e-6, lo, 1.0, n, x, y, z, f, mode, &T);
  if (rc == 0) {
    int64_t no = 0;
    rc = ora_eval(T, n < 64 ? n : 64, x, y, z, out, &no);
    ora_free(T);
  }
  free(x); free(y); free(z); free(f);
  return rc == expect ? 0 : 1;
}
int main(void) {
  int bad = 0;
  for (int mode = 0; mode < 3; ++mode)
    for (int deg = 0; deg <= 4; deg += 2) bad += run(6000, deg, mode, 0, 0);  /* omp tasks above 2048 points */
  bad += run(1500, 3, 0, 1, 0);   /* coplanar: rank truncation */
  bad += run(12, 4, 2, 0, 0);     /* fewer points than monomials: root degree clamp */
  bad += run(500, 2, 1, 0, 1);    /* NaN value: EINVAL, nothing allocated survives */
  return bad;
}
"""


def test_oracle_frees_everything(tmp_path):
    src = tmp_path / "driver.c"
    src.write_text(DRIVER)
    exe = str(tmp_path / "driver")
    subprocess.run(["gcc", "-std=c11", "-O1", "-g", *SAN, "-fopenmp", "-ffp-contract=off", "-o", exe,
                    os.path.join(ROOT, "oracle", "fmt_oracle.c"), str(src), "-lm"], check=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", OMP_NUM_THREADS="4")
    p = subprocess.run([exe], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-4000:]


def test_library_host_code_under_asan_ubsan(tmp_path):
    from paper_1511_01353_gb300 import build as B
    lib = B.compile_library(str(tmp_path / "libfmt_san.so"), str(tmp_path / "obj"), host_flags=["-g", *SAN])
    rc, out = _pytest_child({"FMT_LIBRARY": lib}, "test_abi.py", "test_serve_cpu.py")
    assert rc == 0, out
