"""The oracle's plain-C deposit loop under AddressSanitizer and UndefinedBehaviorSanitizer
(host-side code only): a small driver built with -fsanitize=address,undefined runs
every kernel, with and without the half-cell shift, on particles that include the box
faces, points a rounding step below the far face, and points outside the box (indices
wrap).  Any sanitizer report aborts the test program; its mesh must equal the numpy deposit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.assignment import ORDER, _deposit

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "oracle", "c", "deposit.c")

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
void oracle_deposit(const float *x, const float *y, const float *z, const double *w, int64_t n,
                    const double *box_min, double H, int N, int kind, double shift, double *mesh);
static void *slurp(const char *path, size_t bytes) {
  FILE *f = fopen(path, "rb");
  if (!f) exit(3);
  void *p = malloc(bytes);
  if (!p || fread(p, 1, bytes, f) != bytes) exit(4);
  fclose(f);
  return p;
}
int main(int argc, char **argv) {
  /* argv: dir n N kind shift box_min[3] H */
  const char *dir = argv[1];
  const int64_t n = atoll(argv[2]);
  const int N = atoi(argv[3]), kind = atoi(argv[4]);
  const double shift = atof(argv[5]);
  const double bm[3] = {atof(argv[6]), atof(argv[7]), atof(argv[8])};
  const double H = atof(argv[9]);
  char path[4096];
  snprintf(path, sizeof path, "%s/x.bin", dir); float *x = slurp(path, sizeof(float) * n);
  snprintf(path, sizeof path, "%s/y.bin", dir); float *y = slurp(path, sizeof(float) * n);
  snprintf(path, sizeof path, "%s/z.bin", dir); float *z = slurp(path, sizeof(float) * n);
  snprintf(path, sizeof path, "%s/w.bin", dir); double *w = slurp(path, sizeof(double) * n);
  double *mesh = calloc((size_t)N * N * N, sizeof(double));
  oracle_deposit(x, y, z, w, n, bm, H, N, kind, shift, mesh);
  snprintf(path, sizeof path, "%s/mesh.bin", dir);
  FILE *f = fopen(path, "wb");
  fwrite(mesh, sizeof(double), (size_t)N * N * N, f);
  fclose(f);
  free(x); free(y); free(z); free(w); free(mesh);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("asan")
    (d / "driver.c").write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run(["gcc", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        str(d / "driver.c"), SRC, "-o", str(exe), "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer build unavailable: " + r.stderr[-200:])
    return str(exe)


def _particles(n_mesh, box_min, L):
    gal, _, _ = synth.poisson_cube(3000, 1, side=L, center=tuple(b + 0.5 * L for b in box_min), seed=17)
    pos = gal.positions().astype(np.float32)
    lo = np.asarray(box_min, dtype=np.float32)
    hi = np.nextafter(lo + np.float32(L), np.float32(-np.inf)).astype(np.float32)
    extra = np.array([lo, hi, [lo[0], hi[1], lo[2]], lo - np.float32(0.3 * L), hi + np.float32(1.7 * L),
                      lo + np.float32(L / n_mesh) * np.float32(3.0)], dtype=np.float32)
    pos = np.concatenate([pos, extra])
    w = np.linspace(-0.4, 1.3, pos.shape[0])
    return pos, w


@pytest.mark.parametrize("kind", ["ngp", "cic", "tsc"])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_c_deposit_is_clean_under_sanitizers(driver, tmp_path, kind, shift):
    n, box_min, L = 16, (-37.25, 12.5, 100.0), 64.0
    pos, w = _particles(n, box_min, L)
    for i, name in enumerate("xyz"):
        np.ascontiguousarray(pos[:, i]).tofile(tmp_path / f"{name}.bin")
    w.astype(np.float64).tofile(tmp_path / "w.bin")
    H = L / n
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([driver, str(tmp_path), str(pos.shape[0]), str(n), str(ORDER[kind]), repr(shift),
                        *(repr(b) for b in box_min), repr(H)], capture_output=True, text=True, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.fromfile(tmp_path / "mesh.bin", dtype=np.float64)
    want = np.zeros(n ** 3)
    _deposit(want, pos, w, box_min, H, n, kind, shift)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
