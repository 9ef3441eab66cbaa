"""The FP64 HMF stages' sine and cosine (csrc/sincos_fp64.cuh), compiled for the host and
checked on the CPU against long-double libm sin and cos.

The header writes every floating-point step as an explicitly rounded operation (no
contraction), so its host build computes what the GPU computes.  Pinned here:
* |sin - sinl| and |cos - cosl| stay below one unit of 2^-52 (an FP64 result within a unit
  in the last place of 1) for angles spread over up to +-(2^20 - tiny), at the table points
  k pi/2048, half way between them (the largest |r|) and next to those, at tiny and
  subnormal angles, and on both sides of 2^20 (beyond it the libm fallback);
* the bit moves it uses: int -> double and float -> double exact, double -> float rounded
  to nearest, over random samples against the C casts.
A table index off by one (|r| up to 3 pi/4096) or a dropped or wrong Taylor term leaves
errors of several units of 2^-52 and fails the bound."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1212_0262_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstdint>
#include "sincos_fp64.cuh"

static double2 tab[sc64::kTabN];
static uint64_t st = 0x9e3779b97f4a7c15ull;
static double urand() { st = st * 6364136223846793005ull + 1442695040888963407ull; return (double)(st >> 11) * 0x1p-53; }
static double worst = 0.0;
static void one(double th) {
  double s, c;
  sc64::sincos_tab(th, tab, &s, &c);
  const long double S = sinl((long double)th), C = cosl((long double)th);
  const double e = fmax((double)fabsl((long double)s - S), (double)fabsl((long double)c - C)) / 0x1p-52;
  if (!(e <= worst)) worst = e;
}
int main(int argc, char **argv) {
  const long n = atol(argv[1]);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < sc64::kTabN; k++) {
    const long double x = (long double)k * pi / 2048.0L;
    tab[k] = make_double2((double)sinl(x), (double)cosl(x));
  }
  const double spans[] = {1e-3, 1.0, 100.0, 1e4, 1e6, 0x1p20 * 0.9999999, 0x1p21};
  for (double sp : spans)
    for (long i = 0; i < n; i++) one((2 * urand() - 1) * sp);
  const double h = 0x1.921fb54442d18p-10;
  for (long k = -6000; k < 6000; k++) {
    for (long kk : {k, 667000000L + k, -667000000L - k}) {
      one(kk * h);
      const double m = (kk + 0.5) * h;
      one(m);
      one(nextafter(m, 1e30));
      one(nextafter(m, -1e30));
    }
  }
  const double pts[] = {0.0, -0.0, 5e-324, -5e-324, 2.2e-308, 1e-300, 1e-40, 0x1p-74, 0x1p-75, 1e-10, 7.669e-4};
  for (double t : pts) { one(t); one(-t); }
  for (int e = -1074; e < 22; e++) { one(ldexp(1.0, e)); one(-ldexp(1.7, e)); one(nextafter(ldexp(1.0, e), 0.0)); }
  long bad = 0;
  for (int i = 0; i < 2000000; i++) {
    const int v = (int)(urand() * 2147483647.0) * ((i & 1) ? -1 : 1);
    if (sc64::i2d(v) != (double)v) bad++;
    const double d = (2 * urand() - 1) * ldexp(1.0, (int)(urand() * 250) - 125);
    if (fabs(d) >= 0x1p-126 && sc64::d2f_rn(d) != (float)d) bad++;
    const float f = (float)d;
    if (fabs(f) >= 0x1p-126f && sc64::f2d(f) != (double)f) bad++;
  }
  printf("%.6f %ld\n", worst, bad);
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_fp64_table_sincos_within_one_unit_of_libm(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "sc.cu"
    src.write_text(SRC)
    exe = tmp_path / "sc"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-Xcompiler", "-ffp-contract=off", "-o", str(exe),
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe), "150000"], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    worst, bad = out.stdout.split()
    assert bad == "0"
    assert float(worst) < 1.0, worst
