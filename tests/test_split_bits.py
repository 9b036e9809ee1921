"""The integer FP64 -> FP32 rounding and hi/lo split of the CUDA path
(csrc/afd_split.cuh), compiled here as plain C and compared bit for bit with
the FP64 conversions it replaces: hi = RN(v), lo = RN(v - hi) with the
subtraction in FP64. Random bit patterns over every exponent, with the low
29 bits forced onto ties, near-ties and carries, plus the edge values."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1907_02290_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#include "afd_split.cuh"

static uint32_t fb(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static double dv(uint64_t u) { double v; memcpy(&v, &u, 8); return v; }

static long bad = 0, checked = 0, in_range = 0;

static void check(uint64_t u) {
  const double v = dv(u);
  float h, l;
  afd_split2(v, &h, &l);
  const float hr = (float)v;
  const float lr = isnan(v) ? hr : (float)(v - (double)hr);
  const float r1 = afd_round_f32(v);
  const int fin = afd_finite_bits(v);
  checked++;
  const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
  if (e >= AFD_SPLIT_EMIN && e < AFD_SPLIT_EMAX) in_range++;
  if (isnan(v)) {
    if (!isnan(h) || !isnan(r1) || fin) bad++;
    return;
  }
  if (fb(h) != fb(hr) || fb(l) != fb(lr) || fb(r1) != fb(hr) || fin != (isfinite(v) != 0)) {
    if (bad < 5)
      fprintf(stderr, "mismatch %016llx: hi %08x/%08x lo %08x/%08x\n", (unsigned long long)u,
              fb(h), fb(hr), fb(l), fb(lr));
    bad++;
  }
}

int main(int argc, char **argv) {
  const long n = atol(argv[1]);
  uint64_t s = 0x9e3779b97f4a7c15ull;
  for (long i = 0; i < n; i++) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    uint64_t u = s;
    if (i & 1) {  /* exponent inside or near the integer range */
      const uint64_t e = 930u + (uint64_t)((s >> 20) % 210u);
      u = (u & ~(0x7ffull << 52)) | (e << 52);
    }
    const uint64_t low = (1ull << 29) - 1ull;
    switch ((i >> 1) & 7) {
      case 1: u = (u & ~low) | (1ull << 28); break;            /* exact tie */
      case 2: u = (u & ~low) | ((1ull << 28) + 1ull); break;   /* just above */
      case 3: u = (u & ~low) | ((1ull << 28) - 1ull); break;   /* just below */
      case 4: u |= ((1ull << 52) - 1ull); break;               /* carry into the exponent */
      case 5: u &= ~low; break;                                /* FP32-exact: lo = 0 */
      case 6: u = (u & ~((1ull << 52) - 1ull)) | (1ull << 29) | (1ull << 28); break; /* odd q, tie */
      default: break;
    }
    check(u);
  }
  /* edge values: zeros, the range's boundaries, FP32 limits, subnormals, inf, nan */
  const uint64_t edges[] = {
      0x0000000000000000ull, 0x8000000000000000ull, 0x0000000000000001ull,
      0x000fffffffffffffull, 0x0010000000000000ull, 0x7fefffffffffffffull,
      0x7ff0000000000000ull, 0xfff0000000000000ull, 0x7ff8000000000000ull,
      (uint64_t)AFD_SPLIT_EMIN << 52, ((uint64_t)AFD_SPLIT_EMIN << 52) - 1ull,
      (uint64_t)AFD_SPLIT_EMAX << 52, ((uint64_t)AFD_SPLIT_EMAX << 52) - 1ull,
      0x47efffffe0000000ull, 0x47efffffefffffffull, 0x47effffff0000000ull,
      0x3810000000000000ull, 0x380fffffffffffffull, 0x36a0000000000000ull,
      0x3ff0000000000000ull, 0xbff0000010000000ull, 0x3ff0000030000000ull};
  for (unsigned k = 0; k < sizeof edges / sizeof edges[0]; k++) {
    check(edges[k]);
    check(edges[k] ^ 0x8000000000000000ull);
  }
  printf("%ld %ld %ld\n", checked, in_range, bad);
  return bad != 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("split")
    src = d / "split_check.c"
    src.write_text(HARNESS)
    exe = d / "split_check"
    # -ffp-contract=off and no fast-math: the reference conversions are the
    # IEEE ones
    subprocess.run([cc, "-O2", "-std=c99", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe), "-lm"], check=True)
    return str(exe)


def test_split_matches_fp64_conversions(harness):
    r = subprocess.run([harness, "4000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    checked, in_range, bad = (int(v) for v in r.stdout.split())
    assert bad == 0
    assert in_range > checked // 3  # the integer path is what is exercised
