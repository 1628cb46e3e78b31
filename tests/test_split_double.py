"""The integer conversions between FP64 and double-float of the FP32 path (csrc/df64.cuh) against
the FP64 definitions they replace: split_double, hi = fl32(x), lo = fl32(x - hi), and
df_to_double, fl64((double)hi + (double)lo), both rounding to nearest even.

Both are __host__ __device__ functions: a small host program built with nvcc from the same
header runs them on about a million inputs each and counts the bit differences.  Splits:
random magnitudes across the float range and past both ends of the integer fast path, both
signs, halfway cases that round to even either way, significands that carry into the
exponent, exact floats.  Sums: renormalised and lazy (hi, lo) pairs of both signs, low parts
from just below hi's last bit down to far below double precision, halfway cases, hi a power of
two with a low part of the other sign (the sum drops a binade), carries into the next binade.
Runs on the CPU; needs nvcc."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1907_01724_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include "df64.cuh"
static int sums(const char* path)
{
  FILE* f = fopen(path, "rb");
  std::vector<float> v;
  float t;
  while (fread(&t, sizeof(t), 1, f) == 1) v.push_back(t);
  fclose(f);
  long bad = 0, fast = 0;
  for (size_t k = 0; k + 1 < v.size(); k += 2) {
    hsma::df x;
    x.hi = v[k];
    x.lo = v[k + 1];
    const double a = hsma::df_to_double(x), b = (double)x.hi + (double)x.lo;
    uint64_t ba, bb;
    memcpy(&ba, &a, 8); memcpy(&bb, &b, 8);
    uint32_t hb, lb;
    memcpy(&hb, &x.hi, 4); memcpy(&lb, &x.lo, 4);
    const int eh = (hb >> 23) & 0xFF, el = (lb >> 23) & 0xFF;
    if (eh >= 1 && eh <= 254 && ((lb & 0x7FFFFFFFu) == 0 || (el >= 1 && el <= eh - 2))) ++fast;
    if (ba != bb) {
      if (bad < 5) printf("mismatch hi=%.9g lo=%.9g %016llx/%016llx\n", x.hi, x.lo, (unsigned long long)ba,
                          (unsigned long long)bb);
      ++bad;
    }
  }
  printf("%ld %ld %zu\n", bad, fast, v.size() / 2);
  return 0;
}

int main(int argc, char** argv)
{
  if (argc > 2) return sums(argv[2]);
  FILE* f = fopen(argv[1], "rb");
  std::vector<double> x;
  double v;
  while (fread(&v, sizeof(v), 1, f) == 1) x.push_back(v);
  fclose(f);
  long bad = 0, fast = 0;
  for (double d : x) {
    float hi, lo;
    hsma::split_double(d, hi, lo);
    const float h0 = (float)d;
    const float l0 = (float)(d - (double)h0);
    uint32_t a, b, c, e;
    memcpy(&a, &hi, 4); memcpy(&b, &h0, 4); memcpy(&c, &lo, 4); memcpy(&e, &l0, 4);
    uint64_t bits;
    memcpy(&bits, &d, 8);
    const int E = (int)((bits >> 52) & 0x7FF) - 1023;
    if (E >= -74 && E <= 126) ++fast;
    if (a != b || c != e) {
      if (bad < 5) printf("mismatch x=%.17g hi %08x/%08x lo %08x/%08x\n", d, a, b, c, e);
      ++bad;
    }
  }
  printf("%ld %ld %zu\n", bad, fast, x.size());
  return 0;
}
"""


def _values(rng):
    n = 200000
    out = []
    # random significands and exponents across (and past) the fast-path range, both signs
    e = rng.integers(-90, 135, n)
    out.append(rng.uniform(1.0, 2.0, n) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], n))
    # halfway cases: a float plus half an ulp of it (rounds to even), and just either side
    f = rng.uniform(0.5, 1.0, n).astype(np.float32).astype(np.float64) * np.ldexp(1.0, rng.integers(-70, 120, n))
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    out += [f + 0.5 * ulp, f + 0.5 * ulp * (1 + 2.0 ** -40), f + 0.5 * ulp * (1 - 2.0 ** -40), -(f + 0.5 * ulp)]
    # exact floats (lo = 0) and significands of all ones in the first 24 bits (carry on rounding up)
    out.append(f)
    out.append(np.ldexp(2.0 - 2.0 ** -23 + rng.uniform(0.5, 1.0, n) * 2.0 ** -24, rng.integers(-74, 127, n)))
    # the boundaries of the fast path and values used by the library (unit charges, zero)
    edge = [0.0, -0.0, 1.0, -1.0, 1e-13, -2e-13, 2.0 ** -74, 2.0 ** -75, 2.0 ** 126, 2.0 ** 127 * 1.5,
            np.nextafter(2.0 ** -74, 0), 1e-300, 5e-324]
    out.append(np.array(edge))
    return np.concatenate(out)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("split")
    src = d / "split.cu"
    src.write_text(HARNESS)
    exe = d / "split"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return exe, d


def test_split_double_matches_fp64_rounding(harness):
    exe, d = harness
    x = _values(np.random.default_rng(20240611))
    path = d / "x.bin"
    x.astype(np.float64).tofile(path)
    out = subprocess.run([str(exe), str(path)], check=True, capture_output=True, text=True).stdout.split("\n")
    bad, fast, total = (int(t) for t in out[-2].split())
    assert total == x.size
    assert fast > 0.8 * total  # most values take the integer path
    assert bad == 0, "\n".join(out[:-2])


def _pairs(rng):
    n = 150000
    out = []
    e = rng.integers(-100, 120, n)
    hi = (rng.uniform(1.0, 2.0, n) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    sgn = rng.choice([-1.0, 1.0], n)
    # renormalised and lazy low parts, and low parts far below double precision
    for scale in (rng.uniform(0.0, 0.5, n), rng.uniform(0.0, 2.0, n), rng.uniform(0, 1, n) * 2.0 ** -30,
                  np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-60, -2, n))):
        out.append(np.stack([hi, (sgn * scale * ulp).astype(np.float32)], 1))
    # halfway cases of the double sum: lo = (odd or even) * 2^-53 ulp_double(hi) exactly
    h2 = np.ldexp(rng.integers(2 ** 23, 2 ** 24, n).astype(np.float64), rng.integers(-60, 60, n)).astype(np.float32)
    half = np.abs(h2.astype(np.float64)) * 2.0 ** -53
    out.append(np.stack([h2, (sgn * half).astype(np.float32)], 1))
    out.append(np.stack([h2, (sgn * half * 3).astype(np.float32)], 1))
    # hi a power of two, lo of the other sign: the sum drops a binade
    p2 = np.ldexp(1.0, rng.integers(-60, 60, n)).astype(np.float32)
    out.append(np.stack([p2, (-rng.uniform(0.0, 2.0, n) * np.spacing(p2).astype(np.float64) / 2).astype(np.float32)], 1))
    # carries: hi with an all-ones significand
    c = np.ldexp(2.0 - 2.0 ** -23, rng.integers(-60, 60, n)).astype(np.float32)
    out.append(np.stack([c, (rng.uniform(0.0, 1.0, n) * np.spacing(c).astype(np.float64)).astype(np.float32)], 1))
    edge = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1e-30], [1e-40, 1e-45], [3e38, 1e31], [1.0, 1.0], [1.0, -0.75]],
                    dtype=np.float32)
    out.append(edge)
    return np.concatenate(out).astype(np.float32)


def test_df_to_double_matches_fp64_sum(harness):
    exe, d = harness
    x = _pairs(np.random.default_rng(77))
    path = d / "p.bin"
    x.astype(np.float32).tofile(path)
    out = subprocess.run([str(exe), "-", str(path)], check=True, capture_output=True, text=True).stdout.split("\n")
    bad, fast, total = (int(t) for t in out[-2].split())
    assert total == x.shape[0]
    assert fast > 0.8 * total
    assert bad == 0, "\n".join(out[:-2])
