// Host check of the integer-ALU conversions of step_math.cuh: f32_rn(x)
// against the C conversion (float)x, which rounds to nearest, ties to even
// (IEEE 754), and f64_of(f) against (double)f, bit for bit.  Inputs: random
// bit patterns of every class, doubles whose exponents straddle FP32's range
// with the 29 dropped fraction bits at, just below and just above the
// rounding tie, and the special values.  Exit status 0 when all agree.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "step_math.cuh"

using csph::f32_rn;
using csph::f64_of;

static uint64_t g_state = 0x243f6a8885a308d3ull;
static uint64_t next_bits() {   // splitmix64
  uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static long g_bad32 = 0, g_bad64 = 0, g_n = 0;

static void check32(double x) {
  const float a = f32_rn(x), b = (float)x;
  uint32_t ua, ub;
  memcpy(&ua, &a, 4);
  memcpy(&ub, &b, 4);
  ++g_n;
  if (ua != ub && !(std::isnan(a) && std::isnan(b))) {
    if (g_bad32 < 8) printf("f32_rn(%a) = %a, (float) gives %a\n", x, a, b);
    ++g_bad32;
  }
}

static void check64(float f) {
  const double a = f64_of(f), b = (double)f;
  uint64_t ua, ub;
  memcpy(&ua, &a, 8);
  memcpy(&ub, &b, 8);
  if (ua != ub && !(std::isnan(a) && std::isnan(b))) {
    if (g_bad64 < 8) printf("f64_of(%a) = %a, (double) gives %a\n", f, a, b);
    ++g_bad64;
  }
}

int main(int argc, char** argv) {
  const long iters = argc > 1 ? atol(argv[1]) : 2000000;
  for (long i = 0; i < iters; ++i) {
    uint64_t r = next_bits();
    double x;
    memcpy(&x, &r, 8);
    check32(x);
    const uint64_t e = 850 + next_bits() % 350;                  // exponents 2^-173 .. 2^176
    uint64_t m = next_bits() & 0xfffffffffffffull;
    switch (next_bits() % 4) {
      case 0: m = (m & ~0x1fffffffull) | 0x10000000ull; break;    // exactly half an FP32 ulp
      case 1: m = (m & ~0x1fffffffull) | 0x0fffffffull; break;    // just below
      case 2: m = (m & ~0x1fffffffull) | 0x10000001ull; break;    // just above
      default: break;
    }
    const uint64_t bb = ((next_bits() & 1ull) << 63) | (e << 52) | m;
    memcpy(&x, &bb, 8);
    check32(x);
    const uint32_t fr = (uint32_t)next_bits();
    float f;
    memcpy(&f, &fr, 4);
    check64(f);
  }
  const double sd[] = {0.0, -0.0, 1.0, -1.0, DBL_MIN, DBL_MAX, FLT_MIN, -FLT_MIN, FLT_MAX, -FLT_MAX,
                       0x1.fffffefffffffp127, 0x1.ffffffp127, 0x1.fffffe8p127, INFINITY, -INFINITY, NAN,
                       0x1p-126, 0x1.fffffffffffffp-127, 0x1p-149, 0x1p-150, 0x1.8p-150, 1e-300, -1e300};
  for (double v : sd) check32(v);
  const float sf[] = {0.f, -0.f, FLT_MIN, -FLT_MIN, FLT_MAX, -FLT_MAX, 0x1p-149f, 0x1.fffffcp-127f,
                      INFINITY, -INFINITY, NAN, 1.f, -3.5f};
  for (float v : sf) check64(v);
  printf("f32_rn: %ld mismatches in %ld; f64_of: %ld mismatches\n", g_bad32, g_n, g_bad64);
  return (g_bad32 || g_bad64) ? 1 : 0;
}
