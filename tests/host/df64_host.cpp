// Host build of the device double-float header, for its unit test only.
//
// The header's building blocks use the CUDA float intrinsics __fadd_rn,
// __fsub_rn, __fmul_rn, __fmaf_rn (each an IEEE-754 binary32 operation with
// round-to-nearest-even, the fused multiply-add with one rounding), __frcp_rn
// and __fdiv_rn (correctly rounded reciprocal and quotient) and bit casts.
// Here they are the host's own IEEE binary32 operations (compile with
// -ffp-contract=off so that no expression is fused behind our back).  The
// program draws seeded inputs (splitmix64), applies one operation and prints
// the bit patterns of inputs and outputs; tests/test_df64_host.py checks them
// with exact rational arithmetic.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#define __device__
#define __forceinline__ inline

static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __frcp_rn(float a) { return 1.0f / a; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}
static inline long long __double_as_longlong(double d) {
  long long l;
  std::memcpy(&l, &d, 8);
  return l;
}
static inline float __uint2float_rn(unsigned u) { return (float)u; }

#include "df64.cuh"

using ehl::df;

static uint64_t g_state = 0;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double uniform01() { return (double)(next_u64() >> 11) * 0x1.0p-53; }
// a double with a random 52-bit significand, random sign and exponent in [e_lo, e_hi]
static double random_double(int e_lo, int e_hi) {
  const uint64_t m = next_u64() & ((1ull << 52) - 1);
  const int e = e_lo + (int)(next_u64() % (uint64_t)(e_hi - e_lo + 1));
  const uint64_t s = next_u64() & 1ull;
  const uint64_t bits = (s << 63) | ((uint64_t)(e + 1023) << 52) | m;
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}
static unsigned fb(float f) { return __float_as_uint(f); }
static unsigned long long dbits(double d) { return (unsigned long long)__double_as_longlong(d); }
static df rdf(int e_lo, int e_hi) { return ehl::df_from_double(random_double(e_lo, e_hi)); }
static void pdf(df x) { std::printf(" %08x %08x", fb(x.hi), fb(x.lo)); }

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const char* op = argv[1];
  const int n = std::atoi(argv[2]);
  g_state = std::strtoull(argv[3], nullptr, 10);
  for (int k = 0; k < n; ++k) {
    if (!std::strcmp(op, "from_double") || !std::strcmp(op, "from_double_sel")) {
      double d;
      const int kind = k % 8;
      if (kind < 5) {
        d = random_double(-74, 127);  // the fast window
      } else if (kind == 5) {
        d = random_double(-1022, 1023);  // anywhere in the float64 range
      } else if (kind == 6) {
        d = random_double(-140, -60);  // around the flush-to-zero edge
      } else {
        const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1.0, -1.0, 0x1.fffffffffffffp+127,
                             0x1p+128, 0x1p-100, 0x1.fffffffffffffp-101, 4.9e-324, 0x1p-74, 0x1.fffffffp-75};
        d = sp[(k / 8) % (int)(sizeof(sp) / sizeof(sp[0]))];
      }
      const df r = std::strcmp(op, "from_double") ? ehl::df_from_double_sel(d) : ehl::df_from_double(d);
      std::printf("%016llx", dbits(d));
      pdf(r);
      std::printf("\n");
    } else if (!std::strcmp(op, "add") || !std::strcmp(op, "mul") || !std::strcmp(op, "div")) {
      const df x = rdf(-30, 30), y = rdf(-30, 30);
      const df r = !std::strcmp(op, "add") ? ehl::df_add(x, y) : !std::strcmp(op, "mul") ? ehl::df_mul(x, y)
                                                                                        : ehl::df_div(x, y);
      pdf(x);
      pdf(y);
      pdf(r);
      std::printf("\n");
    } else if (!std::strcmp(op, "rcp")) {
      const df y = rdf(-60, 60);
      pdf(y);
      pdf(ehl::df_rcp(y));
      std::printf("\n");
    } else if (!std::strcmp(op, "sub_two_prods")) {
      const df z = rdf(-10, 10), a = rdf(-5, 5), b = rdf(-5, 5), c = rdf(-5, 5), d = rdf(-5, 5);
      pdf(z);
      pdf(a);
      pdf(b);
      pdf(c);
      pdf(d);
      pdf(ehl::df_sub_two_prods(z, a, b, c, d));
      std::printf("\n");
    } else if (!std::strcmp(op, "mul_floats")) {  // lo = 0 on both sides, away from underflow: exact
      const df x = ehl::make_df((float)random_double(-40, 40), 0.f);
      const df y = ehl::make_df((float)random_double(-40, 40), 0.f);
      pdf(x);
      pdf(y);
      pdf(ehl::df_mul(x, y));
      std::printf("\n");
    } else if (!std::strcmp(op, "mul_f")) {
      const df x = rdf(-30, 30);
      const float y = (float)random_double(-30, 30);
      pdf(x);
      std::printf(" %08x", fb(y));
      pdf(ehl::df_mul_f(x, y));
      std::printf("\n");
    } else {
      return 2;
    }
  }
  (void)uniform01;
  return 0;
}
