// Host check of the library's integer-arithmetic binary64 addition against the
// hardware addition: random pairs over the whole exponent range, near-cancelling
// pairs, subnormals, ties, signed zeros, infinities and NaNs.  Prints mismatches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#define __host__
#define __device__
#define __forceinline__ inline
#include "int_fadd.h"

static uint64_t bits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static double from(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 2000000;
  std::mt19937_64 g(12345);
  long bad = 0, checked = 0;
  auto check = [&](double a, double b) {
    for (int neg = 0; neg < 2; ++neg) {
      const double want = neg ? a - b : a + b;
      const double got = sgb::int_fadd(a, b, neg != 0);
      const bool ok = std::isnan(want) ? std::isnan(got) : bits(want) == bits(got);
      ++checked;
      if (!ok && bad++ < 20)
        std::printf("MISMATCH %.17g %c %.17g: want %.17g (%016llx) got %.17g (%016llx)\n", a, neg ? '-' : '+', b,
                    want, (unsigned long long)bits(want), got, (unsigned long long)bits(got));
    }
  };
  for (long i = 0; i < n; ++i) {
    const uint64_t r1 = g(), r2 = g();
    const int mode = (int)(r1 & 7);
    double a, b;
    if (mode == 0) {  // arbitrary bit patterns
      a = from(r1); b = from(r2);
    } else if (mode == 1) {  // same binade neighbourhood: heavy cancellation
      a = from(r1 & ~0x7ff0000000000000ULL | (uint64_t)(1023 + (int)((r2 >> 60) & 7)) << 52);
      b = from((bits(a) ^ (r2 & 0xfffULL)) ^ (r2 & 0x8000000000000000ULL));
    } else if (mode == 2) {  // subnormals and tiny normals
      a = from(r1 & 0x801fffffffffffffULL);
      b = from(r2 & 0x801fffffffffffffULL);
    } else if (mode == 3) {  // exponent gaps around the 56-bit alignment window
      a = std::ldexp(1.0 + (double)(r1 >> 12) / 4503599627370496.0, (int)(r2 % 200) - 100);
      b = std::ldexp(1.0 + (double)(r2 >> 12) / 4503599627370496.0, (int)(r2 % 200) - 100 - (int)(r1 % 70));
      if (r1 & 1) b = -b;
    } else if (mode == 4) {  // ties: b exactly half an ulp of a, and odd/even mantissas
      a = from((r1 & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL);
      const int gap = 53 + (int)(r2 % 3);
      b = std::ldexp(1.0, -gap + 0) * ((r2 >> 8) & 1 ? 1.0 : -1.0);
    } else if (mode == 5) {  // near overflow
      a = from((r1 & 0x800fffffffffffffULL) | (uint64_t)(2046 - (r2 % 2)) << 52);
      b = from((r2 & 0x800fffffffffffffULL) | (uint64_t)(2046 - (r1 % 3)) << 52);
    } else {  // uniform moderate values, the staging workload
      std::uniform_real_distribution<double> u(-1.0, 1.0);
      a = u(g); b = u(g);
    }
    check(a, b);
  }
  const double special[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 4.9406564584124654e-324,
                            -4.9406564584124654e-324, 2.2250738585072014e-308, 1.7976931348623157e308,
                            -1.7976931348623157e308, 0.5, 1.1102230246251565e-16};
  for (double a : special)
    for (double b : special) check(a, b);
  std::printf("checked %ld mismatches %ld\n", checked, bad);
  return bad != 0;
}
