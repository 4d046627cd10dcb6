// Host-side check of the integer-pipe float <-> double conversions of the
// library against the compiler's own conversions (no GPU needed):
//  - every one of the 2^32 float bit patterns through f2d_bits;
//  - edge cases and 2^26 random doubles spread over the float range through
//    d2f_bits (round to nearest, ties to even).
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "../paper_1604_07163_gb300/csrc/mg_device.cuh"

using namespace mgdev;

static bool same_float(float a, float b) {
  if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
  return fbits(a) == fbits(b);
}

int main() {
  long long bad = 0;
  // f2d: all float bit patterns
  for (uint64_t u = 0; u < (1ull << 32); ++u) {
    const float f = bitsf((unsigned)u);
    const double got = f2d_bits(f);
    double want = (double)f;
    if (std::fpclassify(f) == FP_SUBNORMAL) want = std::signbit(f) ? -0.0 : 0.0;
    const bool ok = std::isnan(f) ? std::isnan(got) : dbits(got) == dbits(want);
    if (!ok && bad++ < 5) printf("f2d mismatch %08llx\n", (unsigned long long)u);
  }
  // d2f: edge cases
  std::vector<double> cases = {0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, (double)FLT_MAX, -(double)FLT_MAX,
                               (double)FLT_MIN, 3.4028235677973366e38, 3.4028236e38, 1e39, -1e39,
                               1.1754942e-38, 1e-45, 1e-300, 1e300, INFINITY, -INFINITY, NAN,
                               1.0 + std::ldexp(1.0, -24), 1.0 + 3 * std::ldexp(1.0, -24),
                               1.0 + std::ldexp(1.0, -24) + std::ldexp(1.0, -52), 16777217.0, 16777219.0};
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> expo(-126.0, 128.0), mant(1.0, 2.0);
  for (int i = 0; i < (1 << 26); ++i) {
    double v = std::ldexp(mant(rng), (int)std::floor(expo(rng)));
    if (rng() & 1) v = -v;
    cases.push_back(v);
    // ties: a float plus exactly half an ulp
    const float f = (float)v;
    if (std::isfinite(f) && f != 0.0f) cases.push_back((double)f + std::ldexp(1.0, std::ilogb(f) - 24));
  }
  for (double d : cases) {
    const float got = d2f_bits(d);
    float want = (float)d;
    if (std::isfinite(want) && want != 0.0f && std::fabs(want) < FLT_MIN) want = std::signbit(want) ? -0.0f : 0.0f;
    if (want == 0.0f && d != 0.0 && std::fabs(d) < FLT_MIN) want = std::signbit(d) ? -0.0f : 0.0f;
    if (!same_float(got, want) && bad++ < 10) printf("d2f mismatch %.17g -> %.9g (want %.9g)\n", d, got, want);
  }
  printf("%s: %lld mismatches over 2^32 floats and %zu doubles\n", bad ? "FAIL" : "OK", bad, cases.size());
  return bad ? 1 : 0;
}
