// Checks the integer FP32 <-> FP64 conversions of the CUDA library's looper
// update against the host's IEEE conversions: widen() on every 32-bit
// pattern, narrow() on random doubles over the whole exponent range and on
// constructed rounding ties and range edges.  Prints the number of
// mismatches and exits non-zero on any.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "tpc_fp64.cuh"

static uint64_t dbits64(double d) {
  uint64_t b;
  std::memcpy(&b, &d, 8);
  return b;
}
static double from64(uint64_t b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}
static uint32_t fbits32(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

static bool same_f(float a, float b) {
  return (std::isnan(a) && std::isnan(b)) || fbits32(a) == fbits32(b);
}

int main() {
  long bad = 0, n = 0;
  // widen: all 2^32 float bit patterns
  for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
    const float f = tpc::bitsf((uint32_t)u);
    const double a = tpc::widen(f), b = (double)f;
    const bool ok = (std::isnan(a) && std::isnan(b)) || dbits64(a) == dbits64(b);
    if (!ok && bad++ < 5) std::printf("widen mismatch at 0x%08llx\n", (unsigned long long)u);
    ++n;
  }
  // narrow: random doubles (xorshift64*), exponents over the whole range
  uint64_t s = 0x9e3779b97f4a7c15ull;
  for (long i = 0; i < 200000000; ++i) {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    const uint64_t r = s * 0x2545f4914f6cdd1dull;
    // bias half of the draws to the float range and its edges
    uint64_t b = r;
    if (i & 1) {
      const uint64_t e = 860 + (r >> 52) % 330;  // 860..1189
      b = (r & 0x800fffffffffffffull) | (e << 52);
    }
    const double d = from64(b);
    const float a = tpc::narrow(d), c = (float)d;
    if (!same_f(a, c) && bad++ < 5) std::printf("narrow mismatch at 0x%016llx\n", (unsigned long long)b);
    ++n;
  }
  // narrow: exact ties and neighbours of ties, every exponent of the float range
  for (uint64_t e = 890; e <= 1160; ++e)
    for (uint64_t m23 = 0; m23 < (1u << 23); m23 += 4097)
      for (int sign = 0; sign < 2; ++sign)
        for (int delta = -2; delta <= 2; ++delta) {
          const uint64_t mant = (m23 << 29) | (1ull << 28);
          const uint64_t b = ((uint64_t)sign << 63) | (e << 52) | (mant + (int64_t)delta);
          const double d = from64(b);
          const float a = tpc::narrow(d), c = (float)d;
          if (!same_f(a, c) && bad++ < 5)
            std::printf("narrow tie mismatch at 0x%016llx\n", (unsigned long long)b);
          ++n;
        }
  // largest float, overflow threshold, smallest normal
  const double edges[] = {3.4028234663852886e38, 3.4028235677973366e38, 3.4028235677973362e38,
                          1.1754943508222875e-38, 1.1754942807573643e-38, 0.0, -0.0, 1.0, -1.0};
  for (double d : edges) {
    if (!same_f(tpc::narrow(d), (float)d) && bad++ < 10) std::printf("narrow edge mismatch %.17g\n", d);
    ++n;
  }
  std::printf("checked %ld conversions, %ld mismatches\n", n, bad);
  return bad ? 1 : 0;
}
