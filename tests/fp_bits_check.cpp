// Host check of the integer-pipe float conversions in csrc/fp_bits.cuh
// against the host compiler's own IEEE 754 conversions: every binary32 bit
// pattern is widened; binary64 operands of every kind (random bit patterns,
// every binary32 binade and the ones around it, exact ties of both parities,
// the overflow and underflow edges) are narrowed.  Prints "ok" or the first
// mismatch.
#include <cstdio>
#include <cstdint>
#include <cstring>

#include "fp_bits.cuh"

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static bool check_narrow(uint64_t b) {
  const double x = crn::fpb_double(b);
  const float want = (float)x;
  const float got = crn::narrow_f64(x);
  if (crn::fpb_bits32(want) != crn::fpb_bits32(got)) {
    std::printf("narrow mismatch: x bits %016llx want %08x got %08x\n", (unsigned long long)b,
                crn::fpb_bits32(want), crn::fpb_bits32(got));
    return false;
  }
  return true;
}

int main() {
  // widening: all 2^32 binary32 patterns
  for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
    const float x = crn::fpb_float((uint32_t)u);
    const double want = (double)x;
    const double got = crn::widen_f32(x);
    if (crn::fpb_bits64(want) != crn::fpb_bits64(got)) {
      std::printf("widen mismatch: x bits %08x\n", (unsigned)u);
      return 1;
    }
  }
  long n = 0;
  // random bit patterns
  for (int t = 0; t < 20000000; ++t, ++n)
    if (!check_narrow(next())) return 1;
  // every exponent from below the subnormal binary32 range to above overflow,
  // random significands, both signs
  for (uint64_t e = 860; e <= 1160; ++e)
    for (int t = 0; t < 200000; ++t, ++n) {
      const uint64_t r = next();
      if (!check_narrow((r & 0x8000000000000000ull) | (e << 52) | (r & 0xfffffffffffffull))) return 1;
    }
  // dropped 29 bits at, just below and just above one half, kept part odd
  // and even, across all binary32 binades
  const uint64_t tails[] = {0x10000000u, 0x0fffffffu, 0x10000001u, 0u, 1u, 0x1fffffffu};
  for (uint64_t e = 895; e <= 1151; ++e)
    for (uint64_t tail : tails)
      for (int t = 0; t < 2000; ++t, ++n) {
        const uint64_t r = next();
        const uint64_t kept = (r >> 11) & 0x7fffffull;
        for (uint64_t s = 0; s < 2; ++s)
          if (!check_narrow((s << 63) | (e << 52) | (kept << 29) | tail)) return 1;
      }
  // all-ones kept significand: the rounding carry crosses into the next
  // binade, and out of the largest one to infinity
  for (uint64_t e = 895; e <= 1151; ++e)
    for (uint64_t tail : tails)
      if (!check_narrow((e << 52) | (0x7fffffull << 29) | tail)) return 1;
  std::printf("ok widen=4294967296 narrow=%ld\n", n);
  return 0;
}
