// Host check of the integer FP64 -> double-float split (df_split_int in df64.cuh) against
// the definition hi = RN_FP32(x), lo = RN_FP32(x - hi) evaluated with plain C conversions.
// Prints the number of values tried, of values the integer path handled and of mismatches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "df64.cuh"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double from_bits(uint64_t b) {
  double x;
  memcpy(&x, &b, sizeof(x));
  return x;
}
static uint32_t fbits(float f) {
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  return u;
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  long tried = 0, handled = 0, bad = 0;
  auto check = [&](double x) {
    ++tried;
    h1w::df r;
    if (!h1w::df_split_int(x, r)) return;
    ++handled;
    const float hi = static_cast<float>(x);
    const float lo = static_cast<float>(x - static_cast<double>(hi));
    if (fbits(hi) != fbits(r.hi) || fbits(lo) != fbits(r.lo)) {
      if (bad < 5) printf("mismatch x=%a int=(%a,%a) ref=(%a,%a)\n", x, r.hi, r.lo, hi, lo);
      ++bad;
    }
  };
  // random bit patterns with exponents across the handled range and beyond
  for (long i = 0; i < n; ++i) {
    const uint64_t r = next_u64();
    const uint64_t ex = 1023 - 70 + (next_u64() % 210);
    check(from_bits((r & 0x800FFFFFFFFFFFFFull) | (ex << 52)));
  }
  // ties and near-ties of the 24-bit rounding, binade carries, signs
  for (int e = -62; e <= 128; ++e)
    for (uint64_t low : {0ull, 1ull, (1ull << 28) - 1, 1ull << 28, (1ull << 28) + 1, (1ull << 29) - 1})
      for (uint64_t top : {0ull, 1ull, 0x7FFFFFull, 0x7FFFFEull})
        for (int sg = 0; sg < 2; ++sg) {
          const uint64_t b = (uint64_t)sg << 63 | (uint64_t)(e + 1023) << 52 | top << 29 | low;
          check(from_bits(b));
        }
  check(0.0);
  check(-0.0);
  printf("%ld %ld %ld\n", tried, handled, bad);
  return bad ? 1 : 0;
}
