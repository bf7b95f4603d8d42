// Host test of pair_to_double (csrc/pair2d.cuh): the double built from a double-float pair by
// integer operations must equal, bit for bit, the correctly rounded h 2^sc + l 2^sc.  For a
// normalized pair (|l| <= ulp(h) / 2), pair_to_double_fast must give the same double or, at an
// exact tie, the other of the two nearest doubles.
#include <cmath>
#include <cstdio>
#include <random>

#include "pair2d.cuh"

static long fails = 0, checked = 0, fast_checked = 0, fast_fails = 0, fast_ties = 0;
static long split_checked = 0, split_fast = 0, split_fails = 0;

// double_to_pair_fast against the conversions: h = (float)x, l = (float)(x - h), bit for bit,
// whenever it takes the fast path
static void check_split(double x) {
  float h, l;
  ++split_checked;
  if (!odmd::double_to_pair_fast(x, h, l)) return;
  ++split_fast;
  const float wh = (float)x;
  const float wl = (float)(x - (double)wh);
  if (std::memcmp(&h, &wh, 4) != 0 || std::memcmp(&l, &wl, 4) != 0) {
    if (split_fails < 10) std::printf("split: x=%a got (%a, %a) want (%a, %a)\n", x, h, l, wh, wl);
    ++split_fails;
  }
}

// a tie: h + l lies exactly halfway between want and its neighbour `other`
static bool is_tie(float h, float l, double want, double other) {
  // h - want is exact (want lies within an ulp of h), and so is adding l to it here
  const double rest = ((double)h - want) + (double)l;
  return rest != 0.0 && 2.0 * rest == other - want;
}

static void check_fast(float h, float l, int sc) {
  int e;
  std::frexp(h, &e);
  if (h != 0.f && std::fabs((double)l) > std::ldexp(1.0, e - 25)) return;  // not normalized
  const double want = std::ldexp((double)h + (double)l, sc);
  const double got = odmd::pair_to_double_fast(h, l, sc);
  ++fast_checked;
  if (std::memcmp(&got, &want, 8) == 0) return;
  const double want0 = (double)h + (double)l;
  const double got0 = std::ldexp(got, -sc);
  if ((got0 == std::nextafter(want0, INFINITY) || got0 == std::nextafter(want0, -INFINITY)) &&
      is_tie(h, l, want0, got0)) {
    ++fast_ties;
    return;
  }
  if (fast_fails < 10) std::printf("fast: h=%a l=%a sc=%d got %a want %a\n", h, l, sc, got, want);
  ++fast_fails;
}

static void check(float h, float l, int sc) {
  const double want = std::ldexp((double)h + (double)l, sc);  // one rounding, then exact scaling
  const double got = odmd::pair_to_double(h, l, sc);
  ++checked;
  check_fast(h, l, sc);
  if (std::memcmp(&got, &want, 8) != 0) {
    if (fails < 10) std::printf("h=%a l=%a sc=%d got %a want %a\n", h, l, sc, got, want);
    ++fails;
  }
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-60, 60), scd(-300, 300), gap(24, 90);
  for (int i = 0; i < 2000000; ++i) {
    // a normalized pair from a double: h = fl(x), l = fl(x - h)
    const double x = std::ldexp(u(rng), ex(rng));
    const float h = (float)x;
    const float l = (float)(x - (double)h);
    check(h, l, scd(rng));
    // a low word far below the high word's last bit (the rounded and sticky paths)
    const float h2 = (float)std::ldexp(u(rng), ex(rng));
    if (h2 != 0.f) {
      int e;
      std::frexp(h2, &e);
      const float l2 = (float)std::ldexp(u(rng), e - gap(rng));
      check(h2, l2, scd(rng));
    }
  }
  // ties to even, borrows at a power of two, zeros
  const float hs[] = {1.0f, -1.0f, 1.5f, 0.75f, 3.0f, -2.0f, 1.0f + 0x1p-23f};
  for (float h : hs) {
    int e;
    std::frexp(h, &e);
    for (int k = 24; k <= 40; ++k)
      for (float sgn : {1.f, -1.f}) {
        const float l = sgn * (float)std::ldexp(1.0, e - 1 - k);
        if (std::fabs(l) <= std::ldexp(1.0, e - 25)) check(h, l, 0);
        check(h, sgn * (float)std::ldexp(1.0 + 0x1p-23, e - 1 - k), 7);
      }
  }
  check(0.f, 0.f, 5);
  check(-0.f, 0.f, 5);
  // doubles to pairs: random significands over the float range, ties of the high word (the
  // low 29 bits exactly half), carries into the next binade, and values whose low word would
  // be subnormal (slow path)
  std::uniform_int_distribution<int> exd(-140, 140);
  std::uniform_int_distribution<uint64_t> bits52(0, (1ull << 52) - 1);
  for (int i = 0; i < 2000000; ++i) {
    check_split(std::ldexp(u(rng), exd(rng)));
    const uint64_t mb = (bits52(rng) & ~((1ull << 29) - 1)) | (1ull << 28);  // a tie for h
    const double t = std::ldexp(1.0 + std::ldexp((double)mb, -52), exd(rng));
    check_split(i & 1 ? t : -t);
  }
  for (int e = -120; e <= 120; e += 7) {
    check_split(std::ldexp(2.0 - 0x1p-52, e));  // rounds up to the next power of two
    check_split(-std::ldexp(1.0 + 0x1p-52, e));
    check_split(std::ldexp(1.0, e));
  }
  check_split(0.0);
  std::printf("%ld checked, %ld mismatches\n", checked, fails);
  std::printf("fast: %ld checked, %ld ties rounded the other way, %ld failures\n", fast_checked, fast_ties,
              fast_fails);
  std::printf("split: %ld checked, %ld on the fast path, %ld failures\n", split_checked, split_fast, split_fails);
  return fails == 0 && fast_fails == 0 && split_fails == 0 && split_fast > split_checked / 2 ? 0 : 1;
}
