// Host check of the integer bf16 split (split.cuh): split3_bits against the
// FP64 split3 on random values over a wide exponent range, on constructed
// round-to-nearest ties in each plane and on special values.  Prints the
// number of mismatching planes; exit status 1 if any.
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_2203_13283_gb300/csrc/split.cuh"

using namespace wcs;

static long long bad = 0, total = 0;

static void check(double x) {
  for (int planes = 1; planes <= 3; ++planes) {
    uint16_t a[3] = {1, 1, 1}, b[3] = {1, 1, 1};
    split3(x, planes, &a[0], &a[1], &a[2]);
    split3_bits(x, planes, &b[0], &b[1], &b[2]);
    for (int p = 0; p < planes; ++p)
      if (a[p] != b[p]) {
        if (bad < 10) printf("mismatch x=%a planes=%d plane %d: %04x vs %04x\n", x, planes, p, a[p], b[p]);
        ++bad;
      }
  }
  ++total;
}

int main(int argc, char** argv) {
  const long long n = argc > 1 ? atoll(argv[1]) : 2000000;
  std::mt19937_64 g(20221213);
  std::uniform_real_distribution<double> U(1.0, 2.0);
  std::uniform_int_distribution<int> E(-90, 115);   // across both ends of the window 2^-74 .. 2^100
  for (long long i = 0; i < n; ++i) {
    double x = std::ldexp(U(g), E(g));
    check((g() & 1) ? -x : x);
  }
  // ties: 8 leading bits, then exactly half an ulp of plane 0, 1 or 2
  for (long long i = 0; i < n / 4; ++i) {
    uint64_t M = (128 + g() % 128) << 45;
    const int kind = (int)(g() % 4);
    if (kind == 0) {
      M |= 1ull << 44;
    } else {
      const int s1 = 20 + (int)(g() % 17);
      M = (M | ((g() & 1) ? (1ull << 44) : 0)) & ~((1ull << 44) - 1);
      M |= (128 + g() % 128) << s1;
      if (kind == 2) M |= 1ull << (s1 - 1);
      if (kind == 3) {
        const int s2 = (int)(g() % (s1 - 9));
        M |= ((128 + g() % 128) << s2) | (s2 ? (1ull << (s2 - 1)) : 0);
      }
    }
    const double x = std::ldexp((double)M, -52 + (int)(g() % 60) - 30);
    check((g() & 1) ? -x : x);
  }
  const double special[] = {0.0, -0.0, 1.0, -1.0, std::ldexp(1.0, -74), std::ldexp(1.0, -75), std::ldexp(1.0, 100),
                            std::ldexp(1.999, 99), INFINITY, -INFINITY, NAN, 5e-324, 1e-310, 3.3e38,
                            1.0 + std::ldexp(1.0, -8), 1.0 + std::ldexp(1.0, -8) + std::ldexp(1.0, -40), 255.5, 511.0,
                            1.0 - std::ldexp(1.0, -9)};
  for (double x : special) check(x);
  printf("checked %lld values, mismatching planes %lld\n", total, bad);
  return bad ? 1 : 0;
}
