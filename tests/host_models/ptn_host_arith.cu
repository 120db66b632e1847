// Host build of the bit-field FP32 <-> FP64 conversions that the kernels' FP64 solves use
// (ptn_common.cuh, __host__ __device__), checked against the host's IEEE-754 conversions.
// Mode "F": every FP32 bit pattern widened to FP64.  Mode "D <n> <seed>": n FP64 values
// rounded to FP32 (normal-range values across all exponents, exact ties and their
// neighbours, values near the overflow threshold, infinities, NaNs).  Prints the number
// of mismatches and the number of values checked; the documented exceptions (FP32
// subnormals to signed zeros; NaNs compared as NaNs) are checked as such.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ptn_common.cuh"

using namespace ptn;

static uint64_t bits_of(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static double of_bits(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static float f_of(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static unsigned fbits(float f) { unsigned u; memcpy(&u, &f, 4); return u; }

static uint64_t state;
static uint64_t next() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static void check_d2f(double d, unsigned long long& bad) {
  const uint64_t u = bits_of(d);
  const unsigned got = f64_bits_to_f32_bits((unsigned)(u >> 32), (unsigned)u);
  const float g = f_of(got);
  bool ok;
  if (std::isnan(d)) ok = std::isnan(g);
  else if (std::fabs(d) < 0x1p-126) ok = (got & 0x7fffffffu) == 0u && (got >> 31) == (unsigned)(u >> 63);
  else ok = got == fbits((float)d);
  if (!ok && bad < 5) fprintf(stderr, "d2f mismatch %a -> %08x (host %08x)\n", d, got, fbits((float)d));
  bad += ok ? 0 : 1;
}

int main(int argc, char** argv) {
  if (argc >= 2 && argv[1][0] == 'F') {
    unsigned long long bad = 0, n = 0;
    for (uint64_t b = 0; b <= 0xffffffffull; b++, n++) {
      const float f = f_of((unsigned)b);
      unsigned hi, lo;
      f32_bits_to_f64_bits((unsigned)b, hi, lo);
      const uint64_t got = ((uint64_t)hi << 32) | lo;
      const unsigned e = ((unsigned)b >> 23) & 0xffu, m = (unsigned)b & 0x7fffffu;
      bool ok;
      if (e == 0u && m != 0u) ok = got == ((uint64_t)((unsigned)b & 0x80000000u) << 32);  // subnormal -> signed zero
      else if (std::isnan(f)) ok = std::isnan(of_bits(got)) && (got & (1ull << 51)) != 0 &&
                                  ((got >> 29) & 0x3fffffull) == (m & 0x3fffffu);  // payload kept, quieted
      else ok = got == bits_of((double)f);
      if (!ok && bad < 5) fprintf(stderr, "f2d mismatch %08x -> %016llx\n", (unsigned)b, (unsigned long long)got);
      bad += ok ? 0 : 1;
    }
    printf("%llu %llu\n", bad, n);
    return 0;
  }
  if (argc >= 4 && argv[1][0] == 'D') {
    const long long n = atoll(argv[2]);
    state = (uint64_t)atoll(argv[3]);
    unsigned long long bad = 0, cnt = 0;
    for (long long i = 0; i < n; i++) {
      // a double with a random mantissa and an exponent across (and just beyond) the FP32 range
      const uint64_t r = next();
      const int ex = (int)(r % 300) - 150;
      const double d = std::ldexp(1.0 + (double)(next() >> 11) * 0x1p-53, ex) * ((r >> 40) & 1 ? -1.0 : 1.0);
      check_d2f(d, bad);
      cnt++;
      // an exact tie between two FP32 neighbours, and the doubles on either side
      const float f = (float)d;
      if (std::isfinite(f) && std::fabs(f) >= 0x1p-126f) {
        const double t = (double)f + 0.5 * ((double)std::nextafter(f, INFINITY) - (double)f);
        check_d2f(t, bad);
        check_d2f(std::nextafter(t, INFINITY), bad);
        check_d2f(std::nextafter(t, -INFINITY), bad);
        cnt += 3;
      }
    }
    const double fmax = 3.4028234663852886e38;
    const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, -NAN, fmax, -fmax, fmax * (1 + 0x1p-25),
                              fmax * (1 + 0x1p-24), fmax * (1 + 0x1p-23), 1e39, 1e300, -1e300, 1e-300, 0x1p-126,
                              0x1p-126 * (1 - 0x1p-30), 0x1p-149, 1.0, -1.0, 0x1.fffffffp0, 0x1.000001p0, 0x1.0000018p0};
    for (double v : special) {
      check_d2f(v, bad);
      cnt++;
    }
    printf("%llu %llu\n", bad, cnt);
    return 0;
  }
  fprintf(stderr, "usage: %s F | D <n> <seed>\n", argv[0]);
  return 2;
}
