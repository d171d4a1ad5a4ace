// Host-only check of the multiply-high division constants of kcs_internal.cuh
// (div_magic32 / div_magic64): for every divisor and dividend in the ranges the
// kernels use, the high half of n * mul equals the exact quotient n / d.
// Built and run by tests/test_host_divmagic.py; needs no GPU.
#include <cstdio>
#include <cstdint>
#include <random>

#include "../../paper_1803_10045_b300/csrc/kcs_internal.cuh"

int main() {
  long long bad = 0, checked = 0;
  // 32-bit form: divisors 2..4096, every dividend n with n (d - 1) < 2^32, up to 2^16
  for (unsigned d = 2; d <= 4096; ++d) {
    const unsigned mul = kcs::div_magic32(d);
    const unsigned long long nmax = std::min<unsigned long long>(1ull << 16, 0xffffffffull / (d - 1));
    for (unsigned long long n = 0; n < nmax; ++n) {
      const unsigned q = (unsigned)((n * (unsigned long long)mul) >> 32);
      bad += q != n / d;
      ++checked;
    }
  }
  // 64-bit form: divisors 1..2^24 and dividends below 2^40 (random), plus edges
  std::mt19937_64 rng(7);
  for (int k = 0; k < 2000000; ++k) {
    const unsigned long long d = 1 + rng() % (1ull << 24);
    const unsigned long long n = rng() % (1ull << 40);
    const unsigned long long mul = kcs::div_magic64(d);
    const unsigned long long q =
        mul ? (unsigned long long)(((unsigned __int128)n * mul) >> 64) : n;
    bad += q != n / d;
    ++checked;
  }
  for (unsigned long long d : {1ull, 2ull, 3ull, 344ull, 118336ull, 15028672ull}) {
    const unsigned long long mul = kcs::div_magic64(d);
    for (unsigned long long n : {0ull, d - 1, d, d + 1, 15028671ull, (1ull << 40) - 1}) {
      const unsigned long long q =
          mul ? (unsigned long long)(((unsigned __int128)n * mul) >> 64) : n;
      bad += q != n / d;
      ++checked;
    }
  }
  std::printf("checked %lld bad %lld\n", checked, bad);
  return bad == 0 ? 0 : 1;
}
