// Host harness for the GPU path's fixed-point accumulators (fixed192.cuh):
// reads groups of doubles (count, then values as hex bit patterns) from stdin
// and prints the rounded sum of each group (grid anchored to the group's
// largest exponent, as on the device) as a hex bit pattern.  Argument "128"
// selects the 128-bit accumulator, otherwise the 192-bit one.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "../paper_2303_05688_gb300/csrc/fixed192.cuh"

int main(int argc, char **argv) {
  const bool w128 = argc > 1 && strcmp(argv[1], "128") == 0;
  unsigned long long cnt;
  while (scanf("%llu", &cnt) == 1) {
    double xs[4096];
    if (cnt > 4096) return 1;
    int emax = 1;
    for (unsigned long long i = 0; i < cnt; ++i) {
      unsigned long long b;
      if (scanf("%llx", &b) != 1) return 1;
      memcpy(&xs[i], &b, 8);
      const int e = asci::fx_exponent(xs[i]);
      emax = e > emax ? e : emax;
    }
    unsigned ovf = 0;
    double s;
    if (w128) {
      const int frac = asci::fx128_frac_for(emax);
      asci::Fx128 acc = {0, 0};
      for (unsigned long long i = 0; i < cnt; ++i) {
        asci::Fx128 v = asci::fx128_from_double(xs[i], frac, &ovf);
        asci::fx128_add(acc, v);
      }
      s = asci::fx128_to_double(acc, frac);
    } else {
      const int frac = asci::fx_frac_for(emax);
      asci::Fx192 acc = {0, 0, 0};
      for (unsigned long long i = 0; i < cnt; ++i) {
        asci::Fx192 v = asci::fx_from_double(xs[i], frac, &ovf);
        asci::fx_add(acc, v);
      }
      s = asci::fx_to_double(acc, frac);
    }
    uint64_t sb;
    memcpy(&sb, &s, 8);
    printf("%llx %u\n", (unsigned long long)sb, ovf);
  }
  return 0;
}
