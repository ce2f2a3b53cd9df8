// Host program for tests/test_fixed_point.py: reads float32 bit patterns (hex,
// one per line) and prints, per value, fix_split's result: ok hi lo.
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include "gp_step_device.cuh"

int main() {
  unsigned int bits;
  while (scanf("%x", &bits) == 1) {
    float v;
    memcpy(&v, &bits, sizeof(v));
    long long hi = 0, lo = 0;
    const bool ok = fix_split(v, hi, lo);
    printf("%d %lld %lld\n", ok ? 1 : 0, hi, lo);
  }
  return 0;
}
