// Host harness for the bit-field FP64 helpers of the tensor-core element
// set-up (fei_geom.cuh), driven by test_geom_bits_cpu.py.  Each input line
// is "mode x y" with x, y given as FP64 bit patterns in hex; the output line
// holds the results as FP32 bit patterns in hex:
//   mode 1: split_f64_bits(x)  -> in_range hi lo
//   mode 2: f64_to_f32_bits(x) -> 1 f 0
#include <stdio.h>
#include <string.h>

#include "fei_geom.cuh"

static unsigned fbits(float f) {
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
}

int main() {
  int mode;
  unsigned long long bx, by;
  while (scanf("%d %llx %llx", &mode, &bx, &by) == 3) {
    double x, y;
    memcpy(&x, &bx, 8);
    memcpy(&y, &by, 8);
    bool ok = true;
    float2 r = make_float2(0.f, 0.f);
    (void)y;
    if (mode == 1) r = fei::split_f64_bits(x, &ok);
    else r.x = fei::f64_to_f32_bits(x);
    printf("%d %08x %08x\n", ok ? 1 : 0, fbits(r.x), fbits(r.y));
  }
  return 0;
}
