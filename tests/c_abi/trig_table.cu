// Prints the compile-time twiddle constants of the composite butterflies (trig::cos2pi /
// trig::sin2pi) for every m < R of the radices used, one "R m cos sin" line each, so that a
// CPU test can compare them with the mathematical values.  Host code only.
#include <stdio.h>

#include "../../paper_2004_13904_gb300/csrc/tf_fft.cuh"

template <int R> void table() {
  for (int m = 0; m < R; ++m)
    printf("%d %d %.17e %.17e\n", R, m, tfk::trig::cos2pi(m, R), tfk::trig::sin2pi(m, R));
}

int main() {
  static_assert(tfk::trig::cos2pi(0, 7) == 1.0, "constexpr evaluation");
  table<3>(); table<5>(); table<7>(); table<8>(); table<14>(); table<16>(); table<20>();
  table<25>(); table<28>(); table<32>(); table<49>(); table<64>();
  return 0;
}
