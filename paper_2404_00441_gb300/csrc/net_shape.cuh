// net_shape.cuh -- parameter layout of the proposal encoder (learned.cu,
// encoder_tc.cu): conv 3x3 C->32, conv 3x3 32->32 stride 2, conv 3x3 32->32
// stride 2, linear (32 h3 h3)->64, each weight block followed by its bias.
#pragma once

#include <stdint.h>

namespace ccw {

struct NetShape {
  int C, tj, h2, h3, flat;
  int64_t o_w1, o_b1, o_w2, o_b2, o_w3, o_b3, o_wf, o_bf, n;
};

inline NetShape net_shape(int C, int tj) {
  NetShape s;
  s.C = C;
  s.tj = tj;
  s.h2 = (tj - 1) / 2 + 1;
  s.h3 = (s.h2 - 1) / 2 + 1;
  s.flat = 32 * s.h3 * s.h3;
  int64_t o = 0;
  s.o_w1 = o; o += 32LL * C * 9;
  s.o_b1 = o; o += 32;
  s.o_w2 = o; o += 32LL * 32 * 9;
  s.o_b2 = o; o += 32;
  s.o_w3 = o; o += 32LL * 32 * 9;
  s.o_b3 = o; o += 32;
  s.o_wf = o; o += 64LL * s.flat;
  s.o_bf = o; o += 64;
  s.n = o;
  return s;
}

}  // namespace ccw
