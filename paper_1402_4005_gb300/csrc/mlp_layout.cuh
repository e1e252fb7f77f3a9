// Parameter layout of the interpolation network (64 -> 64 -> 64 -> 16), one
// float vector: W1 [64 x 64] (row n = output n), b1 [64], W2 [64 x 64],
// b2 [64], W3 [16 x 64], b3 [16].
#pragma once

namespace bamg {
constexpr int kF = 64, kH = 64, kO = 16;
constexpr int kW1 = 0, kB1 = kW1 + kH * kF, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kO * kH, kNParam = kB3 + kO;   // 9360 parameters
}  // namespace bamg
