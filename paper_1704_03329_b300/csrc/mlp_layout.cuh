// Layout of the classifier parameter vector (PPMD_MLP_NPARAM FP32 values):
//   mu[30] | isd[30] | W1[30][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
// with x' = (x - mu) isd and y = x' W + b (input-major weights).
#pragma once

namespace ppmd {

constexpr int OFF_MU = 0, OFF_ISD = 30, OFF_W1 = 60, OFF_B1 = 1980, OFF_W2 = 2044, OFF_B2 = 6140, OFF_W3 = 6204,
              OFF_B3 = 6460, NPARAM = 6464;

}  // namespace ppmd
