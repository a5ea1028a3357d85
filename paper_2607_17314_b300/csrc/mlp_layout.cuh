// Parameter layout of the proposer network (8 -> 128 -> 128 -> 1): W1 [128][8],
// b1 [128], W2 [128][128], b2 [128], W3 [128], b3, FP32 master values.
#pragma once

namespace isdf {
namespace mlpl {

constexpr int MF = 8, MH = 128;  // features, width
constexpr int O_W1 = 0, O_B1 = O_W1 + MH * MF, O_W2 = O_B1 + MH, O_B2 = O_W2 + MH * MH,
              O_W3 = O_B2 + MH, O_B3 = O_W3 + MH, N_PAR = O_B3 + 1;

}  // namespace mlpl
}  // namespace isdf
