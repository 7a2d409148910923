// colpass_five.cu -- the specialized column passes for N1 in {80, 160, 320, 640, 1280}: the splits
// of the transform lengths 5 * 2^k (radix 5 first, Sec. 4.5's smoother length set).
#include "colpass.cuh"

namespace dml {
DMUL_COLPASS_SET(five, 80, 160, 320, 640, 1280)
}  // namespace dml
