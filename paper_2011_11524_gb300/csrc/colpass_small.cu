// colpass_small.cu -- the specialized column passes for N1 in {64, 96, 128, 192, 256, 384} (the
// splits of transform lengths 2^15 .. 2^18, the medium products of batched and served work).
#include "colpass.cuh"

namespace dml {
DMUL_COLPASS_SET(small, 64, 96, 128, 192, 256, 384)
}  // namespace dml
