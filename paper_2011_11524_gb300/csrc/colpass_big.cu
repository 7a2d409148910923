// colpass_big.cu -- the specialized column passes for N1 in {512, 768, 1024, 1536}.
#include "colpass.cuh"

namespace dml {
DMUL_COLPASS_SET(big, 512, 768, 1024, 1536)
}  // namespace dml
