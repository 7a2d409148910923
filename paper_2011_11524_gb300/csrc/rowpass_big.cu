// rowpass_big.cu -- the specialized row pass for N2 in {1024, 2048, 4096, 8192}.
#include "rowpass.cuh"

namespace dml {
DMUL_ROWPASS_SET(big, 1024, 2048, 4096, 8192)
}  // namespace dml
