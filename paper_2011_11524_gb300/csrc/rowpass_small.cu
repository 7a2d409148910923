// rowpass_small.cu -- the specialized row pass for N2 in {256, 512} (splits of the medium products
// of batched and served work).
#include "rowpass.cuh"

namespace dml {
DMUL_ROWPASS_SET(small, 256, 512)
}  // namespace dml
