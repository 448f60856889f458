// Per-subcarrier contractions with cf16 operands.
#include "bingemm.cuh"

namespace fdk {
FD_BIN_TYPE(f16, cf16)
}  // namespace fdk
