// Per-subcarrier contractions with c32 operands.
#include "bingemm.cuh"

namespace fdk {
FD_BIN_TYPE(f32, c32)
}  // namespace fdk
