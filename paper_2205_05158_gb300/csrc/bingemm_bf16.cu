// Per-subcarrier contractions with cbf16 operands.
#include "bingemm.cuh"

namespace fdk {
FD_BIN_TYPE(bf16, cbf16)
}  // namespace fdk
