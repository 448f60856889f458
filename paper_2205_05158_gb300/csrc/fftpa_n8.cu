// Instantiations of the OFDM + PA row kernels for N = 256.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(8)
}  // namespace fdk
