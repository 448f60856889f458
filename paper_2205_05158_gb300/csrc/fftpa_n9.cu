// Instantiations of the OFDM + PA row kernels for N = 512.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(9)
}  // namespace fdk
