// Instantiations of the OFDM + PA row kernels for N = 64.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(6)
}  // namespace fdk
