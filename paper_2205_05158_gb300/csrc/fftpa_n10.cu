// Instantiations of the OFDM + PA row kernels for N = 1024.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(10)
}  // namespace fdk
