// Instantiations of the OFDM + PA row kernels for N = 2048.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(11)
}  // namespace fdk
