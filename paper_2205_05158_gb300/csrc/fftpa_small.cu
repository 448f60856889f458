// Instantiations of the OFDM + PA row kernels for N = 64, 128, 256, 512.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(6)
FD_FFTPA_SIZE(7)
FD_FFTPA_SIZE(8)
FD_FFTPA_SIZE(9)
}  // namespace fdk
