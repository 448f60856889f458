// Instantiations of the OFDM + PA row kernels for N = 128.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(7)
}  // namespace fdk
