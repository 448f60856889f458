// Instantiations of the OFDM + PA row kernels for N = 4096.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE(12)
}  // namespace fdk
