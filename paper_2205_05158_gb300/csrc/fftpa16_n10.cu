// Instantiations of the OFDM + PA row kernels with BF16 frequency-domain planes for N = 1024.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE16(10)
}  // namespace fdk
