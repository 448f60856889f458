// Instantiations of the OFDM + PA row kernels with BF16 frequency-domain planes for N = 256.
#include "fftpa.cuh"

namespace fdk {
FD_FFTPA_SIZE16(8)
}  // namespace fdk
