"""GB300-native frequency-domain DPD for the massive MU-MIMO-OFDM downlink (arxiv 2205.05158).

The compute lives in the sm_103a CUDA library built from ``csrc/`` (C-ABI in
``include/fddpd.h``); this package is its thin Python binding.
"""
from .binding import (FDDPD_ADAM, FDDPD_BF16, FDDPD_ERR_ARG, FDDPD_ERR_CUDA, FDDPD_ERR_LAYOUT,  # noqa: F401
                      FDDPD_ERR_NOMEM, FDDPD_ERR_SINGULAR, FDDPD_ERR_TIMEOUT, FDDPD_ERR_UNSUPPORTED, FDDPD_FP16,
                      FDDPD_FP32, FDDPD_GD, FDDPD_OK, FDDPD_OPT_FACTOR_FP64, FDDPD_OPT_HOST_CHUNKS,
                      FDDPD_OPT_KEEP_PA_INPUT, FDDPD_OPT_ROW_CTAS, FDDPD_OPT_CONTRACTION_CTAS, FDDPD_OPT_CONTRACTION_ITEM,
                      FDDPD_OPT_TENSOR_CONTRACTIONS, FddpdError, Graph,
                      Plan, alu_peak, autotune_forget, debug_fail_allocs, library_path, load,
                      precode_noalloc)
from .autograd import FddpdLoss, fddpd_loss  # noqa: F401,E402
