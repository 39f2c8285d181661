"""GB300-native ph-AFQMC walker step (Shee et al., arXiv:1804.03310).

The walker step runs in libafqmc.so (hand-written sm_103a CUDA behind the C
ABI of include/afqmc.h); this package is the thin Python binding.
"""
from .afqmc import (  # noqa: F401
    Afqmc,
    AfqmcError,
    Batch,
    Inputs,
    Server,
    afqmc_footprint,
    KERNEL_IDS,
    PRECISIONS,
    decode_state,
    encode_state,
    load_library,
)
