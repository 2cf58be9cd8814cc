"""GB300-native BP+DC decoder (arXiv 2510.08695): batched flooding min-sum BP
with degeneracy cutting, as hand-written sm_103a CUDA behind the C-ABI of
``libbpdc.so`` (declared in ``include/bpdc.h``)."""
from ._bpdc import (  # noqa: F401
    BpdcError, Graph, Options, check_status, debug_fail_allocations, decode_host, decode_multi, decode_multi_noalloc, declared_symbols, library_path, load,
    measure_smem_peak, version,
)
