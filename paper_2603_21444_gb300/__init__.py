"""GB300 (sm_103a) hot path of the trident distributed SpGEMM (arXiv 2603.21444).

The local CSR product C = A B (symbolic + numeric, row-binned), the ordered
sum of trident partial products, the batched trident grid on one GPU and the
autograd backward, all computed by hand-written CUDA kernels behind the C ABI
in include/trident_spgemm.h.  PyTorch supplies device memory and streams.
"""
from .api import (BatchPlan, DeviceCSR, Handle, Plan, TridentPlan, batched, default_handle, default_tune,  # noqa: F401
                  fused_into, mcl_step, merge, numeric_into, permute, products, spgemm, spgemm_host, spgemm_single_pass, symbolic,
                  tile_split, trident_bounds, trident_loads, trident_schedule, tune_cache_clear, tune_cache_entries,
                  tune_cache_open, tune_cache_store)
from .autograd import Pattern, SpGEMMFunction, spgemm_values, transpose  # noqa: F401,E402
