"""GB300-native (sm_103a) Radial Intersection Count Image generation and clutter-resistant search.

The computation lives in the CUDA library ``_build/librici.so`` (sources in ``csrc/``, C ABI
in ``include/rici.h``); ``binding`` marshals torch CUDA tensors into it.  Build the library
with ``paper_2007_02306_gb300.build.build()``.
"""
from .binding import (  # noqa: F401
    GEN_DEFAULT, GEN_FP64, SEARCH_AUTO, SEARCH_CUDA_CORE, SEARCH_DEFAULT, SEARCH_EXACT_SLOW,
    SEARCH_INT8_TC, SEARCH_SPARSE, SEARCH_TENSOR, RiciError,
    autotune_generate_batch, autotune_search_batch, batch_run, clutter_areas, crss_search,
    crss_search_batch,
    get_tuning,
    load_library, rici_generate, rici_generate_batch, set_tuning, spin_images, sync_status,
    version,
)
