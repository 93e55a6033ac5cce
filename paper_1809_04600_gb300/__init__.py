"""GB300 (sm_103a) library for the variational hot path of fast semistochastic
heat-bath configuration interaction (arXiv:1809.04600).

The compute lives in the CUDA library ``libshci.so`` (C ABI: include/shci.h);
this package only builds and binds it.  Importing the package does not load
the library; the first call does, and fails loudly if it was not built.
"""
from .binding import (  # noqa: F401
    EXPORTED, SHCI_AUTO, SHCI_MEM_DEVICE, SHCI_MEM_HOST, SHCI_ON_THE_FLY, SHCI_STORED, SHCI_STORED_UPPER, Context,
    ShciError,
    load_library, shci_build_connectivity, shci_create, shci_davidson, shci_davidson_history, shci_destroy,
    shci_get_diag,
    shci_get_pairs, shci_get_row, shci_get_stats, shci_last_error, shci_load_integrals, shci_set_timing, shci_sigma,
)
from .binding import shci_energy_backward, shci_pt2, shci_select, shci_sigma_noalloc  # noqa: F401
from .binding import shci_extend_connectivity  # noqa: F401
from .binding import shci_alias_draw, shci_pt2_3step, shci_pt2_samples, shci_pt2_semistochastic  # noqa: F401
from .binding import (  # noqa: F401
    shci_batch_create, shci_batch_davidson, shci_batch_destroy, shci_batch_get_modes, shci_batch_get_stats,
    shci_batch_set_wait_limit,
)
from .binding import (  # noqa: F401
    SHCI_ERR_CUDA, SHCI_ERR_INVALID, SHCI_ERR_NOT_CONVERGED, SHCI_ERR_OOM, SHCI_ERR_STATE, SHCI_ERR_TIMEOUT, SHCI_OK,
)
from .build_lib import build  # noqa: F401


def __getattr__(name):
    # the autograd wrapper needs torch; import it on first use only
    if name == "Energy":
        from .autograd import Energy
        return Energy
    raise AttributeError(name)
