"""GB300-native hot path of FIRM (Wang, Shkolnisky & Singer): type-1 NUFFT spreading of
the central-slice samples into the Toeplitz kernel and A*b, and CG on the normal
equations with the kernel applied by 2N circulant FFT convolution.

The computation lives in the CUDA library libfirm.so (C ABI in include/firm.h).
`_lib` is its ctypes binding; `Reconstructor` owns a plan and a torch-allocated
workspace and calls the C ABI.  There is no CPU fallback: without the built
library every call raises.
"""
from . import _lib  # noqa: F401
from ._lib import (  # noqa: F401
    FirmError, firm_backproject, firm_cg_solve, firm_copy_out, firm_destroy, firm_kernel,
    firm_lambda_eff, firm_plan, firm_set_timing, firm_stage_times, strerror,
    firm_toeplitz_apply, firm_workspace_size, make_groups, make_params,
)
from .recon import Reconstructor  # noqa: F401
from .batch import BatchReconstructor  # noqa: F401
