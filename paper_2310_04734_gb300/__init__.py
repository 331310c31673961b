"""GB300-native frequency-response sweep and rational Arnoldi MOR for coupled
shell-cavity FE models (arXiv 2310.04734, Blech et al.).

The computation lives in the CUDA library ``libfsi.so`` (C ABI in
include/fsi.h); ``api`` is its Python binding.
"""
from . import api  # noqa: F401
from .api import (DeviceModel, fsi_assemble, fsi_assemble_host, fsi_batched_lu,  # noqa: F401
                  fsi_model_dims, fsi_residual, frf_sweep_full, rom_build, rom_project, rom_sweep)
