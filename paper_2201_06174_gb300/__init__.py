"""GB300-native (sm_103a) seismic saliency: local 3D DFT -> spectral projection ->
directional center-surround -> adaptive combination, behind the C ABI of include/sal.h."""
from .sal import (SAL_ERR_CUDA, SAL_ERR_DEVICE_CHECK, SAL_ERR_INVALID_ARG, SAL_ERR_OOM, SAL_ERR_TIMEOUT,  # noqa: F401
                  SAL_ERR_UNSUPPORTED, SAL_OK, ENTRY_POINTS, Params, SalError, Saliency, directional_window, load,  # noqa: F401
                  sal_adapt_weights, sal_center_surround, sal_check_bounded_wait, sal_measure_mufu_rate, sal_measure_mma_rate,
                  sal_center_surround_backward, sal_combine,
                  sal_combine_backward, sal_combine_noalloc, sal_create, sal_destroy, sal_last_error_text,
                  sal_launch_count, sal_local_spectra_project, sal_local_spectra_project_backward, sal_saliency,
                  sal_saliency_backward, sal_set_alpha, sal_workspace_size)
