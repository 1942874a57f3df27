"""GB300 (sm_103a) stepper for the 3D constant-density acoustic wave equation.

Implements the hot path of arXiv 2204.03775 -- the time loop of Algorithm 1
with the leapfrog update of Eq. 2 and the 25-point, 8th-order star Laplacian
of Section II -- as hand-written CUDA kernels behind the C ABI of
``include/wavestep.h``. ``binding`` is the thin Python binding with the same
names; ``synthetic`` builds the seeded workloads.
"""

from .binding import (  # noqa: F401
    WS_ADJ_DATA, WS_ADJ_RESIDUAL, WS_ERR_BADARG, WS_ERR_CFL, WS_ERR_CUDA, WS_ERR_OOM, WS_ERR_STATE, WS_ERR_TIMEOUT,
    WS_KERNEL_AUTO, WS_KERNEL_DIRECT, WS_KERNEL_STREAM, WS_MAX_SOURCES, WS_OK, WS_STORAGE_BF16,
    WS_STORAGE_FP16, WS_STORAGE_FP32, Batch, Handle,
    WaveStepError, load_library, ws_add_source, ws_adjoint_gradient, ws_adjoint_gradient_shots,
    ws_autotune,
    ws_batch_create, ws_batch_destroy, ws_batch_get_tiling, ws_batch_launch_count,
    ws_batch_set_tiling, ws_batch_step, ws_batch_synchronize, ws_clear_sources, ws_create, ws_destroy, ws_energy, ws_forward,
    ws_energy_noalloc,
    ws_get_step, ws_last_error, ws_launch_count, ws_read_field, ws_read_traces, ws_set_kernel,
    ws_set_receivers, ws_set_slowness2, ws_set_sponge, ws_set_storage, ws_set_stream, ws_set_velocity, ws_step,
    ws_synchronize, ws_test_check_padding, ws_test_fill_padding, ws_test_stall,
    ws_write_field)
