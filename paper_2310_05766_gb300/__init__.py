"""GB300-native TSDF map-generation backend (FeatSense, Section "TSDF Map Generation").

The compute path lives in libtsdf_gb300.so (hand-written sm_103a CUDA behind a
C ABI, include/tsdf.h); `binding` is a thin ctypes layer over it with the same
function names. `synth` generates seeded synthetic LiDAR workloads.
"""
from .binding import (  # noqa: F401
    TSDF_BATCH_OPT_AUTOTUNE, TSDF_BATCH_OPT_CONFIG, TSDF_BATCH_OPT_GRAPH, TSDF_BATCH_OPT_SPIN_LIMIT,
    TSDF_BATCH_OPT_TEST_MISSING_ARRIVALS, tsdf_batch_create, tsdf_batch_destroy, tsdf_batch_get_config,
    tsdf_batch_integrate, tsdf_batch_set_option, tsdf_batch_sync, tsdf_integrate_batch,
    tsdf_server_close_session, tsdf_server_create, tsdf_server_destroy, tsdf_server_get_stats, tsdf_server_open_session,
    tsdf_server_session_map, tsdf_server_submit, tsdf_server_submit_many, tsdf_server_wait, tsdf_server_wait_many,
    TSDF_ERR_ADMISSION, TSDF_ERR_BUSY, TSDF_ERR_CAPACITY, TSDF_ERR_CUDA, TSDF_ERR_DEGENERATE, TSDF_ERR_IO, TSDF_ERR_INVALID, TSDF_ERR_OOM, TSDF_ERR_TIMEOUT,
    TSDF_FLAG_SCAN_WEIGHT, TSDF_FLAG_STEP_VALUE, TSDF_MAX_POINTS, TSDF_OK, TSDF_OPT_PDL, TSDF_OPT_REDUCTION, TSDF_OPT_SORT_CAPACITY, TSDF_OPT_HOST_ZERO_COPY, TSDF_OPT_STEPS_PER_THREAD, TSDF_OPT_WARP_MERGE, TSDF_REDUCTION_ATOMIC, TSDF_REDUCTION_AUTO, TSDF_REDUCTION_POOL, TSDF_REDUCTION_SORT, TSDF_OPT_POOL_BRICKS, TSDF_OPT_STORE_DEVICE_CHUNKS, TSDF_OPT_STORE_SPILL_AGE, TSDF_REDUCE_MIN_ABS, TSDF_REDUCE_WSUM, TsdfError, TsdfMap, lib, library_path,
    make_params, tsdf_error_string, tsdf_get_origin, tsdf_grid_device_ptr, tsdf_integrate, tsdf_integrate_host, tsdf_integrate_static,
    tsdf_last_cuda_error, tsdf_map_create, tsdf_map_load, tsdf_map_save, read_map_file, tsdf_extract_surface, tsdf_map_device_bytes, tsdf_map_reserve_store, tsdf_get_store_stats, tsdf_map_set_store_file, tsdf_register, tsdf_register_system, tsdf_extract_mesh, tsdf_get_reduction, tsdf_probe_reduction_rate, tsdf_profile_enable, tsdf_profile_read, tsdf_set_option, tsdf_map_destroy, tsdf_read, tsdf_shift, tsdf_stats, tsdf_write,
)
