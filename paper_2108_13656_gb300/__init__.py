"""GB300-native colour-temperature decolorization with fused tone mapping.

Implements the luminance of Eq. 1-6 (Sec. II-B) of arXiv 2108.13656 and the global
(Sec. III-B-1) and local (Sec. III-B-2) tone-mapping passes applied to it, as
hand-written CUDA kernels for sm_103a behind the C ABI of include/decolor.h.  This
package is the Python binding (argument marshalling only) plus the seeded synthetic
input generators; PyTorch provides device memory and streams.  No CPU fallback
exists: calls raise when libdecolor.so cannot be loaded.
"""
from ._abi import (  # noqa: F401
    BETA_K,
    BETA_R,
    DC_F16,
    DC_F32,
    DC_HISTEQ,
    DC_LUMA_OURS,
    DC_LUMA_V,
    DC_LUMA_Y,
    DC_OP_DECOLORIZE,
    DC_OP_GLOBAL,
    DC_OP_LOCAL,
    DC_SIGMOID,
    DC_U8,
    STATS_BYTES,
    DcError,
    PreparedCall,
    VideoLocalStreams,
    VideoStreams,
    Workspace,
    debug_bounds,
    debug_fail_launch,
    debug_profile,
    decolorize,
    decolorize_tonemap_global,
    decolorize_tonemap_local,
    get_tuning,
    last_launch_count,
    library_path,
    load,
    local_params,
    local_tile_cols,
    parse_stats,
    preset,
    query_status,
    read_profile,
    set_tuning,
    status_string,
    workspace_bytes,
)
from .pipeline import CallStreams, HostPipeline  # noqa: F401
