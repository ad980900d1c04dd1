// Engine kernels for DC_F32 input (all operations, all batch capacities).
#include "dc_engine_impl.cuh"

namespace dc {

int launch_engine_f32(const void* batch, int cap, int opk, LaunchShape ls, void* stream)
{
    return launch_dispatch<DC_F32>(batch, cap, opk, ls, stream);
}

int occupancy_f32(int cap, int opk)
{
    return occupancy_dispatch<DC_F32>(cap, opk);
}

}  // namespace dc
