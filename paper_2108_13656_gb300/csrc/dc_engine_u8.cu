// Engine kernels for DC_U8 input (all operations, all batch capacities).
#include "dc_engine_impl.cuh"

namespace dc {

int launch_engine_u8(const void* batch, int cap, int opk, LaunchShape ls, void* stream)
{
    return launch_dispatch<DC_U8>(batch, cap, opk, ls, stream);
}

int occupancy_u8(int cap, int opk)
{
    return occupancy_dispatch<DC_U8>(cap, opk);
}

}  // namespace dc
