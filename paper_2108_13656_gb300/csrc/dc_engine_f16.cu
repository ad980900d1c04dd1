// Engine kernels for DC_F16 input (all operations, all batch capacities).
#include "dc_engine_impl.cuh"

namespace dc {

int launch_engine_f16(const void* batch, int cap, int opk, LaunchShape ls, void* stream)
{
    return launch_dispatch<DC_F16>(batch, cap, opk, ls, stream);
}

int occupancy_f16(int cap, int opk)
{
    return occupancy_dispatch<DC_F16>(cap, opk);
}

}  // namespace dc
