// Pass kernels for DC_F32 input (all operations and pass kinds, all batch capacities).
#include "dc_engine_impl.cuh"

namespace dc {

int launch_engine_f32(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream)
{
    return launch_dispatch<DC_F32>(batch, cap, opk, kind, ph, pl, ls, stream);
}

int occupancy_f32(int cap, int opk, int kind, int pl)
{
    return occupancy_dispatch<DC_F32>(cap, opk, kind, pl);
}

int bounds_f32(uint32_t* flags)
{
    return bounds_take<DC_F32>(flags);
}

}  // namespace dc
