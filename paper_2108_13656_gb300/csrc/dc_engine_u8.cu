// Pass kernels for DC_U8 input (all operations and pass kinds, all batch capacities).
#include "dc_engine_impl.cuh"

namespace dc {

int launch_engine_u8(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream)
{
    return launch_dispatch<DC_U8>(batch, cap, opk, kind, ph, pl, ls, stream);
}

int occupancy_u8(int cap, int opk, int kind, int pl)
{
    return occupancy_dispatch<DC_U8>(cap, opk, kind, pl);
}

int bounds_u8(uint32_t* flags)
{
    return bounds_take<DC_U8>(flags);
}

}  // namespace dc
