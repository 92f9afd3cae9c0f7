// mp_mixed.cu - mixed-precision tracking kernels (FP32 in-cell coordinates
// and velocities, the cumulative travel time as an FP32 pair; the engine is
// in mp_mixed.cuh).  Compiled with FMA contraction on.
#include "mp_mixed.cuh"

namespace mp {

cudaError_t launch_track_mixed(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                               int blocks_per_sm_cap, cudaStream_t s)
{
    MixEngine<false> e{f, b};
    return launch_tracking(e, modes, schedule, block, blocks_per_sm_cap, s);
}

}  // namespace mp
