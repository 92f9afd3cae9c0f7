// mp_mixed_f64t.cu - the mixed-precision engine with FP64 kept for the
// cumulative travel time and for the near-zero branch of the exit time
// (MP_PREC_MIXED_F64T): the accuracy reference for the FP32 pair and the
// FP32 series of the default mixed form.
#include "mp_mixed.cuh"

namespace mp {

cudaError_t launch_track_mixed_f64t(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                                    int blocks_per_sm_cap, cudaStream_t s)
{
    MixEngine<true> e{f, b};
    return launch_tracking(e, modes, schedule, block, blocks_per_sm_cap, s);
}

}  // namespace mp
