// bbe_win_time.cu -- the win-count rollout kernels of the time law of responsiveness (kernel
// code: bbe_win.cuh), compiled apart from the position law's to halve the build's longest unit.
#include "bbe_win.cuh"

namespace bbe {

namespace win {

cudaError_t launch_time_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    return launch_law<BBE_LAW_TIME, 0>(l, slots_per_lane, stream);
}

int resident_time_law(int dist, int slots_per_lane, int block)
{
    return resident_law<BBE_LAW_TIME, 0>(dist, slots_per_lane, block, 0);
}

}  // namespace win

}  // namespace bbe
