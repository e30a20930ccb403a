// bbe_win.cu -- the win-count rollout kernels of the position law of responsiveness, and the
// library's entry points to the win-count rollout kernels (kernel code: bbe_win.cuh).
#include "bbe_win.cuh"

namespace bbe {

namespace win {

cudaError_t launch_position_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    return launch_law<BBE_LAW_POSITION, 0>(l, slots_per_lane, stream);
}

int resident_position_law(int dist, int slots_per_lane, int block)
{
    return resident_law<BBE_LAW_POSITION, 0>(dist, slots_per_lane, block, 0);
}

}  // namespace win

cudaError_t launch_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    return l.b.law == BBE_LAW_TIME ? win::launch_time_law(l, slots_per_lane, stream)
                                   : win::launch_position_law(l, slots_per_lane, stream);
}

int rollout_resident_blocks(int dist, int slots_per_lane, int block)
{
    win::resident_time_law(dist, slots_per_lane, block);  // sets the time-law kernels' shared-memory limit too
    return win::resident_position_law(dist, slots_per_lane, block);
}

}  // namespace bbe
