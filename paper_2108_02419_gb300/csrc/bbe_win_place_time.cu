// bbe_win_place_time.cu -- the place-count rollout kernels of the time law of responsiveness
// (kernel code: bbe_win.cuh, MODE 1), compiled apart from the position law's.
#include "bbe_win.cuh"

namespace bbe {

namespace win {

cudaError_t launch_place_time_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    return launch_law<BBE_LAW_TIME, 1>(l, slots_per_lane, stream);
}

int resident_place_time_law(int dist, int slots_per_lane, int block, int place_cells)
{
    return resident_law<BBE_LAW_TIME, 1>(dist, slots_per_lane, block, place_cells);
}

}  // namespace win

}  // namespace bbe
