// bbe_win.cu -- the win-count rollout kernels of the position law of responsiveness, and the
// library's entry points to the win-count rollout kernels (kernel code: bbe_win.cuh).
#include <array>
#include <map>
#include <mutex>

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
    // the occupancy of a (device, distribution, layout, block size) does not change: asked once
    static std::mutex mu;
    static std::map<std::array<int, 4>, int> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    const std::array<int, 4> key{dev, dist, slots_per_lane, block};
    {
        std::lock_guard<std::mutex> g(mu);
        const auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    win::resident_time_law(dist, slots_per_lane, block);  // sets the time-law kernels' shared-memory limit too
    const int nb = win::resident_position_law(dist, slots_per_lane, block);
    std::lock_guard<std::mutex> g(mu);
    known[key] = nb;
    return nb;
}

}  // namespace bbe
