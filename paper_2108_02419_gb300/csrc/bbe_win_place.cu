// bbe_win_place.cu -- the place-count rollout kernels (kernel code: bbe_win.cuh, MODE 1): every
// rollout runs to the K-th finisher for bbe_place_counts, bbe_order_counts and
// bbe_order_histogram; the position law's kernels here, the time law's in bbe_win_place_time.cu
// (translation units of their own, so that the build compiles the kernel families in parallel).
#include <array>
#include <map>
#include <mutex>

#include "bbe_win.cuh"

namespace bbe {

namespace win {
cudaError_t launch_place_time_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
int resident_place_time_law(int dist, int slots_per_lane, int block, int place_cells);
}  // namespace win

cudaError_t launch_place_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    return l.b.law == BBE_LAW_TIME ? win::launch_place_time_law(l, slots_per_lane, stream)
                                   : win::launch_law<BBE_LAW_POSITION, 1>(l, slots_per_lane, stream);
}

int place_resident_blocks(int dist, int slots_per_lane, int block, int place_cells)
{
    // asked once per (device, distribution, layout, block size, place table size)
    static std::mutex mu;
    static std::map<std::array<int, 5>, int> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    const std::array<int, 5> key{dev, dist, slots_per_lane, block, place_cells};
    {
        std::lock_guard<std::mutex> g(mu);
        const auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    win::resident_place_time_law(dist, slots_per_lane, block, place_cells);  // sets its shared-memory limit too
    const int nb = win::resident_law<BBE_LAW_POSITION, 1>(dist, slots_per_lane, block, place_cells);
    std::lock_guard<std::mutex> g(mu);
    known[key] = nb;
    return nb;
}

}  // namespace bbe
