// rt_tma_plan.h -- which device instances the tile kernels fetch with TMA
// tensor copies, as plain host logic with no CUDA, so that it can be checked
// on a machine without a GPU.
//
// A TMA group is a maximal run of consecutive device instances of one grid
// shape (their state planes lie back to back in a slot, so one 4-D tensor
// map (x, y, component, instance) covers the run). A run qualifies when its
// rows are a multiple of 16 bytes (nx * element size) and its grid holds the
// largest box any tile kernel fetches (min_nx columns, min_ny rows). At most
// max_groups runs become groups, the largest (cells times instances) first,
// ties to the earlier run; their instances are numbered from 0 within the
// group. Every other instance keeps plain loads.
#pragma once

#include <algorithm>
#include <cstddef>
#include <vector>

namespace rt {

struct TmaRun {
  int first, count, nx, ny;  // device instances [first, first + count), all nx x ny
};

// Qualifying runs of the instance shapes (nx[i], ny[i]), largest first,
// at most max_groups of them.
inline std::vector<TmaRun> tma_plan(const int* nx, const int* ny, int n, std::size_t elem_bytes, int min_nx,
                                    int min_ny, int max_groups) {
  std::vector<TmaRun> runs;
  for (int d = 0; d < n;) {
    int e = d + 1;
    while (e < n && nx[e] == nx[d] && ny[e] == ny[d]) ++e;
    if ((static_cast<std::size_t>(nx[d]) * elem_bytes) % 16 == 0 && nx[d] >= min_nx && ny[d] >= min_ny)
      runs.push_back({d, e - d, nx[d], ny[d]});
    d = e;
  }
  std::stable_sort(runs.begin(), runs.end(), [](const TmaRun& a, const TmaRun& b) {
    return static_cast<long long>(a.count) * a.nx * a.ny > static_cast<long long>(b.count) * b.nx * b.ny;
  });
  if (static_cast<int>(runs.size()) > max_groups) runs.resize(max_groups < 0 ? 0 : max_groups);
  return runs;
}

}  // namespace rt
