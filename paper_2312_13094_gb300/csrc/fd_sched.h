// Column-wave schedule of a persistent sweep (fd_sched.cu).
#pragma once

#include <vector>

#include "fd_internal.h"

namespace fd {

// One grid of a scheduled launch: its index in the launch's descriptors, its
// tile columns and the planes each column updates.
struct SchedGrid {
  int shot, tiles, nz;
};

// Work items of a wave schedule of `grids` (in the order given) over at most G
// persistent CTAs: CTA c runs items [start[c], start[c+1]).  Returns the
// number of CTAs that received work (the launch's grid size).
int wave_schedule(const std::vector<SchedGrid>& grids, int G, int R,
                  std::vector<int32_t>& start, std::vector<WorkItem>& items);

}  // namespace fd
