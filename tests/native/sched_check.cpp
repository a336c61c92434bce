// Host-side check of the column-wave scheduler (paper_2312_13094_gb300/csrc/
// fd_sched.cu), built with g++ by tests/test_sched_host.py: for a set of
// single-grid and multi-grid launches, every (grid, tile, plane) unit must be
// covered by exactly one work item, every CTA index must be below the CTA
// count, and items must be non-empty z ranges of existing tiles.  Prints one
// line per case: name, CTAs used, items, the busiest CTA's planes, and the
// number of faults.
#include <cstdio>
#include <vector>

#include "fd_sched.h"

using namespace fd;

static int check(const char* name, const std::vector<SchedGrid>& grids, int G, int R) {
  std::vector<int32_t> start;
  std::vector<WorkItem> items;
  const int used = wave_schedule(grids, G, R, start, items);
  int bad = 0;
  if (used < 0 || used > G) ++bad;
  if ((int)start.size() != used + 1 || start[0] != 0 || start[used] != (int)items.size()) ++bad;
  std::vector<std::vector<int>> cover;
  int maxshot = 0;
  for (const SchedGrid& g : grids) maxshot = g.shot > maxshot ? g.shot : maxshot;
  cover.resize(maxshot + 1);
  for (const SchedGrid& g : grids) cover[g.shot].assign((size_t)g.tiles * g.nz, 0);
  long long busiest = 0;
  for (int c = 0; c < used && !bad; ++c) {
    long long planes = 0;
    for (int i = start[c]; i < start[c + 1]; ++i) {
      const WorkItem& w = items[i];
      const SchedGrid* g = nullptr;
      for (const SchedGrid& q : grids)
        if (q.shot == w.shot) g = &q;
      if (!g || w.tile < 0 || w.tile >= g->tiles || w.zb < 0 || w.zb >= w.ze || w.ze > g->nz) {
        ++bad;
        continue;
      }
      for (int z = w.zb; z < w.ze; ++z) cover[w.shot][(size_t)w.tile * g->nz + z]++;
      planes += w.ze - w.zb;
    }
    busiest = planes > busiest ? planes : busiest;
  }
  for (const SchedGrid& g : grids)
    for (int v : cover[g.shot]) bad += v != 1;
  printf("%s %d %zu %lld %d\n", name, used, items.size(), busiest, bad);
  return bad;
}

int main() {
  int bad = 0;
  bad += check("single_fits", {{0, 740, 592}}, 760, 4);
  bad += check("single_waves", {{0, 370, 592}}, 304, 4);
  bad += check("single_many", {{0, 1152, 768}}, 760, 4);
  bad += check("so16", {{0, 703, 592}}, 608, 8);
  bad += check("tiny", {{0, 3, 10}}, 760, 4);
  bad += check("one_cell", {{0, 1, 1}}, 760, 8);
  bad += check("one_cta", {{0, 17, 33}}, 1, 2);
  std::vector<SchedGrid> shots;
  for (int s = 0; s < 32; ++s) shots.push_back({s, 40 + (s * 37) % 200, 168 + (s * 53) % 193});
  bad += check("batch", shots, 304, 4);
  bad += check("batch_wide", shots, 1520, 4);
  std::vector<SchedGrid> gaps = {{3, 12, 40}, {0, 5, 90}, {7, 30, 12}};
  bad += check("unordered_ids", gaps, 64, 3);
  return bad ? 1 : 0;
}
