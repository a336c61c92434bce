// Column-wave schedule of a persistent sweep.
//
// The equal-share sweep gives every resident CTA the same number of planes,
// but when the tile columns outnumber the CTAs a CTA's share starts part way
// through a column, so neighbouring columns are streamed at unrelated z and
// the halo rows one column loads are gone from L2 before its neighbour needs
// them.  The lockstep mode keeps neighbours in step, but only when all
// columns fit on the GPU at once.  A wave schedule does the same for any
// number of columns and grids:
//  * every column is cut into k_s z chunks of about the same height H (the
//    same H for every grid of the launch, so all work items cost about the
//    same);
//  * the items are ordered grid by grid, chunk by chunk, tile by tile (tile
//    columns in row-major order), so consecutive items are neighbouring
//    columns at the same depth;
//  * item i goes to CTA (i mod G) in wave i / G, every other wave in reverse
//    order so that short and long items even out; the G CTAs of a wave then
//    stream G consecutive items side by side, as in lockstep.
// H is picked by simulating the load of the busiest CTA, counting each item
// as its planes plus the 2R halo planes its ring must load before the first
// output plane and a few planes' worth of set-up.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fd_internal.h"
#include "fd_sched.h"

namespace fd {

namespace {

// Chunks of a column of nz planes at target height H: ceil(nz / H).
int chunks_of(int nz, double H) { return std::max(1, int(std::ceil(nz / H - 1e-9))); }

long long max_load(const std::vector<SchedGrid>& grids, double H, int G, int R, long long* items) {
  const long long over = 2LL * R + 4;
  std::vector<long long> load(G, 0);
  long long i = 0;
  for (const SchedGrid& g : grids) {
    const int k = chunks_of(g.nz, H);
    for (int j = 0; j < k; ++j) {
      const long long h = (long long)g.nz * (j + 1) / k - (long long)g.nz * j / k;
      for (int t = 0; t < g.tiles; ++t, ++i) {
        const long long w = i / G, p = i % G;
        load[(w & 1) ? G - 1 - p : p] += h + over;
      }
    }
  }
  *items = i;
  return *std::max_element(load.begin(), load.end());
}

}  // namespace

int wave_schedule(const std::vector<SchedGrid>& grids, int G, int R,
                  std::vector<int32_t>& start, std::vector<WorkItem>& items) {
  start.clear();
  items.clear();
  long long planes = 0;
  int nzmax = 1;
  for (const SchedGrid& g : grids) {
    planes += (long long)g.tiles * g.nz;
    nzmax = std::max(nzmax, g.nz);
  }
  if (G < 1 || planes == 0) return 0;
  // candidate heights: the tallest column in k = 1 .. 64 chunks, and all
  // planes spread over W = 1 .. 64 full waves; none below 4R planes
  std::vector<double> cand;
  for (int k = 1; k <= 64; ++k) cand.push_back(double(nzmax) / k);
  for (int W = 1; W <= 64; ++W) cand.push_back(double(planes) / (double(W) * G));
  double bestH = nzmax;
  long long n_items = 0;
  long long best = max_load(grids, bestH, G, R, &n_items);
  for (double H : cand) {
    if (H > nzmax || H < 4.0 * R) continue;
    const long long l = max_load(grids, H, G, R, &n_items);
    if (l < best) {
      best = l;
      bestH = H;
    }
  }
  // the items in wave order, then grouped per CTA
  std::vector<std::vector<WorkItem>> per(G);
  long long i = 0;
  for (size_t s = 0; s < grids.size(); ++s) {
    const SchedGrid& g = grids[s];
    const int k = chunks_of(g.nz, bestH);
    for (int j = 0; j < k; ++j) {
      const int zb = int((long long)g.nz * j / k), ze = int((long long)g.nz * (j + 1) / k);
      for (int t = 0; t < g.tiles; ++t, ++i) {
        const long long w = i / G, p = i % G;
        per[(w & 1) ? G - 1 - p : p].push_back({g.shot, t, zb, ze});
      }
    }
  }
  int used = 0;
  for (int c = 0; c < G; ++c)
    if (!per[c].empty()) used = c + 1;
  start.assign(used + 1, 0);
  for (int c = 0; c < used; ++c) {
    start[c + 1] = start[c] + int(per[c].size());
    items.insert(items.end(), per[c].begin(), per[c].end());
  }
  return used;
}

}  // namespace fd
