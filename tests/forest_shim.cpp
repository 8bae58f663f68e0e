// Test shim: the library's host quadtree (gf_forest.cpp) behind one C entry
// point, so that CPU tests can drive its regrid rule directly.
#include <cstdint>
#include <vector>

#include "../paper_2403_15435_gb300/csrc/gf_forest.h"

// New leaf list (written to olev/opx/opy, at most cap leaves) of the forest
// with leaves (lev, px, py)[n] after a regrid with per-leaf flags (0 keep,
// 1 refine, 2 coarsen).  Returns the number of leaves, or -1 if cap is too
// small.
extern "C" int forest_regrid(int mi, int mj, int minlevel, int maxlevel, int n,
                             const int* lev, const int* px, const int* py,
                             const uint8_t* flags, int cap, int* olev, int* opx,
                             int* opy) {
  gf::HostForest f(mi, mj, minlevel, maxlevel);
  std::vector<gf::Leaf> v((size_t)n);
  for (int k = 0; k < n; ++k) v[(size_t)k] = gf::Leaf{lev[k], px[k], py[k]};
  f.set_leaves(v);
  const std::vector<gf::Leaf> out = f.regrid(flags);
  if ((int)out.size() > cap) return -1;
  for (size_t k = 0; k < out.size(); ++k) {
    olev[k] = out[k].level;
    opx[k] = out[k].px;
    opy[k] = out[k].py;
  }
  return (int)out.size();
}
