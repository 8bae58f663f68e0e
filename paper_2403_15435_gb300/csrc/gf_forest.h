// Host-side quadtree forest of one scenario: the leaf list in Morton order
// and the regrid rule (Sec. 4, Sec. 6.6).  The forest has mi x mj level-0
// blocks; a leaf is (level, px, py) on that level's patch grid.
#pragma once

#include <cstdint>
#include <vector>

namespace gf {

struct Leaf {
  int level, px, py;
};

class HostForest {
 public:
  HostForest(int mi, int mj, int minlevel, int maxlevel)
      : mi_(mi), mj_(mj), minl_(minlevel), maxl_(maxlevel) {}

  // All leaves at one level, Morton ordered.
  void uniform(int level);

  // New leaf list from per-leaf flags (0 keep, 1 refine, 2 coarsen):
  // refine flagged leaves one level, refine until every face/corner
  // neighbour differs by at most one level, coarsen complete quartets of
  // sibling leaves that all ask for it when no leaf touching the parent is
  // finer than the siblings.  Morton ordered.
  std::vector<Leaf> regrid(const uint8_t* flags) const;

  const std::vector<Leaf>& leaves() const { return leaves_; }
  void set_leaves(std::vector<Leaf> l) { leaves_ = std::move(l); }

  // Position of a leaf on the finest patch grid, bits interleaved
  // (x in even bits, y in odd bits).
  uint64_t morton(const Leaf& l) const;
  void sort(std::vector<Leaf>& v) const;

 private:
  int mi_, mj_, minl_, maxl_;
  std::vector<Leaf> leaves_;
};

}  // namespace gf
