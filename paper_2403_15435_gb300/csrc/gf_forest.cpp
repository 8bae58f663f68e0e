// Host quadtree: regrid with 2:1 balance.  The balance test works on the set
// of tree nodes (leaves and their ancestors): a leaf of level L touches a
// leaf of level >= L+2 exactly when some node of level L+2 sits in the ring
// of level-(L+2) positions around the leaf.
#include "gf_forest.h"

#include <algorithm>
#include <unordered_set>

namespace gf {

namespace {

inline uint64_t key(int L, long long x, long long y) {
  return ((uint64_t)L << 58) | ((uint64_t)x << 29) | (uint64_t)y;
}

// The set of tree nodes (leaves and their ancestors).  A dense bit map per
// level when the levels' patch grids are small enough (every lookup is one
// load), else a hash set.
class NodeSet {
 public:
  NodeSet(int mi, int mj, int maxl) : mi_(mi), mj_(mj) {
    size_t total = 0;
    for (int l = 0; l <= maxl; ++l) total += ((size_t)mi << l) * ((size_t)mj << l);
    dense_ = total <= kDenseLimit;
    if (dense_) {
      off_.resize(maxl + 2, 0);
      for (int l = 0; l <= maxl; ++l)
        off_[l + 1] = off_[l] + ((size_t)mi << l) * ((size_t)mj << l);
      bits_.assign(total, 0);
    }
  }
  void add_leaf(int L, int x, int y) {
    for (int l = L; l >= 0; --l) {
      const long long xl = x >> (L - l), yl = y >> (L - l);
      if (dense_) {
        uint8_t& b = bits_[index(l, xl, yl)];
        if (b) break;
        b = 1;
      } else if (!s_.insert(key(l, xl, yl)).second) {
        break;
      }
    }
  }
  bool has(int L, long long x, long long y) const {
    if (x < 0 || y < 0 || x >= ((long long)mi_ << L) || y >= ((long long)mj_ << L))
      return false;
    if (dense_) return bits_[index(L, x, y)] != 0;
    return s_.count(key(L, x, y)) != 0;
  }
  // any node of level Lr in the one-position ring around the square
  // [x0, x0+n) x [y0, y0+n) of that level
  bool ring_has(int Lr, long long x0, long long y0, long long n) const {
    for (long long x = x0 - 1; x <= x0 + n; ++x) {
      if (has(Lr, x, y0 - 1) || has(Lr, x, y0 + n)) return true;
    }
    for (long long y = y0; y < y0 + n; ++y) {
      if (has(Lr, x0 - 1, y) || has(Lr, x0 + n, y)) return true;
    }
    return false;
  }

 private:
  static constexpr size_t kDenseLimit = size_t(1) << 26;  // 64 MB of flags
  size_t index(int L, long long x, long long y) const {
    return off_[L] + (size_t)y * ((size_t)mi_ << L) + (size_t)x;
  }
  int mi_, mj_;
  bool dense_ = false;
  std::vector<size_t> off_;
  std::vector<uint8_t> bits_;
  std::unordered_set<uint64_t> s_;
};

}  // namespace

namespace {

// Spread the low 32 bits of v to the even bit positions (bit b -> 2b).
inline uint64_t spread_bits(uint64_t v) {
  v &= 0xffffffffull;
  v = (v | (v << 16)) & 0x0000ffff0000ffffull;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

}  // namespace

uint64_t HostForest::morton(const Leaf& l) const {
  const uint64_t X = (uint64_t)l.px << (maxl_ - l.level);
  const uint64_t Y = (uint64_t)l.py << (maxl_ - l.level);
  return spread_bits(X) | (spread_bits(Y) << 1);
}

void HostForest::sort(std::vector<Leaf>& v) const {
  // keys computed once per leaf, then sorted with their leaves
  std::vector<std::pair<uint64_t, Leaf>> kv(v.size());
  for (size_t k = 0; k < v.size(); ++k) kv[k] = {morton(v[k]), v[k]};
  std::sort(kv.begin(), kv.end(), [](const std::pair<uint64_t, Leaf>& a,
                                     const std::pair<uint64_t, Leaf>& b) {
    return a.first < b.first;
  });
  for (size_t k = 0; k < v.size(); ++k) v[k] = kv[k].second;
}

void HostForest::uniform(int level) {
  leaves_.clear();
  const int w = mi_ << level, h = mj_ << level;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) leaves_.push_back(Leaf{level, x, y});
  sort(leaves_);
}

std::vector<Leaf> HostForest::regrid(const uint8_t* flags) const {
  const size_t n0 = leaves_.size();
  // 1. refinement of tagged leaves
  std::vector<Leaf> cur;
  std::vector<int> from;  // original index, -1 for new leaves
  cur.reserve(n0 * 2);
  for (size_t k = 0; k < n0; ++k) {
    const Leaf& l = leaves_[k];
    if (flags[k] == 1 && l.level < maxl_) {
      for (int c = 0; c < 4; ++c) {
        cur.push_back(Leaf{l.level + 1, 2 * l.px + (c & 1), 2 * l.py + (c >> 1)});
        from.push_back(-1);
      }
    } else {
      cur.push_back(l);
      from.push_back((int)k);
    }
  }
  // 2. balance: refine leaves that touch a leaf two or more levels finer
  NodeSet nodes(mi_, mj_, maxl_);
  for (const Leaf& l : cur) nodes.add_leaf(l.level, l.px, l.py);
  for (bool changed = true; changed;) {
    changed = false;
    const size_t n = cur.size();
    for (size_t k = 0; k < n; ++k) {
      const Leaf l = cur[k];
      const int Lr = l.level + 2;
      if (Lr > maxl_) continue;
      if (!nodes.ring_has(Lr, 4LL * l.px, 4LL * l.py, 4)) continue;
      const Leaf c0{l.level + 1, 2 * l.px, 2 * l.py};
      cur[k] = c0;
      from[k] = -1;
      nodes.add_leaf(c0.level, c0.px, c0.py);
      for (int c = 1; c < 4; ++c) {
        const Leaf ch{l.level + 1, 2 * l.px + (c & 1), 2 * l.py + (c >> 1)};
        cur.push_back(ch);
        from.push_back(-1);
        nodes.add_leaf(ch.level, ch.px, ch.py);
      }
      changed = true;
    }
  }
  // 3. coarsening of untouched complete quartets
  std::vector<int> where(n0, -1);
  for (size_t k = 0; k < cur.size(); ++k)
    if (from[k] >= 0) where[from[k]] = (int)k;
  std::vector<char> drop(cur.size(), 0);
  std::vector<Leaf> parents;
  // The leaves are in Morton order and four sibling leaves tile their
  // parent, so a complete quartet occupies four consecutive entries, in the
  // order (0,0), (1,0), (0,1), (1,1) of the children.
  for (size_t k = 0; k < n0; ++k) {
    const Leaf& l = leaves_[k];
    if (l.level <= minl_ || (l.px & 1) || (l.py & 1)) continue;
    int sib[4];
    bool ok = k + 3 < n0;
    for (int c = 0; c < 4 && ok; ++c) {
      const size_t o = k + c;
      const Leaf& m = leaves_[o];
      if (m.level != l.level || m.px != l.px + (c & 1) || m.py != l.py + (c >> 1) ||
          flags[o] != 2 || where[o] < 0)
        ok = false;
      else sib[c] = (int)o;
    }
    if (!ok) continue;
    // parent at level L-1 spans 4x4 positions of level L+1
    const int Lr = l.level + 1;
    if (Lr <= maxl_ && nodes.ring_has(Lr, 2LL * l.px, 2LL * l.py, 4)) continue;
    for (int c = 0; c < 4; ++c) drop[where[sib[c]]] = 1;
    parents.push_back(Leaf{l.level - 1, l.px / 2, l.py / 2});
  }
  std::vector<Leaf> out;
  out.reserve(cur.size());
  for (size_t k = 0; k < cur.size(); ++k)
    if (!drop[k]) out.push_back(cur[k]);
  for (const Leaf& p : parents) out.push_back(p);
  sort(out);
  return out;
}

}  // namespace gf
