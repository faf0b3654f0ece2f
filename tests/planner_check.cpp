// Host-side checks of the hierarchy planner's regrid fill (test infrastructure,
// compiled by tests/test_planner_host.py with the planner source).
//
// Input (stdin): base_n0 base_n1 base_n2 max_level, then two patch lists (old,
// new), each "count" followed by "level lo0 lo1 lo2 n0 n1 n2" lines.  For every
// kept level k = 0 .. max_level - 1 the fill of each new patch above level k
// must cover each of its cells exactly once: copy segments from old patches of
// the same level (whose source cells lie inside the old patch) plus fresh
// (prolonged) boxes.  Prints "ok" or the first violation.
#include <cstdio>
#include <string>
#include <vector>

#include "hierarchy.h"

using namespace amr;

static bool read_list(std::vector<HPatch>& v) {
  int n = 0;
  if (scanf("%d", &n) != 1) return false;
  v.resize(n);
  for (HPatch& p : v)
    if (scanf("%d %d %d %d %d %d %d", &p.level, &p.lo[0], &p.lo[1], &p.lo[2], &p.n[0], &p.n[1], &p.n[2]) != 7)
      return false;
  return true;
}

int main() {
  int bn[3], ml;
  if (scanf("%d %d %d %d", &bn[0], &bn[1], &bn[2], &ml) != 4) return 2;
  std::vector<HPatch> oldp, newp;
  if (!read_list(oldp) || !read_list(newp)) return 2;
  long long segs = 0, fresh = 0;
  for (int keep = 0; keep < ml; ++keep) {
    RegridFill fill;
    build_regrid_fill(oldp, newp, keep, fill);
    std::vector<std::vector<unsigned char>> count(newp.size());
    for (size_t i = 0; i < newp.size(); ++i)
      if (newp[i].level > keep) count[i].assign((size_t)newp[i].n[0] * newp[i].n[1] * newp[i].n[2], 0);
    auto mark = [&](int i, const int lo[3], const int n[3]) -> bool {
      const HPatch& p = newp[i];
      for (int d = 0; d < 3; ++d)
        if (lo[d] < 0 || n[d] <= 0 || lo[d] + n[d] > p.n[d]) return false;
      for (int z = lo[2]; z < lo[2] + n[2]; ++z)
        for (int y = lo[1]; y < lo[1] + n[1]; ++y)
          for (int x = lo[0]; x < lo[0] + n[0]; ++x) count[i][((size_t)z * p.n[1] + y) * p.n[0] + x] += 1;
      return true;
    };
    for (size_t l = 0; l < fill.copy.size(); ++l) {
      for (const CopySeg& s : fill.copy[l]) {
        const HPatch& d = newp[s.dst_patch];
        const HPatch& o = oldp[s.src_patch];
        if (d.level != (int)l || o.level != (int)l || d.level <= keep) { printf("copy segment on a wrong level\n"); return 1; }
        int lo[3], n[3];
        for (int k = 0; k < 3; ++k) {
          lo[k] = s.dlo[k];
          n[k] = s.dn[k];
          const int s0 = s.dlo[k] + s.sh[k], s1 = s0 + s.dn[k];   // source cells, old patch local
          if (s.mode[k] != 0 || s0 < 0 || s1 > o.n[k]) { printf("copy source outside its old patch\n"); return 1; }
          if (d.lo[k] + s.dlo[k] != o.lo[k] + s0) { printf("copy segment moves cells\n"); return 1; }
        }
        if (!mark(s.dst_patch, lo, n)) { printf("copy segment outside its new patch\n"); return 1; }
        ++segs;
      }
      for (const ProlongBox& b : fill.fresh[l]) {
        if (newp[b.patch].level != (int)l) { printf("fresh box on a wrong level\n"); return 1; }
        const int lo[3] = {b.lo[0], b.lo[1], b.lo[2]}, n[3] = {b.n[0], b.n[1], b.n[2]};
        if (!mark(b.patch, lo, n)) { printf("fresh box outside its new patch\n"); return 1; }
        ++fresh;
      }
    }
    for (size_t i = 0; i < newp.size(); ++i)
      for (unsigned char c : count[i])
        if (c != 1) {
          printf("keep %d: a cell of new patch %zu is filled %d times\n", keep, i, (int)c);
          return 1;
        }
  }
  printf("ok %lld %lld\n", segs, fresh);
  return 0;
}
