// Host-side checks of the hierarchy planner (test infrastructure, compiled by
// tests/test_planner_host.py with the planner source).  Prints "ok ..." or the
// first violation.
//
// "fill": base_n0 base_n1 base_n2 max_level, then two patch lists (old, new),
// each "count" followed by "level lo0 lo1 lo2 n0 n1 n2" lines.  For every kept
// level k = 0 .. max_level - 1 the fill of each new patch above level k must
// cover each of its cells exactly once: copy segments from old patches of the
// same level (whose source cells lie inside the old patch) plus fresh
// (prolonged) boxes.
//
// "ghost": base_n0 base_n1 base_n2 max_level bc0 .. bc5, then one patch list.
// Each of the two ghost layers of every patch face is covered exactly once by
// the plan's ghost segments and prolongation boxes, and nothing else is; a
// segment copies, for every ghost cell, the level cell at that cell's position
// (wrapped on periodic axes) or, across an outflow face, the boundary cell of
// the patch itself.
//
// "registers": same input as "ghost".  The flux-register rectangles of each
// fine patch face hold exactly the coarse cells next to that face that no
// patch of the fine level covers (wrapped on periodic axes, none beyond an
// outflow face), each once, each in the coarse patch that holds it, with the
// coarse cell on the right side of the face; a rectangle marked unordered has
// no cell that another rectangle also holds.
//
// "items": same input as "ghost" plus the tile shape (max_wx max_cols zchunk).
// The stage work items of every level, the per-patch ones and the batched ones
// (blocks over the z-layers of patches that tile a rectangle included), cover
// every interior cell of the level exactly once, each block column inside one
// patch of the block over the block's whole z range.
//
// "gathers": same input as "ghost".  For every refined patch, each parent-tile
// cell that its prolongation reads (the parents of its prolongation boxes and
// their face neighbours) is gathered exactly once, from the coarse cell at that
// position (wrapped on periodic axes, the boundary cell beyond an outflow face).
//
// "restrict": same input as "ghost".  Every coarse cell under a finer patch is
// restricted exactly once, from the fine patch that holds its eight children,
// and the coverage boxes (which exclude covered cells from the leaf totals)
// mark exactly those coarse cells.
//
// "faces": same input as "ghost".  Where a patch face is read in place (its
// face-table entry is not the patch's own ghost cells), the entry maps each
// cell of the face's two ghost layers to the interior cell that holds that
// level position (wrapped on periodic axes) in a patch of the same level, or,
// across an outflow face, to the patch's own boundary cell; the entry's
// variable stride is that patch's.
//
// "flat": same input as "ghost".  The flattened lists the batched kernels walk
// address the same cells as the boxes they come from: each prolongation box,
// walked by parent cell as box_prolong_kernel does (children 2p + i - odd in
// the box), writes each of its fine cells once, at that cell's arena index,
// from the parent-tile cell above it; each ghost copy box reads and writes the
// cells of its segment.
//
// "cluster": base_n0 base_n1 base_n2 max_level bc0 .. bc5 buffer block
// max_patch min_level, one patch list, then per patch "0" (not flagged) or "1"
// and its n0 n1 n2 flags (z, y, x order).  Prints "ok", the number of new
// patches and one "level lo0 lo1 lo2 n0 n1 n2" line each: the host clustering
// from byte flags, for comparison with the oracle's.
#include <algorithm>
#include <array>
#include <cstdio>
#include <map>
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

static int check_ghost() {
  int bn[3], ml, bc[6];
  if (scanf("%d %d %d %d %d %d %d %d %d %d", &bn[0], &bn[1], &bn[2], &ml, &bc[0], &bc[1], &bc[2], &bc[3], &bc[4],
            &bc[5]) != 10)
    return 2;
  std::vector<HPatch> P;
  if (!read_list(P)) return 2;
  amr_config cfg{};
  cfg.nvar = 5;
  cfg.precision = AMR_FP32;
  cfg.gamma = 1.4;
  cfg.theta = 1.5;
  cfg.cfl = 0.4;
  cfg.ref_ratio = 2;
  for (int d = 0; d < 3; ++d) {
    cfg.base_n[d] = bn[d];
    cfg.domain_lo[d] = 0;
    cfg.domain_hi[d] = 1;
  }
  for (int f = 0; f < 6; ++f) cfg.bc[f] = bc[f];
  cfg.max_level = ml;
  cfg.batched = 1;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  long long segs = 0, boxes = 0;
  for (const LevelPlan& L : plan.levels) {
    for (int ii = 0; ii < L.count; ++ii) {
      const int i = L.first + ii;
      const HPatch& p = P[i];
      const int g0 = kGhost, m[3] = {p.n[0] + 2 * kGhost, p.n[1] + 2 * kGhost, p.n[2] + 2 * kGhost};
      std::vector<unsigned char> cnt((size_t)m[0] * m[1] * m[2], 0);
      auto at = [&](int x, int y, int z) -> unsigned char& {
        return cnt[((size_t)(z + g0) * m[1] + (y + g0)) * m[0] + (x + g0)];
      };
      for (int e = L.ghost_first[ii]; e < L.ghost_first[ii + 1]; ++e) {
        const CopySeg& s = L.ghost[e];
        const HPatch& o = P[s.src_patch];
        if (s.dst_patch != i || o.level != p.level) { printf("ghost segment of a wrong patch or level\n"); return 1; }
        for (int z = s.dlo[2]; z < s.dlo[2] + s.dn[2]; ++z)
          for (int y = s.dlo[1]; y < s.dlo[1] + s.dn[1]; ++y)
            for (int x = s.dlo[0]; x < s.dlo[0] + s.dn[0]; ++x) {
              const int c[3] = {x, y, z};
              for (int d = 0; d < 3; ++d) {
                const int src = s.mode[d] ? s.sh[d] : c[d] + s.sh[d];   // source-local coordinate
                if (src < 0 || src >= o.n[d]) { printf("ghost source outside its patch\n"); return 1; }
                const int N = p.level == 0 ? bn[d] : bn[d] << p.level;
                const int G = p.lo[d] + c[d];
                if (s.mode[d]) {   // outflow: the patch's own boundary cell
                  if (s.src_patch != i || (G >= 0 && G < N) || src != (G < 0 ? 0 : p.n[d] - 1)) {
                    printf("outflow ghost not the boundary cell\n");
                    return 1;
                  }
                } else if (((G % N) + N) % N != o.lo[d] + src) {
                  printf("ghost copies a cell from another position\n");
                  return 1;
                }
              }
              ++at(x, y, z);
            }
        ++segs;
      }
      if (p.level > 0)
        for (int e = L.prolong_first[ii]; e < L.prolong_first[ii + 1]; ++e) {
          const ProlongBox& b = L.prolong[e];
          if (b.patch != i) { printf("prolongation box of a wrong patch\n"); return 1; }
          for (int z = b.lo[2]; z < b.lo[2] + b.n[2]; ++z)
            for (int y = b.lo[1]; y < b.lo[1] + b.n[1]; ++y)
              for (int x = b.lo[0]; x < b.lo[0] + b.n[0]; ++x) ++at(x, y, z);
          ++boxes;
        }
      for (int z = -g0; z < p.n[2] + g0; ++z)
        for (int y = -g0; y < p.n[1] + g0; ++y)
          for (int x = -g0; x < p.n[0] + g0; ++x) {
            const int c[3] = {x, y, z};
            int out = 0;
            for (int d = 0; d < 3; ++d) out += (c[d] < 0 || c[d] >= p.n[d]) ? 1 : 0;
            const int want = out == 1 ? 1 : 0;   // face layers only (no edges, corners or interior)
            if (at(x, y, z) != want) {
              printf("patch %d cell (%d, %d, %d): covered %d times, want %d\n", i, x, y, z, (int)at(x, y, z), want);
              return 1;
            }
          }
    }
  }
  printf("ok %lld %lld\n", segs, boxes);
  return 0;
}

static bool read_config(amr_config& cfg, int bn[3], int& ml, std::vector<HPatch>& P) {
  int bc[6];
  if (scanf("%d %d %d %d %d %d %d %d %d %d", &bn[0], &bn[1], &bn[2], &ml, &bc[0], &bc[1], &bc[2], &bc[3], &bc[4],
            &bc[5]) != 10)
    return false;
  if (!read_list(P)) return false;
  cfg = amr_config{};
  cfg.nvar = 5;
  cfg.precision = AMR_FP32;
  cfg.gamma = 1.4;
  cfg.theta = 1.5;
  cfg.cfl = 0.4;
  cfg.ref_ratio = 2;
  for (int d = 0; d < 3; ++d) {
    cfg.base_n[d] = bn[d];
    cfg.domain_lo[d] = 0;
    cfg.domain_hi[d] = 1;
  }
  for (int f = 0; f < 6; ++f) cfg.bc[f] = bc[f];
  cfg.max_level = ml;
  cfg.batched = 1;
  return true;
}

static int check_registers() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  auto level_n = [&](int l, int d) { return bn[d] << l; };
  auto periodic = [&](int d) { return cfg.bc[2 * d] == AMR_BC_PERIODIC; };
  long long nreg = 0;
  for (int l = 1; l < (int)plan.levels.size(); ++l) {
    const LevelPlan& L = plan.levels[l];
    const LevelPlan& C = plan.levels[l - 1];
    // coarse cell (global, level l-1) -> (coarse patch, count) of the registers on each fine face
    std::map<std::array<int, 6>, int> got;   // (fpatch, 2d+side, cx, cy, cz, 0) -> count
    std::map<std::array<int, 6>, int> all_cells;   // (cx, cy, cz, 0, 0, 0) -> registers on the cell
    for (const RegRect& r : L.regs.boxes) {
      const HPatch& cp = P[r.cpatch];
      if (cp.level != l - 1 || P[r.fpatch].level != l) { printf("register on a wrong level\n"); return 1; }
      const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int a = 0; a < r.na; ++a)
        for (int b = 0; b < r.nb; ++b) {
          int c[3] = {r.clo[0], r.clo[1], r.clo[2]};
          c[t1] += a;
          c[t2] += b;
          for (int k = 0; k < 3; ++k)
            if (c[k] < 0 || c[k] >= cp.n[k]) { printf("register cell outside its coarse patch\n"); return 1; }
          if (r.cside != (r.side ? -1 : 1)) { printf("register on the wrong side of its coarse cell\n"); return 1; }
          std::array<int, 6> key{r.fpatch, 2 * d + r.side, cp.lo[0] + c[0], cp.lo[1] + c[1], cp.lo[2] + c[2], 0};
          got[key] += 1;
          all_cells[{cp.lo[0] + c[0], cp.lo[1] + c[1], cp.lo[2] + c[2], 0, 0, 0}] += 1;
          ++nreg;
        }
    }
    for (const RegRect& r : L.regs.boxes) {
      if (r.ordered) continue;
      const HPatch& cp = P[r.cpatch];
      const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int a = 0; a < r.na; ++a)
        for (int b = 0; b < r.nb; ++b) {
          int c[3] = {r.clo[0], r.clo[1], r.clo[2]};
          c[t1] += a;
          c[t2] += b;
          if (all_cells[{cp.lo[0] + c[0], cp.lo[1] + c[1], cp.lo[2] + c[2], 0, 0, 0}] != 1) {
            printf("unordered rectangle shares a cell with another register\n");
            return 1;
          }
        }
    }
    // expected: every coarse cell next to a fine face that no level-l patch covers
    std::map<std::array<int, 6>, int> want;
    for (int i = L.first; i < L.first + L.count; ++i) {
      const HPatch& p = P[i];
      for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int Cd = side ? (p.lo[d] + p.n[d]) / 2 : p.lo[d] / 2 - 1;
          const int Nc = level_n(l - 1, d);
          if (Cd < 0 || Cd >= Nc) {
            if (!periodic(d)) continue;
            Cd = ((Cd % Nc) + Nc) % Nc;
          }
          for (int u = p.lo[t1] / 2; u < (p.lo[t1] + p.n[t1]) / 2; ++u)
            for (int v = p.lo[t2] / 2; v < (p.lo[t2] + p.n[t2]) / 2; ++v) {
              int c[3];
              c[d] = Cd; c[t1] = u; c[t2] = v;
              bool covered = false;
              for (int q = L.first; q < L.first + L.count && !covered; ++q) {
                const HPatch& o = P[q];
                bool in = true;
                for (int k = 0; k < 3 && in; ++k) in = 2 * c[k] >= o.lo[k] && 2 * c[k] < o.lo[k] + o.n[k];
                covered = in;
              }
              if (covered) continue;
              bool held = false;
              for (int q = C.first; q < C.first + C.count && !held; ++q) {
                const HPatch& o = P[q];
                bool in = true;
                for (int k = 0; k < 3 && in; ++k) in = c[k] >= o.lo[k] && c[k] < o.lo[k] + o.n[k];
                held = in;
              }
              if (!held) { printf("coarse cell next to a fine face outside the coarse level\n"); return 1; }
              want[{i, 2 * d + side, c[0], c[1], c[2], 0}] = 1;
            }
        }
    }
    if (got != want) {
      printf("level %d: registers %zu cells, expected %zu\n", l, got.size(), want.size());
      return 1;
    }
  }
  printf("ok %lld\n", nreg);
  return 0;
}

static int check_items() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  TileParams tp;
  if (scanf("%d %d %d", &tp.max_wx, &tp.max_cols, &tp.zchunk) != 3) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, tp) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  long long nitems = 0, nspan = 0;
  for (const LevelPlan& L : plan.levels) {
    for (int pass = 0; pass < 2; ++pass) {   // 0: per-patch items, 1: batched items
      std::vector<std::vector<unsigned char>> cnt(L.count);
      for (int ii = 0; ii < L.count; ++ii) {
        const HPatch& p = P[L.first + ii];
        cnt[ii].assign((size_t)p.n[0] * p.n[1] * p.n[2], 0);
      }
      const std::vector<StageItem>& items = pass ? L.bitems : L.items;
      for (const StageItem& it : items) {
        if (it.wx <= 0 || it.wy <= 0 || it.wz <= 0 || it.wx * it.wy > 256) { printf("bad block shape\n"); return 1; }
        int ox, oy, oz;
        std::vector<int> cand;
        if (it.span >= 0) {
          if (!pass) { printf("spanning block among the per-patch items\n"); return 1; }
          const ItemSpan& S = plan.spans[it.span];
          ox = S.ox; oy = S.oy; oz = S.oz;
          cand.assign(S.patch, S.patch + S.n);
          ++nspan;
        } else {
          const HPatch& q = P[it.patch];
          ox = q.lo[0] + it.x0; oy = q.lo[1] + it.y0; oz = q.lo[2] + it.z0;
          cand.push_back(it.patch);
        }
        for (int ty = 0; ty < it.wy; ++ty)
          for (int tx = 0; tx < it.wx; ++tx) {
            const int gx = ox + tx, gy = oy + ty;
            int qc = -1;
            for (int q : cand) {
              const HPatch& o = P[q];
              if (gx >= o.lo[0] && gx < o.lo[0] + o.n[0] && gy >= o.lo[1] && gy < o.lo[1] + o.n[1]) { qc = q; break; }
            }
            if (qc < 0 || qc < L.first || qc >= L.first + L.count) { printf("block column outside its patches\n"); return 1; }
            const HPatch& o = P[qc];
            if (oz < o.lo[2] || oz + it.wz > o.lo[2] + o.n[2]) { printf("block z range leaves its patch\n"); return 1; }
            for (int z = oz; z < oz + it.wz; ++z)
              cnt[qc - L.first][((size_t)(z - o.lo[2]) * o.n[1] + (gy - o.lo[1])) * o.n[0] + (gx - o.lo[0])] += 1;
          }
        ++nitems;
      }
      for (int ii = 0; ii < L.count; ++ii)
        for (unsigned char c : cnt[ii])
          if (c != 1) {
            printf("%s items: a cell of patch %d covered %d times\n", pass ? "batched" : "per-patch", L.first + ii, c);
            return 1;
          }
    }
  }
  printf("ok %lld %lld\n", nitems, nspan);
  return 0;
}

static int check_gathers() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  auto fdiv = [](int g) { return g >= 0 ? g / 2 : -((1 - g) / 2); };
  long long ncell = 0;
  for (int l = 1; l < (int)plan.levels.size(); ++l) {
    const LevelPlan& L = plan.levels[l];
    std::vector<std::vector<unsigned char>> need(L.count), got(L.count);
    for (int ii = 0; ii < L.count; ++ii) {
      const HPatch& p = P[L.first + ii];
      const size_t tv = (size_t)(p.n[0] / 2 + 4) * (p.n[1] / 2 + 4) * (p.n[2] / 2 + 4);
      need[ii].assign(tv, 0);
      got[ii].assign(tv, 0);
    }
    for (const ProlongBox& b : L.prolong) {
      const HPatch& p = P[b.patch];
      const int ii = b.patch - L.first;
      const int tn[3] = {p.n[0] / 2 + 4, p.n[1] / 2 + 4, p.n[2] / 2 + 4};
      for (int z = b.lo[2]; z < b.lo[2] + b.n[2]; ++z)
        for (int y = b.lo[1]; y < b.lo[1] + b.n[1]; ++y)
          for (int x = b.lo[0]; x < b.lo[0] + b.n[0]; ++x) {
            const int f[3] = {x, y, z};
            int t[3];
            for (int d = 0; d < 3; ++d) t[d] = fdiv(p.lo[d] + f[d]) - (fdiv(p.lo[d]) - 2);
            for (int k = -1; k < 6; ++k) {   // the parent and its six face neighbours
              int u[3] = {t[0], t[1], t[2]};
              if (k >= 0) u[k / 2] += (k & 1) ? 1 : -1;
              for (int d = 0; d < 3; ++d)
                if (u[d] < 0 || u[d] >= tn[d]) { printf("stencil outside the parent tile\n"); return 1; }
              need[ii][((size_t)u[2] * tn[1] + u[1]) * tn[0] + u[0]] = 1;
            }
          }
    }
    for (const CopySeg& s : L.gather_ghost) {
      const HPatch& p = P[s.dst_patch];
      const HPatch& o = P[s.src_patch];
      if (p.level != l || o.level != l - 1) { printf("gather segment on a wrong level\n"); return 1; }
      const int ii = s.dst_patch - L.first;
      const int tn[3] = {p.n[0] / 2 + 4, p.n[1] / 2 + 4, p.n[2] / 2 + 4};
      for (int z = s.dlo[2]; z < s.dlo[2] + s.dn[2]; ++z)
        for (int y = s.dlo[1]; y < s.dlo[1] + s.dn[1]; ++y)
          for (int x = s.dlo[0]; x < s.dlo[0] + s.dn[0]; ++x) {
            const int t[3] = {x, y, z};
            for (int d = 0; d < 3; ++d) {
              if (t[d] < 0 || t[d] >= tn[d]) { printf("gather outside the parent tile\n"); return 1; }
              const int src = s.mode[d] ? s.sh[d] : t[d] + s.sh[d];   // coarse-patch local
              if (src < 0 || src >= o.n[d]) { printf("gather source outside its coarse patch\n"); return 1; }
              const int Nc = bn[d] << (l - 1);
              int G = fdiv(p.lo[d]) - 2 + t[d];   // the coarse cell under tile cell t
              if (G < 0 || G >= Nc) {
                if (cfg.bc[2 * d] == AMR_BC_PERIODIC) G = ((G % Nc) + Nc) % Nc;
                else G = G < 0 ? 0 : Nc - 1;
              }
              if (o.lo[d] + src != G) { printf("gather reads another coarse cell\n"); return 1; }
            }
            got[ii][((size_t)z * tn[1] + y) * tn[0] + x] += 1;
          }
    }
    for (int ii = 0; ii < L.count; ++ii)
      for (size_t c = 0; c < need[ii].size(); ++c) {
        if (got[ii][c] > 1) { printf("a tile cell gathered twice\n"); return 1; }
        if (need[ii][c] && !got[ii][c]) { printf("a needed tile cell not gathered\n"); return 1; }
        ncell += got[ii][c];
      }
  }
  printf("ok %lld\n", ncell);
  return 0;
}

static int check_restrict() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  long long ncell = 0;
  const int np = (int)P.size();
  std::vector<std::vector<unsigned char>> rcnt(np), ccnt(np);
  for (int i = 0; i < np; ++i) {
    rcnt[i].assign((size_t)P[i].n[0] * P[i].n[1] * P[i].n[2], 0);
    ccnt[i].assign(rcnt[i].size(), 0);
  }
  for (int l = 1; l < (int)plan.levels.size(); ++l)
    for (const RestrictSeg& r : plan.levels[l].restrict_segs) {
      const HPatch& f = P[r.fine];
      const HPatch& c = P[r.coarse];
      if (f.level != l || c.level != l - 1) { printf("restriction on a wrong level\n"); return 1; }
      for (int z = r.clo[2]; z < r.clo[2] + r.cn[2]; ++z)
        for (int y = r.clo[1]; y < r.clo[1] + r.cn[1]; ++y)
          for (int x = r.clo[0]; x < r.clo[0] + r.cn[0]; ++x) {
            const int cc[3] = {x, y, z};
            for (int d = 0; d < 3; ++d) {
              if (cc[d] < 0 || cc[d] >= c.n[d]) { printf("restricted cell outside its coarse patch\n"); return 1; }
              const int g = 2 * (c.lo[d] + cc[d]);   // first child, level l
              if (g < f.lo[d] || g + 2 > f.lo[d] + f.n[d]) { printf("children outside the fine patch\n"); return 1; }
            }
            rcnt[r.coarse][((size_t)z * c.n[1] + y) * c.n[0] + x] += 1;
          }
    }
  for (int i = 0; i < np; ++i)
    for (int e = plan.cover_first[i]; e < plan.cover_first[i + 1]; ++e) {
      const CoverBox& b = plan.cover[e];
      const HPatch& c = P[i];
      for (int z = b.lo[2]; z < b.lo[2] + b.n[2]; ++z)
        for (int y = b.lo[1]; y < b.lo[1] + b.n[1]; ++y)
          for (int x = b.lo[0]; x < b.lo[0] + b.n[0]; ++x) ccnt[i][((size_t)z * c.n[1] + y) * c.n[0] + x] += 1;
    }
  for (int i = 0; i < np; ++i) {
    const HPatch& c = P[i];
    for (int z = 0; z < c.n[2]; ++z)
      for (int y = 0; y < c.n[1]; ++y)
        for (int x = 0; x < c.n[0]; ++x) {
          // covered: some patch one level finer holds the cell's first child
          bool covered = false;
          for (int q = 0; q < np && !covered; ++q) {
            const HPatch& f = P[q];
            if (f.level != c.level + 1) continue;
            const int g[3] = {2 * (c.lo[0] + x), 2 * (c.lo[1] + y), 2 * (c.lo[2] + z)};
            bool in = true;
            for (int d = 0; d < 3 && in; ++d) in = g[d] >= f.lo[d] && g[d] < f.lo[d] + f.n[d];
            covered = in;
          }
          const size_t k = ((size_t)z * c.n[1] + y) * c.n[0] + x;
          if (rcnt[i][k] != (covered ? 1 : 0)) { printf("patch %d: a coarse cell restricted %d times\n", i, rcnt[i][k]); return 1; }
          if (ccnt[i][k] != (covered ? 1 : 0)) { printf("patch %d: a coverage box count %d\n", i, ccnt[i][k]); return 1; }
          ncell += covered ? 1 : 0;
        }
  }
  printf("ok %lld\n", ncell);
  return 0;
}

static int check_faces() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  const int np = (int)P.size();
  std::vector<std::pair<int64_t, int>> starts(np);   // (arena offset, patch), ascending
  for (int i = 0; i < np; ++i) starts[i] = {plan.desc[i].off, i};
  std::sort(starts.begin(), starts.end());
  long long ndirect = 0;
  for (int i = 0; i < np; ++i) {
    const PatchDesc& D = plan.desc[i];
    const HPatch& p = P[i];
    const int64_t own = D.off + ((int64_t)kGhost * D.m1 + kGhost) * D.pitch + kGhost;
    for (int f = 0; f < 6; ++f) {
      const FaceSrc& fs = D.face[f];
      if (fs.base == own && fs.sx == 1 && fs.sy == D.pitch && fs.sz == D.pitch * D.m1) continue;   // own ghosts
      ++ndirect;
      const int d = f / 2, side = f % 2, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int g = 0; g < kGhost; ++g)
        for (int b = 0; b < p.n[t2]; ++b)
          for (int a = 0; a < p.n[t1]; ++a) {
            int c[3];
            c[d] = side ? p.n[d] + g : -1 - g;
            c[t1] = a;
            c[t2] = b;
            const int64_t o = fs.base + (int64_t)c[0] * fs.sx + (int64_t)c[1] * fs.sy + (int64_t)c[2] * fs.sz;
            auto it = std::upper_bound(starts.begin(), starts.end(), std::make_pair(o, np));
            if (it == starts.begin()) { printf("face entry points before the arena\n"); return 1; }
            const int q = std::prev(it)->second;
            const PatchDesc& Q = plan.desc[q];
            const int64_t idx = o - Q.off;
            if (idx >= Q.vstride) { printf("face entry points past a patch\n"); return 1; }
            const int lz = (int)(idx / ((int64_t)Q.pitch * Q.m1)) - kGhost;
            const int ly = (int)((idx / Q.pitch) % Q.m1) - kGhost;
            const int lx = (int)(idx % Q.pitch) - kGhost;
            const int l[3] = {lx, ly, lz};
            for (int k = 0; k < 3; ++k)
              if (l[k] < 0 || l[k] >= P[q].n[k]) { printf("face entry reads a ghost cell\n"); return 1; }
            if (P[q].level != p.level || fs.vs != (int)Q.vstride) { printf("face source of another level\n"); return 1; }
            for (int k = 0; k < 3; ++k) {
              const int N = bn[k] << p.level;
              int G = p.lo[k] + c[k];
              if (G < 0 || G >= N) {
                if (cfg.bc[2 * k] == AMR_BC_PERIODIC) G = ((G % N) + N) % N;
                else G = G < 0 ? 0 : N - 1;   // outflow: the boundary cell of the patch itself
              }
              if (P[q].lo[k] + l[k] != G) { printf("patch %d face %d reads another position\n", i, f); return 1; }
            }
          }
    }
  }
  printf("ok %lld\n", ndirect);
  return 0;
}

static int check_flat() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  if (!read_config(cfg, bn, ml, P)) return 2;
  Plan plan;
  std::string msg;
  if (build_plan(cfg, P, plan, msg, TileParams()) != AMR_OK) {
    printf("plan failed: %s\n", msg.c_str());
    return 1;
  }
  auto fdiv = [](int g) { return g >= 0 ? g / 2 : -((1 - g) / 2); };
  long long nb = 0;
  for (const LevelPlan& L : plan.levels) {
    if (L.fprolong.boxes.size() != L.prolong.size()) { printf("flattened prolongation list length\n"); return 1; }
    for (size_t k = 0; k < L.prolong.size(); ++k) {
      const ProlongBox& b = L.prolong[k];
      const FlatProlong& g = L.fprolong.boxes[k];
      const PatchDesc& D = plan.desc[b.patch];
      const int np2 = L.fprolong.first[k + 1] - L.fprolong.first[k];
      if (np2 % (g.np0 * g.np1) != 0) { printf("parent count not a whole number of planes\n"); return 1; }
      std::map<int64_t, int> written;   // arena index -> times
      for (int q = 0; q < np2; ++q) {   // as box_prolong_kernel: q -> (pa, pb, pc)
        const int r = q / g.np0, pa = q - r * g.np0, pc = r / g.np1, pb = r - pc * g.np1;
        const int a0 = 2 * pa - (g.odd & 1), b0 = 2 * pb - ((g.odd >> 1) & 1), c0 = 2 * pc - ((g.odd >> 2) & 1);
        const int64_t tile = g.tp0 + pa + (int64_t)pb * g.tsy + (int64_t)pc * g.tsz;
        for (int kz = 0; kz < 2; ++kz)
          for (int jy = 0; jy < 2; ++jy)
            for (int ix = 0; ix < 2; ++ix) {
              const int a = a0 + ix, bb = b0 + jy, c = c0 + kz;
              if (a < 0 || a >= g.n[0] || bb < 0 || bb >= g.n[1] || c < 0 || c >= g.n[2]) continue;
              const int f[3] = {b.lo[0] + a, b.lo[1] + bb, b.lo[2] + c};   // fine cell, patch local
              const int64_t di = g.dst0 + a + (int64_t)bb * g.dsy + (int64_t)c * g.dsz;
              if (di != D.off + cell_index(D, f[0], f[1], f[2])) { printf("prolongation writes another cell\n"); return 1; }
              int t[3];
              for (int d = 0; d < 3; ++d) t[d] = fdiv(D.lo[d] + f[d]) - (fdiv(D.lo[d]) - 2);
              const int64_t want = D.tile_off + t[0] + (int64_t)t[1] * D.tn[0] + (int64_t)t[2] * D.tn[0] * D.tn[1];
              if (tile != want) { printf("prolongation reads another parent\n"); return 1; }
              written[di] += 1;
            }
      }
      if ((int64_t)written.size() != (int64_t)b.n[0] * b.n[1] * b.n[2]) { printf("prolongation box cells missed\n"); return 1; }
      for (auto& w : written)
        if (w.second != 1) { printf("prolongation writes a cell twice\n"); return 1; }
      ++nb;
    }
    // ghost copies: the flattened box's source and destination of every cell
    if (L.fghost_all.boxes.size() != L.ghost.size()) { printf("flattened ghost list length\n"); return 1; }
    for (size_t k = 0; k < L.ghost.size(); ++k) {
      const CopySeg& sgm = L.ghost[k];
      const FlatCopy& c = L.fghost_all.boxes[k];
      const PatchDesc& D = plan.desc[sgm.dst_patch];
      const PatchDesc& S = plan.desc[sgm.src_patch];
      for (int z = 0; z < sgm.dn[2]; ++z)
        for (int y = 0; y < sgm.dn[1]; ++y)
          for (int x = 0; x < sgm.dn[0]; ++x) {
            const int dl[3] = {sgm.dlo[0] + x, sgm.dlo[1] + y, sgm.dlo[2] + z};
            int sl[3];
            for (int d = 0; d < 3; ++d) sl[d] = sgm.mode[d] ? sgm.sh[d] : dl[d] + sgm.sh[d];
            const int64_t di = c.dst0 + x + (int64_t)y * c.dsy + (int64_t)z * c.dsz;
            const int64_t si = c.src0 + (int64_t)x * c.ssx + (int64_t)y * c.ssy + (int64_t)z * c.ssz;
            if (di != D.off + cell_index(D, dl[0], dl[1], dl[2]) || si != S.off + cell_index(S, sl[0], sl[1], sl[2])) {
              printf("flattened ghost copy moves another cell\n");
              return 1;
            }
          }
      if (c.dvs != (int)D.vstride || c.svs != (int)S.vstride) { printf("flattened ghost copy variable stride\n"); return 1; }
      ++nb;
    }
  }
  printf("ok %lld\n", nb);
  return 0;
}

static int run_cluster() {
  int bn[3], ml;
  amr_config cfg;
  std::vector<HPatch> P;
  int bc[6];
  RegridParams rp;
  if (scanf("%d %d %d %d %d %d %d %d %d %d", &bn[0], &bn[1], &bn[2], &ml, &bc[0], &bc[1], &bc[2], &bc[3], &bc[4],
            &bc[5]) != 10)
    return 2;
  if (scanf("%d %d %d %d", &rp.buffer, &rp.block, &rp.max_patch, &rp.min_level) != 4) return 2;
  if (!read_list(P)) return 2;
  cfg = amr_config{};
  cfg.nvar = 5;
  cfg.precision = AMR_FP32;
  cfg.gamma = 1.4;
  cfg.theta = 1.5;
  cfg.cfl = 0.4;
  cfg.ref_ratio = 2;
  for (int d = 0; d < 3; ++d) {
    cfg.base_n[d] = bn[d];
    cfg.domain_lo[d] = 0;
    cfg.domain_hi[d] = 1;
  }
  for (int f = 0; f < 6; ++f) cfg.bc[f] = bc[f];
  cfg.max_level = ml;
  std::vector<std::vector<uint8_t>> flags(P.size());
  for (size_t i = 0; i < P.size(); ++i) {
    int has = 0;
    if (scanf("%d", &has) != 1) return 2;
    if (!has) continue;
    flags[i].resize((size_t)P[i].n[0] * P[i].n[1] * P[i].n[2]);
    for (auto& f : flags[i]) {
      int v;
      if (scanf("%d", &v) != 1) return 2;
      f = (uint8_t)v;
    }
  }
  std::vector<HPatch> out;
  std::string msg;
  if (cluster_patches(cfg, P, flags, rp, out, msg) != AMR_OK) {
    printf("cluster failed: %s\n", msg.c_str());
    return 1;
  }
  printf("ok %zu\n", out.size());
  for (const HPatch& p : out) printf("%d %d %d %d %d %d %d\n", p.level, p.lo[0], p.lo[1], p.lo[2], p.n[0], p.n[1], p.n[2]);
  return 0;
}

int main() {
  char mode[16] = {0};
  if (scanf("%15s", mode) != 1) return 2;
  if (std::string(mode) == "ghost") return check_ghost();
  if (std::string(mode) == "registers") return check_registers();
  if (std::string(mode) == "items") return check_items();
  if (std::string(mode) == "gathers") return check_gathers();
  if (std::string(mode) == "restrict") return check_restrict();
  if (std::string(mode) == "faces") return check_faces();
  if (std::string(mode) == "flat") return check_flat();
  if (std::string(mode) == "cluster") return run_cluster();
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
