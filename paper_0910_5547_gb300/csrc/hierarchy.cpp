// hierarchy.cpp -- host planner for the AMR patch hierarchy (Sec. 3:
// Berger-Colella block-structured refinement, each grid an IBVP).  Builds the
// launch tables of every kernel from the patch list.  No CUDA calls.
#include "hierarchy.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <set>
#include <tuple>
#include <memory>
#include <array>
#include <thread>
#include <mutex>
#include <condition_variable>
#include <functional>
#include <unistd.h>
#include <atomic>
#include <climits>
#include <unordered_map>
#include <unordered_set>

namespace amr {

namespace {

int level_n(const amr_config& c, int l, int d) { return c.base_n[d] << l; }
bool periodic(const amr_config& c, int d) { return c.bc[2 * d] == AMR_BC_PERIODIC; }
int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

std::string fmt(const char* f, int a = 0, int b = 0, int c = 0, int d = 0) {
  char buf[256];
  std::snprintf(buf, sizeof buf, f, a, b, c, d);
  return buf;
}

bool boxes_overlap(const HPatch& a, const HPatch& b) {
  for (int d = 0; d < 3; ++d)
    if (a.lo[d] + a.n[d] <= b.lo[d] || b.lo[d] + b.n[d] <= a.lo[d]) return false;
  return true;
}

// Intervals [lo, hi) of axis d at level l after periodic wrap / clipping at outflow faces.
std::vector<std::pair<int, int>> wrap_interval(const amr_config& c, int l, int d, int lo, int hi) {
  int N = level_n(c, l, d);
  std::vector<std::pair<int, int>> out;
  if (!periodic(c, d)) {
    lo = std::max(lo, 0);
    hi = std::min(hi, N);
    if (lo < hi) out.push_back({lo, hi});
    return out;
  }
  if (hi - lo >= N) {
    out.push_back({0, N});
    return out;
  }
  int a = ((lo % N) + N) % N;
  int len = hi - lo;
  if (a + len <= N) {
    out.push_back({a, a + len});
  } else {
    out.push_back({a, N});
    out.push_back({0, a + len - N});
  }
  return out;
}

// Decompose the cells with mask == 0 of an A x B grid into rectangles
// (row runs merged across consecutive rows with identical extent).
struct Rect { int a0, na, b0, nb; };
void mask_rects(const unsigned char* m, int A, int B, std::vector<Rect>& done) {
  done.clear();
  // runs of the previous row that are still open: (a0, na, index into done)
  thread_local std::vector<std::array<int, 3>> open, next;
  open.clear();
  for (int b = 0; b < B; ++b) {
    next.clear();
    size_t oi = 0;   // open runs are in increasing a0 order, like the runs of this row
    int a = 0;
    while (a < A) {
      if (m[(size_t)b * A + a]) { ++a; continue; }
      int s = a;
      while (a < A && !m[(size_t)b * A + a]) ++a;
      while (oi < open.size() && open[oi][0] < s) ++oi;
      if (oi < open.size() && open[oi][0] == s && open[oi][1] == a - s) {
        done[open[oi][2]].nb += 1;
        next.push_back(open[oi]);
      } else {
        done.push_back({s, a - s, b, 1});
        next.push_back({s, a - s, (int)done.size() - 1});
      }
    }
    open.swap(next);
  }
}
std::vector<Rect> mask_rects(const unsigned char* m, int A, int B) {
  std::vector<Rect> done;
  mask_rects(m, A, B, done);
  return done;
}
std::vector<Rect> mask_rects(const std::vector<unsigned char>& m, int A, int B) { return mask_rects(m.data(), A, B); }

// Disjoint boxes covering the cells with need != 0 of an n0 x n1 x n2 grid:
// rectangles of each z slice, merged across consecutive slices with identical
// rectangles.
struct Box3 { int lo[3], n[3]; };
std::vector<Box3> need_boxes(const std::vector<unsigned char>& need, int n0, int n1, int n2) {
  std::vector<Box3> done;
  std::vector<std::pair<Rect, int>> open, next;
  std::vector<unsigned char> inv((size_t)n0 * n1);
  std::vector<Rect> rects;
  for (int z = 0; z < n2; ++z) {
    for (size_t e = 0; e < inv.size(); ++e) inv[e] = need[(size_t)z * n0 * n1 + e] ? 0 : 1;
    next.clear();
    mask_rects(inv.data(), n0, n1, rects);
    for (const Rect& r : rects) {
      int hit = -1;
      for (const auto& o : open)
        if (o.first.a0 == r.a0 && o.first.na == r.na && o.first.b0 == r.b0 && o.first.nb == r.nb) hit = o.second;
      if (hit >= 0) {
        done[hit].n[2] += 1;
      } else {
        done.push_back({{r.a0, r.b0, z}, {r.na, r.nb, 1}});
        hit = (int)done.size() - 1;
      }
      next.push_back({r, hit});
    }
    open.swap(next);
  }
  return done;
}

// Persistent worker threads for the planner's parallel loops (spawning threads
// per loop costs a few hundred microseconds, and a rebuild runs dozens of loops).
// A job is f(i) for i in [0, n), grabbed in chunks of 8 by the caller and the
// workers.  run() returns false (the caller then loops serially) when called
// from inside a job, while another thread's job is running, or in a child
// process forked after the workers started.
class WorkerPool {
 public:
  static WorkerPool& instance() {
    static WorkerPool pool;
    return pool;
  }
  bool run(int n, const std::function<void(int)>& f, int grain = 8) {
    if (inside_ || nt_ <= 1 || getpid() != pid_) return false;
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &f;
      n_ = n;
      grain_ = grain;
      next_.store(0);
      pending_ = (int)threads_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
    return true;
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_)
      if (t.joinable()) t.join();
  }

 private:
  WorkerPool() : pid_(getpid()) {
    nt_ = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u);
    for (int t = 1; t < nt_; ++t) threads_.emplace_back([this] { loop(); });
  }
  void work() {
    inside_ = true;
    for (;;) {
      const int i0 = next_.fetch_add(grain_);
      if (i0 >= n_) break;
      const int i1 = std::min(i0 + grain_, n_);
      for (int i = i0; i < i1; ++i) (*job_)(i);
    }
    inside_ = false;
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lk(m_);
      cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      lk.unlock();
      work();
      lk.lock();
      if (--pending_ == 0) done_.notify_one();
    }
  }
  static thread_local bool inside_;
  const pid_t pid_;
  int nt_ = 1;
  std::vector<std::thread> threads_;
  std::mutex busy_, m_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* job_ = nullptr;
  int n_ = 0;
  int grain_ = 8;
  std::atomic<int> next_{0};
  int pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};
thread_local bool WorkerPool::inside_ = false;

// f(i) for i in [0, n) on the host's cores; every caller writes only to slot i
// of its outputs, so the result does not depend on the thread count.
template <class F>
void parallel_for(int n, F&& f) {
  if (n >= 64) {
    const std::function<void(int)> job = [&](int i) { f(i); };
    if (WorkerPool::instance().run(n, job)) return;
  }
  for (int i = 0; i < n; ++i) f(i);
}

// A few large independent tasks, handed out one at a time.
template <class F>
void parallel_tasks(int n, F&& f) {
  if (n >= 2) {
    const std::function<void(int)> job = [&](int i) { f(i); };
    if (WorkerPool::instance().run(n, job, 1)) return;
  }
  for (int i = 0; i < n; ++i) f(i);
}

// Bucket index of the patches of one level: a query returns the patches whose
// box intersects a box (each patch listed once, ascending), so neighbour
// searches cost O(neighbours) instead of O(patches).  Buckets form a dense
// grid over the patches' bounding box (cells of edge bs_, bs_ doubled until
// the grid has at most 4M buckets), stored as CSR.
class PatchIndex {
 public:
  PatchIndex(const std::vector<HPatch>& P, int first, int count, int bs = 32) : P_(P), bs_(bs) {
    if (count <= 0) {
      for (int d = 0; d < 3; ++d) { g0_[d] = 0; gn_[d] = 1; }
      start_.assign(2, 0);
      return;
    }
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int i = first; i < first + count; ++i)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], P[i].lo[d]);
        hi[d] = std::max(hi[d], P[i].lo[d] + P[i].n[d]);
      }
    for (;;) {
      int64_t nbk = 1;
      for (int d = 0; d < 3; ++d) {
        g0_[d] = fl(lo[d]);
        gn_[d] = fl(hi[d] - 1) - g0_[d] + 1;
        nbk *= gn_[d];
      }
      if (nbk <= (int64_t)1 << 22) break;
      bs_ *= 2;
    }
    const size_t nbk = (size_t)gn_[0] * gn_[1] * gn_[2];
    start_.assign(nbk + 1, 0);
    auto each_bucket = [&](const HPatch& p, auto&& f) {
      for (int z = fl(p.lo[2]); z <= fl(p.lo[2] + p.n[2] - 1); ++z)
        for (int y = fl(p.lo[1]); y <= fl(p.lo[1] + p.n[1] - 1); ++y)
          for (int x = fl(p.lo[0]); x <= fl(p.lo[0] + p.n[0] - 1); ++x) f(bucket(x, y, z));
    };
    for (int i = first; i < first + count; ++i) each_bucket(P[i], [&](size_t k) { start_[k + 1]++; });
    for (size_t k = 0; k < nbk; ++k) start_[k + 1] += start_[k];
    items_.resize(start_[nbk]);
    std::vector<int> fillp(start_.begin(), start_.end() - 1);
    for (int i = first; i < first + count; ++i) each_bucket(P[i], [&](size_t k) { items_[fillp[k]++] = i; });
  }
  // patches intersecting [lo, hi) (no periodic images), ascending patch order;
  // const and safe to call from several threads
  void query(const int lo[3], const int hi[3], std::vector<int>& out) const {
    out.clear();
    if (lo[0] >= hi[0] || lo[1] >= hi[1] || lo[2] >= hi[2] || items_.empty()) return;
    int b0[3], b1[3];
    for (int d = 0; d < 3; ++d) {
      b0[d] = std::max(fl(lo[d]) - g0_[d], 0);
      b1[d] = std::min(fl(hi[d] - 1) - g0_[d], gn_[d] - 1);
      if (b0[d] > b1[d]) return;
    }
    for (int z = b0[2]; z <= b1[2]; ++z)
      for (int y = b0[1]; y <= b1[1]; ++y)
        for (int x = b0[0]; x <= b1[0]; ++x) {
          const size_t k = ((size_t)z * gn_[1] + y) * gn_[0] + x;
          for (int e = start_[k]; e < start_[k + 1]; ++e) {
            const int i = items_[e];
            const HPatch& p = P_[i];
            bool hit = true;
            for (int d = 0; d < 3 && hit; ++d) hit = p.lo[d] < hi[d] && lo[d] < p.lo[d] + p.n[d];
            if (hit) out.push_back(i);
          }
        }
    // one bucket: its patches are listed once each, in ascending order already
    if (b0[0] == b1[0] && b0[1] == b1[1] && b0[2] == b1[2]) return;
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  }

 private:
  int fl(int c) const { return c >= 0 ? c / bs_ : -((-c + bs_ - 1) / bs_); }
  size_t bucket(int x, int y, int z) const {
    return ((size_t)(z - g0_[2]) * gn_[1] + (y - g0_[1])) * gn_[0] + (x - g0_[0]);
  }
  const std::vector<HPatch>& P_;
  int bs_;
  int g0_[3], gn_[3];
  std::vector<int> start_, items_;
};

// Split boxes with more than `maxc` cells along their longest axis so that
// one CTA per box keeps the GPU busy for large patches.
constexpr int kMaxBoxCells = 4096;

void split_copy(std::vector<CopySeg>& v, size_t from) {
  bool any = false;   // nothing to split (the common case): keep v as it is
  for (size_t i = from; i < v.size() && !any; ++i) any = v[i].dn[0] * v[i].dn[1] * v[i].dn[2] > kMaxBoxCells;
  if (!any) return;
  std::vector<CopySeg> out(v.begin(), v.begin() + from);
  for (size_t i = from; i < v.size(); ++i) {
    if (v[i].dn[0] * v[i].dn[1] * v[i].dn[2] <= kMaxBoxCells) { out.push_back(v[i]); continue; }
    std::vector<CopySeg> work{v[i]};
    while (!work.empty()) {
      CopySeg s = work.back();
      work.pop_back();
      int vol = s.dn[0] * s.dn[1] * s.dn[2];
      if (vol <= kMaxBoxCells) { out.push_back(s); continue; }
      int k = 0;
      for (int a = 1; a < 3; ++a) if (s.dn[a] > s.dn[k]) k = a;
      CopySeg a = s, b = s;
      a.dn[k] = (int16_t)(s.dn[k] / 2);
      b.dn[k] = (int16_t)(s.dn[k] - a.dn[k]);
      b.dlo[k] = (int16_t)(s.dlo[k] + a.dn[k]);
      work.push_back(b);
      work.push_back(a);
    }
  }
  v.swap(out);
}

void split_prolong(std::vector<ProlongBox>& v, size_t from) {
  bool any = false;   // nothing to split (the common case): keep v as it is
  for (size_t i = from; i < v.size() && !any; ++i) any = v[i].n[0] * v[i].n[1] * v[i].n[2] > kMaxBoxCells;
  if (!any) return;
  std::vector<ProlongBox> out(v.begin(), v.begin() + from);
  for (size_t i = from; i < v.size(); ++i) {
    if (v[i].n[0] * v[i].n[1] * v[i].n[2] <= kMaxBoxCells) { out.push_back(v[i]); continue; }
    std::vector<ProlongBox> work{v[i]};
    while (!work.empty()) {
      ProlongBox s = work.back();
      work.pop_back();
      if (s.n[0] * s.n[1] * s.n[2] <= kMaxBoxCells) { out.push_back(s); continue; }
      int k = 0;
      for (int a = 1; a < 3; ++a) if (s.n[a] > s.n[k]) k = a;
      ProlongBox a = s, b = s;
      a.n[k] = (int16_t)((s.n[k] / 2 + 1) & ~1);   // even: no parent cell split between the halves
      b.n[k] = (int16_t)(s.n[k] - a.n[k]);
      b.lo[k] = (int16_t)(s.lo[k] + a.n[k]);
      work.push_back(b);
      work.push_back(a);
    }
  }
  v.swap(out);
}

void split_restrict(std::vector<RestrictSeg>& v) {
  std::vector<RestrictSeg> out;
  out.reserve(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    if (v[i].cn[0] * v[i].cn[1] * v[i].cn[2] <= kMaxBoxCells / 2) { out.push_back(v[i]); continue; }
    std::vector<RestrictSeg> work{v[i]};
    while (!work.empty()) {
      RestrictSeg s = work.back();
      work.pop_back();
      if (s.cn[0] * s.cn[1] * s.cn[2] <= kMaxBoxCells / 2) { out.push_back(s); continue; }
      int k = 0;
      for (int a = 1; a < 3; ++a) if (s.cn[a] > s.cn[k]) k = a;
      RestrictSeg a = s, b = s;
      a.cn[k] = (int16_t)(s.cn[k] / 2);
      b.cn[k] = (int16_t)(s.cn[k] - a.cn[k]);
      b.clo[k] = (int16_t)(s.clo[k] + a.cn[k]);
      work.push_back(b);
      work.push_back(a);
    }
  }
  v.swap(out);
}

}  // namespace

amr_status validate_config(const amr_config& c, std::string& msg) {
  if (c.nvar != 5 && c.nvar != 9) { msg = "nvar must be 5 (Euler) or 9 (GLM-MHD)"; return AMR_ERR_ARG; }
  if (c.precision != AMR_FP64 && c.precision != AMR_FP32) { msg = "precision must be AMR_FP64 or AMR_FP32"; return AMR_ERR_ARG; }
  if (c.riemann != AMR_HLL && c.riemann != AMR_LLF && c.riemann != AMR_FLUXREC) {
    msg = "riemann must be AMR_HLL, AMR_LLF or AMR_FLUXREC";
    return AMR_ERR_ARG;
  }
  if (c.riemann == AMR_FLUXREC && c.nvar != 5) { msg = "AMR_FLUXREC is for the Euler system (nvar 5)"; return AMR_ERR_ARG; }
  if (c.recon != AMR_PLM && c.recon != AMR_WENO3) { msg = "recon must be AMR_PLM or AMR_WENO3"; return AMR_ERR_ARG; }
  if (c.item_span != AMR_SPAN_LAYERS && c.item_span != AMR_SPAN_PATCH) {
    msg = "item_span must be AMR_SPAN_LAYERS or AMR_SPAN_PATCH";
    return AMR_ERR_ARG;
  }
  if (c.ghost_fill != AMR_GHOST_DIRECT && c.ghost_fill != AMR_GHOST_COPY) {
    msg = "ghost_fill must be AMR_GHOST_DIRECT or AMR_GHOST_COPY";
    return AMR_ERR_ARG;
  }
  if (c.recon == AMR_WENO3 && c.riemann == AMR_FLUXREC) {
    msg = "AMR_WENO3 reconstructs the states of an AMR_HLL / AMR_LLF solve, not split fluxes";
    return AMR_ERR_ARG;
  }
  if (!(c.gamma > 1.0) || !std::isfinite(c.gamma)) { msg = "gamma must be > 1"; return AMR_ERR_ARG; }
  if (!(c.theta >= 0.0 && c.theta <= 2.0)) { msg = "theta must lie in [0, 2]"; return AMR_ERR_ARG; }
  if (!(c.cfl > 0.0 && c.cfl <= 1.0)) { msg = "cfl must lie in (0, 1]"; return AMR_ERR_ARG; }
  if (c.max_level < 0 || c.max_level > 12) { msg = "max_level must lie in [0, 12]"; return AMR_ERR_ARG; }
  if (c.ref_ratio != 0 && c.ref_ratio != 2) { msg = "only refinement ratio 2 is supported"; return AMR_ERR_ARG; }
  for (int d = 0; d < 3; ++d) {
    if (c.base_n[d] < 1 || c.base_n[d] > 4096) { msg = "base_n must lie in [1, 4096]"; return AMR_ERR_ARG; }
    if ((int64_t)c.base_n[d] << c.max_level > (1 << 24)) { msg = "base_n * 2^max_level too large"; return AMR_ERR_ARG; }
    if (!(c.domain_hi[d] > c.domain_lo[d]) || !std::isfinite(c.domain_hi[d] - c.domain_lo[d])) {
      msg = "domain_hi must exceed domain_lo"; return AMR_ERR_ARG;
    }
    for (int s = 0; s < 2; ++s)
      if (c.bc[2 * d + s] != AMR_BC_OUTFLOW && c.bc[2 * d + s] != AMR_BC_PERIODIC) { msg = "bad boundary code"; return AMR_ERR_ARG; }
    if ((c.bc[2 * d] == AMR_BC_PERIODIC) != (c.bc[2 * d + 1] == AMR_BC_PERIODIC)) {
      msg = "periodic boundaries must be set on both faces of an axis"; return AMR_ERR_ARG;
    }
  }
  if (c.batched != 0 && c.batched != 1) { msg = "batched must be 0 or 1"; return AMR_ERR_ARG; }
  if (c.nvar == 9 && c.ch > 0.0 && !std::isfinite(c.ch)) { msg = "ch must be finite"; return AMR_ERR_ARG; }
  if (!(c.p_floor >= 0.0) || !std::isfinite(c.p_floor)) { msg = "p_floor must be finite and >= 0"; return AMR_ERR_ARG; }
  if (!(c.glm_alpha >= 0.0) || !std::isfinite(c.glm_alpha)) { msg = "glm_alpha must be finite and >= 0"; return AMR_ERR_ARG; }
  return AMR_OK;
}

amr_status validate_patches(const amr_config& c, const std::vector<HPatch>& P, std::string& msg) {
  amr_status st = validate_config(c, msg);
  if (st != AMR_OK) return st;
  if (P.empty()) { msg = "no patches"; return AMR_ERR_ARG; }
  int maxl = 0;
  for (size_t i = 0; i < P.size(); ++i) {
    const HPatch& p = P[i];
    if (p.level < 0 || p.level > c.max_level) { msg = fmt("patch %d: level %d outside [0, max_level]", (int)i, p.level); return AMR_ERR_ARG; }
    if (i > 0 && p.level < P[i - 1].level) { msg = fmt("patch %d: patches must be sorted by level", (int)i); return AMR_ERR_ARG; }
    maxl = std::max(maxl, p.level);
    for (int d = 0; d < 3; ++d) {
      if (p.n[d] < 2 || p.n[d] > 1024) { msg = fmt("patch %d: size %d outside [2, 1024] on axis %d", (int)i, p.n[d], d); return AMR_ERR_ARG; }
      if (p.lo[d] < 0 || p.lo[d] + p.n[d] > level_n(c, p.level, d)) {
        msg = fmt("patch %d: outside the level-%d domain on axis %d", (int)i, p.level, d); return AMR_ERR_NESTING;
      }
      if ((int64_t)(p.n[0] + 4) * (p.n[1] + 4) * (p.n[2] + 4) * c.nvar > (int64_t)1 << 30) {
        msg = fmt("patch %d: ghosted size times nvar exceeds 2^30 cells", (int)i); return AMR_ERR_ARG;
      }
      if (p.level > 0 && ((p.lo[d] & 1) || (p.n[d] & 1))) {
        msg = fmt("patch %d: refined patches need even lo and n (axis %d)", (int)i, d); return AMR_ERR_NESTING;
      }
    }
  }
  std::vector<int> first(maxl + 2, 0);
  for (const HPatch& p : P) first[p.level + 1]++;
  for (int l = 0; l <= maxl; ++l) {
    if (first[l + 1] == 0) { msg = fmt("level %d has no patches", l); return AMR_ERR_NESTING; }
    first[l + 1] += first[l];
  }
  // no same-level overlap (patches checked in parallel; the first failing one
  // in patch order is reported)
  for (int l = 0; l <= maxl; ++l) {
    PatchIndex ix(P, first[l], first[l + 1] - first[l]);
    const int n = first[l + 1] - first[l];
    std::vector<int> hit(n, -1);
    parallel_for(n, [&](int k) {
      const int a = first[l] + k;
      std::vector<int> cand;
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) { lo[d] = P[a].lo[d]; hi[d] = P[a].lo[d] + P[a].n[d]; }
      ix.query(lo, hi, cand);
      for (int b : cand)
        if (b != a && boxes_overlap(P[a], P[b])) {
          hit[k] = b;
          return;
        }
    });
    for (int k = 0; k < n; ++k)
      if (hit[k] >= 0) {
        const int a = first[l] + k, b = hit[k];
        msg = fmt("patches %d and %d overlap on level %d", std::min(a, b), std::max(a, b), l);
        return AMR_ERR_NESTING;
      }
  }
  // level 0 tiles the domain
  int64_t vol0 = 0;
  for (int i = first[0]; i < first[1]; ++i) vol0 += (int64_t)P[i].n[0] * P[i].n[1] * P[i].n[2];
  if (vol0 != (int64_t)c.base_n[0] * c.base_n[1] * c.base_n[2]) {
    msg = "level-0 patches must tile the whole domain"; return AMR_ERR_NESTING;
  }
  // proper nesting: footprint grown by two parent cells is covered by the parent level
  for (int l = 1; l <= maxl; ++l) {
    PatchIndex cix(P, first[l - 1], first[l] - first[l - 1]);
    const int n = first[l + 1] - first[l];
    std::vector<unsigned char> bad(n, 0);
    parallel_for(n, [&](int k) {
      const int i = first[l] + k;
      std::vector<int> cand;
      const HPatch& p = P[i];
      std::vector<std::pair<int, int>> iv[3];
      int64_t need = 1;
      for (int d = 0; d < 3; ++d) {
        iv[d] = wrap_interval(c, l - 1, d, p.lo[d] / 2 - 2, (p.lo[d] + p.n[d]) / 2 + 2);
        int64_t len = 0;
        for (auto& q : iv[d]) len += q.second - q.first;
        need *= len;
      }
      int64_t got = 0;
      // candidate parents: patches meeting the bounding box of the wrapped pieces
      int blo[3], bhi[3];
      for (int d = 0; d < 3; ++d) {
        blo[d] = INT32_MAX; bhi[d] = INT32_MIN;
        for (auto& r : iv[d]) { blo[d] = std::min(blo[d], r.first); bhi[d] = std::max(bhi[d], r.second); }
      }
      cix.query(blo, bhi, cand);
      for (int q : cand) {
        const HPatch& o = P[q];
        int64_t v = 1;
        for (int d = 0; d < 3 && v; ++d) {
          int64_t len = 0;
          for (auto& r : iv[d]) {
            int a = std::max(r.first, o.lo[d]), b = std::min(r.second, o.lo[d] + o.n[d]);
            if (a < b) len += b - a;
          }
          v *= len;
        }
        got += v;
      }
      bad[k] = got != need;
    });
    for (int k = 0; k < n; ++k)
      if (bad[k]) {
        msg = fmt("patch %d (level %d) is not properly nested: its footprint grown by 2 parent cells "
                  "is not covered by level %d", first[l] + k, l, l - 1);
        return AMR_ERR_NESTING;
      }
  }
  return AMR_OK;
}

void build_items(Plan& plan, const TileParams& tp) {
  const int max_cols = tp.max_cols > 0 ? std::min(tp.max_cols, kStageThreads) : kStageThreads;
  // a tile row plus its four halo rows must fit the threads: 4 (wx + 1) <= max_cols
  const int max_wx = std::min(tp.max_wx > 0 ? std::min(tp.max_wx, kMaxTileX) : kMaxTileX, max_cols / 4 - 1);
  const int zchunk = tp.zchunk > 0 ? tp.zchunk : 32;
  const std::vector<HPatch>& P = plan.patches;
  auto split = [](int n, int parts, std::vector<std::pair<int, int>>& out) {
    out.clear();
    int base = n / parts, rem = n % parts, s = 0;
    for (int k = 0; k < parts; ++k) {
      int w = base + (k < rem ? 1 : 0);
      out.push_back({s, w});
      s += w;
    }
  };
  auto zsplit = [&](int nz, std::vector<std::pair<int, int>>& zs) {
    const int zparts = nz <= zchunk + zchunk / 2 ? 1 : (nz + zchunk - 1) / zchunk;
    split(nz, zparts, zs);
  };
  // one halo cell per thread: 4 (wx + wy) <= threads (= max_cols); plane with halo within
  // the shared-memory plane of the CTA size that runs the tile
  auto wy_max = [&](int wx) {
    const int w = std::min(std::min(max_cols / wx, stage_plane_max(max_cols) / (wx + 4) - 4), max_cols / 4 - wx);
    return std::max(w, 1);
  };
  // tiles of an n0 x n1 rectangle, each with its z chunks, as (x0, wx, y0, wy)
  auto tiles = [&](int n0, int n1, std::vector<std::array<int, 4>>& out) {
    out.clear();
    std::vector<std::pair<int, int>> xs, ys;
    split(n0, (n0 + max_wx - 1) / max_wx, xs);
    for (auto& x : xs) {
      const int wymax = wy_max(x.second);
      split(n1, (n1 + wymax - 1) / wymax, ys);
      for (auto& y : ys) out.push_back({x.first, x.second, y.first, y.second});
    }
  };
  plan.spans.clear();
  for (size_t l = 0; l < plan.levels.size(); ++l) {
    LevelPlan& L = plan.levels[l];
    L.items.clear();
    L.item_first.clear();
    L.item_first.push_back(0);
    std::vector<std::pair<int, int>> zs;
    std::vector<std::array<int, 4>> ts;
    for (int i = L.first; i < L.first + L.count; ++i) {
      const HPatch& p = P[i];
      zsplit(p.n[2], zs);
      for (auto& z : zs) {
        tiles(p.n[0], p.n[1], ts);
        for (auto& tl : ts) {
          StageItem it{};
          it.patch = i;
          it.x0 = (int16_t)tl[0]; it.wx = (int16_t)tl[1];
          it.y0 = (int16_t)tl[2]; it.wy = (int16_t)tl[3];
          it.z0 = (int16_t)z.first; it.wz = (int16_t)z.second;
          it.span = -1;
          L.items.push_back(it);
        }
      }
      L.item_first.push_back((int)L.items.size());
    }
    // batched launches: the z-layers of the level whose patches tile a rectangle
    // (same z range) are tiled as one region, so a column block may take cells of
    // several patches and small patches fill whole CTAs; other patches keep
    // their own blocks
    L.bitems.clear();
    if (!tp.span || plan.cfg.item_span != AMR_SPAN_LAYERS || plan.cfg.riemann == AMR_FLUXREC) {
      L.bitems = L.items;
      continue;
    }
    std::map<std::pair<int, int>, std::vector<int>> layers;   // (lo z, n z) -> patches
    for (int i = L.first; i < L.first + L.count; ++i) layers[{P[i].lo[2], P[i].n[2]}].push_back(i);
    std::vector<char> spanned(L.count, 0);
    for (auto& kv : layers) {
      const std::vector<int>& ps = kv.second;
      if (ps.size() < 2) continue;
      int lo0 = INT32_MAX, lo1 = INT32_MAX, hi0 = INT32_MIN, hi1 = INT32_MIN;
      int64_t area = 0;
      for (int i : ps) {
        lo0 = std::min(lo0, P[i].lo[0]); hi0 = std::max(hi0, P[i].lo[0] + P[i].n[0]);
        lo1 = std::min(lo1, P[i].lo[1]); hi1 = std::max(hi1, P[i].lo[1] + P[i].n[1]);
        area += (int64_t)P[i].n[0] * P[i].n[1];
      }
      if (area != (int64_t)(hi0 - lo0) * (hi1 - lo1)) continue;   // not a full rectangle (patches never overlap)
      tiles(hi0 - lo0, hi1 - lo1, ts);
      zsplit(kv.first.second, zs);
      // span the layer only where that fills the CTAs markedly better than the
      // patches' own blocks (a block over several patches pays a patch lookup per
      // column and halo cell)
      {
        int64_t own_blocks = 0;
        for (int i : ps) own_blocks += L.item_first[i - L.first + 1] - L.item_first[i - L.first];
        own_blocks /= std::max<int64_t>(1, (int64_t)zs.size());   // per z chunk of the layer's patches
        const double own_fill = (double)area / ((double)own_blocks * max_cols);
        const double span_fill = (double)area / ((double)ts.size() * max_cols);
        if (span_fill < own_fill + 0.05) continue;
      }
      std::vector<ItemSpan> sp;
      bool ok = true;
      for (auto& tl : ts) {
        ItemSpan S{};
        S.ox = lo0 + tl[0];
        S.oy = lo1 + tl[2];
        const int gx0 = S.ox - kGhost, gx1 = S.ox + tl[1] + kGhost, gy0 = S.oy - kGhost, gy1 = S.oy + tl[3] + kGhost;
        for (int i : ps)
          if (std::max(gx0, P[i].lo[0]) < std::min(gx1, P[i].lo[0] + P[i].n[0]) &&
              std::max(gy0, P[i].lo[1]) < std::min(gy1, P[i].lo[1] + P[i].n[1])) {
            if (S.n == kSpanMax) { ok = false; break; }
            S.patch[S.n++] = i;
          }
        if (!ok) break;
        sp.push_back(S);
      }
      if (!ok) continue;
      for (auto& z : zs)
        for (size_t k = 0; k < ts.size(); ++k) {
          ItemSpan S = sp[k];
          S.oz = kv.first.first + z.first;
          StageItem it{};
          it.patch = S.patch[0];
          it.wx = (int16_t)ts[k][1];
          it.wy = (int16_t)ts[k][3];
          it.wz = (int16_t)z.second;
          it.span = (int)plan.spans.size();
          plan.spans.push_back(S);
          L.bitems.push_back(it);
        }
      for (int i : ps) spanned[i - L.first] = 1;
    }
    for (int ii = 0; ii < L.count; ++ii)
      if (!spanned[ii])
        L.bitems.insert(L.bitems.end(), L.items.begin() + L.item_first[ii], L.items.begin() + L.item_first[ii + 1]);
  }
}

namespace {

template <class B>
void finish_flat(FlatList<B>& f, const std::vector<int>& cells, int chunk) {
  f.first.assign(cells.size() + 1, 0);
  for (size_t i = 0; i < cells.size(); ++i) f.first[i + 1] = f.first[i] + cells[i];
  f.total = f.first.back();
  const int nch = (f.total + chunk - 1) / chunk;
  f.chunk_box.assign(nch, 0);
  size_t b = 0;
  for (int k = 0; k < nch; ++k) {
    const int e = k * chunk;
    while (f.first[b + 1] <= e) ++b;
    f.chunk_box[k] = (int)b;
  }
}

// Copy boxes with the source mapping of CopySeg folded into strides: per axis
// the source coordinate is dlo + i + sh (translate) or sh (constant).
void flatten_copies(const Plan& plan, const std::vector<CopySeg>& segs, bool gather, FlatList<FlatCopy>& f) {
  f = FlatList<FlatCopy>();
  std::vector<int> cells;
  f.boxes.reserve(segs.size());
  cells.reserve(segs.size());
  for (const CopySeg& g : segs) {
    const PatchDesc& D = plan.desc[g.dst_patch];
    const PatchDesc& S = plan.desc[g.src_patch];
    FlatCopy c{};
    int s0[3];
    for (int d = 0; d < 3; ++d) s0[d] = g.mode[d] ? g.sh[d] : g.dlo[d] + g.sh[d];
    c.src0 = S.off + ((int64_t)(s0[2] + kGhost) * S.m1 + (s0[1] + kGhost)) * S.pitch + (s0[0] + kGhost);
    c.svs = (int)S.vstride;
    c.ssx = g.mode[0] ? 0 : 1;
    c.ssy = g.mode[1] ? 0 : S.pitch;
    c.ssz = g.mode[2] ? 0 : S.pitch * S.m1;
    if (gather) {
      c.dst0 = D.tile_off + ((int64_t)g.dlo[2] * D.tn[1] + g.dlo[1]) * D.tn[0] + g.dlo[0];
      c.dvs = D.tn[0] * D.tn[1] * D.tn[2];
      c.dsy = D.tn[0];
      c.dsz = D.tn[0] * D.tn[1];
    } else {
      c.dst0 = D.off + ((int64_t)(g.dlo[2] + kGhost) * D.m1 + (g.dlo[1] + kGhost)) * D.pitch + (g.dlo[0] + kGhost);
      c.dvs = (int)D.vstride;
      c.dsy = D.pitch;
      c.dsz = D.pitch * D.m1;
    }
    c.n0 = g.dn[0];
    c.n1 = g.dn[1];
    f.boxes.push_back(c);
    cells.push_back(g.dn[0] * g.dn[1] * g.dn[2]);
  }
  finish_flat(f, cells, kCopyChunk);
}

int floor_half(int g) { return g >= 0 ? g / 2 : -((1 - g) / 2); }

void flatten_prolong(const Plan& plan, const std::vector<ProlongBox>& boxes, FlatList<FlatProlong>& f) {
  f = FlatList<FlatProlong>();
  std::vector<int> cells;
  for (const ProlongBox& b : boxes) {
    const PatchDesc& D = plan.desc[b.patch];
    FlatProlong c{};
    c.dst0 = D.off + cell_index(D, b.lo[0], b.lo[1], b.lo[2]);
    c.dvs = (int)D.vstride;
    c.dsy = D.pitch;
    c.dsz = D.pitch * D.m1;
    c.tvol = D.tn[0] * D.tn[1] * D.tn[2];
    c.tsy = D.tn[0];
    c.tsz = D.tn[0] * D.tn[1];
    int p0[3], np[3];
    for (int d = 0; d < 3; ++d) {
      const int g0 = D.lo[d] + b.lo[d];
      p0[d] = floor_half(g0) - (floor_half(D.lo[d]) - 2);   // tile-local parent of the first fine cell
      np[d] = floor_half(g0 + b.n[d] - 1) - floor_half(g0) + 1;
      c.n[d] = b.n[d];
      if (g0 & 1) c.odd |= 1 << d;
    }
    c.tp0 = D.tile_off + p0[0] + (int64_t)p0[1] * c.tsy + (int64_t)p0[2] * c.tsz;
    c.np0 = np[0];
    c.np1 = np[1];
    f.boxes.push_back(c);
    cells.push_back(np[0] * np[1] * np[2]);
  }
  finish_flat(f, cells, kProlongChunk);
}

void flatten_restrict(const Plan& plan, const std::vector<RestrictSeg>& segs, FlatList<FlatCopy>& f) {
  f = FlatList<FlatCopy>();
  std::vector<int> cells;
  for (const RestrictSeg& r : segs) {
    const PatchDesc& C = plan.desc[r.coarse];
    const PatchDesc& F = plan.desc[r.fine];
    FlatCopy c{};
    int f0[3];
    for (int d = 0; d < 3; ++d) f0[d] = 2 * (C.lo[d] + r.clo[d]) - F.lo[d];
    c.dst0 = C.off + cell_index(C, r.clo[0], r.clo[1], r.clo[2]);
    c.dvs = (int)C.vstride;
    c.dsy = C.pitch;
    c.dsz = C.pitch * C.m1;
    c.src0 = F.off + cell_index(F, f0[0], f0[1], f0[2]);
    c.svs = (int)F.vstride;
    c.ssx = 1;
    c.ssy = F.pitch;
    c.ssz = F.pitch * F.m1;
    c.n0 = r.cn[0];
    c.n1 = r.cn[1];
    f.boxes.push_back(c);
    cells.push_back(r.cn[0] * r.cn[1] * r.cn[2]);
  }
  finish_flat(f, cells, kRestrictChunk);
}

}  // namespace

void parallel_run(int n, const std::function<void(int)>& f) { parallel_for(n, f); }

namespace {
// Bits of x spread to every third position (x < 2^21).
uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}
}  // namespace

std::vector<int> morton_partition(const amr_config& cfg, const std::vector<HPatch>& P, int nranks) {
  const int np = (int)P.size();
  std::vector<int> owner(np, 0);
  if (nranks <= 1 || np == 0) return owner;
  int L = 0;
  for (const HPatch& p : P) L = std::max(L, p.level);
  // coarsen the curve so the finest level's coordinates fit 21 bits per axis
  int sh = 0;
  for (int d = 0; d < 3; ++d)
    while (((int64_t)std::max(cfg.base_n[d], 1) << L) >> sh >= ((int64_t)1 << 21)) ++sh;
  for (int l = 0; l <= L; ++l) {
    // the level's patches in Morton order of their centres (finest-level cells,
    // so that the orders of different levels follow the same curve)
    std::vector<std::pair<uint64_t, int>> ord;
    int64_t total = 0;
    for (int i = 0; i < np; ++i) {
      if (P[i].level != l) continue;
      uint64_t c[3];
      for (int d = 0; d < 3; ++d)
        c[d] = (uint64_t)((((int64_t)2 * P[i].lo[d] + P[i].n[d]) << (L - l)) >> (1 + sh));
      const uint64_t key = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
      ord.push_back({key, i});
      total += (int64_t)P[i].n[0] * P[i].n[1] * P[i].n[2];
    }
    std::sort(ord.begin(), ord.end());
    // contiguous ranges: rank r takes the patches whose cell-count prefix midpoint
    // falls in [r, r+1) * total / nranks
    int64_t run = 0;
    for (const auto& e : ord) {
      const HPatch& p = P[e.second];
      const int64_t w = (int64_t)p.n[0] * p.n[1] * p.n[2];
      const int64_t mid2 = 2 * run + w;   // twice the midpoint
      owner[e.second] = (int)std::min<int64_t>(nranks - 1, mid2 * nranks / (2 * std::max<int64_t>(total, 1)));
      run += w;
    }
  }
  return owner;
}

// Gather segments into the parent tile of fine patch i (level l >= 1) for the
// tile cells that the prolongation of `boxes` (fine local cells of patch i)
// reads: the parents of those cells and their face neighbours (the minmod
// stencil), as disjoint boxes of the tile, each split over the parent-level
// patches (periodic images, outflow clamps) that hold it.  cix indexes level
// l - 1.  err is set if a needed parent cell lies outside level l - 1.
void prolong_gathers(const amr_config& cfg, const Plan& plan, const PatchIndex& cix, int i, const ProlongBox* boxes,
                     int nbox, std::vector<CopySeg>& out, std::string& err) {
  const std::vector<HPatch>& P = plan.patches;
  const HPatch& p = P[i];
  const PatchDesc& dsc = plan.desc[i];
  const int l = p.level;
  struct Piece { int a, len, mode, src; };
  std::vector<int> cand;
  // gathers of the tile cells [blo, bhi) per axis; returns the cells covered
  auto gather_box = [&](const int* blo, const int* bhi) -> int64_t {
    // at most three pieces per axis (below the domain, inside, above: the kind only grows along an axis)
    struct Pieces {
      Piece v[3];
      int n = 0;
      void push_back(const Piece& x) { v[n++] = x; }
      const Piece* begin() const { return v; }
      const Piece* end() const { return v + n; }
    } pieces[3];
    for (int d = 0; d < 3; ++d) {
      const int Nc = level_n(cfg, l - 1, d);
      const int T0 = p.lo[d] / 2 - 2;
      int t = blo[d];
      while (t < bhi[d]) {
        const int Cg = T0 + t;
        const int kind = Cg < 0 ? 0 : (Cg < Nc ? 1 : 2);
        int e = t;
        while (e < bhi[d]) {
          const int Cc = T0 + e;
          if ((Cc < 0 ? 0 : (Cc < Nc ? 1 : 2)) != kind) break;
          ++e;
        }
        Piece pc{t, e - t, 0, 0};
        if (kind == 1) { pc.mode = 0; pc.src = Cg; }
        else if (periodic(cfg, d)) { pc.mode = 0; pc.src = kind == 0 ? Cg + Nc : Cg - Nc; }
        else { pc.mode = 1; pc.src = kind == 0 ? 0 : Nc - 1; }
        pieces[d].push_back(pc);
        t = e;
      }
    }
    int64_t covered = 0;
    for (const Piece& p0 : pieces[0])
      for (const Piece& p1 : pieces[1])
        for (const Piece& p2 : pieces[2]) {
          const Piece* pp[3] = {&p0, &p1, &p2};
          int qlo[3], qhi[3];
          for (int d = 0; d < 3; ++d) {
            qlo[d] = pp[d]->src;
            qhi[d] = pp[d]->mode == 1 ? pp[d]->src + 1 : pp[d]->src + pp[d]->len;
          }
          cix.query(qlo, qhi, cand);
          for (int q : cand) {
            const HPatch& o = P[q];
            CopySeg s{};
            s.dst_patch = i; s.src_patch = q;
            bool ok = true;
            int64_t vol = 1;
            for (int d = 0; d < 3 && ok; ++d) {
              const Piece& pc = *pp[d];
              if (pc.mode == 1) {
                if (pc.src < o.lo[d] || pc.src >= o.lo[d] + o.n[d]) { ok = false; break; }
                s.dlo[d] = (int16_t)pc.a; s.dn[d] = (int16_t)pc.len; s.mode[d] = 1;
                s.sh[d] = (int16_t)(pc.src - o.lo[d]);
                vol *= pc.len;
              } else {
                const int a = std::max(pc.src, o.lo[d]), b = std::min(pc.src + pc.len, o.lo[d] + o.n[d]);
                if (a >= b) { ok = false; break; }
                const int dst0 = pc.a + (a - pc.src);
                s.dlo[d] = (int16_t)dst0; s.dn[d] = (int16_t)(b - a); s.mode[d] = 0;
                s.sh[d] = (int16_t)((a - o.lo[d]) - dst0);
                vol *= (b - a);
              }
            }
            if (!ok) continue;
            covered += vol;
            out.push_back(s);
          }
        }
    return covered;
  };
  std::vector<unsigned char> need((size_t)dsc.tn[0] * dsc.tn[1] * dsc.tn[2], 0);
  int64_t nneed = 0;
  int blo_all[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, bhi_all[3] = {-1, -1, -1};   // bounding box (inclusive)
  for (int b = 0; b < nbox; ++b) {
    const ProlongBox& pb = boxes[b];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      const int t0 = ((p.lo[a] + pb.lo[a]) >> 1) - (p.lo[a] >> 1) + 2;
      const int t1 = ((p.lo[a] + pb.lo[a] + pb.n[a] - 1) >> 1) - (p.lo[a] >> 1) + 2;
      lo[a] = std::max(t0 - 1, 0);
      hi[a] = std::min(t1 + 1, dsc.tn[a] - 1);
      blo_all[a] = std::min(blo_all[a], lo[a]);
      bhi_all[a] = std::max(bhi_all[a], hi[a]);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          unsigned char& m = need[((size_t)z * dsc.tn[1] + y) * dsc.tn[0] + x];
          nneed += m ? 0 : 1;
          m = 1;
        }
  }
  if (nneed == 0) return;
  const size_t first = out.size();
  int64_t got = 0, want = nneed;
  const int64_t bvol = (int64_t)(bhi_all[0] - blo_all[0] + 1) * (bhi_all[1] - blo_all[1] + 1) *
                       (bhi_all[2] - blo_all[2] + 1);
  if (2 * nneed >= bvol) {
    // the needed cells fill at least half of their bounding box: gather the box
    // (fewer, larger copies; the extra cells are read but never used)
    const int blo[3] = {blo_all[0], blo_all[1], blo_all[2]};
    const int bhi[3] = {bhi_all[0] + 1, bhi_all[1] + 1, bhi_all[2] + 1};
    got = gather_box(blo, bhi);
    want = bvol;
  } else {
    for (const Box3& bx : need_boxes(need, dsc.tn[0], dsc.tn[1], dsc.tn[2])) {
      const int blo[3] = {bx.lo[0], bx.lo[1], bx.lo[2]};
      const int bhi[3] = {bx.lo[0] + bx.n[0], bx.lo[1] + bx.n[1], bx.lo[2] + bx.n[2]};
      got += gather_box(blo, bhi);
    }
  }
  split_copy(out, first);
  if (got != want) err = fmt("patch %d: parent cells of its prolongation not covered by level %d", i, l - 1);
}

void build_fill_gathers(const amr_config& cfg, const Plan& plan, const std::vector<std::vector<ProlongBox>>& fresh,
                        std::vector<std::vector<CopySeg>>& out, std::string& msg) {
  out.assign(fresh.size(), {});
  for (size_t l = 1; l < fresh.size() && l < plan.levels.size(); ++l) {
    const std::vector<ProlongBox>& F = fresh[l];
    if (F.empty()) continue;
    // the fresh boxes grouped by patch (they come grouped, patch by patch)
    std::vector<std::pair<int, int>> runs;   // [begin, end) of each patch's boxes
    for (int b = 0; b < (int)F.size();) {
      int e = b + 1;
      while (e < (int)F.size() && F[e].patch == F[b].patch) ++e;
      runs.push_back({b, e});
      b = e;
    }
    PatchIndex cix(plan.patches, plan.levels[l - 1].first, plan.levels[l - 1].count);
    std::vector<std::vector<CopySeg>> segs(runs.size());
    std::vector<std::string> err(runs.size());
    parallel_for((int)runs.size(), [&](int r) {
      prolong_gathers(cfg, plan, cix, F[runs[r].first].patch, F.data() + runs[r].first,
                      runs[r].second - runs[r].first, segs[r], err[r]);
    });
    for (size_t r = 0; r < runs.size(); ++r) {
      if (!err[r].empty() && msg.empty()) msg = err[r];
      out[l].insert(out[l].end(), segs[r].begin(), segs[r].end());
    }
  }
}

// The stage kernel's view of a face read from the patch's own ghost cells.
FaceSrc own_face(const PatchDesc& d) {
  FaceSrc f;
  f.base = d.off + cell_index(d, 0, 0, 0);
  f.sx = 1;
  f.sy = d.pitch;
  f.sz = d.pitch * d.m1;
  f.vs = (int)d.vstride;
  return f;
}

// Face (2 axis + side) of the patch that a ghost segment fills.
int seg_face(const CopySeg& s, const HPatch& p) {
  for (int a = 0; a < 3; ++a) {
    if (s.dlo[a] < 0) return 2 * a;
    if (s.dlo[a] >= p.n[a]) return 2 * a + 1;
  }
  return 0;   // not reached: ghost segments lie outside the interior along one axis
}

// Faces of patch i whose two ghost layers come, whole, from one source cell box
// through one mapping (one same-level patch by translation, the patch itself
// across a periodic boundary, or its boundary cells at an outflow face): the
// stage kernel can read them there (desc.face), and the ghost copy skips them.
void classify_faces(Plan& plan, int i, const std::vector<CopySeg>& segs, std::array<uint8_t, 6>& direct) {
  const HPatch& p = plan.patches[i];
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const CopySeg* first = nullptr;
    bool same = true;
    int64_t vol = 0;
    for (const CopySeg& s : segs) {
      if (seg_face(s, p) != f) continue;
      if (!first) first = &s;
      for (int a = 0; a < 3; ++a)
        same = same && s.src_patch == first->src_patch && s.mode[a] == first->mode[a] && s.sh[a] == first->sh[a];
      vol += (int64_t)s.dn[0] * s.dn[1] * s.dn[2];
    }
    direct[f] = 0;
    if (!first || !same || vol != (int64_t)kGhost * p.n[t1] * p.n[t2]) continue;
    if (first->mode[t1] != 0 || first->mode[t2] != 0) continue;
    const PatchDesc& q = plan.desc[first->src_patch];
    FaceSrc& fs = plan.desc[i].face[f];
    fs.base = q.off + cell_index(q, first->sh[0], first->sh[1], first->sh[2]);
    fs.sx = first->mode[0] ? 0 : 1;
    fs.sy = first->mode[1] ? 0 : q.pitch;
    fs.sz = first->mode[2] ? 0 : q.pitch * q.m1;
    fs.vs = (int)q.vstride;
    direct[f] = 1;
  }
}

void build_flat(Plan& plan) {
  // five independent lists per level, flattened in parallel
  parallel_tasks(5 * (int)plan.levels.size(), [&](int t) {
    LevelPlan& L = plan.levels[t / 5];
    switch (t % 5) {
      case 0: flatten_copies(plan, L.ghost_stage, false, L.fghost); break;
      case 1: flatten_copies(plan, L.gather_ghost, true, L.fgather); break;
      case 2: flatten_prolong(plan, L.prolong, L.fprolong); break;
      case 3: flatten_copies(plan, L.ghost, false, L.fghost_all); break;
      default: flatten_restrict(plan, L.restrict_segs, L.frestrict); break;
    }
  });
}

amr_status build_plan(const amr_config& cfg, const std::vector<HPatch>& P, Plan& plan, std::string& msg,
                      const TileParams& tp) {
  amr_status st = validate_patches(cfg, P, msg);
  if (st != AMR_OK) return st;
  plan = Plan();
  plan.cfg = cfg;
  plan.nvar = cfg.nvar;
  plan.patches = P;
  const int np = (int)P.size();
  int nlev = P.back().level + 1;
  plan.levels.resize(nlev);
  for (int i = 0; i < np; ++i) {
    LevelPlan& L = plan.levels[P[i].level];
    if (L.count == 0) L.first = i;
    L.count++;
    L.cells += (int64_t)P[i].n[0] * P[i].n[1] * P[i].n[2];
  }

  // ---- device descriptors and arena layout ----
  plan.desc.resize(np);
  int64_t off = 0, toff = 0, poff = 0;
  plan.packed_off.resize(np);
  for (int i = 0; i < np; ++i) {
    PatchDesc& d = plan.desc[i];
    const HPatch& p = P[i];
    for (int a = 0; a < 3; ++a) { d.n[a] = p.n[a]; d.lo[a] = p.lo[a]; }
    d.level = p.level;
    d.pitch = (int)round_up(p.n[0] + 2 * kGhost, 4);
    d.m1 = p.n[1] + 2 * kGhost;
    d.vstride = round_up((int64_t)d.pitch * d.m1 * (p.n[2] + 2 * kGhost), 32);
    d.off = off;
    off += d.vstride * plan.nvar;
    if (p.level > 0) {
      d.tile_off = (int)toff;
      for (int a = 0; a < 3; ++a) d.tn[a] = p.n[a] / 2 + 4;
      toff += (int64_t)d.tn[0] * d.tn[1] * d.tn[2] * plan.nvar;
    } else {
      d.tile_off = -1;
      d.tn[0] = d.tn[1] = d.tn[2] = 0;
    }
    plan.packed_off[i] = poff;
    poff += (int64_t)p.n[0] * p.n[1] * p.n[2] * plan.nvar;
  }
  if (toff > INT32_MAX) { msg = "parent tiles exceed 2^31 elements"; return AMR_ERR_ARG; }
  for (int i = 0; i < np; ++i)
    for (int f = 0; f < 6; ++f) plan.desc[i].face[f] = own_face(plan.desc[i]);
  plan.arena_elems = off;
  plan.tile_elems = toff;
  plan.packed_elems = poff;

  // ---- stage work items ----
  build_items(plan, tp);
  // faces whose ghost layers a stage reads straight from a neighbour (or outflow boundary cells)
  const bool direct_ok = cfg.ghost_fill == AMR_GHOST_DIRECT && cfg.riemann != AMR_FLUXREC;
  std::vector<std::array<uint8_t, 6>> direct(np);
  // bit 2d+side: the ghost layer of that face two cells out on the low side (one on
  // the high side) -- the fine cells of the coarse cells next to the face -- lies
  // in same-level patches all over, so the face has no flux register
  std::vector<uint8_t> face_full(np, 0);
  for (auto& a : direct) a.fill(0);

  // ---- ghost fill: sibling copies (incl. periodic images), outflow, prolongation boxes ----
  for (int l = 0; l < nlev; ++l) {
    LevelPlan& L = plan.levels[l];
    PatchIndex six(P, L.first, L.count);
    std::vector<std::vector<CopySeg>> gs(L.count);
    std::vector<std::vector<ProlongBox>> ps(L.count);
    std::vector<std::string> err(L.count);
    parallel_for(L.count, [&](int ii) {
      const int i = L.first + ii;
      std::vector<CopySeg>& Gv = gs[ii];
      std::vector<ProlongBox>& Pv = ps[ii];
      std::vector<int> cand;
      const HPatch& p = P[i];
        for (int d = 0; d < 3; ++d) {
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int Nl = level_n(cfg, l, d);
          for (int side = 0; side < 2; ++side) {
            // one neighbour query for both ghost layers of the face when they are
            // adjacent level cells (the loop below keeps the patches of each layer)
            int qd_lo = 0, qd_hi = 0;   // layer range along d the current cand covers
            for (int gg = 0; gg < kGhost; ++gg) {
              int loc = side ? p.n[d] + gg : -1 - gg;
              int G = p.lo[d] + loc;
              if (G < 0 || G >= Nl) {
                if (!periodic(cfg, d)) {  // outflow: zero-gradient copy of the boundary cell
                  CopySeg s{};
                  s.dst_patch = i; s.src_patch = i;
                  s.dlo[d] = (int16_t)loc; s.dn[d] = 1; s.mode[d] = 1;
                  s.sh[d] = (int16_t)(side ? p.n[d] - 1 : 0);
                  s.dlo[t1] = 0; s.dn[t1] = (int16_t)p.n[t1]; s.mode[t1] = 0; s.sh[t1] = 0;
                  s.dlo[t2] = 0; s.dn[t2] = (int16_t)p.n[t2]; s.mode[t2] = 0; s.sh[t2] = 0;
                  Gv.push_back(s);
                  continue;
                }
                G = ((G % Nl) + Nl) % Nl;
              }
              int A = p.n[t1], B = p.n[t2];
              if (!(G >= qd_lo && G < qd_hi)) {
                int qlo[3], qhi[3];
                qlo[d] = G; qhi[d] = G + 1;
                if (gg + 1 < kGhost) {   // the next layer, if it lies next to this one in the level
                  const int Gn = p.lo[d] + (side ? p.n[d] + gg + 1 : -2 - gg);
                  if (Gn >= 0 && Gn < Nl && (Gn == G + 1 || Gn == G - 1)) {
                    qlo[d] = std::min(G, Gn);
                    qhi[d] = std::max(G, Gn) + 1;
                  }
                }
                qlo[t1] = p.lo[t1]; qhi[t1] = p.lo[t1] + p.n[t1];
                qlo[t2] = p.lo[t2]; qhi[t2] = p.lo[t2] + p.n[t2];
                six.query(qlo, qhi, cand);
                qd_lo = qlo[d];
                qd_hi = qhi[d];
              }
              const size_t g0 = Gv.size();
              int64_t area = 0;      // same-level patches do not overlap: the covered area sums
              for (int q : cand) {
                const HPatch& o = P[q];
                if (G < o.lo[d] || G >= o.lo[d] + o.n[d]) continue;
                int a0 = std::max(p.lo[t1], o.lo[t1]), a1 = std::min(p.lo[t1] + p.n[t1], o.lo[t1] + o.n[t1]);
                int b0 = std::max(p.lo[t2], o.lo[t2]), b1 = std::min(p.lo[t2] + p.n[t2], o.lo[t2] + o.n[t2]);
                if (a0 >= a1 || b0 >= b1) continue;
                CopySeg s{};
                s.dst_patch = i; s.src_patch = q;
                s.dlo[d] = (int16_t)loc; s.dn[d] = 1; s.mode[d] = 0;
                s.sh[d] = (int16_t)((G - o.lo[d]) - loc);
                s.dlo[t1] = (int16_t)(a0 - p.lo[t1]); s.dn[t1] = (int16_t)(a1 - a0); s.sh[t1] = (int16_t)(p.lo[t1] - o.lo[t1]);
                s.dlo[t2] = (int16_t)(b0 - p.lo[t2]); s.dn[t2] = (int16_t)(b1 - b0); s.sh[t2] = (int16_t)(p.lo[t2] - o.lo[t2]);
                Gv.push_back(s);
                area += (int64_t)(a1 - a0) * (b1 - b0);
              }
              if (area == (int64_t)A * B && gg == (side ? 0 : 1)) face_full[i] |= (uint8_t)(1u << (2 * d + side));
              std::vector<Rect> rects;
              if (area < (int64_t)A * B) {   // uncovered parts of the face layer: prolongation boxes
                std::vector<unsigned char> mask((size_t)A * B, 0);
                for (size_t e = g0; e < Gv.size(); ++e) {
                  const CopySeg& c = Gv[e];
                  for (int b = c.dlo[t2]; b < c.dlo[t2] + c.dn[t2]; ++b)
                    for (int a = c.dlo[t1]; a < c.dlo[t1] + c.dn[t1]; ++a) mask[(size_t)b * A + a] = 1;
                }
                mask_rects(mask.data(), A, B, rects);
              }
              if (!rects.empty() && l == 0) {
                err[ii] = fmt("level-0 patch %d has uncovered ghost cells", i);
                return;
              }
              for (const Rect& r : rects) {
                ProlongBox pb{};
                pb.patch = i;
                pb.lo[d] = (int16_t)loc; pb.n[d] = 1;
                pb.lo[t1] = (int16_t)r.a0; pb.n[t1] = (int16_t)r.na;
                pb.lo[t2] = (int16_t)r.b0; pb.n[t2] = (int16_t)r.nb;
                Pv.push_back(pb);
              }
            }
          }
        }
        // merge the two ghost layers of a face into one two-deep segment where
        // both layers copy from the same source with the same mapping
        {
          const int g0 = 0;
          std::vector<CopySeg> segs(Gv.begin() + g0, Gv.end());
          std::vector<char> used(segs.size(), 0);
          std::vector<CopySeg> merged;
          for (size_t a = 0; a < segs.size(); ++a) {
            if (used[a]) continue;
            CopySeg m = segs[a];
            for (size_t b = a + 1; b < segs.size(); ++b) {
              if (used[b]) continue;
              const CopySeg& o = segs[b];
              int d = -1;
              for (int k = 0; k < 3; ++k)
                if (m.dn[k] == 1 && o.dn[k] == 1 && (o.dlo[k] == m.dlo[k] - 1 || o.dlo[k] == m.dlo[k] + 1)) d = k;
              if (d < 0 || o.src_patch != m.src_patch) continue;
              bool same = true;
              for (int k = 0; k < 3 && same; ++k) {
                same = o.mode[k] == m.mode[k] && o.sh[k] == m.sh[k];
                if (k != d) same = same && o.dlo[k] == m.dlo[k] && o.dn[k] == m.dn[k];
              }
              if (!same) continue;
              m.dlo[d] = std::min(m.dlo[d], o.dlo[d]);
              m.dn[d] = 2;
              used[b] = 1;
              break;
            }
            merged.push_back(m);
          }
          Gv.resize(g0);
          Gv.insert(Gv.end(), merged.begin(), merged.end());
          split_copy(Gv, g0);
        }
        split_prolong(Pv, 0);
        if (direct_ok) classify_faces(plan, i, Gv, direct[i]);
    });
    L.ghost_first.push_back(0);
    L.prolong_first.push_back(0);
    for (int ii = 0; ii < L.count; ++ii) {
      if (!err[ii].empty()) {
        msg = err[ii];
        return AMR_ERR_NESTING;
      }
      L.ghost.insert(L.ghost.end(), gs[ii].begin(), gs[ii].end());
      L.prolong.insert(L.prolong.end(), ps[ii].begin(), ps[ii].end());
      L.ghost_first.push_back((int)L.ghost.size());
      L.prolong_first.push_back((int)L.prolong.size());
    }
  }

  // ---- parent-cell gathers (level >= 1) ----
  // each stage gathers, time-interpolated, only the parent cells the
  // prolongation of the patch's coarse-fine ghost cells reads (a patch whose
  // ghost cells all come from siblings gathers nothing); the regrid fill
  // gathers for its own prolongation boxes (build_fill_gathers)
  for (int l = 1; l < nlev; ++l) {
    LevelPlan& L = plan.levels[l];
    PatchIndex cix(P, plan.levels[l - 1].first, plan.levels[l - 1].count);
    std::vector<std::vector<CopySeg>> gs_ghost(L.count);
    std::vector<std::string> err(L.count);
    parallel_for(L.count, [&](int ii) {
      const int a = L.prolong_first[ii], b = L.prolong_first[ii + 1];
      if (b > a) prolong_gathers(cfg, plan, cix, L.first + ii, L.prolong.data() + a, b - a, gs_ghost[ii], err[ii]);
    });
    for (int ii = 0; ii < L.count; ++ii) {
      if (!err[ii].empty()) {
        msg = err[ii];
        return AMR_ERR_NESTING;
      }
      L.gather_ghost.insert(L.gather_ghost.end(), gs_ghost[ii].begin(), gs_ghost[ii].end());
    }
  }

  // ---- restriction segments and coverage boxes ----
  plan.cover_first.assign(np + 1, 0);
  std::vector<std::vector<CoverBox>> cov(np);
  for (int l = 1; l < nlev; ++l) {
    LevelPlan& L = plan.levels[l];
    const LevelPlan& C = plan.levels[l - 1];
    PatchIndex cix(P, C.first, C.count);
    std::vector<std::vector<RestrictSeg>> rsegs(L.count);   // per fine patch, concatenated in patch order
    parallel_for(L.count, [&](int ii) {
      const int i = L.first + ii;
      const HPatch& f = P[i];
      std::vector<int> cand;
      {
        int qlo[3], qhi[3];
        for (int d = 0; d < 3; ++d) { qlo[d] = f.lo[d] / 2; qhi[d] = (f.lo[d] + f.n[d]) / 2; }
        cix.query(qlo, qhi, cand);
      }
      for (int q : cand) {
        const HPatch& o = P[q];
        int lo[3], hi[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::max(f.lo[d] / 2, o.lo[d]);
          hi[d] = std::min((f.lo[d] + f.n[d]) / 2, o.lo[d] + o.n[d]);
          if (lo[d] >= hi[d]) ok = false;
        }
        if (!ok) continue;
        RestrictSeg r{};
        r.fine = i; r.coarse = q;
        for (int d = 0; d < 3; ++d) {
          r.clo[d] = (int16_t)(lo[d] - o.lo[d]);
          r.cn[d] = (int16_t)(hi[d] - lo[d]);
        }
        rsegs[ii].push_back(r);
      }
    });
    for (int ii = 0; ii < L.count; ++ii)
      for (const RestrictSeg& r : rsegs[ii]) {
        L.restrict_segs.push_back(r);
        CoverBox cb{};
        for (int d = 0; d < 3; ++d) { cb.lo[d] = r.clo[d]; cb.n[d] = r.cn[d]; }
        cov[r.coarse].push_back(cb);
      }
  }
  for (int l = 1; l < nlev; ++l) split_restrict(plan.levels[l].restrict_segs);
  for (int i = 0; i < np; ++i) {
    plan.cover_first[i + 1] = plan.cover_first[i] + (int)cov[i].size();
    for (auto& b : cov[i]) plan.cover.push_back(b);
  }

  // ---- flux registers (level >= 1): fine patch faces against uncovered parent cells ----
  for (int l = 1; l < nlev; ++l) {
    LevelPlan& L = plan.levels[l];
    const LevelPlan& C = plan.levels[l - 1];
    PatchIndex fix(P, L.first, L.count), cix(P, C.first, C.count);
    // tasks in (d, side, patch) order; concatenated in that order below
    const int ntask = 6 * L.count;
    std::vector<std::vector<RegRect>> rs(ntask);
    std::vector<std::string> err(ntask);
    parallel_for(ntask, [&](int task) {
      const int d = task / (2 * L.count), side = (task / L.count) % 2, i = L.first + task % L.count;
      if (face_full[i] & (1u << (2 * d + side))) return;   // the fine level covers the cells next to the face
      std::vector<RegRect>& Rv = rs[task];
      std::vector<int> cand;
          const HPatch& p = P[i];
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int xf = side ? p.lo[d] + p.n[d] : p.lo[d];
          int Cd = side ? xf / 2 : xf / 2 - 1;
          int Nc = level_n(cfg, l - 1, d);
          if (Cd < 0 || Cd >= Nc) {
            if (!periodic(cfg, d)) return;
            Cd = ((Cd % Nc) + Nc) % Nc;
          }
          int a0 = p.lo[t1] / 2, A = p.n[t1] / 2, b0 = p.lo[t2] / 2, B = p.n[t2] / 2;
          // covered by a level-l patch?
          std::vector<unsigned char> cov2((size_t)A * B, 0);
          {
            int qlo[3], qhi[3];
            qlo[d] = 2 * Cd; qhi[d] = 2 * Cd + 1;
            qlo[t1] = 2 * a0; qhi[t1] = 2 * (a0 + A);
            qlo[t2] = 2 * b0; qhi[t2] = 2 * (b0 + B);
            fix.query(qlo, qhi, cand);
          }
          int64_t covered = 0;   // same-level patches do not overlap: their areas add up
          for (int q : cand) {
            const HPatch& o = P[q];
            if (2 * Cd < o.lo[d] || 2 * Cd >= o.lo[d] + o.n[d]) continue;
            int x0 = std::max(a0, o.lo[t1] / 2), x1 = std::min(a0 + A, (o.lo[t1] + o.n[t1]) / 2);
            int y0 = std::max(b0, o.lo[t2] / 2), y1 = std::min(b0 + B, (o.lo[t2] + o.n[t2]) / 2);
            for (int y = y0; y < y1; ++y)
              for (int x = x0; x < x1; ++x) cov2[(size_t)(y - b0) * A + (x - a0)] = 1;
            if (x1 > x0 && y1 > y0) covered += (int64_t)(x1 - x0) * (y1 - y0);
          }
          if (covered == (int64_t)A * B) return;   // the face borders level l all over: no register
          std::vector<int> owner((size_t)A * B, -1);
          {
            int qlo[3], qhi[3];
            qlo[d] = Cd; qhi[d] = Cd + 1;
            qlo[t1] = a0; qhi[t1] = a0 + A;
            qlo[t2] = b0; qhi[t2] = b0 + B;
            cix.query(qlo, qhi, cand);
          }
          for (int q : cand) {
            const HPatch& o = P[q];
            if (Cd < o.lo[d] || Cd >= o.lo[d] + o.n[d]) continue;
            int x0 = std::max(a0, o.lo[t1]), x1 = std::min(a0 + A, o.lo[t1] + o.n[t1]);
            int y0 = std::max(b0, o.lo[t2]), y1 = std::min(b0 + B, o.lo[t2] + o.n[t2]);
            for (int y = y0; y < y1; ++y)
              for (int x = x0; x < x1; ++x) owner[(size_t)(y - b0) * A + (x - a0)] = q;
          }
          // one rectangle per run of uncovered cells with the same coarse owner
          std::vector<int> qs;
          for (size_t e = 0; e < owner.size(); ++e)
            if (!cov2[e]) {
              if (owner[e] < 0) { err[task] = fmt("patch %d: coarse neighbour cell outside level %d", i, l - 1); return; }
              if (std::find(qs.begin(), qs.end(), owner[e]) == qs.end()) qs.push_back(owner[e]);
            }
          std::sort(qs.begin(), qs.end());
          // level-l patches near the face: coarse cells [Cd - 1, Cd + 2) along d and one
          // cell beyond the face's extent in-plane (every box covered_any asks about
          // that does not wrap lies inside)
          std::vector<int> near;
          int nlo[3], nhi[3];
          nlo[d] = Cd - 1; nhi[d] = Cd + 2;
          nlo[t1] = a0 - 1; nhi[t1] = a0 + A + 1;
          nlo[t2] = b0 - 1; nhi[t2] = b0 + B + 1;
          {
            int qlo[3], qhi[3];
            for (int k = 0; k < 3; ++k) { qlo[k] = 2 * nlo[k]; qhi[k] = 2 * nhi[k]; }
            fix.query(qlo, qhi, near);
          }
          // does a level-l patch cover any coarse cell of [lo, hi) (level l-1 indices; a
          // cell beyond an outflow face is not covered, periodic axes wrap)
          std::vector<int> cc;
          auto covered_any = [&](int lo[3], int hi[3]) {
            bool wrapped = false;
            for (int k = 0; k < 3; ++k) {
              const int Nk = level_n(cfg, l - 1, k);
              if (lo[k] < 0 || hi[k] > Nk) {
                if (!periodic(cfg, k) || hi[k] - lo[k] != 1) return false;   // only single-cell strips leave the box
                lo[k] = ((lo[k] % Nk) + Nk) % Nk;
                hi[k] = lo[k] + 1;
                wrapped = true;
              }
            }
            const std::vector<int>* cands = &near;
            if (wrapped) {
              int qlo[3], qhi[3];
              for (int k = 0; k < 3; ++k) { qlo[k] = 2 * lo[k]; qhi[k] = 2 * hi[k]; }
              fix.query(qlo, qhi, cc);
              cands = &cc;
            }
            for (int q2 : *cands) {
              const HPatch& o = P[q2];
              bool hit = true;
              for (int k = 0; k < 3 && hit; ++k)
                hit = std::max(lo[k], o.lo[k] / 2) < std::min(hi[k], (o.lo[k] + o.n[k]) / 2);
              if (hit) return true;
            }
            return false;
          };
          std::vector<unsigned char> other((size_t)A * B);
          std::vector<Rect> orects;
          for (int q : qs) {
            for (size_t e = 0; e < other.size(); ++e) other[e] = (cov2[e] || owner[e] != q) ? 1 : 0;
            const HPatch& o = P[q];
            mask_rects(other.data(), A, B, orects);
            for (const Rect& rc : orects) {
              RegRect r{};
              r.fpatch = i; r.cpatch = q;
              r.d = (int8_t)d; r.side = (int8_t)side; r.cside = (int8_t)(side ? -1 : 1);
              int Cc[3];
              Cc[d] = Cd; Cc[t1] = a0 + rc.a0; Cc[t2] = b0 + rc.b0;
              for (int kk = 0; kk < 3; ++kk) r.clo[kk] = (int16_t)(Cc[kk] - o.lo[kk]);
              r.flo[d] = (int16_t)(side ? p.n[d] : 0);
              r.flo[t1] = (int16_t)(2 * (a0 + rc.a0) - p.lo[t1]);
              r.flo[t2] = (int16_t)(2 * (b0 + rc.b0) - p.lo[t2]);
              r.na = (int16_t)rc.na;
              r.nb = (int16_t)rc.nb;
              // another register on one of these coarse cells (a one-cell gap along d, or a
              // covered in-plane neighbour of a boundary cell): its reflux is ordered
              {
                const int cl[3] = {Cd, a0 + rc.a0, b0 + rc.b0};
                const int ch[3] = {Cd + 1, a0 + rc.a0 + rc.na, b0 + rc.b0 + rc.nb};
                int lo[3], hi[3];
                auto box = [&](int dd, int v) {   // the rectangle's cells shifted to coordinate v on axis dd
                  for (int k = 0; k < 3; ++k) { lo[k] = 0; hi[k] = 0; }
                  int m[3];
                  m[d] = 0; m[t1] = 1; m[t2] = 2;
                  for (int k = 0; k < 3; ++k) { lo[k] = cl[m[k]]; hi[k] = ch[m[k]]; }
                  lo[dd] = v;
                  hi[dd] = v + 1;
                };
                bool conflict = false;
                box(d, Cd - r.cside);
                conflict = conflict || covered_any(lo, hi);
                box(t1, a0 + rc.a0 - 1);
                conflict = conflict || covered_any(lo, hi);
                box(t1, a0 + rc.a0 + rc.na);
                conflict = conflict || covered_any(lo, hi);
                box(t2, b0 + rc.b0 - 1);
                conflict = conflict || covered_any(lo, hi);
                box(t2, b0 + rc.b0 + rc.nb);
                conflict = conflict || covered_any(lo, hi);
                r.ordered = conflict ? 1 : 0;
              }
              Rv.push_back(r);
            }
          }
            });
    for (int task = 0; task < ntask; ++task)
      if (!err[task].empty()) {
        msg = err[task];
        return AMR_ERR_NESTING;
      }
    // rectangles in task order, (d, side, fine patch): the reflux passes go over
    // (d, side) = 0 .. 5 in turn, and in one pass every coarse cell has at most
    // one register (a coarse face borders one fine patch)
    L.regs = FlatList<RegRect>();
    std::vector<int> cells;
    int64_t run = 0;
    for (int task = 0; task < ntask; ++task) {
      for (const RegRect& r : rs[task]) {
        L.regs.boxes.push_back(r);
        cells.push_back((int)r.na * r.nb);
        run += (int64_t)r.na * r.nb;
        if (r.ordered) L.reg_ordered[task / L.count] = 1;
      }
      L.reg_pass[task / L.count + 1] = (int)run;   // pass = task / count = 2 d + side
    }
    finish_flat(L.regs, cells, kBoxThreads);
  }
  // the coarse-side register flux reads two cells on either side of a coarse-fine
  // face: where that stencil leaves the coarse patch, its ghost cells are read,
  // so that face of the coarse patch keeps copied ghost cells
  for (int l = 1; l < nlev && direct_ok; ++l)
    for (const RegRect& r : plan.levels[l].regs.boxes) {
      const int f = r.clo[r.d] + (r.cside > 0 ? 1 : 0);   // face index between cells f-1 and f
      if (f - 2 < 0) direct[r.cpatch][2 * r.d] = 0;
      if (f + 1 >= P[r.cpatch].n[r.d]) direct[r.cpatch][2 * r.d + 1] = 0;
    }
  for (int i = 0; i < np; ++i)
    for (int f = 0; f < 6; ++f)
      if (!direct[i][f]) plan.desc[i].face[f] = own_face(plan.desc[i]);
  // per-stage ghost copies: the segments of the faces that are not read directly
  for (LevelPlan& L : plan.levels) {
    L.ghost_stage.clear();
    L.ghost_stage_first.assign(1, 0);
    for (int ii = 0; ii < L.count; ++ii) {
      const int i = L.first + ii;
      for (int e = L.ghost_first[ii]; e < L.ghost_first[ii + 1]; ++e)
        if (!direct[i][seg_face(L.ghost[e], P[i])]) L.ghost_stage.push_back(L.ghost[e]);
      L.ghost_stage_first.push_back((int)L.ghost_stage.size());
    }
  }
  build_flat(plan);
  return AMR_OK;
}


// ---------------------------------------------------------------------------
// Regridding (Sec. 3: hierarchy creation stays on the host)
// ---------------------------------------------------------------------------

namespace {

struct Key {
  int x, y, z;
  bool operator<(const Key& o) const { return std::tie(z, y, x) < std::tie(o.z, o.y, o.x); }
};

// block coordinates packed into one integer (each in [-2^20, 2^20))
int64_t pack(int x, int y, int z) {
  return ((int64_t)(z + (1 << 20)) << 42) | ((int64_t)(y + (1 << 20)) << 21) | (int64_t)(x + (1 << 20));
}
Key unpack(int64_t k) {
  Key r;
  r.x = (int)(k & ((1 << 21) - 1)) - (1 << 20);
  r.y = (int)((k >> 21) & ((1 << 21) - 1)) - (1 << 20);
  r.z = (int)(k >> 42) - (1 << 20);
  return r;
}

// Set of packed block keys (all >= 0): open addressing with linear probing in
// a power-of-two table kept at most half full; the slot hash is the 64-bit
// finaliser of MurmurHash3.  Membership only -- iteration order is not used
// for any result.
class KeySet {
 public:
  KeySet() : slots_(16, kEmpty), mask_(15) {}
  bool insert(int64_t k) {
    if (2 * (n_ + 1) > slots_.size()) grow();
    size_t h = mix(k) & mask_;
    while (slots_[h] != kEmpty) {
      if (slots_[h] == k) return false;
      h = (h + 1) & mask_;
    }
    slots_[h] = k;
    ++n_;
    return true;
  }
  size_t count(int64_t k) const {
    size_t h = mix(k) & mask_;
    while (slots_[h] != kEmpty) {
      if (slots_[h] == k) return 1;
      h = (h + 1) & mask_;
    }
    return 0;
  }
  size_t size() const { return n_; }
  bool empty() const { return n_ == 0; }
  void swap(KeySet& o) {
    slots_.swap(o.slots_);
    std::swap(n_, o.n_);
    std::swap(mask_, o.mask_);
  }
  std::vector<int64_t> keys() const {
    std::vector<int64_t> out;
    out.reserve(n_);
    for (int64_t k : slots_)
      if (k != kEmpty) out.push_back(k);
    return out;
  }

 private:
  static constexpr int64_t kEmpty = -1;
  static size_t mix(int64_t k) {
    uint64_t x = (uint64_t)k;
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return (size_t)x;
  }
  void grow() {
    std::vector<int64_t> old(slots_.size() * 2, kEmpty);
    old.swap(slots_);
    mask_ = slots_.size() - 1;
    n_ = 0;
    for (int64_t k : old)
      if (k != kEmpty) insert(k);
  }
  std::vector<int64_t> slots_;
  size_t n_ = 0, mask_;
};

// Set of block coordinates inside a known box [lo, hi): a dense bitmap when the
// box has at most 2^28 blocks, else a KeySet.  Coordinates outside the box are
// never members.
class BlockSet {
 public:
  void reset(const int lo[3], const int hi[3]) {
    int64_t vol = 1;
    for (int d = 0; d < 3; ++d) {
      lo_[d] = lo[d];
      n_[d] = std::max(hi[d] - lo[d], 0);
      vol *= n_[d];
    }
    dense_ = vol <= ((int64_t)1 << 28);
    bits_.assign(dense_ ? (size_t)((vol + 63) / 64) : 0, 0);
    hash_ = KeySet();
    count_ = 0;
  }
  void insert(int x, int y, int z) {
    if (dense_) {
      int64_t i;
      if (!index(x, y, z, i)) return;
      uint64_t& w = bits_[i >> 6];
      const uint64_t m = (uint64_t)1 << (i & 63);
      if (!(w & m)) { w |= m; ++count_; }
    } else if (inside(x, y, z) && hash_.insert(pack(x, y, z))) {
      ++count_;
    }
  }
  bool count(int x, int y, int z) const {
    if (dense_) {
      int64_t i;
      return index(x, y, z, i) && ((bits_[i >> 6] >> (i & 63)) & 1);
    }
    return inside(x, y, z) && hash_.count(pack(x, y, z));
  }
  bool empty() const { return count_ == 0; }

 private:
  bool inside(int x, int y, int z) const {
    return x >= lo_[0] && x < lo_[0] + n_[0] && y >= lo_[1] && y < lo_[1] + n_[1] && z >= lo_[2] &&
           z < lo_[2] + n_[2];
  }
  bool index(int x, int y, int z, int64_t& i) const {
    if (!inside(x, y, z)) return false;
    i = ((int64_t)(z - lo_[2]) * n_[1] + (y - lo_[1])) * n_[0] + (x - lo_[0]);
    return true;
  }
  int lo_[3] = {0, 0, 0}, n_[3] = {0, 0, 0};
  bool dense_ = true;
  std::vector<uint64_t> bits_;
  KeySet hash_;
  size_t count_ = 0;
};

// Tagged blocks of one level over its whole block grid [0, n): a dense bitmap
// whose set() may be called from many threads when the grid has at most 2^28
// blocks, else a KeySet (set() from one thread only).  keys() lists the members
// in (z, y, x) order.
class TagGrid {
 public:
  void reset(const int n[3]) {
    int64_t vol = 1;
    for (int d = 0; d < 3; ++d) {
      n_[d] = std::max(n[d], 0);
      vol *= n_[d];
    }
    dense_ = vol <= ((int64_t)1 << 28);
    bits_.assign(dense_ ? (size_t)((vol + 63) / 64) : 0, 0);
    hash_ = KeySet();
  }
  bool dense() const { return dense_; }
  // take a dense bitmap made elsewhere (bit i = block (x, y, z) with
  // i = (z n1 + y) n0 + x, 64 bits per word); false if the grid is not dense or
  // the size differs
  bool adopt(std::vector<uint64_t>& words) {
    if (!dense_ || words.size() != bits_.size()) return false;
    bits_.swap(words);
    return true;
  }
  void set(int x, int y, int z) {
    if (dense_) {
      const int64_t i = ((int64_t)z * n_[1] + y) * n_[0] + x;
      __atomic_fetch_or(&bits_[(size_t)(i >> 6)], (uint64_t)1 << (i & 63), __ATOMIC_RELAXED);
    } else {
      hash_.insert(pack(x, y, z));
    }
  }
  std::vector<Key> keys() const {
    std::vector<Key> out;
    if (!dense_) {
      for (int64_t k : hash_.keys()) out.push_back(unpack(k));
      std::sort(out.begin(), out.end());
      return out;
    }
    // runs of words in parallel, each run's members in order, concatenated
    const size_t nw = bits_.size();
    const int nrun = (int)std::min<size_t>(256, (nw + 4095) / 4096);
    std::vector<std::vector<Key>> part(std::max(nrun, 1));
    parallel_for(nrun, [&](int r) {
      const size_t w0 = nw * r / nrun, w1 = nw * (r + 1) / nrun;
      for (size_t w = w0; w < w1; ++w) {
        uint64_t b = bits_[w];
        while (b) {
          const int64_t i = (int64_t)(w << 6) + __builtin_ctzll(b);
          b &= b - 1;
          const int64_t row = i / n_[0];
          part[r].push_back(Key{(int)(i - row * n_[0]), (int)(row % n_[1]), (int)(row / n_[1])});
        }
      }
    });
    size_t tot = 0;
    for (const auto& v : part) tot += v.size();
    out.reserve(tot);
    for (const auto& v : part) out.insert(out.end(), v.begin(), v.end());
    return out;
  }

 private:
  int n_[3] = {0, 0, 0};
  bool dense_ = true;
  std::vector<uint64_t> bits_;
  KeySet hash_;
};

}  // namespace

amr_status check_regrid_params(const amr_config& cfg, const RegridParams& rp, std::string& msg) {
  const int B = rp.block;
  if (B < 2 || (B & 1) || rp.buffer < 0 || rp.buffer > B || rp.max_patch < 2 * B || rp.max_patch % (2 * B) ||
      rp.min_level < 0 || rp.min_level > cfg.max_level) {
    msg = "bad regrid parameters (block even >= 2, 0 <= buffer <= block, max_patch a multiple of 2 block)";
    return AMR_ERR_ARG;
  }
  return AMR_OK;
}

int64_t regrid_tag_blocks(const amr_config& cfg, const RegridParams& rp, int level, int nb[3]) {
  int64_t v = 1;
  for (int d = 0; d < 3; ++d) {
    nb[d] = (level_n(cfg, level, d) + rp.block - 1) / rp.block;
    v *= nb[d];
  }
  return v;
}

namespace {
amr_status cluster_tagged(const amr_config& cfg, const std::vector<HPatch>& old, std::vector<TagGrid>& tags,
                          const RegridParams& rp, std::vector<HPatch>& out, std::string& msg);
}  // namespace

amr_status cluster_patches(const amr_config& cfg, const std::vector<HPatch>& old,
                           const std::vector<std::vector<uint8_t>>& flags, const RegridParams& rp,
                           std::vector<HPatch>& out, std::string& msg) {
  amr_status st = check_regrid_params(cfg, rp, msg);
  if (st != AMR_OK) return st;
  const int B = rp.block, L = cfg.max_level, l0 = rp.min_level;
  auto nb = [&](int l, int d) { return (level_n(cfg, l, d) + B - 1) / B; };
  auto per = [&](int d) { return periodic(cfg, d); };
  std::vector<TagGrid> tags(L + 1);   // level L (the finest allowed) is never flagged
  for (int l = l0; l < L; ++l) {
    const int n[3] = {nb(l, 0), nb(l, 1), nb(l, 2)};
    tags[l].reset(n);
  }
  // 1. flagged cells, grown by the buffer, mark blocks of their level (first on a
  //    per-patch block grid, so each block is listed once per patch; patches in
  //    parallel, straight into a dense tag grid, else listed and inserted after)
  std::vector<std::vector<int64_t>> pk(old.size());
  parallel_for((int)old.size(), [&](int i) {
    const HPatch& p = old[i];
    if (p.level < l0 || p.level >= L || flags[i].empty()) return;
    const int l = p.level;
    int g0[3], gn[3];
    for (int d = 0; d < 3; ++d) {
      g0[d] = (int)std::floor((double)(p.lo[d] - rp.buffer) / B);
      gn[d] = (int)std::floor((double)(p.lo[d] + p.n[d] - 1 + rp.buffer) / B) - g0[d] + 1;
    }
    std::vector<unsigned char> mark((size_t)gn[0] * gn[1] * gn[2], 0);
    for (int k = 0; k < p.n[2]; ++k)
      for (int j = 0; j < p.n[1]; ++j)
        for (int ii = 0; ii < p.n[0]; ++ii) {
          if (!flags[i][((size_t)k * p.n[1] + j) * p.n[0] + ii]) continue;
          const int c[3] = {p.lo[0] + ii, p.lo[1] + j, p.lo[2] + k};
          int b0[3], b1[3];
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            // blocks touched by [c - buffer, c + buffer]
            int lo = c[d] - rp.buffer, hi = c[d] + rp.buffer;
            int N = level_n(cfg, l, d);
            if (!per(d)) { lo = std::max(lo, 0); hi = std::min(hi, N - 1); }
            b0[d] = (int)std::floor((double)lo / B) - g0[d];
            b1[d] = (int)std::floor((double)hi / B) - g0[d];
            if (b1[d] < b0[d]) ok = false;
          }
          if (!ok) continue;
          for (int z = b0[2]; z <= b1[2]; ++z)
            for (int y = b0[1]; y <= b1[1]; ++y)
              for (int x = b0[0]; x <= b1[0]; ++x) mark[((size_t)z * gn[1] + y) * gn[0] + x] = 1;
        }
    for (int z = 0; z < gn[2]; ++z)
      for (int y = 0; y < gn[1]; ++y)
        for (int x = 0; x < gn[0]; ++x) {
          if (!mark[((size_t)z * gn[1] + y) * gn[0] + x]) continue;
          int q[3] = {x + g0[0], y + g0[1], z + g0[2]};
          for (int d = 0; d < 3; ++d) {
            int n = nb(l, d);
            if (per(d)) q[d] = ((q[d] % n) + n) % n;
          }
          if (tags[l].dense()) tags[l].set(q[0], q[1], q[2]);
          else pk[i].push_back(pack(q[0], q[1], q[2]));
        }
  });
  for (size_t i = 0; i < old.size(); ++i)
    for (int64_t k : pk[i]) {
      const Key b = unpack(k);
      tags[old[i].level].set(b.x, b.y, b.z);
    }
  return cluster_tagged(cfg, old, tags, rp, out, msg);
}

namespace {
// Greedy box merge of the refinable blocks `order` of level l (in (z, y, x)
// order, bounding box [rlo, rhi)): from each block not yet taken, extend along
// x, then y, then z while every block is refinable and free, up to max_patch
// fine cells; each box becomes a patch of level l+1.  `refine` receives the
// refinable set.
void merge_boxes(const amr_config& cfg, const RegridParams& rp, int l, const std::vector<Key>& order,
                 const int rlo[3], const int rhi[3], std::vector<HPatch>& out, BlockSet& refine) {
  const int B = rp.block;
  const int maxb = rp.max_patch / (2 * B);
  BlockSet done;
  refine.reset(rlo, rhi);
  done.reset(rlo, rhi);
  for (const Key& b : order) refine.insert(b.x, b.y, b.z);
  // greedy box merge in (z, y, x) order (the order of the tags): extend along x,
  // then y, then z
  for (const Key& b : order) {
    if (done.count(b.x, b.y, b.z)) continue;
    auto free_ = [&](int x, int y, int z) { return refine.count(x, y, z) && !done.count(x, y, z); };
    int nx = 1, ny = 1, nz = 1;
    while (nx < maxb && free_(b.x + nx, b.y, b.z)) ++nx;
    auto row_ok = [&](int y, int z) {
      for (int i = 0; i < nx; ++i)
        if (!free_(b.x + i, y, z)) return false;
      return true;
    };
    while (ny < maxb && row_ok(b.y + ny, b.z)) ++ny;
    auto slab_ok = [&](int z) {
      for (int j = 0; j < ny; ++j)
        if (!row_ok(b.y + j, z)) return false;
      return true;
    };
    while (nz < maxb && slab_ok(b.z + nz)) ++nz;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) done.insert(b.x + x, b.y + y, b.z + z);
    HPatch f{};
    f.level = l + 1;
    const int bl[3] = {b.x, b.y, b.z}, bn[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
      const int Nf = level_n(cfg, l + 1, d);
      f.lo[d] = 2 * B * bl[d];
      f.n[d] = std::min(2 * B * bn[d], Nf - f.lo[d]);
    }
    out.push_back(f);
  }
}

// Steps 2-3 of the clustering from the block tags of levels min_level .. L-1.
amr_status cluster_tagged(const amr_config& cfg, const std::vector<HPatch>& old, std::vector<TagGrid>& tags,
                          const RegridParams& rp, std::vector<HPatch>& out, std::string& msg) {
  (void)msg;
  const int B = rp.block, L = cfg.max_level, l0 = rp.min_level;
  auto nb = [&](int l, int d) { return (level_n(cfg, l, d) + B - 1) / B; };
  auto per = [&](int d) { return periodic(cfg, d); };
  // 2. a tag on level l needs its parent region (and a ring for nesting) refined on level l-1
  for (int l = L - 1; l > l0; --l) {
    TagGrid parents;   // parent blocks of the tags (8 children share one)
    {
      const int n[3] = {nb(l - 1, 0), nb(l - 1, 1), nb(l - 1, 2)};
      parents.reset(n);
    }
    const std::vector<Key> tk = tags[l].keys();
    auto parent_of = [&](int t) { parents.set(tk[t].x >> 1, tk[t].y >> 1, tk[t].z >> 1); };
    if (parents.dense()) parallel_for((int)tk.size(), parent_of);
    else for (int t = 0; t < (int)tk.size(); ++t) parent_of(t);
    const std::vector<Key> pk2 = parents.keys();
    auto ring = [&](int t) {
      const int pb[3] = {pk2[t].x, pk2[t].y, pk2[t].z};
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int q[3] = {pb[0] + dx, pb[1] + dy, pb[2] + dz};
            bool ok = true;
            for (int d = 0; d < 3 && ok; ++d) {
              int n = nb(l - 1, d);
              if (q[d] < 0 || q[d] >= n) {
                if (per(d)) q[d] = ((q[d] % n) + n) % n;
                else ok = false;
              }
            }
            if (ok) tags[l - 1].set(q[0], q[1], q[2]);
          }
    };
    if (tags[l - 1].dense()) parallel_for((int)pk2.size(), ring);
    else for (int t = 0; t < (int)pk2.size(); ++t) ring(t);
  }
  // 3. top-down: keep levels <= l0, then cluster refinable blocks of each level
  out.clear();
  for (const HPatch& p : old)
    if (p.level <= l0) out.push_back(p);
  // blocks of level l0 fully covered by its patches
  BlockSet cover;
  {
    auto block_range = [&](const HPatch& p, int* a0, int* a1) {
      for (int d = 0; d < 3; ++d) {
        a0[d] = (p.lo[d] + B - 1) / B;
        a1[d] = (p.lo[d] + p.n[d]) / B;
        // a partial block at the domain's end counts when the patch reaches the end
        if (p.lo[d] + p.n[d] == level_n(cfg, l0, d) && level_n(cfg, l0, d) % B) a1[d] += 1;
      }
    };
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (const HPatch& p : old) {
      if (p.level != l0) continue;
      int a0[3], a1[3];
      block_range(p, a0, a1);
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], a0[d]); hi[d] = std::max(hi[d], a1[d]); }
    }
    if (lo[0] > hi[0]) for (int d = 0; d < 3; ++d) lo[d] = hi[d] = 0;
    cover.reset(lo, hi);
    for (const HPatch& p : old) {
      if (p.level != l0) continue;
      int a0[3], a1[3];
      block_range(p, a0, a1);
      for (int z = a0[2]; z < a1[2]; ++z)
        for (int y = a0[1]; y < a1[1]; ++y)
          for (int x = a0[0]; x < a1[0]; ++x) cover.insert(x, y, z);
    }
  }
  // blocks of level l covered by its patches: `cover` for l0, afterwards the
  // refined blocks of level l-1 seen through the parent coordinates
  BlockSet prev_refine;
  bool coarse_cover = false;
  auto cover_count = [&](int x, int y, int z) {
    return coarse_cover ? prev_refine.count(x >> 1, y >> 1, z >> 1) : cover.count(x, y, z);
  };
  for (int l = l0; l < L; ++l) {
    const std::vector<Key> tl = tags[l].keys();   // (z, y, x) order
    std::vector<unsigned char> refinable(tl.size(), 0);
    parallel_for((int)tl.size(), [&](int ti) {
      const Key b = tl[ti];
      bool ok = true;
      for (int dz = -1; dz <= 1 && ok; ++dz)
        for (int dy = -1; dy <= 1 && ok; ++dy)
          for (int dx = -1; dx <= 1 && ok; ++dx) {
            int q[3] = {b.x + dx, b.y + dy, b.z + dz};
            bool outside = false;
            for (int d = 0; d < 3; ++d) {
              int n = nb(l, d);
              if (q[d] < 0 || q[d] >= n) {
                if (per(d)) q[d] = ((q[d] % n) + n) % n;
                else outside = true;
              }
            }
            if (!outside && !cover_count(q[0], q[1], q[2])) ok = false;
          }
      refinable[ti] = ok;
    });
    std::vector<Key> order;
    int rlo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, rhi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (size_t ti = 0; ti < tl.size(); ++ti)
      if (refinable[ti]) {
        const Key b = tl[ti];
        order.push_back(b);
        const int c[3] = {b.x, b.y, b.z};
        for (int d = 0; d < 3; ++d) { rlo[d] = std::min(rlo[d], c[d]); rhi[d] = std::max(rhi[d], c[d] + 1); }
      }
    if (order.empty()) break;
    BlockSet refine;
    merge_boxes(cfg, rp, l, order, rlo, rhi, out, refine);
    // every refinable block is now in a new patch: a block of level l+1 lies in
    // the new patches exactly when its parent block (coordinates halved) is one
    std::swap(prev_refine, refine);
    coarse_cover = true;
  }
  return AMR_OK;
}
}  // namespace

std::vector<uint64_t> regrid_base_cover(const amr_config& cfg, const std::vector<HPatch>& old,
                                        const RegridParams& rp) {
  const int B = rp.block, l0 = rp.min_level;
  int nb[3];
  const int64_t nbt = regrid_tag_blocks(cfg, rp, l0, nb);
  std::vector<uint64_t> w((size_t)((nbt + 63) / 64), 0);
  for (const HPatch& p : old) {
    if (p.level != l0) continue;
    int a0[3], a1[3];
    for (int d = 0; d < 3; ++d) {   // the blocks fully inside p (as the clustering's cover)
      a0[d] = (p.lo[d] + B - 1) / B;
      a1[d] = (p.lo[d] + p.n[d]) / B;
      if (p.lo[d] + p.n[d] == level_n(cfg, l0, d) && level_n(cfg, l0, d) % B) a1[d] += 1;
    }
    for (int z = a0[2]; z < a1[2]; ++z)
      for (int y = a0[1]; y < a1[1]; ++y)
        for (int x = a0[0]; x < a1[0]; ++x) {
          const int64_t i = ((int64_t)z * nb[1] + y) * nb[0] + x;
          w[(size_t)(i >> 6)] |= (uint64_t)1 << (i & 63);
        }
  }
  return w;
}

amr_status cluster_patches_refinable(const amr_config& cfg, const std::vector<HPatch>& old,
                                     std::vector<std::vector<uint64_t>>& refinable, const RegridParams& rp,
                                     std::vector<HPatch>& out, std::string& msg) {
  amr_status st = check_regrid_params(cfg, rp, msg);
  if (st != AMR_OK) return st;
  const int L = cfg.max_level, l0 = rp.min_level;
  out.clear();
  for (const HPatch& p : old)
    if (p.level <= l0) out.push_back(p);
  for (int l = l0; l < L; ++l) {
    int n[3];
    regrid_tag_blocks(cfg, rp, l, n);
    TagGrid R;
    R.reset(n);
    if (l >= (int)refinable.size() || !R.adopt(refinable[l])) {
      msg = "regrid: refinable blocks of a level do not match its block grid";
      return AMR_ERR_ARG;
    }
    const std::vector<Key> order = R.keys();   // (z, y, x) order
    if (order.empty()) break;
    int rlo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, rhi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (const Key& b : order) {
      const int c[3] = {b.x, b.y, b.z};
      for (int d = 0; d < 3; ++d) { rlo[d] = std::min(rlo[d], c[d]); rhi[d] = std::max(rhi[d], c[d] + 1); }
    }
    BlockSet refine;
    merge_boxes(cfg, rp, l, order, rlo, rhi, out, refine);
  }
  return AMR_OK;
}

void build_regrid_fill(const std::vector<HPatch>& oldp, const std::vector<HPatch>& newp, int keep_level,
                       RegridFill& fill) {
  int L = 0;
  for (const HPatch& p : newp) L = std::max(L, p.level);
  fill.copy.assign(L + 1, {});
  fill.fresh.assign(L + 1, {});
  std::vector<int> ofirst, ocount;
  for (size_t q = 0; q < oldp.size(); ++q) {
    const int l = oldp[q].level;
    if ((int)ofirst.size() <= l) { ofirst.resize(l + 1, (int)q); ocount.resize(l + 1, 0); }
    ocount[l]++;
  }
  std::vector<std::unique_ptr<PatchIndex>> oix(ofirst.size());
  for (size_t l = 0; l < ofirst.size(); ++l) oix[l].reset(new PatchIndex(oldp, ofirst[l], ocount[l]));
  const int nnew = (int)newp.size();
  std::vector<std::vector<CopySeg>> cs(nnew);
  std::vector<std::vector<ProlongBox>> fs(nnew);
  parallel_for(nnew, [&](int ii) {
    const size_t i = (size_t)ii;
    const HPatch& p = newp[i];
    if (p.level <= keep_level) return;
    const int l = p.level;
    std::vector<int> cand;
    std::vector<CopySeg>& Cv = cs[ii];
    std::vector<ProlongBox>& Fv = fs[ii];
    // the new patch's cells outside every old patch of its level, as boxes: the
    // patch box minus each overlapping old box in turn (a box minus a box is at
    // most six boxes: below and above in z, then in y, then in x)
    struct B3 { int lo[3], hi[3]; };
    std::vector<B3> rest{{{p.lo[0], p.lo[1], p.lo[2]}, {p.lo[0] + p.n[0], p.lo[1] + p.n[1], p.lo[2] + p.n[2]}}}, next;
    if (l < (int)oix.size()) {
      int qlo[3], qhi[3];
      for (int d = 0; d < 3; ++d) { qlo[d] = p.lo[d]; qhi[d] = p.lo[d] + p.n[d]; }
      oix[l]->query(qlo, qhi, cand);
    }
    for (int q : cand) {
      const HPatch& o = oldp[q];
      if (o.level != l) continue;
      int lo[3], hi[3];
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::max(p.lo[d], o.lo[d]);
        hi[d] = std::min(p.lo[d] + p.n[d], o.lo[d] + o.n[d]);
        if (lo[d] >= hi[d]) ok = false;
      }
      if (!ok) continue;
      CopySeg sg{};
      sg.dst_patch = (int)i;
      sg.src_patch = (int)q;
      for (int d = 0; d < 3; ++d) {
        sg.dlo[d] = (int16_t)(lo[d] - p.lo[d]);
        sg.dn[d] = (int16_t)(hi[d] - lo[d]);
        sg.sh[d] = (int16_t)(p.lo[d] - o.lo[d]);
        sg.mode[d] = 0;
      }
      Cv.push_back(sg);
      next.clear();
      for (const B3& a : rest) {
        int c0[3], c1[3];
        bool meet = true;
        for (int d = 0; d < 3; ++d) {
          c0[d] = std::max(a.lo[d], lo[d]);
          c1[d] = std::min(a.hi[d], hi[d]);
          if (c0[d] >= c1[d]) meet = false;
        }
        if (!meet) { next.push_back(a); continue; }
        B3 core = a;   // shrinks to the overlap axis by axis, z first
        for (int d = 2; d >= 0; --d) {
          if (core.lo[d] < c0[d]) { B3 b = core; b.hi[d] = c0[d]; next.push_back(b); }
          if (c1[d] < core.hi[d]) { B3 b = core; b.lo[d] = c1[d]; next.push_back(b); }
          core.lo[d] = c0[d];
          core.hi[d] = c1[d];
        }
      }
      rest.swap(next);
    }
    split_copy(Cv, 0);
    for (const B3& a : rest) {
      ProlongBox b{};
      b.patch = (int)i;
      for (int d = 0; d < 3; ++d) {
        b.lo[d] = (int16_t)(a.lo[d] - p.lo[d]);
        b.n[d] = (int16_t)(a.hi[d] - a.lo[d]);
      }
      Fv.push_back(b);
    }
    split_prolong(Fv, 0);
  });
  for (int ii = 0; ii < nnew; ++ii) {
    const int l = newp[ii].level;
    fill.copy[l].insert(fill.copy[l].end(), cs[ii].begin(), cs[ii].end());
    fill.fresh[l].insert(fill.fresh[l].end(), fs[ii].begin(), fs[ii].end());
  }
}

}  // namespace amr
