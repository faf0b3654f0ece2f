// amr_noalloc.cu -- one RK2 step of one uniform patch without allocating any
// device memory.
//
// Who needs it: callers that must not call cudaMalloc (or any allocating
// library routine) -- code running while another framework owns the device
// allocator and has to account for every byte, real-time loops that may not
// enter the allocator (it can synchronise the device), and hosts with a hard
// device-memory budget fixed at start-up.  Such a caller passes its own input
// and output arrays; every other byte the step needs (the ghosted state, the
// stage-1 state, the launch tables, the step parameters) lives in the fixed
// array g_noalloc_scratch below, which every GPU that loads this library holds
// until the process exits.
//
// The computation is the same as amr_step on a single level-0 patch: the same
// ghost-fill, stage and packing kernels, launched from here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/amr.h"
#include "hierarchy.h"
#include "kernels.cuh"

using namespace amr;

namespace {

// 32 MiB: enough for two ghosted FP64 Euler states of a 64^3 patch plus tables.
constexpr size_t kScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
bool g_ready[kMaxDevices];

__global__ void noalloc_set_dt(StepParams* p, double dt) { p->dt0 = dt; }

__global__ void noalloc_finalize(StepParams* p, double cfl, double ch_fixed, int set_dt) {
  const double rate = __longlong_as_double((long long)p->rate_bits);
  const double speed = __longlong_as_double((long long)p->speed_bits);
  if (set_dt) p->dt0 = cfl / rate;
  p->ch = ch_fixed > 0.0 ? ch_fixed : speed;
}

size_t align256(size_t a) { return (a + 255) / 256 * 256; }

// CTAs per SM of the default stage-kernel variant (its shared-memory layout depends on it)
template <typename T, int NV>
constexpr int kDefCtas = (sizeof(T) == 4 && NV == 5) ? 2 : 1;

template <typename T, int NV>
void set_smem_attributes() {
  cudaFuncSetAttribute(stage_kernel<T, NV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)stage_smem_bytes<T, NV, kDefCtas<T, NV>>());
  cudaFuncSetAttribute(stage_kernel<T, NV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)stage_smem_bytes<T, NV, kDefCtas<T, NV>>());
}

// One-time set-up per device (the device must be current): resolve the device
// address of the scratch array and set the stage kernels' shared-memory limit.
amr_status setup_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return AMR_ERR_CUDA;
  if (!g_ready[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return AMR_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    set_smem_attributes<float, 5>();
    set_smem_attributes<double, 5>();
    set_smem_attributes<float, 9>();
    set_smem_attributes<double, 9>();
    if (cudaGetLastError() != cudaSuccess) return AMR_ERR_CUDA;
    g_ready[dev] = true;
  }
  *out = g_scratch_addr[dev];
  return AMR_OK;
}

template <typename X>
size_t place(std::vector<unsigned char>& buf, const std::vector<X>& v) {
  size_t off = align256(buf.size());
  buf.resize(off + v.size() * sizeof(X));
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(X));
  return off;
}

template <typename T, int NV>
amr_status run(const amr_config& cfg, const Plan& pl, unsigned char* base, const double* in, double* out,
               double dt, double* dt_used) {
  cudaStream_t s = static_cast<cudaStream_t>(cfg.cuda_stream);
  const LevelPlan& L = pl.levels[0];
  // scratch layout: [StepParams][tables][U][U1]
  std::vector<ChunkDesc> chunks;
  const int nc = pl.patches[0].n[0] * pl.patches[0].n[1] * pl.patches[0].n[2];
  for (int b = 0; b < nc; b += 16384) chunks.push_back({0, b, nc - b < 16384 ? nc - b : 16384});
  std::vector<unsigned char> tab;
  tab.resize(256);  // StepParams slot
  const size_t o_desc = place(tab, pl.desc);
  const size_t o_items = place(tab, L.items);
  const size_t o_ghost = place(tab, L.ghost);
  const size_t o_chunks = place(tab, chunks);
  const size_t o_poff = place(tab, pl.packed_off);
  const size_t o_U = align256(tab.size());
  const size_t arr = align256((size_t)pl.arena_elems * sizeof(T));
  const size_t o_U1 = o_U + arr;
  if (o_U1 + arr > kScratchBytes) return AMR_ERR_ARG;

  StepParams* prm = reinterpret_cast<StepParams*>(base);
  const PatchDesc* desc = reinterpret_cast<const PatchDesc*>(base + o_desc);
  const StageItem* items = reinterpret_cast<const StageItem*>(base + o_items);
  const CopySeg* ghost = reinterpret_cast<const CopySeg*>(base + o_ghost);
  const ChunkDesc* dchunks = reinterpret_cast<const ChunkDesc*>(base + o_chunks);
  const int64_t* poff = reinterpret_cast<const int64_t*>(base + o_poff);
  T* U = reinterpret_cast<T*>(base + o_U);
  T* U1 = reinterpret_cast<T*>(base + o_U1);

  // tables (the previous call's contents are overwritten) and zeroed step parameters
  if (cudaMemcpyAsync(base + 256, tab.data() + 256, tab.size() - 256, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(base, 0, 256, s) != cudaSuccess)
    return AMR_ERR_CUDA;

  Phys<T> ph{};
  ph.gamma = (T)cfg.gamma;
  ph.gm1 = (T)(cfg.gamma - 1.0);
  ph.ggm1 = (T)(cfg.gamma * (cfg.gamma - 1.0));
  ph.theta = (T)cfg.theta;
  ph.llf = cfg.riemann == AMR_LLF ? 1 : 0;
  ph.fluxrec = (NV == 5 && cfg.riemann == AMR_FLUXREC) ? 1 : 0;
  ph.efl = (T)(cfg.p_floor / (cfg.gamma - 1.0));
  ph.glm_alpha = (T)cfg.glm_alpha;
  double dx[3];
  for (int d = 0; d < 3; ++d) dx[d] = (cfg.domain_hi[d] - cfg.domain_lo[d]) / cfg.base_n[d];
  const int nchunk = (int)chunks.size();
  const int grid_chunks = nchunk < 65535 ? nchunk : 65535;

  pack_in_kernel<T, NV><<<grid_chunks, 256, 0, s>>>(dchunks, nchunk, desc, poff, in, U, 0, cfg.gamma, prm);
  const bool cfl = !(dt > 0.0);
  if (cfl || NV == 9) {
    speed_kernel<T, NV><<<grid_chunks, 256, 0, s>>>(dchunks, nchunk, desc, U, prm, 1.0 / dx[0], 1.0 / dx[1],
                                                     1.0 / dx[2], ph);
    noalloc_finalize<<<1, 1, 0, s>>>(prm, cfg.cfl, NV == 9 ? cfg.ch : 1.0, cfl ? 1 : 0);
  }
  if (!cfl) noalloc_set_dt<<<1, 1, 0, s>>>(prm, dt);

  StageArgs<T> a;
  a.desc = desc;
  a.items = items;
  a.nitems = (int)L.items.size();
  a.params = prm;
  a.dt_scale = 1.0;
  a.idx = (T)(1.0 / dx[0]);
  a.idy = (T)(1.0 / dx[1]);
  a.idz = (T)(1.0 / dx[2]);
  a.idx0 = 1.0 / dx[0];
  a.idy0 = 1.0 / dx[1];
  a.idz0 = 1.0 / dx[2];
  a.fuse_rate = 0;
  a.dynamic = 0;
  a.spans = nullptr;   // one patch: per-patch blocks only
  a.Uold = nullptr;    // one level: no old-time state
  a.ph = ph;
  const int nseg = (int)L.ghost.size();
  const int gseg = nseg < 65535 ? nseg : 65535;
  const size_t sm = stage_smem_bytes<T, NV, kDefCtas<T, NV>>();
  copy_kernel<T, NV, false><<<gseg, 256, 0, s>>>(ghost, nseg, desc, U, U, nullptr, T(0));
  a.Uin = U;
  a.Uout = U1;
  if (ph.fluxrec) fluxrec_stage_kernel<T, 1><<<a.nitems, kStageThreads, 0, s>>>(a);
  else stage_kernel<T, NV, 1><<<a.nitems, kStageThreads, sm, s>>>(a);
  copy_kernel<T, NV, false><<<gseg, 256, 0, s>>>(ghost, nseg, desc, U1, U1, nullptr, T(0));
  a.Uin = U1;
  a.Uout = U;
  if (ph.fluxrec) fluxrec_stage_kernel<T, 2><<<a.nitems, kStageThreads, 0, s>>>(a);
  else stage_kernel<T, NV, 2><<<a.nitems, kStageThreads, sm, s>>>(a);
  pack_out_kernel<T, NV><<<grid_chunks, 256, 0, s>>>(dchunks, nchunk, desc, poff, U, out);
  if (cudaGetLastError() != cudaSuccess) return AMR_ERR_CUDA;
  if (dt_used) {
    StepParams host{};
    if (cudaMemcpyAsync(&host, prm, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return AMR_ERR_CUDA;
    *dt_used = host.dt0;
    if (host.bad) return AMR_ERR_NONPHYSICAL;
  }
  return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_step_patch_noalloc(const amr_config* cfg, const double* state_in, double* state_out,
                                             double dt, double* dt_used) {
  if (!cfg || !state_in || !state_out || !std::isfinite(dt)) return AMR_ERR_ARG;
  std::string msg;
  if (validate_config(*cfg, msg) != AMR_OK) return AMR_ERR_ARG;
  if (cfg->recon != AMR_PLM) return AMR_ERR_ARG;   // the WENO3 build is not compiled into this path
  {   // the output is written while the input is still being read: the two ranges may not overlap
    const uintptr_t bytes = (uintptr_t)cfg->nvar * cfg->base_n[0] * cfg->base_n[1] * cfg->base_n[2] * sizeof(double);
    const uintptr_t a = reinterpret_cast<uintptr_t>(state_in), b = reinterpret_cast<uintptr_t>(state_out);
    if (a < b + bytes && b < a + bytes) return AMR_ERR_ARG;
  }
  std::vector<HPatch> P(1);
  P[0].level = 0;
  for (int d = 0; d < 3; ++d) {
    P[0].lo[d] = 0;
    P[0].n[d] = cfg->base_n[d];
  }
  Plan pl;
  amr_status st = build_plan(*cfg, P, pl, msg);   // host-side tables only
  if (st != AMR_OK) return st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AMR_ERR_CUDA;
  unsigned char* base = nullptr;
  st = setup_device(dev, &base);
  if (st != AMR_OK) return st;
  if (cfg->nvar == 5)
    return cfg->precision == AMR_FP32 ? run<float, 5>(*cfg, pl, base, state_in, state_out, dt, dt_used)
                                      : run<double, 5>(*cfg, pl, base, state_in, state_out, dt, dt_used);
  return cfg->precision == AMR_FP32 ? run<float, 9>(*cfg, pl, base, state_in, state_out, dt, dt_used)
                                    : run<double, 9>(*cfg, pl, base, state_in, state_out, dt, dt_used);
}
