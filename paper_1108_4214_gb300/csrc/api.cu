// Host side of libdynbond: the C ABI of include/dynbond.h.  A context owns
// the device topology (bond slots, per-replica angle / dihedral lists sized
// for the worst case), the per-call scratch, and two CUDA graphs (one call of
// the fix; one force evaluation) replayed with new arguments each call.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace dynbond;

struct dynbond_ctx {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;                        // the breakage nomination's branch of a call
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // its fork from and join into `stream`
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;  // the bond forces' branch of a combined call
  dynbond_params prm{};
  RuleTab rt{};
  RuleTab* d_rt = nullptr;  // device copy read by the kernels
  FF ff{};
  long long N = 0;
  int R = 0;
  long long n_cells = 0;
  long long W = 0;  // bitmap words
  Dev d{};
  std::vector<void*> allocs;
  cudaGraphExec_t g_step = nullptr, g_forces = nullptr;
  cudaGraphExec_t g_both = nullptr;  // step + forces in one graph (dynbond_step_forces)
  bool use_graph = true;
  bool pdl = true;  // programmatic dependent launch between the kernels of a call
  int block = 256;
  int grid_bead = 0, grid_scan = 0, grid_cand = 0, grid_match = 0, grid_seg = 0, grid_edit = 0, grid_purge = 0;
  int grid_adf = 0, grid_bf = 0;
  long long st_scan_n = 0;
  void* small = nullptr;
  size_t small_bytes = 0;
  void* status_all = nullptr;
  size_t status_bytes = 0;
  dynbond_status sticky = DYNBOND_OK;
  std::string last_error;
  bool profile = false;
  std::vector<cudaEvent_t> ev_step, ev_forces;
  std::vector<const char*> names_step, names_forces;
  std::vector<float> last_step_ms, last_forces_ms;
  int last_profiled = 0;  // 1 = step, 2 = forces
  int4* h2d_pos = nullptr;
  float4* d2h_force = nullptr;
  double* d2h_ev = nullptr;
  // cell geometry (re-chosen by the autotuner; never changes results)
  std::vector<long long> h_box;
  long long reach = 0;
  bool octant = false;          // candidate search by octant (see set_geometry)          // smallest integer cell width covering the largest creation distance
  long long max_cells = 0;      // cells allocated (geometry at scale 1)
  int* d_nc = nullptr;
  int* d_ncz = nullptr;
  int4* d_geo = nullptr;
  long long* d_cb = nullptr;
  dynbond_tuning tuning{};
  unsigned long long* d_hash = nullptr;  // per-replica topology hashes
  // candidate search by staged tiles (k_candidates_tile): work items of the
  // current geometry, or none (global-memory search)
  int4* d_ctile = nullptr;
  long long ctile_cap = 0;
  bool cand_tiles = false;      // the search runs on staged tiles (tiles_avail && tiles_on)
  bool tiles_avail = false;     // the current geometry has staged work items
  bool tiles_on = false;        // autotuner's choice between staged and global search (global until timed)
  bool global_search = false;   // DYNBOND_FLAG_GLOBAL_SEARCH
  bool staged_search = false;   // DYNBOND_FLAG_STAGED_SEARCH
  bool persistent = false;      // DYNBOND_FLAG_PERSISTENT (and not profiling)
  int grid_persist = 0;
  int grid_ctile = 0;
  bool tuned = false;
};

namespace {

thread_local std::string g_create_error;  // message of the last failed dynbond_create

dynbond_status fail(dynbond_ctx* c, dynbond_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      return fail(ctx, DYNBOND_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    }                                                                                         \
  } while (0)

template <class T>
dynbond_status dalloc(dynbond_ctx* c, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DYNBOND_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return DYNBOND_OK;
}

// floor((dist * 2^20)^2), exact for the double dist: with dist * 2^20 = m 2^e
// (m an integer below 2^53) the square m^2 2^(2e) fits 128-bit integers.
long long quantized_r2(double dist) {
  if (!(dist > 0.0) || !std::isfinite(dist)) return 0;
  int e;
  double f = std::frexp(std::ldexp(dist, 20), &e);  // dist 2^20 = f 2^e, f in [0.5, 1)
  unsigned long long m = (unsigned long long)std::ldexp(f, 53);
  int sh = 2 * (e - 53);
  unsigned __int128 sq = (unsigned __int128)m * m;
  const unsigned __int128 cap = (unsigned __int128)0x7FFFFFFFFFFFFFFFull;
  if (sh >= 0) {
    if (sh >= 63 || (sq << sh) > cap) return 0x7FFFFFFFFFFFFFFFll;
    return (long long)(sq << sh);
  }
  if (-sh >= 128) return 0;
  unsigned __int128 v = sq >> (-sh);
  return v > cap ? 0x7FFFFFFFFFFFFFFFll : (long long)v;
}

unsigned long long prob_threshold(double p) {
  if (!(p > 0.0)) return 0ull;
  if (p >= 1.0) return 1ull << 32;
  return (unsigned long long)(p * 4294967296.0);
}

bool mask_ok(uint32_t m) { return m != 0 && (m >> DYNBOND_MAX_TYPES) == 0; }
bool btype_ok(int t) { return t >= 1 && t < DYNBOND_MAX_TYPES; }

dynbond_status build_rules(dynbond_ctx* c, const dynbond_rule* rules, int n) {
  if (n < 0 || n > MAXR) return fail(c, DYNBOND_EINVAL, "n_rules must be in [0, 32]");
  if (n > 0 && !rules) return fail(c, DYNBOND_EINVAL, "rules is NULL");
  RuleTab& rt = c->rt;
  std::memset(&rt, 0, sizeof(rt));
  rt.n = n;
  for (int k = 0; k < n; ++k) {
    const dynbond_rule& r = rules[k];
    std::string where = "rule " + std::to_string(k) + ": ";
    rt.kind[k] = r.kind;
    rt.type[k] = r.type;
    rt.type2[k] = r.type2;
    rt.maxn[k] = r.maxn;
    for (int q = 0; q < 4; ++q) rt.bead[k][q] = r.bead_mask[q];
    for (int q = 0; q < 3; ++q) rt.bond[k][q] = r.bond_mask[q];
    bool dist_ok = std::isfinite(r.dist) && r.dist >= 0.0;
    bool prob_ok = std::isfinite(r.prob) && r.prob >= 0.0;
    switch (r.kind) {
      case DYNBOND_CREATEBOND:
      case DYNBOND_CREATEDIRBOND:
        if (!btype_ok(r.type) || (r.kind == DYNBOND_CREATEDIRBOND && !btype_ok(r.type2)))
          return fail(c, DYNBOND_EINVAL, where + "bond type out of range 1..15");
        if (!mask_ok(r.bead_mask[0]) || !mask_ok(r.bead_mask[1]))
          return fail(c, DYNBOND_EINVAL, where + "bead type masks must be nonzero over types 0..15");
        if (!dist_ok || !prob_ok) return fail(c, DYNBOND_EINVAL, where + "bad distance or probability");
        rt.r2[k] = quantized_r2(r.dist);
        break;
      case DYNBOND_BREAKBOND:
      case DYNBOND_KILLBOND:
        if (!btype_ok(r.type)) return fail(c, DYNBOND_EINVAL, where + "bond type out of range 1..15");
        if (!dist_ok || (r.kind == DYNBOND_BREAKBOND && !prob_ok))
          return fail(c, DYNBOND_EINVAL, where + "bad distance or probability");
        rt.r2[k] = quantized_r2(r.dist);
        break;
      case DYNBOND_CONVERTBOND:
        if (!btype_ok(r.type) || !btype_ok(r.type2) || !prob_ok)
          return fail(c, DYNBOND_EINVAL, where + "bad bond types or probability");
        break;
      case DYNBOND_CREATEANGLE:
        if (!btype_ok(r.type)) return fail(c, DYNBOND_EINVAL, where + "angle type out of range 1..15");
        for (int q = 0; q < 3; ++q)
          if (!mask_ok(r.bead_mask[q])) return fail(c, DYNBOND_EINVAL, where + "bead masks must be nonzero");
        for (int q = 0; q < 2; ++q)
          if (!mask_ok(r.bond_mask[q])) return fail(c, DYNBOND_EINVAL, where + "bond masks must be nonzero");
        rt.angle_idx[rt.n_angle++] = k;
        break;
      case DYNBOND_CREATEDIHEDRAL:
        if (!btype_ok(r.type)) return fail(c, DYNBOND_EINVAL, where + "dihedral type out of range 1..15");
        for (int q = 0; q < 4; ++q)
          if (!mask_ok(r.bead_mask[q])) return fail(c, DYNBOND_EINVAL, where + "bead masks must be nonzero");
        for (int q = 0; q < 3; ++q)
          if (!mask_ok(r.bond_mask[q])) return fail(c, DYNBOND_EINVAL, where + "bond masks must be nonzero");
        rt.dihedral_idx[rt.n_dihedral++] = k;
        break;
      case DYNBOND_MAXBOND:
        if (!mask_ok(r.bond_mask[0]) || !mask_ok(r.bead_mask[0]) || r.maxn < 0)
          return fail(c, DYNBOND_EINVAL, where + "maxbond needs bond and bead masks and maxn >= 0");
        rt.maxbond_idx[rt.n_maxbond++] = k;
        break;
      default:
        return fail(c, DYNBOND_EINVAL, where + "unknown rule kind " + std::to_string(r.kind));
    }
    if (r.kind == DYNBOND_CREATEBOND || r.kind == DYNBOND_CREATEDIRBOND) {
      rt.r2max = std::max(rt.r2max, rt.r2[k]);
      for (int a = 0; a < 16; ++a) {
        if ((r.bead_mask[0] >> a) & 1u || (r.bead_mask[1] >> a) & 1u) rt.role_rules[a] |= 1u << k;
        for (int b = 0; b < 16; ++b)
          if ((((r.bead_mask[0] >> a) & 1u) && ((r.bead_mask[1] >> b) & 1u)) ||
              (((r.bead_mask[0] >> b) & 1u) && ((r.bead_mask[1] >> a) & 1u)))
            rt.pair_rules[a][b] |= 1u << k;
      }
    }
    if (r.kind == DYNBOND_BREAKBOND || r.kind == DYNBOND_CONVERTBOND || r.kind == DYNBOND_KILLBOND)
      rt.breakish |= 1u << r.type;
  }
  // precompiled lookups: stored types per bead type; break/convert/kill
  // rules grouped by bond type (list order kept within a type)
  for (int k = 0; k < n; ++k) {
    const dynbond_rule& r = rules[k];
    if (r.kind != DYNBOND_CREATEBOND && r.kind != DYNBOND_CREATEDIRBOND) continue;
    int t2 = r.kind == DYNBOND_CREATEDIRBOND ? r.type2 : r.type;
    for (int a = 0; a < 16; ++a) {
      if ((r.bead_mask[0] >> a) & 1u) rt.role_store[a] |= 1u << r.type;
      if ((r.bead_mask[1] >> a) & 1u) rt.role_store[a] |= 1u << t2;
    }
  }
  int nbk = 0;
  for (int t = 0; t < 16; ++t) {
    rt.bk_start[t] = nbk;
    for (int k = 0; k < n; ++k) {
      const dynbond_rule& r = rules[k];
      if ((r.kind == DYNBOND_BREAKBOND || r.kind == DYNBOND_CONVERTBOND || r.kind == DYNBOND_KILLBOND) && r.type == t)
        rt.bk_list[nbk++] = k;
    }
  }
  rt.bk_start[16] = nbk;
  const dynbond_params& p = c->prm;
  rt.reactive = p.reactive_mask;
  rt.pc13 = p.paircheck13 != 0;
  rt.pc14 = p.paircheck14 != 0;
  rt.max_rounds = p.max_rounds;
  rt.prob_mode = p.prob_mode;
  rt.key0 = (uint32_t)p.seed;
  rt.key1 = (uint32_t)(p.seed >> 32);
  // one cell-list class per creation-capable type (binned by k_bead)
  rt.n_cls = 0;
  for (int t = 0; t < 16; ++t)
    rt.cls_of[t] = (rt.role_store[t] && ((rt.reactive >> t) & 1u)) ? rt.n_cls++ : -1;
  for (int t = 0; t < 16; ++t) {
    rt.cls_mask[t] = 0;
    for (int u = 0; u < 16; ++u)
      if (rt.pair_rules[t][u] && rt.cls_of[u] >= 0) rt.cls_mask[t] |= 1u << rt.cls_of[u];
  }
  if (rt.n_cls == 0) rt.n_cls = 1;  // nothing is binned; keep the arrays non-empty
  return DYNBOND_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int occupancy_grid(dynbond_ctx* c, const void* fn, int block, int per_sm_cap, size_t smem = 0) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return c->nsm * std::min(nb, per_sm_cap);
}

int bounded_grid(long long work, int block, int cap) {
  long long g = (work + block - 1) / block;
  return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

// ---------------------------------------------------------------------------
// launch sequences
// ---------------------------------------------------------------------------

void mark(dynbond_ctx* c, std::vector<cudaEvent_t>& ev, size_t k) {
  if (c->profile && k < ev.size()) cudaEventRecord(ev[k], c->stream);
}

// Launch on the context's stream, with programmatic stream serialization
// unless the context disables it (every kernel waits for its predecessor with
// griddepcontrol.wait before touching memory) or profiles (events between
// phases would measure the overlap, not the phases).
#define E(x)                              \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

template <typename... KArgs, typename... Args>
cudaError_t launch_smem(dynbond_ctx* c, void (*kern)(KArgs...), int grid, int block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c->pdl && !c->profile ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch(dynbond_ctx* c, void (*kern)(KArgs...), int grid, int block, Args... args) {
  return launch_smem(c, kern, grid, block, 0, args...);
}
// a launch after an event wait (a graph branch or its join): plain stream order
template <typename... KArgs, typename... Args>
cudaError_t launch_plain(cudaStream_t st, void (*kern)(KArgs...), int grid, int block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_match(dynbond_ctx* c) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(c->grid_match);
  cfg.blockDim = dim3(MATCH_THREADS);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_match, c->d, (const RuleTab*)c->d_rt);
}

// the candidate search: staged tiles when the geometry has them, else the
// per-bead search in global memory
cudaError_t launch_candidates(dynbond_ctx* c) {
  if (c->cand_tiles)
    return launch_smem(c, c->octant ? k_candidates_tile_oct : k_candidates_tile, c->grid_ctile, 256,
                       (size_t)CAND_TILE_SMEM, c->d, (const RuleTab*)c->d_rt);
  return launch(c, c->octant ? k_candidates_oct : k_candidates, c->grid_cand, 256, c->d, (const RuleTab*)c->d_rt);
}

// the whole call as one persistent cooperative launch (DYNBOND_FLAG_PERSISTENT)
cudaError_t launch_persistent(dynbond_ctx* c) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(c->grid_persist);
  cfg.blockDim = dim3(256);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, c->octant ? k_step_persistent_oct : k_step_persistent, c->d,
                            (const RuleTab*)c->d_rt);
}

// The step's launch sequence; with bond_branch, the bond forces of the new
// topology run on a branch forked after the edit (they read only the slots
// and the positions, which nothing after the edit writes) beside the purge,
// hole filling and rebuild, joined at the end.
cudaError_t enqueue_step_seq(dynbond_ctx* c, bool bond_branch) {
  const Dev& d = c->d;
  size_t k = 0;
  if (c->persistent) {
    E(launch_persistent(c));
    return cudaGetLastError();
  }
  mark(c, c->ev_step, k++);
  E(launch(c, k_setup, c->nsm * 4, 256, d));
  // the breakage nomination needs only the zeroed per-call state: it runs on
  // a branch beside the binning, cell list and candidate search, joined
  // before the matching
  E(cudaEventRecord(c->ev_fork, c->stream));
  E(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  k_breakage<<<c->nsm * 4, 256, 0, c->side>>>(d, c->d_rt);
  E(cudaEventRecord(c->ev_join, c->side));
  mark(c, c->ev_step, k++);
  E(launch(c, k_bead, c->grid_bead, 256, d, c->d_rt));
  mark(c, c->ev_step, k++);
  E(launch(c, k_scan_cells, c->grid_scan, 256, d));
  E(launch(c, k_scatter, c->grid_bead, 256, d));
  mark(c, c->ev_step, k++);
  E(launch_candidates(c));
  E(launch(c, k_cand_overflow, c->nsm, 128, d, c->d_rt));
  mark(c, c->ev_step, k++);
  E(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  E(launch_match(c));
  mark(c, c->ev_step, k++);
  E(launch(c, k_edit, c->grid_edit, 256, d, c->d_rt));
  if (bond_branch) {
    E(cudaEventRecord(c->ev_fork2, c->stream));
    E(cudaStreamWaitEvent(c->side, c->ev_fork2, 0));
    E(launch_plain(c->side, k_bond_forces, c->grid_bf, BF_THREADS, (size_t)BF_SMEM_BYTES, d, c->ff));
    E(cudaEventRecord(c->ev_join2, c->side));
  }
  mark(c, c->ev_step, k++);
  E(launch(c, k_purge, c->grid_purge, PURGE_TILE / PURGE_PER_THREAD, d));
  E(launch(c, k_fill, c->nsm * 4, FILL_TILE, d));
  mark(c, c->ev_step, k++);
  E(launch(c, k_rebuild, c->grid_seg, 256, d, c->d_rt, 0));
  mark(c, c->ev_step, k++);
  if (bond_branch) E(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
  return cudaGetLastError();
}
cudaError_t enqueue_step(dynbond_ctx* c) { return enqueue_step_seq(c, false); }

// The angle / dihedral forces (after the bonds') and the energy / virial output.
cudaError_t enqueue_ad_forces(dynbond_ctx* c, bool after_join) {
  const Dev& d = c->d;
  if (after_join)
    E(launch_plain(c->stream, k_angle_dihedral_forces, c->grid_adf, AD_THREADS, (size_t)AD_SMEM_BYTES, d, c->ff));
  else
    E(launch_smem(c, k_angle_dihedral_forces, c->grid_adf, AD_THREADS, (size_t)AD_SMEM_BYTES, d, c->ff));
  return cudaSuccess;
}

// dynbond_step_forces: the step with the bond forces on a branch, then the
// angle / dihedral forces and the energy / virial output
cudaError_t enqueue_both(dynbond_ctx* c) {
  E(enqueue_step_seq(c, true));
  E(enqueue_ad_forces(c, true));
  E(launch(c, k_ev_out, bounded_grid(7ll * c->R, 256, c->nsm), 256, c->d));
  return cudaGetLastError();
}

cudaError_t enqueue_forces(dynbond_ctx* c) {
  const Dev& d = c->d;
  size_t k = 0;
  mark(c, c->ev_forces, k++);
  E(launch_smem(c, k_bond_forces, c->grid_bf, BF_THREADS, (size_t)BF_SMEM_BYTES, d, c->ff));
  mark(c, c->ev_forces, k++);
  E(launch_smem(c, k_angle_dihedral_forces, c->grid_adf, AD_THREADS, (size_t)AD_SMEM_BYTES, d, c->ff));
  mark(c, c->ev_forces, k++);
  E(launch(c, k_ev_out, bounded_grid(7ll * c->R, 256, c->nsm), 256, d));
  return cudaGetLastError();
}

cudaError_t capture(dynbond_ctx* c, cudaError_t (*enqueue)(dynbond_ctx*), cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = enqueue(c);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e1 != cudaSuccess ? e1 : e2;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
  }
  return e;
}

dynbond_status device_status(dynbond_ctx* c) {
  unsigned err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, c->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->sticky = DYNBOND_ECUDA;
    return fail(c, DYNBOND_ECUDA, std::string("device execution: ") + cudaGetErrorString(e));
  }
  if (!err) return DYNBOND_OK;
  dynbond_status s;
  std::string msg;
  if (err & ERR_POS) {
    s = DYNBOND_EINVAL;
    msg = "a position lies outside [0, box_q) of its replica";
  } else if (err & ERR_TIMEOUT) {
    s = DYNBOND_ETIMEOUT;
    msg = "a bounded device-side wait gave up (grid barrier or look-back)";
  } else if (err & ERR_ROUNDS) {
    s = DYNBOND_ENOTCONVERGED;
    msg = "matching did not reach a fixpoint within DYNBOND_MAX_ROUNDS rounds";
  } else if (err & ERR_CAND_CAP) {
    s = DYNBOND_ECAPACITY;
    msg = "candidate buffer exhausted";
  } else if (err & ERR_INTERNAL) {
    s = DYNBOND_ECAPACITY;
    msg = "internal consistency check failed (interaction record out of range)";
  } else {
    s = DYNBOND_ECAPACITY;
    msg = "bond slot capacity exceeded";
  }
  c->sticky = s;
  return fail(c, s, msg);
}

void collect_profile(dynbond_ctx* c, int which) {
  std::vector<cudaEvent_t>& ev = which == 1 ? c->ev_step : c->ev_forces;
  std::vector<float>& out = which == 1 ? c->last_step_ms : c->last_forces_ms;
  out.assign(ev.size() - 1, 0.f);
  for (size_t k = 0; k + 1 < ev.size(); ++k) cudaEventElapsedTime(&out[k], ev[k], ev[k + 1]);
}

// Cell grid of every replica for a cell edge of `scale` x the reach (at least
// the reach, at most 1024 cells per axis); uploads it and sizes the scan.
dynbond_status set_geometry(dynbond_ctx* c, double scale, int zdiv) {
  const int R = c->R;
  std::vector<int> nc(R), nz(R);
  std::vector<long long> cb(R + 1, 0);
  bool octant = true;
  for (int r = 0; r < R; ++r) {
    long long L = c->h_box[r];
    long long ncap = c->reach > 0 ? L / c->reach : 1;
    long long n = c->reach > 0 ? (long long)((double)L / (scale * (double)c->reach)) : 1;
    n = std::max<long long>(1, std::min<long long>({n, ncap, 1024}));
    // z: zdiv cells per x / y edge (any count works: the search takes the
    // z cells overlapping the reach interval)
    long long m = c->reach > 0 ? (long long)((double)L * zdiv / (scale * (double)c->reach)) : 1;
    m = std::max<long long>(1, std::min<long long>(m, 4096));
    nc[r] = (int)n;
    nz[r] = (int)m;
    cb[r + 1] = cb[r] + n * n * m;
    // cells at least twice the reach on every axis: the octant search suffices
    octant = octant && n >= 3 && 2 * c->reach * n <= L;
  }
  if (c->max_cells && cb[R] > c->max_cells) return fail(c, DYNBOND_ECAPACITY, "cell geometry larger than allocated");
  if (cb[R] * c->rt.n_cls >= 0x7FFFFFFFll)
    return fail(c, DYNBOND_EINVAL, "cell grid too large: boxes over 2^31 cell keys (cell classes x cells)");
  // work items of the staged search: per replica and class with partner
  // classes, tiles of CT x CT columns and Z z cells; along z the stage adds hz
  // cells on each side, hz = floor(reach nz / L) + 1 >= the cells a reach
  // interval extends beyond its bead's cell
  std::vector<int4> tiles;
  bool tiles_ok = !c->global_search && c->reach > 0;
  for (int r = 0; r < R && tiles_ok; ++r) {
    const long long L = c->h_box[r];
    const long long hz = c->reach * nz[r] / L + 1;
    if (2 * hz >= CZS_MAX) {
      tiles_ok = false;
      break;
    }
    const int Z = nz[r] <= CZS_MAX ? nz[r] : (int)std::min<long long>(16, CZS_MAX - 2 * hz);
    const int ntx = (nc[r] + CT - 1) / CT, ntz = (nz[r] + Z - 1) / Z;
    for (int t = 0; t < 16; ++t) {
      const int cls = c->rt.cls_of[t];
      const unsigned pm = c->rt.cls_mask[t];
      if (cls < 0 || !pm) continue;
      for (int tx = 0; tx < ntx; ++tx)
        for (int ty = 0; ty < ntx; ++ty)
          for (int tz = 0; tz < ntz; ++tz)
            tiles.push_back(make_int4(r, cls | (int)(hz << 8) | (int)(pm << 16), tx | ty << 16, tz | Z << 16));
    }
  }
  c->n_cells = cb[R];
  c->octant = octant;
  c->d.n_cells = c->n_cells;
  c->d.n_keys = c->n_cells * c->rt.n_cls;
  c->grid_scan = bounded_grid(c->d.n_keys, 256 * SCAN_PER_THREAD, c->nsm * 4);
  std::vector<int4> geo(2 * R);
  for (int r = 0; r < R; ++r) {
    const long long L = c->h_box[r];
    const float fxy = (float)nc[r] / (float)L, fz = (float)nz[r] / (float)L;
    int bxy, bz;
    std::memcpy(&bxy, &fxy, 4);
    std::memcpy(&bz, &fz, 4);
    const long long hz = (c->reach * nz[r] + L - 1) / L;
    geo[2 * r] = make_int4((int)L, nc[r], nz[r], (int)hz);
    geo[2 * r + 1] = make_int4(bxy, bz, (int)cb[r], 0);
  }
  if (c->d_nc) {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_geo, geo.data(), sizeof(int4) * 2 * R, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_nc, nc.data(), 4 * R, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ncz, nz.data(), 4 * R, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_cb, cb.data(), 8 * (R + 1), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->tiles_avail = tiles_ok && !tiles.empty();
  c->cand_tiles = c->tiles_avail && c->tiles_on;
  c->d.n_ctile = c->tiles_avail ? (int)tiles.size() : 0;
  if (c->tiles_avail && c->d_nc) {
    if ((long long)tiles.size() > c->ctile_cap) {  // outside any captured work: the graphs are recaptured after
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      if (c->d_ctile) cudaFree(c->d_ctile);
      c->d_ctile = nullptr;
      c->ctile_cap = 0;
      CUDA_TRY(c, cudaMalloc(&c->d_ctile, sizeof(int4) * tiles.size()));
      c->ctile_cap = (long long)tiles.size();
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ctile, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->d.ctile = c->d_ctile;
  c->tuning.cell_scale = scale;
  c->tuning.cell_zdiv = zdiv;
  c->tuning.octant = octant ? 1 : 0;
  c->tuning.tiles = c->cand_tiles ? 1 : 0;
  return DYNBOND_OK;
}

// The combined call runs its own graph unless the context profiles phases or
// runs each step as one persistent launch (then it is the two calls in turn).
bool combined_graph(const dynbond_ctx* c) { return !c->profile && !c->persistent; }

dynbond_status capture_graphs(dynbond_ctx* c) {
  if (c->g_step) cudaGraphExecDestroy(c->g_step);
  if (c->g_forces) cudaGraphExecDestroy(c->g_forces);
  if (c->g_both) cudaGraphExecDestroy(c->g_both);
  c->g_step = c->g_forces = c->g_both = nullptr;
  if (!c->use_graph) return DYNBOND_OK;
  if (capture(c, enqueue_step, &c->g_step) != cudaSuccess || capture(c, enqueue_forces, &c->g_forces) != cudaSuccess) {
    if (c->g_step) cudaGraphExecDestroy(c->g_step);
    if (c->g_forces) cudaGraphExecDestroy(c->g_forces);
    c->g_step = c->g_forces = nullptr;
    c->use_graph = false;
    cudaGetLastError();
    c->last_error = "CUDA graph capture unavailable; launching kernels directly";
    return DYNBOND_OK;
  }
  if (combined_graph(c) && capture(c, enqueue_both, &c->g_both) != cudaSuccess) {
    c->g_both = nullptr;  // the combined call falls back to the two graphs
    cudaGetLastError();
  }
  return DYNBOND_OK;
}

// The front of a call up to the candidate lists; it writes per-call scratch
// only, so it can be timed repeatedly without changing the topology.
cudaError_t enqueue_front(dynbond_ctx* c) {
  const Dev& d = c->d;
  E(launch(c, k_setup, c->nsm * 2, 1024, d));
  E(launch(c, k_bead, c->grid_bead, 256, d, c->d_rt));
  E(launch(c, k_scan_cells, c->grid_scan, 256, d));
  E(launch(c, k_scatter, c->grid_bead, 256, d));
  E(launch_candidates(c));
  E(launch(c, k_cand_overflow, c->nsm, 128, d, c->d_rt));
  return cudaGetLastError();
}

}  // namespace

const uint4* dynbond::internal_slots(const dynbond_ctx* c, long long* n_beads, long long* box_q, int* n_replicas,
                                     cudaStream_t* stream) {
  *n_beads = c->N;
  *box_q = c->h_box.empty() ? 0 : c->h_box[0];
  *n_replicas = c->R;
  *stream = c->stream;
  return c->d.slots;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* dynbond_status_string(dynbond_status s) {
  switch (s) {
    case DYNBOND_OK: return "ok";
    case DYNBOND_EINVAL: return "invalid argument";
    case DYNBOND_ENOMEM: return "out of memory";
    case DYNBOND_ECAPACITY: return "capacity exceeded";
    case DYNBOND_ECUDA: return "CUDA error";
    case DYNBOND_ETIMEOUT: return "device wait timed out";
    case DYNBOND_ENOTCONVERGED: return "matching did not converge";
  }
  return "unknown status";
}

const char* dynbond_last_error(const dynbond_ctx* c) { return c ? c->last_error.c_str() : g_create_error.c_str(); }

void dynbond_destroy(dynbond_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->g_step) cudaGraphExecDestroy(c->g_step);
  if (c->g_forces) cudaGraphExecDestroy(c->g_forces);
  if (c->g_both) cudaGraphExecDestroy(c->g_both);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_fork2) cudaEventDestroy(c->ev_fork2);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  for (cudaEvent_t e : c->ev_step) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_forces) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->d_ctile) cudaFree(c->d_ctile);
  delete c;
}

}  // extern "C"

namespace {


dynbond_status create_impl(dynbond_ctx* c, const dynbond_params* params, const dynbond_rule* rules, int32_t n_rules,
                           const dynbond_system* sys, const dynbond_forcefield* ff, dynbond_stream stream) {
  if (!params || !sys || !ff) return (fail(c, DYNBOND_EINVAL, "params, system and forcefield are required"));
  c->prm = *params;
  c->stream = (cudaStream_t)stream;
  c->profile = (params->flags & DYNBOND_FLAG_PROFILE) != 0;
  c->use_graph = (params->flags & DYNBOND_FLAG_NO_GRAPH) == 0;
  c->pdl = (params->flags & DYNBOND_FLAG_NO_PDL) == 0;
  c->global_search = (params->flags & DYNBOND_FLAG_GLOBAL_SEARCH) != 0;
  c->persistent = (params->flags & DYNBOND_FLAG_PERSISTENT) != 0 && !c->profile;
  c->staged_search = !c->global_search && (params->flags & DYNBOND_FLAG_STAGED_SEARCH) != 0;
  c->tiles_on = c->staged_search;
  if (params->max_rounds < 0 || params->prob_mode < 0 || params->prob_mode > 1 || params->cell_scale < 0)
    return (fail(c, DYNBOND_EINVAL, "bad max_rounds, prob_mode or cell_scale"));
  dynbond_status st = build_rules(c, rules, n_rules);
  if (st) return (st);

  // ---- system validation (host)
  const int R = sys->n_replicas;
  if (R < 1 || !sys->bead_offset || !sys->box_q || !sys->bead_type)
    return (fail(c, DYNBOND_EINVAL, "n_replicas >= 1 with bead_offset, box_q and bead_type required"));
  if (sys->bead_offset[0] != 0) return (fail(c, DYNBOND_EINVAL, "bead_offset[0] must be 0"));
  for (int r = 0; r < R; ++r) {
    if (sys->bead_offset[r + 1] <= sys->bead_offset[r])
      return (fail(c, DYNBOND_EINVAL, "every replica needs at least one bead (offsets increasing)"));
    if (sys->box_q[r] < 2 || sys->box_q[r] >= (1ll << 31))
      return (fail(c, DYNBOND_EINVAL, "box_q must lie in [2, 2^31)"));
  }
  const long long N = sys->bead_offset[R];
  if (N >= (1ll << 28)) return (fail(c, DYNBOND_EINVAL, "at most 2^28 - 1 beads"));
  c->N = N;
  c->R = R;
  std::vector<int> rep(N);
  for (int r = 0; r < R; ++r)
    for (long long i = sys->bead_offset[r]; i < sys->bead_offset[r + 1]; ++i) rep[i] = r;
  std::vector<unsigned char> type(N);
  for (long long i = 0; i < N; ++i) {
    if (sys->bead_type[i] < 0 || sys->bead_type[i] >= DYNBOND_MAX_TYPES)
      return (fail(c, DYNBOND_EINVAL, "bead types must lie in 0..15"));
    type[i] = (unsigned char)sys->bead_type[i];
  }
  std::vector<uint4> slots(N, make_uint4(0, 0, 0, 0));
  std::vector<int> deg(N, 0);
  std::vector<long long> nb_rep(R, 0);
  if (sys->n_bonds < 0 || (sys->n_bonds > 0 && !sys->bonds)) return (fail(c, DYNBOND_EINVAL, "bad bond list"));
  for (long long k = 0; k < sys->n_bonds; ++k) {
    long long i = sys->bonds[4 * k], j = sys->bonds[4 * k + 1];
    int ti = sys->bonds[4 * k + 2], tj = sys->bonds[4 * k + 3];
    if (i < 0 || j < 0 || i >= N || j >= N || i == j || rep[i] != rep[j] || !btype_ok(ti) || !btype_ok(tj))
      return (fail(c, DYNBOND_EINVAL, "bond " + std::to_string(k) + " is malformed"));
    for (int q = 0; q < deg[i]; ++q)
      if ((int)(((unsigned*)&slots[i])[q] >> 4) == j)
        return (fail(c, DYNBOND_EINVAL, "bond " + std::to_string(k) + " is listed twice"));
    if (deg[i] >= SLOTS || deg[j] >= SLOTS)
      return (fail(c, DYNBOND_EINVAL, "more than 4 bonds on one bead"));
    ((unsigned*)&slots[i])[deg[i]++] = ((unsigned)j << 4) | (unsigned)ti;
    ((unsigned*)&slots[j])[deg[j]++] = ((unsigned)i << 4) | (unsigned)tj;
    nb_rep[rep[i]] += 1;
  }
  if (!make_ff(*ff, c->ff)) return fail(c, DYNBOND_EINVAL, "angle_style must be 0 (cosine) or 1 (harmonic)");

  // ---- device
  CUDA_TRY(c, cudaGetDevice(&c->device));
  CUDA_TRY(c, cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));

  // cells: edge >= the largest creation distance; the default (and the
  // autotuner's largest grid) is cells exactly as wide as that reach
  c->h_box.assign(sys->box_q, sys->box_q + R);
  c->reach = 0;
  while (c->reach * c->reach < c->rt.r2max) ++c->reach;
  st = set_geometry(c, params->cell_scale > 0 ? (double)params->cell_scale : 1.0,
                    params->cell_scale > 0 && params->cell_zdiv > 0 ? params->cell_zdiv : 1);
  if (st) return st;
  c->max_cells = c->n_cells;
  c->W = N / 32 + 1;
  c->d.W = c->W;

  Dev& d = c->d;
  d.N = N;
  d.R = R;
  d.n_cells = c->n_cells;
  d.spin_limit = params->spin_limit > 0 ? params->spin_limit : (1 << 24);
  long long* p_off;
  long long* p_box;
  long long* p_cb;
  int* p_nc;
  int* p_ncz;
  int* p_rep;
  unsigned char* p_type;
  unsigned* p_stream;
  unsigned long long *p_tf, *p_tb;
#define ALLOC(ptr, n)                         \
  do {                                        \
    dynbond_status s_ = dalloc(c, &(ptr), (size_t)(n)); \
    if (s_) return (s_);                  \
  } while (0)
  ALLOC(p_off, R + 1);
  ALLOC(p_box, R);
  ALLOC(p_cb, R + 1);
  ALLOC(p_nc, R);
  ALLOC(p_ncz, R);
  ALLOC(c->d_geo, 2 * R);
  c->d_nc = p_nc;
  c->d_ncz = p_ncz;
  c->d_cb = p_cb;
  ALLOC(p_rep, N);
  ALLOC(p_type, N);
  ALLOC(p_stream, R);
  ALLOC(p_tf, (size_t)R * MAXR);
  ALLOC(p_tb, (size_t)R * MAXR);
  ALLOC(d.args, 1);
  ALLOC(c->d_rt, 1);
  ALLOC(d.slots, N);
  ALLOC(d.ang, 6 * N);
  ALLOC(d.dih, 18 * N);
  ALLOC(d.n_ang, R);
  ALLOC(d.n_dih, R);
  ALLOC(d.n_bonds, R);
  ALLOC(d.cnt, 1);
  ALLOC(d.err, 1);
  // 4 leading ints (16 B, keeping the scan's vector loads aligned): element -1
  // stays 0, so cell k's range after the scatter is [cell_start[k-1], cell_start[k])
  ALLOC(d.cell_start, c->n_cells * c->rt.n_cls + 5);
  CUDA_TRY(c, cudaMemsetAsync(d.cell_start, 0, 4 * (size_t)(c->n_cells * c->rt.n_cls + 5), c->stream));
  d.cell_start += 4;
  ALLOC(d.binned, N);
  ALLOC(d.binned_n, (N + BIN_SEG - 1) / BIN_SEG);
  ALLOC(d.sorted, N);
  d.cand_fixed = N * CAND_FAST;
  d.cand_pool = 2 * N + 65536;
  if (d.cand_fixed + d.cand_pool >= 0x7FFFFFFFll) return fail(c, DYNBOND_EINVAL, "too many beads for one context");
  ALLOC(d.cand, d.cand_fixed + d.cand_pool);
  ALLOC(d.cand_start, N);
  ALLOC(d.cand_len, N);
  ALLOC(d.ovf, N);
  ALLOC(d.brk, 4 * N);
  ALLOC(d.brk_len, N);
  ALLOC(d.killmask, N);
  ALLOC(d.bm_ca, c->W);
  ALLOC(d.bm_ba, c->W);
  ALLOC(d.bm_bn, c->W);
  ALLOC(d.bm_bk, c->W);
  ALLOC(d.bm_elig, c->W);
  ALLOC(d.bm_dirty, c->W);
  // coarse dirty bitmap: one bit per 2^dc_shift words, at most PURGE_COARSE_WORDS words
  d.dc_shift = 0;
  while (((c->W >> d.dc_shift) + 31) / 32 > PURGE_COARSE_WORDS) ++d.dc_shift;
  d.Wc = ((c->W >> d.dc_shift) + 1 + 31) / 32;
  ALLOC(d.bm_dirtyc, d.Wc);
  ALLOC(d.bm_new, c->W);
  ALLOC(d.live[0], 2 * N);
  ALLOC(d.live[1], 2 * N);
  ALLOC(d.mate, 2 * N);
  ALLOC(d.nom, 2 * N);
  ALLOC(d.ptr, 2 * N);
  ALLOC(d.rem, N);
  ALLOC(d.newp, N);
  ALLOC(d.nbl, 2 * N + 1);
  ALLOC(d.rm_ang, 6 * N);
  ALLOC(d.rm_dih, 18 * N);
  ALLOC(d.pr_ang, 6 * N);
  ALLOC(d.pr_dih, 18 * N);
  ALLOC(d.tb_ang, R + 1);
  ALLOC(d.tb_dih, R + 1);
  ALLOC(d.tb_fill, R + 1);
  ALLOC(d.tb_beads, R + 1);
  ALLOC(d.tb_fang, R + 1);
  ALLOC(d.tb_fdih, R + 1);
  ALLOC(d.ev_acc, 7 * (size_t)R * EV_COPIES);
  // per-call counters zeroed together: removed / added counts, k_fill
  // counters and items, round flags, statistics
  {
    size_t ints = 13 * (size_t)R;
    size_t bytes = ((ints * sizeof(int) + 15) / 16) * 16 + (size_t)R * NSTAT * sizeof(long long);
    char* base;
    ALLOC(base, bytes);
    c->small = base;
    c->small_bytes = bytes;
    d.small = (int*)base;
    d.small_words = (long long)(bytes / sizeof(int));
    int* ip = (int*)base;
    d.m_ang = ip;
    d.m_dih = ip + R;
    d.added_ang = ip + 2 * R;
    d.added_dih = ip + 3 * R;
    d.fill_items = ip + 4 * R;
    d.fillc = ip + 5 * R;      // 4R
    d.round_hit = ip + 9 * R;  // 4R: two buffers of (creation, breakage) x R
    d.stats = (long long*)(base + ((ints * sizeof(int) + 15) / 16) * 16);
  }
  {
    c->st_scan_n = c->n_cells * c->rt.n_cls / (256 * SCAN_PER_THREAD) + 2;  // tiles of the cell scan
    long long tot = c->st_scan_n;
    unsigned long long* base;
    ALLOC(base, tot);
    c->status_all = base;
    c->status_bytes = (size_t)tot * 8;
    d.status_all = base;
    d.status_words = tot;
    d.st_scan = base;
  }
  ALLOC(c->h2d_pos, N);
  ALLOC(c->d2h_force, N);
  ALLOC(c->d2h_ev, 7 * R);
  ALLOC(c->d_hash, R);
#undef ALLOC
  d.off = p_off;
  d.box = p_box;
  d.cell_base = p_cb;
  d.nc = p_nc;
  d.ncz = p_ncz;
  d.geo = c->d_geo;
  d.reach = c->reach;
  d.rep = p_rep;
  d.type = p_type;
  d.stream = p_stream;
  d.T_form = p_tf;
  d.T_break = p_tb;

  // ---- upload
  std::vector<unsigned long long> tf((size_t)R * MAXR, 0), tb((size_t)R * MAXR, 0);
  std::vector<unsigned> strm(R);
  std::vector<int> tbeads(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    double fs = sys->form_scale ? sys->form_scale[r] : 1.0, bs = sys->break_scale ? sys->break_scale[r] : 1.0;
    if (!std::isfinite(fs) || !std::isfinite(bs) || fs < 0 || bs < 0)
      return (fail(c, DYNBOND_EINVAL, "probability scales must be finite and >= 0"));
    for (int k = 0; k < n_rules; ++k) {
      tf[(size_t)r * MAXR + k] = prob_threshold(std::min(1.0, rules[k].prob * fs));
      tb[(size_t)r * MAXR + k] = prob_threshold(std::min(1.0, rules[k].prob * bs));
    }
    strm[r] = sys->rng_stream ? sys->rng_stream[r] : (unsigned)r;
    long long n = sys->bead_offset[r + 1] - sys->bead_offset[r];
    tbeads[r + 1] = tbeads[r] + (int)((n + BEAD_TILE - 1) / BEAD_TILE);
  }
  std::vector<long long> boxv(sys->box_q, sys->box_q + R), offv(sys->bead_offset, sys->bead_offset + R + 1);
  std::vector<int> zeros(R, 0);
  cudaStream_t s = c->stream;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_rt, &c->rt, sizeof(RuleTab), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_off, offv.data(), 8 * (R + 1), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_box, boxv.data(), 8 * R, cudaMemcpyHostToDevice, s));
  st = set_geometry(c, c->tuning.cell_scale, c->tuning.cell_zdiv);
  if (st) return st;
  CUDA_TRY(c, cudaMemcpyAsync(p_rep, rep.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_type, type.data(), N, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_stream, strm.data(), 4 * R, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_tf, tf.data(), 8 * tf.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(p_tb, tb.data(), 8 * tb.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(d.slots, slots.data(), 16 * N, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(d.n_bonds, nb_rep.data(), 8 * R, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(d.tb_beads, tbeads.data(), 4 * (R + 1), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemsetAsync(d.err, 0, sizeof(unsigned), s));
  for (unsigned* bm : {d.bm_ca, d.bm_ba, d.bm_bn, d.bm_bk, d.bm_elig, d.bm_dirty, d.bm_new})
    CUDA_TRY(c, cudaMemsetAsync(bm, 0, sizeof(unsigned) * (size_t)c->W, s));
  CUDA_TRY(c, cudaMemsetAsync(d.bm_dirtyc, 0, sizeof(unsigned) * (size_t)d.Wc, s));
  CUDA_TRY(c, cudaMemsetAsync(d.n_ang, 0, 4 * R, s));
  CUDA_TRY(c, cudaMemsetAsync(d.n_dih, 0, 4 * R, s));
  CUDA_TRY(c, cudaMemsetAsync(d.args, 0, sizeof(CallArgs), s));

  // ---- launch geometry
  c->grid_bead = bounded_grid(N, 256, c->nsm * 8);
  // angle / dihedral forces: one persistent wave (the blocks pipeline their tiles)
  CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_angle_dihedral_forces,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, AD_SMEM_BYTES));
  c->grid_adf = occupancy_grid(c, (const void*)k_angle_dihedral_forces, AD_THREADS, 8, AD_SMEM_BYTES);
  CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_bond_forces, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   BF_SMEM_BYTES));
  c->grid_bf = occupancy_grid(c, (const void*)k_bond_forces, BF_THREADS, 8, BF_SMEM_BYTES);
  c->grid_edit = bounded_grid((c->W + 7) / 8, 8, c->nsm * 8);  // a warp per 8 bitmap words
  c->tuning.bead_blocks_per_sm = 8;
  c->tuning.candidate_blocks_per_sm = 8;
  c->grid_cand = bounded_grid(N, 256, c->nsm * 8);
  for (auto fn : {(const void*)k_candidates_tile, (const void*)k_candidates_tile_oct})
    CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, CAND_TILE_SMEM));
  c->grid_ctile = occupancy_grid(c, (const void*)k_candidates_tile, 256, 8, CAND_TILE_SMEM);
  // persistent call: every block resident (cooperative launch), at most two per SM
  c->grid_persist = std::min(occupancy_grid(c, (const void*)k_step_persistent, 256, 2),
                             occupancy_grid(c, (const void*)k_step_persistent_oct, 256, 2));
  c->grid_seg = c->nsm * 4;
  // purge: every block resident, so every tile's records are in flight in one wave
  c->grid_purge = occupancy_grid(c, (const void*)k_purge, PURGE_TILE / PURGE_PER_THREAD, 8);
  // matching: co-resident blocks (cooperative launch), at most two per SM so
  // the grid barriers between rounds stay short; round 0 gives each lane one
  // 32-bead bitmap word
  c->grid_match = std::max(1, std::min(occupancy_grid(c, (const void*)k_match, MATCH_THREADS, 2),
                                       bounded_grid((N + 31) / 32, MATCH_THREADS, c->nsm * 2)));

  // ---- initial interactions: the typed set of every path of the initial graph
  CUDA_TRY(c, cudaMemsetAsync(d.cnt, 0, sizeof(Counters), s));
  CUDA_TRY(c, cudaMemsetAsync(c->small, 0, c->small_bytes, s));
  CUDA_TRY(c, cudaMemsetAsync(c->status_all, 0, c->status_bytes, s));
  k_bead_flags<<<c->grid_bead, 256, 0, s>>>(d, c->d_rt);
  k_allbonds<<<c->grid_bead, 256, 0, s>>>(d);
  k_rebuild<<<c->grid_seg, 256, 0, s>>>(d, c->d_rt, 1);
  CUDA_TRY(c, cudaMemsetAsync(d.ev_acc, 0, sizeof(double) * 7 * (size_t)R * EV_COPIES, s));
  CUDA_TRY(c, cudaGetLastError());
  st = device_status(c);
  if (st) return (st);

  // ---- the side branch of a call, profiling events and graphs
  CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming));
  CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming));
  if (c->profile) {
    c->names_step = {"setup", "bead", "cells", "candidates", "match", "edit", "purge", "rebuild"};
    c->names_forces = {"bond_forces", "angle_dihedral_forces"};
    c->ev_step.resize(c->names_step.size() + 1);
    c->ev_forces.resize(c->names_forces.size() + 1);
    for (auto& e : c->ev_step) CUDA_TRY(c, cudaEventCreate(&e));
    for (auto& e : c->ev_forces) CUDA_TRY(c, cudaEventCreate(&e));
  }
  c->tuned = params->cell_scale > 0 || (params->flags & DYNBOND_FLAG_NO_AUTOTUNE);
  return capture_graphs(c);
}

}  // namespace

extern "C" {

dynbond_status dynbond_create(const dynbond_params* params, const dynbond_rule* rules, int32_t n_rules,
                              const dynbond_system* sys, const dynbond_forcefield* ff, dynbond_stream stream,
                              dynbond_ctx** out) {
  if (!out) return DYNBOND_EINVAL;
  *out = nullptr;
  dynbond_ctx* c = new dynbond_ctx();
  dynbond_status st = create_impl(c, params, rules, n_rules, sys, ff, stream);
  if (st != DYNBOND_OK) {
    g_create_error = c->last_error;
    dynbond_destroy(c);
    return st;
  }
  *out = c;
  return DYNBOND_OK;
}

dynbond_status dynbond_step(dynbond_ctx* c, const int32_t* d_pos, uint64_t step, dynbond_stats* h_stats) {
  if (!c || !d_pos) return DYNBOND_EINVAL;
  if (!aligned16(d_pos)) return fail(c, DYNBOND_EINVAL, "d_pos must be 16-byte aligned (int4 per bead)");
  if (c->sticky) return c->sticky;
  if (!c->tuned) {
    dynbond_status st = dynbond_autotune(c, d_pos, nullptr);
    if (st) return st;
  }
  k_set_args<<<1, 1, 0, c->stream>>>(c->d.args, (const int4*)d_pos, nullptr, nullptr, step, 1, 0,
                                     c->persistent ? &c->d.cnt->bar[1] : nullptr);
  cudaError_t e = c->use_graph ? cudaGraphLaunch(c->g_step, c->stream) : enqueue_step(c);
  if (e != cudaSuccess) {
    c->sticky = DYNBOND_ECUDA;
    return fail(c, DYNBOND_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  if (c->profile) c->last_profiled |= 1;
  if (h_stats) {
    dynbond_status st = device_status(c);
    if (st) return st;
    static_assert(sizeof(dynbond_stats) == NSTAT * sizeof(long long), "stats layout");
    CUDA_TRY(c, cudaMemcpy(h_stats, c->d.stats, sizeof(dynbond_stats) * c->R, cudaMemcpyDeviceToHost));
  }
  return DYNBOND_OK;
}

dynbond_status dynbond_forces(dynbond_ctx* c, const int32_t* d_pos, float* d_force, double* d_ev) {
  if (!c || !d_pos || !d_force || !d_ev) return DYNBOND_EINVAL;
  if (!aligned16(d_pos) || !aligned16(d_force))
    return fail(c, DYNBOND_EINVAL, "d_pos and d_force must be 16-byte aligned (4-vectors per bead)");
  if (c->sticky) return c->sticky;
  k_set_args<<<1, 1, 0, c->stream>>>(c->d.args, (const int4*)d_pos, (float4*)d_force, d_ev, 0, 0, 1, nullptr);
  cudaError_t e = c->use_graph ? cudaGraphLaunch(c->g_forces, c->stream) : enqueue_forces(c);
  if (e != cudaSuccess) {
    c->sticky = DYNBOND_ECUDA;
    return fail(c, DYNBOND_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  if (c->profile) c->last_profiled |= 2;
  return DYNBOND_OK;
}

dynbond_status dynbond_step_forces(dynbond_ctx* c, const int32_t* d_pos, uint64_t step, float* d_force,
                                   double* d_ev, dynbond_stats* h_stats) {
  if (!c || !d_pos || !d_force || !d_ev) return DYNBOND_EINVAL;
  if (!aligned16(d_pos) || !aligned16(d_force))
    return fail(c, DYNBOND_EINVAL, "d_pos and d_force must be 16-byte aligned (4-vectors per bead)");
  if (c->sticky) return c->sticky;
  if (!c->tuned) {
    dynbond_status st = dynbond_autotune(c, d_pos, nullptr);
    if (st) return st;
  }
  if (!combined_graph(c) || (c->use_graph && !c->g_both)) {
    dynbond_status st = dynbond_step(c, d_pos, step, nullptr);
    if (!st) st = dynbond_forces(c, d_pos, d_force, d_ev);
    if (st) return st;
  } else {
    k_set_args<<<1, 1, 0, c->stream>>>(c->d.args, (const int4*)d_pos, (float4*)d_force, d_ev, step, 1, 1, nullptr);
    cudaError_t e = c->use_graph ? cudaGraphLaunch(c->g_both, c->stream) : enqueue_both(c);
    if (e != cudaSuccess) {
      c->sticky = DYNBOND_ECUDA;
      return fail(c, DYNBOND_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
  }
  if (h_stats) {
    dynbond_status st = device_status(c);
    if (st) return st;
    CUDA_TRY(c, cudaMemcpy(h_stats, c->d.stats, sizeof(dynbond_stats) * c->R, cudaMemcpyDeviceToHost));
  }
  return DYNBOND_OK;
}

dynbond_status dynbond_run_host(dynbond_ctx* c, const int32_t* h_pos, uint64_t step, float* h_force, double* h_ev,
                                dynbond_stats* h_stats) {
  if (!c || !h_pos || !h_force || !h_ev) return DYNBOND_EINVAL;
  if (c->sticky) return c->sticky;
  CUDA_TRY(c, cudaMemcpyAsync(c->h2d_pos, h_pos, 16 * c->N, cudaMemcpyHostToDevice, c->stream));
  dynbond_status st =
      dynbond_step_forces(c, (const int32_t*)c->h2d_pos, step, (float*)c->d2h_force, c->d2h_ev, nullptr);
  if (st) return st;
  CUDA_TRY(c, cudaMemcpyAsync(h_force, c->d2h_force, 16 * c->N, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h_ev, c->d2h_ev, 8 * 7 * c->R, cudaMemcpyDeviceToHost, c->stream));
  st = device_status(c);
  if (st) return st;
  if (h_stats) CUDA_TRY(c, cudaMemcpy(h_stats, c->d.stats, sizeof(dynbond_stats) * c->R, cudaMemcpyDeviceToHost));
  return DYNBOND_OK;
}

dynbond_status dynbond_autotune(dynbond_ctx* c, const int32_t* d_pos, dynbond_tuning* out) {
  if (!c || !d_pos) return DYNBOND_EINVAL;
  if (!aligned16(d_pos)) return fail(c, DYNBOND_EINVAL, "d_pos must be 16-byte aligned (int4 per bead)");
  if (c->sticky) return c->sticky;
  dynbond_status st = DYNBOND_OK;
  if (c->max_cells) {
    const double scales[] = {1.0, 1.25, 1.5, 2.0, 3.0};
    const int grids[] = {4, 8, 16};
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    k_set_args<<<1, 1, 0, c->stream>>>(c->d.args, (const int4*)d_pos, nullptr, nullptr, 0, 1, 0, nullptr);
    const int zdivs[] = {1, 2, 4};
    float best = 1e30f;
    double best_scale = 1.0;
    int best_grid = 8, best_zdiv = 1;
    bool best_tiles = false;
    for (int g = 0; g < 15; ++g) {
      const double sc = scales[g / 3];
      const int zd = zdivs[g % 3];
      st = set_geometry(c, sc, zd);
      if (st == DYNBOND_ECAPACITY) {  // more cells than allocated: not a candidate
        st = DYNBOND_OK;
        continue;
      }
      if (st) break;
      // staged tiles, then the global search (a flag fixes one of them)
      const int mode0 = c->tiles_avail && !c->global_search ? 0 : 1, mode1 = c->staged_search ? 1 : 2;
      for (int mode = mode0; mode < std::max(mode1, mode0 + 1); ++mode) {
        c->cand_tiles = c->tiles_avail && mode == 0;
        for (int gm : grids) {
          c->grid_bead = c->grid_cand = bounded_grid(c->N, 256, c->nsm * gm);
          float ms = 1e30f;
          for (int rep = 0; rep < 4; ++rep) {  // the first run warms caches and clocks; best of three
            cudaEventRecord(e0, c->stream);
            enqueue_front(c);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep) ms = std::min(ms, t);
          }
          if (ms < best) {
            best = ms;
            best_scale = sc;
            best_zdiv = zd;
            best_grid = gm;
            best_tiles = c->cand_tiles;
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tiles_on = best_tiles;  // kept: later geometry changes stay with the timed choice
    if (!st) st = set_geometry(c, best_scale, best_zdiv);
    c->grid_bead = c->grid_cand = bounded_grid(c->N, 256, c->nsm * best_grid);
    c->tuning.bead_blocks_per_sm = c->tuning.candidate_blocks_per_sm = best_grid;
    c->tuning.front_ms = best;
    if (!st) st = device_status(c);
    if (!st) st = capture_graphs(c);
  }
  c->tuned = true;
  c->tuning.tuned = 1;
  if (out) *out = c->tuning;
  return st;
}

dynbond_status dynbond_get_tuning(dynbond_ctx* c, dynbond_tuning* out) {
  if (!c || !out) return DYNBOND_EINVAL;
  *out = c->tuning;
  return DYNBOND_OK;
}

dynbond_status dynbond_sync(dynbond_ctx* c) {
  if (!c) return DYNBOND_EINVAL;
  if (c->sticky) return c->sticky;
  return device_status(c);
}

dynbond_status dynbond_topology_hash(dynbond_ctx* c, uint64_t* h_out) {
  if (!c || !h_out) return DYNBOND_EINVAL;
  if (c->sticky) return c->sticky;
  const int R = c->R;
  unsigned long long* d_h = c->d_hash;
  cudaError_t e = cudaMemsetAsync(d_h, 0, 8 * (size_t)R, c->stream);
  if (e == cudaSuccess) {
    k_topo_hash<<<c->nsm * 4, 256, 0, c->stream>>>(c->d, d_h);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_h, 8 * (size_t)R, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return fail(c, DYNBOND_ECUDA, std::string("topology hash: ") + cudaGetErrorString(e));
  return device_status(c);
}

dynbond_status dynbond_get_topology(dynbond_ctx* c, dynbond_topology* t) {
  if (!c || !t) return DYNBOND_EINVAL;
  dynbond_status st = device_status(c);
  if (st && st != DYNBOND_OK && c->sticky == DYNBOND_ECUDA) return st;
  const long long N = c->N;
  const int R = c->R;
  std::vector<uint4> slots(N);
  std::vector<int> na(R), nd(R);
  std::vector<long long> off(R + 1);
  CUDA_TRY(c, cudaMemcpy(slots.data(), c->d.slots, 16 * N, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(na.data(), c->d.n_ang, 4 * R, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(nd.data(), c->d.n_dih, 4 * R, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(off.data(), c->d.off, 8 * (R + 1), cudaMemcpyDeviceToHost));
  auto part = [](unsigned v) { return v ? (int)(v >> 4) : -1; };
  auto stored = [&](long long x, long long y) {
    const unsigned* s = (const unsigned*)&slots[x];
    for (int q = 0; q < SLOTS; ++q)
      if (s[q] && part(s[q]) == y) return (int)(s[q] & 15u);
    return 0;
  };
  long long nb = 0, sa = 0, sd = 0;
  for (long long i = 0; i < N; ++i) {
    const unsigned* s = (const unsigned*)&slots[i];
    for (int q = 0; q < SLOTS; ++q) nb += part(s[q]) > i;
  }
  for (int r = 0; r < R; ++r) {
    sa += na[r];
    sd += nd[r];
  }
  bool fill = t->bonds || t->angles || t->dihedrals;
  if (fill) {
    if ((t->bonds && t->n_bonds < nb) || (t->angles && t->n_angles < sa) || (t->dihedrals && t->n_dihedrals < sd))
      return fail(c, DYNBOND_EINVAL, "topology arrays smaller than the counts");
    if (t->bonds) {
      std::vector<std::array<int, 4>> B;
      B.reserve(nb);
      for (long long i = 0; i < N; ++i) {
        const unsigned* s = (const unsigned*)&slots[i];
        for (int q = 0; q < SLOTS; ++q)
          if (part(s[q]) > i) B.push_back({(int)i, part(s[q]), (int)(s[q] & 15u), stored(part(s[q]), i)});
      }
      std::sort(B.begin(), B.end());
      std::memcpy(t->bonds, B.data(), B.size() * sizeof(B[0]));
    }
    if (t->angles) {
      std::vector<std::array<int, 4>> A(sa);
      long long at = 0;
      for (int r = 0; r < R; ++r) {
        if (na[r]) CUDA_TRY(c, cudaMemcpy(&A[at], c->d.ang + 6 * off[r], 16 * (size_t)na[r], cudaMemcpyDeviceToHost));
        at += na[r];
      }
      std::sort(A.begin(), A.end());
      std::memcpy(t->angles, A.data(), A.size() * sizeof(A[0]));
    }
    if (t->dihedrals) {
      std::vector<std::array<int, 4>> D4(sd);
      long long at = 0;
      for (int r = 0; r < R; ++r) {
        if (nd[r])
          CUDA_TRY(c, cudaMemcpy(&D4[at], c->d.dih + 18 * off[r], 16 * (size_t)nd[r], cudaMemcpyDeviceToHost));
        at += nd[r];
      }
      std::vector<std::array<int, 5>> D(sd);
      for (long long k = 0; k < sd; ++k)
        D[k] = {D4[k][0], D4[k][1], D4[k][2], D4[k][3] & 0x0FFFFFFF, (int)((unsigned)D4[k][3] >> 28)};
      std::sort(D.begin(), D.end());
      std::memcpy(t->dihedrals, D.data(), D.size() * sizeof(D[0]));
    }
  }
  t->n_bonds = nb;
  t->n_angles = sa;
  t->n_dihedrals = sd;
  return c->sticky;
}

dynbond_status dynbond_phase_times(dynbond_ctx* c, float* ms, const char** names, int32_t n, int32_t* n_out) {
  if (!c) return DYNBOND_EINVAL;
  if (!c->profile) return fail(c, DYNBOND_EINVAL, "context created without DYNBOND_FLAG_PROFILE");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->last_profiled & 1) collect_profile(c, 1);
  if (c->last_profiled & 2) collect_profile(c, 2);
  c->last_profiled = 0;
  int k = 0;
  for (size_t q = 0; q < c->last_step_ms.size(); ++q, ++k)
    if (k < n) {
      if (ms) ms[k] = c->last_step_ms[q];
      if (names) names[k] = c->names_step[q];
    }
  for (size_t q = 0; q < c->last_forces_ms.size(); ++q, ++k)
    if (k < n) {
      if (ms) ms[k] = c->last_forces_ms[q];
      if (names) names[k] = c->names_forces[q];
    }
  if (n_out) *n_out = k;
  return DYNBOND_OK;
}

}  // extern "C"
