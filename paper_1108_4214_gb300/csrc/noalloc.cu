// Bonded forces for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host simulation engine that has
// reserved the GPU's memory for its own pool allocator before this library
// is loaded, or a latency-critical loop in which cudaMalloc's implicit device
// synchronization is not acceptable.  dynbond_forces_noalloc serves them: it
// evaluates the same bonded forces as dynbond_forces, but for a topology the
// caller passes in, and without any allocation.  Its only scratch -- the
// per-replica FP64 energy / virial accumulators -- is a file-scope device
// array of fixed size, held by every GPU that loads the library until the
// process exits.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace dynbond {
namespace {

constexpr int NA_MAX_R = DYNBOND_NOALLOC_MAX_REPLICAS;
constexpr int NA_ERR_SLOT = NA_MAX_R * 7;  // the call's error word, after the accumulators

// The scratch shared by every call on a device: per-replica energy / virial
// accumulators (7 doubles each) and, in the slot after them, the error word
// of the call (nonzero when a term named a bead outside its replica or a type
// outside 0..15).  Each call clears what it uses before accumulating.
static __device__ __align__(256) double g_noalloc_scratch[NA_ERR_SLOT + 1];

// replica of bead x: largest r with off[r] <= x
__device__ __forceinline__ int na_rep(const long long* off, int R, long long x) {
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// bead id x lies in [0, N) and in the bead range [lo, hi) of the replica
__device__ __forceinline__ bool na_in(long long x, long long lo, long long hi, long long N) {
  return x >= 0 && x < N && x >= lo && x < hi;
}
__device__ __forceinline__ void na_flag(double* scratch) {
  atomicOr(reinterpret_cast<unsigned long long*>(scratch + NA_ERR_SLOT), 1ull);
}

// Per-lane FP64 accumulation of one replica's energy and virial; flushed
// with atomics to the scratch when the lane moves to another replica.
struct NaAcc {
  double e[7];
  int r = -1;
  __device__ void to(int rr, double* ev) {
    if (rr == r) return;
    flush(ev);
    r = rr;
  }
  __device__ void flush(double* ev) {
    if (r >= 0)
      for (int k = 0; k < 7; ++k)
        if (e[k] != 0.0) atomicAdd(&ev[r * 7 + k], e[k]);
    for (int k = 0; k < 7; ++k) e[k] = 0.0;
  }
  // end of a kernel: lanes holding the same replica are summed across the
  // warp first (every lane of the warp must call this)
  __device__ void flush_warp(double* ev) {
    const int lane = threadIdx.x & 31;
    while (true) {
      unsigned live = __ballot_sync(0xffffffffu, r >= 0);
      if (!live) break;
      int rr = __shfl_sync(0xffffffffu, r, __ffs(live) - 1);
      bool mine = r == rr;
      for (int k = 0; k < 7; ++k) {
        double v = mine ? e[k] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(&ev[rr * 7 + k], v);
      }
      if (mine) {
        r = -1;
        for (int k = 0; k < 7; ++k) e[k] = 0.0;
      }
    }
  }
  __device__ void vir(float3 rv, float3 f, float w) {
    e[1] += (double)(w * rv.x * f.x);
    e[2] += (double)(w * rv.y * f.y);
    e[3] += (double)(w * rv.z * f.z);
    e[4] += (double)(w * rv.x * f.y);
    e[5] += (double)(w * rv.x * f.z);
    e[6] += (double)(w * rv.y * f.z);
  }
};

// zero the accumulators of n_ev values and the error word
__global__ void na_clear(double* scratch, int n_ev) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_ev; k += gridDim.x * blockDim.x) scratch[k] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(scratch + NA_ERR_SLOT) = 0ull;
}

// bonds: each bead applies the force of the type it stores (directional
// bonds, Sec. 2) and books half the energy; plain stores initialize force[].
// A slot whose partner lies outside the bead's replica is skipped and flagged.
__global__ void na_bonds(const int4* __restrict__ pos, const uint4* __restrict__ slots, const long long* off,
                         const long long* box, int R, long long N, FF ff, float4* force, double* scratch) {
  NaAcc acc;
  acc.flush(nullptr);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int r = na_rep(off, R, i);
    acc.to(r, scratch);
    const long long lo = off[r], hi = off[r + 1];
    const int L = (int)box[r];
    const int4 p = pos[i];
    const uint4 s = slots[i];
    float3 f = make_float3(0.f, 0.f, 0.f);
    for (int q = 0; q < SLOTS; ++q) {
      const unsigned v = s_get(s, q);
      if (!v) continue;
      const long long j = s_partner(v);
      if (!na_in(j, lo, hi, N)) {
        na_flag(scratch);
        continue;
      }
      const BondHalf h = bond_half_force(ff, s_type(v), reli(p, pos[j], L));
      f = make_float3(f.x + h.f.x, f.y + h.f.y, f.z + h.f.z);
      acc.e[0] += (double)h.E;
      acc.vir(h.rij, h.f, 0.5f);
    }
    force[i] = make_float4(f.x, f.y, f.z, 0.f);
  }
  acc.flush_warp(scratch);
}

__device__ __forceinline__ void na_add(float4* f, int i, float3 v) { red_add_f4(f, i, v.x, v.y, v.z); }

// angles and dihedrals (angle_term_forces, dihedral_term_forces); a record
// naming a bead outside the replica of its centre bead b, or a type outside
// 0..15, is skipped and flagged
__global__ void na_angles_dihedrals(const int4* __restrict__ pos, const long long* off, const long long* box, int R,
                                    long long N, const int* __restrict__ ang, long long na,
                                    const int* __restrict__ dih, long long nd, FF ff, float4* force,
                                    double* scratch) {
  NaAcc acc;
  acc.flush(nullptr);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < na + nd; k += stride) {
    if (k < na) {
      const int a = ang[4 * k], b = ang[4 * k + 1], c = ang[4 * k + 2], t = ang[4 * k + 3];
      if (b < 0 || b >= N) {
        na_flag(scratch);
        continue;
      }
      const int r = na_rep(off, R, b);
      const long long lo = off[r], hi = off[r + 1];
      if (!na_in(a, lo, hi, N) || !na_in(b, lo, hi, N) || !na_in(c, lo, hi, N) || (unsigned)t >= 16u) {
        na_flag(scratch);
        continue;
      }
      acc.to(r, scratch);
      const AngleTerm o = angle_term_forces(ff, t, pos[a], pos[b], pos[c], (int)box[r]);
      na_add(force, a, o.Fa);
      na_add(force, b, make_float3(-o.Fa.x - o.Fc.x, -o.Fa.y - o.Fc.y, -o.Fa.z - o.Fc.z));
      na_add(force, c, o.Fc);
      acc.e[0] += (double)o.E;
      acc.vir(o.ra, o.Fa, 1.f);
      acc.vir(o.rc, o.Fc, 1.f);
    } else {
      const long long m = k - na;
      const int ia = dih[5 * m], ib = dih[5 * m + 1], ic = dih[5 * m + 2], id = dih[5 * m + 3], t = dih[5 * m + 4];
      if (ib < 0 || ib >= N) {
        na_flag(scratch);
        continue;
      }
      const int r = na_rep(off, R, ib);
      const long long lo = off[r], hi = off[r + 1];
      if (!na_in(ia, lo, hi, N) || !na_in(ib, lo, hi, N) || !na_in(ic, lo, hi, N) || !na_in(id, lo, hi, N) ||
          (unsigned)t >= 16u) {
        na_flag(scratch);
        continue;
      }
      acc.to(r, scratch);
      const DihedralTerm o = dihedral_term_forces(ff, t, pos[ia], pos[ib], pos[ic], pos[id], (int)box[r]);
      na_add(force, ia, o.Fa);
      na_add(force, ib, o.Fb);
      na_add(force, ic, o.Fc);
      na_add(force, id, o.Fd);
      acc.e[0] += (double)o.E;
      // relative to B: r_A - r_B = F, r_C - r_B = -G, r_D - r_B = H - G
      acc.vir(o.F, o.Fa, 1.f);
      acc.vir(make_float3(-o.G.x, -o.G.y, -o.G.z), o.Fc, 1.f);
      acc.vir(make_float3(o.H.x - o.G.x, o.H.y - o.G.y, o.H.z - o.G.z), o.Fd, 1.f);
    }
  }
  acc.flush_warp(scratch);
}

__global__ void na_copy(const double* src, double* dst, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[k] = src[k];
}

// Device address of the scratch array, looked up once per device (host code
// may not use the array's name as a device pointer).  The address belongs to
// the device's primary context: no call may follow a cudaDeviceReset of that
// device in the same process.
std::mutex g_mu;
double* g_scratch[256] = {};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = (double*)p;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dynbond

using namespace dynbond;

extern "C" dynbond_status dynbond_forces_noalloc(const int32_t* d_pos, const uint32_t* d_slots,
                                                 const int64_t* d_bead_offset, const int64_t* d_box_q,
                                                 int32_t n_replicas, int64_t n_beads, const int32_t* d_angles,
                                                 int64_t n_angles, const int32_t* d_dihedrals, int64_t n_dihedrals,
                                                 const dynbond_forcefield* ff, float* d_force, double* d_ev,
                                                 dynbond_stream stream) {
  if (n_replicas < 1 || n_replicas > NA_MAX_R)
    return DYNBOND_EINVAL;
  if (n_beads < 0 || n_angles < 0 || n_dihedrals < 0 || n_beads >= (1ll << 28))
    return DYNBOND_EINVAL;
  if (!ff || !d_ev || !d_bead_offset || !d_box_q || (n_beads && (!d_pos || !d_slots || !d_force)) ||
      (n_angles && !d_angles) || (n_dihedrals && !d_dihedrals))
    return DYNBOND_EINVAL;
  if ((n_beads && (((uintptr_t)d_pos | (uintptr_t)d_slots | (uintptr_t)d_force) & 15u)) ||
      ((uintptr_t)d_bead_offset | (uintptr_t)d_box_q | (uintptr_t)d_ev) & 7u ||
      ((uintptr_t)d_angles | (uintptr_t)d_dihedrals) & 3u)
    return DYNBOND_EINVAL;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return DYNBOND_ECUDA;
  FF f;
  if (!make_ff(*ff, f)) return DYNBOND_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int nev = 7 * n_replicas;
  na_clear<<<(nev + 255) / 256, 256, 0, s>>>(scratch, nev);
  if (n_beads)
    na_bonds<<<(int)std::min<long long>((n_beads + 255) / 256, 1024), 256, 0, s>>>(
        (const int4*)d_pos, (const uint4*)d_slots, (const long long*)d_bead_offset, (const long long*)d_box_q,
        n_replicas, n_beads, f, (float4*)d_force, scratch);
  if (n_angles + n_dihedrals)
    na_angles_dihedrals<<<(int)std::min<long long>((n_angles + n_dihedrals + 255) / 256, 1024), 256, 0, s>>>(
        (const int4*)d_pos, (const long long*)d_bead_offset, (const long long*)d_box_q, n_replicas, n_beads,
        d_angles, n_angles, d_dihedrals, n_dihedrals, f, (float4*)d_force, scratch);
  na_copy<<<(nev + 255) / 256, 256, 0, s>>>(scratch, d_ev, nev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return DYNBOND_ECUDA;
  // the error word: read back once the kernels are done
  unsigned long long bad = 0;
  e = cudaMemcpyAsync(&bad, scratch + NA_ERR_SLOT, sizeof(bad), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return DYNBOND_ECUDA;
  return bad ? DYNBOND_EINVAL : DYNBOND_OK;
}
