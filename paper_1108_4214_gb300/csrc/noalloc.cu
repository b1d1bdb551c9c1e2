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

// Per-replica energy / virial accumulators (7 doubles each), shared by every
// call on a device; each call clears the part it uses before accumulating.
static __device__ __align__(256) double g_noalloc_ev[NA_MAX_R * 7];

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

__device__ __forceinline__ float3 na_rel(const int4& a, const int4& b, int L) {
  const float q = 1.0f / 1048576.0f;
  return make_float3((float)wrap_dx(a.x - b.x, L) * q, (float)wrap_dx(a.y - b.y, L) * q,
                     (float)wrap_dx(a.z - b.z, L) * q);
}
__device__ __forceinline__ float na_dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

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

__global__ void na_clear(double* ev, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) ev[k] = 0.0;
}

// bonds: each bead applies the force of the type it stores (directional
// bonds, Sec. 2) and books half the energy; plain stores initialize force[]
__global__ void na_bonds(const int4* __restrict__ pos, const uint4* __restrict__ slots, const long long* off,
                         const long long* box, int R, long long N, FF ff, float4* force, double* ev) {
  NaAcc acc;
  acc.flush(nullptr);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int r = na_rep(off, R, i);
    acc.to(r, ev);
    int L = (int)box[r];
    int4 p = pos[i];
    uint4 s = slots[i];
    float3 f = make_float3(0.f, 0.f, 0.f);
    for (int q = 0; q < SLOTS; ++q) {
      unsigned v = s_get(s, q);
      if (!v) continue;
      int t = s_type(v);
      float3 rij = na_rel(p, pos[s_partner(v)], L);
      float rr = sqrtf(na_dot(rij, rij));
      float dr = rr - ff.bond_r0[t];
      float fs = -2.0f * ff.bond_k[t] * dr / rr;
      float3 fq = make_float3(fs * rij.x, fs * rij.y, fs * rij.z);
      f = make_float3(f.x + fq.x, f.y + fq.y, f.z + fq.z);
      acc.e[0] += (double)(0.5f * ff.bond_k[t] * dr * dr);
      acc.vir(rij, fq, 0.5f);
    }
    force[i] = make_float4(f.x, f.y, f.z, 0.f);
  }
  acc.flush_warp(ev);
}

__device__ __forceinline__ void na_add(float4* f, int i, float3 v) { red_add_f4(f, i, v.x, v.y, v.z); }

// angles E = K (1 + cos theta); dihedrals E = K (1 + d cos phi) with the
// Blondel-Karplus derivatives of phi
__global__ void na_angles_dihedrals(const int4* __restrict__ pos, const long long* off, const long long* box, int R,
                                    const int* __restrict__ ang, long long na, const int* __restrict__ dih,
                                    long long nd, FF ff, float4* force, double* ev) {
  NaAcc acc;
  acc.flush(nullptr);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < na + nd; k += stride) {
    if (k < na) {
      int a = ang[4 * k], b = ang[4 * k + 1], c = ang[4 * k + 2], t = ang[4 * k + 3];
      int r = na_rep(off, R, b);
      acc.to(r, ev);
      int L = (int)box[r];
      int4 pb = pos[b];
      float3 ra = na_rel(pos[a], pb, L), rc = na_rel(pos[c], pb, L);
      float la2 = na_dot(ra, ra), lc2 = na_dot(rc, rc);
      float inv = rsqrtf(la2 * lc2);
      float cs = na_dot(ra, rc) * inv;
      float Ea;
      const float cf = angle_coef(ff, t, pos[a], pb, pos[c], L, cs, inv, &Ea);
      float3 Fa = make_float3(cf * (rc.x * inv - cs * ra.x / la2), cf * (rc.y * inv - cs * ra.y / la2),
                              cf * (rc.z * inv - cs * ra.z / la2));
      float3 Fc = make_float3(cf * (ra.x * inv - cs * rc.x / lc2), cf * (ra.y * inv - cs * rc.y / lc2),
                              cf * (ra.z * inv - cs * rc.z / lc2));
      na_add(force, a, Fa);
      na_add(force, b, make_float3(-Fa.x - Fc.x, -Fa.y - Fc.y, -Fa.z - Fc.z));
      na_add(force, c, Fc);
      acc.e[0] += (double)Ea;
      acc.vir(ra, Fa, 1.f);
      acc.vir(rc, Fc, 1.f);
    } else {
      long long m = k - na;
      int ia = dih[5 * m], ib = dih[5 * m + 1], ic = dih[5 * m + 2], id = dih[5 * m + 3], t = dih[5 * m + 4];
      int r = na_rep(off, R, ib);
      acc.to(r, ev);
      int L = (int)box[r];
      int4 pb = pos[ib], pc = pos[ic], pa = pos[ia], pd = pos[id];
      // F = r_A - r_B, G = r_B - r_C, H = r_D - r_C; A = F x G, B = H x G,
      // products formed exactly from the integer displacements
      int3 Fi = make_int3(wrap_dx(pa.x - pb.x, L), wrap_dx(pa.y - pb.y, L), wrap_dx(pa.z - pb.z, L));
      int3 Gi = make_int3(wrap_dx(pb.x - pc.x, L), wrap_dx(pb.y - pc.y, L), wrap_dx(pb.z - pc.z, L));
      int3 Hi = make_int3(wrap_dx(pd.x - pc.x, L), wrap_dx(pd.y - pc.y, L), wrap_dx(pd.z - pc.z, L));
      long long Ax = (long long)Fi.y * Gi.z - (long long)Fi.z * Gi.y, Ay = (long long)Fi.z * Gi.x - (long long)Fi.x * Gi.z,
                Az = (long long)Fi.x * Gi.y - (long long)Fi.y * Gi.x;
      long long Bx = (long long)Hi.y * Gi.z - (long long)Hi.z * Gi.y, By = (long long)Hi.z * Gi.x - (long long)Hi.x * Gi.z,
                Bz = (long long)Hi.x * Gi.y - (long long)Hi.y * Gi.x;
      const float s20 = 1.0f / 1048576.0f, s40 = s20 * s20;
      float3 F = make_float3(Fi.x * s20, Fi.y * s20, Fi.z * s20), G = make_float3(Gi.x * s20, Gi.y * s20, Gi.z * s20);
      float3 H = make_float3(Hi.x * s20, Hi.y * s20, Hi.z * s20);
      float3 A = make_float3((float)Ax * s40, (float)Ay * s40, (float)Az * s40);
      float3 B = make_float3((float)Bx * s40, (float)By * s40, (float)Bz * s40);
      float A2 = na_dot(A, A), B2 = na_dot(B, B);
      float rg = sqrtf((float)((long long)Gi.x * Gi.x + (long long)Gi.y * Gi.y + (long long)Gi.z * Gi.z) * s40);
      float rab = rsqrtf(A2 * B2);
      float cs = na_dot(A, B) * rab;
      // sin phi = -|G| (F . B) / (|A||B|), with F . B exact in 128 bits
      __int128 tp = (__int128)Fi.x * Bx + (__int128)Fi.y * By + (__int128)Fi.z * Bz;
      int e2 = -60;
      while (tp > (__int128)0x3FFFFFFFFFFFFFFFll || tp < -(__int128)0x3FFFFFFFFFFFFFFFll) {
        tp >>= 8;
        e2 += 8;
      }
      float sn = -rg * ldexpf((float)(long long)tp, e2) * rab;
      float K = ff.dih_k[t], dd = ff.dih_d[t];
      float mdE = K * dd * sn;
      float fg = (float)((long long)Fi.x * Gi.x + (long long)Fi.y * Gi.y + (long long)Fi.z * Gi.z) * s40;
      float hg = (float)((long long)Hi.x * Gi.x + (long long)Hi.y * Gi.y + (long long)Hi.z * Gi.z) * s40;
      float c1 = -rg / A2, c4 = rg / B2, cbA = rg / A2 + fg / (A2 * rg), cbB = -hg / (B2 * rg);
      float ccA = -fg / (A2 * rg), ccB = hg / (B2 * rg) - rg / B2;
      float3 Fa = make_float3(mdE * c1 * A.x, mdE * c1 * A.y, mdE * c1 * A.z);
      float3 Fd = make_float3(mdE * c4 * B.x, mdE * c4 * B.y, mdE * c4 * B.z);
      float3 Fb = make_float3(mdE * (cbA * A.x + cbB * B.x), mdE * (cbA * A.y + cbB * B.y),
                              mdE * (cbA * A.z + cbB * B.z));
      float3 Fc = make_float3(mdE * (ccA * A.x + ccB * B.x), mdE * (ccA * A.y + ccB * B.y),
                              mdE * (ccA * A.z + ccB * B.z));
      na_add(force, ia, Fa);
      na_add(force, ib, Fb);
      na_add(force, ic, Fc);
      na_add(force, id, Fd);
      acc.e[0] += (double)(K * (1.0f + dd * cs));
      acc.vir(F, Fa, 1.f);
      acc.vir(make_float3(-G.x, -G.y, -G.z), Fc, 1.f);
      acc.vir(make_float3(H.x - G.x, H.y - G.y, H.z - G.z), Fd, 1.f);
    }
  }
  acc.flush_warp(ev);
}

__global__ void na_copy(const double* src, double* dst, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[k] = src[k];
}

// Device address of the scratch array, looked up once per device (host code
// may not use the array's name as a device pointer).
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
    e = cudaGetSymbolAddress(&p, g_noalloc_ev);
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
        (const int4*)d_pos, (const long long*)d_bead_offset, (const long long*)d_box_q, n_replicas, d_angles,
        n_angles, d_dihedrals, n_dihedrals, f, (float4*)d_force, scratch);
  na_copy<<<(nev + 255) / 256, 256, 0, s>>>(scratch, d_ev, nev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return DYNBOND_ECUDA;
  return DYNBOND_OK;
}
