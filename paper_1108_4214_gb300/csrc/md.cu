// Molecular-dynamics harness around the dynamic-bonding pass: velocity-Verlet
// with the DPD force field of Sec. 3 (conservative a w(r), dissipative
// -gamma w(r)^2 (rhat . v_ij), random sigma w(r) xi / sqrt(dt), sigma^2 =
// 2 kT gamma, w(r) = 1 - r / rc), non-bonded pairs switched off between beads
// fewer than 3 bonds apart, plus the bonded forces of the context.  Positions
// stay on the int32 grid of 2^-20 sigma: each drift adds the rounded
// displacement v dt.  One replica (one periodic box) per context.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace dynbond {
namespace {

struct MdDev {
  long long N;
  int L, nc;
  long long n_cells;
  float a, gamma, sigma_over_sqrt_dt, rc, inv_rc, dt, inv_m;
  long long rc_q2;  // (rc 2^20)^2 floor, pair cutoff in quantized units
  unsigned key0, key1;
  int* cell_count;  // [n_cells + 1] -> cell starts
  int* bead_cell;   // [N]
  int* bead_rank;   // [N]
  int4* sorted;     // [N] (x, y, z, bead)
  float4* fdpd;     // [N]
  unsigned long long* status;
  int* ticket;
  unsigned* err;
  int spin_limit;
};

__global__ void md_clear(MdDev m) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k <= m.n_cells;
       k += (long long)gridDim.x * blockDim.x)
    m.cell_count[k] = 0;
  long long nt = (m.n_cells + 2047) / 2048 + 2;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += (long long)gridDim.x * blockDim.x)
    m.status[k] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) *m.ticket = 0;
}

__global__ void md_bin(MdDev m, const int4* __restrict__ pos) {
  if (aborted(m.err)) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x) {
    int4 p = pos[i];
    long long c = (((long long)p.x * m.nc / m.L) * m.nc + (long long)p.y * m.nc / m.L) * m.nc +
                  (long long)p.z * m.nc / m.L;
    m.bead_cell[i] = (int)c;
    m.bead_rank[i] = atomicAdd(&m.cell_count[c], 1);
  }
}

__global__ void __launch_bounds__(256) md_scan(MdDev m) {
  __shared__ long long sh[33];
  __shared__ long long s_excl, s_tile;
  const long long n = m.n_cells, per_tile = 2048, ntiles = (n + per_tile - 1) / per_tile;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(m.ticket, 1);
    __syncthreads();
    long long t = s_tile;
    if (t >= ntiles) break;
    long long beg = t * per_tile + threadIdx.x * 8;
    int v[8];
    long long sum = 0;
    for (int k = 0; k < 8; ++k) {
      v[k] = beg + k < n ? m.cell_count[beg + k] : 0;
      sum += v[k];
    }
    long long tot, ex = block_excl_scan(sum, sh, &tot);
    if (threadIdx.x < 32) {
      long long x = lookback(m.status, t, 0, (unsigned long long)tot, m.spin_limit, m.err);
      if (threadIdx.x == 0) s_excl = x;
    }
    __syncthreads();
    if (s_excl < 0) return;
    long long pre = s_excl + ex;
    for (int k = 0; k < 8; ++k) {
      if (beg + k < n) m.cell_count[beg + k] = (int)pre;
      pre += v[k];
    }
    if (t == ntiles - 1 && threadIdx.x == blockDim.x - 1) m.cell_count[n] = (int)pre;
    __syncthreads();
  }
}

__global__ void md_scatter(MdDev m, const int4* __restrict__ pos) {
  if (aborted(m.err)) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x) {
    int4 p = pos[i];
    p.w = (int)i;
    m.sorted[m.cell_count[m.bead_cell[i]] + m.bead_rank[i]] = p;
  }
}

// pairs closer than 3 bonds (1-2, 1-3) carry no non-bonded force
__device__ __forceinline__ bool md_excluded(const uint4* __restrict__ slots, const uint4& si, int j) {
  int ni[SLOTS];
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    ni[q] = s_partner(s_get(si, q));
    if (ni[q] == j) return true;
  }
  uint4 sj = slots[j];
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    int b = s_partner(s_get(sj, q));
    if (b < 0) continue;
#pragma unroll
    for (int w = 0; w < SLOTS; ++w)
      if (ni[w] == b) return true;
  }
  return false;
}

// Gaussian of pair (lo, hi) at a step: Box-Muller on two Philox words; the
// counter is symmetric in the pair so both beads draw the same number.  The
// uniforms u1 = ((x0 >> 9) + 1/2) 2^-23 in (0, 1) and u2 = (x1 >> 9) 2^-23
// are exact in FP32.
__device__ __forceinline__ float md_gauss(const MdDev& m, int lo, int hi, unsigned long long step) {
  uint4 u = philox4x32_10(make_uint4((unsigned)lo, (unsigned)hi, (unsigned)step, (unsigned)(step >> 32) ^ 0x3D000000u),
                          make_uint2(m.key0, m.key1));
  float u1 = ((float)(u.x >> 9) + 0.5f) * (1.0f / 8388608.0f);
  float u2 = (float)(u.y >> 9) * (1.0f / 8388608.0f);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// The DPD force on bead i (sorted entry me, velocity vi, slots si) from
// entry o within r_c: conservative, dissipative and random parts, zero for a
// pair fewer than 3 bonds apart.
__device__ __forceinline__ float3 md_pair_force(const MdDev& m, const int4& me, int i, const float4& vi, const uint4& si,
                                                const int4& o, const float4* __restrict__ vel,
                                                const uint4* __restrict__ slots, unsigned long long step) {
  const int j = o.w;
  if (md_excluded(slots, si, j)) return make_float3(0.f, 0.f, 0.f);
  const float s20 = 1.0f / 1048576.0f;
  float3 r = make_float3((float)wrap_dx(me.x - o.x, m.L) * s20, (float)wrap_dx(me.y - o.y, m.L) * s20,
                         (float)wrap_dx(me.z - o.z, m.L) * s20);
  float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
  if (rr <= 0.f) return make_float3(0.f, 0.f, 0.f);
  float w = 1.0f - rr * m.inv_rc;
  float4 vj = vel[j];
  float rv = (r.x * (vi.x - vj.x) + r.y * (vi.y - vj.y) + r.z * (vi.z - vj.z)) / rr;
  float xi = md_gauss(m, min(i, j), max(i, j), step);
  float fs = m.a * w - m.gamma * w * w * rv + m.sigma_over_sqrt_dt * w * xi;
  return make_float3(fs * r.x / rr, fs * r.y / rr, fs * r.z / rr);
}

// DPD pair forces on every bead (both orders of a pair are evaluated, with the
// same random number), written with plain stores.  A bead first walks its
// 27 neighbouring cells keeping the entries within r_c (a short loop); the
// pair forces then run in lockstep across the warp, the k-th neighbour of
// every lane together, so the random number and the weight are computed
// with all lanes that have one instead of one lane at a time.  The pairs are
// summed in cell order either way.
constexpr int MD_NB = 32;  // neighbours within r_c a bead keeps for the lockstep loop
__global__ void __launch_bounds__(256) md_dpd(MdDev m, const int4* __restrict__ pos, const float4* __restrict__ vel,
                                               const uint4* __restrict__ slots, unsigned long long step) {
  if (aborted(m.err)) return;
  const int nc = m.nc, noff = nc >= 3 ? 3 : nc;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < m.N; base += stride) {  // warp-uniform
    const long long e = base + threadIdx.x;
    int4 me = make_int4(0, 0, 0, 0);
    int i = 0, np = 0;
    float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
    uint4 si = make_uint4(0, 0, 0, 0);
    int nb[MD_NB];
    bool more = false;
    int xs[3], ys[3], zs[3];
    if (e < m.N) {
      me = m.sorted[e];
      i = me.w;
      vi = vel[i];
      si = slots[i];
      const int cx = (int)((long long)me.x * nc / m.L), cy = (int)((long long)me.y * nc / m.L),
                cz = (int)((long long)me.z * nc / m.L);
      // the cells at offsets 0, +1, -1 (periodic) along each axis, distinct ones only
      xs[0] = cx, xs[1] = cx + 1 == nc ? 0 : cx + 1, xs[2] = cx == 0 ? nc - 1 : cx - 1;
      ys[0] = cy, ys[1] = cy + 1 == nc ? 0 : cy + 1, ys[2] = cy == 0 ? nc - 1 : cy - 1;
      zs[0] = cz, zs[1] = cz + 1 == nc ? 0 : cz + 1, zs[2] = cz == 0 ? nc - 1 : cz - 1;
      for (int a = 0; a < noff; ++a)
        for (int b = 0; b < noff; ++b)
          for (int c = 0; c < noff; ++c) {
            const long long cell = ((long long)xs[a] * nc + ys[b]) * nc + zs[c];
            const int q0 = m.cell_count[cell], q1 = m.cell_count[cell + 1];
            for (int q = q0; q < q1; ++q) {
              const int4 o = m.sorted[q];
              if (o.w == i || dist2(me, o, m.L) >= m.rc_q2) continue;
              if (np < MD_NB) nb[np++] = q;
              else more = true;
            }
          }
    }
    float3 f = make_float3(0.f, 0.f, 0.f);
    const int kmax = __reduce_max_sync(FULL, (unsigned)np);
    for (int k = 0; k < kmax; ++k) {
      if (k >= np) continue;
      const float3 df = md_pair_force(m, me, i, vi, si, m.sorted[nb[k]], vel, slots, step);
      f.x += df.x;
      f.y += df.y;
      f.z += df.z;
    }
    if (more) {  // more than MD_NB neighbours (dense spot): the pairs after the kept ones, in the same order
      int seen = 0;
      for (int a = 0; a < noff; ++a)
        for (int b = 0; b < noff; ++b)
          for (int c = 0; c < noff; ++c) {
            const long long cell = ((long long)xs[a] * nc + ys[b]) * nc + zs[c];
            const int q0 = m.cell_count[cell], q1 = m.cell_count[cell + 1];
            for (int q = q0; q < q1; ++q) {
              const int4 o = m.sorted[q];
              if (o.w == i || dist2(me, o, m.L) >= m.rc_q2) continue;
              if (seen++ < MD_NB) continue;
              const float3 df = md_pair_force(m, me, i, vi, si, o, vel, slots, step);
              f.x += df.x;
              f.y += df.y;
              f.z += df.z;
            }
          }
    }
    if (e < m.N) m.fdpd[i] = make_float4(f.x, f.y, f.z, 0.f);
  }
}

// v += dt/2 F/m, then (drift) x += v dt rounded onto the grid and wrapped
__global__ void md_kick(MdDev m, float4* vel, const float4* __restrict__ fb, int4* pos, int drift) {
  if (aborted(m.err)) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x) {
    float4 v = vel[i], a = fb[i], b = m.fdpd[i];
    float h = 0.5f * m.dt * m.inv_m;
    v.x += h * (a.x + b.x);
    v.y += h * (a.y + b.y);
    v.z += h * (a.z + b.z);
    vel[i] = v;
    if (drift) {
      int4 p = pos[i];
      const float q = 1048576.0f * m.dt;
      int dx = __float2int_rn(v.x * q), dy = __float2int_rn(v.y * q), dz = __float2int_rn(v.z * q);
      p.x = (int)(((long long)p.x + dx) % m.L);
      p.y = (int)(((long long)p.y + dy) % m.L);
      p.z = (int)(((long long)p.z + dz) % m.L);
      if (p.x < 0) p.x += m.L;
      if (p.y < 0) p.y += m.L;
      if (p.z < 0) p.z += m.L;
      pos[i] = p;
    }
  }
}

}  // namespace
}  // namespace dynbond

using namespace dynbond;

struct dynbond_md {
  dynbond_ctx* ctx = nullptr;
  MdDev m{};
  const uint4* slots = nullptr;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  float4* fbond = nullptr;
  double* ev = nullptr;
  std::vector<void*> allocs;
};

extern "C" {

void dynbond_md_destroy(dynbond_md* md) {
  if (!md) return;
  if (md->stream) cudaStreamSynchronize(md->stream);
  for (void* p : md->allocs) cudaFree(p);
  delete md;
}

dynbond_status dynbond_md_create(dynbond_ctx* ctx, const dynbond_dpd* prm, dynbond_md** out) {
  if (!ctx || !prm || !out) return DYNBOND_EINVAL;
  *out = nullptr;
  long long N = 0, box = 0;
  int R = 0;
  cudaStream_t s = nullptr;
  const uint4* slots = dynbond::internal_slots(ctx, &N, &box, &R, &s);
  if (R != 1 || !(prm->rc > 0) || !(prm->dt > 0) || !(prm->mass > 0) || prm->gamma < 0 || prm->kT < 0)
    return DYNBOND_EINVAL;
  dynbond_md* md = new dynbond_md();
  md->ctx = ctx;
  md->slots = slots;
  md->stream = s;
  cudaGetDevice(&md->nsm);
  cudaDeviceGetAttribute(&md->nsm, cudaDevAttrMultiProcessorCount, md->nsm);
  MdDev& m = md->m;
  m.N = N;
  m.L = (int)box;
  double rcq = prm->rc * 1048576.0;
  long long w = (long long)std::ceil(rcq);
  m.nc = (int)std::max<long long>(1, std::min<long long>(box / std::max<long long>(w, 1), 1024));
  m.n_cells = (long long)m.nc * m.nc * m.nc;
  m.a = (float)prm->a;
  m.gamma = (float)prm->gamma;
  m.sigma_over_sqrt_dt = (float)(std::sqrt(2.0 * prm->kT * prm->gamma) / std::sqrt(prm->dt));
  m.rc = (float)prm->rc;
  m.inv_rc = (float)(1.0 / prm->rc);
  m.dt = (float)prm->dt;
  m.inv_m = (float)(1.0 / prm->mass);
  m.rc_q2 = (long long)std::floor(rcq * rcq);
  m.key0 = (unsigned)prm->seed;
  m.key1 = (unsigned)(prm->seed >> 32);
  m.spin_limit = 1 << 24;
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    md->allocs.push_back(*p);
    return true;
  };
  bool ok = alloc((void**)&m.cell_count, 4 * (m.n_cells + 1)) && alloc((void**)&m.bead_cell, 4 * N) &&
            alloc((void**)&m.bead_rank, 4 * N) && alloc((void**)&m.sorted, 16 * N) && alloc((void**)&m.fdpd, 16 * N) &&
            alloc((void**)&m.status, 8 * ((m.n_cells + 2047) / 2048 + 2)) && alloc((void**)&m.ticket, 4) &&
            alloc((void**)&m.err, 4) && alloc((void**)&md->fbond, 16 * N) && alloc((void**)&md->ev, 8 * 7);
  if (!ok || cudaMemsetAsync(m.err, 0, 4, s) != cudaSuccess) {
    cudaGetLastError();
    dynbond_md_destroy(md);
    return DYNBOND_ENOMEM;
  }
  *out = md;
  return DYNBOND_OK;
}

namespace {
// DPD pair forces of step `step` into m.fdpd (cell binning, scan, scatter, pairs)
dynbond_status md_pair(dynbond_md* md, const int32_t* d_pos, const float* d_vel, unsigned long long step) {
  const MdDev& m = md->m;
  cudaStream_t s = md->stream;
  int g = std::max(1, std::min<int>((int)((m.N + 255) / 256), md->nsm * 8));
  md_clear<<<md->nsm * 2, 256, 0, s>>>(m);
  md_bin<<<g, 256, 0, s>>>(m, (const int4*)d_pos);
  md_scan<<<md->nsm * 4, 256, 0, s>>>(m);
  md_scatter<<<g, 256, 0, s>>>(m, (const int4*)d_pos);
  md_dpd<<<g, 256, 0, s>>>(m, (const int4*)d_pos, (const float4*)d_vel, md->slots, step);
  return cudaGetLastError() != cudaSuccess ? DYNBOND_ECUDA : DYNBOND_OK;
}

dynbond_status md_forces(dynbond_md* md, int32_t* d_pos, const float* d_vel, unsigned long long step) {
  dynbond_status st = md_pair(md, d_pos, d_vel, step);
  if (st) return st;
  return dynbond_forces(md->ctx, d_pos, (float*)md->fbond, md->ev);
}

dynbond_status md_wait(dynbond_md* md) {
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, md->m.err, 4, cudaMemcpyDeviceToHost, md->stream) != cudaSuccess ||
      cudaStreamSynchronize(md->stream) != cudaSuccess)
    return DYNBOND_ECUDA;
  return err ? DYNBOND_ETIMEOUT : DYNBOND_OK;
}
}  // namespace

dynbond_status dynbond_md_pair_forces(dynbond_md* md, const int32_t* d_pos, const float* d_vel, uint64_t step,
                                      float* d_force) {
  if (!md || !d_pos || !d_vel || !d_force) return DYNBOND_EINVAL;
  if (((uintptr_t)d_pos | (uintptr_t)d_vel | (uintptr_t)d_force) & 15u) return DYNBOND_EINVAL;
  dynbond_status st = md_pair(md, d_pos, d_vel, step);
  if (st) return st;
  if (cudaMemcpyAsync(d_force, md->m.fdpd, 16 * (size_t)md->m.N, cudaMemcpyDeviceToDevice, md->stream) !=
      cudaSuccess)
    return DYNBOND_ECUDA;
  return md_wait(md);
}

dynbond_status dynbond_md_advance(dynbond_md* md, int32_t* d_pos, float* d_vel, int64_t n_steps, uint64_t first_step,
                                  double* d_ev) {
  if (!md || !d_pos || !d_vel || n_steps < 0) return DYNBOND_EINVAL;
  const MdDev& m = md->m;
  cudaStream_t s = md->stream;
  int g = std::max(1, std::min<int>((int)((m.N + 255) / 256), md->nsm * 8));
  // forces at the current time (the topology may have changed since the last call)
  dynbond_status st = md_forces(md, d_pos, d_vel, first_step);
  if (st) return st;
  for (int64_t k = 0; k < n_steps; ++k) {
    md_kick<<<g, 256, 0, s>>>(m, (float4*)d_vel, md->fbond, (int4*)d_pos, 1);
    st = md_forces(md, d_pos, d_vel, first_step + (uint64_t)k + 1);
    if (st) return st;
    md_kick<<<g, 256, 0, s>>>(m, (float4*)d_vel, md->fbond, (int4*)d_pos, 0);
  }
  if (d_ev && cudaMemcpyAsync(d_ev, md->ev, 8 * 7, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return DYNBOND_ECUDA;
  return md_wait(md);
}

}  // extern "C"
