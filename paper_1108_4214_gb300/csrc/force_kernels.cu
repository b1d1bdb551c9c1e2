// Bonded forces of the current topology: FP32 arithmetic per interaction
// from exact integer minimum-image displacements (scaled by 2^-20), FP64
// block reductions of the energy and the virial per replica.
//   bonds     each bead sums the harmonic force of the type IT stores for
//             each of its bonds (directional bonds, Sec. 2) -- no atomics;
//   angles    E = K (1 + cos theta), forces added with float4 atomics;
//   dihedrals E = K (1 + d cos phi) (Sec. 3), forces from the
//             Blondel-Karplus (J. Comput. Chem. 17, 1132 (1996)) derivatives
//             of phi, free of the sin(phi) = 0 singularity.
// Work items are (replica, tile) pairs so each block reduces one replica.
#include "common.cuh"
#include "kernels.h"

namespace dynbond {

__device__ __forceinline__ float3 relq(const int4& a, const int4& b, int L) {
  const float q = 1.0f / 1048576.0f;
  return make_float3((float)wrap_dx(a.x - b.x, L) * q, (float)wrap_dx(a.y - b.y, L) * q,
                     (float)wrap_dx(a.z - b.z, L) * q);
}
// exact integer minimum-image displacement a - b (quantized units)
__device__ __forceinline__ int3 reli(const int4& a, const int4& b, int L) {
  return make_int3(wrap_dx(a.x - b.x, L), wrap_dx(a.y - b.y, L), wrap_dx(a.z - b.z, L));
}
struct L3 {
  long long x, y, z;
};
__device__ __forceinline__ L3 crossi(int3 a, int3 b) {
  return L3{(long long)a.y * b.z - (long long)a.z * b.y, (long long)a.z * b.x - (long long)a.x * b.z,
            (long long)a.x * b.y - (long long)a.y * b.x};
}
__device__ __forceinline__ long long doti(int3 a, int3 b) {
  return (long long)a.x * b.x + (long long)a.y * b.y + (long long)a.z * b.z;
}
// a . b formed exactly in 128 bits, returned as FP32 times 2^e2
__device__ __forceinline__ float triplei(int3 a, L3 b, int e2) {
  __int128 t = (__int128)a.x * b.x + (__int128)a.y * b.y + (__int128)a.z * b.z;
  const __int128 lim = (__int128)0x3FFFFFFFFFFFFFFFll;
  while (t > lim || t < -lim) {  // drop low bits: relative change below 2^-54
    t >>= 8;
    e2 += 8;
  }
  return ldexpf((float)(long long)t, e2);
}
__device__ __forceinline__ float3 tof(int3 v, float s) {
  return make_float3((float)v.x * s, (float)v.y * s, (float)v.z * s);
}
__device__ __forceinline__ float3 tof(L3 v, float s) {
  return make_float3((float)v.x * s, (float)v.y * s, (float)v.z * s);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 axpy(float a, float3 x, float3 y) {
  return make_float3(a * x.x + y.x, a * x.y + y.y, a * x.z + y.z);
}
__device__ __forceinline__ float3 scale(float a, float3 x) { return make_float3(a * x.x, a * x.y, a * x.z); }

// Energy / virial accumulators: each FP32 term is added with an error-free
// transformation (TwoSum), so a thread's partial sum is a float pair with
// about twice the FP32 precision; warps combine the pairs the same way, and
// only the per-warp totals enter FP64 (block sum, then one FP64 atomic per
// component per block).  FP64 is thus used only where the reduction needs it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

struct EV {
  float hi[7], lo[7];
  __device__ EV() {
#pragma unroll
    for (int k = 0; k < 7; ++k) hi[k] = lo[k] = 0.f;
  }
  __device__ void add(int k, float x) {
    float s, e;
    two_sum(hi[k], x, s, e);
    hi[k] = s;
    lo[k] = __fadd_rn(lo[k], e);
  }
  // W_ab += w r_a F_b (xx, yy, zz, xy, xz, yz)
  __device__ void vir(float3 r, float3 f, float w) {
    add(1, __fmul_rn(__fmul_rn(w, r.x), f.x));
    add(2, __fmul_rn(__fmul_rn(w, r.y), f.y));
    add(3, __fmul_rn(__fmul_rn(w, r.z), f.z));
    add(4, __fmul_rn(__fmul_rn(w, r.x), f.y));
    add(5, __fmul_rn(__fmul_rn(w, r.x), f.z));
    add(6, __fmul_rn(__fmul_rn(w, r.y), f.z));
  }
};

// block-reduce the 7 accumulators and add them to replica r
__device__ void flush_ev(const Dev& d, EV& acc, int r) {
  __shared__ double sh[7][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    float h = acc.hi[k], l = acc.lo[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float h2 = __shfl_down_sync(FULL, h, o), l2 = __shfl_down_sync(FULL, l, o);
      float s, e;
      two_sum(h, h2, s, e);
      h = s;
      l = __fadd_rn(__fadd_rn(l, l2), e);
    }
    if (lane == 0) sh[k][wid] = (double)h + (double)l;
    acc.hi[k] = acc.lo[k] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
    atomicAdd(&d.ev_acc[r * 7 + threadIdx.x], s);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_bond_forces(Dev d, FF ff) {
  const int4* __restrict__ pos = d.args->pos;
  float4* __restrict__ force = d.args->force;
  const int R = d.R, nitems = d.tb_beads[R];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int r = find_seg(d.tb_beads, R, it);
    long long beg = d.off[r] + (long long)(it - d.tb_beads[r]) * BEAD_TILE;
    long long end = min(beg + BEAD_TILE, d.off[r + 1]);
    int L = (int)d.box[r];
    EV acc;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
      int4 p = pos[i];
      uint4 s = d.slots[i];
      float3 f = make_float3(0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        unsigned v = s_get(s, q);
        if (!v) continue;
        int t = s_type(v);
        float3 rij = relq(p, pos[s_partner(v)], L);
        float rr = sqrtf(dot3(rij, rij));
        float dr = rr - ff.bond_r0[t];
        float fscal = -2.0f * ff.bond_k[t] * dr / rr;
        float3 fq = scale(fscal, rij);
        f = make_float3(f.x + fq.x, f.y + fq.y, f.z + fq.z);
        acc.add(0, __fmul_rn(__fmul_rn(0.5f * ff.bond_k[t], dr), dr));
        acc.vir(rij, fq, 0.5f);
      }
      force[i] = make_float4(f.x, f.y, f.z, 0.f);
    }
    flush_ev(d, acc, r);
  }
}

__device__ __forceinline__ void add_force(float4* f, int i, float3 v) {
  atomicAdd(f + i, make_float4(v.x, v.y, v.z, 0.f));
}

__global__ void __launch_bounds__(256) k_angle_forces(Dev d, FF ff) {
  const int4* __restrict__ pos = d.args->pos;
  float4* force = d.args->force;
  const int R = d.R, nitems = d.tb_ang[R];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int r = find_seg(d.tb_ang, R, it);
    int lt = it - d.tb_ang[r];
    const int4* recs = d.ang + 6 * d.off[r];
    int beg = lt * FORCE_TILE, end = min(beg + FORCE_TILE, d.n_ang[r]);
    int L = (int)d.box[r];
    EV acc;
    for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
      int4 a = recs[k];
      if ((unsigned)a.x >= (unsigned)d.N || (unsigned)a.y >= (unsigned)d.N || (unsigned)a.z >= (unsigned)d.N) {
        atomicOr(d.err, ERR_INTERNAL);
        continue;
      }
      int4 pb = pos[a.y];
      float3 ra = relq(pos[a.x], pb, L), rc = relq(pos[a.z], pb, L);
      float K = ff.angle_k[a.w];
      float la2 = dot3(ra, ra), lc2 = dot3(rc, rc);
      float inv = rsqrtf(la2 * lc2);
      float cs = dot3(ra, rc) * inv;
      // F_A = -K d(cos)/d(r_A), F_C likewise, F_B = -(F_A + F_C)
      float3 Fa = scale(-K, axpy(-cs / la2, ra, scale(inv, rc)));
      float3 Fc = scale(-K, axpy(-cs / lc2, rc, scale(inv, ra)));
      float3 Fb = make_float3(-Fa.x - Fc.x, -Fa.y - Fc.y, -Fa.z - Fc.z);
      add_force(force, a.x, Fa);
      add_force(force, a.y, Fb);
      add_force(force, a.z, Fc);
      acc.add(0, __fmul_rn(K, 1.0f + cs));
      acc.vir(ra, Fa, 1.f);
      acc.vir(rc, Fc, 1.f);
    }
    flush_ev(d, acc, r);
  }
}

__global__ void __launch_bounds__(256) k_dihedral_forces(Dev d, FF ff) {
  const int4* __restrict__ pos = d.args->pos;
  float4* force = d.args->force;
  const int R = d.R, nitems = d.tb_dih[R];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int r = find_seg(d.tb_dih, R, it);
    int lt = it - d.tb_dih[r];
    const int4* recs = d.dih + 18 * d.off[r];
    int beg = lt * FORCE_TILE, end = min(beg + FORCE_TILE, d.n_dih[r]);
    int L = (int)d.box[r];
    EV acc;
    for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
      int4 rec = recs[k];
      int ia = rec.x, ib = rec.y, ic = rec.z, id = rec.w & 0x0FFFFFFF;
      int t = (int)((unsigned)rec.w >> 28);
      if ((unsigned)ia >= (unsigned)d.N || (unsigned)ib >= (unsigned)d.N || (unsigned)ic >= (unsigned)d.N ||
          (unsigned)id >= (unsigned)d.N) {
        atomicOr(d.err, ERR_INTERNAL);
        continue;
      }
      int4 pb = pos[ib], pc = pos[ic];
      // Blondel-Karplus: F = r_A - r_B, G = r_B - r_C, H = r_D - r_C,
      // A = F x G, B = H x G; cos phi = A.B / (|A||B|), phi = 180 deg trans.
      // The cross, dot and triple products are formed exactly from the integer
      // displacements and rounded once, so near-collinear quartets keep FP32
      // accuracy; the rest is FP32.
      int3 Fi = reli(pos[ia], pb, L), Gi = reli(pb, pc, L), Hi = reli(pos[id], pc, L);
      L3 Ai = crossi(Fi, Gi), Bi = crossi(Hi, Gi);
      const float s20 = 1.0f / 1048576.0f, s40 = s20 * s20;
      float3 F = tof(Fi, s20), G = tof(Gi, s20), H = tof(Hi, s20);
      float3 A = tof(Ai, s40), B = tof(Bi, s40);
      float A2 = dot3(A, A), B2 = dot3(B, B);
      float rg = sqrtf((float)doti(Gi, Gi) * s40);
      float rab = rsqrtf(A2 * B2);
      float cs = dot3(A, B) * rab;
      // (B x A).G = -|G|^2 F.B, so sin phi = -|G| (F.B) / (|A||B|)
      float sn = -rg * triplei(Fi, Bi, -60) * rab;
      float K = ff.dih_k[t], dd = ff.dih_d[t];
      // E = K (1 + d cos phi): -dE/dphi = K d sin phi
      float mdE = K * dd * sn;
      float fg = (float)doti(Fi, Gi) * s40, hg = (float)doti(Hi, Gi) * s40;
      float ia2 = 1.0f / A2, ib2 = 1.0f / B2;
      // dphi/dr_A = -|G|/A^2 A ; dphi/dr_D = |G|/B^2 B
      // dphi/dr_B = (|G|/A^2 + F.G/(A^2|G|)) A - H.G/(B^2|G|) B
      // dphi/dr_C = -F.G/(A^2|G|) A + (H.G/(B^2|G|) - |G|/B^2) B
      float3 dA = scale(-rg * ia2, A);
      float3 dD = scale(rg * ib2, B);
      float3 dB = axpy(-hg * ib2 / rg, B, scale(rg * ia2 + fg * ia2 / rg, A));
      float3 dC = axpy(hg * ib2 / rg - rg * ib2, B, scale(-fg * ia2 / rg, A));
      float3 Fa = scale(mdE, dA), Fb = scale(mdE, dB), Fc = scale(mdE, dC), Fd = scale(mdE, dD);
      add_force(force, ia, Fa);
      add_force(force, ib, Fb);
      add_force(force, ic, Fc);
      add_force(force, id, Fd);
      acc.add(0, __fmul_rn(K, 1.0f + dd * cs));
      // virial relative to B: r_A - r_B = F, r_C - r_B = -G, r_D - r_B = H - G
      acc.vir(F, Fa, 1.f);
      acc.vir(make_float3(-G.x, -G.y, -G.z), Fc, 1.f);
      acc.vir(make_float3(H.x - G.x, H.y - G.y, H.z - G.z), Fd, 1.f);
    }
    flush_ev(d, acc, r);
  }
}

__global__ void k_ev_out(Dev d) {
  double* out = d.args->ev;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 7 * d.R; k += gridDim.x * blockDim.x) out[k] = d.ev_acc[k];
}

}  // namespace dynbond
