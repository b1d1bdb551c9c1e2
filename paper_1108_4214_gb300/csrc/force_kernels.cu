// Bonded forces of the current topology: FP32 arithmetic per interaction
// from exact integer minimum-image displacements (scaled by 2^-20), FP64
// block reductions of the energy and the virial per replica.
//   bonds     each bead sums the harmonic force of the type IT stores for
//             each of its bonds (directional bonds, Sec. 2) -- no atomics;
//   angles    E = K (1 + cos theta), forces added with float4 atomics;
//   dihedrals E = K (1 + d cos phi) (Sec. 3), forces from the
//             Blondel-Karplus (J. Comput. Chem. 17, 1132 (1996)) derivatives
//             of phi, free of the sin(phi) = 0 singularity.
// Work items are (replica, tile) pairs; a block reduces its energy / virial
// when it moves to another replica and at its end.
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

// Energy / virial accumulators: a thread sums its own few terms (at most a
// few tens: its beads' bonds or its records over the launch) in plain FP32;
// warps combine the threads' partials with an error-free transformation
// (TwoSum), so a warp total is a float pair with about twice the FP32
// precision, and only the per-warp totals enter FP64 (block sum, then one
// striped FP64 atomic per component per block).  FP64 is thus used only
// where the reduction needs it, and a thread holds 7 registers for it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

struct EV {
  float hi[7];
  __device__ EV() {
#pragma unroll
    for (int k = 0; k < 7; ++k) hi[k] = 0.f;
  }
  __device__ void add(int k, float x) { hi[k] = __fadd_rn(hi[k], x); }
  // W_ab += r_a F_b + q_a G_b, the two terms summed in FP32 first
  __device__ void vir2(float3 r, float3 f, float3 q, float3 g) {
    add(1, r.x * f.x + q.x * g.x);
    add(2, r.y * f.y + q.y * g.y);
    add(3, r.z * f.z + q.z * g.z);
    add(4, r.x * f.y + q.x * g.y);
    add(5, r.x * f.z + q.x * g.z);
    add(6, r.y * f.z + q.y * g.z);
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
    float h = acc.hi[k], l = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float h2 = __shfl_down_sync(FULL, h, o), l2 = __shfl_down_sync(FULL, l, o);
      float s, e;
      two_sum(h, h2, s, e);
      h = s;
      l = __fadd_rn(__fadd_rn(l, l2), e);
    }
    if (lane == 0) sh[k][wid] = (double)h + (double)l;
    acc.hi[k] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
    // striped: blocks add to one of EV_COPIES copies, so the FP64 atomics
    // of a launch do not all meet at the same seven addresses
    atomicAdd(&d.ev_acc[((long long)r * EV_COPIES + blockIdx.x % EV_COPIES) * 7 + threadIdx.x], s);
  }
  __syncthreads();
}

// bonds: BEAD_TILE beads per work item, BEAD_PER_THREAD per thread with
// every load issued before the arithmetic
constexpr int BEAD_PER_THREAD = BEAD_TILE / 256;

__global__ void __launch_bounds__(256) k_bond_forces(Dev d, FF ff) {
  pdl_enter();
  if (aborted(d.err)) return;
  const int4* __restrict__ pos = d.args->pos;
  float4* __restrict__ force = d.args->force;
  const int R = d.R, nitems = d.tb_beads[R];
  EV acc;
  int racc = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int r = find_seg(d.tb_beads, R, it);
    if (r != racc) {
      if (racc >= 0) flush_ev(d, acc, racc);
      racc = r;
    }
    long long beg = d.off[r] + (long long)(it - d.tb_beads[r]) * BEAD_TILE;
    long long end = min(beg + BEAD_TILE, d.off[r + 1]);
    int L = (int)d.box[r];
    int4 p[BEAD_PER_THREAD];
    uint4 s[BEAD_PER_THREAD];
#pragma unroll
    for (int u = 0; u < BEAD_PER_THREAD; ++u) {
      long long i = beg + threadIdx.x + u * 256;
      s[u] = make_uint4(0, 0, 0, 0);
      if (i < end) {
        p[u] = pos[i];
        s[u] = d.slots[i];
      }
    }
    int4 q[BEAD_PER_THREAD][SLOTS];
#pragma unroll
    for (int u = 0; u < BEAD_PER_THREAD; ++u)
#pragma unroll
      for (int k = 0; k < SLOTS; ++k) {
        unsigned v = s_get(s[u], k);
        if (v) q[u][k] = pos[s_partner(v)];
      }
    float e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < BEAD_PER_THREAD; ++u) {
      long long i = beg + threadIdx.x + u * 256;
      if (i >= end) continue;
      float3 f = make_float3(0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < SLOTS; ++k) {
        unsigned v = s_get(s[u], k);
        if (!v) continue;
        int t = s_type(v);
        float3 rij = relq(p[u], q[u][k], L);
        float ir = rsqrtf(dot3(rij, rij));
        float dr = dot3(rij, rij) * ir - ff.bond_r0[t];
        float fscal = -2.0f * ff.bond_k[t] * dr * ir;
        float3 fq = scale(fscal, rij);
        f = make_float3(f.x + fq.x, f.y + fq.y, f.z + fq.z);
        e += 0.5f * ff.bond_k[t] * dr * dr;
        w[0] += rij.x * fq.x;
        w[1] += rij.y * fq.y;
        w[2] += rij.z * fq.z;
        w[3] += rij.x * fq.y;
        w[4] += rij.x * fq.z;
        w[5] += rij.y * fq.z;
      }
      force[i] = make_float4(f.x, f.y, f.z, 0.f);
    }
    acc.add(0, e);
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.add(k + 1, 0.5f * w[k]);
  }
  if (racc >= 0) flush_ev(d, acc, racc);
}

__device__ __forceinline__ void add_force(float4* f, int i, float3 v) {
  red_add_f4(f, i, v.x, v.y, v.z);
}

constexpr int ANG_PER_THREAD = FORCE_TILE / 256;
constexpr int DIH_PER_THREAD = FORCE_TILE / 256;

// Angles and dihedrals in one launch: items [0, tb_fang[R]) are angle tiles,
// the rest dihedral tiles; both add their forces with float4 atomics.
__global__ void __launch_bounds__(256) k_angle_dihedral_forces(Dev d, FF ff) {
  pdl_enter();
  if (aborted(d.err)) return;
  const int4* __restrict__ pos = d.args->pos;
  float4* force = d.args->force;
  const int R = d.R, na_items = d.tb_fang[R], nitems = na_items + d.tb_fdih[R];
  const unsigned N = (unsigned)d.N;
  EV acc;
  int racc = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const bool dih = it >= na_items;
    const int* tb = dih ? d.tb_fdih : d.tb_fang;
    int t0 = dih ? it - na_items : it;
    int r = find_seg(tb, R, t0);
    if (r != racc) {
      if (racc >= 0) flush_ev(d, acc, racc);
      racc = r;
    }
    int lt = t0 - tb[r];
    int L = (int)d.box[r];
    float e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!dih) {
      const int4* recs = d.ang + 6 * d.off[r];
      int beg = lt * FORCE_TILE, end = min(beg + FORCE_TILE, d.n_ang[r]);
      int4 a[ANG_PER_THREAD], pa[ANG_PER_THREAD], pb[ANG_PER_THREAD], pc[ANG_PER_THREAD];
      bool ok[ANG_PER_THREAD];
#pragma unroll
      for (int u = 0; u < ANG_PER_THREAD; ++u) {
        int k = beg + threadIdx.x + u * 256;
        ok[u] = k < end;
        if (ok[u]) a[u] = recs[k];
        ok[u] = ok[u] && (unsigned)a[u].x < N && (unsigned)a[u].y < N && (unsigned)a[u].z < N;
        if (k < end && !ok[u]) atomicOr(d.err, ERR_INTERNAL);
      }
#pragma unroll
      for (int u = 0; u < ANG_PER_THREAD; ++u)
        if (ok[u]) {
          pa[u] = pos[a[u].x];
          pb[u] = pos[a[u].y];
          pc[u] = pos[a[u].z];
        }
#pragma unroll
      for (int u = 0; u < ANG_PER_THREAD; ++u) {
        if (!ok[u]) continue;
        float3 ra = relq(pa[u], pb[u], L), rc = relq(pc[u], pb[u], L);
        float K = ff.angle_k[a[u].w];
        float ia = rsqrtf(dot3(ra, ra)), ic = rsqrtf(dot3(rc, rc));
        float inv = ia * ic;
        float cs = dot3(ra, rc) * inv;
        // F_A = -K d(cos)/d(r_A), F_C likewise, F_B = -(F_A + F_C)
        float3 Fa = scale(-K, axpy(-cs * ia * ia, ra, scale(inv, rc)));
        float3 Fc = scale(-K, axpy(-cs * ic * ic, rc, scale(inv, ra)));
        float3 Fb = make_float3(-Fa.x - Fc.x, -Fa.y - Fc.y, -Fa.z - Fc.z);
        add_force(force, a[u].x, Fa);
        add_force(force, a[u].y, Fb);
        add_force(force, a[u].z, Fc);
        e += K * (1.0f + cs);
        w[0] += ra.x * Fa.x + rc.x * Fc.x;
        w[1] += ra.y * Fa.y + rc.y * Fc.y;
        w[2] += ra.z * Fa.z + rc.z * Fc.z;
        w[3] += ra.x * Fa.y + rc.x * Fc.y;
        w[4] += ra.x * Fa.z + rc.x * Fc.z;
        w[5] += ra.y * Fa.z + rc.y * Fc.z;
      }
    } else {
      const int4* recs = d.dih + 18 * d.off[r];
      int beg = lt * FORCE_TILE, end = min(beg + FORCE_TILE, d.n_dih[r]);
      int4 rec[DIH_PER_THREAD], P[DIH_PER_THREAD][4];
      bool ok[DIH_PER_THREAD];
#pragma unroll
      for (int u = 0; u < DIH_PER_THREAD; ++u) {
        int k = beg + threadIdx.x + u * 256;
        ok[u] = k < end;
        if (ok[u]) rec[u] = recs[k];
        unsigned id = (unsigned)(rec[u].w & 0x0FFFFFFF);
        ok[u] = ok[u] && (unsigned)rec[u].x < N && (unsigned)rec[u].y < N && (unsigned)rec[u].z < N && id < N;
        if (k < end && !ok[u]) atomicOr(d.err, ERR_INTERNAL);
      }
#pragma unroll
      for (int u = 0; u < DIH_PER_THREAD; ++u)
        if (ok[u]) {
          P[u][0] = pos[rec[u].x];
          P[u][1] = pos[rec[u].y];
          P[u][2] = pos[rec[u].z];
          P[u][3] = pos[rec[u].w & 0x0FFFFFFF];
        }
#pragma unroll
      for (int u = 0; u < DIH_PER_THREAD; ++u) {
        if (!ok[u]) continue;
        int ia = rec[u].x, ib = rec[u].y, ic = rec[u].z, id = rec[u].w & 0x0FFFFFFF;
        int t = (int)((unsigned)rec[u].w >> 28);
        // Blondel-Karplus: F = r_A - r_B, G = r_B - r_C, H = r_D - r_C,
        // A = F x G, B = H x G; cos phi = A.B / (|A||B|), phi = 180 deg trans.
        // The cross, dot and triple products are formed exactly from the
        // integer displacements and rounded once, so near-collinear quartets
        // keep FP32 accuracy; the rest is FP32.
        int3 Fi = reli(P[u][0], P[u][1], L), Gi = reli(P[u][1], P[u][2], L), Hi = reli(P[u][3], P[u][2], L);
        L3 Ai = crossi(Fi, Gi), Bi = crossi(Hi, Gi);
        const float s20 = 1.0f / 1048576.0f, s40 = s20 * s20;
        float3 F = tof(Fi, s20), G = tof(Gi, s20), H = tof(Hi, s20);
        float3 A = tof(Ai, s40), B = tof(Bi, s40);
        float A2 = dot3(A, A), B2 = dot3(B, B);
        float gg = (float)doti(Gi, Gi) * s40;
        float irg = rsqrtf(gg), rg = gg * irg;
        float rab = rsqrtf(A2 * B2);
        float cs = dot3(A, B) * rab;
        // (B x A).G = -|G|^2 F.B, so sin phi = -|G| (F.B) / (|A||B|)
        float sn = -rg * triplei(Fi, Bi, -60) * rab;
        float K = ff.dih_k[t], dd = ff.dih_d[t];
        // E = K (1 + d cos phi): -dE/dphi = K d sin phi
        float mdE = K * dd * sn;
        float fg = (float)doti(Fi, Gi) * s40, hg = (float)doti(Hi, Gi) * s40;
        float ia2 = __frcp_rn(A2), ib2 = __frcp_rn(B2);
        // dphi/dr_A = -|G|/A^2 A ; dphi/dr_D = |G|/B^2 B
        // dphi/dr_B = (|G|/A^2 + F.G/(A^2|G|)) A - H.G/(B^2|G|) B
        // dphi/dr_C = -F.G/(A^2|G|) A + (H.G/(B^2|G|) - |G|/B^2) B
        float3 dA = scale(-rg * ia2, A);
        float3 dD = scale(rg * ib2, B);
        float3 dB = axpy(-hg * ib2 * irg, B, scale(rg * ia2 + fg * ia2 * irg, A));
        float3 dC = axpy(hg * ib2 * irg - rg * ib2, B, scale(-fg * ia2 * irg, A));
        float3 Fa = scale(mdE, dA), Fb = scale(mdE, dB), Fc = scale(mdE, dC), Fd = scale(mdE, dD);
        add_force(force, ia, Fa);
        add_force(force, ib, Fb);
        add_force(force, ic, Fc);
        add_force(force, id, Fd);
        e += K * (1.0f + dd * cs);
        // virial relative to B: r_A - r_B = F, r_C - r_B = -G, r_D - r_B = H - G
        float3 mg = make_float3(-G.x, -G.y, -G.z), hm = make_float3(H.x - G.x, H.y - G.y, H.z - G.z);
        w[0] += F.x * Fa.x + mg.x * Fc.x + hm.x * Fd.x;
        w[1] += F.y * Fa.y + mg.y * Fc.y + hm.y * Fd.y;
        w[2] += F.z * Fa.z + mg.z * Fc.z + hm.z * Fd.z;
        w[3] += F.x * Fa.y + mg.x * Fc.y + hm.x * Fd.y;
        w[4] += F.x * Fa.z + mg.x * Fc.z + hm.x * Fd.z;
        w[5] += F.y * Fa.z + mg.y * Fc.z + hm.y * Fd.z;
      }
    }
    acc.add(0, e);
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.add(k + 1, w[k]);
  }
  if (racc >= 0) flush_ev(d, acc, racc);
}

// Order-independent topology hash (see dynbond_topology_hash): per replica,
// the sum of splitmix64-mixed bond ends and interaction records.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_topo_hash(Dev d, unsigned long long* h) {
  if (aborted(d.err)) return;
  const int R = d.R;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += stride) {
    const int r = rep_of(d, i);
    const long long o = d.off[r];
    const uint4 s = d.slots[i];
    unsigned long long acc = 0;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      const unsigned v = s_get(s, q);
      if (!v) continue;
      const unsigned long long j = (unsigned long long)(s_partner(v) - o);
      acc += mix64(((unsigned long long)(i - o) << 32) | (j << 4) | (unsigned long long)s_type(v));
    }
    if (acc) atomicAdd(h + r, acc);
  }
  for (int r = 0; r < R; ++r) {
    const long long o = d.off[r];
    const int4* ang = d.ang + 6 * o;
    const int4* dih = d.dih + 18 * o;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < d.n_ang[r]; k += stride) {
      const int4 a = ang[k];
      unsigned long long z = mix64(0xA);
      z = mix64(z ^ (unsigned long long)(a.x - o));
      z = mix64(z ^ (unsigned long long)(a.y - o));
      z = mix64(z ^ (unsigned long long)(a.z - o));
      atomicAdd(h + r, mix64(z ^ (unsigned long long)a.w));
    }
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < d.n_dih[r]; k += stride) {
      const int4 a = dih[k];
      unsigned long long z = mix64(0xD);
      z = mix64(z ^ (unsigned long long)(a.x - o));
      z = mix64(z ^ (unsigned long long)(a.y - o));
      z = mix64(z ^ (unsigned long long)(a.z - o));
      z = mix64(z ^ (unsigned long long)((a.w & 0x0FFFFFFF) - o));
      atomicAdd(h + r, mix64(z ^ (unsigned long long)((unsigned)a.w >> 28)));
    }
  }
}

// sum the striped copies of the energy / virial, write them out and clear
// the accumulators for the next force call
__global__ void k_ev_out(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  double* out = d.args->ev;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 7 * d.R; k += gridDim.x * blockDim.x) {
    const int r = k / 7, c = k % 7;
    double s = 0.0;
    for (int q = 0; q < EV_COPIES; ++q) {
      double* p = d.ev_acc + ((long long)r * EV_COPIES + q) * 7 + c;
      s += *p;
      *p = 0.0;
    }
    out[k] = s;
  }
}

}  // namespace dynbond
