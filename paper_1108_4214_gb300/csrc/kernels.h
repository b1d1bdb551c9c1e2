// Kernel declarations and tile sizes shared by the kernel translation units
// and the host context.
#pragma once

#include <cmath>

#include "common.cuh"

namespace dynbond {

constexpr int PURGE_TILE = 1024;   // 256 threads x 4 records (small tiles balance the blocks)
constexpr int PURGE_PER_THREAD = 4;
constexpr int PURGE_COARSE_WORDS = 4096;  // coarse dirty bitmap of the purge, held in shared memory (16 KB)
constexpr int FILL_TILE = 256;     // hole / tail items per k_fill work item, one per thread
constexpr int BIN_SEG = 128;      // beads per binning segment (a warp, four loads per lane)
constexpr int SCAN_PER_THREAD = 32;  // cell keys per thread in the histogram scan (a multiple of 4)
constexpr int FORCE_TILE = 512;    // records per force work item (2 per thread)
constexpr int AD_THREADS = 256;    // threads of the angle / dihedral force blocks
constexpr int AD_PER_THREAD = FORCE_TILE / AD_THREADS;
// shared memory of an angle / dihedral block: records of three tiles and four
// positions per record of two tiles, 16 bytes each
constexpr int AD_SMEM_BYTES = 16 * AD_THREADS * AD_PER_THREAD * (3 + 2 * 4);
constexpr int BEAD_TILE = 512;     // beads per force work item (2 per thread)
constexpr int BF_THREADS = 256;    // threads of the bond force blocks
constexpr int BF_PER_THREAD = BEAD_TILE / BF_THREADS;
// shared memory of a bond force block: slots of three tiles, own and partner
// positions of two tiles, 16 bytes each
constexpr int BF_SMEM_BYTES = 16 * BF_THREADS * BF_PER_THREAD * (3 + 2 * (1 + DYNBOND_SLOTS));
constexpr int EV_COPIES = 32;      // striped copies of each replica's energy / virial sums
constexpr int FORCE_TILE_TABLE = 256;  // work items per force block looked up ahead (shared memory)
constexpr int MATCH_THREADS = 256; // threads of the (cooperative) matching blocks
// candidate search by staged tiles (k_candidates_tile): cell columns per tile
// side, staged z cells per column, and the stage's capacities
constexpr int CT = 8;
constexpr int CZS_MAX = 24;
constexpr int C_COL_CAP = 200;     // staged columns
constexpr int C_ENT_CAP = 2048;    // staged entries (16 bytes each)
constexpr int CAND_TILE_SMEM = 48 * 1024;

// bonded force-field tables in FP32 (kernel parameter space)
struct FF {
  float bond_k[16], bond_r0[16], angle_k[16], dih_k[16], dih_d[16];
  long long bond_r0q2[16];  // (r0 2^20)^2 rounded: r0^2 in quantized units^2
  float angle_pt0[16];  // pi - theta0 of the harmonic angle types
  unsigned angle_harm;  // bit t: angle type t is harmonic in theta
};

// Device copy of a force field (FP32 parameters); false for an unknown angle style.
inline bool make_ff(const dynbond_forcefield& in, FF& out) {
  out = FF{};
  for (int t = 0; t < 16; ++t) {
    out.bond_k[t] = (float)in.bond_k[t];
    out.bond_r0[t] = (float)in.bond_r0[t];
    const double r0q = in.bond_r0[t] * 1048576.0;
    out.bond_r0q2[t] = (long long)std::llround(r0q * r0q);
    out.angle_k[t] = (float)in.angle_k[t];
    out.dih_k[t] = (float)in.dihedral_k[t];
    out.dih_d[t] = (float)in.dihedral_d[t];
    out.angle_pt0[t] = (float)(3.14159265358979323846 - in.angle_theta0[t]);
    if (in.angle_style[t] != 0 && in.angle_style[t] != 1) return false;
    if (in.angle_style[t] == 1) out.angle_harm |= 1u << t;
  }
  return true;
}

// The block's copy of a force field in shared memory.  Terms of different
// types meet in one warp, and a per-type lookup with lane-dependent indices
// replays in the constant bank once per distinct address; from shared memory
// it is one access.  Every thread of the block must call it.
__device__ __forceinline__ const FF& ff_to_shared(const FF& ff, FF& s) {
  const int t = threadIdx.x;
  if (t < 16) {
    s.bond_k[t] = ff.bond_k[t];
    s.bond_r0[t] = ff.bond_r0[t];
    s.angle_k[t] = ff.angle_k[t];
    s.dih_k[t] = ff.dih_k[t];
    s.dih_d[t] = ff.dih_d[t];
    s.bond_r0q2[t] = ff.bond_r0q2[t];
    s.angle_pt0[t] = ff.angle_pt0[t];
  }
  if (t == 0) s.angle_harm = ff.angle_harm;
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// Per-term force arithmetic shared by the context's force kernels and the
// allocation-free entry point.  Every term starts from exact integer
// minimum-image displacements (quantized units, 2^-20 sigma); cross, dot and
// triple products are formed exactly in 64 / 128-bit integers and rounded
// once, the rest is FP32.
// ---------------------------------------------------------------------------
struct L3 {
  long long x, y, z;
};
__device__ __forceinline__ int3 reli(const int4& a, const int4& b, int L) {
  return make_int3(wrap_dx(a.x - b.x, L), wrap_dx(a.y - b.y, L), wrap_dx(a.z - b.z, L));
}
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

// One end of a bond, seen from the bead that stores type t, from the exact
// integer displacement d = r_i - r_j (quantized units): the end feels the
// full force of E = K (r - r0)^2 of the type IT stores and books half the
// energy (directional bonds, Sec. 2).  r - r0 is formed as (|d|^2 - r0^2) /
// (r + r0) with the difference of squares exact in 64-bit integers, so a bond
// near its rest length keeps FP32 relative accuracy in r - r0 (sqrt(|d|^2) -
// r0 in FP32 would cancel down to the rounding of r).
struct BondHalf {
  float3 rij, f;
  float E;
};
__device__ __forceinline__ BondHalf bond_half_force(const FF& ff, int t, int3 d) {
  const float s20 = 1.0f / 1048576.0f;
  BondHalf o;
  o.rij = tof(d, s20);
  const long long q2 = doti(d, d);
  const float q2f = (float)q2, rs = rsqrtf(q2f);  // 1 / |d| in quantized units
  const float r = q2f * rs * s20;
  const float dr = __fdividef((float)(q2 - ff.bond_r0q2[t]) * (s20 * s20), r + ff.bond_r0[t]);
  o.f = scale(-2.0f * ff.bond_k[t] * dr * (rs * 1048576.0f), o.rij);
  o.E = 0.5f * ff.bond_k[t] * dr * dr;
  return o;
}

// One angle term of type t (ends A and C, centre B): end forces Fa, Fc
// (F_B = -(Fa + Fc)), the relative vectors ra = r_A - r_B, rc = r_C - r_B
// for the virial, and the energy.
//   cosine    E = K (1 + cos theta): F_A = -K dcos/dr_A, F_C likewise.
//   harmonic  E = K (theta - theta0)^2 (the DNA angles of Sec. 3), with theta
//             = atan2(|ra x rc|, ra . rc) from the exact integer products.
//             The gradient of theta is taken through the unit normal n of the
//             plane ABC: dtheta/dr_A = (ra x n) / |ra|^2 and dtheta/dr_C =
//             -(rc x n) / |rc|^2, which has magnitude 1 / |r| at every angle
//             (no division by sin theta), so F_A = -2K (theta - theta0)
//             (ra x n) / |ra|^2 and F_C = 2K (theta - theta0) (rc x n) /
//             |rc|^2 are exact up to rounding arbitrarily close to 0 and
//             180 degrees.  Exactly collinear beads (ra x rc = 0) have no
//             plane and get no angle force (for theta0 = 180 deg that is the
//             exact force).
struct AngleTerm {
  float3 ra, rc, Fa, Fc;
  float E;
};
__device__ __forceinline__ AngleTerm angle_term_forces(const FF& ff, int t, const int4& pa, const int4& pb,
                                                       const int4& pc, int L) {
  const float s20 = 1.0f / 1048576.0f;
  const int3 u = reli(pa, pb, L), v = reli(pc, pb, L);
  AngleTerm o;
  o.ra = tof(u, s20);
  o.rc = tof(v, s20);
  const float K = ff.angle_k[t];
  if (!((ff.angle_harm >> t) & 1u)) {
    const float ia = rsqrtf(dot3(o.ra, o.ra)), ic = rsqrtf(dot3(o.rc, o.rc));
    const float inv = ia * ic;
    const float cs = dot3(o.ra, o.rc) * inv;
    // F_A = -K dcos/dr_A = -K (rc / (|ra||rc|) - cos ra / |ra|^2), F_C likewise
    o.Fa = scale(-K, axpy(-cs * ia * ia, o.ra, scale(inv, o.rc)));
    o.Fc = scale(-K, axpy(-cs * ic * ic, o.rc, scale(inv, o.ra)));
    o.E = K * (1.0f + cs);
    return o;
  }
  const L3 w = crossi(u, v);  // |w| = |ra||rc| sin theta (units^2), exact
  const float wx = (float)w.x, wy = (float)w.y, wz = (float)w.z;
  const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
  const float pth = atan2f(wn, -(float)doti(u, v));  // pi - theta
  const float dth = ff.angle_pt0[t] - pth;          // theta - theta0
  o.E = K * dth * dth;
  if (wn == 0.0f) {
    o.Fa = o.Fc = make_float3(0.f, 0.f, 0.f);
    return o;
  }
  const float3 n = make_float3(wx / wn, wy / wn, wz / wn);
  const float ga = -2.0f * K * dth / dot3(o.ra, o.ra), gc = 2.0f * K * dth / dot3(o.rc, o.rc);
  o.Fa = scale(ga, cross3(o.ra, n));
  o.Fc = scale(gc, cross3(o.rc, n));
  return o;
}

// One dihedral term of type t: E = K (1 + d cos phi), phi = 180 deg trans
// (Sec. 3).  Blondel-Karplus (J. Comput. Chem. 17, 1132 (1996)): F = r_A -
// r_B, G = r_B - r_C, H = r_D - r_C, A = F x G, B = H x G; cos phi = A.B /
// (|A||B|), sin phi = -|G| (F.B) / (|A||B|) since (B x A).G = -|G|^2 F.B; the
// derivatives of phi carry no 1 / sin phi.  Returns the four forces, the
// energy and the vectors F, G, H for the virial (r_A - r_B = F, r_C - r_B =
// -G, r_D - r_B = H - G).
struct DihedralTerm {
  float3 F, G, H, Fa, Fb, Fc, Fd;
  float E;
};
__device__ __forceinline__ DihedralTerm dihedral_term_forces(const FF& ff, int t, const int4& P0, const int4& P1,
                                                             const int4& P2, const int4& P3, int L) {
  const int3 Fi = reli(P0, P1, L), Gi = reli(P1, P2, L), Hi = reli(P3, P2, L);
  const L3 Ai = crossi(Fi, Gi), Bi = crossi(Hi, Gi);
  const float s20 = 1.0f / 1048576.0f, s40 = s20 * s20;
  DihedralTerm o;
  o.F = tof(Fi, s20);
  o.G = tof(Gi, s20);
  o.H = tof(Hi, s20);
  const float3 A = tof(Ai, s40), B = tof(Bi, s40);
  const float A2 = dot3(A, A), B2 = dot3(B, B);
  const float gg = (float)doti(Gi, Gi) * s40;
  const float irg = rsqrtf(gg), rg = gg * irg;
  const float rab = rsqrtf(A2 * B2);
  const float cs = dot3(A, B) * rab;
  const float sn = -rg * triplei(Fi, Bi, -60) * rab;
  const float K = ff.dih_k[t], dd = ff.dih_d[t];
  const float mdE = K * dd * sn;  // -dE/dphi = K d sin phi
  const float fg = (float)doti(Fi, Gi) * s40, hg = (float)doti(Hi, Gi) * s40;
  const float ia2 = __frcp_rn(A2), ib2 = __frcp_rn(B2);
  // dphi/dr_A = -|G|/A^2 A ; dphi/dr_D = |G|/B^2 B
  // dphi/dr_B = (|G|/A^2 + F.G/(A^2|G|)) A - H.G/(B^2|G|) B
  // dphi/dr_C = -F.G/(A^2|G|) A + (H.G/(B^2|G|) - |G|/B^2) B
  o.Fa = scale(mdE, scale(-rg * ia2, A));
  o.Fd = scale(mdE, scale(rg * ib2, B));
  o.Fb = scale(mdE, axpy(-hg * ib2 * irg, B, scale(rg * ia2 + fg * ia2 * irg, A)));
  o.Fc = scale(mdE, axpy(hg * ib2 * irg - rg * ib2, B, scale(-fg * ia2 * irg, A)));
  o.E = K * (1.0f + dd * cs);
  return o;
}

__global__ void k_bead(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_bead_flags(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_scan_cells(Dev d);
__global__ void k_scatter(Dev d);
__global__ void k_breakage(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_candidates(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_candidates_oct(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_candidates_tile(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_candidates_tile_oct(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_cand_overflow(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_match(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_edit(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_allbonds(Dev d);
__global__ void k_purge(Dev d);
__global__ void k_fill(Dev d);
__global__ void k_rebuild(Dev d, const RuleTab* __restrict__ rtp, int all_new);
__global__ void k_setup(Dev d);
__global__ void k_step_persistent(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_step_persistent_oct(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_set_args(CallArgs* a, const int4* pos, float4* force, double* ev, unsigned long long step,
                           int set_pos, int set_force, unsigned* bar_reset);

// the context's bond slots and geometry, for the MD harness (defined in api.cu)
const uint4* internal_slots(const dynbond_ctx* ctx, long long* n_beads, long long* box_q, int* n_replicas,
                            cudaStream_t* stream);

__global__ void k_bond_forces(Dev d, FF ff);
__global__ void k_angle_dihedral_forces(Dev d, FF ff);
__global__ void k_ev_out(Dev d);
__global__ void k_topo_hash(Dev d, unsigned long long* h);

}  // namespace dynbond
