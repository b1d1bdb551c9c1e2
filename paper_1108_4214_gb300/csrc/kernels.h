// Kernel declarations and tile sizes shared by the kernel translation units
// and the host context.
#pragma once

#include "common.cuh"

namespace dynbond {

constexpr int PURGE_TILE = 1024;   // 256 threads x 4 records (small tiles balance the blocks)
constexpr int PURGE_PER_THREAD = 4;
constexpr int FILL_TILE = 256;     // hole / tail items per k_fill work item, one per thread
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

// bonded force-field tables in FP32 (kernel parameter space)
struct FF {
  float bond_k[16], bond_r0[16], angle_k[16], dih_k[16], dih_d[16];
  float angle_pt0[16];  // pi - theta0 of the harmonic angle types
  unsigned angle_harm;  // bit t: angle type t is harmonic in theta
};

// Device copy of a force field (FP32 parameters); false for an unknown angle style.
inline bool make_ff(const dynbond_forcefield& in, FF& out) {
  out = FF{};
  for (int t = 0; t < 16; ++t) {
    out.bond_k[t] = (float)in.bond_k[t];
    out.bond_r0[t] = (float)in.bond_r0[t];
    out.angle_k[t] = (float)in.angle_k[t];
    out.dih_k[t] = (float)in.dihedral_k[t];
    out.dih_d[t] = (float)in.dihedral_d[t];
    out.angle_pt0[t] = (float)(3.14159265358979323846 - in.angle_theta0[t]);
    if (in.angle_style[t] != 0 && in.angle_style[t] != 1) return false;
    if (in.angle_style[t] == 1) out.angle_harm |= 1u << t;
  }
  return true;
}

// Coefficient c and energy of an angle term of type t (centre bead B, ends A
// and C; cos theta = cs, inv = 1 / (|r_A - r_B| |r_C - r_B|) in sigma^-2):
// F_A = c dcos/dr_A, F_C = c dcos/dr_C.  Cosine: E = K (1 + cos), c = -K.
// Harmonic: E = K (theta - theta0)^2, c = 2 K (theta - theta0) / sin theta
// (d theta / d cos = -1 / sin), sin clamped below at 1e-3.  For the harmonic
// form pi - theta = atan2(|u x v|, -u.v) is taken from the exact integer
// cross and dot products of the displacements u, v, so nearly straight
// angles keep FP32 relative accuracy.
__device__ __forceinline__ float angle_coef(const FF& ff, int t, const int4& pa, const int4& pb, const int4& pc, int L,
                                            float cs, float inv, float* E) {
  const float K = ff.angle_k[t];
  if (!((ff.angle_harm >> t) & 1u)) {
    *E = K * (1.0f + cs);
    return -K;
  }
  const long long ux = wrap_dx(pa.x - pb.x, L), uy = wrap_dx(pa.y - pb.y, L), uz = wrap_dx(pa.z - pb.z, L);
  const long long vx = wrap_dx(pc.x - pb.x, L), vy = wrap_dx(pc.y - pb.y, L), vz = wrap_dx(pc.z - pb.z, L);
  const float cx = (float)(uy * vz - uz * vy), cy = (float)(uz * vx - ux * vz), cz = (float)(ux * vy - uy * vx);
  const float sr = sqrtf(cx * cx + cy * cy + cz * cz);          // |u x v|, units^2
  const float pth = atan2f(sr, -(float)(ux * vx + uy * vy + uz * vz));  // pi - theta
  const float dth = ff.angle_pt0[t] - pth;                         // theta - theta0
  const float s = fmaxf(sr * (1.0f / 1099511627776.0f) * inv, 1e-3f);  // sin theta (units^2 -> sigma^2)
  *E = K * dth * dth;
  return 2.0f * K * dth / s;
}

__global__ void k_bead(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_bead_flags(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_scan_cells(Dev d);
__global__ void k_scatter(Dev d, const RuleTab* __restrict__ rtp, int scatter_blocks);
__global__ void k_candidates(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_candidates_oct(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_cand_overflow(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_match(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_edit(Dev d, const RuleTab* __restrict__ rtp);
__global__ void k_allbonds(Dev d);
__global__ void k_purge(Dev d);
__global__ void k_fill(Dev d);
__global__ void k_rebuild(Dev d, const RuleTab* __restrict__ rtp, int all_new);
__global__ void k_setup(Dev d);
__global__ void k_set_args(CallArgs* a, const int4* pos, float4* force, double* ev, unsigned long long step,
                           int set_pos, int set_force);

// the context's bond slots and geometry, for the MD harness (defined in api.cu)
const uint4* internal_slots(const dynbond_ctx* ctx, long long* n_beads, long long* box_q, int* n_replicas,
                            cudaStream_t* stream);

__global__ void k_bond_forces(Dev d, FF ff);
__global__ void k_angle_dihedral_forces(Dev d, FF ff);
__global__ void k_ev_out(Dev d);
__global__ void k_topo_hash(Dev d, unsigned long long* h);

}  // namespace dynbond
