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
};

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
