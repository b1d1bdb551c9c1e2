// Bonded forces of the current topology: FP32 arithmetic per interaction
// from exact integer minimum-image displacements (scaled by 2^-20), FP64
// block reductions of the energy and the virial per replica.
//   bonds     each bead sums the harmonic force of the type IT stores for
//             each of its bonds (directional bonds, Sec. 2) -- no atomics;
//   angles    E = K (1 + cos theta) or K (theta - theta0)^2 (per type),
//             forces added with 16-byte reductions;
//   dihedrals E = K (1 + d cos phi) (Sec. 3), forces from the
//             Blondel-Karplus (J. Comput. Chem. 17, 1132 (1996)) derivatives
//             of phi, free of the sin(phi) = 0 singularity.
// Work items are (replica, tile) pairs; each warp adds its energy / virial
// partials to the replica's sums when its block moves to another replica and
// at its end.
#include "common.cuh"
#include "kernels.h"

namespace dynbond {

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

// Add the warp's 7 accumulators to replica r and clear them: a TwoSum
// butterfly over the lanes (every lane ends with the warp totals as float
// pairs), then lane k adds component k with one FP64 atomic to one of
// EV_COPIES striped copies (so the atomics of a launch do not all meet at
// the same seven addresses).  No block barrier: a block whose consecutive
// tiles belong to different replicas flushes at every change.  Every lane
// of the warp must call it.
__device__ __forceinline__ void flush_ev(const Dev& d, EV& acc, int r) {
  const int lane = threadIdx.x & 31;
  double mine = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    float h = acc.hi[k], l = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(FULL, h, o), l2 = __shfl_xor_sync(FULL, l, o);
      float s2, e;
      two_sum(h, h2, s2, e);
      h = s2;
      l = __fadd_rn(__fadd_rn(l, l2), e);
    }
    if (lane == k) mine = (double)h + (double)l;
    acc.hi[k] = 0.f;
  }
  const long long copy = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % EV_COPIES;
  if (lane < 7 && mine != 0.0) atomicAdd(&d.ev_acc[((long long)r * EV_COPIES + copy) * 7 + lane], mine);
}

// The work items of block b of G under the chunked-strided order: chunk j
// holds items (j G + b) 2^cs .. (j G + b) 2^cs + 2^cs - 1.  cs = 0 is the
// plain strided order (at any time the grid works on neighbouring items);
// with several replicas, cs > 0 keeps a block's consecutive items in one
// replica, so its energy / virial partials are flushed about once per chunk
// instead of at every item.
struct ItemOrder {
  int b, G, cs;
  __device__ int item(int k) const { return (((k >> cs) * G + b) << cs) + (k & ((1 << cs) - 1)); }
  __device__ int count(int nitems) const {
    const int first = b << cs;
    if (nitems <= first) return 0;
    const int S = G << cs;
    const int J = (nitems - first + S - 1) / S;  // chunks that start below nitems
    const int last = (((J - 1) * G + b) << cs);
    return ((J - 1) << cs) + min(1 << cs, nitems - last);
  }
};
__device__ __forceinline__ ItemOrder item_order(const Dev& d) {
  return ItemOrder{(int)blockIdx.x, (int)gridDim.x, d.R > 1 ? 3 : 0};
}

// Bonds: each bead sums, over its occupied slots, the harmonic force of the
// type it stores for that bond (directional bonds, Sec. 2) and books half the
// energy; no atomics.  Software-pipelined per thread like the angle /
// dihedral launch: the slots of the tile after next and the positions (own
// and partners') of the next tile are in flight while the current tile is
// computed.
struct BondStage {
  uint4 slot[3][BF_PER_THREAD][BF_THREADS];
  int4 pos[2][BF_PER_THREAD][1 + SLOTS][BF_THREADS];
};
static_assert(sizeof(BondStage) == BF_SMEM_BYTES, "bond shared memory layout");

__global__ void __launch_bounds__(BF_THREADS) k_bond_forces(Dev d, FF ffp) {
  pdl_enter();
  if (aborted(d.err)) return;
  __shared__ FF s_ff;
  const FF& ff = ff_to_shared(ffp, s_ff);
  extern __shared__ __align__(16) unsigned char bf_smem[];
  BondStage& sm = *reinterpret_cast<BondStage*>(bf_smem);
  const int4* __restrict__ pos = d.args->pos;
  float4* __restrict__ force = d.args->force;
  const int R = d.R, nitems = d.tb_beads[R];
  const unsigned N = (unsigned)d.N;
  const int tid = threadIdx.x;
  // work items in the chunked-strided order: at any time the grid works on
  // neighbouring tiles (shared partner positions stay in L2); each tile's
  // replica is looked up once, when its slots are issued
  const ItemOrder order = item_order(d);
  const int ntiles = order.count(nitems);
  struct Tile {
    long long beg = 0, end = 0;
    int r = 0, L = 0;
  };
  // the block's tiles are looked up before the pipeline starts, a warp per
  // tile (the lookups are independent), so no tile waits on a lookup
  __shared__ int4 s_tiles[FORCE_TILE_TABLE];
  const int nlook = min(ntiles, FORCE_TILE_TABLE);
  for (int k = tid >> 5; k < nlook; k += BF_THREADS >> 5) {
    const int it = order.item(k);
    const int r = find_seg_warp(d.tb_beads, R, it);
    if ((tid & 31) == 0) {
      const long long beg = d.off[r] + (long long)(it - d.tb_beads[r]) * BEAD_TILE;
      s_tiles[k] = make_int4(r, (int)beg, (int)min(beg + BEAD_TILE, d.off[r + 1]), (int)d.box[r]);
    }
  }
  __syncthreads();
  auto tile = [&](int k) {
    Tile t;
    if (k >= ntiles) return t;
    if (k < FORCE_TILE_TABLE) {
      const int4 e = s_tiles[k];
      t.r = e.x;
      t.beg = e.y;
      t.end = e.z;
      t.L = e.w;
      return t;
    }
    const int it = order.item(k);
    t.r = find_seg_warp(d.tb_beads, R, it);
    t.beg = d.off[t.r] + (long long)(it - d.tb_beads[t.r]) * BEAD_TILE;
    t.end = min(t.beg + BEAD_TILE, d.off[t.r + 1]);
    t.L = (int)d.box[t.r];
    return t;
  };
  auto issue_slots = [&](const Tile& t, int k) {
#pragma unroll
    for (int u = 0; u < BF_PER_THREAD; ++u) {
      const long long i = t.beg + tid + u * BF_THREADS;
      cp_async16(&sm.slot[k % 3][u][tid], i < t.end ? (const void*)(d.slots + i) : (const void*)d.slots, i < t.end);
    }
    cp_async_commit();
  };
  auto issue_pos = [&](const Tile& t, int k) {
#pragma unroll
    for (int u = 0; u < BF_PER_THREAD; ++u) {
      const long long i = t.beg + tid + u * BF_THREADS;
      const bool ok = i < t.end;
      const uint4 sl = sm.slot[k % 3][u][tid];
      cp_async16(&sm.pos[k & 1][u][0][tid], pos + (ok ? i : 0), ok);
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const unsigned v = s_get(sl, q);
        const bool has = ok && v && (unsigned)s_partner(v) < N;
        cp_async16(&sm.pos[k & 1][u][1 + q][tid], pos + (has ? s_partner(v) : 0), has);
      }
    }
    cp_async_commit();
  };
  EV acc;
  int racc = -1;
  // commit order: S0 S1 P0 | S2 P1 | S3 P2 ...; wait_group 2 leaves the two
  // newest groups in flight.  t0, t1, t2: tiles k, k + 1, k + 2.
  Tile t0 = tile(0), t1 = tile(1);
  issue_slots(t0, 0);
  issue_slots(t1, 1);
  cp_async_wait<1>();
  issue_pos(t0, 0);
  for (int k = 0; k < ntiles; ++k) {
    const Tile t2 = tile(k + 2);
    issue_slots(t2, k + 2);  // past the last tile: an empty group
    cp_async_wait<2>();      // slots of tile k + 1 have landed
    issue_pos(t1, k + 1);
    cp_async_wait<2>();      // positions of tile k have landed
    const long long beg = t0.beg, end = t0.end;
    const int r = t0.r, L = t0.L;
    t0 = t1;
    t1 = t2;
    if (r != racc) {
      if (racc >= 0) flush_ev(d, acc, racc);
      racc = r;
    }
    float e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < BF_PER_THREAD; ++u) {
      const long long i = beg + tid + u * BF_THREADS;
      if (i >= end) continue;
      const uint4 sl = sm.slot[k % 3][u][tid];
      const int4 p = sm.pos[k & 1][u][0][tid];
      float3 f = make_float3(0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const unsigned v = s_get(sl, q);
        if (!v) continue;
        if ((unsigned)s_partner(v) >= N) {
          atomicOr(d.err, ERR_INTERNAL);
          continue;
        }
        const BondHalf h = bond_half_force(ff, s_type(v), reli(p, sm.pos[k & 1][u][1 + q][tid], L));
        const float3 rij = h.rij, fq = h.f;
        f = make_float3(f.x + fq.x, f.y + fq.y, f.z + fq.z);
        e += h.E;
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
    for (int c = 0; c < 6; ++c) acc.add(c + 1, 0.5f * w[c]);
  }
  cp_async_wait<0>();
  if (racc >= 0) flush_ev(d, acc, racc);
}

__device__ __forceinline__ void add_force(float4* f, int i, float3 v) {
  red_add_f4(f, i, v.x, v.y, v.z);
}

// One angle (angle_term_forces); F_B = -(F_A + F_C).
__device__ __forceinline__ void angle_term(float4* force, const int4& a, const int4& pa, const int4& pb,
                                           const int4& pc, int L, const FF& ff, float& e, float* w) {
  const AngleTerm o = angle_term_forces(ff, a.w, pa, pb, pc, L);
  const float3 Fb = make_float3(-o.Fa.x - o.Fc.x, -o.Fa.y - o.Fc.y, -o.Fa.z - o.Fc.z);
  add_force(force, a.x, o.Fa);
  add_force(force, a.y, Fb);
  add_force(force, a.z, o.Fc);
  e += o.E;
  w[0] += o.ra.x * o.Fa.x + o.rc.x * o.Fc.x;
  w[1] += o.ra.y * o.Fa.y + o.rc.y * o.Fc.y;
  w[2] += o.ra.z * o.Fa.z + o.rc.z * o.Fc.z;
  w[3] += o.ra.x * o.Fa.y + o.rc.x * o.Fc.y;
  w[4] += o.ra.x * o.Fa.z + o.rc.x * o.Fc.z;
  w[5] += o.ra.y * o.Fa.z + o.rc.y * o.Fc.z;
}

// One dihedral (dihedral_term_forces); the record's fourth bead carries the
// type in its top 4 bits.
__device__ __forceinline__ void dihedral_term(float4* force, const int4& rec, const int4& P0, const int4& P1,
                                              const int4& P2, const int4& P3, int L, const FF& ff, float& e,
                                              float* w) {
  const int id = rec.w & 0x0FFFFFFF, t = (int)((unsigned)rec.w >> 28);
  const DihedralTerm o = dihedral_term_forces(ff, t, P0, P1, P2, P3, L);
  add_force(force, rec.x, o.Fa);
  add_force(force, rec.y, o.Fb);
  add_force(force, rec.z, o.Fc);
  add_force(force, id, o.Fd);
  e += o.E;
  // virial relative to B: r_A - r_B = F, r_C - r_B = -G, r_D - r_B = H - G
  const float3 F = o.F, mg = make_float3(-o.G.x, -o.G.y, -o.G.z);
  const float3 hm = make_float3(o.H.x - o.G.x, o.H.y - o.G.y, o.H.z - o.G.z);
  w[0] += F.x * o.Fa.x + mg.x * o.Fc.x + hm.x * o.Fd.x;
  w[1] += F.y * o.Fa.y + mg.y * o.Fc.y + hm.y * o.Fd.y;
  w[2] += F.z * o.Fa.z + mg.z * o.Fc.z + hm.z * o.Fd.z;
  w[3] += F.x * o.Fa.y + mg.x * o.Fc.y + hm.x * o.Fd.y;
  w[4] += F.x * o.Fa.z + mg.x * o.Fc.z + hm.x * o.Fd.z;
  w[5] += F.y * o.Fa.z + mg.y * o.Fc.z + hm.y * o.Fd.z;
}

// A work item of the angle / dihedral launch: tiles [0, tb_fang[R]) of the
// angle lists, then the dihedral tiles.
struct AdTile {
  bool valid = false, dih = false;
  int r = 0, beg = 0, end = 0, L = 0;
  const int4* recs = nullptr;
};
__device__ __forceinline__ AdTile ad_tile(const Dev& d, int it, int na_items, int nitems) {
  AdTile t;
  if (it >= nitems) return t;
  t.valid = true;
  t.dih = it >= na_items;
  const int* tb = t.dih ? d.tb_fdih : d.tb_fang;
  const int t0 = t.dih ? it - na_items : it;
  t.r = find_seg_warp(tb, d.R, t0);
  t.recs = t.dih ? d.dih + 18 * d.off[t.r] : d.ang + 6 * d.off[t.r];
  t.beg = (t0 - tb[t.r]) * FORCE_TILE;
  t.end = min(t.beg + FORCE_TILE, (t.dih ? d.n_dih : d.n_ang)[t.r]);
  t.L = (int)d.box[t.r];
  return t;
}

// Angles and dihedrals in one launch, software-pipelined per thread: the
// records of the tile after next and the bead positions of the next tile are
// in flight (cp.async into this thread's own shared-memory slots) while the
// current tile is computed, so the dependent record -> position loads of a
// tile overlap the arithmetic of the previous one.  Forces are added with
// 16-byte reductions.  Each thread reads back only what it copied itself, so
// no block barrier is needed between the stages.
struct AdStage {
  int4 rec[3][AD_PER_THREAD][AD_THREADS];     // records, three tiles
  int4 pos[2][AD_PER_THREAD][4][AD_THREADS];  // gathered positions, two tiles
};

static_assert(sizeof(AdStage) == AD_SMEM_BYTES, "angle / dihedral shared memory layout");

__global__ void __launch_bounds__(AD_THREADS) k_angle_dihedral_forces(Dev d, FF ffp) {
  pdl_enter();
  if (aborted(d.err)) return;
  __shared__ FF s_ff;
  const FF& ff = ff_to_shared(ffp, s_ff);
  extern __shared__ __align__(16) unsigned char ad_smem[];
  AdStage& sm = *reinterpret_cast<AdStage*>(ad_smem);
  const int4* __restrict__ pos = d.args->pos;
  float4* force = d.args->force;
  const int na_items = d.tb_fang[d.R], nitems = na_items + d.tb_fdih[d.R];
  const unsigned N = (unsigned)d.N;
  const int tid = threadIdx.x;
  // work items in the chunked-strided order (neighbouring records in flight
  // together); each tile is looked up once, when its records are issued
  const ItemOrder order = item_order(d);
  const int ntiles = order.count(nitems);
  // the block's tiles looked up first, a warp per tile (independent lookups)
  __shared__ AdTile s_tiles[FORCE_TILE_TABLE];
  const int nlook = min(ntiles, FORCE_TILE_TABLE);
  for (int k = tid >> 5; k < nlook; k += AD_THREADS >> 5) {
    const AdTile t = ad_tile(d, order.item(k), na_items, nitems);
    if ((tid & 31) == 0) s_tiles[k] = t;
  }
  __syncthreads();
  auto tile = [&](int k) {
    if (k < nlook) return s_tiles[k];
    return ad_tile(d, k < ntiles ? order.item(k) : nitems, na_items, nitems);
  };
  auto issue_rec = [&](const AdTile& t, int k) {
#pragma unroll
    for (int u = 0; u < AD_PER_THREAD; ++u) {
      const int q = t.beg + tid + u * AD_THREADS;
      const bool ok = t.valid && q < t.end;
      cp_async16(&sm.rec[k % 3][u][tid], ok ? (const void*)(t.recs + q) : (const void*)pos, ok);
    }
    cp_async_commit();
  };
  auto issue_pos = [&](const AdTile& t, int k) {
#pragma unroll
    for (int u = 0; u < AD_PER_THREAD; ++u) {
      const int q = t.beg + tid + u * AD_THREADS;
      const int4 a = sm.rec[k % 3][u][tid];
      const int b3 = t.dih ? (a.w & 0x0FFFFFFF) : a.z;
      bool ok = t.valid && q < t.end;
      const bool inb = (unsigned)a.x < N && (unsigned)a.y < N && (unsigned)a.z < N && (unsigned)b3 < N;
      if (ok && !inb) atomicOr(d.err, ERR_INTERNAL);
      ok = ok && inb;
      cp_async16(&sm.pos[k & 1][u][0][tid], pos + (ok ? a.x : 0), ok);
      cp_async16(&sm.pos[k & 1][u][1][tid], pos + (ok ? a.y : 0), ok);
      cp_async16(&sm.pos[k & 1][u][2][tid], pos + (ok ? a.z : 0), ok);
      cp_async16(&sm.pos[k & 1][u][3][tid], pos + (ok ? b3 : 0), ok && t.dih);
    }
    cp_async_commit();
  };
  EV acc;
  int racc = -1;
  // commit order: R0 R1 P0 | R2 P1 | R3 P2 ...; wait_group 2 leaves the two
  // newest groups in flight.  t0, t1: tiles k, k + 1.
  AdTile t0 = tile(0), t1 = tile(1);
  issue_rec(t0, 0);
  issue_rec(t1, 1);
  cp_async_wait<1>();
  issue_pos(t0, 0);
  for (int k = 0; k < ntiles; ++k) {
    const AdTile t2 = tile(k + 2);
    issue_rec(t2, k + 2);  // past the last tile: an empty group
    cp_async_wait<2>();    // records of tile k + 1 have landed
    issue_pos(t1, k + 1);
    cp_async_wait<2>();    // positions of tile k have landed
    const AdTile t = t0;
    t0 = t1;
    t1 = t2;
    if (t.r != racc) {
      if (racc >= 0) flush_ev(d, acc, racc);
      racc = t.r;
    }
    const int L = t.L;
    float e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < AD_PER_THREAD; ++u) {
      const int q = t.beg + tid + u * AD_THREADS;
      if (q >= t.end) continue;
      const int4 a = sm.rec[k % 3][u][tid];
      const int b3 = t.dih ? (a.w & 0x0FFFFFFF) : a.z;
      if ((unsigned)a.x >= N || (unsigned)a.y >= N || (unsigned)a.z >= N || (unsigned)b3 >= N) continue;
      const int4 P0 = sm.pos[k & 1][u][0][tid], P1 = sm.pos[k & 1][u][1][tid], P2 = sm.pos[k & 1][u][2][tid];
      if (t.dih) dihedral_term(force, a, P0, P1, P2, sm.pos[k & 1][u][3][tid], L, ff, e, w);
      else angle_term(force, a, P0, P1, P2, L, ff, e, w);
    }
    acc.add(0, e);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc.add(c + 1, w[c]);
  }
  cp_async_wait<0>();
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
