// Device-side building blocks of the dynamic-bonding library: the context
// view passed to every kernel, the rule table, exact integer geometry, the
// Philox4x32-10 generator, bitmaps, warp / block scans, a bounded single-pass
// look-back for ordered compaction, and a bounded grid barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dynbond.h"

namespace dynbond {

constexpr int SLOTS = DYNBOND_SLOTS;
constexpr int MAXR = DYNBOND_MAX_RULES;
constexpr int MAXC = DYNBOND_MAX_CANDIDATES;
constexpr int CAND_FAST = 8;  // candidate slots of each sorted entry (longer lists use the pool)
constexpr int MAX_ROUNDS = DYNBOND_MAX_ROUNDS;
constexpr int NSTAT = 17;
constexpr unsigned FULL = 0xffffffffu;

// bits of the sticky device error word
enum : unsigned {
  ERR_POS = 1u,        // a position outside [0, box)
  ERR_CAND_CAP = 4u,   // candidate buffer exhausted
  ERR_SLOTS = 8u,      // a bead would exceed SLOTS bonds (internal)
  ERR_TIMEOUT = 16u,   // a bounded wait gave up
  ERR_ROUNDS = 32u,    // matching needed more than MAX_ROUNDS rounds
  ERR_INTERNAL = 64u,  // an internal consistency check failed (record out of range)
};

enum StatIdx {
  ST_CANDIDATES, ST_CREATE_MATCHED, ST_FORMED, ST_BREAK_CANDIDATES, ST_BREAK_MATCHED, ST_BROKEN, ST_KILLED,
  ST_CONVERTED, ST_ANG_REMOVED, ST_ANG_ADDED, ST_DIH_REMOVED, ST_DIH_ADDED, ST_NBONDS, ST_NANGLES,
  ST_NDIHEDRALS, ST_CREATE_ROUNDS, ST_BREAK_ROUNDS
};

enum { TAG_FORM = 1u, TAG_BREAK = 2u };

// Rule table, passed by value (kernel parameter space) so every lane reads it
// through the constant cache.
struct RuleTab {
  int n;
  int kind[MAXR];
  int type[MAXR];
  int type2[MAXR];
  int maxn[MAXR];
  uint32_t bead[MAXR][4];
  uint32_t bond[MAXR][3];
  long long r2[MAXR];
  uint32_t pair_rules[16][16];  // creation rules whose bead masks admit (ti, tj) in some orientation
  uint32_t role_rules[16];      // creation rules naming bead type t in either role
  long long r2max;              // largest creation threshold
  uint32_t breakish;            // bond types named by breakbond / convertbond / killbond
  uint32_t reactive;
  int n_maxbond, n_angle, n_dihedral;
  int maxbond_idx[MAXR], angle_idx[MAXR], dihedral_idx[MAXR];
  int pc13, pc14, max_rounds, prob_mode;
  uint32_t key0, key1;
  // precompiled lookups
  uint32_t role_store[16];      // bond types a bead of type t could store under some creation rule
  int bk_start[17];             // breakbond / convertbond / killbond rules of bond type t:
  int bk_list[MAXR];            //   bk_list[bk_start[t] .. bk_start[t+1]) in list order
  // cell-list classes: creation-capable bead types are binned apart, and a
  // bead searches only the classes of the types it can pair with
  int n_cls;
  int cls_of[16];               // class of bead type t, -1 if never binned
  uint32_t cls_mask[16];        // classes holding partner types of bead type t
};

// Arguments that change from call to call, read from device memory so that a
// captured CUDA graph can be replayed with new positions and call index.
struct CallArgs {
  const int4* pos;
  float4* force;
  double* ev;
  unsigned long long step;
};

struct Counters {
  int n_sorted;
  int cand_used;
  int n_nbl;
  int n_ovf;
  int ticket[8];
  int done[4];                 // blocks finished (last-block hand-off)
  unsigned bar[2];
  int rounds_done;
  int round_matched[MAX_ROUNDS];
  int round_live[MAX_ROUNDS];  // entries carried into the next round
};

// Device view of a context.  Arrays marked [N] are indexed by global bead id.
struct Dev {
  long long N;
  int R;
  int spin_limit;
  const long long* off;        // [R+1]
  const long long* box;        // [R]
  const int* nc;               // [R] cells along x and y
  const int* ncz;              // [R] cells along z
  // [2R] per replica: (L, nc, nz, hz) and (nc / L, nz / L as float bits, cell_base, 0); hz = ceil(reach nz / L),
  // the z cells a reach interval can extend beyond its bead's cell on either side
  const int4* geo;
  long long reach;              // smallest integer >= the largest creation distance (quantised units)
  const long long* cell_base;  // [R+1]
  long long n_cells;            // cells of one class (all replicas)
  const int4* ctile;           // [n_ctile] work items of the staged candidate search
  int n_ctile;
  long long n_keys;             // n_cls * n_cells binned keys
  const int* rep;              // [N]
  const unsigned char* type;   // [N]
  const unsigned* stream;      // [R]
  const unsigned long long* T_form;   // [R*MAXR]
  const unsigned long long* T_break;  // [R*MAXR]
  CallArgs* args;
  // topology
  uint4* slots;                // [N] (partner << 4 | stored type), 0 = empty
  int4* ang;                   // replica r owns [6*off[r], 6*off[r+1])
  int4* dih;                   // replica r owns [18*off[r], 18*off[r+1]); w = d | type << 28
  int* n_ang;                  // [R]
  int* n_dih;                  // [R]
  int* m_ang;                  // [R] records removed in this call
  int* m_dih;                  // [R]
  int* added_ang;              // [R] records added in this call
  int* added_dih;              // [R]
  int* fillc;                  // [4R] hole / mover arrival counters of k_fill
  int* fill_items;             // [R]
  int* rm_ang;                 // [6N] positions of removed records (replica regions as ang)
  int* rm_dih;                 // [18N]
  int* pr_ang;                 // [6N] rendezvous words of k_fill
  int* pr_dih;                 // [18N]
  long long* n_bonds;          // [R]
  // per-call scratch
  Counters* cnt;
  unsigned* err;               // sticky error word
  int* cell_start;             // [-1, n_keys], key = class * n_cells + cell: counts, then starts
                               // (exclusive scan), then ends after the scatter; cell_start[-1] = 0
  int2* binned;                // [N] per segment of BIN_SEG beads, its binned beads (bead, cell key) first
  int* binned_n;               // [N / BIN_SEG] binned beads per segment
  int4* sorted;                // [N] (x, y, z, gid << 4 | type)
  int4* cand;                  // (partner, rule | mytype << 8, d2 lo, d2 hi): CAND_FAST slots per
                               // sorted entry, then a pool of cand_pool entries for longer lists
  long long cand_fixed;        // N * CAND_FAST
  long long cand_pool;
  int* cand_start;             // [N]
  int* cand_len;               // [N]
  int* ovf;                    // [N] sorted indices of beads with more than MAXC candidates
  int4* brk;                   // [N*4] (partner, rule, key lo, key hi), key = -d2
  unsigned char* brk_len;      // [N]
  unsigned char* killmask;     // [N]
  unsigned* bm_ca;             // [W] creation-active beads
  unsigned* bm_ba;             // [W] breakage/kill-active beads
  unsigned* bm_bn;             // [W] beads nominating a breakage partner
  unsigned* bm_bk;             // [W] beads holding a bond of a type named by a breakage rule (kept current)
  unsigned* bm_elig;           // [W] beads that can form a bond (creation_eligible; kept current)
  unsigned* bm_dirty;          // [W] beads that lost or retyped a bond
  unsigned* bm_dirtyc;         // [Wc] coarse: bit b set if a bead of words [b << dc_shift, (b + 1) << dc_shift) is dirty
  long long Wc;                // coarse words (at most PURGE_COARSE_WORDS)
  int dc_shift;
  unsigned* bm_new;            // [W] beads with a formed or retyped bond
  int* live[2];                // [2*N] each: active (system << 31 | bead) entries between rounds
  long long* mate;             // [2*N] creation / breakage match: partner | round << 32, -1 = none
  int* nom;                    // [2*N]
  int* ptr;                    // [2*N]
  int* round_hit;              // [2*R]
  int4* rem;                   // [N] partners whose bond was removed or retyped
  int2* newp;                  // [N] formed partner, retyped partner
  int4* nbl;                   // new-bond list (u, v, replica, 0), u < v, unordered
  int* tb_ang;                 // [R+1] purge tile bases
  int* tb_dih;                 // [R+1]
  int* tb_fill;                // [R+1] k_fill tile bases
  int* tb_beads;               // [R+1] (static)
  int* tb_fang;                // [R+1] force tile bases of the final lists
  int* tb_fdih;                // [R+1]
  long long W;                 // bitmap words
  int* small;                  // per-call per-replica scratch, zeroed by k_setup
  long long small_words;
  unsigned long long* status_all;  // all look-back status words, zeroed by k_setup
  long long status_words;
  unsigned long long* st_scan; // look-back status words of the cell scan
  long long* stats;            // [R*NSTAT]
  double* ev_acc;              // [R * EV_COPIES * 7] striped energy / virial sums
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int s_partner(unsigned v) { return v ? (int)(v >> 4) : -1; }
__device__ __forceinline__ int s_type(unsigned v) { return (int)(v & 15u); }
__device__ __forceinline__ unsigned s_get(const uint4& s, int k) {
  return k == 0 ? s.x : k == 1 ? s.y : k == 2 ? s.z : s.w;
}
__device__ __forceinline__ void s_set(uint4& s, int k, unsigned v) {
  if (k == 0) s.x = v;
  else if (k == 1) s.y = v;
  else if (k == 2) s.z = v;
  else s.w = v;
}
__device__ __forceinline__ int s_deg(const uint4& s) { return (s.x != 0) + (s.y != 0) + (s.z != 0) + (s.w != 0); }
// type that the bead with slots s stores for its bond to q, or 0 if none
__device__ __forceinline__ int s_type_to(const uint4& s, int q) {
  unsigned want = (unsigned)q << 4;
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    unsigned v = s_get(s, k);
    if (v && (v & ~15u) == want) return s_type(v);
  }
  return 0;
}
__device__ __forceinline__ bool has_bit(uint32_t m, int t) { return (m >> t) & 1u; }

// minimum-image component of xi - xj for a box edge L (2 dx in (-L, L])
__device__ __forceinline__ int wrap_dx(int dx, int L) {
  int half_dn = L >> 1, half_up = (L >> 1) + (L & 1);
  if (dx > half_dn) dx -= L;
  else if (dx <= -half_up) dx += L;
  return dx;
}
// Cell of coordinate x in [0, L) on an axis of nc cells: floor(x nc / L)
// exactly.  The FP32 estimate is within one of the true quotient (relative
// error below 2^-22 on a value below 1024), and one integer-exact comparison
// step corrects it.
__device__ __forceinline__ int cell_of(int x, int nc, int L, float nc_over_L) {
  int q = min(max((int)((float)x * nc_over_L), 0), nc - 1);
  const long long p = (long long)x * nc;
  if ((long long)q * L > p) --q;
  else if ((long long)(q + 1) * L <= p) ++q;
  return q;
}

__device__ __forceinline__ long long dist2(const int4& a, const int4& b, int L) {
  long long x = wrap_dx(a.x - b.x, L), y = wrap_dx(a.y - b.y, L), z = wrap_dx(a.z - b.z, L);
  return x * x + y * y + z * z;
}

// Largest r in [0, R) with base[r] <= x (base non-decreasing, base[0] <= x),
// for a warp whose 32 lanes all ask for the same x (every lane must call
// it): each round probes 32 evenly spaced entries of [lo, hi] at once and
// keeps the part between the last probe at or below x and the next one, so
// R segments take ceil(log32 R) dependent loads (two for 512 replicas)
// instead of log2 R.
__device__ __forceinline__ int find_seg_warp(const int* base, int R, int x) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    const int step = (hi - lo + 31) >> 5;  // 32 probes cover (lo, hi]
    const int idx = lo + (lane + 1) * step;
    const bool le = idx <= hi && base[idx] <= x;
    lo += __popc(__ballot_sync(FULL, le)) * step;  // the true probes are a prefix of the lanes
    hi = min(hi, lo + step - 1);
  }
  return lo;
}

__device__ __forceinline__ int ld_cg(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Once any device error is recorded (a bounded wait gave up, a capacity or
// consistency check failed, a bad position), every later kernel of the call
// returns at once, so no kernel consumes half-built data.
// Programmatic dependent launch.  Kernels of a call are launched with
// programmatic stream serialization, so the next kernel's blocks may be
// scheduled while this one drains.  Every kernel first waits for its
// predecessor to complete and flush (griddepcontrol.wait returns at once for
// a kernel launched without the attribute), then lets its own successor be
// scheduled; the successor's blocks only take resources this kernel's
// blocks leave free, and they wait in turn before touching memory, so each
// kernel still sees everything all earlier kernels wrote.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// f[i] += (x, y, z, 0) as one 16-byte reduction at L2 (no value returned, so
// the issuing warp neither waits for it nor keeps registers for a result)
__device__ __forceinline__ void red_add_f4(float4* f, long long i, float x, float y, float z) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(f + i), "f"(x), "f"(y), "f"(z), "f"(0.f)
               : "memory");
}

// 16-byte asynchronous copy global -> shared (cp.async; zero-filled when
// !pred, the source address is then not read)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Replica of bead i: the common single-system case needs no load, so later
// loads that depend on the replica (box, offsets, streams) are not delayed.
__device__ __forceinline__ int rep_of(const Dev& d, long long i) { return d.R == 1 ? 0 : d.rep[i]; }

// a match of the matching rounds: the partner and the round it was made in
__device__ __forceinline__ long long mate_pack(int round, int j) { return ((long long)round << 32) | (unsigned)j; }
__device__ __forceinline__ int mate_partner(long long m) { return m < 0 ? -1 : (int)(unsigned)m; }

__device__ __forceinline__ bool aborted(const unsigned* err) { return *(const volatile unsigned*)err != 0u; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round the counter
// words 0 and 2 are multiplied by the two round multipliers, high halves are
// xored with the other counter words and the round key, and the key advances
// by the two Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    unsigned h0 = __umulhi(m0, c.x), l0 = m0 * c.x;
    unsigned h1 = __umulhi(m1, c.z), l1 = m1 * c.z;
    c = make_uint4(h1 ^ c.y ^ k.x, l1, h0 ^ c.w ^ k.y, l0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// One Bernoulli trial of the pair (a, b), a < b, global ids.
__device__ __forceinline__ bool trial(const Dev& d, const RuleTab& rt, int a, int b, int r, unsigned tag,
                                      unsigned long long T) {
  long long o = d.off[r];
  uint4 c = make_uint4((unsigned)(a - o), (unsigned)(b - o), (unsigned)d.args->step,
                       (tag << 24) | (d.stream[r] & 0xFFFFFFu));
  uint4 u = philox4x32_10(c, make_uint2(rt.key0, rt.key1));
  if (rt.prob_mode == 0) return (unsigned long long)u.x < T;
  return (unsigned long long)u.x + (unsigned long long)u.y < 2ull * T;
}

// ---------------------------------------------------------------------------
// rules
// ---------------------------------------------------------------------------

// May a bead of bead type bt with slots s receive one more bond stored as nt?
__device__ __forceinline__ bool maxbond_ok(const RuleTab& rt, int bt, const uint4& s, int nt) {
  if (s_deg(s) >= SLOTS) return false;
  for (int m = 0; m < rt.n_maxbond; ++m) {
    int k = rt.maxbond_idx[m];
    if (!has_bit(rt.bead[k][0], bt) || !has_bit(rt.bond[k][0], nt)) continue;
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      unsigned v = s_get(s, q);
      cnt += (v != 0) && has_bit(rt.bond[k][0], s_type(v));
    }
    if (cnt >= rt.maxn[k]) return false;
  }
  return true;
}

// Can the bead take part in any creation pair (reactive, named by a creation
// rule in some role with room for the type it would store)?
// Does a reactive bead of type bt hold a bond of a type named by a breakage
// (break / convert / kill) rule?
__device__ __forceinline__ bool holds_breakable(const RuleTab& rt, int bt, const uint4& s) {
  if (!rt.breakish || !has_bit(rt.reactive, bt)) return false;
  bool b = false;
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    const unsigned v = s_get(s, q);
    b |= v && has_bit(rt.breakish, s_type(v));
  }
  return b;
}

__device__ __forceinline__ bool creation_eligible(const RuleTab& rt, int bt, const uint4& s) {
  if (!has_bit(rt.reactive, bt) || s_deg(s) >= SLOTS) return false;
  uint32_t m = rt.role_store[bt];
  while (m) {
    int t = __ffs(m) - 1;
    m &= m - 1;
    if (maxbond_ok(rt, bt, s, t)) return true;
  }
  return false;
}

// Last creation rule matching the pair (a < b): bead types, distance and
// maxbond at both ends; orientation a-first is tried first.  Returns the rule
// (or -1) and the types a and b would store.
__device__ __forceinline__ int creation_rule(const RuleTab& rt, int ta, int tb, const uint4& sa, const uint4& sb,
                                             long long d2, int* sta, int* stb) {
  uint32_t m = rt.pair_rules[ta][tb];
  while (m) {
    int k = 31 - __clz(m);
    m &= ~(1u << k);
    if (d2 > rt.r2[k]) continue;
    int t1 = rt.type[k], t2 = rt.kind[k] == DYNBOND_CREATEDIRBOND ? rt.type2[k] : rt.type[k];
    if (has_bit(rt.bead[k][0], ta) && has_bit(rt.bead[k][1], tb) && maxbond_ok(rt, ta, sa, t1) &&
        maxbond_ok(rt, tb, sb, t2)) {
      *sta = t1;
      *stb = t2;
      return k;
    }
    if (has_bit(rt.bead[k][0], tb) && has_bit(rt.bead[k][1], ta) && maxbond_ok(rt, tb, sb, t1) &&
        maxbond_ok(rt, ta, sa, t2)) {
      *sta = t2;
      *stb = t1;
      return k;
    }
  }
  return -1;
}

__device__ __forceinline__ int angle_type(const RuleTab& rt, int ta, int tb, int tc, int t_ba, int t_bc) {
  for (int q = 0; q < rt.n_angle; ++q) {
    int k = rt.angle_idx[q];
    const uint32_t* bm = rt.bead[k];
    bool fwd = has_bit(bm[0], ta) && has_bit(bm[1], tb) && has_bit(bm[2], tc) && has_bit(rt.bond[k][0], t_ba) &&
               has_bit(rt.bond[k][1], t_bc);
    bool rev = has_bit(bm[0], tc) && has_bit(bm[1], tb) && has_bit(bm[2], ta) && has_bit(rt.bond[k][0], t_bc) &&
               has_bit(rt.bond[k][1], t_ba);
    if (fwd || rev) return rt.type[k];
  }
  return 0;
}

// r = type B stores toward A, s = C toward B, sp = B toward C, t = C toward D
__device__ __forceinline__ int dihedral_type(const RuleTab& rt, int ta, int tb, int tc, int td, int r, int s, int sp,
                                             int t) {
  for (int q = 0; q < rt.n_dihedral; ++q) {
    int k = rt.dihedral_idx[q];
    const uint32_t* bm = rt.bead[k];
    const uint32_t* bd = rt.bond[k];
    bool fwd = has_bit(bm[0], ta) && has_bit(bm[1], tb) && has_bit(bm[2], tc) && has_bit(bm[3], td) &&
               has_bit(bd[0], r) && (has_bit(bd[1], s) || has_bit(bd[1], sp)) && has_bit(bd[2], t);
    bool rev = has_bit(bm[0], td) && has_bit(bm[1], tc) && has_bit(bm[2], tb) && has_bit(bm[3], ta) &&
               has_bit(bd[0], t) && (has_bit(bd[1], sp) || has_bit(bd[1], s)) && has_bit(bd[2], r);
    if (fwd || rev) return rt.type[k];
  }
  return 0;
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Exclusive block scan (blockDim.x a multiple of 32, <= 1024); returns the
// exclusive prefix of v and the block total in *total.  Uses `sh` (>= 33 T).
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* sh, T* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? sh[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < nw) sh[lane] = wi - w;
    if (lane == nw - 1) sh[32] = wi;
  }
  __syncthreads();
  T r = sh[wid] + inc - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// single-pass look-back, called by one full warp of the block.  Tiles are
// taken in ticket order, so every predecessor has started; each tile
// publishes its aggregate after reading its input and its inclusive prefix
// after the look-back.  status[t] = flag << 62 | value; flag 1 = aggregate,
// 2 = inclusive prefix.  The warp inspects 32 predecessors per poll.
// Returns (in every lane) the exclusive prefix within the segment starting at
// seg_first, or -1 after spin_limit unsuccessful polls (error bit set).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long lookback(unsigned long long* status, long long t, long long seg_first,
                                              unsigned long long agg, int spin_limit, unsigned* err) {
  const unsigned long long FA = 1ull << 62, FP = 2ull << 62, VM = (1ull << 62) - 1;
  const int lane = threadIdx.x & 31;
  if (t == seg_first) {
    if (lane == 0) st_release(status + t, FP | agg);
    return 0;
  }
  if (lane == 0) st_release(status + t, FA | agg);
  unsigned long long excl = 0;
  long long p = t - 1;
  int spins = 0;
  while (true) {
    long long idx = p - lane;
    unsigned long long s = idx >= seg_first ? ld_acquire(status + idx) : FP;
    unsigned long long f = s >> 62;
    unsigned inc = __ballot_sync(FULL, f == 2), zero = __ballot_sync(FULL, f == 0);
    unsigned need = inc ? ((inc & (0u - inc)) << 1) - 1 : FULL;  // lanes up to the first prefix
    if (zero & need) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        return -1;
      }
      if (spins > 4096) __nanosleep(32);  // predecessors are normally microseconds away: poll first
      continue;
    }
    unsigned long long v = ((need >> lane) & 1u) ? (s & VM) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    excl += __shfl_sync(FULL, v, 0);
    if (inc) break;
    p -= 32;
  }
  if (lane == 0) st_release(status + t, FP | (excl + agg));
  return (long long)excl;
}

// Add v (per lane) to statistic k of replica r with one atomic per replica
// present in the warp.  Every lane of the warp must call it.
__device__ __forceinline__ void stat_add_warp(long long* stats, int r, int k, unsigned v) {
  if (!__ballot_sync(FULL, v != 0)) return;
  unsigned grp = __match_any_sync(FULL, r);
  int lane = threadIdx.x & 31;
  if (grp == FULL) {
    unsigned sum = __reduce_add_sync(FULL, v);
    if (lane == 0) atomicAdd((unsigned long long*)&stats[(long long)r * NSTAT + k], (unsigned long long)sum);
  } else if (v) {
    atomicAdd((unsigned long long*)&stats[(long long)r * NSTAT + k], (unsigned long long)v);
  }
}

// Same for an int counter array indexed by replica.
__device__ __forceinline__ void count_add_warp(int* counts, int r, unsigned v) {
  if (!__ballot_sync(FULL, v != 0)) return;
  unsigned grp = __match_any_sync(FULL, r);
  int lane = threadIdx.x & 31;
  if (grp == FULL) {
    unsigned sum = __reduce_add_sync(FULL, v);
    if (lane == 0) atomicAdd(&counts[r], (int)sum);
  } else if (v) {
    atomicAdd(&counts[r], (int)v);
  }
}

// ---------------------------------------------------------------------------
// Block-aggregated counters.  Atomics on one address from every warp of a
// launch serialize in L2 (a few ns each, thousands per launch), so list
// appends and per-replica counts are combined per block first.
// ---------------------------------------------------------------------------

// Exclusive prefix of `want` over the block, then one atomicAdd on `counter`
// for the block total (none if it is 0); returns this thread's first slot.
// Every thread of the block must call it.
__device__ __forceinline__ int block_alloc(int* counter, int want) {
  __shared__ int s_off[32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int incl = warp_incl_scan(want);
  if (lane == 31) s_off[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = lane < nw ? s_off[lane] : 0;
    int inc = warp_incl_scan(v);
    if (lane < nw) s_off[lane] = inc - v;
    if (lane == 31) s_base = inc ? atomicAdd(counter, inc) : 0;
  }
  __syncthreads();
  const int at = s_base + s_off[wid] + incl - want;
  __syncthreads();
  return at;
}

// block_alloc for four counters at once: each thread takes one slot of
// counter[role] (role 0..3) or none (role < 0); the four block totals are
// added with independent atomics by four lanes, so the block waits for one
// round trip.  Returns this thread's slot.  Every thread of the block must
// call it.
__device__ __forceinline__ int block_alloc4(int* counter, int role) {
  __shared__ int s_cnt[32][4];
  __shared__ int s_base[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned bal[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) bal[q] = __ballot_sync(FULL, role == q);
  if (lane < 4) s_cnt[wid][lane] = __popc(lane == 0 ? bal[0] : lane == 1 ? bal[1] : lane == 2 ? bal[2] : bal[3]);
  __syncthreads();
  if (wid == 0 && lane < 4) {
    int run = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = s_cnt[w][lane];
      s_cnt[w][lane] = run;
      run += c;
    }
    s_base[lane] = run ? atomicAdd(counter + lane, run) : 0;
  }
  __syncthreads();
  int at = 0;
  if (role >= 0) {
    const unsigned b = role == 0 ? bal[0] : role == 1 ? bal[1] : role == 2 ? bal[2] : bal[3];
    at = s_base[role] + s_cnt[wid][role] + __popc(b & ((1u << lane) - 1u));
  }
  __syncthreads();
  return at;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Address of per-replica counter k: base[k] + r * stride[k].
template <int K>
struct CountTargets {
  long long* base[K];
  int stride[K];
  __device__ unsigned long long* at(int r, int k) const {
    return (unsigned long long*)(base[k] + (long long)r * stride[k]);
  }
};

// Per-thread partial sums of K per-replica counters.  A thread keeps the
// replica it last counted for and flushes with atomics when that changes
// (rare: threads walk beads in id order, replicas are contiguous in id);
// flush_block() adds the partials of the whole block with one atomic per
// counter when they all belong to one replica, else one per thread.
template <int K>
struct ReplicaCounts {
  int r = -1;
  long long v[K];
  __device__ ReplicaCounts() {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0;
  }
  __device__ void flush_thread(const CountTargets<K>& t) {
    if (r >= 0) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (v[k]) atomicAdd(t.at(r, k), (unsigned long long)v[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0;
  }
  __device__ void add(const CountTargets<K>& t, int rr, int k, long long x) {
    if (!x) return;
    if (rr != r) {
      flush_thread(t);
      r = rr;
    }
    v[k] += x;
  }
  // Barrier-free variant for kernels whose warps finish at different times:
  // begin_block() (every thread, once, before any end_warp) clears the shared
  // partials; end_warp() (every lane of a warp, once) adds the warp's partials
  // there, and the last warp of the block to finish adds them to the
  // counters.  Partials of a replica other than the block's first are added
  // directly.
  struct Shared {
    long long sum[K];
    int r, done;
  };
  __device__ static Shared& shared() {
    __shared__ Shared sh;
    return sh;
  }
  __device__ static void begin_block() {
    Shared& sh = shared();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) sh.sum[k] = 0;
      sh.r = -1;
      sh.done = 0;
    }
    __syncthreads();
  }
  __device__ void end_warp(const CountTargets<K>& t) {
    Shared& sh = shared();
    const int lane = threadIdx.x & 31;
    bool any = false;
#pragma unroll
    for (int k = 0; k < K; ++k) any |= v[k] != 0;
    const int rr = any ? r : -1;
    const unsigned have = __ballot_sync(FULL, any);
    const int wr = __shfl_sync(FULL, rr, have ? __ffs(have) - 1 : 0);
    // warp-uniform: every lane with partials counts for replica wr
    const bool uniform = __all_sync(FULL, !any || rr == wr) && have;
    bool local = false;  // this warp's partials go to the shared sums
    if (uniform) {
      int cur = 0;
      if (lane == 0) {
        cur = atomicCAS(&sh.r, -1, wr);
        cur = cur == -1 ? wr : cur;
      }
      local = __shfl_sync(FULL, cur, 0) == wr;
    }
    if (local) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const long long x = warp_sum64(v[k]);
        if (lane == 0 && x) atomicAdd((unsigned long long*)&sh.sum[k], (unsigned long long)x);
        v[k] = 0;
      }
    } else {
      flush_thread(t);
    }
    __threadfence_block();
    int last = 0;
    if (lane == 0) last = atomicAdd(&sh.done, 1) == (int)(blockDim.x >> 5) - 1;
    last = __shfl_sync(FULL, last, 0);
    if (last && lane < K) {
      const long long x = *(volatile long long*)&sh.sum[lane];
      const int br = *(volatile int*)&sh.r;
      if (x && br >= 0) atomicAdd(t.at(br, lane), (unsigned long long)x);
    }
  }
  // every thread of the block must call it
  __device__ void flush_block(const CountTargets<K>& t) {
    __shared__ int s_lo, s_hi;
    __shared__ long long s_sum[K];
    if (threadIdx.x == 0) {
      s_lo = 0x7FFFFFFF;
      s_hi = -1;
#pragma unroll
      for (int k = 0; k < K; ++k) s_sum[k] = 0;
    }
    __syncthreads();
    bool any = false;
#pragma unroll
    for (int k = 0; k < K; ++k) any |= v[k] != 0;
    if (any) {
      atomicMin(&s_lo, r);
      atomicMax(&s_hi, r);
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    if (hi >= 0 && lo == hi) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        long long x = warp_sum64(v[k]);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd((unsigned long long*)&s_sum[k], (unsigned long long)x);
        v[k] = 0;
      }
      __syncthreads();
      if (threadIdx.x < K && s_sum[threadIdx.x]) atomicAdd(t.at(lo, threadIdx.x), (unsigned long long)s_sum[threadIdx.x]);
    } else if (hi >= 0) {
      flush_thread(t);
    }
    __syncthreads();
  }
};

// Flag replica r (-1: none) in flags; one store per block when every thread
// of the block names the same replica.  Every thread of the block must call it.
__device__ __forceinline__ void block_flag(int* flags, int r) {
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = 0x7FFFFFFF;
    s_hi = -1;
  }
  __syncthreads();
  if (r >= 0) {
    atomicMin(&s_lo, r);
    atomicMax(&s_hi, r);
  }
  __syncthreads();
  const int lo = s_lo, hi = s_hi;
  if (hi >= 0) {
    if (lo == hi) {
      if (threadIdx.x == 0) flags[lo] = 1;
    } else if (r >= 0) {
      flags[r] = 1;
    }
  }
  __syncthreads();
}

// Visit the beads whose bit is set in bitmap a or b (words [0, W), bits of
// beads below N) over the chunks [c_begin, c_end) of 8 words.  Loops are
// block-uniform: each warp compacts one chunk and its lanes take the set
// bits 32 at a time; fn(valid, i, in_a, in_b) is called by every thread of
// the block the same number of times (valid = false for idle lanes), so fn
// may use block-wide collectives.
constexpr int CHUNK_WORDS = 8;

// position of the n-th (from 0) set bit of m; n < popc(m)
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    unsigned lo = m & ((1u << w) - 1u);
    int c = __popc(lo);
    if (n >= c) {
      n -= c;
      m >>= w;
      pos += w;
    } else {
      m = lo;
    }
  }
  return pos;
}

template <class F>
__device__ __forceinline__ void for_bits_block(const unsigned* a, const unsigned* b, long long W, long long N,
                                               long long c_begin, long long c_end, F&& fn) {
  __shared__ int s_rounds;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (long long c0 = c_begin; c0 < c_end; c0 += nwarps) {
    const long long ch = c0 + warp;
    const long long w0 = ch * CHUNK_WORDS;
    unsigned wa = 0, wb = 0;
    if (ch < c_end && lane < CHUNK_WORDS && w0 + lane < W) {
      const long long b0 = 32 * (w0 + lane);  // the last word may extend past N
      const unsigned vmask = b0 + 32 <= N ? FULL : (b0 >= N ? 0u : (1u << (N - b0)) - 1u);
      if (a) wa = a[w0 + lane] & vmask;
      if (b) wb = b[w0 + lane] & vmask;
    }
    const unsigned act = wa | wb;
    const int incl = warp_incl_scan(__popc(act));
    const int total = __shfl_sync(FULL, incl, 31);
    if (threadIdx.x == 0) s_rounds = 0;
    __syncthreads();
    if (lane == 0 && total) atomicMax(&s_rounds, (total + 31) >> 5);
    __syncthreads();
    const int rounds = s_rounds;
    __syncthreads();
    for (int rr = 0; rr < rounds; ++rr) {
      const int want = rr * 32 + lane;
      int k = 0;
#pragma unroll
      for (int q = 0; q < CHUNK_WORDS; ++q) k += __shfl_sync(FULL, incl, q) <= want;
      const int ks = k & (CHUNK_WORDS - 1);
      const unsigned act_k = __shfl_sync(FULL, act, ks);
      const unsigned wa_k = __shfl_sync(FULL, wa, ks);
      const unsigned wb_k = __shfl_sync(FULL, wb, ks);
      const int prev = __shfl_sync(FULL, incl, (k - 1) & (CHUNK_WORDS - 1));
      bool valid = want < total;
      long long i = 0;
      int bit = 0;
      if (valid) {
        bit = nth_set_bit(act_k, want - (k ? prev : 0));
        i = 32 * (w0 + k) + bit;
        valid = i < N;
      }
      fn(valid, i, valid && ((wa_k >> bit) & 1u), valid && ((wb_k >> bit) & 1u));
    }
  }
}

// ---------------------------------------------------------------------------
// grid barrier for co-resident (cooperative) launches, bounded: returns false
// (error bit set) if the other blocks do not arrive within spin_limit polls.
// bar[0] counts arrivals monotonically within a launch (zeroed before it):
// the k-th barrier completes when the count reaches k * gridDim.x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_sync(unsigned* bar, int spin_limit, unsigned* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    unsigned target = (old / gridDim.x + 1) * gridDim.x;
    int spins = 0;
    while ((int)(ld_acquire_u32(bar) - target) < 0) {
      if (++spins > spin_limit || (*(volatile unsigned*)err & ERR_TIMEOUT)) {
        atomicOr(err, ERR_TIMEOUT);
        ok = 0;
        break;
      }
      if (spins > 512) __nanosleep(32);
    }
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace dynbond
