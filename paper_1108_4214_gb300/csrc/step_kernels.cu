// Kernels of one dynamic-bonding call (Svaneborg, arXiv:1108.4214, Appendix
// steps 1-10), in launch order:
//   k_setup       zero the per-call scratch and cell counts
//   k_bead        per bead: bounds check, cell histogram of the beads whose
//                 eligibility bit is set (step 2)
//   k_scan_cells  exclusive scan of the cell histogram (single pass)
//   k_scatter     counting-sort scatter of eligible beads into cell order;
//                 beside it, breakage nomination lists and killbond marks of
//                 the beads holding breakable bonds (steps 3, 5)
//   k_candidates(_oct)  per eligible bead: every creation partner in the
//                 neighbouring cell columns (an octant of them when columns
//                 are twice the reach wide) within the z reach interval,
//                 last-rule-wins typing, graph-distance exclusion, maxbond
//                 (step 2); sorted per-bead lists (k_cand_overflow finishes
//                 beads with more than MAXC candidates)
//   k_match       rounds of mutual nomination for creation and breakage at
//                 once (step 4), cooperative launch with a bounded barrier
//   k_edit        trials, kill / break / convert / form applied to each
//                 bead's own bond slots (steps 5, 7, 8); lists the new bonds
//   k_purge       positions of the angle / dihedral records on removed or
//                 retyped bonds (step 6)
//   k_fill        surviving tail records moved into the holes: dense lists
//   k_rebuild     typed records of every path through a new bond (step 9);
//                 per-replica counts and statistics (step 10)
#include "common.cuh"
#include "kernels.h"

namespace dynbond {

constexpr int SCAN_BATCH = 2;  // candidate entries loaded together
template <int N>
struct IntC {
  static constexpr int value = N;
};
constexpr int FO_BATCH = 4;     // list entries examined together by first_open
constexpr int SOLO_LIVE = 512;   // live beads below which block 0 finishes the matching alone

__device__ __forceinline__ void stat_add(const Dev& d, int r, int k, long long v) {
  if (v) atomicAdd((unsigned long long*)&d.stats[(long long)r * NSTAT + k], (unsigned long long)v);
}

// warp-aggregated append of `want` items; returns this lane's first index
__device__ __forceinline__ int warp_alloc(int* counter, int want) {
  int lane = threadIdx.x & 31;
  int incl = warp_incl_scan(want);
  int total = __shfl_sync(FULL, incl, 31);
  int base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, total);
  base = __shfl_sync(FULL, base, 31);
  return base + incl - want;
}

// ---------------------------------------------------------------------------
// k_bead
// ---------------------------------------------------------------------------
// Breakage nomination of bead i (Appendix steps 3 and 5): its symmetric bonds
// of a type named by breakbond / convertbond / killbond with both ends
// reactive, sorted by (-d2, partner); killbond marks; settled pairs.
// Returns the flags of the activity bitmaps (bit 0: active in the edit,
// bit 1: nominates in the matching).
__device__ __forceinline__ unsigned bead_breakage(const Dev& d, const RuleTab& rt, const int4* __restrict__ pos,
                                                  long long i, int r, const CountTargets<2>& tg, ReplicaCounts<2>& cnt,
                                                  int& hit_r) {
  const long long N = d.N;
  const uint4 s = d.slots[i];
  const int4 p = pos[i];
  const int L = (int)d.box[r];
  unsigned km = 0;
  int4 ent[SLOTS];
  int nbrk = 0, ncand_b = 0;
  int nbt = 0;        // slots of i holding a type named by break / convert / kill rules
  uint4 sj_one = s;   // slots of the partner (meaningful when nbrk == 1)
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    unsigned v = s_get(s, q);
    if (!v || !has_bit(rt.breakish, s_type(v))) continue;
    ++nbt;
    int bty = s_type(v), j = s_partner(v);
    if (!has_bit(rt.reactive, d.type[j])) continue;
    const uint4 sj = d.slots[j];
    if (s_type_to(sj, (int)i) != bty) continue;
    sj_one = sj;
    long long dd = dist2(p, pos[j], L);
    int rule = -1;
    for (int q2 = rt.bk_start[bty], q3 = rt.bk_start[bty + 1]; q2 < q3; ++q2) {
      int k = rt.bk_list[q2];
      int kd = rt.kind[k];
      if (kd == DYNBOND_KILLBOND && dd > rt.r2[k]) km |= 1u << q;
      if ((kd == DYNBOND_BREAKBOND && dd > rt.r2[k]) || kd == DYNBOND_CONVERTBOND) rule = k;
    }
    if (rule < 0) continue;
    // insert sorted by (-d2, partner)
    long long key = -dd;
    int at = nbrk;
    while (at > 0) {
      long long pk = ((long long)(unsigned)ent[at - 1].w << 32) | (unsigned)ent[at - 1].z;
      if (pk < key || (pk == key && ent[at - 1].x < j)) break;
      ent[at] = ent[at - 1];
      --at;
    }
    ent[at] = make_int4(j, rule, (int)(unsigned)(unsigned long long)key, (int)(key >> 32));
    ++nbrk;
    ncand_b += j > i;
  }
  cnt.add(tg, r, 0, ncand_b);
  // A settled pair: both ends hold exactly one bond of a type named by
  // break / convert / kill rules -- each other.  They nominate each other in
  // round 0 and nobody else can nominate either, so they match there
  // whatever else happens; the trial (step 5) is drawn now and only a
  // successful one reaches the edit.
  bool settled = false;
  if (nbrk == 1 && nbt == 1) {
    int nbt_j = 0;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      unsigned v = s_get(sj_one, q);
      nbt_j += v && has_bit(rt.breakish, s_type(v));
    }
    settled = nbt_j == 1;
  }
  bool broken = false;
  if (settled) {
    const int j = ent[0].x, k = ent[0].y;
    const int a = (int)min((long long)j, i), b = (int)max((long long)j, i);
    broken = trial(d, rt, a, b, r, TAG_BREAK, d.T_break[(long long)r * MAXR + k]);
    if (j > i) {
      cnt.add(tg, r, 1, 1);  // the pair matched in round 0
      if (hit_r != r) {
        if (hit_r >= 0) d.round_hit[d.R + hit_r] = 1;
        hit_r = r;
      }
    }
  }
  const bool ba = km || (nbrk && !settled) || broken;
  if (ba) {
    d.killmask[i] = (unsigned char)km;
    d.brk_len[i] = (unsigned char)nbrk;
    for (int q = 0; q < nbrk; ++q) d.brk[4 * i + q] = ent[q];
    if (nbrk) {
      d.mate[N + i] = broken ? mate_pack(0, ent[0].x) : -1;
      d.ptr[N + i] = 0;
      d.nom[N + i] = ent[0].x;  // round 0 nomination: the most distant partner
    }
  }
  return (ba ? 1u : 0u) | (nbrk > 0 && !settled ? 2u : 0u);
}

// Per bead: bounds check and binning of the beads that can form bonds
// (Appendix step 2; occupancy counts only, the scatter assigns the slots).
// Which beads can form a bond, and which hold a breakable bond, depends on
// their bonds only: both bitmaps are computed at creation (k_bead_flags) and
// kept current by the edit, so this pass reads positions and the bitmap.
__device__ __forceinline__ void bead_body(const Dev& d, const RuleTab* __restrict__ rtp) {
  const RuleTab& rt = *rtp;
  const int4* __restrict__ pos = d.args->pos;
  const long long N = d.N;
  const int lane = threadIdx.x & 31;
  // a warp takes segments of BIN_SEG consecutive beads (32 per load, the
  // segment's loads issued together) and writes its binned beads, (bead, cell
  // key), to the front of the segment's own part of `binned` with their count
  // in binned_n: no shared counter
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long sg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sg * BIN_SEG < N; sg += nwarps) {
    const long long i0 = sg * BIN_SEG + lane;
    constexpr int U = BIN_SEG / 32;
    int4 p[U];
    unsigned ew[U];
    int rr[U], bt[U], cell[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + 32 * u;
      if (i < N) {
        p[u] = pos[i];
        ew[u] = d.bm_elig[i >> 5];
        rr[u] = rep_of(d, i);
        bt[u] = d.type[i];
      }
    }
    int nb = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + 32 * u;
      cell[u] = -1;
      if (i >= N) continue;
      const int r = rr[u];
      const int4 g0 = d.geo[2 * r];
      const int L = g0.x;
      if (p[u].x < 0 || p[u].y < 0 || p[u].z < 0 || p[u].x >= L || p[u].y >= L || p[u].z >= L) {
        atomicOr(d.err, ERR_POS);
      } else if ((ew[u] >> (i & 31)) & 1u) {
        const int4 g1 = d.geo[2 * r + 1];
        const int nc = g0.y, nz = g0.z;
        const float f = __int_as_float(g1.x);
        long long cx = cell_of(p[u].x, nc, L, f), cy = cell_of(p[u].y, nc, L, f);
        long long cz = cell_of(p[u].z, nz, L, __int_as_float(g1.y));
        long long c = rt.cls_of[bt[u]] * d.n_cells + g1.z + (cx * nc + cy) * nz + cz;
        atomicAdd(&d.cell_start[c], 1);  // count only; the scatter assigns the slots
        cell[u] = (int)c;
        ++nb;
      }
    }
    const int incl = warp_incl_scan(nb);
    int at = (int)(sg * BIN_SEG) + incl - nb;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cell[u] >= 0) d.binned[at++] = make_int2((int)(i0 + 32 * u), cell[u]);
    if (lane == 31) d.binned_n[sg] = incl;
  }
}

__global__ void __launch_bounds__(256) k_bead(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_enter();
  bead_body(d, rtp);
}

// Both bead bitmaps from the bonds, for every bead (at creation).
__global__ void __launch_bounds__(256) k_bead_flags(Dev d, const RuleTab* __restrict__ rtp) {
  const RuleTab& rt = *rtp;
  const long long N = d.N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += stride) {
    const long long i = base + threadIdx.x;
    bool el = false, bk = false;
    if (i < N) {
      const int bt = d.type[i];
      const uint4 s = d.slots[i];
      el = creation_eligible(rt, bt, s);
      bk = holds_breakable(rt, bt, s);
    }
    const unsigned me = __ballot_sync(FULL, el), mb = __ballot_sync(FULL, bk);
    if ((threadIdx.x & 31) == 0 && i < N) {
      d.bm_elig[i >> 5] = me;
      d.bm_bk[i >> 5] = mb;
    }
  }
}

// ---------------------------------------------------------------------------
// k_scan_cells: in-place exclusive scan of the cell histogram
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scan_cells_body(const Dev& d) {
  __shared__ long long sh[33];
  __shared__ long long s_excl;
  __shared__ long long s_tile;
  const long long n = d.n_keys;
  const long long per_tile = (long long)blockDim.x * SCAN_PER_THREAD;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&d.cnt->ticket[0], 1);
    __syncthreads();
    long long t = s_tile;
    if (t >= ntiles) break;
    long long beg = t * per_tile + (long long)threadIdx.x * SCAN_PER_THREAD;
    int v[SCAN_PER_THREAD];
    const bool full = beg + SCAN_PER_THREAD <= n;
    if (full) {
      const int4* src = reinterpret_cast<const int4*>(d.cell_start + beg);
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD / 4; ++k) {
        int4 x = src[k];
        v[4 * k] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD; ++k) v[k] = beg + k < n ? d.cell_start[beg + k] : 0;
    }
    long long sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) sum += v[k];
    long long tot;
    long long ex = block_excl_scan(sum, sh, &tot);
    if (threadIdx.x < 32) {
      long long x = lookback(d.st_scan, t, 0, (unsigned long long)tot, d.spin_limit, d.err);
      if (threadIdx.x == 0) s_excl = x;
    }
    __syncthreads();
    if (s_excl < 0) return;
    long long pre = s_excl + ex;
    if (full) {
      int4* dst = reinterpret_cast<int4*>(d.cell_start + beg);
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD / 4; ++k) {
        int4 x;
        x.x = (int)pre;
        pre += v[4 * k];
        x.y = (int)pre;
        pre += v[4 * k + 1];
        x.z = (int)pre;
        pre += v[4 * k + 2];
        x.w = (int)pre;
        pre += v[4 * k + 3];
        dst[k] = x;
      }
    } else {
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (beg + k < n) d.cell_start[beg + k] = (int)pre;
        pre += v[k];
      }
    }
    if (t == ntiles - 1 && threadIdx.x == blockDim.x - 1) {
      d.cell_start[n] = (int)pre;
      d.cnt->n_sorted = (int)pre;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_scan_cells(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  scan_cells_body(d);
}

// Counting-sort scatter of the binned beads into cell order, by blocks
// b = 0 .. nb - 1 of the caller's: a warp per segment of k_bead, only the
// segment's binned beads.
__device__ __forceinline__ void scatter_part(const Dev& d, int b, int nb) {
  const int4* __restrict__ pos = d.args->pos;
  const int lane = threadIdx.x & 31;
  const long long nseg = (d.N + BIN_SEG - 1) / BIN_SEG;
  const long long nwarps = (long long)nb * (blockDim.x >> 5);
  constexpr int U = BIN_SEG / 32;
  for (long long sg = (long long)b * (blockDim.x >> 5) + (threadIdx.x >> 5); sg < nseg; sg += nwarps) {
    const int cnt = d.binned_n[sg];
    int2 e[U];
    int at[U];
    int4 p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = 32 * u + lane < cnt ? d.binned[sg * BIN_SEG + 32 * u + lane] : make_int2(-1, -1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e[u].x >= 0) {
        p[u] = pos[e[u].x];
        p[u].w = (int)(((long long)e[u].x << 4) | d.type[e[u].x]);
      }
    }
    // after the scatter cell_start[c] holds the end of cell c, i.e. the start
    // of cell c + 1 (the search reads cell c as [cell_start[c-1], cell_start[c]))
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e[u].x >= 0) at[u] = atomicAdd(&d.cell_start[e[u].y], 1);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e[u].x >= 0) d.sorted[at[u]] = p[u];
  }
}

// Breakage nomination of the beads of the breakage bitmap by blocks b = 0 ..
// nb - 1 of the caller's, with their edit / nomination bits OR-ed into the
// activity bitmaps.  It needs neither the positions' binning nor the cell
// list, so it runs beside them.
__device__ __forceinline__ void breakage_part(const Dev& d, const RuleTab* __restrict__ rtp, int b, int nb) {
  const int4* __restrict__ pos = d.args->pos;
  const RuleTab& rt = *rtp;
  const CountTargets<2> tg{{d.stats + ST_BREAK_CANDIDATES, d.stats + ST_BREAK_MATCHED}, {NSTAT, NSTAT}};
  ReplicaCounts<2> cnt;
  int hit_r = -1;  // replica of the settled breakage pairs this thread counted
  const long long nchunks = (d.W + CHUNK_WORDS - 1) / CHUNK_WORDS;
  const long long cpb = (nchunks + nb - 1) / nb;
  const long long c0 = (long long)b * cpb, c1 = min(nchunks, c0 + cpb);
  for_bits_block(d.bm_bk, nullptr, d.W, d.N, c0, c1, [&](bool valid, long long i, bool, bool) {
    if (!valid) return;
    const unsigned fl = bead_breakage(d, rt, pos, i, rep_of(d, i), tg, cnt, hit_r);
    if (fl & 1u) atomicOr(&d.bm_ba[i >> 5], 1u << (i & 31));
    if (fl & 2u) atomicOr(&d.bm_bn[i >> 5], 1u << (i & 31));
  });
  cnt.flush_block(tg);
  // settled pairs count as round-0 breakage matches of their replica
  block_flag(d.round_hit + d.R, hit_r);
}

// The persistent call's form: the first gridDim.x - scatter_blocks blocks
// nominate (their longer dependent chains start with the first wave instead
// of trailing the scatter), the last scatter_blocks scatter.
__device__ __forceinline__ void scatter_body(const Dev& d, const RuleTab* __restrict__ rtp, int scatter_blocks) {
  const int nb = gridDim.x - scatter_blocks;
  if ((int)blockIdx.x >= nb) scatter_part(d, blockIdx.x - nb, scatter_blocks);
  else breakage_part(d, rtp, blockIdx.x, nb);
}

__global__ void __launch_bounds__(256) k_scatter(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  scatter_part(d, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_breakage(Dev d, const RuleTab* __restrict__ rtp) {
  if (aborted(d.err)) return;
  breakage_part(d, rtp, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// k_candidates
// ---------------------------------------------------------------------------

// Graph distance test on the bond graph before the call: never at distance 1,
// at 2 only with paircheck13, at 3 only with paircheck14, always beyond.
__device__ __forceinline__ bool pair_eligible(const uint4* __restrict__ slots, const RuleTab& rt, int i, int j,
                                              const uint4& si, const uint4& sj) {
  int ni[SLOTS], nj[SLOTS];
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    ni[q] = s_partner(s_get(si, q));
    nj[q] = s_partner(s_get(sj, q));
    if (ni[q] == j) return false;
  }
  bool g2 = false;
#pragma unroll
  for (int q = 0; q < SLOTS; ++q)
#pragma unroll
    for (int w = 0; w < SLOTS; ++w) g2 |= ni[q] >= 0 && ni[q] == nj[w];
  if (g2) return rt.pc13 != 0;
  bool g3 = false;
  for (int q = 0; q < SLOTS && !g3; ++q) {
    if (ni[q] < 0) continue;
    uint4 sa = slots[ni[q]];
#pragma unroll
    for (int q2 = 0; q2 < SLOTS; ++q2) {
      int b = s_partner(s_get(sa, q2));
      if (b < 0) continue;
#pragma unroll
      for (int w = 0; w < SLOTS; ++w) g3 |= nj[w] == b;
    }
  }
  if (g3) return rt.pc14 != 0;
  return true;
}

// Per-bead candidate list kept in registers / local memory by the fast path.
struct LocalList {
  long long kd[MAXC];
  int kp[MAXC], ki[MAXC];
  int cnt, pairs, me;
  bool overflow;
};

// Rule and graph-distance tests of a pair within the largest creation
// distance: the last matching creation rule and the type bead i would store
// (code = rule | stored type << 8), or -1.  Kept out of line so the scan
// loops stay small.
__device__ __noinline__ int eval_pair(const uint4* __restrict__ slots, const RuleTab* __restrict__ rtp, int i, int j,
                                      int ti, int tj, long long dd, uint4 si) {
  const RuleTab& rt = *rtp;
  uint4 sj = slots[j];
  int sta, stb, k;
  if (i < j) k = creation_rule(rt, ti, tj, si, sj, dd, &sta, &stb);
  else k = creation_rule(rt, tj, ti, sj, si, dd, &stb, &sta);
  if (k < 0 || !pair_eligible(slots, rt, i, j, si, sj)) return -1;
  return k | (sta << 8);
}

// insert (dd, j, code) into the bead's list, sorted by (d2, partner)
__device__ __forceinline__ void list_insert(LocalList* ll, long long dd, int j, int code) {
  if (ll->cnt == MAXC) {
    ll->overflow = true;
    return;
  }
  int at = ll->cnt;
  while (at > 0 && (ll->kd[at - 1] > dd || (ll->kd[at - 1] == dd && ll->kp[at - 1] > j))) {
    ll->kd[at] = ll->kd[at - 1];
    ll->kp[at] = ll->kp[at - 1];
    ll->ki[at] = ll->ki[at - 1];
    --at;
  }
  ll->kd[at] = dd;
  ll->kp[at] = j;
  ll->ki[at] = code;
  ++ll->cnt;
}

// The overflow passes: mode 1 counts the bead's candidates, mode 2 writes
// them to *out (sorted afterwards).
__device__ __forceinline__ void cand_slow(const uint4* __restrict__ slots, const RuleTab* __restrict__ rtp, int i,
                                          int j, int ti, int tj, long long dd, uint4 si, LocalList* ll, int mode,
                                          int4** out) {
  const int code = eval_pair(slots, rtp, i, j, ti, tj, dd, si);
  if (code < 0) return;
  ll->pairs += j > i;
  if (mode == 2) *(*out)++ = make_int4(j, code, (int)(unsigned)(unsigned long long)dd, (int)(dd >> 32));
  else ++ll->cnt;
}

// The cells eligible bead `me` (replica r) searches in each cell-list class:
// NA x NA cell columns (xs x ys, nx distinct per axis; NA = 2 octant, else 3)
// and along z a window of cells holding every cell that [z - reach, z + reach]
// overlaps (periodic), as a main run [z0, z1] and, across the boundary, a
// wrapped run [w0, w1] (empty if w1 < w0; the whole column when it covers it).  The cells of a column are
// contiguous in cell order, so each run of each column is one contiguous
// range of the sorted array.  GEO 1: every replica's columns are at least
// twice the reach wide, and a bead's reach only touches the neighbouring
// column on the side of the half it sits in (octant of columns); GEO 0: 3 x 3
// columns, correct for any geometry with columns at least the reach wide.
struct BeadGeo {
  int L, nc, nz, cb, nx;
  int xs[3], ys[3];
  int z0, z1, w0, w1;
};
template <int GEO>
__device__ __forceinline__ BeadGeo bead_geo(const Dev& d, const int4& me, int r) {
  BeadGeo g;
  const int4 g0 = d.geo[2 * r], g1 = d.geo[2 * r + 1];
  const int L = g0.x, nc = g0.y, nz = g0.z, hz = g0.w;
  g.L = L;
  g.nc = nc;
  g.nz = nz;
  g.cb = g1.z;  // cell keys fit in 32 bits (n_cls * n_cells < 2^31 is checked on the host)
  const float f = __int_as_float(g1.x), fz = __int_as_float(g1.y);
  const int cx = cell_of(me.x, nc, L, f), cy = cell_of(me.y, nc, L, f);
  g.nx = nc >= 3 ? 3 : nc;
  g.xs[0] = cx;
  g.xs[1] = cx + 1 == nc ? 0 : cx + 1;
  g.xs[2] = cx == 0 ? nc - 1 : cx - 1;
  g.ys[0] = cy;
  g.ys[1] = cy + 1 == nc ? 0 : cy + 1;
  g.ys[2] = cy == 0 ? nc - 1 : cy - 1;
  // is coordinate x in the lower half of its cell c (exactly: 2 (x nc - c L) < L)?
  auto lower = [&](int x, int c) { return 2 * ((long long)x * nc - (long long)c * L) < (long long)L; };
  if (GEO == 1) {
    g.nx = 2;
    if (lower(me.x, cx)) g.xs[1] = g.xs[2];
    if (lower(me.y, cy)) g.ys[1] = g.ys[2];
  }
  // z: the cells cz - hz .. cz + hz (periodic), which hold every cell the
  // reach interval overlaps (floor(a - b) >= floor(a) - ceil(b) and
  // floor(a + b) <= floor(a) + ceil(b)); the whole column when they cover it
  const int cz = cell_of(me.z, nz, L, fz);
  g.w0 = 0;
  g.w1 = -1;
  if (2 * hz + 1 >= nz) {
    g.z0 = 0;
    g.z1 = nz - 1;
  } else {
    const int lo = cz - hz, hi = cz + hz;
    g.z0 = max(lo, 0);
    g.z1 = min(hi, nz - 1);
    if (lo < 0) {
      g.w0 = lo + nz;
      g.w1 = nz - 1;
    } else if (hi >= nz) {
      g.w0 = 0;
      g.w1 = hi - nz;
    }
  }
  return g;
}

// Visit every creation candidate of eligible bead i (sorted entry `me`):
// for each cell-list class holding partner types of bead i, the entries
// within the largest creation distance (the reach) among the cells of
// bead_geo are collected first; the rule and graph-distance tests then run on
// them after the scan, so the lanes of a warp take the rare path together
// instead of one after another.
template <int GEO>
__device__ __forceinline__ void scan_candidates(const Dev& d, const RuleTab* __restrict__ rtp, unsigned cmask,
                                                long long r2max, const int4& me, int i, LocalList* ll, int mode,
                                                int4** out, int* pj, long long* pd, int* np_out) {
  const int ti = me.w & 15;
  const int r = rep_of(d, i);
  const BeadGeo g = bead_geo<GEO>(d, me, r);
  const int L = g.L, nc = g.nc, nz = g.nz, cb = g.cb, ncl = (int)d.n_cells, nx = g.nx;
  const int *xs = g.xs, *ys = g.ys;
  const int z0 = g.z0, z1 = g.z1, w0 = g.w0, w1 = g.w1;
  int np = 0;
  bool more = false;
  // entries of the NA x NA column runs (NA = 2 octant, else 3), fetched
  // SCAN_BATCH at a time with independent loads (runs are short, many are
  // empty).  Entry k of the concatenated runs is sorted[k + dl[u]] for the
  // last run u starting at or before k (an empty run is never the last).
  auto scan_runs = [&](auto na_c, int lo, int hi, int cbk) {
    constexpr int NA = decltype(na_c)::value, NR = NA * NA;
    int dl[NR], ex[NR + 1];  // run offsets; exclusive prefix of the run lengths
    ex[0] = 0;
#pragma unroll
    for (int ab = 0; ab < NR; ++ab) {
      const int a = ab / NA, b = ab % NA;
      int len = 0, q0 = 0;
      if (a < nx && b < nx) {
        const int row = cbk + (xs[a] * nc + ys[b]) * nz;
        q0 = d.cell_start[row + lo - 1];
        len = d.cell_start[row + hi] - q0;
      }
      dl[ab] = q0 - ex[ab];
      ex[ab + 1] = ex[ab] + len;
    }
    const int total = ex[NR];
    for (int k0 = 0; k0 < total; k0 += SCAN_BATCH) {
      int4 o[SCAN_BATCH];
#pragma unroll
      for (int v = 0; v < SCAN_BATCH; ++v) {
        const int k = k0 + v;
        int dk = dl[0];
#pragma unroll
        for (int u = 1; u < NR; ++u)
          if (k >= ex[u]) dk = dl[u];
        if (k < total) o[v] = d.sorted[k + dk];
      }
#pragma unroll
      for (int v = 0; v < SCAN_BATCH; ++v) {
        if (k0 + v >= total) break;
        const long long dd = dist2(me, o[v], L);
        if (dd > r2max || (o[v].w >> 4) == i) continue;
        if (np < MAXC) {
          pj[np] = o[v].w;
          pd[np] = dd;
          ++np;
        } else {
          more = true;
        }
      }
    }
  };
  for (unsigned cm = cmask; cm; cm &= cm - 1) {
    const int cbk = (__ffs(cm) - 1) * ncl + cb;  // this class's cells of the replica
    scan_runs(IntC<GEO == 1 ? 2 : 3>{}, z0, z1, cbk);
    if (w1 >= w0) scan_runs(IntC<GEO == 1 ? 2 : 3>{}, w0, w1, cbk);  // next to a periodic boundary in z
  }
  if (mode == 0) {  // survivors go back to the caller; the warp tests them together
    ll->overflow = more;  // finished exactly by k_cand_overflow
    *np_out = more ? 0 : np;
    return;
  }
  if (more) {  // counting / writing passes of the overflow path: rescan without a buffer
    uint4 si = d.slots[i];
    for (unsigned cm = cmask; cm; cm &= cm - 1) {
      const int cbk = (__ffs(cm) - 1) * ncl + cb;
      for (int a = 0; a < nx; ++a)
        for (int b = 0; b < nx; ++b) {
          const int row = cbk + (xs[a] * nc + ys[b]) * nz;
          for (int run = 0; run < 2; ++run) {
            int lo = run ? w0 : z0, hi = run ? w1 : z1;
            if (hi < lo) continue;
            int q0 = d.cell_start[row + lo - 1], q1 = d.cell_start[row + hi];
            for (int q = q0; q < q1; ++q) {
              int4 o = d.sorted[q];
              long long dd = dist2(me, o, L);
              if (dd > r2max || (o.w >> 4) == i) continue;
              cand_slow(d.slots, rtp, i, o.w >> 4, ti, o.w & 15, dd, si, ll, mode, out);
            }
          }
        }
    }
    return;
  }
  if (np == 0) return;
  uint4 si = d.slots[i];
  for (int k = 0; k < np; ++k) cand_slow(d.slots, rtp, i, pj[k] >> 4, ti, pj[k] & 15, pd[k], si, ll, mode, out);
}

// The rule and graph-distance tests of the survivors of a whole warp: the
// lanes' survivors are queued in shared memory and tested 32 at a time, so
// a lane with many survivors does not hold the warp for each of them; the
// results go back to the owners' sorted lists.  Every lane must call it.
constexpr int SURV_CAP = 64;  // queued survivors per warp (more: each lane tests its own)
struct SurvQueue {
  int j[SURV_CAP], code[SURV_CAP];
  long long dd[SURV_CAP];
  unsigned char owner[SURV_CAP];
};
__device__ __forceinline__ void warp_survivors(const Dev& d, const RuleTab* __restrict__ rtp, int i, int ti,
                                               const uint4& si, const int* pj, const long long* pd, int np,
                                               LocalList* ll, SurvQueue& q) {
  const int lane = threadIdx.x & 31;
  const int incl = warp_incl_scan(np);
  const int total = __shfl_sync(FULL, incl, 31);
  if (total == 0) return;
  if (total > SURV_CAP) {
    for (int k = 0; k < np; ++k) {
      const int code = eval_pair(d.slots, rtp, i, pj[k] >> 4, ti, pj[k] & 15, pd[k], si);
      if (code < 0) continue;
      ll->pairs += (pj[k] >> 4) > i;
      list_insert(ll, pd[k], pj[k] >> 4, code);
    }
    return;
  }
  const int off = incl - np;
  for (int k = 0; k < np; ++k) {
    q.j[off + k] = pj[k];
    q.dd[off + k] = pd[k];
    q.owner[off + k] = (unsigned char)lane;
  }
  __syncwarp();
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + lane;
    const bool valid = t < total;
    const int o = valid ? q.owner[t] : lane;
    const int oi = __shfl_sync(FULL, i, o), oti = __shfl_sync(FULL, ti, o);
    const uint4 osi = make_uint4(__shfl_sync(FULL, si.x, o), __shfl_sync(FULL, si.y, o), __shfl_sync(FULL, si.z, o),
                                 __shfl_sync(FULL, si.w, o));
    if (valid) q.code[t] = eval_pair(d.slots, rtp, oi, q.j[t] >> 4, oti, q.j[t] & 15, q.dd[t], osi);
  }
  __syncwarp();
  for (int k = 0; k < np; ++k) {
    const int code = q.code[off + k];
    if (code < 0) continue;
    const int j = pj[k] >> 4;
    ll->pairs += j > i;
    list_insert(ll, pd[k], j, code);
  }
  __syncwarp();
}

// first: the list's first partner (round 0: nobody is matched yet, so the
// bead nominates its nearest partner)
__device__ __forceinline__ void activate_creator(const Dev& d, int i, int start, int len, int first) {
  d.cand_start[i] = start;
  d.cand_len[i] = len;
  d.mate[i] = -1;
  d.ptr[i] = 0;
  d.nom[i] = first;
  atomicOr(&d.bm_ca[i >> 5], 1u << (i & 31));
}

// per bead type: the cell-list classes holding its partner types
__device__ __forceinline__ void load_type_masks(const RuleTab& rt, unsigned* s_mask) {
  if (threadIdx.x < 16) s_mask[threadIdx.x] = rt.cls_mask[threadIdx.x];
  __syncthreads();
}

// The sorted candidate list of sorted entry e (bead i; i < 0: no bead): lists
// of up to CAND_FAST entries go to the entry's own slots, longer ones (rare)
// take room from the shared pool behind them; a bead with more than MAXC
// candidates is queued for k_cand_overflow.  Every lane of the warp must call it.
__device__ __forceinline__ void emit_list(const Dev& d, int e, int i, const LocalList& ll) {
  const int oslot = warp_alloc(&d.cnt->n_ovf, ll.overflow ? 1 : 0);
  if (ll.overflow) d.ovf[oslot] = e;
  int cnt = ll.overflow ? 0 : ll.cnt;
  if (cnt > 0) {
    long long at = (long long)e * CAND_FAST;
    if (cnt > CAND_FAST) {
      const int a = atomicAdd(&d.cnt->cand_used, cnt);
      at = d.cand_fixed + a;
      if ((long long)a + cnt > d.cand_pool) {
        atomicOr(d.err, ERR_CAND_CAP);
        cnt = 0;
      }
    }
    if (cnt > 0) {
      for (int q = 0; q < cnt; ++q)
        d.cand[at + q] =
            make_int4(ll.kp[q], ll.ki[q], (int)(unsigned)(unsigned long long)ll.kd[q], (int)(ll.kd[q] >> 32));
      activate_creator(d, i, (int)at, cnt, ll.kp[0]);
    }
  }
}

template <int GEO>
__device__ __forceinline__ void candidates_body(const Dev& d, const RuleTab* __restrict__ rtp) {
  __shared__ unsigned s_mask[16];
  load_type_masks(*rtp, s_mask);
  const long long r2max = rtp->r2max;
  const int n = d.cnt->n_sorted;
  const int stride = gridDim.x * blockDim.x;
  const CountTargets<1> tg{{d.stats + ST_CANDIDATES}, {NSTAT}};
  ReplicaCounts<1> pairs;
  ReplicaCounts<1>::begin_block();
  __shared__ SurvQueue s_q[8];  // one per warp (256 threads)
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    int e = base + threadIdx.x;
    int i = -1, r = 0, ti = 0, np = 0;
    int pj[MAXC];
    long long pd[MAXC];
    uint4 si = make_uint4(0, 0, 0, 0);
    LocalList ll;
    ll.cnt = ll.pairs = 0;
    ll.overflow = false;
    if (e < n) {
      int4 me = d.sorted[e];
      i = me.w >> 4;
      ti = me.w & 15;
      r = rep_of(d, i);
      ll.me = i;
      scan_candidates<GEO>(d, rtp, s_mask[ti], r2max, me, i, &ll, 0, nullptr, pj, pd, &np);
      if (np) si = d.slots[i];
    }
    warp_survivors(d, rtp, i, ti, si, pj, pd, np, &ll, s_q[threadIdx.x >> 5]);
    emit_list(d, e, i, ll);
    if (e < n && !ll.overflow) pairs.add(tg, r, 0, ll.pairs);
  }
  pairs.end_warp(tg);
}

__global__ void __launch_bounds__(256, 3) k_candidates(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_enter();
  if (aborted(d.err)) return;
  candidates_body<0>(d, rtp);
}
__global__ void __launch_bounds__(256, 4) k_candidates_oct(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_enter();
  if (aborted(d.err)) return;
  candidates_body<1>(d, rtp);
}

// ---------------------------------------------------------------------------
// k_candidates_tile: the same search by tiles of cell columns staged in
// shared memory.  A work item is one replica's cell-list class c over CT x CT
// cell columns and a window of z cells.  The block stages, for every partner
// class of c, the entries of the columns one step around the tile (x and y,
// periodic, distinct) over the z window widened by hz cells on each side
// (the whole column when that covers it): first the cell counts (one pass
// over the cell ends, a block scan gives each staged cell its place), then
// the entries themselves with 16-byte cp.async.  Every owned bead of the tile
// then runs the search of scan_candidates on the staged copy, so its
// neighbour-cell loop walks shared memory instead of issuing dependent global
// loads.  Survivors are tested and listed exactly as by k_candidates.  Tiles
// whose staged data would not fit (dense cells, many partner classes) run the
// global-memory search for their beads.  Work items are taken from a ticket.
// ---------------------------------------------------------------------------
struct CandStage {
  int4 ent[C_ENT_CAP];
  unsigned short off[C_COL_CAP][CZS_MAX + 1];  // column-relative start of staged cell lz; [Zs] = column total
  int cbase[C_COL_CAP + 1];                    // first staged entry of each column; [n_cols] = total
  int colA[C_COL_CAP], colLenA[C_COL_CAP], colB[C_COL_CAP];  // per staged column: its run up to the
                                                             // end of the column, then from z cell 0
  int own_g[CT * CT], own_pre[CT * CT + 1];                  // owned column runs of sorted entries
  int r, c, pmask, P, nc, nz, L, hx0, hy0, HX, HY, hz0, Zs, whole, n_cols, n_own_cols, x0, y0, Ty, z0, Tz, fallback;
};
static_assert(sizeof(CandStage) <= CAND_TILE_SMEM, "candidate tile shared memory layout");

// Tile parameters from the work item and its replica's geometry.  Tile
// record: x = replica, y = class | hz << 8 | partner classes << 16, z = tile
// x | tile y << 16, w = tile z | z cells per tile << 16.
__device__ __forceinline__ void tile_params(const int4& t, int nc, int nz, int L, CandStage& S) {
  S.r = t.x;
  S.c = t.y & 0xFF;
  const int hz = (t.y >> 8) & 0xFF;
  S.pmask = (int)((unsigned)t.y >> 16);
  S.P = __popc(S.pmask);
  S.nc = nc;
  S.nz = nz;
  S.L = L;
  const int x0 = (t.z & 0xFFFF) * CT, y0 = ((unsigned)t.z >> 16) * CT;
  const int Tx = min(CT, nc - x0), Ty = min(CT, nc - y0);
  const int Z = (unsigned)t.w >> 16;
  S.z0 = (t.w & 0xFFFF) * Z;
  S.Tz = min(Z, nz - S.z0);
  S.x0 = x0;
  S.y0 = y0;
  S.Ty = Ty;
  // halo columns: one step around the tile, distinct; all of them when that wraps
  S.HX = Tx + 2 >= nc ? nc : Tx + 2;
  S.hx0 = Tx + 2 >= nc ? 0 : (x0 == 0 ? nc - 1 : x0 - 1);
  S.HY = Ty + 2 >= nc ? nc : Ty + 2;
  S.hy0 = Ty + 2 >= nc ? 0 : (y0 == 0 ? nc - 1 : y0 - 1);
  S.whole = S.Tz + 2 * hz >= nz;
  S.Zs = S.whole ? nz : S.Tz + 2 * hz;
  S.hz0 = S.whole ? 0 : (S.z0 >= hz ? S.z0 - hz : S.z0 - hz + nz);
  S.n_cols = S.P * S.HX * S.HY;
  S.n_own_cols = Tx * Ty;
  S.fallback = S.n_cols > C_COL_CAP || S.Zs > CZS_MAX;
}

// a - b for two indices in [0, n): in [0, n)
__device__ __forceinline__ int cyc(int a, int b, int n) { return a >= b ? a - b : a - b + n; }

// The owned bead's candidates from the staged columns: the same neighbour
// columns and z cells as scan_candidates, read from shared memory.
template <int GEO>
__device__ __forceinline__ void scan_staged(const CandStage& S, long long r2max, long long reach, const int4& me,
                                            int i, int* pj, long long* pd, int& np, bool& more) {
  const int L = S.L, nc = S.nc, nz = S.nz;
  const float f = (float)nc / (float)L;
  const int cx = cell_of(me.x, nc, L, f), cy = cell_of(me.y, nc, L, f);
  int nx = nc >= 3 ? 3 : nc;
  int xs[3] = {cx, cx + 1 == nc ? 0 : cx + 1, cx == 0 ? nc - 1 : cx - 1};
  int ys[3] = {cy, cy + 1 == nc ? 0 : cy + 1, cy == 0 ? nc - 1 : cy - 1};
  auto lower = [&](int x, int cc) { return 2 * ((long long)x * nc - (long long)cc * L) < (long long)L; };
  if (GEO == 1) {
    nx = 2;
    if (lower(me.x, cx)) xs[1] = xs[2];
    if (lower(me.y, cy)) ys[1] = ys[2];
  }
  // z runs in staged (local) cells
  int ra0, ra1, rb0 = 0, rb1 = -1;
  {
    const float fz = (float)nz / (float)L;
    const long long zlo = (long long)me.z - reach, zhi = (long long)me.z + reach;
    if (!S.whole) {
      // the window holds every cell within hz of the bead's: one local run
      const int cz = cell_of(me.z, nz, L, fz);
      const int lo = cell_of((int)(zlo < 0 ? zlo + L : zlo), nz, L, fz);
      const int hi = cell_of((int)(zhi >= L ? zhi - L : zhi), nz, L, fz);
      const int lzb = cyc(cz, S.hz0, nz);
      ra0 = lzb - cyc(cz, lo, nz);
      ra1 = lzb + cyc(hi, cz, nz);
    } else if (zlo >= 0 && zhi < L) {
      ra0 = cell_of((int)zlo, nz, L, fz);
      ra1 = cell_of((int)zhi, nz, L, fz);
    } else if (zlo < 0 && zhi < L) {
      const int a = cell_of((int)(zlo + L), nz, L, fz), b = cell_of((int)zhi, nz, L, fz);
      ra0 = 0;
      ra1 = a > b ? b : nz - 1;
      if (a > b) {
        rb0 = a;
        rb1 = nz - 1;
      }
    } else if (zlo >= 0 && zhi >= L) {
      const int a = cell_of((int)zlo, nz, L, fz), b = cell_of((int)(zhi - L), nz, L, fz);
      ra0 = b < a ? a : 0;
      ra1 = nz - 1;
      if (b < a) {
        rb0 = 0;
        rb1 = b;
      }
    } else {
      ra0 = 0;
      ra1 = nz - 1;
    }
  }
  for (int pi = 0; pi < S.P; ++pi)
    for (int a = 0; a < nx; ++a) {
      const int colx = (pi * S.HX + cyc(xs[a], S.hx0, nc)) * S.HY;
      for (int b = 0; b < nx; ++b) {
        const int col = colx + cyc(ys[b], S.hy0, nc);
        const int base = S.cbase[col];
        const unsigned short* off = S.off[col];
        for (int run = 0; run < 2; ++run) {
          const int la = run ? rb0 : ra0, lb = run ? rb1 : ra1;
          if (lb < la) continue;
          const int q1 = base + off[lb + 1];
          for (int q = base + off[la]; q < q1; ++q) {
            const int4 o = S.ent[q];
            const long long dd = dist2(me, o, L);
            if (dd > r2max || (o.w >> 4) == i) continue;
            if (np < MAXC) {
              pj[np] = o.w;
              pd[np] = dd;
              ++np;
            } else {
              more = true;
            }
          }
        }
      }
    }
}

// largest k in [0, n) with a[k] <= x (a non-decreasing, a[0] <= x), shared memory
__device__ __forceinline__ int smem_upper(const int* a, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int GEO>
__device__ __forceinline__ void cand_tile_body(const Dev& d, const RuleTab* __restrict__ rtp, CandStage& S) {
  pdl_enter();
  if (aborted(d.err)) return;
  __shared__ unsigned s_mask[16];
  load_type_masks(*rtp, s_mask);
  __shared__ SurvQueue s_q[8];  // one per warp (256 threads)
  __shared__ long long s_scan[33];
  __shared__ int s_tile;
  const long long r2max = rtp->r2max;
  const CountTargets<1> tg{{d.stats + ST_CANDIDATES}, {NSTAT}};
  ReplicaCounts<1> pairs;
  ReplicaCounts<1>::begin_block();
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int* cs = d.cell_start;
  // thread 0 holds the next work item and its replica's geometry, loaded
  // while the current tile is processed
  int4 nxt = make_int4(0, 0, 0, 0);
  int nxt_id = 0, nxt_nc = 0, nxt_nz = 0, nxt_L = 0;
  auto fetch = [&]() {
    nxt_id = atomicAdd(&d.cnt->ticket[1], 1);
    if (nxt_id < d.n_ctile) {
      nxt = d.ctile[nxt_id];
      nxt_nc = d.nc[nxt.x];
      nxt_nz = d.ncz[nxt.x];
      nxt_L = (int)d.box[nxt.x];
    }
  };
  if (tid == 0) fetch();
  while (true) {
    if (tid == 0) {
      s_tile = nxt_id;
      if (nxt_id < d.n_ctile) {
        tile_params(nxt, nxt_nc, nxt_nz, nxt_L, S);
        fetch();
      }
    }
    __syncthreads();
    if (s_tile >= d.n_ctile) break;
    const int r = S.r, nc = S.nc, nz = S.nz, Zs = S.Zs, HX = S.HX, HY = S.HY;
    const int cb = (int)d.cell_base[r], ncl = (int)d.n_cells;
    // owned column runs of class c: one contiguous run of sorted entries each
    if (tid < S.n_own_cols) {
      const int gx = S.x0 + tid / S.Ty, gy = S.y0 + tid % S.Ty;
      const int k0 = S.c * ncl + cb + (gx * nc + gy) * nz + S.z0;
      const int g = cs[k0 - 1];
      S.own_g[tid] = g;
      S.own_pre[tid + 1] = cs[k0 + S.Tz - 1] - g;
    }
    bool fb = S.fallback;
    if (!fb) {
      // staged columns, a warp each: lane lz reads the end of cell lz - 1 of
      // the column's run from hz0 (and, past the end of the column, of its
      // run from z cell 0), so one coalesced load per run gives every staged
      // cell's offset within the column
      const int nA = min(Zs, nz - S.hz0), nB = Zs - nA;
      for (int col = warp; col < S.n_cols; col += nwarps) {
        const int pi = col / (HX * HY), rem = col - pi * HX * HY, lx = rem / HY, ly = rem - lx * HY;
        const int p = nth_set_bit((unsigned)S.pmask, pi);
        int gx = S.hx0 + lx, gy = S.hy0 + ly;
        if (gx >= nc) gx -= nc;
        if (gy >= nc) gy -= nc;
        const int kb = p * ncl + cb + (gx * nc + gy) * nz;
        const int rawA = lane <= nA ? cs[kb + S.hz0 + lane - 1] : 0;
        const int rawB = nB > 0 && lane <= nB ? cs[kb + lane - 1] : 0;
        const int colA = __shfl_sync(FULL, rawA, 0), endA = __shfl_sync(FULL, rawA, nA);
        const int colB = __shfl_sync(FULL, rawB, 0), endB = __shfl_sync(FULL, rawB, nB);
        const int fromB = __shfl_sync(FULL, rawB, lane > nA ? lane - nA : 0);
        const int lenA = endA - colA;
        const int off = lane <= nA ? rawA - colA : lenA + fromB - colB;
        const int tot = lenA + (nB > 0 ? endB - colB : 0);
        if (lane <= Zs) S.off[col][lane] = (unsigned short)min(off, 65535);
        if (lane == 0) {
          S.colA[col] = colA;
          S.colLenA[col] = lenA;
          S.colB[col] = colB;
          S.cbase[col] = min(tot, C_ENT_CAP + 1);  // column totals, scanned below
        }
      }
    }
    __syncthreads();
    if (!fb) {
      // column totals -> first staged entry of each column (n_cols <= blockDim)
      const int v = tid < S.n_cols ? S.cbase[tid] : 0;
      long long tot;
      const long long ex = block_excl_scan((long long)v, s_scan, &tot);
      if (tid < S.n_cols) S.cbase[tid] = (int)ex;
      if (tid == 0) S.cbase[S.n_cols] = (int)min(tot, (long long)C_ENT_CAP + 1);
      fb = tot > C_ENT_CAP;
    }
    if (warp == 0) {  // owned column runs: exclusive prefix of their lengths
      const int n = S.n_own_cols;
      const int v0 = 2 * lane < n ? S.own_pre[2 * lane + 1] : 0, v1 = 2 * lane + 1 < n ? S.own_pre[2 * lane + 2] : 0;
      const int inc = warp_incl_scan(v0 + v1);
      __syncwarp();
      if (2 * lane < n) S.own_pre[2 * lane] = inc - v0 - v1;
      if (2 * lane + 1 < n) S.own_pre[2 * lane + 1] = inc - v1;
      if (lane == 31) S.own_pre[n] = inc;
    }
    __syncthreads();
    if (!fb) {
      // the staged entries, 16 bytes each, a warp per column
      for (int col = warp; col < S.n_cols; col += nwarps) {
        const int base = S.cbase[col], len = S.cbase[col + 1] - base;
        const int a = S.colA[col], la = S.colLenA[col], bq = S.colB[col];
        for (int q = lane; q < len; q += 32) cp_async16(&S.ent[base + q], d.sorted + (q < la ? a + q : bq + (q - la)), true);
      }
      cp_async_commit();
      cp_async_wait<0>();
    }
    __syncthreads();
    // the owned beads, one per thread
    const int n_own = S.own_pre[S.n_own_cols];
    for (int base = 0; base < n_own; base += nthr) {
      const int fo = base + tid;
      int e = -1, i = -1, ti = 0, np = 0;
      int pj[MAXC];
      long long pd[MAXC];
      uint4 si = make_uint4(0, 0, 0, 0);
      LocalList ll;
      ll.cnt = ll.pairs = 0;
      ll.overflow = false;
      if (fo < n_own) {
        const int oc = smem_upper(S.own_pre, S.n_own_cols, fo);
        e = S.own_g[oc] + (fo - S.own_pre[oc]);
        const int4 me = d.sorted[e];
        i = me.w >> 4;
        ti = me.w & 15;
        ll.me = i;
        if (fb) {
          scan_candidates<GEO>(d, rtp, s_mask[ti], r2max, me, i, &ll, 0, nullptr, pj, pd, &np);
        } else {
          bool more = false;
          scan_staged<GEO>(S, r2max, d.reach, me, i, pj, pd, np, more);
          ll.overflow = more;  // finished exactly by k_cand_overflow
          if (more) np = 0;
        }
        if (np) si = d.slots[i];
      }
      warp_survivors(d, rtp, i, ti, si, pj, pd, np, &ll, s_q[warp]);
      emit_list(d, e, i, ll);
      if (fo < n_own && !ll.overflow) pairs.add(tg, r, 0, ll.pairs);
    }
    __syncthreads();  // the stage is reused by the next tile
  }
  pairs.end_warp(tg);
}

__global__ void __launch_bounds__(256, 3) k_candidates_tile(Dev d, const RuleTab* __restrict__ rtp) {
  extern __shared__ __align__(16) unsigned char ct_smem[];
  cand_tile_body<0>(d, rtp, *reinterpret_cast<CandStage*>(ct_smem));
}
__global__ void __launch_bounds__(256, 3) k_candidates_tile_oct(Dev d, const RuleTab* __restrict__ rtp) {
  extern __shared__ __align__(16) unsigned char ct_smem[];
  cand_tile_body<1>(d, rtp, *reinterpret_cast<CandStage*>(ct_smem));
}

// Exact path for beads with more than MAXC candidates: count, allocate,
// write, then sort the bead's list by (d2, partner) in place.
__device__ __forceinline__ void cand_overflow_body(const Dev& d, const RuleTab* __restrict__ rtp) {
  if (ld_cg(&d.cnt->n_ovf) == 0) return;  // the common case: nothing overflowed (every thread reads the same count)
  __shared__ unsigned s_mask[16];
  load_type_masks(*rtp, s_mask);
  const long long r2max = rtp->r2max;
  const int n = d.cnt->n_ovf;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int4 me = d.sorted[d.ovf[k]];
    int i = me.w >> 4;
    LocalList cv;
    cv.cnt = cv.pairs = 0;
    cv.me = i;
    int pj[MAXC], np = 0;
    long long pd[MAXC];
    scan_candidates<0>(d, rtp, s_mask[me.w & 15], r2max, me, i, &cv, 1, nullptr, pj, pd, &np);
    const int a = atomicAdd(&d.cnt->cand_used, cv.cnt);
    if ((long long)a + cv.cnt > d.cand_pool) {
      atomicOr(d.err, ERR_CAND_CAP);
      continue;
    }
    const long long at = d.cand_fixed + a;
    int pairs = cv.pairs;
    int4* w = d.cand + at;
    scan_candidates<0>(d, rtp, s_mask[me.w & 15], r2max, me, i, &cv, 2, &w, pj, pd, &np);
    int4* lst = d.cand + at;
    for (int a = 1; a < cv.cnt; ++a) {
      int4 x = lst[a];
      long long kx = ((long long)x.w << 32) | (unsigned)x.z;
      int b = a;
      while (b > 0) {
        int4 y = lst[b - 1];
        long long ky = ((long long)y.w << 32) | (unsigned)y.z;
        if (ky < kx || (ky == kx && y.x < x.x)) break;
        lst[b] = y;
        --b;
      }
      lst[b] = x;
    }
    // more than MAXC beads within the reach need not leave any candidate
    // once the rule, maxbond and graph-distance tests run: such a bead takes
    // no part in the matching (its nomination would read a stale entry)
    if (cv.cnt > 0) activate_creator(d, i, (int)at, cv.cnt, lst[0].x);
    stat_add(d, rep_of(d, i), ST_CANDIDATES, pairs);
  }
}

__global__ void __launch_bounds__(128) k_cand_overflow(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_enter();
  if (aborted(d.err)) return;
  cand_overflow_body(d, rtp);
}

// ---------------------------------------------------------------------------
// k_match: rounds of mutual nomination (creation: nearest partner; breakage:
// most distant; ties to the lower partner id), until a round matches nothing
// or max_rounds rounds.  Per-bead lists are sorted, so a bead's nominee is
// its first entry whose partner is still unmatched.
// ---------------------------------------------------------------------------
// First entry, from position p on, of bead i's list (system sys) whose
// partner was unmatched when round `round` began; p is left at it (or at the
// list's end, returning -1).
__device__ __forceinline__ int first_open(const Dev& d, int sys, int i, int& p, int round) {
  const long long o = sys ? d.N : 0;
  const int len = sys ? d.brk_len[i] : d.cand_len[i];
  const int4* lst = sys ? d.brk + 4 * (long long)i : d.cand + d.cand_start[i];
  // FO_BATCH list entries and then their partners' match states are loaded
  // together, so skipping matched partners costs no extra dependent loads
  for (; p < len; p += FO_BATCH) {
    int q[FO_BATCH];
    long long m[FO_BATCH];
#pragma unroll
    for (int u = 0; u < FO_BATCH; ++u) q[u] = p + u < len ? lst[p + u].x : -1;
#pragma unroll
    for (int u = 0; u < FO_BATCH; ++u) m[u] = q[u] >= 0 ? __ldcg(d.mate + o + q[u]) : 0;
#pragma unroll
    for (int u = 0; u < FO_BATCH; ++u)
      if (q[u] >= 0 && (m[u] < 0 || (m[u] >> 32) == round)) {
        p += u;
        return q[u];
      }
  }
  p = len;
  return -1;
}

// Flag replica r (-1: none) as having matched in this round (flags of round
// k live in buffer k & 1, so block 0 can count and clear one round's flags
// while the next round sets the other buffer's).
__device__ __forceinline__ void flag_round(const Dev& d, int round, int sys, int r) {
  if (r >= 0) d.round_hit[(round & 1) * 2 * d.R + sys * d.R + r] = 1;
}

// Rounds run over the grid with warp-level list appends and counters (no
// block barrier inside a round) and one bounded grid barrier between rounds;
// once few beads are left, block 0 finishes alone with block barriers.
__device__ __forceinline__ void match_body(const Dev& d, const RuleTab* __restrict__ rtp, unsigned* bar) {
  constexpr int MQ = 4;                              // round-0 jobs per lane and pass
  __shared__ int s_mq[MATCH_THREADS / 32][32 * 32];  // round-0 job queue per warp (32 words x 32 beads)
  const RuleTab& rt = *rtp;
  const long long N = d.N;
  const int R = d.R;
  const int lane = threadIdx.x & 31;
  const CountTargets<2> tg{{d.stats + ST_CREATE_MATCHED, d.stats + ST_BREAK_MATCHED}, {NSTAT, NSTAT}};
  ReplicaCounts<2> matched_pairs;
  int n = 0, round = 0;
  bool solo = false;
  int nb = gridDim.x, bi = blockIdx.x;  // participating blocks, this block's rank
  while (true) {
    const int* src = round ? d.live[(round - 1) & 1] : nullptr;
    int* dst = d.live[round & 1];
    int hits = 0;            // pairs (i < j) this thread matched in this round
    int hr[2] = {-1, -1};    // replica of those pairs, per system (flagged when it changes)
    auto count_hit = [&](int sys, int i) {
      const int r = rep_of(d, i);
      ++hits;
      matched_pairs.add(tg, r, sys, 1);
      if (hr[sys] != r) {
        flag_round(d, round, sys, hr[sys]);
        hr[sys] = r;
      }
    };
    const int tthreads = nb * blockDim.x, tid = bi * blockDim.x + threadIdx.x;
    if (round == 0) {
      // nominations were written by the list producers; a mutual pair is a
      // match, an unmatched nominator carries over.  Each lane reads one
      // bitmap word; the warp queues the (bead, system) jobs of its 32 words
      // in shared memory and takes them MQ per lane at a time, every load of
      // a pass issued together, so a word with many active beads does not
      // hold its warp for one dependent chain per bead.
      int* q = s_mq[threadIdx.x >> 5];
      for (long long w0 = (long long)tid - lane; w0 < d.W; w0 += tthreads) {
        const long long w = w0 + lane;
        unsigned ca = 0, bn = 0;
        if (w < d.W) {
          const long long b0 = 32 * w;  // the last word may extend past N
          const unsigned vmask = b0 + 32 <= N ? FULL : (b0 >= N ? 0u : (1u << (N - b0)) - 1u);
          ca = d.bm_ca[w] & vmask;
          bn = d.bm_bn[w] & vmask;
        }
        // job = bead | creation bit << 28 | breakage bit << 29 (beads < 2^28)
        unsigned todo = ca | bn;
        const int nj = __popc(todo);
        const int incl = warp_incl_scan(nj);
        const int total = __shfl_sync(FULL, incl, 31);
        for (int at = incl - nj; todo; todo &= todo - 1) {
          const int bit = __ffs(todo) - 1;
          q[at++] = (int)(32 * w + bit) | (int)(((ca >> bit) & 1u) << 28) | (int)(((bn >> bit) & 1u) << 29);
        }
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32 * MQ) {
          int job[MQ], j[MQ][2], back[MQ][2];
#pragma unroll
          for (int u = 0; u < MQ; ++u) {
            const int t = t0 + u * 32 + lane;
            job[u] = t < total ? q[t] : 0;
          }
#pragma unroll
          for (int u = 0; u < MQ; ++u)
#pragma unroll
            for (int sys = 0; sys < 2; ++sys)
              j[u][sys] = (job[u] >> (28 + sys)) & 1 ? d.nom[(sys ? N : 0) + (job[u] & 0x0FFFFFFF)] : -1;
#pragma unroll
          for (int u = 0; u < MQ; ++u)
#pragma unroll
            for (int sys = 0; sys < 2; ++sys)
              back[u][sys] = j[u][sys] >= 0 ? ld_cg(d.nom + (sys ? N : 0) + j[u][sys]) : -1;
          int want = 0;
#pragma unroll
          for (int u = 0; u < MQ; ++u) {
            const int i = job[u] & 0x0FFFFFFF;
#pragma unroll
            for (int sys = 0; sys < 2; ++sys) {
              if (j[u][sys] < 0) continue;
              if (back[u][sys] == i) {
                d.mate[(sys ? N : 0) + i] = mate_pack(0, j[u][sys]);
                if (i < j[u][sys]) count_hit(sys, i);
                j[u][sys] = -1;  // matched: no carry
              } else {
                ++want;
              }
            }
          }
          int at = warp_alloc(&d.cnt->round_live[0], want);
#pragma unroll
          for (int u = 0; u < MQ; ++u) {
            const int i = job[u] & 0x0FFFFFFF;
            if (j[u][0] >= 0) dst[at++] = i;
            if (j[u][1] >= 0) dst[at++] = (int)(1u << 31 | (unsigned)i);
          }
        }
        __syncwarp();
      }
    } else {
      // One phase per round: a live bead's nominee is its first list entry
      // that was unmatched when the round began (a match stamped with this
      // round does not count yet), and the nominee's own nominee is found
      // the same way from the nominee's list; a mutual pair is a match.  The
      // two ends decide alike, so a round needs a single barrier.
      for (int base = tid - lane; base < n; base += tthreads) {
        const int idx = base + lane;
        bool keep = false;
        int e = 0;
        if (idx < n) {
          e = src[idx];
          const int sys = (unsigned)e >> 31, i = e & 0x7FFFFFFF;
          const long long o = sys ? N : 0;
          int p = ld_cg(d.ptr + o + i);  // written in an earlier round, maybe on another SM
          const int j = first_open(d, sys, i, p, round);
          d.ptr[o + i] = p;
          if (j >= 0) {
            // the nominee's pointer only ever skips partners matched before
            // this round, whichever value is read
            int pj = ld_cg(d.ptr + o + j);
            if (first_open(d, sys, j, pj, round) == i) {
              d.mate[o + i] = mate_pack(round, j);
              if (i < j) count_hit(sys, i);
            } else {
              keep = true;
            }
          }
        }
        const int at = warp_alloc(&d.cnt->round_live[round], keep ? 1 : 0);
        if (keep) dst[at] = e;
      }
    }
    // pairs matched in the round (one atomic per warp), replicas that matched any
    const int wh = __reduce_add_sync(FULL, hits);
    if (lane == 0 && wh) atomicAdd(&d.cnt->round_matched[round], wh);
    flag_round(d, round, 0, hr[0]);
    flag_round(d, round, 1, hr[1]);
    if (solo) __syncthreads();
    else if (!grid_sync(bar, d.spin_limit, d.err)) return;
    const int matched = ld_cg(&d.cnt->round_matched[round]);
    if (blockIdx.x == 0) {
      int* flags = d.round_hit + (round & 1) * 2 * R;
      for (int k = threadIdx.x; k < 2 * R; k += blockDim.x) {
        if (ld_cg(flags + k)) {
          d.stats[(long long)(k % R) * NSTAT + (k < R ? ST_CREATE_ROUNDS : ST_BREAK_ROUNDS)] += 1;
          flags[k] = 0;
        }
      }
    }
    n = ld_cg(&d.cnt->round_live[round]);
    ++round;
    if (matched == 0 || n == 0) break;
    if (rt.max_rounds && round >= rt.max_rounds) break;
    if (round >= MAX_ROUNDS) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(d.err, ERR_ROUNDS);
      break;
    }
    if (!solo && n <= SOLO_LIVE) {
      if (blockIdx.x != 0) {
        matched_pairs.flush_block(tg);
        return;
      }
      solo = true;
      nb = 1;
      bi = 0;
    }
  }
  matched_pairs.flush_block(tg);
  if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt->rounds_done = round;
}

__global__ void __launch_bounds__(MATCH_THREADS) k_match(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_wait();  // cooperative: its successor is scheduled only when it ends
  if (aborted(d.err)) return;
  match_body(d, rtp, d.cnt->bar);
}

// ---------------------------------------------------------------------------
// k_edit: trials and in-place edit of each bead's own slots.  Only beads
// marked creation- or breakage-active are visited (bitmap compaction).
// ---------------------------------------------------------------------------
struct EditOut {
  bool dirty = false, fresh = false;
  int form_hi = -1, conv_hi = -1;
  unsigned n_killed = 0, n_broken = 0, n_conv = 0, n_formed = 0;
};

__device__ __forceinline__ void edit_bead(const Dev& d, const RuleTab& rt, long long i, int r, bool ca, bool ba,
                                          EditOut& o) {
  const long long N = d.N;
  uint4 s = d.slots[i];
  unsigned removed = 0, changed = 0;
  int conv_partner = -1, form_partner = -1, form_type = 0;
  // the per-bead words of both systems are read together, before any of them
  // is needed (one round trip instead of a chain)
  long long mb = -1, mc = -1;
  int pb = 0, pc = 0, cs = 0;
  unsigned km = 0, bl = 0;
  if (ba) {
    km = d.killmask[i];
    bl = d.brk_len[i];
    mb = d.mate[N + i];
    pb = d.ptr[N + i];
  }
  if (ca) {
    mc = d.mate[i];
    pc = d.ptr[i];
    cs = d.cand_start[i];
  }
  if (ba) {
    removed = km;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q)
      if ((removed >> q) & 1u) o.n_killed += s_partner(s_get(s, q)) > i;
    int j = bl ? mate_partner(mb) : -1;
    if (j >= 0) {
      int4 ent = d.brk[4 * i + pb];
      int k = ent.y;
      int a = (int)min((long long)j, i), b = (int)max((long long)j, i);
      if (trial(d, rt, a, b, r, TAG_BREAK, d.T_break[(long long)r * MAXR + k])) {
        int q = 0;
        while (q < SLOTS && s_partner(s_get(s, q)) != j) ++q;
        bool killed = q < SLOTS && ((removed >> q) & 1u);
        if (q == SLOTS) {
          atomicOr(d.err, ERR_INTERNAL);
        } else if (rt.kind[k] == DYNBOND_BREAKBOND) {
          removed |= 1u << q;
          o.n_broken += !killed && j > i;
        } else if (!killed) {
          changed |= 1u << q;
          s_set(s, q, ((unsigned)j << 4) | (unsigned)rt.type2[k]);
          conv_partner = j;
          o.n_conv += j > i;
        }
      }
    }
  }
  if (ca) {
    int j = mate_partner(mc);
    if (j >= 0) {
      int4 ent = d.cand[cs + pc];
      int k = ent.y & 0xFF;
      int a = (int)min((long long)j, i), b = (int)max((long long)j, i);
      if (trial(d, rt, a, b, r, TAG_FORM, d.T_form[(long long)r * MAXR + k])) {
        form_partner = j;
        form_type = (ent.y >> 8) & 15;
        o.n_formed += j > i;
      }
    }
    if (form_partner == (int)i) {  // a matching that paired a bead with itself: report, never form it
      atomicOr(d.err, ERR_INTERNAL);
      form_partner = -1;
    }
  }
  if (!(removed | changed | (unsigned)(form_partner >= 0))) return;
  uint4 ns = make_uint4(0, 0, 0, 0);
  int4 rp = make_int4(-1, -1, -1, -1);
  int nk = 0, nr = 0;
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    unsigned v = s_get(s, q);
    if (!v) continue;
    if (((removed | changed) >> q) & 1u) {
      if (nr == 0) rp.x = s_partner(v);
      else if (nr == 1) rp.y = s_partner(v);
      else if (nr == 2) rp.z = s_partner(v);
      else rp.w = s_partner(v);
      ++nr;
      if ((removed >> q) & 1u) continue;
    }
    s_set(ns, nk++, v);
  }
  if (form_partner >= 0) {
    if (nk >= SLOTS) atomicOr(d.err, ERR_SLOTS);
    else s_set(ns, nk++, ((unsigned)form_partner << 4) | (unsigned)form_type);
  }
  d.slots[i] = ns;
  // the bead's bonds changed: refresh its bits in the two bead bitmaps
  {
    const int bt = d.type[i];
    const unsigned bit = 1u << (i & 31);
    if (creation_eligible(rt, bt, ns)) atomicOr(&d.bm_elig[i >> 5], bit);
    else atomicAnd(&d.bm_elig[i >> 5], ~bit);
    if (holds_breakable(rt, bt, ns)) atomicOr(&d.bm_bk[i >> 5], bit);
    else atomicAnd(&d.bm_bk[i >> 5], ~bit);
  }
  o.dirty = (removed | changed) != 0;
  o.fresh = form_partner >= 0 || conv_partner >= 0;
  if (o.dirty) d.rem[i] = rp;
  if (o.fresh) d.newp[i] = make_int2(form_partner, conv_partner);
  if (form_partner > i) o.form_hi = form_partner;
  if (conv_partner > i) o.conv_hi = conv_partner;
}

__device__ __forceinline__ void edit_body(const Dev& d, const RuleTab* __restrict__ rtp) {
  const RuleTab& rt = *rtp;
  const CountTargets<5> tg{{d.stats + ST_KILLED, d.stats + ST_BROKEN, d.stats + ST_CONVERTED, d.stats + ST_FORMED,
                            d.n_bonds},
                           {NSTAT, NSTAT, NSTAT, NSTAT, 1}};
  ReplicaCounts<5> counts;
  const long long nchunks = (d.W + CHUNK_WORDS - 1) / CHUNK_WORDS;
  const long long cpb = (nchunks + gridDim.x - 1) / gridDim.x;
  const long long c0 = (long long)blockIdx.x * cpb, c1 = min(nchunks, c0 + cpb);
  for_bits_block(d.bm_ca, d.bm_ba, d.W, d.N, c0, c1, [&](bool valid, long long i, bool ca, bool ba) {
    EditOut o;
    int r = 0;
    if (valid) {
      r = rep_of(d, i);
      edit_bead(d, rt, i, r, ca, ba, o);
      counts.add(tg, r, 0, o.n_killed);
      counts.add(tg, r, 1, o.n_broken);
      counts.add(tg, r, 2, o.n_conv);
      counts.add(tg, r, 3, o.n_formed);
      counts.add(tg, r, 4, (long long)o.n_formed - (long long)o.n_broken - (long long)o.n_killed);
      if (o.dirty) {
        atomicOr(&d.bm_dirty[i >> 5], 1u << (i & 31));
        const long long cb = (i >> 5) >> d.dc_shift;
        atomicOr(&d.bm_dirtyc[cb >> 5], 1u << (cb & 31));
      }
      if (o.fresh) atomicOr(&d.bm_new[i >> 5], 1u << (i & 31));
    }
    // new-bond list for the rebuild: bonds formed or retyped, listed by
    // their lower end
    const bool nf = o.form_hi >= 0, nv = o.conv_hi >= 0;
    int at = block_alloc(&d.cnt->n_nbl, (int)nf + (int)nv);
    if (nf) d.nbl[at++] = make_int4((int)i, o.form_hi, r, 0);
    if (nv) d.nbl[at] = make_int4((int)i, o.conv_hi, r, 0);
  });
  counts.flush_block(tg);
}

__global__ void __launch_bounds__(256) k_edit(Dev d, const RuleTab* __restrict__ rtp) {
  pdl_enter();
  if (aborted(d.err)) return;
  edit_body(d, rtp);
}

// per-replica tile bases: base[r] = tiles of replicas before r, base[R] = all
__device__ void block_tile_bases(const int* count, int R, int per_tile, int* base, int* first) {
  __shared__ long long sh[33];
  __shared__ long long carry, carry2;
  if (threadIdx.x == 0) {
    carry = 0;
    carry2 = 0;
  }
  __syncthreads();
  for (int r0 = 0; r0 < R; r0 += blockDim.x) {
    int r = r0 + threadIdx.x;
    long long c = r < R ? count[r] : 0;
    long long tiles = (c + per_tile - 1) / per_tile;
    long long tot, tot2;
    long long ex = block_excl_scan(tiles, sh, &tot);
    long long ex2 = first ? block_excl_scan(c, sh, &tot2) : 0;
    if (r < R) {
      base[r] = (int)(carry + ex);
      if (first) first[r] = (int)(carry2 + ex2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry += tot;
      if (first) carry2 += tot2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) base[R] = (int)carry;
}

// ---------------------------------------------------------------------------
// Interaction-list maintenance (Appendix steps 6 and 9).  The order of the
// records inside a replica's angle / dihedral list carries no meaning (the
// exported topology is sorted), so the lists stay dense without any ordered
// scan or look-back chain:
//   k_allbonds  every bond (u, v), u < v, of the initial graph (creation)
//   k_purge     lists the position of every record holding a bond removed or
//               retyped in this call: m of the replica's n records go
//   k_fill      moves the surviving records of the tail [n - m, n) into the
//               holes below n - m; the i-th hole and the i-th mover to arrive
//               meet at rendezvous word i, and the second one moves the record
//   k_rebuild   appends the typed records of every path through a new bond
//               after the n - m kept ones; its last block finalizes the
//               counts, the statistics and the force tiles
// New bonds are listed by k_edit (or k_allbonds) as (u, v, replica, 0).
// ---------------------------------------------------------------------------

// Last block of the grid to get here (after all its threads' writes are
// visible device-wide); the caller then finishes the per-replica work alone.
__device__ __forceinline__ bool last_block(int* done) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

__global__ void __launch_bounds__(256) k_allbonds(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  const long long N = d.N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += stride) {
    long long u = base + threadIdx.x;
    int out[SLOTS], n = 0, r = 0;
    if (u < N) {
      uint4 su = d.slots[u];
      r = rep_of(d, u);
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        int v = s_partner(s_get(su, q));
        if (v > u) out[n++] = v;
      }
    }
    int at = warp_alloc(&d.cnt->n_nbl, n);
    for (int q = 0; q < n; ++q) d.nbl[at + q] = make_int4((int)u, out[q], r, 0);
  }
}

__device__ __forceinline__ bool is_dirty(const Dev& d, int x) { return (d.bm_dirty[x >> 5] >> (x & 31)) & 1u; }

__device__ __forceinline__ bool bond_gone(const Dev& d, int a, int b) {
  if (!is_dirty(d, a) || !is_dirty(d, b)) return false;
  int4 rp = d.rem[a];
  return rp.x == b || rp.y == b || rp.z == b || rp.w == b;
}

// Might bead x be dirty?  The coarse bitmap in shared memory (one bit per
// 32 << dc_shift beads) is clear for every bead range without a dirty bead.
__device__ __forceinline__ bool maybe_dirty(const unsigned* s_coarse, int shift, int x) {
  const int b = (x >> 5) >> shift;
  return (s_coarse[b >> 5] >> (b & 31)) & 1u;
}

// Does the record hold a bond removed or retyped in this call (step 6)?
// Every bond of an angle contains its middle bead, every bond of a dihedral
// one of its two middle beads, so those beads' dirty bits decide most records.
__device__ __forceinline__ bool record_gone(const Dev& d, const int4& v, bool dih) {
  if (!dih) return is_dirty(d, v.y) && (bond_gone(d, v.x, v.y) || bond_gone(d, v.y, v.z));
  const bool db = is_dirty(d, v.y), dc = is_dirty(d, v.z);
  if (!db && !dc) return false;
  return bond_gone(d, v.x, v.y) || bond_gone(d, v.y, v.z) || bond_gone(d, v.z, v.w & 0x0FFFFFFF);
}

// the same, the coarse bits in shared memory checked first
__device__ __forceinline__ bool record_gone(const Dev& d, const unsigned* s_coarse, const int4& v, bool dih) {
  if (!dih) return maybe_dirty(s_coarse, d.dc_shift, v.y) && is_dirty(d, v.y) &&
                   (bond_gone(d, v.x, v.y) || bond_gone(d, v.y, v.z));
  if (!maybe_dirty(s_coarse, d.dc_shift, v.y) && !maybe_dirty(s_coarse, d.dc_shift, v.z)) return false;
  return record_gone(d, v, dih);
}

__device__ __forceinline__ void purge_body(const Dev& d) {
  __shared__ unsigned s_coarse[PURGE_COARSE_WORDS];
  for (long long k = threadIdx.x; k < d.Wc; k += blockDim.x) s_coarse[k] = d.bm_dirtyc[k];
  __syncthreads();
  const int R = d.R;
  const int na_tiles = d.tb_ang[R];
  const int ntiles = na_tiles + d.tb_dih[R];
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int tg = blockIdx.x; tg < ntiles; tg += gridDim.x) {
    // tiles [0, na_tiles) scan the angle lists, the rest the dihedral lists
    const bool dih = tg >= na_tiles;
    const int t = dih ? tg - na_tiles : tg;
    const int* tb = dih ? d.tb_dih : d.tb_ang;
    const int r = find_seg_warp(tb, R, t);
    const long long base = (dih ? 18 : 6) * d.off[r];
    const int4* recs = (dih ? d.dih : d.ang) + base;
    const int n = (dih ? d.n_dih : d.n_ang)[r];
    const int beg = (t - tb[r]) * PURGE_TILE + threadIdx.x;
    int4 v[PURGE_PER_THREAD];
#pragma unroll
    for (int k = 0; k < PURGE_PER_THREAD; ++k) {
      int idx = beg + k * (int)blockDim.x;
      if (idx < n) v[k] = recs[idx];
    }
    unsigned bal[PURGE_PER_THREAD];
    int tot = 0;
#pragma unroll
    for (int k = 0; k < PURGE_PER_THREAD; ++k) {
      int idx = beg + k * (int)blockDim.x;
      bal[k] = __ballot_sync(FULL, idx < n && record_gone(d, s_coarse, v[k], dih));
      tot += __popc(bal[k]);
    }
    // one atomic per tile (the tile lies in one replica)
    int wbase = block_alloc((dih ? d.m_dih : d.m_ang) + r, lane == 0 ? tot : 0);
    wbase = __shfl_sync(FULL, wbase, 0);
    int* rm = (dih ? d.rm_dih : d.rm_ang) + base;
    int* pr = (dih ? d.pr_dih : d.pr_ang) + base;
#pragma unroll
    for (int k = 0; k < PURGE_PER_THREAD; ++k) {
      if ((bal[k] >> lane) & 1u) {
        int at = wbase + __popc(bal[k] & lt_mask);
        rm[at] = beg + k * (int)blockDim.x;
        pr[at] = 0;  // rendezvous word of k_fill
      }
      wbase += __popc(bal[k]);
    }
  }
  // the last block sizes k_fill: per replica, m holes-or-not and m tail
  // positions of each list
  if (!last_block(&d.cnt->done[0])) return;
  for (int r = threadIdx.x; r < R; r += blockDim.x) d.fill_items[r] = 2 * (ld_cg(d.m_ang + r) + ld_cg(d.m_dih + r));
  __syncthreads();
  block_tile_bases(d.fill_items, R, FILL_TILE, d.tb_fill, nullptr);
}

__global__ void __launch_bounds__(PURGE_TILE / PURGE_PER_THREAD) k_purge(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  purge_body(d);
}

__device__ __forceinline__ void fill_body(const Dev& d) {
  const int R = d.R;
  const int ntiles = d.tb_fill[R];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r = find_seg_warp(d.tb_fill, R, t);
    const int k = (t - d.tb_fill[r]) * FILL_TILE + threadIdx.x;
    const int ma = d.m_ang[r], md = d.m_dih[r];
    // item k: [0, ma) removed angles, [ma, 2 ma) the angle tail, then the
    // same for the dihedrals
    const bool dih = k >= 2 * ma;
    const int kk = dih ? k - 2 * ma : k;
    const int m = dih ? md : ma;
    const long long base = (dih ? 18 : 6) * d.off[r];
    int4* recs = (dih ? d.dih : d.ang) + base;
    const int keep = (dih ? d.n_dih : d.n_ang)[r] - m;
    int role = -1, pos = 0;  // role 0 / 1: angle hole / mover, 2 / 3: dihedral
    if (kk < m) {
      int p = (dih ? d.rm_dih : d.rm_ang)[base + kk];
      if (p < keep) {
        role = dih ? 2 : 0;
        pos = p;
      }
    } else if (kk < 2 * m) {
      int p = keep + (kk - m);
      if (!record_gone(d, recs[p], dih)) {
        role = dih ? 3 : 1;
        pos = p;
      }
    }
    const int at = block_alloc4(&d.fillc[4 * r], role);  // the tile lies in one replica
    if (role < 0) continue;
    int code = (role & 1) ? -(pos + 1) : pos + 1;
    int other = atomicExch((dih ? d.pr_dih : d.pr_ang) + base + at, code);
    if (other != 0) {  // both ends arrived: move the tail record into the hole
      int hole = code > 0 ? code - 1 : other - 1;
      int mover = code < 0 ? -code - 1 : -other - 1;
      recs[hole] = recs[mover];
    }
  }
}

__global__ void __launch_bounds__(FILL_TILE) k_fill(Dev d) {
  pdl_enter();
  if (aborted(d.err)) return;
  fill_body(d);
}

// ---------------------------------------------------------------------------
// k_rebuild: typed angle / dihedral records of every non-cyclic path of the
// new bond graph that contains a new bond (Appendix step 9; typing rules of
// Sec. 2).  A path holding several new bonds is written by its lowest one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long bkey(int a, int b) {
  return a < b ? ((unsigned long long)(unsigned)a << 32) | (unsigned)b
               : ((unsigned long long)(unsigned)b << 32) | (unsigned)a;
}

struct Rebuild {
  const Dev& d;
  const RuleTab& rt;
  int all_new;
  __device__ bool is_new(int p, int q) const {
    if (all_new) return true;
    if (!((d.bm_new[p >> 5] >> (p & 31)) & 1u) || !((d.bm_new[q >> 5] >> (q & 31)) & 1u)) return false;
    int2 np = d.newp[p];
    return np.x == q || np.y == q;
  }
  // true if another bond (p, q) of the path is new and ranks below (u, v)
  __device__ bool outranked(int p, int q, unsigned long long kuv) const { return bkey(p, q) < kuv && is_new(p, q); }

  // part 0: angles centred at u; 1: angles centred at v; 2: dihedrals with
  // (u, v) in the middle; 3 / 4: dihedrals starting at u / at v.  The parts
  // are independent and run on different threads.
  template <class Emit>
  __device__ void run(int u, int v, int part, Emit& emit) const {
    const unsigned long long kuv = bkey(u, v);
    uint4 su = d.slots[u], sv = d.slots[v];
    int tu = d.type[u], tv = d.type[v];
    int st_uv = s_type_to(su, v), st_vu = s_type_to(sv, u);
    // angles centred at u: (x, u, v) and at v: (u, v, y)
    if (part == 0)
    for (int q = 0; q < SLOTS; ++q) {
      unsigned w = s_get(su, q);
      int x = s_partner(w);
      if (x < 0 || x == v || outranked(x, u, kuv)) continue;
      int t = angle_type(rt, d.type[x], tu, tv, s_type(w), st_uv);
      if (t) emit.angle(min(x, v), u, max(x, v), t);
    }
    if (part == 1)
    for (int q = 0; q < SLOTS; ++q) {
      unsigned w = s_get(sv, q);
      int y = s_partner(w);
      if (y < 0 || y == u || outranked(v, y, kuv)) continue;
      int t = angle_type(rt, tu, tv, d.type[y], st_vu, s_type(w));
      if (t) emit.angle(min(u, y), v, max(u, y), t);
    }
    // dihedrals with (u, v) in the middle: (x, u, v, y)
    if (part == 2)
    for (int q = 0; q < SLOTS; ++q) {
      unsigned wx = s_get(su, q);
      int x = s_partner(wx);
      if (x < 0 || x == v || outranked(x, u, kuv)) continue;
      int tx = d.type[x];
      for (int q2 = 0; q2 < SLOTS; ++q2) {
        unsigned wy = s_get(sv, q2);
        int y = s_partner(wy);
        if (y < 0 || y == u || y == x || outranked(v, y, kuv)) continue;
        // r = st(u->x), s = st(v->u), s' = st(u->v), t = st(v->y)
        int t = dihedral_type(rt, tx, tu, tv, d.type[y], s_type(wx), st_vu, st_uv, s_type(wy));
        if (t) {
          if (x < y) emit.dihedral(x, u, v, y, t);
          else emit.dihedral(y, v, u, x, t);
        }
      }
    }
    // dihedrals starting at u: (u, v, y, z) and starting at v: (v, u, x, w)
    if (part >= 3) {
      const int side = part - 3;
      int a = side ? v : u, b = side ? u : v;  // path a - b - y - z
      const uint4& sb = side ? su : sv;
      int ta = side ? tv : tu, tb = side ? tu : tv;
      int st_ba = side ? st_uv : st_vu;
      for (int q = 0; q < SLOTS; ++q) {
        unsigned wy = s_get(sb, q);
        int y = s_partner(wy);
        if (y < 0 || y == a || outranked(b, y, kuv)) continue;
        uint4 sy = d.slots[y];
        int ty = d.type[y];
        int st_yb = s_type_to(sy, b);
        for (int q2 = 0; q2 < SLOTS; ++q2) {
          unsigned wz = s_get(sy, q2);
          int z = s_partner(wz);
          if (z < 0 || z == b || z == a || outranked(y, z, kuv)) continue;
          // path (a, b, y, z): r = st(b->a), s = st(y->b), s' = st(b->y), t = st(y->z)
          int t = dihedral_type(rt, ta, tb, ty, d.type[z], st_ba, st_yb, s_type(wy), s_type(wz));
          if (t) {
            if (a < z) emit.dihedral(a, b, y, z, t);
            else emit.dihedral(z, y, b, a, t);
          }
        }
      }
    }
  }
};

struct CountEmit {
  int na = 0, nd = 0;
  __device__ void angle(int, int, int, int) { ++na; }
  __device__ void dihedral(int, int, int, int, int) { ++nd; }
};
struct WriteEmit {
  int4* ang;
  int4* dih;
  const int4* ang_end;  // end of the replica's region (worst-case capacity)
  const int4* dih_end;
  unsigned* err;
  __device__ void angle(int a, int b, int c, int t) {
    if (ang < ang_end) *ang++ = make_int4(a, b, c, t);
    else atomicOr(err, ERR_INTERNAL);
  }
  __device__ void dihedral(int a, int b, int c, int dd, int t) {
    if (dih < dih_end) *dih++ = make_int4(a, b, c, dd | (t << 28));
    else atomicOr(err, ERR_INTERNAL);
  }
};

// Room for (na, nd) records after the kept ones of replica r: one atomic pair
// per group of lanes with the same replica; offsets in lane order.
__device__ __forceinline__ void reserve(const Dev& d, int r, int na, int nd, int* oa, int* od) {
  const int lane = threadIdx.x & 31;
  unsigned grp = __match_any_sync(FULL, r);
  int pa = 0, pd = 0, ta = 0, td = 0;
  for (int l = 0; l < 32; ++l) {
    int a = __shfl_sync(FULL, na, l), b = __shfl_sync(FULL, nd, l);
    if ((grp >> l) & 1u) {
      ta += a;
      td += b;
      if (l < lane) {
        pa += a;
        pd += b;
      }
    }
  }
  int leader = __ffs(grp) - 1;
  int ba = 0, bd = 0;
  if (lane == leader && r >= 0) {
    if (ta) ba = atomicAdd(d.added_ang + r, ta);
    if (td) bd = atomicAdd(d.added_dih + r, td);
  }
  *oa = __shfl_sync(FULL, ba, leader) + pa;
  *od = __shfl_sync(FULL, bd, leader) + pd;
}

__device__ __forceinline__ void rebuild_body(const Dev& d, const RuleTab* __restrict__ rtp, int all_new) {
  const RuleTab& rt = *rtp;
  const Rebuild rb{d, rt, all_new};
  // five independent parts per new bond, part-major: the lanes of a warp run
  // the same part on consecutive bonds (convergent, and the records of a
  // chain's consecutive bonds land next to each other)
  const long long nn = d.cnt->n_nbl, n = 5 * nn;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    const bool valid = i < n;
    const int part = valid ? (int)(i / nn) : 0;
    int4 e = valid ? d.nbl[i - part * nn] : make_int4(0, 0, -1, 0);
    CountEmit ce;
    if (valid) rb.run(e.x, e.y, part, ce);
    int oa, od;
    reserve(d, e.z, ce.na, ce.nd, &oa, &od);
    if (valid && (ce.na || ce.nd)) {
      const int r = e.z;
      WriteEmit we{d.ang + 6 * d.off[r] + (d.n_ang[r] - d.m_ang[r]) + oa,
                   d.dih + 18 * d.off[r] + (d.n_dih[r] - d.m_dih[r]) + od, d.ang + 6 * d.off[r + 1],
                   d.dih + 18 * d.off[r + 1], d.err};
      rb.run(e.x, e.y, part, we);
    }
  }
  // the last block: per-replica counts and statistics (step 10), then the
  // force tiles of the final lists
  if (!last_block(&d.cnt->done[1])) return;
  for (int r = threadIdx.x; r < d.R; r += blockDim.x) {
    long long* st = d.stats + (long long)r * NSTAT;
    int ma = ld_cg(d.m_ang + r), md = ld_cg(d.m_dih + r);
    int aa = ld_cg(d.added_ang + r), ad = ld_cg(d.added_dih + r);
    int na = d.n_ang[r] - ma + aa, nd = d.n_dih[r] - md + ad;
    st[ST_ANG_REMOVED] = ma;
    st[ST_DIH_REMOVED] = md;
    st[ST_ANG_ADDED] = aa;
    st[ST_DIH_ADDED] = ad;
    d.n_ang[r] = na;
    d.n_dih[r] = nd;
    st[ST_NBONDS] = __ldcg(d.n_bonds + r);
    st[ST_NANGLES] = na;
    st[ST_NDIHEDRALS] = nd;
  }
  __syncthreads();
  block_tile_bases(d.n_ang, d.R, FORCE_TILE, d.tb_fang, nullptr);
  __syncthreads();
  block_tile_bases(d.n_dih, d.R, FORCE_TILE, d.tb_fdih, nullptr);
}

__global__ void __launch_bounds__(256) k_rebuild(Dev d, const RuleTab* __restrict__ rtp, int all_new) {
  pdl_enter();
  if (aborted(d.err)) return;
  rebuild_body(d, rtp, all_new);
}

// Per-call setup (one launch): zero the counters, the cell histogram, the
// creation-active bitmap, the per-replica scratch and the look-back status
// words; block 0 also computes the purge tile bases from the list counts.
// keep_bar: leave the persistent call's barrier counter (bar[1]) alone, for
// the setup phase of k_step_persistent, whose blocks count on it
__device__ __forceinline__ void setup_body(const Dev& d, bool keep_bar) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int* cnt = reinterpret_cast<int*>(d.cnt);
  const long long bar1 = (reinterpret_cast<const char*>(&d.cnt->bar[1]) - reinterpret_cast<const char*>(d.cnt)) /
                         (long long)sizeof(int);
  for (long long k = g; k < (long long)(sizeof(Counters) / sizeof(int)); k += stride)
    if (!keep_bar || k != bar1) cnt[k] = 0;
  {  // cell counts [0, n_keys]: 16-byte stores (the array is 256-byte aligned), then the last few words
    const long long n4 = (d.n_keys + 1) / 4;
    int4* c4 = reinterpret_cast<int4*>(d.cell_start);
    for (long long k = g; k < n4; k += stride) c4[k] = make_int4(0, 0, 0, 0);
    for (long long k = 4 * n4 + g; k <= d.n_keys; k += stride) d.cell_start[k] = 0;
  }
  for (long long k = g; k < d.W; k += stride) {
    d.bm_ca[k] = 0;
    d.bm_ba[k] = 0;
    d.bm_bn[k] = 0;
    d.bm_dirty[k] = 0;
    if (k < d.Wc) d.bm_dirtyc[k] = 0;
    d.bm_new[k] = 0;
  }
  for (long long k = g; k < d.small_words; k += stride) d.small[k] = 0;
  for (long long k = g; k < d.status_words; k += stride) d.status_all[k] = 0ull;
  if (blockIdx.x == 0) {
    block_tile_bases(d.n_ang, d.R, PURGE_TILE, d.tb_ang, nullptr);
    __syncthreads();
    block_tile_bases(d.n_dih, d.R, PURGE_TILE, d.tb_dih, nullptr);
  }
}

__global__ void __launch_bounds__(1024) k_setup(Dev d) {
  pdl_enter();
  setup_body(d, false);
}

// ---------------------------------------------------------------------------
// k_step_persistent: the whole call as one cooperative launch.  The blocks
// stay resident and run the phases of the launch sequence above one after
// another -- setup, binning, scan, scatter and breakage nomination, candidate
// search, overflow lists, matching rounds, edit, purge, hole filling,
// rebuild -- each over all blocks' work items, separated by bounded grid
// barriers on bar[1] (which keeps counting across calls: every call adds the
// same number of arrivals per block).  After a device error every phase is
// skipped but every barrier is still met.
// ---------------------------------------------------------------------------
template <int GEO>
__device__ __forceinline__ void step_persistent_body(const Dev& d, const RuleTab* __restrict__ rtp) {
  unsigned* bar = &d.cnt->bar[1];
  setup_body(d, true);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  bead_body(d, rtp);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) scan_cells_body(d);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) scatter_body(d, rtp, gridDim.x / 2);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) candidates_body<GEO>(d, rtp);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) cand_overflow_body(d, rtp);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) match_body(d, rtp, bar);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) edit_body(d, rtp);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) purge_body(d);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) fill_body(d);
  if (!grid_sync(bar, d.spin_limit, d.err)) return;
  if (!aborted(d.err)) rebuild_body(d, rtp, 0);
}

static_assert(MATCH_THREADS == 256, "the persistent call runs the matching in its 256-thread blocks");
__global__ void __launch_bounds__(256, 2) k_step_persistent(Dev d, const RuleTab* __restrict__ rtp) {
  step_persistent_body<0>(d, rtp);
}
__global__ void __launch_bounds__(256, 2) k_step_persistent_oct(Dev d, const RuleTab* __restrict__ rtp) {
  step_persistent_body<1>(d, rtp);
}

// bar_reset (nullable): the persistent call's barrier counter, restarted at
// zero before each call (it counts every block's arrivals within a call)
__global__ void k_set_args(CallArgs* a, const int4* pos, float4* force, double* ev, unsigned long long step,
                           int set_pos, int set_force, unsigned* bar_reset) {
  if (bar_reset) *bar_reset = 0u;
  if (set_pos) {
    a->pos = pos;
    a->step = step;
  }
  if (set_force) {
    a->pos = pos;
    a->force = force;
    a->ev = ev;
  }
}

}  // namespace dynbond
