// CPU ORACLE FOR THE DYNAMIC-BONDING PASS — TEST INFRASTRUCTURE ONLY.
//
// A plain, serial, deliberately slow statement of one call of the dynamic
// bonding fix of C. Svaneborg, "LAMMPS Framework for Dynamic Bonding and an
// Application Modeling DNA" (arXiv:1108.4214), and of the bonded forces on the
// resulting topology.  Only the test suite, the package smoke check and the
// benchmark's CPU-baseline leg may load it; the product path never does.  It
// shares no code, header or table with the CUDA library.
//
// The steps follow the order of the paper's Appendix ("Implementation
// details", steps 1-10):
//   step 2  creation nomination  -> creation_candidates() + match_rounds()
//   step 3  breakage nomination  -> breakage_candidates() + match_rounds()
//   step 4  aggregation          -> mutual nomination inside match_rounds()
//   step 5  breakage / killbond  -> trials, kill set
//   step 6  interaction removal  -> purge of every angle/dihedral on a removed
//                                   or converted bond
//   step 7  table update         -> bonds removed / converted
//   step 8  creation             -> trials, bonds added
//   step 9  interaction creation -> typed records for every non-cyclic 3-/4-path
//                                   of the new graph that contains a new bond
//   step 10 statistics
// Beside the call: the FP64 bonded forces of the resulting topology
// (orc_forces) and the DPD pair forces of Sec. 3 on a snapshot
// (orc_dpd_forces), each pinned by its own tests.
// Readings taken where the paper is silent or ambiguous (all listed in the
// design notes):
//   * distances: positions are int32 on a 2^-20 sigma grid, squared distances
//     are exact int64, "within r" is d2 <= floor((r*2^20)^2), "longer than r"
//     is d2 > floor((r*2^20)^2);
//   * pair eligibility for creation: beads at graph distance 1 never, 2 only
//     with paircheck13, 3 only with paircheck14, >= 4 (or unconnected) always;
//   * per pair the LAST creation rule (list order) that matches bead types,
//     distance and maxbond decides the bond types (Sec. 2, Appendix step 2);
//   * nomination keys: creation (d2, lower id, higher id) ascending, breakage
//     (-d2, lower id, higher id) ascending, i.e. nearest / most distant
//     partner, ties to the lower partner id; rounds of mutual nomination are
//     repeated until nothing matches (max_rounds = 0) or max_rounds times
//     (max_rounds = 1 is the paper's single nomination);
//   * a trial draws Philox4x32-10 (Salmon et al., SC'11) on the counter
//     (lower local id, higher local id, call index, tag << 24 | stream) and
//     succeeds iff x0 < floor(p * 2^32) (prob_mode 0) or x0 + x1 < 2 floor(p * 2^32)
//     (prob_mode 1, the paper's average of two uniforms, Appendix steps 5, 8);
//   * breakbond / convertbond / killbond act on symmetric bonds of their type
//     (both endpoints store it), as Sec. 2 describes them;
//   * several angle / dihedral rules matching one path: the first in list
//     order wins, one record per path;
//   * every bead holds at most 4 bonds (an implicit functionality cap).

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <set>
#include <utility>
#include <vector>

namespace {

constexpr int SLOTS = 4;

enum Kind {
  K_CREATEBOND = 1,
  K_CREATEDIRBOND = 2,
  K_BREAKBOND = 3,
  K_CONVERTBOND = 4,
  K_KILLBOND = 5,
  K_CREATEANGLE = 6,
  K_CREATEDIHEDRAL = 7,
  K_MAXBOND = 8,
};

// Layout mirrored by oracle/oracle.py (64 bytes).
struct ORule {
  int32_t kind;
  int32_t type;   // created / matched bond type, or angle / dihedral type
  int32_t type2;  // createdirbond second bond type, convertbond new type
  int32_t maxn;   // maxbond maximum
  uint32_t bead[4];
  uint32_t bond[3];
  uint32_t pad;
  double dist;
  double prob;
};
static_assert(sizeof(ORule) == 64, "rule layout");

using Angle = std::array<int32_t, 4>;     // (a, b, c, type), a < c
using Dihedral = std::array<int32_t, 5>;  // (a, b, c, d, type), a < d

// ---------------------------------------------------------------------------
// exact integer thresholds
// ---------------------------------------------------------------------------

// floor((dist * 2^20)^2) for a finite dist >= 0, exact: dist = M * 2^e with an
// integer mantissa M < 2^53, so the square is M^2 * 2^(2e) with M^2 < 2^106.
int64_t r2_of(double dist) {
  if (!(dist > 0.0)) return 0;
  int e = 0;
  double m = std::frexp(dist, &e);  // dist = m * 2^e, m in [0.5, 1)
  uint64_t M = (uint64_t)std::ldexp(m, 53);
  int shift = 2 * (e + 20 - 53);    // (dist*2^20)^2 = M^2 * 2^shift
  unsigned __int128 sq = (unsigned __int128)M * M;
  if (shift >= 0) {
    if (shift >= 62) return INT64_MAX;
    unsigned __int128 v = sq << shift;
    if (v > (unsigned __int128)INT64_MAX) return INT64_MAX;
    return (int64_t)v;
  }
  int s = -shift;
  if (s >= 127) return 0;
  unsigned __int128 v = sq >> s;
  if (v > (unsigned __int128)INT64_MAX) return INT64_MAX;
  return (int64_t)v;
}

// Integer threshold of a trial probability: floor(p * 2^32), clamped to [0, 2^32].
uint64_t threshold_of(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 1ull << 32;
  return (uint64_t)std::floor(p * 4294967296.0);
}

// ---------------------------------------------------------------------------
// Philox4x32-10, from the definition in Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two
// 32x32->64 multiplications with the counter words crossed and xored with the
// round key, the key advanced by the two Weyl constants between rounds.
// ---------------------------------------------------------------------------

void philox4x32_10(const uint32_t in_ctr[4], const uint32_t in_key[2], uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
  uint32_t k0 = in_key[0], k1 = in_key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = M0 * (uint64_t)c0;
    uint64_t p1 = M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { TAG_FORM = 1, TAG_BREAK = 2 };

// ---------------------------------------------------------------------------
// matching by rounds of mutual nomination (Appendix steps 2-4)
// ---------------------------------------------------------------------------

struct Edge {
  int64_t k1;  // d2 for creation, -d2 for breakage
  int32_t a, b;  // a < b (global ids)
  int32_t rule;
  int32_t ta, tb;  // stored types after creation / conversion
};

bool edge_less(const Edge& x, const Edge& y) {
  if (x.k1 != y.k1) return x.k1 < y.k1;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

// Each round: every bead that still has an edge to an unmatched partner
// nominates its smallest such edge; an edge nominated from both ends is
// matched and both beads leave.  Returns the matched edge ids; rounds_out[r]
// counts, per replica, the rounds in which that replica matched a pair.
std::vector<int> match_rounds(int64_t n_beads, const std::vector<Edge>& E, int max_rounds,
                              const std::vector<int32_t>& rep_of, std::vector<int64_t>* rounds_out) {
  std::vector<std::vector<int>> inc(n_beads);
  for (int e = 0; e < (int)E.size(); ++e) {
    inc[E[e].a].push_back(e);
    inc[E[e].b].push_back(e);
  }
  std::vector<char> matched(n_beads, 0);
  std::vector<int> result;
  for (int round = 0; max_rounds == 0 || round < max_rounds; ++round) {
    std::vector<int> nominee(n_beads, -1);
    for (int64_t x = 0; x < n_beads; ++x) {
      if (matched[x]) continue;
      int best = -1;
      for (int e : inc[x]) {
        int other = E[e].a == x ? E[e].b : E[e].a;
        if (matched[other]) continue;
        if (best < 0 || edge_less(E[e], E[best])) best = e;
      }
      nominee[x] = best;
    }
    std::vector<int> now;
    for (int64_t x = 0; x < n_beads; ++x) {
      int e = nominee[x];
      if (e < 0 || E[e].a != x) continue;
      if (nominee[E[e].b] == e) now.push_back(e);
    }
    if (now.empty()) break;
    std::set<int32_t> reps;
    for (int e : now) {
      matched[E[e].a] = matched[E[e].b] = 1;
      result.push_back(e);
      reps.insert(rep_of[E[e].a]);
    }
    if (rounds_out)
      for (int32_t r : reps) (*rounds_out)[r] += 1;
  }
  return result;
}

// ---------------------------------------------------------------------------
// the system
// ---------------------------------------------------------------------------

enum Stat {
  S_CANDIDATES, S_CREATE_MATCHED, S_FORMED, S_BREAK_CANDIDATES, S_BREAK_MATCHED, S_BROKEN, S_KILLED,
  S_CONVERTED, S_ANG_REMOVED, S_ANG_ADDED, S_DIH_REMOVED, S_DIH_ADDED, S_NBONDS, S_NANGLES, S_NDIHEDRALS,
  S_CREATE_ROUNDS, S_BREAK_ROUNDS, S_COUNT
};

struct Oracle {
  int R = 0;
  std::vector<int64_t> off, L;
  std::vector<double> fscale, bscale;
  std::vector<uint32_t> stream;
  int64_t N = 0;
  std::vector<int32_t> type, rep;
  std::vector<int32_t> nb, st;  // N*SLOTS partner / stored type, -1 = empty
  std::vector<ORule> rules;
  uint64_t seed = 0;
  int pc13 = 0, pc14 = 0, max_rounds = 0, prob_mode = 0, use_cells = 1;
  uint32_t reactive = 0xFFFF;
  std::vector<Angle> angles;
  std::vector<Dihedral> dihedrals;
  const int32_t* pos = nullptr;  // current snapshot, int32 [N*4]

  int deg(int64_t x) const {
    int d = 0;
    for (int s = 0; s < SLOTS; ++s) d += nb[x * SLOTS + s] >= 0;
    return d;
  }
  int stored(int64_t x, int64_t y) const {  // type x stores for its bond to y
    for (int s = 0; s < SLOTS; ++s)
      if (nb[x * SLOTS + s] == y) return st[x * SLOTS + s];
    return -1;
  }
  bool has(uint32_t mask, int t) const { return t >= 0 && t < 32 && ((mask >> t) & 1u); }

  int64_t d2(int64_t i, int64_t j) const {
    int64_t Lr = L[rep[i]], s = 0;
    for (int c = 0; c < 3; ++c) {
      int64_t dx = (int64_t)pos[4 * i + c] - (int64_t)pos[4 * j + c];
      if (2 * dx > Lr) dx -= Lr;
      else if (2 * dx <= -Lr) dx += Lr;
      s += dx * dx;
    }
    return s;
  }
  // minimum-image vector r_i - r_j in sigma
  void rel(int64_t i, int64_t j, double out[3]) const {
    int64_t Lr = L[rep[i]];
    for (int c = 0; c < 3; ++c) {
      int64_t dx = (int64_t)pos[4 * i + c] - (int64_t)pos[4 * j + c];
      if (2 * dx > Lr) dx -= Lr;
      else if (2 * dx <= -Lr) dx += Lr;
      out[c] = (double)dx / 1048576.0;
    }
  }

  // graph distance on the bond graph, capped at 4 (= 4 or more / unconnected)
  int graph_distance(int64_t a, int64_t b) const {
    if (a == b) return 0;
    std::vector<int64_t> frontier{a}, seen{a};
    for (int d = 1; d <= 3; ++d) {
      std::vector<int64_t> next;
      for (int64_t x : frontier)
        for (int s = 0; s < SLOTS; ++s) {
          int64_t y = nb[x * SLOTS + s];
          if (y < 0) continue;
          if (y == b) return d;
          if (std::find(seen.begin(), seen.end(), y) == seen.end()) {
            seen.push_back(y);
            next.push_back(y);
          }
        }
      frontier.swap(next);
    }
    return 4;
  }

  // Maxbond rules (Sec. 2, Appendix step 2): bead x may receive one more bond
  // stored as type t only if every maxbond rule covering (type(x), t) leaves
  // room, counting the bonds x already stores with a type in the rule's list.
  bool maxbond_ok(int64_t x, int t) const {
    if (deg(x) >= SLOTS) return false;
    for (const ORule& m : rules) {
      if (m.kind != K_MAXBOND) continue;
      if (!has(m.bead[0], type[x]) || !has(m.bond[0], t)) continue;
      int cnt = 0;
      for (int s = 0; s < SLOTS; ++s)
        if (nb[x * SLOTS + s] >= 0 && has(m.bond[0], st[x * SLOTS + s])) ++cnt;
      if (cnt >= m.maxn) return false;
    }
    return true;
  }

  // Last creation rule that matches the pair a < b at squared distance d2:
  // bead types (orientation a-as-first tried before b-as-first), distance and
  // maxbond on both ends.  Returns the rule index or -1 and the stored types.
  int creation_rule(int64_t a, int64_t b, int64_t dd, int* ta, int* tb) const {
    for (int k = (int)rules.size() - 1; k >= 0; --k) {
      const ORule& r = rules[k];
      if (r.kind != K_CREATEBOND && r.kind != K_CREATEDIRBOND) continue;
      if (dd > r2_of(r.dist)) continue;
      for (int o = 0; o < 2; ++o) {
        int64_t x = o == 0 ? a : b, y = o == 0 ? b : a;  // x plays beadtype1
        if (!has(r.bead[0], type[x]) || !has(r.bead[1], type[y])) continue;
        int tx = r.type, ty = r.kind == K_CREATEDIRBOND ? r.type2 : r.type;
        if (!maxbond_ok(x, tx) || !maxbond_ok(y, ty)) continue;
        *ta = x == a ? tx : ty;
        *tb = x == a ? ty : tx;
        return k;
      }
    }
    return -1;
  }

  bool pair_eligible(int64_t a, int64_t b) const {
    int g = graph_distance(a, b);
    if (g >= 4) return true;
    if (g == 2) return pc13 != 0;
    if (g == 3) return pc14 != 0;
    return false;
  }

  bool creates_at_all(int64_t x) const {
    if (!has(reactive, type[x])) return false;
    for (const ORule& r : rules)
      if ((r.kind == K_CREATEBOND || r.kind == K_CREATEDIRBOND) &&
          (has(r.bead[0], type[x]) || has(r.bead[1], type[x])))
        return true;
    return false;
  }

  void consider_pair(int64_t a, int64_t b, std::vector<Edge>* out) const {
    if (a > b) std::swap(a, b);
    int64_t dd = d2(a, b);
    int ta = 0, tb = 0;
    int k = creation_rule(a, b, dd, &ta, &tb);
    if (k < 0) return;
    if (!pair_eligible(a, b)) return;
    out->push_back(Edge{dd, (int32_t)a, (int32_t)b, k, ta, tb});
  }

  // Appendix step 2: every candidate creation pair (each unordered pair once).
  std::vector<Edge> creation_candidates(bool brute) const {
    std::vector<Edge> E;
    int64_t rmax2 = 0;
    for (const ORule& r : rules)
      if (r.kind == K_CREATEBOND || r.kind == K_CREATEDIRBOND) rmax2 = std::max(rmax2, r2_of(r.dist));
    for (int r = 0; r < R; ++r) {
      std::vector<int64_t> beads;
      for (int64_t x = off[r]; x < off[r + 1]; ++x)
        if (creates_at_all(x)) beads.push_back(x);
      if (brute) {
        for (size_t i = 0; i < beads.size(); ++i)
          for (size_t j = i + 1; j < beads.size(); ++j) consider_pair(beads[i], beads[j], &E);
        continue;
      }
      // plain cell list: cells at least as wide as the largest creation radius
      int64_t w = (int64_t)std::ceil(std::sqrt((double)rmax2));
      while (w * w < rmax2) ++w;
      while (w > 1 && (w - 1) * (w - 1) >= rmax2) --w;
      int64_t nc = w > 0 ? L[r] / w : 1;
      nc = std::max<int64_t>(1, std::min<int64_t>(nc, 200));  // wider cells stay correct
      auto cell_of = [&](int64_t x) {
        int64_t c[3];
        for (int k = 0; k < 3; ++k) c[k] = (int64_t)pos[4 * x + k] * nc / L[r];
        return (c[0] * nc + c[1]) * nc + c[2];
      };
      // counting sort of the beads by cell
      std::vector<int64_t> start((size_t)(nc * nc * nc + 1), 0), sorted(beads.size());
      for (int64_t x : beads) start[(size_t)cell_of(x) + 1] += 1;
      for (size_t c = 1; c < start.size(); ++c) start[c] += start[c - 1];
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (int64_t x : beads) sorted[(size_t)fill[(size_t)cell_of(x)]++] = x;
      std::vector<int64_t> offs;
      for (int64_t d = -1; d <= 1; ++d) {
        int64_t v = ((d % nc) + nc) % nc;
        if (std::find(offs.begin(), offs.end(), v) == offs.end()) offs.push_back(v);
      }
      for (int64_t x : beads) {
        int64_t cx = (int64_t)pos[4 * x] * nc / L[r], cy = (int64_t)pos[4 * x + 1] * nc / L[r],
                cz = (int64_t)pos[4 * x + 2] * nc / L[r];
        for (int64_t ox : offs)
          for (int64_t oy : offs)
            for (int64_t oz : offs) {
              size_t c = (size_t)((((cx + ox) % nc) * nc + (cy + oy) % nc) * nc + (cz + oz) % nc);
              for (int64_t k = start[c]; k < start[c + 1]; ++k)
                if (sorted[(size_t)k] > x) consider_pair(x, sorted[(size_t)k], &E);
            }
      }
    }
    return E;
  }

  // Appendix step 3: bonds eligible for breakage or conversion (last matching
  // breakbond / convertbond rule per bond), and the killbond set of step 5.
  void breakage_candidates(std::vector<Edge>* E, std::set<std::pair<int32_t, int32_t>>* killed) const {
    for (int64_t a = 0; a < N; ++a)
      for (int s = 0; s < SLOTS; ++s) {
        int64_t b = nb[a * SLOTS + s];
        if (b < 0 || b < a) continue;
        int t = st[a * SLOTS + s];
        if (stored(b, a) != t) continue;  // only symmetric bonds
        if (!has(reactive, type[a]) || !has(reactive, type[b])) continue;
        int64_t dd = d2(a, b);
        for (const ORule& r : rules)
          if (r.kind == K_KILLBOND && r.type == t && dd > r2_of(r.dist)) killed->insert({(int32_t)a, (int32_t)b});
        for (int k = (int)rules.size() - 1; k >= 0; --k) {
          const ORule& r = rules[k];
          bool m = (r.kind == K_BREAKBOND && r.type == t && dd > r2_of(r.dist)) ||
                   (r.kind == K_CONVERTBOND && r.type == t);
          if (!m) continue;
          int nt = r.kind == K_CONVERTBOND ? r.type2 : -1;
          E->push_back(Edge{-dd, (int32_t)a, (int32_t)b, k, nt, nt});
          break;
        }
      }
  }

  bool trial(const Edge& e, int tag, uint64_t step, double scale) const {
    int r = rep[e.a];
    uint32_t ctr[4] = {(uint32_t)(e.a - off[r]), (uint32_t)(e.b - off[r]), (uint32_t)step,
                       ((uint32_t)tag << 24) | (stream[r] & 0xFFFFFFu)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4];
    philox4x32_10(ctr, key, u);
    double p = std::min(1.0, rules[e.rule].prob * scale);
    uint64_t T = threshold_of(p);
    if (prob_mode == 0) return (uint64_t)u[0] < T;
    return (uint64_t)u[0] + (uint64_t)u[1] < 2 * T;
  }

  void remove_bond(int64_t a, int64_t b) {
    for (int64_t x : {a, b}) {
      int64_t y = x == a ? b : a;
      std::vector<std::pair<int32_t, int32_t>> keep;
      for (int s = 0; s < SLOTS; ++s)
        if (nb[x * SLOTS + s] >= 0 && nb[x * SLOTS + s] != y) keep.push_back({nb[x * SLOTS + s], st[x * SLOTS + s]});
      for (int s = 0; s < SLOTS; ++s) {
        nb[x * SLOTS + s] = s < (int)keep.size() ? keep[s].first : -1;
        st[x * SLOTS + s] = s < (int)keep.size() ? keep[s].second : -1;
      }
    }
  }
  void set_type(int64_t x, int64_t y, int t) {
    for (int s = 0; s < SLOTS; ++s)
      if (nb[x * SLOTS + s] == y) st[x * SLOTS + s] = t;
  }
  bool add_half(int64_t x, int64_t y, int t) {
    for (int s = 0; s < SLOTS; ++s)
      if (nb[x * SLOTS + s] < 0) {
        nb[x * SLOTS + s] = (int32_t)y;
        st[x * SLOTS + s] = t;
        return true;
      }
    return false;
  }

  // ------------------------------------------------------------------------
  // interaction typing (Sec. 2): createangle / createdihedral rules tried in
  // list order on ABC then CBA (ABCD then DCBA); bond types are those stored
  // by the beads: angle  t = st(B->A), s = st(B->C);
  //               dihedral r = st(B->A), s = st(C->B) or s' = st(B->C), t = st(C->D).
  // ------------------------------------------------------------------------
  bool angle_match(const ORule& r, int64_t a, int64_t b, int64_t c) const {
    return has(r.bead[0], type[a]) && has(r.bead[1], type[b]) && has(r.bead[2], type[c]) &&
           has(r.bond[0], stored(b, a)) && has(r.bond[1], stored(b, c));
  }
  int angle_type(int64_t a, int64_t b, int64_t c) const {
    for (const ORule& r : rules)
      if (r.kind == K_CREATEANGLE && (angle_match(r, a, b, c) || angle_match(r, c, b, a))) return r.type;
    return 0;
  }
  bool dihedral_match(const ORule& r, int64_t a, int64_t b, int64_t c, int64_t d) const {
    return has(r.bead[0], type[a]) && has(r.bead[1], type[b]) && has(r.bead[2], type[c]) && has(r.bead[3], type[d]) &&
           has(r.bond[0], stored(b, a)) && (has(r.bond[1], stored(c, b)) || has(r.bond[1], stored(b, c))) &&
           has(r.bond[2], stored(c, d));
  }
  int dihedral_type(int64_t a, int64_t b, int64_t c, int64_t d) const {
    for (const ORule& r : rules)
      if (r.kind == K_CREATEDIHEDRAL && (dihedral_match(r, a, b, c, d) || dihedral_match(r, d, c, b, a)))
        return r.type;
    return 0;
  }

  // Every non-cyclic path of 3 and 4 beads of the current bond graph, typed,
  // in canonical orientation.  keep(path-bonds) filters paths by their bonds.
  template <class F>
  void typed_paths(std::vector<Angle>* A, std::vector<Dihedral>* D, F keep) const {
    for (int64_t b = 0; b < N; ++b)
      for (int s1 = 0; s1 < SLOTS; ++s1) {
        int64_t a = nb[b * SLOTS + s1];
        if (a < 0) continue;
        for (int s2 = 0; s2 < SLOTS; ++s2) {
          int64_t c = nb[b * SLOTS + s2];
          if (c < 0 || c == a || a > c) continue;
          std::array<std::pair<int64_t, int64_t>, 2> bonds{{{a, b}, {b, c}}};
          if (!keep(bonds.data(), 2)) continue;
          int t = angle_type(a, b, c);
          if (t) A->push_back(Angle{(int32_t)a, (int32_t)b, (int32_t)c, t});
        }
        // dihedrals with middle bond (b, c)
        for (int s2 = 0; s2 < SLOTS; ++s2) {
          int64_t c = nb[b * SLOTS + s2];
          if (c < 0) continue;
          for (int s3 = 0; s3 < SLOTS; ++s3) {
            int64_t d = nb[c * SLOTS + s3];
            if (d < 0 || d == b) continue;
            if (a == c || a == d) continue;
            if (a > d) continue;  // each undirected path once: first bead below last bead
            std::array<std::pair<int64_t, int64_t>, 3> bonds{{{a, b}, {b, c}, {c, d}}};
            if (!keep(bonds.data(), 3)) continue;
            int t = dihedral_type(a, b, c, d);
            if (t) D->push_back(Dihedral{(int32_t)a, (int32_t)b, (int32_t)c, (int32_t)d, t});
          }
        }
      }
    std::sort(A->begin(), A->end());
    A->erase(std::unique(A->begin(), A->end()), A->end());
    std::sort(D->begin(), D->end());
    D->erase(std::unique(D->begin(), D->end()), D->end());
  }

  void full_rules(std::vector<Angle>* A, std::vector<Dihedral>* D) const {
    typed_paths(A, D, [](const std::pair<int64_t, int64_t>*, int) { return true; });
  }

  // ------------------------------------------------------------------------
  // one call of the fix
  // ------------------------------------------------------------------------
  int step(const int32_t* p, uint64_t s, int64_t* stats) {
    for (int r = 0; r < R; ++r)
      for (int64_t x = off[r]; x < off[r + 1]; ++x)
        for (int c = 0; c < 3; ++c)
          if (p[4 * x + c] < 0 || p[4 * x + c] >= L[r]) return 1;
    pos = p;
    std::vector<int64_t> S((size_t)R * S_COUNT, 0);
    auto stat = [&](int r, int k) -> int64_t& { return S[(size_t)r * S_COUNT + k]; };

    // steps 2 and 4: creation nomination on the pre-call state
    std::vector<Edge> CE = creation_candidates(!use_cells);
    std::sort(CE.begin(), CE.end(), edge_less);
    for (const Edge& e : CE) stat(rep[e.a], S_CANDIDATES) += 1;
    std::vector<int64_t> crounds(R, 0), brounds(R, 0);
    std::vector<int> cm = match_rounds(N, CE, max_rounds, rep, &crounds);

    // steps 3 and 4: breakage nomination on the pre-call state; killbond set
    std::vector<Edge> BE;
    std::set<std::pair<int32_t, int32_t>> killed;
    breakage_candidates(&BE, &killed);
    std::sort(BE.begin(), BE.end(), edge_less);
    for (const Edge& e : BE) stat(rep[e.a], S_BREAK_CANDIDATES) += 1;
    std::vector<int> bm = match_rounds(N, BE, max_rounds, rep, &brounds);

    // steps 5 and 8: stochastic trials of the matched pairs
    std::vector<Edge> formed, broken, converted;
    for (int e : cm) {
      stat(rep[CE[e].a], S_CREATE_MATCHED) += 1;
      if (trial(CE[e], TAG_FORM, s, fscale[rep[CE[e].a]])) formed.push_back(CE[e]);
    }
    for (int e : bm) {
      const Edge& x = BE[e];
      stat(rep[x.a], S_BREAK_MATCHED) += 1;
      if (!trial(x, TAG_BREAK, s, bscale[rep[x.a]])) continue;
      if (killed.count({x.a, x.b})) continue;  // removed by killbond anyway
      if (rules[x.rule].kind == K_BREAKBOND) broken.push_back(x);
      else converted.push_back(x);
    }

    // bonds removed or retyped this call
    std::set<std::pair<int32_t, int32_t>> changed(killed.begin(), killed.end());
    for (const Edge& e : broken) changed.insert({e.a, e.b});
    for (const Edge& e : converted) changed.insert({e.a, e.b});

    // step 6: drop every interaction that contains a removed or converted bond
    auto bond_changed = [&](int64_t x, int64_t y) {
      return changed.count({(int32_t)std::min(x, y), (int32_t)std::max(x, y)}) > 0;
    };
    std::vector<Angle> keepA;
    for (const Angle& a : angles) {
      if (bond_changed(a[0], a[1]) || bond_changed(a[1], a[2])) stat(rep[a[1]], S_ANG_REMOVED) += 1;
      else keepA.push_back(a);
    }
    std::vector<Dihedral> keepD;
    for (const Dihedral& d : dihedrals) {
      if (bond_changed(d[0], d[1]) || bond_changed(d[1], d[2]) || bond_changed(d[2], d[3]))
        stat(rep[d[1]], S_DIH_REMOVED) += 1;
      else keepD.push_back(d);
    }

    // step 7: update the bond tables (kill + break), conversions
    for (auto& k : killed) { remove_bond(k.first, k.second); stat(rep[k.first], S_KILLED) += 1; }
    for (const Edge& e : broken) { remove_bond(e.a, e.b); stat(rep[e.a], S_BROKEN) += 1; }
    for (const Edge& e : converted) {
      set_type(e.a, e.b, rules[e.rule].type2);
      set_type(e.b, e.a, rules[e.rule].type2);
      stat(rep[e.a], S_CONVERTED) += 1;
    }
    // step 8: add the formed bonds
    for (const Edge& e : formed) {
      if (!add_half(e.a, e.b, e.ta) || !add_half(e.b, e.a, e.tb)) return 2;
      stat(rep[e.a], S_FORMED) += 1;
    }

    // step 9: typed interactions of every path that contains a new bond
    std::set<std::pair<int32_t, int32_t>> fresh;
    for (const Edge& e : formed) fresh.insert({e.a, e.b});
    for (const Edge& e : converted) fresh.insert({e.a, e.b});
    std::vector<Angle> addA;
    std::vector<Dihedral> addD;
    typed_paths(&addA, &addD, [&](const std::pair<int64_t, int64_t>* bonds, int n) {
      for (int i = 0; i < n; ++i) {
        int64_t x = bonds[i].first, y = bonds[i].second;
        if (fresh.count({(int32_t)std::min(x, y), (int32_t)std::max(x, y)})) return true;
      }
      return false;
    });
    for (const Angle& a : addA) stat(rep[a[1]], S_ANG_ADDED) += 1;
    for (const Dihedral& d : addD) stat(rep[d[1]], S_DIH_ADDED) += 1;
    angles.clear();
    std::merge(keepA.begin(), keepA.end(), addA.begin(), addA.end(), std::back_inserter(angles));
    dihedrals.clear();
    std::merge(keepD.begin(), keepD.end(), addD.begin(), addD.end(), std::back_inserter(dihedrals));

    // step 10: statistics
    for (int64_t x = 0; x < N; ++x)
      for (int k = 0; k < SLOTS; ++k)
        if (nb[x * SLOTS + k] > x) stat(rep[x], S_NBONDS) += 1;
    for (const Angle& a : angles) stat(rep[a[1]], S_NANGLES) += 1;
    for (const Dihedral& d : dihedrals) stat(rep[d[1]], S_NDIHEDRALS) += 1;
    for (int r = 0; r < R; ++r) {
      stat(r, S_CREATE_ROUNDS) = crounds[r];
      stat(r, S_BREAK_ROUNDS) = brounds[r];
    }
    if (stats) std::memcpy(stats, S.data(), S.size() * sizeof(int64_t));
    pos = nullptr;
    return 0;
  }
};

// ---------------------------------------------------------------------------
// bonded forces in FP64
// ---------------------------------------------------------------------------

void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Half of a harmonic bond seen from one end: the end feels the full force of
// E = K (r - r0)^2 with the type it stores and books half the energy (each
// end of a directional bond applies its own stored type, Sec. 2).
void bond_half(const double rij[3], double K, double r0, double* E, double F[3]) {
  double r = std::sqrt(dot(rij, rij));
  double dEdr = 2.0 * K * (r - r0);
  for (int c = 0; c < 3; ++c) F[c] = -dEdr * rij[c] / r;
  *E = 0.5 * K * (r - r0) * (r - r0);
}

// Cosine angle E = K (1 + cos theta) with ra = r_A - r_B, rc = r_C - r_B.
void angle_cos(const double ra[3], const double rc[3], double K, double* E, double Fa[3], double Fc[3]) {
  double la = std::sqrt(dot(ra, ra)), lc = std::sqrt(dot(rc, rc));
  double cs = dot(ra, rc) / (la * lc);
  for (int c = 0; c < 3; ++c) {
    double ga = rc[c] / (la * lc) - cs * ra[c] / (la * la);
    double gc = ra[c] / (la * lc) - cs * rc[c] / (lc * lc);
    Fa[c] = -K * ga;
    Fc[c] = -K * gc;
  }
  *E = K * (1.0 + cs);
}

// Harmonic angle E = K (theta - theta0)^2 (the DNA angles of Sec. 3) with
// ra = r_A - r_B, rc = r_C - r_B and theta the angle at B.  The gradient of
// theta follows from rotating each end about the unit normal n = (ra x rc) /
// |ra x rc| of the plane ABC: moving A along n x ra opens the angle, so
// dtheta/dr_A = (ra x n) / |ra|^2 and dtheta/dr_C = -(rc x n) / |rc|^2, each
// of magnitude 1 / |r|.  F = -dE/dr = -2K (theta - theta0) dtheta/dr.  This
// holds at every angle where the plane exists; exactly collinear beads have
// no plane and get no angle force.
void angle_harmonic(const double ra[3], const double rc[3], double K, double theta0, double* E, double Fa[3],
                    double Fc[3]) {
  double w[3];
  cross(ra, rc, w);
  double wn = std::sqrt(dot(w, w));
  double theta = std::atan2(wn, dot(ra, rc));  // accurate near 0 and pi
  double g = 2.0 * K * (theta - theta0);        // dE/dtheta
  *E = K * (theta - theta0) * (theta - theta0);
  if (wn == 0.0) {
    for (int k = 0; k < 3; ++k) Fa[k] = Fc[k] = 0.0;
    return;
  }
  double n[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
  double ta[3], tc[3];
  cross(ra, n, ta);
  cross(rc, n, tc);
  double la2 = dot(ra, ra), lc2 = dot(rc, rc);
  for (int k = 0; k < 3; ++k) {
    Fa[k] = -g * ta[k] / la2;
    Fc[k] = g * tc[k] / lc2;
  }
}

// Dihedral E = K (1 + d cos phi), b1 = r_B - r_A, b2 = r_C - r_B, b3 = r_D - r_C,
// cos phi = m.n / (|m||n|) with m = b1 x b2, n = b2 x b3 (trans = 180 deg).
// The gradient is taken of cos phi through m and n directly.
void dihedral_cos(const double b1[3], const double b2[3], const double b3[3], double K, double d, double* E,
                  double Fa[3], double Fb[3], double Fc[3], double Fd[3]) {
  double m[3], n[3];
  cross(b1, b2, m);
  cross(b2, b3, n);
  double lm = std::sqrt(dot(m, m)), ln = std::sqrt(dot(n, n));
  double cs = dot(m, n) / (lm * ln);
  double gm[3], gn[3];
  for (int c = 0; c < 3; ++c) {
    gm[c] = n[c] / (lm * ln) - cs * m[c] / (lm * lm);
    gn[c] = m[c] / (lm * ln) - cs * n[c] / (ln * ln);
  }
  double G1[3], G2a[3], G2b[3], G3[3];
  cross(b2, gm, G1);   // d cos / d b1
  cross(gm, b1, G2a);  // d cos / d b2 through m
  cross(b3, gn, G2b);  // d cos / d b2 through n
  cross(gn, b2, G3);   // d cos / d b3
  for (int c = 0; c < 3; ++c) {
    double G2 = G2a[c] + G2b[c];
    double dA = -G1[c], dB = G1[c] - G2, dC = G2 - G3[c], dD = G3[c];
    Fa[c] = -K * d * dA;
    Fb[c] = -K * d * dB;
    Fc[c] = -K * d * dC;
    Fd[c] = -K * d * dD;
  }
  *E = K * (1.0 + d * cs);
}

void add_virial(double* ev, const double r[3], const double F[3], double w) {
  ev[1] += w * r[0] * F[0];
  ev[2] += w * r[1] * F[1];
  ev[3] += w * r[2] * F[2];
  ev[4] += w * r[0] * F[1];
  ev[5] += w * r[0] * F[2];
  ev[6] += w * r[1] * F[2];
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (called from oracle/oracle.py through ctypes)
// ---------------------------------------------------------------------------
extern "C" {

void* orc_new(int R, const int64_t* off, const int64_t* box, const double* fscale, const double* bscale,
              const uint32_t* stream, const int32_t* types, const int32_t* bonds, int64_t n_bonds,
              const void* rules, int n_rules, uint64_t seed, int pc13, int pc14, int max_rounds, int prob_mode,
              uint32_t reactive, int use_cells) {
  Oracle* o = new Oracle();
  o->R = R;
  o->off.assign(off, off + R + 1);
  o->L.assign(box, box + R);
  o->fscale.assign(fscale, fscale + R);
  o->bscale.assign(bscale, bscale + R);
  o->stream.assign(stream, stream + R);
  o->N = off[R];
  o->type.assign(types, types + o->N);
  o->rep.assign(o->N, 0);
  for (int r = 0; r < R; ++r)
    for (int64_t x = off[r]; x < off[r + 1]; ++x) o->rep[x] = r;
  o->nb.assign(o->N * SLOTS, -1);
  o->st.assign(o->N * SLOTS, -1);
  const ORule* rr = static_cast<const ORule*>(rules);
  o->rules.assign(rr, rr + n_rules);
  o->seed = seed;
  o->pc13 = pc13;
  o->pc14 = pc14;
  o->max_rounds = max_rounds;
  o->prob_mode = prob_mode;
  o->reactive = reactive;
  o->use_cells = use_cells;
  for (int64_t k = 0; k < n_bonds; ++k) {
    int64_t i = bonds[4 * k], j = bonds[4 * k + 1];
    if (i < 0 || j < 0 || i >= o->N || j >= o->N || i == j || o->rep[i] != o->rep[j] || o->stored(i, j) >= 0 ||
        !o->add_half(i, j, bonds[4 * k + 2]) || !o->add_half(j, i, bonds[4 * k + 3])) {
      delete o;
      return nullptr;
    }
  }
  // the initial interaction set is the typed set of every path of the initial graph
  o->full_rules(&o->angles, &o->dihedrals);
  return o;
}

void orc_free(void* h) { delete static_cast<Oracle*>(h); }

int orc_step(void* h, const int32_t* pos, uint64_t step, int64_t* stats) {
  return static_cast<Oracle*>(h)->step(pos, step, stats);
}

int orc_stat_count() { return S_COUNT; }

void orc_counts(void* h, int64_t* out) {
  Oracle* o = static_cast<Oracle*>(h);
  int64_t nbnd = 0;
  for (int64_t x = 0; x < o->N; ++x)
    for (int s = 0; s < SLOTS; ++s) nbnd += o->nb[x * SLOTS + s] > x;
  out[0] = nbnd;
  out[1] = (int64_t)o->angles.size();
  out[2] = (int64_t)o->dihedrals.size();
}

// bonds (i < j, type stored by i, type stored by j) sorted; angles and
// dihedrals canonical and sorted.
void orc_topology(void* h, int32_t* bonds, int32_t* angles, int32_t* dihedrals) {
  Oracle* o = static_cast<Oracle*>(h);
  std::vector<std::array<int32_t, 4>> B;
  for (int64_t x = 0; x < o->N; ++x)
    for (int s = 0; s < SLOTS; ++s) {
      int64_t y = o->nb[x * SLOTS + s];
      if (y > x) B.push_back({(int32_t)x, (int32_t)y, o->st[x * SLOTS + s], o->stored(y, x)});
    }
  std::sort(B.begin(), B.end());
  if (bonds) std::memcpy(bonds, B.data(), B.size() * sizeof(B[0]));
  if (angles) std::memcpy(angles, o->angles.data(), o->angles.size() * sizeof(Angle));
  if (dihedrals) std::memcpy(dihedrals, o->dihedrals.data(), o->dihedrals.size() * sizeof(Dihedral));
}

// 1 if the stored interaction sets equal the typed set of every path of the
// current bond graph.
int orc_check_rules_identity(void* h) {
  Oracle* o = static_cast<Oracle*>(h);
  std::vector<Angle> A;
  std::vector<Dihedral> D;
  o->full_rules(&A, &D);
  return A == o->angles && D == o->dihedrals;
}

// Creation candidate pairs for the given snapshot without changing state:
// rows (a, b, rule, d2_lo, d2_hi) with a < b, sorted.  Returns the count.
int64_t orc_candidates(void* h, const int32_t* pos, int brute, int32_t* out, int64_t cap) {
  Oracle* o = static_cast<Oracle*>(h);
  o->pos = pos;
  std::vector<Edge> E = o->creation_candidates(brute != 0);
  o->pos = nullptr;
  std::sort(E.begin(), E.end(), [](const Edge& x, const Edge& y) {
    return std::make_pair(x.a, x.b) < std::make_pair(y.a, y.b);
  });
  for (int64_t k = 0; k < (int64_t)E.size() && k < cap; ++k) {
    out[5 * k] = E[k].a;
    out[5 * k + 1] = E[k].b;
    out[5 * k + 2] = E[k].rule;
    out[5 * k + 3] = (int32_t)(uint32_t)(uint64_t)E[k].k1;
    out[5 * k + 4] = (int32_t)(E[k].k1 >> 32);
  }
  return (int64_t)E.size();
}

// Rounds of mutual nomination on an arbitrary edge list (for pins): keys
// (k1[e], a[e], b[e]) with a[e] < b[e]; writes 1 into matched[e] for every
// matched edge and returns the number of rounds that matched something.
int orc_match(int64_t n_beads, int64_t n_edges, const int64_t* k1, const int32_t* a, const int32_t* b,
              int max_rounds, int32_t* matched) {
  std::vector<Edge> E((size_t)n_edges);
  for (int64_t e = 0; e < n_edges; ++e) E[e] = Edge{k1[e], a[e], b[e], 0, 0, 0};
  std::vector<int32_t> rep(n_beads, 0);
  std::vector<int64_t> rounds(1, 0);
  std::vector<int> m = match_rounds(n_beads, E, max_rounds, rep, &rounds);
  for (int64_t e = 0; e < n_edges; ++e) matched[e] = 0;
  for (int e : m) matched[e] = 1;
  return (int)rounds[0];
}

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }
int64_t orc_r2(double dist) { return r2_of(dist); }
uint64_t orc_threshold(double p) { return threshold_of(p); }

// Bonded forces (FP64) of the current topology at the given snapshot:
// force[N*3], ev[R*7] = (E, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz) per replica with
// W_ab = sum over interactions of (r_role - r_ref)_a F_role,b.
int orc_forces(void* h, const int32_t* pos, const double* bond_k, const double* bond_r0, const double* angle_k,
               const double* dih_k, const int32_t* dih_d, const double* angle_theta0, const int32_t* angle_style,
               double* force, double* ev) {
  Oracle* o = static_cast<Oracle*>(h);
  o->pos = pos;
  std::memset(force, 0, sizeof(double) * 3 * o->N);
  std::memset(ev, 0, sizeof(double) * 7 * o->R);
  for (int64_t i = 0; i < o->N; ++i)
    for (int s = 0; s < SLOTS; ++s) {
      int64_t j = o->nb[i * SLOTS + s];
      if (j < 0) continue;
      int t = o->st[i * SLOTS + s];
      double rij[3], F[3], E;
      o->rel(i, j, rij);
      bond_half(rij, bond_k[t], bond_r0[t], &E, F);
      double* e = ev + 7 * o->rep[i];
      e[0] += E;
      add_virial(e, rij, F, 0.5);
      for (int c = 0; c < 3; ++c) force[3 * i + c] += F[c];
    }
  for (const Angle& a : o->angles) {
    double ra[3], rc[3], Fa[3], Fc[3], E;
    o->rel(a[0], a[1], ra);
    o->rel(a[2], a[1], rc);
    if (angle_style[a[3]] == 1) angle_harmonic(ra, rc, angle_k[a[3]], angle_theta0[a[3]], &E, Fa, Fc);
    else angle_cos(ra, rc, angle_k[a[3]], &E, Fa, Fc);
    double* e = ev + 7 * o->rep[a[1]];
    e[0] += E;
    add_virial(e, ra, Fa, 1.0);
    add_virial(e, rc, Fc, 1.0);
    for (int c = 0; c < 3; ++c) {
      force[3 * a[0] + c] += Fa[c];
      force[3 * a[2] + c] += Fc[c];
      force[3 * a[1] + c] -= Fa[c] + Fc[c];
    }
  }
  for (const Dihedral& d : o->dihedrals) {
    double b1[3], b2[3], b3[3], Fa[3], Fb[3], Fc[3], Fd[3], E;
    o->rel(d[1], d[0], b1);
    o->rel(d[2], d[1], b2);
    o->rel(d[3], d[2], b3);
    dihedral_cos(b1, b2, b3, dih_k[d[4]], (double)dih_d[d[4]], &E, Fa, Fb, Fc, Fd);
    double* e = ev + 7 * o->rep[d[1]];
    e[0] += E;
    double ra[3], rd[3];
    for (int c = 0; c < 3; ++c) {
      ra[c] = -b1[c];
      rd[c] = b2[c] + b3[c];
    }
    add_virial(e, ra, Fa, 1.0);
    add_virial(e, b2, Fc, 1.0);
    add_virial(e, rd, Fd, 1.0);
    for (int c = 0; c < 3; ++c) {
      force[3 * d[0] + c] += Fa[c];
      force[3 * d[1] + c] += Fb[c];
      force[3 * d[2] + c] += Fc[c];
      force[3 * d[3] + c] += Fd[c];
    }
  }
  o->pos = nullptr;
  return 0;
}

// DPD pair forces of Sec. 3 (FP64), by brute force over every pair of beads
// of a replica: for r = |r_i - r_j| < r_c,
//   F_i += (F^C + F^D + F^R) r_ij / r,  F^C = a w(r),
//   F^D = -gamma w(r)^2 (r_ij . v_ij) / r,  F^R = sigma w(r) xi / sqrt(dt),
// w(r) = 1 - r / r_c, sigma = sqrt(2 kT gamma), r_ij = r_i - r_j, v_ij = v_i
// - v_j; pairs fewer than 3 bonds apart (graph distance 1 or 2) carry no pair
// force (Sec. 3).  "r < r_c" is decided exactly on the integer grid as d2 <
// floor((r_c 2^20)^2).  xi is the unit Gaussian of the pair at this step:
// Philox4x32-10 on the counter (lower id, higher id, step low word, step high
// word xor 0x3D000000) with the 64-bit seed as key; its first two words give
// u1 = ((x0 >> 9) + 1/2) 2^-23 in (0, 1) and u2 = (x1 >> 9) 2^-23 in [0, 1),
// and xi = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller, Ann. Math. Stat. 29,
// 610 (1958)), the same number for both beads of the pair.
void orc_dpd_forces(void* h, const int32_t* pos, const double* vel, double a, double gamma, double kT, double rc,
                    double dt, uint64_t seed, uint64_t step, double* force) {
  Oracle* o = static_cast<Oracle*>(h);
  o->pos = pos;
  std::memset(force, 0, sizeof(double) * 3 * o->N);
  const int64_t rc2 = r2_of(rc);
  const double sigma = std::sqrt(2.0 * kT * gamma);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double pi = 3.14159265358979323846;
  for (int r = 0; r < o->R; ++r)
    for (int64_t i = o->off[r]; i < o->off[r + 1]; ++i)
      for (int64_t j = i + 1; j < o->off[r + 1]; ++j) {
        if (o->d2(i, j) >= rc2) continue;
        if (o->graph_distance(i, j) < 3) continue;
        double rij[3];
        o->rel(i, j, rij);
        const double rr = std::sqrt(dot(rij, rij));
        if (rr <= 0.0) continue;
        const double w = 1.0 - rr / rc;
        double rv = 0.0;
        for (int c = 0; c < 3; ++c) rv += rij[c] * (vel[3 * i + c] - vel[3 * j + c]);
        const uint32_t ctr[4] = {(uint32_t)i, (uint32_t)j, (uint32_t)step, (uint32_t)(step >> 32) ^ 0x3D000000u};
        uint32_t u[4];
        philox4x32_10(ctr, key, u);
        const double u1 = ((double)(u[0] >> 9) + 0.5) / 8388608.0, u2 = (double)(u[1] >> 9) / 8388608.0;
        const double xi = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * pi * u2);
        const double fs = a * w - gamma * w * w * rv / rr + sigma * w * xi / std::sqrt(dt);
        for (int c = 0; c < 3; ++c) {
          force[3 * i + c] += fs * rij[c] / rr;
          force[3 * j + c] -= fs * rij[c] / rr;
        }
      }
  o->pos = nullptr;
}

// Force primitives on explicit relative vectors (for finite-difference pins).
void orc_bond_half(const double* rij, double K, double r0, double* E, double* F) { bond_half(rij, K, r0, E, F); }
void orc_angle(const double* ra, const double* rc, double K, double* E, double* Fa, double* Fc) {
  angle_cos(ra, rc, K, E, Fa, Fc);
}
void orc_angle_harmonic(const double* ra, const double* rc, double K, double theta0, double* E, double* Fa,
                        double* Fc) {
  angle_harmonic(ra, rc, K, theta0, E, Fa, Fc);
}
void orc_dihedral(const double* b1, const double* b2, const double* b3, double K, double d, double* E, double* Fa,
                  double* Fb, double* Fc, double* Fd) {
  dihedral_cos(b1, b2, b3, K, d, E, Fa, Fb, Fc, Fd);
}

}  // extern "C"
