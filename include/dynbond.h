/*
 * dynbond.h — C ABI of the GB300 dynamic-bonding library (libdynbond.so).
 *
 * One call of dynbond_step() is one application of the dynamic-bonding fix of
 * C. Svaneborg, "LAMMPS Framework for Dynamic Bonding and an Application
 * Modeling DNA" (arXiv:1108.4214): creation and breakage nomination on the
 * state before the call, mutual-nomination matching, stochastic trials,
 * killbond / breakbond / convertbond, removal of every angle and dihedral that
 * contains a removed or converted bond, and typed creation of the angles and
 * dihedrals of every new triplet and quartet (Sec. 2; Appendix steps 1-10).
 * dynbond_forces() evaluates the bonded forces of the resulting topology.
 *
 * Conventions shared by every entry point
 *   - Beads of all replicas are numbered globally 0..N-1; replica r owns
 *     [bead_offset[r], bead_offset[r+1]).  Replicas never interact.
 *   - Positions are int32 on a fixed-point grid of 2^-20 sigma per unit,
 *     passed as int4 {x, y, z, w} per bead (16 bytes, w ignored), each
 *     coordinate in [0, box_q[r]).  Squared distances are exact int64; a
 *     distance threshold r is compared as d2 <= floor((r * 2^20)^2) ("within r")
 *     or d2 > floor((r * 2^20)^2) ("longer than r").
 *   - Bond types are 1..15, bead types 0..15; type masks have bit t set for
 *     type t ('*' = all bits).  Each bead holds at most DYNBOND_SLOTS bonds.
 *   - Device pointers (d_*) are caller-owned CUDA global memory; host
 *     pointers (h_*, and every pointer inside dynbond_system / dynbond_rule /
 *     dynbond_topology) are caller-owned host memory that is only read (or
 *     written, for outputs) during the call.
 *   - Every call is ordered on the context's CUDA stream.  Errors found on the
 *     device (capacity, bad positions, timeouts) are reported by the next call
 *     that synchronizes: dynbond_sync(), or dynbond_step() with h_stats.  After
 *     a device error the context refuses further steps (status sticks).
 *   - No entry point throws or aborts; each returns a dynbond_status.
 */
#ifndef DYNBOND_H
#define DYNBOND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dynbond_status {
  DYNBOND_OK = 0,
  DYNBOND_EINVAL = 1,         /* malformed argument, rule, system or position */
  DYNBOND_ENOMEM = 2,         /* device or host allocation failed */
  DYNBOND_ECAPACITY = 3,      /* a fixed capacity was exceeded (see DYNBOND_MAX_*) */
  DYNBOND_ECUDA = 4,          /* a CUDA runtime call failed */
  DYNBOND_ETIMEOUT = 5,       /* a bounded device-side wait gave up */
  DYNBOND_ENOTCONVERGED = 6   /* matching needed more than DYNBOND_MAX_ROUNDS rounds */
} dynbond_status;

enum {
  DYNBOND_MAX_TYPES = 16,     /* bead types 0..15, bond / angle / dihedral types 1..15 */
  DYNBOND_SLOTS = 4,          /* bonds per bead; creation also requires fewer than this */
  DYNBOND_MAX_RULES = 32,
  DYNBOND_MAX_CANDIDATES = 24,/* creation candidates one bead keeps in registers; beads with more
                                 take an exact two-pass path (no limit) */
  DYNBOND_MAX_ROUNDS = 4096,  /* matching rounds of one call */
  DYNBOND_EV = 7,             /* energy + 6 virial components per replica */
  DYNBOND_NOALLOC_MAX_REPLICAS = 4096 /* replicas of one dynbond_forces_noalloc call */
};

/* Rule kinds: the rule set of the fix (Fig. 1). */
typedef enum dynbond_rule_kind {
  DYNBOND_CREATEBOND = 1,     /* type; bead_mask[0..1]; dist (max); prob */
  DYNBOND_CREATEDIRBOND = 2,  /* type (stored by the bead-mask-0 end), type2 (by the other); bead_mask[0..1]; dist; prob */
  DYNBOND_BREAKBOND = 3,      /* type; dist (min, strict); prob */
  DYNBOND_CONVERTBOND = 4,    /* type -> type2; prob */
  DYNBOND_KILLBOND = 5,       /* type; dist (min, strict) */
  DYNBOND_CREATEANGLE = 6,    /* type; bead_mask[0..2]; bond_mask[0] = t, [1] = s */
  DYNBOND_CREATEDIHEDRAL = 7, /* type; bead_mask[0..3]; bond_mask[0] = r, [1] = s / s', [2] = t */
  DYNBOND_MAXBOND = 8         /* bond_mask[0] = counted bond types; bead_mask[0]; maxn */
} dynbond_rule_kind;

/*
 * One rule (64 bytes).  Rules are evaluated in list order:
 *   - creation (createbond / createdirbond): per candidate pair the LAST rule
 *     matching bead types, distance and maxbond decides the stored bond types
 *     (Sec. 2, Appendix step 2); a directional bond is oriented by trying the
 *     lower-id bead as the rule's first bead type first;
 *   - breakage / conversion (breakbond / convertbond): per bond the LAST
 *     matching rule; these rules, and killbond, apply to symmetric bonds of
 *     their type (both endpoints store it), as Sec. 2 describes them;
 *   - typing (createangle / createdihedral): per path the FIRST rule matching
 *     ABC or CBA (ABCD or DCBA) with the directional bond types of Sec. 2:
 *     angle t = type B stores toward A, s = type B stores toward C; dihedral
 *     r = B toward A, s = C toward B or s' = B toward C, t = C toward D;
 *   - maxbond: a bead of a type in bead_mask[0] may receive a bond stored as a
 *     type in bond_mask[0] only while it stores fewer than maxn such bonds.
 *     Conversions are not checked against maxbond (the fix checks it while
 *     nominating creation partners only).
 */
typedef struct dynbond_rule {
  int32_t kind;
  int32_t type;
  int32_t type2;
  int32_t maxn;
  uint32_t bead_mask[4];
  uint32_t bond_mask[3];
  uint32_t reserved;
  double dist;
  double prob;
} dynbond_rule;

enum {
  DYNBOND_FLAG_NO_GRAPH = 1,    /* launch kernels one by one instead of replaying a CUDA graph */
  DYNBOND_FLAG_PROFILE = 2,     /* record CUDA events between phases (dynbond_phase_times) */
  DYNBOND_FLAG_NO_AUTOTUNE = 4, /* with cell_scale 0: use cells as wide as the reach, never autotune */
  DYNBOND_FLAG_NO_PDL = 8,      /* launch each kernel only after the previous one ends (no programmatic
                                   dependent launch); results are identical either way */
  DYNBOND_FLAG_GLOBAL_SEARCH = 16, /* candidate search always walks the cell lists in global memory */
  DYNBOND_FLAG_STAGED_SEARCH = 32, /* candidate search always stages tiles of cell columns in shared memory
                                      where the geometry allows it (without either flag the autotuner
                                      times both; untuned contexts use the global search); results are
                                      identical either way */
  DYNBOND_FLAG_PERSISTENT = 64     /* each dynbond_step is one persistent cooperative launch whose blocks run
                                      the call's phases one after another with bounded grid barriers
                                      (instead of a graph of one kernel per phase; not with
                                      DYNBOND_FLAG_PROFILE, whose phase events need the kernels apart);
                                      the candidate search is then the global one; results are identical */
};

/*
 * Run parameters.
 *   seed          64-bit key of the Philox4x32-10 trials (Salmon et al., SC'11).
 *   paircheck13/14  1 admits creation between beads 2 / 3 bonds apart; beads
 *                 1 bond apart never bond again, beads >= 4 apart always may.
 *   max_rounds    0 = repeat mutual-nomination rounds until none matches;
 *                 k > 0 = at most k rounds (1 = the fix's single nomination).
 *   prob_mode     0 = one uniform per trial: success iff u < floor(p 2^32);
 *                 1 = the fix's average of two uniforms: u0 + u1 < 2 floor(p 2^32).
 *   reactive_mask bead types of the reactive group; every rule acts only on
 *                 pairs / bonds of two reactive beads.
 *   flags         DYNBOND_FLAG_*.
 *   cell_scale    0 = autotune on the first dynbond_step (dynbond_autotune);
 *                 k >= 1: cell edge along x and y = k x the largest creation
 *                 distance (the reach).
 *   cell_zdiv     with cell_scale k >= 1: cells are cell_zdiv times thinner
 *                 along z (0 = 1, cubic cells).  Along z the search reads, in
 *                 each cell column, the cells overlapping [z - reach, z + reach].
 *                 The cell geometry never changes results.
 *   block_size    0 = default (256) threads per block for the bead passes.
 *   spin_limit    0 = default; iterations of every bounded device-side wait.
 */
typedef struct dynbond_params {
  uint64_t seed;
  int32_t paircheck13;
  int32_t paircheck14;
  int32_t max_rounds;
  int32_t prob_mode;
  uint32_t reactive_mask;
  int32_t flags;
  int32_t cell_scale;
  int32_t block_size;
  int32_t spin_limit;
  int32_t cell_zdiv;
  int32_t reserved[4];
} dynbond_params;

/*
 * Bonded force field, indexed by type (entry 0 unused):
 *   bond      E = bond_k (r - bond_r0)^2; each endpoint feels the force of the
 *             type IT stores and books half the energy (directional bonds,
 *             Sec. 2: equal potentials both ways conserve momentum);
 *   angle     angle_style 0: E = angle_k (1 + cos theta), theta the angle at
 *             the centre bead; angle_style 1: E = angle_k (theta -
 *             angle_theta0)^2 (the DNA angles of Sec. 3, theta0 in radians),
 *             its forces taken through the unit normal of the plane of the
 *             three beads, exact up to rounding at every angle; exactly
 *             collinear beads (no plane) get no angle force, which is the
 *             exact force when theta0 is 180 degrees;
 *   dihedral  E = dihedral_k (1 + dihedral_d cos phi) (the form of Sec. 3),
 *             phi = 180 degrees for the trans conformation.
 * An angle_style other than 0 or 1 is EINVAL.
 */
typedef struct dynbond_forcefield {
  double bond_k[DYNBOND_MAX_TYPES];
  double bond_r0[DYNBOND_MAX_TYPES];
  double angle_k[DYNBOND_MAX_TYPES];
  double dihedral_k[DYNBOND_MAX_TYPES];
  int32_t dihedral_d[DYNBOND_MAX_TYPES];
  double angle_theta0[DYNBOND_MAX_TYPES];
  int32_t angle_style[DYNBOND_MAX_TYPES];
} dynbond_forcefield;

/*
 * The system, read during dynbond_create() only.
 *   bead_offset[R+1], box_q[R]  replica bead ranges and periodic box edges
 *                 (quantized units, 2 <= box_q < 2^31).
 *   form_scale[R], break_scale[R]  nullable (= 1): the trial probability of a
 *                 creation (breakage / conversion) rule in replica r is
 *                 min(1, prob x scale[r]).
 *   rng_stream[R] nullable (= r): 24-bit Philox stream id of replica r.
 *   bead_type[N]  0..15.
 *   bonds[n_bonds*4]  rows (i, j, type stored by i, type stored by j), global
 *                 ids, i and j in the same replica; at most DYNBOND_SLOTS
 *                 bonds per bead.  The initial angles and dihedrals are the
 *                 typed set of every non-cyclic 3- and 4-bead path of this
 *                 graph, which every later call keeps exact.
 */
typedef struct dynbond_system {
  int32_t n_replicas;
  int32_t reserved;
  const int64_t* bead_offset;
  const int64_t* box_q;
  const double* form_scale;
  const double* break_scale;
  const uint32_t* rng_stream;
  const int32_t* bead_type;
  const int32_t* bonds;
  int64_t n_bonds;
} dynbond_system;

/* Per-replica statistics of one call (Appendix step 10), 17 int64 values. */
typedef struct dynbond_stats {
  int64_t candidates;       /* creation candidate pairs */
  int64_t create_matched;   /* mutually nominated creation pairs */
  int64_t bonds_formed;
  int64_t break_candidates; /* bonds eligible for breakbond / convertbond */
  int64_t break_matched;
  int64_t bonds_broken;     /* by breakbond trials (not also killed) */
  int64_t bonds_killed;
  int64_t bonds_converted;  /* by convertbond trials (not also killed) */
  int64_t angles_removed;
  int64_t angles_added;
  int64_t dihedrals_removed;
  int64_t dihedrals_added;
  int64_t n_bonds;          /* totals after the call */
  int64_t n_angles;
  int64_t n_dihedrals;
  int64_t create_rounds;    /* rounds in which this replica matched a creation pair */
  int64_t break_rounds;
} dynbond_stats;

/*
 * Topology export (two-call protocol): call once with null arrays to obtain
 * the counts, then again with caller-allocated host arrays of those sizes.
 *   bonds[n_bonds*4]        (i < j, type stored by i, type stored by j), sorted;
 *   angles[n_angles*4]      (a, b, c, type), a < c, sorted;
 *   dihedrals[n_dihedrals*5] (a, b, c, d, type), a < d, sorted.
 */
typedef struct dynbond_topology {
  int64_t n_bonds;
  int64_t n_angles;
  int64_t n_dihedrals;
  int32_t* bonds;
  int32_t* angles;
  int32_t* dihedrals;
} dynbond_topology;

typedef struct dynbond_ctx dynbond_ctx;
typedef struct CUstream_st* dynbond_stream; /* a cudaStream_t; NULL = legacy default stream */

/*
 * Create a context: validates the rules (the fix's parse-time sanity check)
 * and the system, uploads it to the current CUDA device, builds the initial
 * angle / dihedral lists and captures the per-call work.  Device memory for
 * the topology is sized for the worst case (6 angles and 18 dihedrals per
 * bead), so the lists never overflow.  Returns EINVAL on malformed input,
 * ENOMEM / ECUDA on device failure; *out is NULL on failure.
 */
dynbond_status dynbond_create(const dynbond_params* params, const dynbond_rule* rules, int32_t n_rules,
                              const dynbond_system* system, const dynbond_forcefield* forcefield,
                              dynbond_stream stream, dynbond_ctx** out);

/*
 * One call of the fix (Appendix steps 1-10) at call index `step` on the
 * positions d_pos (device int4[N], 16-byte aligned, read only; EINVAL if
 * misaligned).  Trials are keyed by
 * (seed, step, pair), so repeating a step index repeats its random numbers.
 * h_stats (nullable, host [n_replicas]): when given, the call waits for the
 * device and fills the statistics, and device errors are returned.
 */
dynbond_status dynbond_step(dynbond_ctx* ctx, const int32_t* d_pos, uint64_t step, dynbond_stats* h_stats);

/*
 * Bonded forces of the current topology at d_pos (device int4[N], read only).
 * The topology is the state the last dynbond_step left (Appendix steps 7 and
 * 9: the bonds with the type each end stores, and the typed angles and
 * dihedrals); the potentials are those of dynbond_forcefield: each end of a
 * bond feels the force of the type it stores (the directional half bonds of
 * Sec. 2), angles and dihedrals follow the forms of Sec. 3.
 *   d_force  device float4[N], overwritten (w = 0), FP32 per term;
 *   d_ev     device double[R*7], overwritten: per replica (E, Wxx, Wyy, Wzz,
 *            Wxy, Wxz, Wyz) with W_ab = sum over interactions of
 *            (r_role - r_ref)_a F_role,b, reduced in FP64.
 * d_pos and d_force must be 16-byte aligned (EINVAL otherwise, nothing is
 * launched).  Stream-ordered; device errors surface at the next
 * synchronizing call.
 */
dynbond_status dynbond_forces(dynbond_ctx* ctx, const int32_t* d_pos, float* d_force, double* d_ev);

/*
 * dynbond_step followed by dynbond_forces at the same positions, in one call:
 * the results (topology, statistics, d_force, d_ev) are those of the two calls
 * in turn (forces within the same FP32 tolerance: only the order of the
 * floating-point partial sums may differ).  The bond forces of the new
 * topology depend only on the bonds (Appendix step 7) and the positions, so
 * they run beside the removal and re-creation of angles and dihedrals
 * (Appendix steps 6 and 9) instead of after them.  Arguments, alignment and
 * errors as for dynbond_step and dynbond_forces; h_stats nullable (when given
 * the call waits and fills it).  Contexts created with DYNBOND_FLAG_PROFILE or
 * DYNBOND_FLAG_PERSISTENT run the two calls in turn.
 */
dynbond_status dynbond_step_forces(dynbond_ctx* ctx, const int32_t* d_pos, uint64_t step, float* d_force,
                                   double* d_ev, dynbond_stats* h_stats);

/*
 * dynbond_step + dynbond_forces from host buffers: copies h_pos (int4[N]) to
 * the device, runs both (as dynbond_step_forces), and copies the forces
 * (float4[N]) and energies / virials (double[R*7]) back.  Waits for
 * completion.  h_stats nullable.
 */
dynbond_status dynbond_run_host(dynbond_ctx* ctx, const int32_t* h_pos, uint64_t step, float* h_force,
                                double* h_ev, dynbond_stats* h_stats);

/*
 * Export the current topology: the bond set with the type each end stores
 * and the typed angle and dihedral sets that the last dynbond_step left
 * (Appendix steps 7 and 9; at creation, the typed set of every path of the
 * initial bonds).  Two-call protocol of dynbond_topology above: host arrays,
 * canonical records, sorted.  EINVAL if a given array is smaller than its
 * count.  Synchronizes.
 */
dynbond_status dynbond_get_topology(dynbond_ctx* ctx, dynbond_topology* topo);

/*
 * Order-independent 64-bit hash of each replica's topology (not part of the
 * paper; for logging a long run call by call):
 *   h_r = sum over bond ends (i stores t toward j) of mix(i << 32 | j << 4 | t)
 *       + sum over angles (a, b, c, t) of chain(0xA, a, b, c, t)
 *       + sum over dihedrals (a, b, c, d, t) of chain(0xD, a, b, c, d, t)   (mod 2^64),
 * bead ids local to the replica, records canonical as exported, mix the
 * splitmix64 finalizer (Steele, Lea, Flood, OOPSLA 2014) and
 * chain(x0, x1, ...) = mix(...mix(mix(x0) ^ x1)... ^ xn).
 * Writes n_replicas values to h_out (host).  Synchronizes.
 */
dynbond_status dynbond_topology_hash(dynbond_ctx* ctx, uint64_t* h_out);

/*
 * Autotuning of launch geometry (not part of the paper): the cell edge along x
 * and y (1, 1.25, 1.5, 2 or 3 x the largest creation distance), the z edge (the
 * x / y edge divided by 1, 2 or 4; grids larger than the one allocated at
 * creation are skipped), the candidate search (tiles of cell columns staged
 * in shared memory, or the per-bead search in global memory) and the
 * bead-pass grid size (4, 8 or 16 blocks per SM) are chosen by timing the
 * front of a call (cell binning,
 * breakage nomination and candidate search, which write scratch only; best of
 * three runs) on the positions d_pos; the fastest is kept and the captured work
 * is rebuilt.  No choice changes results.
 * Runs by itself on the first dynbond_step of a context created with
 * cell_scale 0.  out (nullable) receives the choice.
 */
typedef struct dynbond_tuning {
  double cell_scale;
  int32_t bead_blocks_per_sm;
  int32_t candidate_blocks_per_sm;
  float front_ms;   /* device time of the timed front at the chosen geometry */
  int32_t tuned;
  int32_t cell_zdiv; /* z edge = x / y edge / cell_zdiv */
  int32_t octant;    /* 1: columns at least twice the reach wide, the search reads 2 x 2 columns */
  int32_t tiles;     /* 1: the search stages tiles of cell columns in shared memory */
} dynbond_tuning;

dynbond_status dynbond_autotune(dynbond_ctx* ctx, const int32_t* d_pos, dynbond_tuning* out);

/* The context's current launch geometry (tuned or fixed at creation) in *out
 * (host).  EINVAL on NULL arguments.  Launches nothing. */
dynbond_status dynbond_get_tuning(dynbond_ctx* ctx, dynbond_tuning* out);

/* Wait for the context's stream and return any device-side error. */
dynbond_status dynbond_sync(dynbond_ctx* ctx);

/*
 * Per-phase device times (ms) of the last dynbond_step and dynbond_forces of a
 * context created with DYNBOND_FLAG_PROFILE (CUDA events recorded between the
 * phases inside the replayed work, so timing adds no host synchronization to
 * the calls themselves).  Synchronizes the stream, writes up to n values and
 * their static names, and returns the number of phases in *n_out.
 */
dynbond_status dynbond_phase_times(dynbond_ctx* ctx, float* ms, const char** names, int32_t n, int32_t* n_out);

/*
 * Bonded forces without any device allocation, for callers that must not
 * call cudaMalloc: for example a host engine that has handed the GPU's memory
 * to its own pool allocator before loading this library, or a latency-critical
 * loop that cannot accept cudaMalloc's implicit device synchronization.  The
 * paper has no counterpart; this is a service of the library.
 *
 * It evaluates the forces of dynbond_forces for a topology the caller passes
 * in (no context needed).  Every array is caller-owned device memory:
 *   d_pos        int4[n_beads] positions (as for dynbond_step);
 *   d_slots      uint32[n_beads*4] bond slots: (partner << 4 | type this bead
 *                stores), 0 = empty slot;
 *   d_bead_offset int64[n_replicas+1], d_box_q int64[n_replicas];
 *   d_angles     int32[n_angles*4] (a, b, c, type), replica = that of b;
 *   d_dihedrals  int32[n_dihedrals*5] (a, b, c, d, type), replica = that of b;
 *   d_force      float4[n_beads] output (overwritten, w = 0);
 *   d_ev         double[n_replicas*7] output (E, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz).
 * Its scratch (the FP64 accumulators of up to DYNBOND_NOALLOC_MAX_REPLICAS
 * replicas and one error word, 229 KB) is a fixed array in device memory that
 * every GPU loading the library holds until the process exits; n_replicas
 * above that limit returns EINVAL.  The first call on a device looks up the
 * array's device address once (cudaGetSymbolAddress), so make that first call
 * outside any stream capture; no call may follow a cudaDeviceReset of that
 * device in the same process.  All calls on a device share the array: calls
 * that overlap on the GPU (different streams, no ordering) race and give
 * wrong energies.
 * Every bead id is checked on the device: a bond partner outside its bead's
 * replica, an angle or dihedral bead outside the replica of its centre bead
 * b, or an angle / dihedral type outside 0..15 is never dereferenced; the
 * term is skipped (the others are still computed) and the call returns
 * EINVAL.  Work is enqueued on `stream` and the call waits for it to finish
 * (to read the error word).  Returns EINVAL for bad sizes, NULL or misaligned
 * pointers (positions, slots and forces 16-byte, offsets, boxes and d_ev
 * 8-byte, records 4-byte aligned) and bad ids, ECUDA if a CUDA call fails.
 */
dynbond_status dynbond_forces_noalloc(const int32_t* d_pos, const uint32_t* d_slots, const int64_t* d_bead_offset,
                                      const int64_t* d_box_q, int32_t n_replicas, int64_t n_beads,
                                      const int32_t* d_angles, int64_t n_angles, const int32_t* d_dihedrals,
                                      int64_t n_dihedrals, const dynbond_forcefield* ff, float* d_force,
                                      double* d_ev, dynbond_stream stream);

/*
 * Molecular-dynamics harness (the DPD systems of Sec. 3): velocity-Verlet
 * with the DPD force field F_ij = (a w - gamma w^2 (rhat . v_ij) +
 * sigma w xi / sqrt(dt)) rhat, sigma^2 = 2 kT gamma, w = 1 - r / rc, between
 * every pair closer than rc except beads fewer than 3 bonds apart, plus the
 * bonded forces of the context.  Positions stay on the int32 grid: each drift
 * adds round(v dt 2^20) and wraps into the box.  xi is a Gaussian drawn from
 * Philox4x32-10 on (lower id, higher id, step), the same for both beads of a
 * pair.  One replica per context.  dynbond_md_advance runs n_steps steps from
 * step index first_step on d_pos (int4[N], updated) and d_vel (float4[N],
 * updated, w ignored), recomputing the forces at first_step first (the
 * topology may have changed since the last call); d_ev (nullable, device
 * double[7]) receives the bonded energy / virial of the last step.  Waits for
 * completion.
 */
typedef struct dynbond_dpd {
  double a;      /* conservative amplitude */
  double gamma;  /* friction */
  double kT;
  double rc;     /* cutoff */
  double dt;
  double mass;
  uint64_t seed;
} dynbond_dpd;

typedef struct dynbond_md dynbond_md;

dynbond_status dynbond_md_create(dynbond_ctx* ctx, const dynbond_dpd* dpd, dynbond_md** out);
dynbond_status dynbond_md_advance(dynbond_md* md, int32_t* d_pos, float* d_vel, int64_t n_steps, uint64_t first_step,
                                  double* d_ev);
/*
 * The DPD pair forces alone (Sec. 3: F^C + F^D + F^R along r_ij for r < r_c,
 * none between beads fewer than 3 bonds apart) at d_pos (int4[N]) and d_vel
 * (float4[N], w ignored) for step index `step` (which selects the Gaussian
 * numbers xi), written to d_force (device float4[N], w = 0).  All three
 * 16-byte aligned (else EINVAL).  Positions and velocities are not changed.
 * Waits for completion.
 */
dynbond_status dynbond_md_pair_forces(dynbond_md* md, const int32_t* d_pos, const float* d_vel, uint64_t step,
                                      float* d_force);
void dynbond_md_destroy(dynbond_md* md);

/* Human-readable text of the last error of ctx (never NULL). */
const char* dynbond_last_error(const dynbond_ctx* ctx);

const char* dynbond_status_string(dynbond_status status);

void dynbond_destroy(dynbond_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DYNBOND_H */
