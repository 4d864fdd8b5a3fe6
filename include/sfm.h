/*
 * sfm.h -- C ABI of the GB300 (sm_103a) implementation of the discrete social
 * field pedestrian model of Yu, Zhu, Wu and Zhang, "Improved OpenCL-based
 * Implementation of Social Field Pedestrian Model".
 *
 * One call of sfm_step() advances the simulation by ticks of the paper's
 * Alg. 1: field superposition (sub-job k-5 of Sec. 3.1, here a per-su gather),
 * each pedestrian's choice among its 9 candidate su (k-2), the election of
 * one registrant per contested su (k-3, the enrollment container of Sec. 3.1
 * item s-2) and the move commit (k-4).
 *
 * Model laws (the paper names the field kinds in Sec. 2 and leaves their
 * formulas to its predecessors; the library implements this reading):
 *   F(c) = sum_p K_P(c-x_p; h_p) + sum_{WALL o} K_O(c-o) + sum_{EXIT e} K_E(c-e)
 *   K_P(d; h) = kP |d|^aP (1 + gamma (h.d)/|d|),  K_O = kO |d|^aO,  K_E = kE |d|^aE
 *   each zero unless 0 < max(|dx|,|dy|) <= r (square (2r+1)^2 geometry; the
 *   paper's "7x7" field is r = 3); minimum-image offsets in periodic dims.
 *   E_p(k) = F(c_k) - [k>0] K_P(Delta_k; h_p) + guide_p(k); choice = argmin,
 *   ties to the smallest k; guide = beta (D(c_k)-D(x_p))/5 for exit-seekers
 *   (D = 5-7 chamfer geodesic distance to the nearest exit), or
 *   -beta Delta_k . u_goal for pedestrians with a fixed desired direction.
 *   Election priority: SplitMix64 output indexed by (seed, tick, id).
 *
 * Conventions for every entry point:
 *   - Lattices are row-major, index y*W + x; x is the column.
 *   - Direction classes 0..8: 0 stay, then (1,0) (1,1) (0,1) (-1,1) (-1,0)
 *     (-1,-1) (0,-1) (1,-1).
 *   - Host buffers passed in are owned by the caller and are copied before
 *     the call returns (or, for device buffers, before the next call on the
 *     context's stream).  Device memory of a context is allocated and owned
 *     by the library and released by sfm_destroy.
 *   - `on_device` flags say whether a pointer is device memory (1) or host
 *     memory (0).  Host destinations of sfm_read_* are written synchronously.
 *   - Every call returns an sfm_status; sfm_last_error() gives the message of
 *     the last failure on that context (or of the last failed sfm_create when
 *     given NULL).  Errors raised by kernels are reported by the next
 *     synchronising call (sfm_sync, sfm_read_*, sfm_stats, sfm_place).
 *   - A context is used from one host thread at a time; all work is issued on
 *     the stream given to sfm_create (NULL = the legacy default stream).
 */
#ifndef SFM_H_
#define SFM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFM_ABI_VERSION 5
#define SFM_MAX_RADIUS 64
#define SFM_NSTAGES 6

typedef struct sfm_ctx sfm_ctx; /* opaque, library-owned */

typedef enum sfm_status {
  SFM_OK = 0,
  SFM_EINVAL = 1,    /* bad argument (sizes, radius, classes, NULL pointer) */
  SFM_ENOMEM = 2,    /* device allocation failed */
  SFM_EBUDGET = 3,   /* the resident lattice arrays exceed hbm_budget_bytes */
  SFM_ECUDA = 4,     /* a CUDA runtime call or a kernel failed */
  SFM_ECONFLICT = 5, /* placement overlaps, sits on a WALL/EXIT su or off-lattice */
  SFM_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  SFM_ESTATE = 7     /* call out of order (e.g. step before place) */
} sfm_status;

/* Lattice geometry. periodic_x / periodic_y wrap that dimension (the paper's
 * experiments use periodic boundaries, Sec. 5); a periodic extent must be at
 * least 2r+1 so that one image at most lies inside a window. */
typedef struct sfm_lattice {
  int32_t W, H;
  int32_t periodic_x, periodic_y;
} sfm_lattice;

/* Model parameters.  r in [0, SFM_MAX_RADIUS].  seed feeds the election hash.
 * hbm_budget_bytes: 0 = unlimited; otherwise the field is computed in row
 * bands whose buffers fit the budget left after the resident arrays (the
 * divide-and-conquer split of Sec. 3.3, Eq. 1).  bin: side of the square
 * pedestrian bins used by the gather (0 = library default). */
typedef struct sfm_params {
  int32_t r;
  int32_t bin;
  float kP, aP, gamma;
  float kO, aO;
  float kE, aE;
  float beta;
  uint64_t seed;
  uint64_t hbm_budget_bytes;
} sfm_params;

typedef struct sfm_stats_t {
  int64_t t;               /* ticks simulated since creation (or sfm_set_time) */
  int64_t n;               /* pedestrians placed */
  int64_t alive;           /* still on the lattice */
  int64_t exited;          /* left through exits */
  int64_t moved_total;     /* committed moves since placement */
  int32_t max_registrants; /* largest enrollment seen in a vote (<= 8) */
  int32_t bands;           /* row bands per field pass (1 = unblocked) */
  uint32_t error_flags;    /* device-side invariant violations (0 = none) */
  int32_t pad_;
  int64_t device_bytes;    /* device memory held by the context */
  int64_t kernel_launches; /* kernels this context has launched since creation */
  int64_t decided;         /* decisions (k-2) taken since placement */
  int64_t near_ties;       /* of those, decisions whose best and second-best
                              admissible energies E_a <= E_b satisfy
                              E_b - E_a <= 1e-5 (M_a + M_b), M = |F| + |own
                              field term| + |guidance term| of the candidate:
                              near ties, which a field rounded otherwise may
                              break either way (counted, not an error) */
} sfm_stats_t;

/* Stage indices for sfm_stage_times. */
enum {
  SFM_STAGE_BIN = 0,    /* S1: counting sort of pedestrians into bins */
  SFM_STAGE_FIELD = 1,  /* S2: field gather (k-5 in the paper) */
  SFM_STAGE_DECIDE = 2, /* S3: 9-candidate decision (k-2) */
  SFM_STAGE_VOTE = 3,   /* S4: election (k-3) */
  SFM_STAGE_COMMIT = 4, /* S5: commit (k-4) */
  SFM_STAGE_STEP = 5    /* whole tick */
};

/* ABI version compiled into the library. */
int32_t sfm_abi_version(void);

/* Bytes of the lattice-sized arrays a context keeps resident whatever the
 * budget (cells, static field, guidance distances, occupancy and its class
 * grid).  A budget of sfm_resident_bytes(lat) + 4*W*(rows+33) leaves room for
 * field bands of `rows` rows (rounded down to a multiple of 32): the band
 * buffer holds a band, the row above it and the next band's first 32 rows. */
uint64_t sfm_resident_bytes(const sfm_lattice* lat);

/* Create a context for one lattice: the discrete space of Sec. 2 (space
 * units, su, with static openings and obstacles whose omnidirectional fields
 * Sec. 2 names), set up once before the loop of Alg. 1 (Sec. 3.1).
 * cell: W*H bytes, 0 FREE, 1 WALL,
 * 2 EXIT (host or device per cell_on_device).  Computes the kernel tables,
 * the static field of WALL and EXIT su and the guidance distances on the
 * device (once per scene).  stream: a cudaStream_t or NULL.  On failure *out
 * is NULL and sfm_last_error(NULL) describes the error.
 * Errors: SFM_EINVAL, SFM_ENOMEM, SFM_EBUDGET, SFM_ECUDA. */
sfm_status sfm_create(const sfm_lattice* lat, const uint8_t* cell, int32_t cell_on_device,
                      const sfm_params* prm, void* stream, sfm_ctx** out);

/* Release every device buffer of the context (synchronises its stream). */
void sfm_destroy(sfm_ctx* ctx);

/* Message of the last failure on ctx (ctx == NULL: last failed sfm_create
 * on this thread).  Never NULL; valid until the next call on ctx. */
const char* sfm_last_error(const sfm_ctx* ctx);

/* Place the crowd that the loop of Alg. 1 (Sec. 3.1) advances: pedestrians
 * of 1 x 1 su with walk period 1, as in the experiments of Sec. 5 (the
 * sized and periodic variants of Sec. 2 are sfm_place_sized and
 * sfm_set_walk_periods).
 * (Re)place n pedestrians, replacing any previous set (the step counter is
 * kept).  xy: n pairs (x, y) int32; heading: n classes 0..8 (NULL = 0);
 * goal: n classes, 0 = exit-seeker, 1..8 = fixed desired direction (NULL = 0);
 * alive: n flags (NULL = all alive).  Validates on the device and returns
 * SFM_ECONFLICT if two live pedestrians share a su or one sits on a WALL or
 * EXIT su or off-lattice.  Synchronising.  A placement of as many
 * pedestrians as the previous one, with the same sizing and no walk periods
 * set, keeps the captured tick graphs (a place / step / read loop replays
 * them); any other placement drops them and its first tick runs stage by
 * stage.  A placement of as many 1 x 1 pedestrians also rewrites the
 * occupancy grids only for the pedestrians whose su, alive flag or heading
 * it changes (the others stay as the previous placement and the ticks since
 * left them), with the same checks; a loop that hands back what it read
 * changes none.  When every array given is device memory or pinned host
 * memory mapped into the device's address space (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister), such a placement reads them in place,
 * without copies; pageable host memory is copied in. */
sfm_status sfm_place(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                     const uint8_t* goal, const uint8_t* alive, int32_t on_device);

/* Set the tick counter used by the election hash. */
sfm_status sfm_set_time(sfm_ctx* ctx, int64_t t);

/* Advance nsteps ticks: nsteps passes of the while loop of Alg. 1 (Sec.
 * 3.1), each k-1 (bins), k-5's superposition computed first as a gather of
 * the tick-start field, k-2 (9-candidate choice), k-3 (election) and k-4
 * (move commit, exits).  Asynchronous on the context's stream. */
sfm_status sfm_step(sfm_ctx* ctx, int32_t nsteps);

/* Compute the field of the current state into the field buffer without
 * moving anybody (bins + gather only).  Asynchronous. */
sfm_status sfm_compute_field(sfm_ctx* ctx);

/* Times the field gather of the current state with each of its warp
 * footprints (see sfm_set_field_footprint) and keeps the fastest for this
 * context (the choice survives later placements).  *shape_out (may be
 * NULL): 0..3.  The fields computed are identical either way.
 * Synchronising; moves nobody. */
sfm_status sfm_autotune(sfm_ctx* ctx, int32_t* shape_out);

/* Checkpoint and resume.  sfm_snapshot writes the context's dynamic state
 * (tick counter, exit and move counters, every pedestrian's position,
 * heading, goal and alive flag, and its walk period and size when set) into
 * buf, a caller-owned host buffer of *len bytes; buf == NULL only stores the
 * size needed in *len (a buffer too small is SFM_EINVAL, *len = size
 * needed).  sfm_restore places that state in a context created with the same
 * lattice, cells and model parameters (lattice size, boundaries, radius and
 * the parameters are checked; SFM_EINVAL otherwise, the context unchanged);
 * the run then continues bit for bit as the snapshotted one would.  The
 * format is this library's (little-endian, versioned).  Both synchronise. */
sfm_status sfm_snapshot(sfm_ctx* ctx, void* buf, size_t* len);
sfm_status sfm_restore(sfm_ctx* ctx, const void* buf, size_t len);

/* Multi-su pedestrians (Sec. 2 of the paper; its Table V): as sfm_place, plus
 * width[n] and height[n] (host or device per on_device): odd sides in
 * [1, 15].  Pedestrian p occupies the width x height rectangle of su centred
 * on xy[p] (wrapped in periodic dimensions; a periodic extent must be at
 * least 2 * side + 3); only the centre emits its field.  A move is
 * admissible iff every su the rectangle newly enters is inside, not WALL and
 * not covered by another pedestrian at tick start; a mover claims those su
 * and wins iff its (priority, id) is the smallest among the movers whose
 * claims meet its own; it leaves when its new rectangle meets an EXIT su.
 * Rectangles must not overlap each other or WALL su, and centres must be on
 * FREE su (else SFM_ECONFLICT, nothing placed).  A later sfm_place returns to
 * 1 x 1 pedestrians.  Not supported by the surrogate or the batch. */
sfm_status sfm_place_sized(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                           const uint8_t* goal, const uint8_t* alive, const uint8_t* width,
                           const uint8_t* height, int32_t on_device);

/* Walk periods (Sec. 2 of the paper, which adopts them to vary walking
 * speeds under a maximal speed of 1 su per tick): pedestrian p may move only
 * on ticks t with t mod period[p] == phase[p] (t = the context's tick
 * counter, see sfm_set_time) and stays on the others, registering nowhere.
 * period, phase: n bytes each (n of the last sfm_place), host or device per
 * on_device; 1 <= period, phase < period, else SFM_EINVAL and nothing
 * changes.  period == NULL switches periods off (every pedestrian active,
 * the plain model).  Every sfm_place switches them off; call this after it.
 * Synchronising. */
sfm_status sfm_set_walk_periods(sfm_ctx* ctx, const uint8_t* period, const uint8_t* phase,
                                int32_t on_device);

/* Pedestrian numbers for the election (k-3 of Alg. 1, Sec. 3.1): by default
 * pedestrian p of the last placement draws its priority as number p (the
 * SplitMix64 output indexed by (seed, tick, p)) and wins ties by the smaller
 * p.  A context that holds one row band of a larger lattice, with its
 * neighbours' pedestrians near the band edges as ghosts (the row-band
 * decomposition across devices; the divide-and-conquer idea of Sec. 3.3),
 * sets each pedestrian's number in the whole lattice here so that its
 * elections match the whole lattice's.  ids: n int32 (n of the last
 * sfm_place), distinct and >= 0, host or device per on_device; NULL goes
 * back to the indices.  Every sfm_place goes back to the indices; call this
 * after it.  Not for multi-su pedestrians (SFM_EINVAL).  Synchronising. */
sfm_status sfm_set_ids(sfm_ctx* ctx, const int32_t* ids, int32_t on_device);

/* Replace the guidance distances (the 5-7 chamfer distances to the nearest
 * exit that exit-seekers follow) by D: W*H int32 in [0, 2^23], host or
 * device per on_device, 2^23 meaning unreachable; WALL su are marked as
 * walls whatever D holds there.  For a context that is one row band of a
 * larger lattice, whose distances run through the other bands: pass the
 * whole lattice's distances for the band's rows (sfm_read_guidance of a
 * context over the whole lattice gives them).  Synchronising; SFM_EINVAL for
 * values out of range (nothing changed). */
sfm_status sfm_set_guidance(sfm_ctx* ctx, const int32_t* D, int32_t on_device);

/* How the pedestrians are sorted into bins each tick (the bin records and
 * every result are identical either way): 1 = by scanning the per-su class
 * grid (cost follows the lattice area), 2 = from the pedestrian list with
 * atomic counts and an in-bin rank (cost follows the crowd), 0 = automatic
 * (the default: the list when n * 64 < W * H).  Anything else is SFM_EINVAL. */
sfm_status sfm_set_binning(sfm_ctx* ctx, int32_t mode);

/* Sets the warp footprint of the field gather by hand: 0 = 16 x 16 su,
 * 1 = 32 x 16 su (every pedestrian visit reads all 16 rows), 2 = 32 x 32 su
 * on the row-trimmed gather (a visit reads only the 8-row blocks the window
 * reaches; radius 1..40, beyond which 2 runs as 1).  Anything else is
 * SFM_EINVAL.  Ignored (but accepted) when the interaction radius exceeds
 * the class-table gather (r > 50). */
sfm_status sfm_set_field_footprint(sfm_ctx* ctx, int32_t shape);

/* Wait for the context's stream and report device-side errors. */
sfm_status sfm_sync(sfm_ctx* ctx);

/* The superposed field that k-5 of Alg. 1 (Sec. 3.1) maintains: the sum of
 * the five field kinds of Sec. 2 (here static openings and obstacles plus
 * the merged pedestrian kernel) at every su.
 * W*H floats: the field at the start of the last tick (or of the last
 * sfm_compute_field).  SFM_ESTATE in banded mode, where no full-lattice field
 * is resident: use sfm_compute_field_into instead. */
sfm_status sfm_read_field(sfm_ctx* ctx, float* dst, int32_t on_device);

/* Compute the field of the current state band by band straight into dst
 * (W*H floats, host or device); works in every mode. */
sfm_status sfm_compute_field_into(sfm_ctx* ctx, float* dst, int32_t on_device);

/* W*H floats: the static field of WALL and EXIT su. */
sfm_status sfm_read_static_field(sfm_ctx* ctx, float* dst, int32_t on_device);

/* W*H int32: chamfer guidance distances (5 per straight step, 7 per diagonal
 * step; 1<<23 where no exit is reachable or on WALL su). */
sfm_status sfm_read_guidance(sfm_ctx* ctx, int32_t* dst, int32_t on_device);

/* The positions k-4 of Alg. 1 (Sec. 3.1) commits, the headings that orient
 * the directional fields of Sec. 2, and whether each pedestrian is still on
 * the lattice (leaving through openings, Sec. 4.2's task no. 11).
 * Pedestrian state: xy (n pairs), heading classes, alive flags (each may be
 * NULL to skip).  on_device: the buffers are device memory (copied device to
 * device); otherwise host memory: pinned host buffers mapped into the
 * device's address space are written in place by one launch, pageable ones
 * are copied out.  Synchronising. */
sfm_status sfm_read_peds(sfm_ctx* ctx, int32_t* xy, uint8_t* heading, uint8_t* alive,
                         int32_t on_device);

/* Decisions of the last tick: choice class (0..8) and election result
 * (1 = moved) per pedestrian (each may be NULL). */
sfm_status sfm_read_decisions(sfm_ctx* ctx, uint8_t* choice, uint8_t* won, int32_t on_device);

/* Counters of the loop of Alg. 1 (Sec. 3.1): the tick t, pedestrians still
 * on the lattice and those that left through openings (Sec. 4.2, task no.
 * 11), committed moves (k-4), the largest enrollment of one su (k-3; at most
 * 8 by the enrollment container of Sec. 3.1, item s-2) and the near-tie
 * decisions of k-2.  Synchronising. */
sfm_status sfm_stats(sfm_ctx* ctx, sfm_stats_t* out);

/* Per-stage timing.  every = 0: off; every = k >= 1: sfm_step records CUDA
 * events around each stage of every k-th tick (the first tick after this call
 * is one), on the context's stream.  Every record waits for the stream's
 * work before it and the next launch waits for it, so it costs a few
 * microseconds of GPU time; sampling (k > 1) keeps that out of most ticks.
 * After the first tick following a placement (launched stage by stage), a
 * timed tick replays a one-tick CUDA graph whose event record nodes are
 * pointed at fresh events before the replay; untimed ticks replay the
 * untimed graphs.  A batch context times every tick (one event pair around
 * its graph) whatever k is.  every < 0: SFM_EINVAL. */
sfm_status sfm_set_timing(sfm_ctx* ctx, int32_t every);

/* Accumulated milliseconds per stage (SFM_NSTAGES doubles) and the number
 * of timed ticks they cover since the last call; resets the accumulators.
 * Synchronising. */
sfm_status sfm_stage_times(sfm_ctx* ctx, double* ms, int64_t* ticks);

/* ---- Batches of independent lattices -------------------------------------
 * Many small or uneven lattices stepped together: every tick is ONE
 * persistent (cooperative) kernel launch that runs bins, field, decisions,
 * vote and commit for all lattices, separated by grid-wide barriers whose
 * waits are bounded (a barrier that times out ends the launch and the next
 * synchronising call returns SFM_ETIMEOUT).  The field stage walks a work
 * list of (lattice, 32-footprint chunk) items sorted by decreasing cost; the
 * tick launch is captured once in a CUDA graph and replayed.  Each lattice
 * evolves exactly as it would in its own context (same bins, same summation
 * order, its own seed and pedestrian numbering), which the tests check bit
 * for bit.  This batches the paper's concurrency technique (several tasks in
 * flight, Sec. 4.2) across scenarios.
 *
 * sfm_batch_create: nscenes lattices (1..65535); lats[i], cells[i] (host,
 *   W*H bytes each), prms[i] (r <= 50).  The context then accepts
 *   sfm_batch_place, sfm_step, sfm_compute_field, sfm_read_field /
 *   _static_field / _guidance (all lattices concatenated in order, offsets
 *   from sfm_batch_offsets), sfm_read_peds / _decisions (pedestrians
 *   concatenated in lattice order), sfm_stats, sfm_set_time, sfm_sync,
 *   sfm_set_timing / sfm_stage_times (one entry per tick) and sfm_destroy.
 *   Errors as sfm_create.
 * sfm_batch_place: counts[nscenes] (host) pedestrians per lattice; xy,
 *   heading, goal, alive concatenated in lattice order, coordinates local to
 *   each lattice (host or device per on_device).  Errors as sfm_place.
 * sfm_batch_offsets: su_off[nscenes+1] and ped_off[nscenes+1] (either may
 *   be NULL) receive where each lattice starts in the concatenated arrays.
 * sfm_batch_autotune: times the field stage of each radius class (lattices
 *   sharing a class-table row stride) with 16 x 16 and 32 x 16 su warp
 *   footprints and keeps the faster; shape_per_class[7] (may be NULL)
 *   receives 0 (16 x 16) or 1 (32 x 16) for the strides 34, 50, 66, 82, 98,
 *   114 (radius <= 1, 9, 17, 25, 33, 41) and 102 (radius 42..50).  Needs
 *   placed pedestrians; moves nobody.
 * sfm_batch_test_missing_ctas: test hook of the bounded barrier wait; the
 *   next tick's barriers wait for `missing` CTAs that are never launched, so
 *   the tick gives up after about a second and returns SFM_ETIMEOUT (the
 *   context stays usable). */
sfm_status sfm_batch_create(int32_t nscenes, const sfm_lattice* lats, const uint8_t* const* cells,
                            const sfm_params* prms, void* stream, sfm_ctx** out);
sfm_status sfm_batch_place(sfm_ctx* ctx, const int32_t* counts, const int32_t* xy,
                           const uint8_t* heading, const uint8_t* goal, const uint8_t* alive,
                           int32_t on_device);
sfm_status sfm_batch_offsets(const sfm_ctx* ctx, int64_t* su_off, int64_t* ped_off);
sfm_status sfm_batch_autotune(sfm_ctx* ctx, int32_t* shape_per_class);
sfm_status sfm_batch_test_missing_ctas(sfm_ctx* ctx, int32_t missing);

/* ---- Learned field surrogate ----------------------------------------------
 * F_sur(c) = F_static(c) + [exact pedestrian field within Chebyshev radius
 * rn of c] + scale * bilinear(Y)(c), where Y is the output of a 4-layer
 * convolutional network (3->32 5x5, 32->32 3x3, 32->32 3x3, 32->1 3x3, ReLU
 * between layers, "valid" correlations) run on a grid coarsened s times:
 * per s x s cell the pedestrian count and the heading sums, / s^2, with a
 * 5-cell border (wrapped in periodic dimensions, zero otherwise).  Weights
 * and activations are BF16, accumulation FP32.  With s = 8 the network sees
 * +-40 su, the radius of the largest workload; s = 1, rn = 0 is the literal
 * fine-grid network (+-5 su).  Trained on the GPU by this library's forward,
 * backward and Adam kernels against the exact field's far part (cell
 * averages of F - F_near, / scale); the exact path stays the judge.  The
 * paper's future work (Sec. 6) names deep learning only for data collection;
 * this surrogate is an addition, not a paper method.
 *
 * Parameters travel in the order W1 b1 W2 b2 W3 b3 W4 b4, each W laid out
 * [out][in][ky][kx]: sfm_surrogate_nparams() floats.  Contexts used with a
 * surrogate are single, unbanded, with W and H multiples of s. */
typedef struct sfm_surrogate sfm_surrogate; /* opaque */
typedef struct sfm_surrogate_cfg {
  int32_t coarsen;     /* s >= 1 */
  int32_t near_radius; /* rn in [0, min(r, 50)] */
  float target_scale;  /* field units per network output unit (> 0) */
  float lr, beta1, beta2, eps; /* Adam */
  float taper_inner;   /* >= 0: the near part's kernel is weighted 1 up to this
                          Euclidean distance and by a raised cosine down to 0
                          at rn, leaving a smooth remainder to the network;
                          >= rn: no taper (hard cut at the Chebyshev window) */
} sfm_surrogate_cfg;
int32_t sfm_surrogate_nparams(void);
sfm_status sfm_surrogate_create(const sfm_surrogate_cfg* cfg, void* stream, sfm_surrogate** out);
void sfm_surrogate_destroy(sfm_surrogate* sur);
const char* sfm_surrogate_last_error(const sfm_surrogate* sur);
/* host arrays of sfm_surrogate_nparams() floats; set resets the Adam state */
sfm_status sfm_surrogate_set_params(sfm_surrogate* sur, const float* params);
sfm_status sfm_surrogate_get_params(sfm_surrogate* sur, float* params);
/* One forward + backward on a given input: X (host, [3][Hin][Win] floats,
 * rounded to BF16), targets T (host, [Hin-10][Win-10]); loss = 0.5 *
 * mean((Y-T)^2) and its gradients (host, nparams floats, public order). */
sfm_status sfm_surrogate_grad(sfm_surrogate* sur, int32_t Hin, int32_t Win, const float* X,
                              const float* T, float* loss, float* grads);
/* Forward pass alone on a given input: X as for sfm_surrogate_grad, Y (host,
 * [Hin-10][Win-10]) the network's output.  tcgen05 != 0: the 3x3 32 -> 32
 * layers on the tcgen05 kernel that every other surrogate call uses, 0: on
 * the mma.sync kernel (a check of the first against the second).
 * SFM_ETIMEOUT: a tcgen05 convolution's bounded wait ran out; from then on
 * the surrogate runs those layers on mma.sync (every synchronising
 * surrogate call reports such a timeout once). */
sfm_status sfm_surrogate_forward(sfm_surrogate* sur, int32_t Hin, int32_t Win, const float* X,
                                 float* Y, int32_t tcgen05);
/* iters training steps on ctx: each takes the exact field of ctx's current
 * state, one Adam step on the whole coarse lattice, then ticks ctx once so
 * the next step sees a new crowd.  loss_curve: iters floats (host) or NULL. */
sfm_status sfm_surrogate_train(sfm_surrogate* sur, sfm_ctx* ctx, int32_t iters, float* loss_curve);
/* surrogate field of ctx's current state into out (W*H floats, host or device) */
sfm_status sfm_surrogate_field(sfm_surrogate* sur, sfm_ctx* ctx, float* out, int32_t on_device);
/* Decisions with the exact field as fallback.  A tick of sfm_surrogate_step
 * runs the network on the tick's coarse inputs and decides every live
 * pedestrian on F_sur composed at its 9 candidates (the values the lattice
 * pass of sfm_surrogate_field writes there, up to FP32 rounding; the fine
 * lattice itself is not written); a pedestrian whose energy margin
 * (second-best minus best candidate) is at most delta (plus a rounding
 * allowance) is decided again on the exact field at its admissible
 * candidates, computed bit for bit as the exact gather computes it.  If
 * F_sur - F varies by less than the margin over a pedestrian's admissible
 * candidates (max - min), its move equals the exact path's: an error common
 * to all candidates cancels.  delta starts at +infinity: every pedestrian
 * falls back, and such a tick runs neither the network nor the surrogate
 * composition -- it is the exact tick with the field computed at each
 * pedestrian's 9 candidates only (moves equal to sfm_step's bit for bit).
 * sfm_surrogate_set_delta: delta >= 0 (or +inf) by hand.
 * sfm_surrogate_calibrate: on ctx's current state, delta = the `quantile`
 *   (in [0, 1]) over live pedestrians of the spread max - min of F_sur - F
 *   over their admissible candidates; *delta_out (may be NULL) receives it.
 *   Overwrites ctx's field buffer.
 * sfm_surrogate_step: nsteps ticks of ctx (clear, bins, network, decisions
 *   with the fallback, vote, commit), asynchronous on ctx's stream.
 *   Field radius <= 50 (the exact fallback reuses the class-table gather).
 * sfm_surrogate_counts: totals over all surrogate ticks so far of the
 *   pedestrians that fell back and of those decided (synchronising). */
sfm_status sfm_surrogate_set_delta(sfm_surrogate* sur, float delta);
sfm_status sfm_surrogate_calibrate(sfm_surrogate* sur, sfm_ctx* ctx, double quantile,
                                   float* delta_out);
sfm_status sfm_surrogate_step(sfm_surrogate* sur, sfm_ctx* ctx, int32_t nsteps);
sfm_status sfm_surrogate_counts(sfm_surrogate* sur, int64_t* fallbacks, int64_t* decided);
/* Test hook of the bounded waits of the tcgen05 convolution: the next
 * layer-2 launch stops issuing its input copies after `after` tiles per CTA,
 * so its MMA and store warps' waits run out (about a second); the launch
 * then waits for the copies and MMAs it did issue, frees its tensor memory
 * and returns, and the next synchronising surrogate call reports
 * SFM_ETIMEOUT and switches layers 2-3 to mma.sync.  after < 0: SFM_EINVAL. */
sfm_status sfm_surrogate_test_stop_copies(sfm_surrogate* sur, int32_t after);
/* sfm_surrogate_eval, on ctx's current state (overwrites ctx's field and
 * decision buffers):
 *   field_rel_err  sum|F_sur - F| / sum|F - F_static| over the lattice;
 *   flip_rate      fraction of live pedestrians whose surrogate decision,
 *                  with the fallback, differs from the exact path's;
 *   flip_rate_raw  the same without the fallback (decisions on F_sur alone);
 *   fallback_rate  fraction that fell back;
 *   ms_surrogate   bins + network + decisions with the fallback (the
 *                  decision part of a surrogate tick);
 *   ms_exact       bins + exact field + decisions (CUDA events, ctx stream);
 *   ms_surrogate_field  network + the lattice pass of sfm_surrogate_field
 *                  (the surrogate field of every su; its field_rel_err). */
typedef struct sfm_surrogate_report {
  double field_rel_err, flip_rate, flip_rate_raw, fallback_rate, ms_surrogate, ms_exact,
      ms_surrogate_field;
  float delta;
  int32_t decided;
} sfm_surrogate_report;
sfm_status sfm_surrogate_eval(sfm_surrogate* sur, sfm_ctx* ctx, sfm_surrogate_report* report);

/* ---- Field superposition that allocates nothing ------------------------
 * The paper has no counterpart of this entry point: it serves callers that
 * cannot call cudaMalloc, such as a host application or framework that
 * reserves all device memory up front in its own pool and forbids further
 * allocations (or cannot afford the device synchronisation an allocation
 * may cause) while it runs.
 *
 * Computes field[c] = base[c] + sum_p K_P(c - x_p; h_p) over the live
 * pedestrians, the same superposition as the context path (summed in another
 * order, so equal up to FP32 rounding).  Pass the static field read with
 * sfm_read_static_field as `base` for the whole field, or zeros for the
 * pedestrian part alone.  No context is needed.
 *   lat, prm: lattice and model parameters (host).  Only r, kP, aP, gamma are
 *             used.  r must be <= SFM_NOALLOC_MAX_RADIUS; the lattice may
 *             need at most SFM_NOALLOC_MAX_BINS bins of 32 x 32 su; n <=
 *             SFM_NOALLOC_MAX_PEDS.
 *   xy (n int32 pairs), heading (n classes 0..8, or NULL = 0), alive
 *             (n flags, or NULL = all alive): device memory, caller-owned.
 *   base, field: device memory, W*H floats each, caller-owned, not aliased.
 *   stream: cudaStream_t or NULL.  The call waits for the stream.
 * Working memory is a fixed array of device memory inside the library
 * (about 5.2 MB, held by every GPU that loads the library until exit); the
 * first call on a device looks its address up, and the call never calls
 * cudaMalloc, cudaFree or an allocating library routine.  Every call reuses
 * the same array, so calls that overlap on the GPU (other streams or host
 * threads) race and must not be made.
 * Returns SFM_EINVAL for sizes beyond the limits above or bad arguments
 * (before any device work), SFM_ECONFLICT if a live pedestrian is
 * off-lattice or has a class > 8, SFM_ECUDA on a CUDA failure. */
#define SFM_NOALLOC_MAX_PEDS (1 << 20)
#define SFM_NOALLOC_MAX_BINS (1 << 16)
#define SFM_NOALLOC_MAX_RADIUS 47
sfm_status sfm_field_noalloc(const sfm_lattice* lat, const sfm_params* prm, int32_t n,
                             const int32_t* xy, const uint8_t* heading, const uint8_t* alive,
                             const float* base, float* field, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFM_H_ */
