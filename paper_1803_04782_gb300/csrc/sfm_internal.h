// sfm_internal.h -- device data layout and kernel launchers shared by the
// C-ABI host code (sfm_api.cu) and the kernels (sfm_kernels.cu, sfm_field.cu,
// sfm_batch.cu, sfm_surrogate.cu, sfm_noalloc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sfm.h"

namespace sfm {

constexpr int kFree = 0, kWall = 1, kExit = 2;
constexpr int32_t kDInf = 1 << 23;  // guidance distance of unreachable su (and WALL su, as exported)
// the guidance array's value on WALL su inside the library: it marks the su
// inadmissible, so a decision needs no read of the cell grid; exported as kDInf
constexpr int32_t kDWall = kDInf + 1;

// Three-component field gather (radius > 50): a CTA owns a 32 x 32 su tile;
// warp w owns rows 4w..4w+3 of it, lane l owns column l.
constexpr int kTile = 32;
// Rows of the band buffer beyond a band's: the row above the band and the
// next band's first tile row (the ring of run_tick's banded field)
constexpr int kBandExtraRows = kTile + 1;
constexpr int kFieldThreads = 256;
constexpr int kRowsPerThread = kTile / (kFieldThreads / 32);  // 4
constexpr int kStageCap = 2048;    // pedestrians staged in shared memory per chunk
constexpr int kMaxHaloBins = 128;  // bins touched by one tile's halo (checked)
constexpr int kBin = 32;           // side of a pedestrian bin (one warp column per su)
// class-table gather: a warp owns a 16 x 16 su footprint (half-warp h = rows
// 8h..8h+7, lane = column) or a 32 x 16 one (lane = column, 16 rows), 32
// warps per CTA.  The 4 heading-class tables sit in shared memory with row
// stride SP = 2 (mod 4), which puts the two half-warps' rows (8 SP apart) on
// disjoint banks.  A "wide" stride leaves >= 31 zero columns after each row's
// 2r + 1, so a lane outside a pedestrian's reach reads a zero and no lane
// needs a range test; the narrow stride 102 (radius 42..50, where wide tables
// would not fit in shared memory) keeps the test.
constexpr int kV2Rows = 8;         // rows per lane of the 16 x 16 footprint
constexpr int kFieldPadRows = 15;  // zero rows above/below each class table
constexpr int kV2Threads = 1024;
constexpr int kTableGuard = 32;    // zero floats in front of the tables in shared memory
constexpr int kNarrowStride = 102;
constexpr int kNumStrideClasses = 7;  // the wide strides 34, 50, ..., 114, then 102
constexpr int kMaxTableRadius = 50;   // largest radius of the class-table gather
constexpr int kMaxTableStride = 114;

constexpr int stride_of_class(int ci) { return ci < 6 ? 34 + 16 * ci : kNarrowStride; }
constexpr int class_of_stride(int sp) { return sp == kNarrowStride ? 6 : (sp - 34) / 16; }
constexpr bool wide_stride(int sp) { return sp != kNarrowStride; }

// Row stride of the class tables for radius r (0: beyond the gather).
constexpr int class_table_stride_of(int r) {
  if (r < 0 || r > kMaxTableRadius) return 0;
  for (int ci = 0; ci < 6; ++ci)
    if (stride_of_class(ci) >= 2 * r + 32) return stride_of_class(ci);
  return kNarrowStride;  // 2r + 1 <= 101
}
constexpr size_t class_table_floats_of(int r) {
  return class_table_stride_of(r)
             ? (size_t)4 * (2 * r + 1 + 2 * kFieldPadRows) * class_table_stride_of(r)
             : 0;
}
constexpr size_t max_class_table_floats(int rmax) {
  size_t m = 0;
  for (int r = 0; r <= rmax; ++r) m = class_table_floats_of(r) > m ? class_table_floats_of(r) : m;
  return m;
}
// shared memory of a gather CTA: guard, tables, per-warp record scratch
static_assert((kTableGuard + max_class_table_floats(kMaxTableRadius)) * 4 +
                      kV2Threads / 32 * 32 * 8 <= 227 * 1024 - 1024,
              "class tables exceed shared memory");

// Row-trimmed class-table gather (sfm_field3.cu): 32 x 32 su footprints,
// lane = column, blocks of 8 rows.  Seven zero rows above
// and below each window (a visit reads whole blocks) and at least 31 zero
// columns after each row; the row stride is one of a few compile-time
// classes.  Radius 1..40.
constexpr int kField3PadRows = 7;
constexpr int kShape16x16 = 0, kShape32x16 = 1, kShape32x32 = 2;
constexpr int field3_stride(int r) {
  // >= 2r + 32: zero columns for 32 lanes
  if (r < 1 || r > 40) return 0;
  for (int sp = 48; sp <= 112; sp += 32)
    if (sp >= 2 * r + 32) return sp;
  return 0;
}
constexpr size_t field3_table_floats(int r) {
  return field3_stride(r) ? (size_t)4 * (2 * r + 1 + 2 * kField3PadRows) * field3_stride(r) : 0;
}
constexpr size_t max_field3_table_floats() {
  size_t m = 0;
  for (int r = 0; r <= kMaxTableRadius; ++r)
    m = field3_table_floats(r) > m ? field3_table_floats(r) : m;
  return m;
}
static_assert((kTableGuard + max_field3_table_floats()) * 4 + kV2Threads / 32 * 32 * 8 <=
                  227 * 1024,
              "row-trimmed gather tables exceed shared memory");
// the row-trimmed footprint `shape` can run at radius r
constexpr bool field3_shape_ok(int shape, int r) {
  return field3_stride(r) != 0 && shape == kShape32x32;
}

// device error flags (sticky until read by a synchronising call)
enum : uint32_t {
  kErrPlaceConflict = 1u,  // two pedestrians on one su, or on a WALL/EXIT su
  kErrPlaceRange = 2u,     // off-lattice position or class > 8
  kErrEnroll = 4u,         // more than 8 registrants for one su (impossible by construction)
  kErrHalo = 8u,           // a tile's halo touched more bins than kMaxHaloBins
  kErrTimeout = 16u,       // a bounded device wait gave up
};

struct Counters {
  unsigned long long moved;
  unsigned long long exited;
  int max_registrants;
  uint32_t err;
  long long t;  // tick counter read by the vote and advanced by the commit
  // the class-table gather's footprint tickets: next ticket, CTAs done; zero
  // between launches (the launch's last CTA puts them back), so launches
  // sharing one context's counters run one at a time, in stream order
  unsigned int field_tickets[2];
  // decisions taken since the placement, and those among them whose best
  // and second-best admissible energies lie within 1e-5 of their magnitude
  // (near ties, which a differently rounded field may break the other way)
  unsigned long long decided;
  unsigned long long near_ties;
};

// Multi-su pedestrians (Sec. 2): pedestrian p occupies the w[p] x h[p]
// rectangle (odd sides) centred on its centre su; occ holds p on every su of
// it.  w == nullptr: every pedestrian is 1 x 1 (the plain model).
struct Sizes {
  const uint8_t* w = nullptr;
  const uint8_t* h = nullptr;
};
constexpr int kMaxPedSide = 15;  // largest width / height of a pedestrian

// Geometry and model constants passed by value to every kernel.
struct Geo {
  int W, H, px, py;
  int r;
  int nbx, nby;  // bins per row / column
  int opitch;    // row pitch (bytes) of the occupancy-class grid, a multiple of 128
};

// A far part added by the class-table gather's epilogue (the learned
// surrogate): F = (Fs + near sum) + scale * Y~, Y~ the bilinear interpolation
// of an Hc x Wc grid of s x s cells between cell centres (wrapped in periodic
// dimensions, clamped otherwise).  Y == nullptr: no far part.
struct FarPart {
  const float* Y = nullptr;
  int s = 1, Hc = 0, Wc = 0;
  float scale = 0.f;
  float inv_s = 1.f;  // 1 / s
};

struct Tables {
  const float* T0;      // (2r+1)^2: kP d^aP          (pedestrian, isotropic part)
  const float* TX;      // (2r+1)^2: kP d^aP gamma dx/d
  const float* TY;      // (2r+1)^2: kP d^aP gamma dy/d
  const float* KO;      // (2r+1)^2: kO d^aO
  const float* KE;      // (2r+1)^2: kE d^aE
  const float* own;     // [9 heading][9 move]: K_P(Delta_move; h)
  const float* dirdot;  // [9 goal][9 move]: Delta_move . u_goal
  const float2* hvec;   // [9]: unit heading vectors
  const float* CT;      // 4 padded heading-class tables of the v2 gather (or NULL)
  const float* CT3 = nullptr;  // the same in the row-trimmed gather's layout (or NULL)
  int shape = 0;        // class-table gather footprint: kShape16x16 .. kShape32x32
};

// footprint of the class-table gather used when none has been tuned
inline int default_field_shape(int r) {
  return r > 30 ? (field3_stride(r) ? kShape32x32 : kShape32x16) : kShape16x16;
}

// ---- launchers (sfm_kernels.cu) ----
void launch_tables(int r, const sfm_params& p, float* T0, float* TX, float* TY, float* KO,
                   float* KE, float* own, float* dirdot, float2* hvec, cudaStream_t s);
void launch_static_field(const Geo& g, const uint8_t* cell, const Tables& tb, float* Fs,
                         cudaStream_t s);
// One relaxation round of the guidance distances; returns via *changed.
void launch_guidance_init(const Geo& g, const uint8_t* cell, int32_t* D, cudaStream_t s);
void launch_guidance_export(int32_t* D, size_t n, cudaStream_t s);
void launch_guidance_import(const uint8_t* cell, int32_t* D, size_t n, cudaStream_t s);
void launch_guidance_round(const Geo& g, const uint8_t* cell, int32_t* D, const uint8_t* act_in,
                           uint8_t* act_out, int* changed, cudaStream_t s);

void launch_place_clear(int n, const int2* xy, const uint8_t* alive, const Geo& g, int32_t* occ,
                        uint8_t* ocls, cudaStream_t s, const Sizes& sz = Sizes());
void launch_place_scatter(int n, const int2* xy, const uint8_t* heading, const uint8_t* goal,
                          const uint8_t* alive, const uint8_t* cell, const Geo& g, int32_t* occ,
                          uint8_t* ocls, Counters* ctr, cudaStream_t s, const Sizes& sz = Sizes());
// placement of as many 1 x 1 pedestrians: grid entries of the changed ones only
// (from the previous state kept in *_prev, or read in place from the caller's
// device-visible buffers and staged in st_*)
void launch_place_direct(int n, const int2* src_xy, const uint8_t* src_h, const uint8_t* src_g,
                         const uint8_t* src_a, int2* st_xy, uint8_t* st_h, uint8_t* st_g,
                         uint8_t* st_a, int2* xy, uint8_t* heading, uint8_t* goal, uint8_t* alive,
                         uint8_t* choice, uint8_t* won, const uint8_t* cell, const Geo& g,
                         int32_t* occ, uint8_t* ocls, Counters* ctr, cudaStream_t s);
void launch_read_peds(int n, const int2* xy, const uint8_t* heading, const uint8_t* alive, int2* dxy,
                      uint8_t* dh, uint8_t* da, cudaStream_t s);
void launch_place_diff(int n, const int2* xy_prev, const uint8_t* alive_prev,
                       const uint8_t* heading_prev, const int2* xy, const uint8_t* heading,
                       const uint8_t* goal, const uint8_t* alive, const uint8_t* cell, const Geo& g,
                       int32_t* occ, uint8_t* ocls, Counters* ctr, cudaStream_t s);

void launch_bin_count(const Geo& g, const uint8_t* ocls, int32_t* count, cudaStream_t s);
void launch_scan(const int32_t* in, int32_t* out, int n, int32_t* block_tmp, cudaStream_t s);
int scan_tmp_elems(int n);
// Records of each bin in row-major su order, and the pedestrian id of each
// record (the per-pedestrian stages walk pedestrians in this spatial order).
void launch_bin_fill(const Geo& g, const uint8_t* ocls, const int32_t* occ, const int32_t* start,
                     uint32_t* rec, int32_t* rec_id, cudaStream_t s);
// choice = won = 0 for pedestrians that are not alive.
void launch_bins_from_peds(const Geo& g, int n, const int2* xy, const uint8_t* alive,
                           const uint8_t* heading, int32_t* count, int32_t* start,
                           int32_t* scan_tmp, int32_t* slot, uint32_t* key, uint32_t* rec,
                           int32_t* rec_id, cudaStream_t s);
void launch_reset_counters(Counters* ctr, cudaStream_t s);
void launch_clear_dead(int n, const uint8_t* alive, uint8_t* choice, uint8_t* won, cudaStream_t s);

// Field gather; stores lattice rows y in [store_lo, store_hi) at
// out[(y - out_row0) * W + x].  Every su is summed in the same order whatever
// the row range, so banded and unbanded passes agree bit for bit.
// the three-component gather (radius > 50), called by launch_field
void launch_field_v1(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const Tables& tb,
                     const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                     Counters* ctr, cudaStream_t s);
// ring > 0: out is a ring of `ring` rows, row y stored at (y - out_row0) mod
// ring (y - out_row0 < 2 ring); only the row-trimmed gather takes one
// (launch_field_v3 returns false otherwise)
void launch_field(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const Tables& tb,
                  const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                  Counters* ctr, cudaStream_t s, const FarPart& far = FarPart(), int ring = 0);
int class_table_stride(int r);
size_t class_table_floats(int r);
// taper_in < r: entries weighted by 1 up to Euclidean distance taper_in and
// a raised cosine down to 0 at r (the surrogate's near part); default none
void launch_class_tables(int r, const sfm_params& p, float* T, cudaStream_t s,
                         double taper_in = 1e30);
// the row-trimmed gather (sfm_field3.cu): false (nothing launched) when the
// radius, the tables or the footprint do not select it
bool launch_field_v3(const Geo& g, const int32_t* bin_start, const uint32_t* rec,
                     const Tables& tb, const float* Fs, float* out, int out_row0, int store_lo,
                     int store_hi, unsigned int* tickets, cudaStream_t s, int ring = 0);
void launch_class_tables3(int r, const sfm_params& p, float* T, cudaStream_t s);

// The per-pedestrian stages visit the live pedestrians of bins [b_lo, b_hi)
// through rec_id (n bounds the launch).  F rows: lattice rows [y_lo, y_hi) at
// buffer row (y - y_lo + main_off), lattice row lo_row at buffer row 0 and
// hi_row at buffer row hi_off.
// Walk periods (Sec. 2): pedestrian p may move only on ticks t with
// t mod period[p] = phase[p] (t = ctr->t, read on the device); period ==
// nullptr: every pedestrian is active.
struct WalkPeriods {
  const uint8_t* period = nullptr;
  const uint8_t* phase = nullptr;
  const Counters* ctr = nullptr;
};

// streaming multiprocessors of the current device (its attribute, cached)
int device_sm_count();
void launch_decide(int n, const int32_t* rec_id, const int32_t* bin_start, int b_lo, int b_hi,
                   const int2* xy, const uint8_t* heading, const uint8_t* goal,
                   const uint8_t* cell, const uint8_t* ocls, const int32_t* D, const float* F,
                   int main_off, int lo_row, int hi_row, int hi_off, int y_lo, int y_hi,
                   const Geo& g, float beta, const Tables& tb, uint8_t* choice, cudaStream_t s,
                   const WalkPeriods& wp = WalkPeriods(), const Sizes& sz = Sizes(),
                   const int32_t* occ = nullptr, Counters* ctr = nullptr, int ring = 0);
void launch_vote(int n, const int32_t* rec_id, const int32_t* bin_start, const int2* xy,
                 const uint8_t* choice, const int32_t* occ, const Geo& g, uint64_t seed,
                 Counters* ctr, uint8_t* won, cudaStream_t s, const Sizes& sz = Sizes(),
                 const int32_t* gid = nullptr);
void launch_commit(int n, const int32_t* rec_id, const int32_t* bin_start, int2* xy,
                   uint8_t* alive, uint8_t* heading, const uint8_t* choice, const uint8_t* won,
                   const uint8_t* cell, int32_t* occ, uint8_t* ocls, const Geo& g, Counters* ctr,
                   cudaStream_t s, const Sizes& sz = Sizes());

}  // namespace sfm
