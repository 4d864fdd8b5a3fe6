// sfm_device.cuh -- device building blocks of one tick, shared by the
// single-lattice kernels (sfm_kernels.cu) and the batched persistent tick
// (sfm_batch.cu).  Every function works on one lattice given by its Geo and
// pointers already offset to that lattice's arrays; pedestrian indices are
// indices into the (possibly concatenated) pedestrian arrays.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfm_internal.h"

namespace sfm {

// move offsets of the direction classes 0..8 and the class of the opposite move
static __constant__ int c_dx[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static __constant__ int c_dy[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
static __constant__ int c_opp[9] = {0, 5, 6, 7, 8, 1, 2, 3, 4};
// heading class -> (stored table, x sign, y sign): tables 0 none, 1 E, 2 N,
// 3 NE; x/y mirrors give W, S, NW, SW, SE.  Two bits per class in two
// immediate constants (the table; x mirrored | y mirrored << 1), so a class
// that differs from lane to lane costs no serialised constant-memory read.
constexpr unsigned kClassTab = 0x3B7B4u, kClassMirror = 0x2B500u;
__host__ __device__ __forceinline__ constexpr int class_table(int c) {
  return (int)(kClassTab >> (2 * c)) & 3;
}
__host__ __device__ __forceinline__ constexpr int class_sx(int c) {
  return ((kClassMirror >> (2 * c)) & 1u) ? -1 : 1;
}
__host__ __device__ __forceinline__ constexpr int class_sy(int c) {
  return ((kClassMirror >> (2 * c)) & 2u) ? -1 : 1;
}
static_assert(class_table(0) == 0 && class_table(1) == 1 && class_table(2) == 3 &&
                  class_table(3) == 2 && class_table(4) == 3 && class_table(5) == 1 &&
                  class_table(6) == 3 && class_table(7) == 2 && class_table(8) == 3,
              "heading class tables");
static_assert(class_sx(0) + class_sx(1) + class_sx(2) + class_sx(3) == 4 && class_sx(4) == -1 &&
                  class_sx(5) == -1 && class_sx(6) == -1 && class_sx(7) == 1 && class_sx(8) == 1,
              "heading class x mirrors");
static_assert(class_sy(0) + class_sy(1) + class_sy(2) + class_sy(3) + class_sy(4) + class_sy(5) == 6 &&
                  class_sy(6) == -1 && class_sy(7) == -1 && class_sy(8) == -1,
              "heading class y mirrors");
// the same in constant memory (the footprint gather decodes a batch's records
// with these; its register allocation is tuned with them)
#define SFM_CLASS_ROW(f) {f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8)}
static __constant__ int c_ctab[9] = SFM_CLASS_ROW(class_table);
static __constant__ int c_csx[9] = SFM_CLASS_ROW(class_sx);
static __constant__ int c_csy[9] = SFM_CLASS_ROW(class_sy);
#undef SFM_CLASS_ROW

constexpr int kFieldPad = kFieldPadRows;

// Entry (dx, dy) of stored heading-class table t (0 none, 1 E, 2 N, 3 NE):
// K_P((dx, dy); h_t) = kP d^aP (1 + gamma h_t . (dx, dy) / d) for 0 <
// max(|dx|, |dy|) <= r, else 0; evaluated in FP64 (and rounded to FP32 by
// the caller) so that every table layout holds the same values.  taper_in <
// r: weighted by 1 up to Euclidean distance taper_in and a raised cosine
// down to 0 at r (the surrogate's near part).
__device__ __forceinline__ double class_kernel_value(int t, int dx, int dy, int r, double kP,
                                                     double aP, double gamma, double taper_in) {
  const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
  double v = 0.0;
  if (adx <= r && ady <= r && (adx | ady) != 0) {
    const double hx = (t == 1) ? 1.0 : (t == 3 ? 0.70710678118654752440 : 0.0);
    const double hy = (t == 2) ? 1.0 : (t == 3 ? 0.70710678118654752440 : 0.0);
    const double d = sqrt((double)(dx * dx + dy * dy));
    v = kP * pow(d, aP) * (1.0 + gamma * (hx * dx + hy * dy) / d);
    if (taper_in < r && d > taper_in)
      v *= d >= r ? 0.0 : 0.5 * (1.0 + cos(3.14159265358979323846 * (d - taper_in) / (r - taper_in)));
  }
  return v;
}

// the same move offsets as compile-time functions, so unrolled loops index
// register arrays with constants
__host__ __device__ __forceinline__ constexpr int move_dx(int k) {
  return (k == 1 || k == 2 || k == 8) ? 1 : ((k >= 4 && k <= 6) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int move_dy(int k) {
  return (k >= 2 && k <= 4) ? 1 : ((k >= 6 && k <= 8) ? -1 : 0);
}

__device__ __forceinline__ bool wrap_coord(int v, int n, int periodic, int& out) {
  if (v >= 0 && v < n) {
    out = v;
    return true;
  }
  if (!periodic) return false;
  v %= n;
  if (v < 0) v += n;
  out = v;
  return true;
}

__device__ __forceinline__ int floor_div(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__device__ __forceinline__ int nonzero_bytes(uint32_t v) {
  return __popc((((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v) & 0x80808080u);
}

// Counter-based election priority: SplitMix64 (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t splitmix_nth(uint64_t s, uint64_t i) {
  return mix64(s + i * 0x9e3779b97f4a7c15ULL);
}

// ---------------------------------------------------------------- S1 bins
// One warp covers bins 4*gx .. 4*gx+3 of bin row by (32 rows of the
// 128-byte-pitched class grid, 4 bytes per lane); lanes 8b..8b+7 cover bin b.
__device__ __forceinline__ void bin_count_group(const Geo& g, const uint8_t* __restrict__ ocls,
                                                int32_t* __restrict__ count, int gx, int by,
                                                int lane) {
  const uint8_t* base = ocls + (size_t)by * kBin * g.opitch + gx * 128 + 4 * lane;
  const int rows = min(kBin, g.H - by * kBin);
  int c = 0;
  for (int row = 0; row < rows; ++row)
    c += nonzero_bytes(*reinterpret_cast<const uint32_t*>(base + (size_t)row * g.opitch));
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  const int bx = gx * 4 + (lane >> 3);
  if ((lane & 7) == 0 && bx < g.nbx) count[by * g.nbx + bx] = c;
}

// Records of the group's bins in row-major su order, with the pedestrian
// index (the occupancy value) of each record.
__device__ __forceinline__ void bin_fill_group(const Geo& g, const uint8_t* __restrict__ ocls,
                                               const int32_t* __restrict__ occ,
                                               const int32_t* __restrict__ start,
                                               uint32_t* __restrict__ rec,
                                               int32_t* __restrict__ rec_id, int gx, int by,
                                               int lane) {
  const int sub = lane & 7;
  const int bx = gx * 4 + (lane >> 3);
  const int x = gx * 128 + 4 * lane;
  const uint8_t* base = ocls + (size_t)by * kBin * g.opitch + x;
  const int rows = min(kBin, g.H - by * kBin);
  int off = bx < g.nbx ? start[by * g.nbx + bx] : 0;
  for (int row = 0; row < rows; ++row) {
    const uint32_t v = *reinterpret_cast<const uint32_t*>(base + (size_t)row * g.opitch);
    const int nz = nonzero_bytes(v);
    int inc = nz;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o, 8);
      if (sub >= o) inc += t;
    }
    const int grp = __shfl_sync(0xffffffffu, inc, 7, 8);
    if (nz) {
      int k = off + inc - nz;
      const int y = by * kBin + row;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t cls = (v >> (8 * b)) & 0xffu;
        if (cls) {
          rec[k] = (uint32_t)(4 * sub + b) | ((uint32_t)row << 8) | ((cls - 1u) << 16);
          rec_id[k] = occ[(size_t)y * g.W + x + b];
          ++k;
        }
      }
    }
    off += grp;
  }
}

// ----------------------------------------------------- multi-su pedestrians
// su (cx + i, cy + j), wrapped in periodic dimensions; false if it leaves a
// closed lattice.
__device__ __forceinline__ bool rect_su(const Geo& g, int cx, int cy, int i, int j, size_t& s) {
  int x, y;
  if (!(wrap_coord(cx + i, g.W, g.px, x) & wrap_coord(cy + j, g.H, g.py, y))) return false;
  s = (size_t)y * g.W + x;
  return true;
}

// Every su that the rectangle of half sides (a, b) centred on (x, y) newly
// enters when its centre moves by class k is inside, not WALL and not
// covered by a pedestrian (occ < 0) at tick start.
__device__ __forceinline__ bool strip_free(const Geo& g, const uint8_t* __restrict__ cell,
                                           const int32_t* __restrict__ occ, int x, int y, int a,
                                           int b, int k) {
  const int dx = move_dx(k), dy = move_dy(k);
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      const int ox = i + dx, oy = j + dy;  // offset from the old centre
      if (ox >= -a && ox <= a && oy >= -b && oy <= b) continue;
      size_t s;
      if (!rect_su(g, x, y, ox, oy, s)) return false;
      if (cell[s] == kWall || occ[s] >= 0) return false;
    }
  return true;
}

// Offset d along a dimension of n su: the minimum image when periodic.
__device__ __forceinline__ int image_offset(int d, int n, int periodic) {
  if (!periodic) return d;
  d %= n;
  if (d > n / 2) d -= n;
  if (d < -(n / 2)) d += n;
  return d;
}

// su (sx, sy) is one that pedestrian q (centre (qx, qy), half sides a, b)
// newly enters with move k.
__device__ __forceinline__ bool in_entered(const Geo& g, int sx, int sy, int qx, int qy, int a, int b,
                                           int k) {
  const int ox = image_offset(sx - qx, g.W, g.px), oy = image_offset(sy - qy, g.H, g.py);
  const bool in_old = ox >= -a && ox <= a && oy >= -b && oy <= b;
  const int nx = ox - move_dx(k), ny = oy - move_dy(k);
  return !in_old && nx >= -a && nx <= a && ny >= -b && ny <= b;
}

// ---------------------------------------------------------------- S3 decide
// E over the 9 candidates (stay + 8 neighbours), admissible iff inside, not
// WALL and unoccupied at tick start; the minimum with ties to the smallest
// class.  F rows: lattice rows [y_lo, y_hi) at buffer row y - y_lo + main_off
// (less `ring` when that is >= ring > 0: a ring buffer of `ring` rows),
// lo_row at buffer row 0 and hi_row at hi_off.  own / dirdot: this lattice's
// 81-entry tables.
// Admissible candidates (stay, or inside, not WALL and unoccupied at tick
// start) and the energy E(k) = F(c_k) - K_P(own heading) + guidance; the
// minimum with ties to the smallest class.  With MARGIN, *margin receives
// E(second best) - E(best) over the admissible candidates (+inf when only
// staying is admissible) and *emag (optional) the larger |E| of the two:
// any field error below margin / 2 at every candidate, less FP32 rounding of
// energies of that size, leaves the choice unchanged.  With TIE, *tie
// receives whether the second-best admissible energy lies within 1e-5 of
// the best, relative to the two candidates' energy magnitudes |F| + |own| +
// |guidance| (a near tie: a field rounded otherwise may break it the other
// way).
template <bool MARGIN, bool TIE = false>
__device__ __forceinline__ int pick_move(const float (&f)[9], const int32_t (&dd)[9],
                                         const uint8_t (&oc)[9],
                                         const bool (&okx)[3], const bool (&oky)[3], int h, int gl,
                                         float beta, const float* __restrict__ own,
                                         const float* __restrict__ dirdot, float* margin,
                                         float* emag = nullptr, bool* tie = nullptr) {
  constexpr bool SECOND = MARGIN || TIE;
  int best = 0;
  float bestE = 0.f, second = __int_as_float(0x7f800000);
  float bestM = 0.f, secondM = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    // a WALL su carries kDWall in the guidance array
    const bool adm = (k == 0) || (okx[xi] && oky[yi] && dd[k] != kDWall && oc[k] == 0);
    const float guide = (gl == 0) ? beta * ((float)(dd[k] - dd[0]) / 5.0f) : -beta * dirdot[gl * 9 + k];
    const float e = f[k] - own[h * 9 + k] + guide;
    const float mag = TIE ? fabsf(f[k]) + fabsf(own[h * 9 + k]) + fabsf(guide) : 0.f;
    if (adm && (k == 0 || e < bestE)) {
      if (SECOND && k != 0) {
        second = bestE;
        secondM = bestM;
      }
      best = k;
      bestE = e;
      bestM = mag;
    } else if (SECOND && adm && e < second) {
      second = e;
      secondM = mag;
    }
  }
  if (TIE)
    *tie = second < __int_as_float(0x7f800000) && second - bestE <= 1e-5f * (bestM + secondM);
  if (MARGIN) {
    *margin = second - bestE;
    // size of the energies compared, for a rounding allowance
    if (emag) *emag = fmaxf(fabsf(bestE), second < __int_as_float(0x7f800000) ? fabsf(second) : 0.f);
  }
  return best;
}

// The 3 x 3 candidate block of a pedestrian at q: columns and rows wrapped
// (periodic) or clamped to q (an out-of-lattice candidate repeats q's own
// row or column and is marked inadmissible by okx / oky) ...
__device__ __forceinline__ void candidate_coords(int2 q, const Geo& g, int (&cx)[3], int (&ry)[3],
                                                 bool (&okx)[3], bool (&oky)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    okx[d] = wrap_coord(q.x + d - 1, g.W, g.px, cx[d]);
    oky[d] = wrap_coord(q.y + d - 1, g.H, g.py, ry[d]);
    if (!okx[d]) cx[d] = q.x;
    if (!oky[d]) ry[d] = q.y;
  }
}

// ... and the guidance distance and occupancy class there (a WALL su is
// recognised by its guidance value kDWall, so the cell grid is not read)
__device__ __forceinline__ void candidate_loads(const Geo& g, const uint8_t* __restrict__ ocls,
                                                const int32_t* __restrict__ D, const int (&cx)[3],
                                                const int (&ry)[3], int32_t (&dd)[9],
                                                uint8_t (&oc)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    dd[k] = D[(size_t)ry[yi] * g.W + cx[xi]];
    oc[k] = ocls[(size_t)ry[yi] * g.opitch + cx[xi]];
  }
}

template <bool TIE = false>
__device__ __forceinline__ uint8_t decide_one(
    int p, const Geo& g, const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
    const uint8_t* __restrict__ goal, const uint8_t* __restrict__ cell,
    const uint8_t* __restrict__ ocls, const int32_t* __restrict__ D, const float* __restrict__ F,
    int main_off, int lo_row, int hi_row, int hi_off, int y_lo, int y_hi, float beta,
    const float* __restrict__ own, const float* __restrict__ dirdot,
    const uint8_t* __restrict__ pw = nullptr, const uint8_t* __restrict__ ph = nullptr,
    const int32_t* __restrict__ occ = nullptr, bool* tie = nullptr, int ring = 0) {
  const int2 q = xy[p];
  const int h = heading[p], gl = goal[p];
  // the 3 x 3 neighbourhood (wrapped or clipped); every load is issued
  // before any use so the 36 reads overlap
  int cx[3], ry[3], fr[3];
  bool okx[3], oky[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    okx[d] = wrap_coord(q.x + d - 1, g.W, g.px, cx[d]);
    oky[d] = wrap_coord(q.y + d - 1, g.H, g.py, ry[d]);
    if (!okx[d]) cx[d] = q.x;
    if (!oky[d]) ry[d] = q.y;
    const int ny = ry[d];
    fr[d] = (ny >= y_lo && ny < y_hi) ? ny - y_lo + main_off
                                      : (ny == lo_row ? 0 : (ny == hi_row ? hi_off : 0));
    if (ring && fr[d] >= ring) fr[d] -= ring;
  }
  float f[9];
  int32_t dd[9];
  uint8_t oc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    f[k] = F[(size_t)fr[yi] * g.W + cx[xi]];
    dd[k] = D[(size_t)ry[yi] * g.W + cx[xi]];  // kDWall on WALL su: no cell read
    oc[k] = ocls[(size_t)ry[yi] * g.opitch + cx[xi]];
  }
  if (pw) {
    // multi-su pedestrian: a move is admissible iff the su its rectangle
    // newly enters are free (walls included in the test)
    const int a = pw[p] >> 1, b = ph[p] >> 1;
#pragma unroll
    for (int k = 1; k < 9; ++k) oc[k] = strip_free(g, cell, occ, q.x, q.y, a, b, k) ? 0 : 1;
  }
  return (uint8_t)pick_move<false, TIE>(f, dd, oc, okx, oky, h, gl, beta, own, dirdot, nullptr,
                                       nullptr, tie);
}

// ------------------------------------------------------------------ S4 vote
// A mover wins iff no other registrant of its target (a pedestrian on one of
// the target's 8 neighbours whose choice points at it) has a smaller
// (priority, id).  Atomic-free: each mover reads the <= 8 competitors.  occ
// holds pedestrian indices; ped_off is the lattice's first index, so the
// priority is indexed by the pedestrian's number within its lattice, or by
// gid[p] when the caller numbered the pedestrians itself (a lattice that is
// one band of a larger one).  Returns the registrant count of the target (0
// for a stay).
__device__ __forceinline__ int vote_one(int p, int ped_off, const Geo& g,
                                        const int2* __restrict__ xy,
                                        const uint8_t* __restrict__ choice,
                                        const int32_t* __restrict__ occ, uint64_t seed,
                                        long long t, uint8_t* __restrict__ won,
                                        const int32_t* __restrict__ gid = nullptr) {
  const int k = choice[p];
  if (k == 0) {
    won[p] = 0;
    return 0;
  }
  const int2 q = xy[p];
  int tx, ty;
  wrap_coord(q.x + c_dx[k], g.W, g.px, tx);
  wrap_coord(q.y + c_dy[k], g.H, g.py, ty);
  const uint64_t st = splitmix_nth(seed, (uint64_t)t + 1);
  const long long idp = gid ? (long long)gid[p] : (long long)(p - ped_off);
  const uint64_t mine = splitmix_nth(st, (uint64_t)idp + 1);
  bool win = true;
  int regs = 1;
#pragma unroll
  for (int j = 1; j <= 8; ++j) {
    int nx, ny;
    if (!(wrap_coord(tx + move_dx(j), g.W, g.px, nx) & wrap_coord(ty + move_dy(j), g.H, g.py, ny)))
      continue;
    const int o = occ[(size_t)ny * g.W + nx];
    if (o < 0 || o == p) continue;
    if (choice[o] != c_opp[j]) continue;  // its move does not point at the target
    ++regs;
    const long long ido = gid ? (long long)gid[o] : (long long)(o - ped_off);
    const uint64_t po = splitmix_nth(st, (uint64_t)ido + 1);
    if (po < mine || (po == mine && ido < idp)) win = false;
  }
  won[p] = win ? 1 : 0;
  return regs;
}

// ---------------------------------------------------------------- S5 commit
// Winners move; occupancy and class grids follow; a winner on an EXIT su
// leaves.  No other pedestrian writes the same su: targets were empty at tick
// start and each has one winner.
__device__ __forceinline__ void commit_one(int p, const Geo& g, int2* __restrict__ xy,
                                           uint8_t* __restrict__ alive,
                                           uint8_t* __restrict__ heading,
                                           const uint8_t* __restrict__ choice,
                                           const uint8_t* __restrict__ won,
                                           const uint8_t* __restrict__ cell,
                                           int32_t* __restrict__ occ,
                                           uint8_t* __restrict__ ocls, bool& moved, bool& left) {
  moved = false;
  left = false;
  if (!won[p]) return;
  const int k = choice[p];
  const int2 q = xy[p];
  int tx, ty;
  wrap_coord(q.x + c_dx[k], g.W, g.px, tx);
  wrap_coord(q.y + c_dy[k], g.H, g.py, ty);
  const size_t c0 = (size_t)q.y * g.W + q.x, c1 = (size_t)ty * g.W + tx;
  occ[c0] = -1;
  ocls[(size_t)q.y * g.opitch + q.x] = 0;
  if (cell[c1] == kExit) {
    alive[p] = 0;
    left = true;
  } else {
    occ[c1] = p;
    ocls[(size_t)ty * g.opitch + tx] = (uint8_t)(1 + k);
  }
  xy[p] = make_int2(tx, ty);
  heading[p] = (uint8_t)k;
  moved = true;
}

// Vote of a multi-su pedestrian: it claims the su its rectangle newly
// enters and wins iff its (priority, id) is smaller than that of every other
// mover claiming one of them.  A rival claiming su s covers a su next to s,
// so the 8 neighbours of each claimed su hold every rival's id.  Returns the
// most claimants of one su.
__device__ __forceinline__ int vote_one_sized(int p, const Geo& g, const int2* __restrict__ xy,
                                              const uint8_t* __restrict__ choice,
                                              const int32_t* __restrict__ occ,
                                              const uint8_t* __restrict__ pw,
                                              const uint8_t* __restrict__ ph, uint64_t seed,
                                              long long t, uint8_t* __restrict__ won) {
  const int k = choice[p];
  if (k == 0) {
    won[p] = 0;
    return 0;
  }
  const int2 q = xy[p];
  const int a = pw[p] >> 1, b = ph[p] >> 1, dx = move_dx(k), dy = move_dy(k);
  const uint64_t st = splitmix_nth(seed, (uint64_t)t + 1);
  const uint64_t mine = splitmix_nth(st, (uint64_t)p + 1);
  bool win = true;
  int regs = 1;
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      const int ox = i + dx, oy = j + dy;
      if (ox >= -a && ox <= a && oy >= -b && oy <= b) continue;  // not newly entered
      int sx, sy;
      if (!(wrap_coord(q.x + ox, g.W, g.px, sx) & wrap_coord(q.y + oy, g.H, g.py, sy))) continue;
      int seen[8], ns = 0;
      for (int e = 1; e <= 8; ++e) {
        int nx, ny;
        if (!(wrap_coord(sx + move_dx(e), g.W, g.px, nx) & wrap_coord(sy + move_dy(e), g.H, g.py, ny)))
          continue;
        const int o = occ[(size_t)ny * g.W + nx];
        if (o < 0 || o == p) continue;
        bool dup = false;
        for (int u = 0; u < ns; ++u) dup |= seen[u] == o;
        if (dup || choice[o] == 0) continue;
        const int2 qo = xy[o];
        if (!in_entered(g, sx, sy, qo.x, qo.y, pw[o] >> 1, ph[o] >> 1, choice[o])) continue;
        seen[ns++] = o;
        const uint64_t po = splitmix_nth(st, (uint64_t)o + 1);
        if (po < mine || (po == mine && o < p)) win = false;
      }
      regs = max(regs, ns + 1);
    }
  won[p] = win ? 1 : 0;
  return regs;
}

// Commit of a multi-su pedestrian: the su it leaves behind are freed and the
// su it enters take its id (claims of winners are disjoint and were free, so
// no two threads write one su); a winner whose new rectangle meets an EXIT su
// leaves and frees its whole rectangle.
__device__ __forceinline__ void commit_one_sized(int p, const Geo& g, int2* __restrict__ xy,
                                                 uint8_t* __restrict__ alive,
                                                 uint8_t* __restrict__ heading,
                                                 const uint8_t* __restrict__ choice,
                                                 const uint8_t* __restrict__ won,
                                                 const uint8_t* __restrict__ cell,
                                                 int32_t* __restrict__ occ,
                                                 uint8_t* __restrict__ ocls,
                                                 const uint8_t* __restrict__ pw,
                                                 const uint8_t* __restrict__ ph, bool& moved,
                                                 bool& left) {
  moved = false;
  left = false;
  if (!won[p]) return;
  const int k = choice[p];
  const int2 q = xy[p];
  const int a = pw[p] >> 1, b = ph[p] >> 1, dx = move_dx(k), dy = move_dy(k);
  int tx, ty;
  wrap_coord(q.x + dx, g.W, g.px, tx);
  wrap_coord(q.y + dy, g.H, g.py, ty);
  bool out = false;
  for (int j = -b; j <= b && !out; ++j)
    for (int i = -a; i <= a && !out; ++i) {
      size_t s;
      if (rect_su(g, tx, ty, i, j, s) && cell[s] == kExit) out = true;
    }
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      size_t s;
      const int ni = i - dx, nj = j - dy;  // offset of this old su from the new centre
      const bool kept = ni >= -a && ni <= a && nj >= -b && nj <= b;
      if ((out || !kept) && rect_su(g, q.x, q.y, i, j, s)) occ[s] = -1;
      const int ei = i + dx, ej = j + dy;  // offset of a new su from the old centre
      const bool entered = !(ei >= -a && ei <= a && ej >= -b && ej <= b);
      if (!out && entered && rect_su(g, q.x, q.y, ei, ej, s)) occ[s] = p;
    }
  ocls[(size_t)q.y * g.opitch + q.x] = 0;
  if (out) {
    alive[p] = 0;
    left = true;
  } else {
    ocls[(size_t)ty * g.opitch + tx] = (uint8_t)(1 + k);
  }
  xy[p] = make_int2(tx, ty);
  heading[p] = (uint8_t)k;
  moved = true;
}

}  // namespace sfm
