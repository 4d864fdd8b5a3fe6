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
// 3 NE; x/y mirrors give W, S, NW, SW, SE
static __constant__ int c_ctab[9] = {0, 1, 3, 2, 3, 1, 3, 2, 3};
static __constant__ int c_csx[9] = {1, 1, 1, 1, -1, -1, -1, 1, 1};
static __constant__ int c_csy[9] = {1, 1, 1, 1, 1, 1, -1, -1, -1};

constexpr int kFieldPad = kFieldPadRows;

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

// -------------------------------------------------------------- S2 gather
// Number of (bin, image) entries overlapping [lo, hi] along one dimension.
__device__ __forceinline__ int halo_count(int lo, int hi, int n, int periodic) {
  if (!periodic) {
    lo = max(lo, 0);
    hi = min(hi, n - 1);
    return lo > hi ? 0 : hi / kBin - lo / kBin + 1;
  }
  const int k0 = floor_div(lo, n), k1 = floor_div(hi, n);
  int c = 0;
  for (int k = k0; k <= k1; ++k) {
    const int a = max(lo - k * n, 0), z = min(hi - k * n, n - 1);
    if (a <= z) c += z / kBin - a / kBin + 1;
  }
  return c;
}

// i-th entry of that list: bin index and offset of the bin origin (image
// coordinates) relative to t0.
__device__ __forceinline__ void halo_entry(int i, int lo, int hi, int n, int periodic, int t0,
                                           int& bin, int& off) {
  if (!periodic) {
    const int b = max(lo, 0) / kBin + i;
    bin = b;
    off = b * kBin - t0;
    return;
  }
  const int k0 = floor_div(lo, n), k1 = floor_div(hi, n);
  bin = 0;
  off = 0;
  for (int k = k0; k <= k1; ++k) {
    const int a = max(lo - k * n, 0), z = min(hi - k * n, n - 1);
    if (a > z) continue;
    const int c = z / kBin - a / kBin + 1;
    if (i < c) {
      const int b = a / kBin + i;
      bin = b;
      off = b * kBin + k * n - t0;
      return;
    }
    i -= c;
  }
}

// Walks the bins overlapping [x0-r, x0+FW-1+r] x [y0-r, y0+FH-1+r] in
// (bin row, bin column, row-major inside the bin) order -- the order of the
// terms summed into one su therefore does not depend on the footprint's
// shape -- and calls visit(item) for every record within reach of the
// footprint, after compacting the batch's records into the warp's scratch.
// item.x: table offset of the record for footprint column 0 / row 0;
// item.y: lane-column range llo | lhi << 5 | x mirror << 10 | y mirror << 11.
// acc[k] += (p[2k S], p[(2k + 1) S]), S = +-SP: one shared-memory read per
// row, one packed FP32 add per row pair (each half rounded as a scalar add).
template <int SP, int NP, bool NEG>
__device__ __forceinline__ void add_row_pairs(const float* __restrict__ p, float2 (&acc)[NP]) {
  constexpr int S = NEG ? -SP : SP;
#pragma unroll
  for (int k = 0; k < NP; ++k)
    acc[k] = __fadd2_rn(acc[k], make_float2(p[2 * k * S], p[(2 * k + 1) * S]));
}

// Visits, in bin-walk order (halo bins row-major, records in bin order), the
// records within reach (Chebyshev r) of some su of the FW x FH window at
// (x0, y0): a batch of 32 records is fetched lane-parallel, each lane turns
// its record (rx, ry relative to (x0, y0), heading class) into an item with
// make(), the items in reach are compacted into the warp's scratch scr (32
// int2) and visit() is called on each, in order, by the whole warp.
template <int FW, int FH, class Make, class Visit>
__device__ __forceinline__ void walk_records(const Geo& g, const int32_t* __restrict__ bin_start,
                                             const uint32_t* __restrict__ rec, int2* scr, int lane,
                                             int x0, int y0, Make make, Visit visit) {
  const int r = g.r;
  const unsigned lt = (1u << lane) - 1u;
  const int xlo = x0 - r, xhi = x0 + FW - 1 + r, ylo = y0 - r, yhi = y0 + FH - 1 + r;
  const int nxl = halo_count(xlo, xhi, g.W, g.px);
  const int ne = nxl * halo_count(ylo, yhi, g.H, g.py);
  for (int e0 = 0; e0 < ne; e0 += 32) {
    const int e = e0 + lane;
    int start = 0, cnt = 0, xoff = 0, yoff = 0;
    if (e < ne) {
      int bx, by;
      halo_entry(e % nxl, xlo, xhi, g.W, g.px, x0, bx, xoff);
      halo_entry(e / nxl, ylo, yhi, g.H, g.py, y0, by, yoff);
      const int id = by * g.nbx + bx;
      start = bin_start[id];
      cnt = bin_start[id + 1] - start;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    const int pre = inc - cnt;
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      // entry holding record q: the last lane whose prefix is <= q
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int p = __shfl_sync(0xffffffffu, pre, lo + step);
        if (p <= q) lo += step;
      }
      const int s_lo = __shfl_sync(0xffffffffu, start, lo);
      const int p_lo = __shfl_sync(0xffffffffu, pre, lo);
      const int xo = __shfl_sync(0xffffffffu, xoff, lo);
      const int yo = __shfl_sync(0xffffffffu, yoff, lo);
      bool keep = false;
      int2 item = make_int2(0, 0);
      if (q < total) {
        const uint32_t rc = rec[s_lo + (q - p_lo)];
        const int rx = xo + (int)(rc & 0xffu), ry = yo + (int)((rc >> 8) & 0xffu);
        const int cls = (int)((rc >> 16) & 0xfu);
        // some row of the footprint and some column within the window
        keep = ry >= -r && ry <= FH - 1 + r && rx >= -r && rx <= FW - 1 + r;
        if (keep) item = make(rx, ry, cls);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) scr[__popc(bal & lt)] = item;
      __syncwarp();
      const int m = __popc(bal);
      for (int j = 0; j < m; ++j) visit(scr[j]);
      __syncwarp();
    }
  }
}

// The footprint gather's walk: items carry the table offset of the
// pedestrian's class and position, its lane range and mirror flags.
template <int SP, int FW, int FH, class Visit>
__device__ __forceinline__ void walk_footprint(const Geo& g, const int32_t* __restrict__ bin_start,
                                               const uint32_t* __restrict__ rec, int TS, int2* scr,
                                               int lane, int x0, int y0, Visit visit) {
  const int r = g.r;
  walk_records<FW, FH>(g, bin_start, rec, scr, lane, x0, y0, [&](int rx, int ry, int cls) {
    const int sx = c_csx[cls], sy = c_csy[cls];
    const int llo = max(0, rx - r), lhi = min(FW - 1, rx + r);
    return make_int2(c_ctab[cls] * TS + (r + kFieldPad - sy * ry) * SP + r - sx * rx,
                     llo | (lhi << 5) | (sx < 0 ? 1024 : 0) | (sy < 0 ? 2048 : 0));
  }, visit);
}

// Adds the pedestrian field of the 16 x 16 footprint at (x0, y0): lane l owns
// column x0 + (l & 15) and rows y0 + 8 (l >> 4) + j, j < 8, row j in
// acc[j / 2] (.x even, .y odd).  One shared-memory read per (su, pedestrian)
// pair; the two half-warps read rows 8 SP apart, on disjoint banks as SP = 2
// (mod 4).  sT: the 4 heading-class tables (row stride SP, TS floats each,
// kFieldPad zero rows above and below the window, kTableGuard zero floats in
// front); scr: 32 int2 of per-warp scratch.  A kept pedestrian lies within r
// columns of the footprint, so with a wide stride every lane's column offset
// lies in [-15, 2r + 15]: out-of-reach lanes read zero columns (of its own
// row, or the row above, or the guard) and need no test.
template <int SP>
__device__ __forceinline__ void gather_footprint16(const Geo& g, const int32_t* __restrict__ bin_start,
                                                   const uint32_t* __restrict__ rec,
                                                   const float* __restrict__ sT, int TS, int2* scr,
                                                   int lane, int x0, int y0, float2 (&acc)[4]) {
  const int col = lane & 15, hoff = (lane >> 4) * 8 * SP;
  walk_footprint<SP, 16, 16>(g, bin_start, rec, TS, scr, lane, x0, y0, [&](const int2 it) {
    const int llo = it.y & 31, lhi = (it.y >> 5) & 31;
    if (SP != kNarrowStride || (col >= llo && col <= lhi)) {
      const float* p = sT + it.x + ((it.y & 1024) ? -col : col);
      if (it.y & 2048)
        add_row_pairs<SP, 4, true>(p - hoff, acc);
      else
        add_row_pairs<SP, 4, false>(p + hoff, acc);
    }
  });
}

// The 32 x 16 footprint: lane l owns column x0 + l and rows y0 + j, j < 16,
// row j in acc[j / 2]; column offsets lie in [-31, 2r + 31].
template <int SP>
__device__ __forceinline__ void gather_footprint32(const Geo& g, const int32_t* __restrict__ bin_start,
                                                   const uint32_t* __restrict__ rec,
                                                   const float* __restrict__ sT, int TS, int2* scr,
                                                   int lane, int x0, int y0, float2 (&acc)[8]) {
  walk_footprint<SP, 32, 16>(g, bin_start, rec, TS, scr, lane, x0, y0, [&](const int2 it) {
    const int llo = it.y & 31, lhi = (it.y >> 5) & 31;
    if (SP != kNarrowStride || (lane >= llo && lane <= lhi)) {
      const float* p = sT + it.x + ((it.y & 1024) ? -lane : lane);
      if (it.y & 2048)
        add_row_pairs<SP, 8, true>(p, acc);
      else
        add_row_pairs<SP, 8, false>(p, acc);
    }
  });
}

// The far part (see FarPart), split into a column part (per lane, once per
// footprint) and a row part (per row): bilinear weights between the centres
// of the coarse cells, indices wrapped or clamped.
struct FarAxis {
  int i0, i1;  // coarse indices of the two neighbouring centres
  float t;     // weight of i1
};
__device__ __forceinline__ FarAxis far_axis(int v, float inv_s, int n, int periodic) {
  const float f = (v + 0.5f) * inv_s - 0.5f;
  int a = (int)floorf(f);
  FarAxis ax;
  ax.t = f - a;
  int b = a + 1;
  if (periodic) {
    a = a < 0 ? a + n : (a >= n ? a - n : a);
    b = b < 0 ? b + n : (b >= n ? b - n : b);
  } else {
    a = min(max(a, 0), n - 1);
    b = min(max(b, 0), n - 1);
  }
  ax.i0 = a;
  ax.i1 = b;
  return ax;
}
__device__ __forceinline__ float far_value(const FarPart& fp, const FarAxis& ay, const FarAxis& ax) {
  const float* r0 = fp.Y + (size_t)ay.i0 * fp.Wc;
  const float* r1 = fp.Y + (size_t)ay.i1 * fp.Wc;
  const float v = (1.f - ay.t) * ((1.f - ax.t) * r0[ax.i0] + ax.t * r0[ax.i1]) +
                  ay.t * ((1.f - ax.t) * r1[ax.i0] + ax.t * r1[ax.i1]);
  return fp.scale * v;
}

// ---------------------------------------------------------------- S3 decide
// E over the 9 candidates (stay + 8 neighbours), admissible iff inside, not
// WALL and unoccupied at tick start; the minimum with ties to the smallest
// class.  F rows: lattice rows [y_lo, y_hi) at buffer row y - y_lo + main_off,
// lo_row at buffer row 0 and hi_row at hi_off.  own / dirdot: this lattice's
// 81-entry tables.
// Admissible candidates (stay, or inside, not WALL and unoccupied at tick
// start) and the energy E(k) = F(c_k) - K_P(own heading) + guidance; the
// minimum with ties to the smallest class.  With MARGIN, *margin receives
// E(second best) - E(best) over the admissible candidates (+inf when only
// staying is admissible) and *emag (optional) the larger |E| of the two:
// any field error below margin / 2 at every candidate, less FP32 rounding of
// energies of that size, leaves the choice unchanged.
template <bool MARGIN>
__device__ __forceinline__ int pick_move(const float (&f)[9], const int32_t (&dd)[9],
                                         const uint8_t (&cl)[9], const uint8_t (&oc)[9],
                                         const bool (&okx)[3], const bool (&oky)[3], int h, int gl,
                                         float beta, const float* __restrict__ own,
                                         const float* __restrict__ dirdot, float* margin,
                                         float* emag = nullptr) {
  int best = 0;
  float bestE = 0.f, second = __int_as_float(0x7f800000);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    const bool adm = (k == 0) || (okx[xi] && oky[yi] && cl[k] != kWall && oc[k] == 0);
    const float guide = (gl == 0) ? beta * ((float)(dd[k] - dd[0]) / 5.0f) : -beta * dirdot[gl * 9 + k];
    const float e = f[k] - own[h * 9 + k] + guide;
    if (adm && (k == 0 || e < bestE)) {
      if (MARGIN && k != 0) second = bestE;
      best = k;
      bestE = e;
    } else if (MARGIN && adm && e < second) {
      second = e;
    }
  }
  if (MARGIN) {
    *margin = second - bestE;
    // size of the energies compared, for a rounding allowance
    if (emag) *emag = fmaxf(fabsf(bestE), second < __int_as_float(0x7f800000) ? fabsf(second) : 0.f);
  }
  return best;
}

// The 3 x 3 neighbourhood of pedestrian p: wrapped or clipped coordinates
// (an out-of-lattice candidate repeats p's own row or column and is marked
// inadmissible by okx / oky), and the guidance, cell and occupancy of each
// candidate.
__device__ __forceinline__ void candidate_cells(int2 q, const Geo& g, const uint8_t* __restrict__ cell,
                                                const uint8_t* __restrict__ ocls,
                                                const int32_t* __restrict__ D, int (&cx)[3],
                                                int (&ry)[3], bool (&okx)[3], bool (&oky)[3],
                                                int32_t (&dd)[9], uint8_t (&cl)[9],
                                                uint8_t (&oc)[9]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    okx[d] = wrap_coord(q.x + d - 1, g.W, g.px, cx[d]);
    oky[d] = wrap_coord(q.y + d - 1, g.H, g.py, ry[d]);
    if (!okx[d]) cx[d] = q.x;
    if (!oky[d]) ry[d] = q.y;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    const size_t c = (size_t)ry[yi] * g.W + cx[xi];
    dd[k] = D[c];
    cl[k] = cell[c];
    oc[k] = ocls[(size_t)ry[yi] * g.opitch + cx[xi]];
  }
}

__device__ __forceinline__ uint8_t decide_one(
    int p, const Geo& g, const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
    const uint8_t* __restrict__ goal, const uint8_t* __restrict__ cell,
    const uint8_t* __restrict__ ocls, const int32_t* __restrict__ D, const float* __restrict__ F,
    int main_off, int lo_row, int hi_row, int hi_off, int y_lo, int y_hi, float beta,
    const float* __restrict__ own, const float* __restrict__ dirdot) {
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
  }
  float f[9];
  int32_t dd[9];
  uint8_t cl[9], oc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    const size_t c = (size_t)ry[yi] * g.W + cx[xi];
    f[k] = F[(size_t)fr[yi] * g.W + cx[xi]];
    dd[k] = D[c];
    cl[k] = cell[c];
    oc[k] = ocls[(size_t)ry[yi] * g.opitch + cx[xi]];
  }
  return (uint8_t)pick_move<false>(f, dd, cl, oc, okx, oky, h, gl, beta, own, dirdot, nullptr);
}

// ------------------------------------------------------------------ S4 vote
// A mover wins iff no other registrant of its target (a pedestrian on one of
// the target's 8 neighbours whose choice points at it) has a smaller
// (priority, id).  Atomic-free: each mover reads the <= 8 competitors.  occ
// holds pedestrian indices; ped_off is the lattice's first index, so the
// priority is indexed by the pedestrian's number within its lattice.
// Returns the registrant count of the target (0 for a stay).
__device__ __forceinline__ int vote_one(int p, int ped_off, const Geo& g,
                                        const int2* __restrict__ xy,
                                        const uint8_t* __restrict__ choice,
                                        const int32_t* __restrict__ occ, uint64_t seed,
                                        long long t, uint8_t* __restrict__ won) {
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
  const uint64_t mine = splitmix_nth(st, (uint64_t)(p - ped_off) + 1);
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
    const uint64_t po = splitmix_nth(st, (uint64_t)(o - ped_off) + 1);
    if (po < mine || (po == mine && o < p)) win = false;
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

}  // namespace sfm
