// sfm_gather.cuh -- device building blocks of the field gather (S2): the
// halo-bin lists, the record walk of a warp footprint, the class-table reads
// of the 16 x 16 and 32 x 16 footprints and the surrogate's far part.  Shared
// by the single-lattice gather (sfm_field.cu), the batched tick (sfm_batch.cu)
// and the surrogate's exact fallback (sfm_surrogate.cu).
#pragma once
#include "sfm_device.cuh"

namespace sfm {

// -------------------------------------------------------------- S2 gather
// n elements global -> shared by the CTA's threads, B loads a thread in
// flight before their stores: a plain strided loop waits out one load's
// latency per element it copies (about 4.5 us for the 170 KB tables of the
// r = 40 gather, against one latency here).
template <int B, class T>
__device__ __forceinline__ void copy_to_shared(T* __restrict__ dst, const T* __restrict__ src,
                                               int n) {
  for (int i0 = threadIdx.x; i0 < n; i0 += B * blockDim.x) {
    T v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int i = i0 + k * blockDim.x;
      if (i < n) v[k] = __ldg(src + i);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int i = i0 + k * blockDim.x;
      if (i < n) dst[i] = v[k];
    }
  }
}

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
// The window's extent FW x FH is a run-time value here (walk_records below
// fixes it at compile time for the footprints).
template <class Make, class Visit>
__device__ __forceinline__ void walk_records_box(const Geo& g, const int32_t* __restrict__ bin_start,
                                                 const uint32_t* __restrict__ rec, int2* scr, int lane,
                                                 int x0, int y0, int FW, int FH, Make make, Visit visit) {
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
      // two items per shared-memory read (one broadcast of 16 bytes; scr is
      // 16-byte aligned and j even)
      const int m = __popc(bal);
      int j = 0;
      for (; j + 1 < m; j += 2) {
        const int4 two = *reinterpret_cast<const int4*>(scr + j);
        visit(make_int2(two.x, two.y));
        visit(make_int2(two.z, two.w));
      }
      if (j < m) visit(scr[j]);
      __syncwarp();
    }
  }
}

template <int FW, int FH, class Make, class Visit>
__device__ __forceinline__ void walk_records(const Geo& g, const int32_t* __restrict__ bin_start,
                                             const uint32_t* __restrict__ rec, int2* scr, int lane,
                                             int x0, int y0, Make make, Visit visit) {
  walk_records_box(g, bin_start, rec, scr, lane, x0, y0, FW, FH, make, visit);
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

}  // namespace sfm
