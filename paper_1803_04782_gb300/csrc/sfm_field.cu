// sfm_field.cu -- the class-table field gather (S2, radius <= 50): the
// per-su superposition of the pedestrian field of one tick, F = F_static +
// sum of K_P over pedestrians in reach (k-5 of the paper's Alg. 1, Sec. 3.1),
// as a gather over binned pedestrians instead of the paper's fan-out scatter.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfm_gather.cuh"
#include "sfm_internal.h"

namespace sfm {

// ---------------------------------------------- S2 (v2): persistent warps
// One CTA of 32 warps per SM loads the 4 heading-class tables into shared
// memory once per launch; each warp then takes footprints of 32 x 16 su
// (SHAPE 1: lane = column, 16 rows) or 16 x 16 su (SHAPE 0: half-warp = 8
// rows) in turn.  For a footprint it walks the bins overlapping the r-halo
// in batches of 32 records (coalesced, L1-shared by the neighbouring
// footprints other warps of the SM work on), compacts the records in reach
// with their table offsets into a per-warp scratch, and adds for each one
// table word per (su, pedestrian) pair: the heading of a pedestrian is one of
// 9 classes and the kernel of every class is stored precomputed (4 tables,
// the other 5 by x/y mirroring).  Zero rows above and below each window and,
// for wide strides, zero columns after each row let every lane read without
// a range test, and the compile-time row stride SP turns the 16 reads into
// immediate offsets.  F = Fs + sum (+ the far part when FAR) is written once.

// Store of a 32 x 16 footprint column with the surrogate's far part: F =
// Fs + near sum + scale * bilinear(Y).  The 16 rows of a footprint need the
// coarse rows a(y0) .. a(y0 + 15) + 1; when these are at most 4 (coarsening
// >= 8), each lane blends its two coarse columns once per coarse row (8
// independent loads) and every row interpolates between two of those; else
// the far part is evaluated row by row.
template <int NJ, int S>
__device__ __forceinline__ void far_epilogue(const Geo& g, const FarPart& far, const FarAxis& fax,
                                             const float* __restrict__ Fs, float* __restrict__ out,
                                             int out_row0, int store_lo, int store_hi, int xx,
                                             int y0, const float2 (&acc)[NJ / 2]) {
  const float is = far.inv_s;
  const int a0 = (int)floorf((y0 + 0.5f) * is - 0.5f);
  const int a1 = (int)floorf((y0 + NJ - 1 + 0.5f) * is - 0.5f);
  const bool col = xx < g.W;  // fax is only valid for columns inside the lattice
  float v[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int y = y0 + j;
    v[j] = (col && y < g.H) ? Fs[(size_t)y * g.W + xx] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x)
                            : 0.f;
  }
  if constexpr (S == 8 && NJ == 16) {
    // coarsening 8, rows y0 .. y0 + 15 with y0 a multiple of 16: row j lies
    // at (y0 + j + 0.5) / 8 - 0.5 = y0 / 8 + (j - 3.5) / 8, so its coarse rows
    // are a0 + m_j, a0 + m_j + 1 (a0 = y0 / 8 - 1, m_j = 0, 1, 2 for j < 4,
    // < 12, < 16) with weight t_j = (j + 4.5) / 8 - m_j of the second: the
    // values the general formula gives, exactly (all are multiples of 1/16)
    float h[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int k = y0 / 8 - 1 + m;
      if (g.py) {
        k %= far.Hc;
        if (k < 0) k += far.Hc;
      } else {
        k = min(max(k, 0), far.Hc - 1);
      }
      const float* row = far.Y + (size_t)k * far.Wc;
      h[m] = col ? (1.f - fax.t) * row[fax.i0] + fax.t * row[fax.i1] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int m = j < 4 ? 0 : (j < 12 ? 1 : 2);
      const float t = (j + 4.5f) * 0.125f - (float)m;
      v[j] += far.scale * ((1.f - t) * h[m] + t * h[m + 1]);
    }
  } else if (a1 - a0 <= 2) {
    float h[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      // coarse row a0 + m, wrapped (periodic) or clamped as far_axis does
      int k = a0 + m;
      if (g.py) {
        k %= far.Hc;
        if (k < 0) k += far.Hc;
      } else {
        k = min(max(k, 0), far.Hc - 1);
      }
      const float* row = far.Y + (size_t)k * far.Wc;
      h[m] = col ? (1.f - fax.t) * row[fax.i0] + fax.t * row[fax.i1] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float f = (y0 + j + 0.5f) * is - 0.5f;
      const float a = floorf(f), t = f - a;
      const int m = (int)a - a0;
      const float h0 = m == 0 ? h[0] : (m == 1 ? h[1] : h[2]);
      const float h1 = m == 0 ? h[1] : (m == 1 ? h[2] : h[3]);
      v[j] += far.scale * ((1.f - t) * h0 + t * h1);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NJ; ++j)
      if (col && y0 + j < g.H) v[j] += far_value(far, far_axis(y0 + j, is, far.Hc, g.py), fax);
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int y = y0 + j;
    if (xx < g.W && y < g.H && y >= store_lo && y < store_hi) out[(size_t)(y - out_row0) * g.W + xx] = v[j];
  }
}

template <int SP, int SHAPE, int FAR>
__global__ void __launch_bounds__(kV2Threads, 1)
    k_field_v2(Geo g, const int32_t* __restrict__ bin_start, const uint32_t* __restrict__ rec,
               const float* __restrict__ CT, const float* __restrict__ Fs,
               float* __restrict__ out, int out_row0, int fy0, int fy1, int store_lo,
               int store_hi, FarPart far, unsigned int* __restrict__ tickets) {
  extern __shared__ __align__(16) float sm[];
  constexpr int FW = SHAPE ? 32 : 16, FH = 16, NJ = SHAPE ? 16 : 8;
  const int r = g.r;
  const int TR = 2 * r + 1 + 2 * kFieldPad, TS = TR * SP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sT = sm + kTableGuard;
  // per-warp scratch: the batch's pedestrians in reach of the footprint
  int2* scr = reinterpret_cast<int2*>(sT + 4 * TS) + warp * 32;
  {
    const float2* src = reinterpret_cast<const float2*>(CT);
    float2* dst = reinterpret_cast<float2*>(sT);
    copy_to_shared<12>(dst, src, 2 * TS);  // 4*TS floats
    if (threadIdx.x < kTableGuard) sm[threadIdx.x] = 0.f;
  }
  __syncthreads();
  const int wpb = blockDim.x >> 5;
  const int tw = gridDim.x * wpb;
  const int nfx = (g.W + FW - 1) / FW;
  const int nf = nfx * (fy1 - fy0);
  // this lane's column and first row inside a footprint
  const int x = SHAPE ? lane : (lane & 15), yl = SHAPE ? 0 : (lane >> 4) * 8;
  // Schedule.  The first footprints go out in rounds of tw, one per warp: a
  // round of a large lattice gives each CTA a run of wpb consecutive
  // footprints (its warps share records through L1); a partial round, or
  // every round of a lattice under 4 footprints per warp of the whole grid,
  // deals footprint base + i to CTA i % gridDim.x, so it spreads over every
  // SM.  With a ticket counter only whole rounds covering about 4/5 of the
  // footprints are dealt so; a warp then takes the rest one at a time, in
  // the order of tickets it draws, so SMs whose share of the crowd was light
  // do more of them and all finish together.  Either way each footprint is
  // computed once, by one warp.
  const bool spread_all = nf < 4 * tw;
  const int nstat = tickets ? (int)((4LL * nf / 5) / tw) * tw : nf;
  auto footprint = [&](int base) {
    return spread_all || nf - base < tw ? base + blockIdx.x + gridDim.x * warp
                                        : base + blockIdx.x * wpb + warp;
  };
  // with the far part (little gather work per footprint) the static-field
  // lines of a footprint (one per row) are fetched into L2 before its
  // gather, so the store's reads of Fs do not wait on HBM
  auto prefetch_fs = [&](int f) {
    if (FAR && f < nf && lane < FH) {
      const int px0 = (f % nfx) * FW, py = (fy0 + f / nfx) * FH + lane;
      if (py < g.H) asm volatile("prefetch.global.L2 [%0];" ::"l"(Fs + (size_t)py * g.W + px0));
    }
  };
  auto visit = [&](int f) {
    const int x0 = (f % nfx) * FW, y0 = (fy0 + f / nfx) * FH;
    FarAxis fax{};
    if constexpr (FAR) fax = far_axis(x0 + x, far.inv_s, far.Wc, g.px);
    float2 acc[NJ / 2];
#pragma unroll
    for (int j = 0; j < NJ / 2; ++j) acc[j] = make_float2(0.f, 0.f);
    if constexpr (SHAPE)
      gather_footprint32<SP>(g, bin_start, rec, sT, TS, scr, lane, x0, y0, acc);
    else
      gather_footprint16<SP>(g, bin_start, rec, sT, TS, scr, lane, x0, y0, acc);
    if constexpr (FAR) {
      far_epilogue<NJ, FAR>(g, far, fax, Fs, out, out_row0, store_lo, store_hi, x0 + x, y0, acc);
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int y = y0 + yl + j, xx = x0 + x;
        if (xx < g.W && y < g.H && y >= store_lo && y < store_hi) {
          const size_t c = (size_t)y * g.W + xx;
          out[(size_t)(y - out_row0) * g.W + xx] = Fs[c] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
        }
      }
    }
  };
  // one loop over both parts, so the footprint's code is inlined once; lane
  // 0 draws a warp's next ticket while the warp works on the current one
  unsigned int t = 0;
  int base = 0, f;
  if (nstat > 0) {
    f = footprint(0);
  } else {
    if (lane == 0) t = atomicAdd(tickets, 1u);
    f = nstat + (int)__shfl_sync(0xffffffffu, t, 0);
  }
  prefetch_fs(f);
  while (f < nf) {  // f >= nf: a partial round had none left, or the tickets ran out
    int fn = nf;
    if (base + tw < nstat) {
      base += tw;
      fn = footprint(base);
    } else if (tickets) {
      if (lane == 0) t = atomicAdd(tickets, 1u);
      fn = -1;
    }
    if (fn >= 0) prefetch_fs(fn);
    visit(f);
    f = fn >= 0 ? fn : nstat + (int)__shfl_sync(0xffffffffu, t, 0);
    if (fn < 0) prefetch_fs(f);
  }
  if (!tickets) return;
  // the last CTA out puts the counter back to zero for the next launch:
  // every warp of every CTA has drawn its final ticket before its CTA counts
  // itself done
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(tickets + 1, 1u) == gridDim.x - 1) {
      atomicExch(tickets, 0u);
      atomicExch(tickets + 1, 0u);
    }
  }
}

static int g_num_sms = 0;

template <int SP, int SHAPE, int FAR>
static void launch_v2(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const float* CT,
                      const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                      cudaStream_t s, const FarPart& far, unsigned int* tickets) {
  constexpr int FW = SHAPE ? 32 : 16, FH = 16;
  const size_t smem = (kTableGuard + class_table_floats(g.r)) * sizeof(float) +
                      kV2Threads / 32 * 32 * sizeof(int2);
  cudaFuncSetAttribute(k_field_v2<SP, SHAPE, FAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  const int fy0 = store_lo / FH, fy1 = (store_hi + FH - 1) / FH;
  const int nf = ((g.W + FW - 1) / FW) * (fy1 - fy0);
  const int wpb = kV2Threads / 32;
  // under 4 footprints per warp of a full grid the kernel spreads single
  // footprints over the CTAs, so a full grid (one CTA per SM) has work
  int blocks = nf < 4 * wpb * g_num_sms ? nf : (nf + wpb - 1) / wpb;
  if (blocks > g_num_sms) blocks = g_num_sms;
  if (blocks < 1) blocks = 1;
  // tickets only where there are whole rounds to rebalance (4 footprints per
  // warp or more); a small lattice keeps the static deal, without the
  // counter's atomics at the start and end of the launch
  if (nf < 4 * wpb * blocks) tickets = nullptr;
  k_field_v2<SP, SHAPE, FAR><<<blocks, kV2Threads, smem, s>>>(g, bin_start, rec, CT, Fs, out, out_row0,
                                                         fy0, fy1, store_lo, store_hi, far,
                                                         tickets);
}

template <int SP>
static void launch_v2_shape(const Geo& g, const int32_t* bin_start, const uint32_t* rec,
                            const Tables& tb, const float* Fs, float* out, int out_row0,
                            int store_lo, int store_hi, cudaStream_t s, const FarPart& far,
                            unsigned int* tickets) {
  // the far part (surrogate) has its own instantiations, 32 x 16 footprint
  // only (one for coarsening 8, one for any), so the exact gather carries no
  // code for it
  if (far.Y && far.s == 8)
    launch_v2<SP, 1, 8>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far, tickets);
  else if (far.Y)
    launch_v2<SP, 1, 1>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far, tickets);
  else if (tb.shape != kShape16x16)  // the row-trimmed shape where that gather is off
    launch_v2<SP, 1, 0>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far, tickets);
  else
    launch_v2<SP, 0, 0>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far, tickets);
}

void launch_field(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const Tables& tb,
                  const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                  Counters* ctr, cudaStream_t s, const FarPart& far, int ring) {
  if (store_hi <= store_lo) return;
  const int sp = tb.CT ? class_table_stride(g.r) : 0;
  if (!sp) {
    launch_field_v1(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, ctr, s);
    return;
  }
  // the context's footprint ticket counter (no counter: a static schedule).
  // The far-part gather keeps the static one: its footprints cost about the
  // same everywhere (a 7 x 7 window and the epilogue), and they are so short
  // that one ticket each would queue on the counter.  So do lattices under 4
  // footprints per warp (launch_v2).
  unsigned int* tickets = ctr && !far.Y ? ctr->field_tickets : nullptr;
  if (!far.Y && launch_field_v3(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi,
                                tickets, s, ring))
    return;
  if (ring) return;  // the caller checked that the row-trimmed gather is in use
  switch (sp) {
    case 34: launch_v2_shape<34>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    case 50: launch_v2_shape<50>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    case 66: launch_v2_shape<66>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    case 82: launch_v2_shape<82>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    case 98: launch_v2_shape<98>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    case 114: launch_v2_shape<114>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
    default: launch_v2_shape<kNarrowStride>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far, tickets); break;
  }
}

}  // namespace sfm
