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

template <int SP, int SHAPE, bool FAR>
__global__ void __launch_bounds__(kV2Threads, 1)
    k_field_v2(Geo g, const int32_t* __restrict__ bin_start, const uint32_t* __restrict__ rec,
               const float* __restrict__ CT, const float* __restrict__ Fs,
               float* __restrict__ out, int out_row0, int fy0, int fy1, int store_lo,
               int store_hi, FarPart far) {
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
    for (int i = threadIdx.x; i < 2 * TS; i += blockDim.x) dst[i] = src[i];  // 4*TS floats
    if (threadIdx.x < kTableGuard) sm[threadIdx.x] = 0.f;
  }
  __syncthreads();
  const int wpb = blockDim.x >> 5;
  const int tw = gridDim.x * wpb;
  const int nfx = (g.W + FW - 1) / FW;
  const int nf = nfx * (fy1 - fy0);
  // this lane's column and first row inside a footprint
  const int x = SHAPE ? lane : (lane & 15), yl = SHAPE ? 0 : (lane >> 4) * 8;
  // large lattices: each CTA takes runs of wpb consecutive footprints (its
  // warps share records through L1); small ones (under 4 footprints per warp
  // of the whole grid): footprint f goes to CTA f % gridDim.x, so every SM
  // gets work.  Either way each footprint is computed once, by one warp.
  // (both walk footprints with the stride of all warps, tw)
  const int f0 = nf < 4 * tw ? blockIdx.x + gridDim.x * warp : blockIdx.x * wpb + warp;
  for (int f = f0; f < nf; f += tw) {
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
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int y = y0 + yl + j, xx = x0 + x;
      if (xx < g.W && y < g.H && y >= store_lo && y < store_hi) {
        const size_t c = (size_t)y * g.W + xx;
        float v = Fs[c] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
        if constexpr (FAR) v += far_value(far, far_axis(y, far.inv_s, far.Hc, g.py), fax);
        out[(size_t)(y - out_row0) * g.W + xx] = v;
      }
    }
  }
}

static int g_num_sms = 0;

template <int SP, int SHAPE, bool FAR>
static void launch_v2(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const float* CT,
                      const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                      cudaStream_t s, const FarPart& far) {
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
  k_field_v2<SP, SHAPE, FAR><<<blocks, kV2Threads, smem, s>>>(g, bin_start, rec, CT, Fs, out, out_row0,
                                                         fy0, fy1, store_lo, store_hi, far);
}

template <int SP>
static void launch_v2_shape(const Geo& g, const int32_t* bin_start, const uint32_t* rec,
                            const Tables& tb, const float* Fs, float* out, int out_row0,
                            int store_lo, int store_hi, cudaStream_t s, const FarPart& far) {
  // the far part (surrogate) has its own instantiation, 32 x 16 footprint only,
  // so the exact gather carries no code for it
  if (far.Y)
    launch_v2<SP, 1, true>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far);
  else if (tb.shape)
    launch_v2<SP, 1, false>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far);
  else
    launch_v2<SP, 0, false>(g, bin_start, rec, tb.CT, Fs, out, out_row0, store_lo, store_hi, s, far);
}

void launch_field(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const Tables& tb,
                  const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
                  Counters* ctr, cudaStream_t s, const FarPart& far) {
  if (store_hi <= store_lo) return;
  const int sp = tb.CT ? class_table_stride(g.r) : 0;
  if (!sp) {
    launch_field_v1(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, ctr, s);
    return;
  }
  switch (sp) {
    case 34: launch_v2_shape<34>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    case 50: launch_v2_shape<50>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    case 66: launch_v2_shape<66>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    case 82: launch_v2_shape<82>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    case 98: launch_v2_shape<98>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    case 114: launch_v2_shape<114>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
    default: launch_v2_shape<kNarrowStride>(g, bin_start, rec, tb, Fs, out, out_row0, store_lo, store_hi, s, far); break;
  }
}

}  // namespace sfm
