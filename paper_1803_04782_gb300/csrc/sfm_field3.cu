// sfm_field3.cu -- the row-trimmed class-table field gather (S2, radius 1
// .. 40): the per-su superposition of the pedestrian field of one tick, F =
// F_static + sum of K_P over the pedestrians in reach (k-5 of the paper's
// Alg. 1, Sec. 3.1), gathered over binned pedestrians.
//
// A warp owns a footprint of 32 x 32 su (lane = column), in blocks of 8
// rows.  A pedestrian visit reads only the blocks its window reaches: each
// block is eight shared-memory reads and four packed FP32 adds per lane,
// behind one test that is uniform over the warp.  The 16-row gathers of
// sfm_field.cu read all 16 rows of every visit, the zero rows above and
// below a window included; the 32 x 32 footprint also visits each pedestrian
// about 40 % fewer times per su than a 32 x 16 one at r = 40.  The tables
// carry 7 zero rows above and below each window (a block may start 7 rows
// before the reach) and at least 31 zero columns after each row (a lane left
// or right of the window reads a zero of its own row or of the row before),
// so no lane needs a range test.  Each su adds its terms in the record-walk
// order of the other gathers, so the field is the same bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfm_gather.cuh"
#include "sfm_internal.h"

namespace sfm {

namespace {

// Rows per block of the visit: a visit reads the blocks its window reaches.
constexpr int kBlockRows = 8;

// Block G of a lane: footprint rows BR G .. BR G + BR - 1 (acc[BR G / 2] ..,
// .x even rows, .y odd) at table offsets (BR G + j) S from the lane's row-0
// address p, S = +-SP the signed row stride: BR reads and BR / 2 packed
// adds, done only when the block is in reach (`on`, uniform over the warp).
template <int S, int G, int NG>
__device__ __forceinline__ void add_block(const float* __restrict__ p, uint32_t on, float2 (&acc)[NG]) {
  constexpr int BR = kBlockRows;
  if (on) {
#pragma unroll
    for (int j = 0; j < BR / 2; ++j)
      acc[BR / 2 * G + j] = __fadd2_rn(acc[BR / 2 * G + j],
                                       make_float2(p[(BR * G + 2 * j) * S], p[(BR * G + 2 * j + 1) * S]));
  }
}

// the blocks of a visit; bit b of `mask` says whether block b is in reach
template <int S, int NB, int NG, int G = 0>
__device__ __forceinline__ void add_blocks(const float* __restrict__ p, uint32_t mask, float2 (&acc)[NG]) {
  add_block<S, G, NG>(p, mask & (1u << G), acc);
  if constexpr (G + 1 < NB) add_blocks<S, NB, NG, G + 1>(p, mask, acc);
}

template <int SP, int FH>
__global__ void __launch_bounds__(kV2Threads, 1)
    k_field_v3(Geo g, const int32_t* __restrict__ bin_start, const uint32_t* __restrict__ rec,
               const float* __restrict__ CT3, const float* __restrict__ Fs,
               float* __restrict__ out, int out_row0, int fy0, int fy1, int store_lo,
               int store_hi, unsigned int* __restrict__ tickets, int ring) {
  static_assert(FH % kBlockRows == 0 && FH / kBlockRows <= 16, "footprint height: whole blocks, at most 16");
  // launched only for radii whose row stride class SP >= 2r + 32 (launch_field_v3)
  extern __shared__ __align__(16) float sm[];
  constexpr int FW = 32, NB = FH / kBlockRows, NG = FH / 2;  // NG: float2 accumulators a lane
  const int r = g.r;
  const int TS = (2 * r + 1 + 2 * kField3PadRows) * SP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sT = sm + kTableGuard;
  int2* scr = reinterpret_cast<int2*>(sT + 4 * TS) + warp * 32;
  {
    const float4* src = reinterpret_cast<const float4*>(CT3);
    float4* dst = reinterpret_cast<float4*>(sT);
    copy_to_shared<8>(dst, src, TS);  // 4 * TS floats
    if (threadIdx.x < kTableGuard) sm[threadIdx.x] = 0.f;
  }
  __syncthreads();
  const int wpb = blockDim.x >> 5;
  const int tw = gridDim.x * wpb;
  const int nfx = (g.W + FW - 1) / FW;
  const int nf = nfx * (fy1 - fy0);
  // the schedule of the 16-row gathers: whole rounds of one footprint per
  // warp (a CTA's warps on consecutive footprints), then tickets; here the
  // rounds deal about half the footprints, not 4/5: once a crowd gathers
  // into clusters, the dealt share of some warps costs far more than that of
  // others, and the tickets must cover the difference (on the 16384^2 floor
  // after 800 ticks: 2.12 ms a tick against 2.28 with 4/5 dealt; the same
  // at the start)
  const bool spread_all = nf < 4 * tw;
  const int nstat = tickets ? (int)((nf / 2) / tw) * tw : nf;
  auto footprint = [&](int base) {
    return spread_all || nf - base < tw ? base + blockIdx.x + gridDim.x * warp
                                        : base + blockIdx.x * wpb + warp;
  };
  auto visit = [&](int f) {
    const int x0 = (f % nfx) * FW, y0 = (fy0 + f / nfx) * FH;
    float2 acc[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) acc[j] = make_float2(0.f, 0.f);
    walk_records_box(
        g, bin_start, rec, scr, lane, x0, y0, FW, FH,
        [&](int rx, int ry, int cls) {
          const int sx = class_sx(cls), sy = class_sy(cls);
          // blocks b0 .. b1 hold the rows in reach
          const int b0 = max(0, ry - r) / kBlockRows, b1 = min(FH - 1, ry + r) / kBlockRows;
          const int mask = (2 << b1) - (1 << b0);
          return make_int2(class_table(cls) * TS + (kField3PadRows + r - sy * ry) * SP + r - sx * rx,
                           mask | (sx < 0 ? 0x10000 : 0) | (sy < 0 ? 0x20000 : 0));
        },
        [&](const int2 it) {
          // the item is the same in every lane; its OR over the warp is a
          // value the compiler knows to be warp-uniform, so the block and
          // mirror tests below are uniform branches
          const uint32_t u = __reduce_or_sync(0xffffffffu, (uint32_t)it.y);
          const float* p = sT + it.x + ((u & 0x10000) ? -lane : lane);
          if (u & 0x20000)
            add_blocks<-SP, NB, NG>(p, u, acc);
          else
            add_blocks<SP, NB, NG>(p, u, acc);
        });
    const int xx = x0 + lane;
#pragma unroll
    for (int j = 0; j < FH; ++j) {
      const int y = y0 + j;
      if (xx < g.W && y < g.H && y >= store_lo && y < store_hi) {
        int row = y - out_row0;
        if (ring && row >= ring) row -= ring;
        out[(size_t)row * g.W + xx] =
            Fs[(size_t)y * g.W + xx] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
      }
    }
  };
  unsigned int t = 0;
  int base = 0, f;
  if (nstat > 0) {
    f = footprint(0);
  } else {
    if (lane == 0) t = atomicAdd(tickets, 1u);
    f = nstat + (int)__shfl_sync(0xffffffffu, t, 0);
  }
  while (f < nf) {
    int fn = nf;
    if (base + tw < nstat) {
      base += tw;
      fn = footprint(base);
    } else if (tickets) {
      if (lane == 0) t = atomicAdd(tickets, 1u);
      fn = -1;
    }
    visit(f);
    f = fn >= 0 ? fn : nstat + (int)__shfl_sync(0xffffffffu, t, 0);
  }
  if (!tickets) return;
  // the last CTA out puts the counter back to zero for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(tickets + 1, 1u) == gridDim.x - 1) {
      atomicExch(tickets, 0u);
      atomicExch(tickets + 1, 0u);
    }
  }
}

template <int SP, int FH>
void launch_v3(const Geo& g, const int32_t* bin_start, const uint32_t* rec, const float* CT3,
               const float* Fs, float* out, int out_row0, int store_lo, int store_hi,
               cudaStream_t s, unsigned int* tickets, int ring) {
  constexpr int FW = 32;
  const size_t smem = (kTableGuard + field3_table_floats(g.r)) * sizeof(float) +
                      kV2Threads / 32 * 32 * sizeof(int2);
  cudaFuncSetAttribute(k_field_v3<SP, FH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nsm = device_sm_count();
  const int fy0 = store_lo / FH, fy1 = (store_hi + FH - 1) / FH;
  const int nf = ((g.W + FW - 1) / FW) * (fy1 - fy0);
  const int wpb = kV2Threads / 32;
  // under 4 footprints per warp of a full grid single footprints are spread
  // over the CTAs; tickets only where whole rounds are left to rebalance
  int blocks = nf < 4 * wpb * nsm ? nf : (nf + wpb - 1) / wpb;
  if (blocks > nsm) blocks = nsm;
  if (blocks < 1) blocks = 1;
  if (nf < 4 * wpb * blocks) tickets = nullptr;
  k_field_v3<SP, FH><<<blocks, kV2Threads, smem, s>>>(g, bin_start, rec, CT3, Fs, out, out_row0,
                                                      fy0, fy1, store_lo, store_hi, tickets, ring);
}

// the class tables in the layout of the row-trimmed gather: [4][2r+3][SP],
// window row dy at table row dy + r + 1, column dx at dx + r
__global__ void k_class_tables3(int r, int SP, double kP, double aP, double gamma,
                                float* __restrict__ T) {
  const int TR = 2 * r + 1 + 2 * kField3PadRows;
  const int n = 4 * TR * SP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = i / (TR * SP), rem = i % (TR * SP);
  const int dy = rem / SP - (r + kField3PadRows), dx = rem % SP - r;
  T[i] = (float)class_kernel_value(t, dx, dy, r, kP, aP, gamma, (double)r);
}

}  // namespace

bool launch_field_v3(const Geo& g, const int32_t* bin_start, const uint32_t* rec,
                     const Tables& tb, const float* Fs, float* out, int out_row0, int store_lo,
                     int store_hi, unsigned int* tickets, cudaStream_t s, int ring) {
  if (!tb.CT3 || !field3_shape_ok(tb.shape, g.r)) return false;
#define SFM_V3(SP) \
  case SP: launch_v3<SP, 32>(g, bin_start, rec, tb.CT3, Fs, out, out_row0, store_lo, store_hi, s, tickets, ring); break;
  // one footprint: 32 x 32 su (measured against 32 x 16 and 16 x 32 row-
  // trimmed footprints, it was the fastest on the 16384^2 floor at r = 40)
  switch (field3_stride(g.r)) {
    SFM_V3(48)
    SFM_V3(80)
    SFM_V3(112)
    default:
      return false;
  }
#undef SFM_V3
  return true;
}

void launch_class_tables3(int r, const sfm_params& p, float* T, cudaStream_t s) {
  const int sp = field3_stride(r);
  if (!sp) return;
  const int n = (int)field3_table_floats(r);
  k_class_tables3<<<(n + 255) / 256, 256, 0, s>>>(r, sp, p.kP, p.aP, p.gamma, T);
}

}  // namespace sfm
