// sfm_surrogate.cu -- learned field surrogate: the exact near field (pedestrians
// within a small Chebyshev radius rn, by the same gather as the exact path)
// plus a 4-layer convolutional network that predicts the far field from
// per-cell occupancy and heading channels of an s-times coarsened grid,
// interpolated back to every su.  BF16 weights and activations, FP32
// accumulation; trained on the GPU by the kernels below (forward, backward,
// Adam) on fields the exact path computes; the exact path stays the judge
// (sfm_surrogate_eval: field error and decision flip rate).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sfm_ctx.h"
#include "sfm_gather.cuh"

using namespace sfm;

namespace {

typedef __nv_bfloat16 bf16;

// network layers: (Cin, Cout, kernel)
constexpr int kL1i = 3, kL1o = 32, kL1k = 5;
constexpr int kLh = 32, kLk = 3;
constexpr int kHalo = (kL1k - 1) / 2 + 3 * ((kLk - 1) / 2);  // 5 cells of context
constexpr int kNW1 = kL1k * kL1k * kL1i * kL1o, kNW2 = kLk * kLk * kLh * kLh,
              kNW4 = kLk * kLk * kLh * 1;
constexpr int kNParams = kNW1 + kL1o + 2 * (kNW2 + kLh) + kNW4 + 1;
// parameter blocks in the internal flat order: W1 b1 W2 b2 W3 b3 W4 b4, each W
// stored [ky][kx][cin][cout]
constexpr int kOffW[4] = {0, kNW1 + kL1o, kNW1 + kL1o + kNW2 + kLh,
                          kNW1 + kL1o + 2 * (kNW2 + kLh)};
constexpr int kOffB[4] = {kNW1, kNW1 + kL1o + kNW2, kNW1 + kL1o + 2 * kNW2 + kLh,
                          kNW1 + kL1o + 2 * (kNW2 + kLh) + kNW4};
constexpr int kTile = 16;  // output pixels per CTA side
static_assert(kNParams == 3 * 32 * 25 + 32 + 2 * (32 * 32 * 9 + 32) + 32 * 9 + 1, "params");

// ------------------------------------------- tensor-core 3x3 (mma.sync)
// Implicit GEMM on mma.sync m16n8k16 (BF16 operands, FP32 accumulators) for
// the 32 -> 1 last layer, and for the 32 -> 32 layers when the tcgen05
// kernel below is not used: a CTA computes 4 MT output rows x 16 pixels;
// warp w owns rows MT w .. MT w + MT - 1 (one m16 tile each) and the NT n8
// tiles of output channels.  K runs over the 9 kernel offsets x 2 blocks of
// 16 input channels.  The input tile and the weights sit in shared memory
// channel-last with rows padded to 40 channels (80 bytes), which keeps the
// ldmatrix row fetches free of bank conflicts.  Weights in shared memory:
// [ky][kx][out][in], BF16.  The CTAs are persistent: each loads the weights
// once and takes the tiles with the grid's stride, copying the next tile's
// input with cp.async into the second of two buffers while it computes the
// current one.  (Layer 1 uses the 8 x 16 tiles of kTcRows.)
constexpr int kTcRows = 8, kTcCols = 16, kTcPad = 40;

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// input tile of a CTA computing 4 MT output rows, and the shared memory of
// weights plus two input buffers (BF16 elements / bytes)
__host__ __device__ constexpr int conv3_in_elems(int MT) { return (4 * MT + 2) * (kTcCols + 2) * kTcPad; }
constexpr int kC3W = 9 * 32 * kTcPad;
constexpr size_t conv3_smem(int MT) { return (size_t)(kC3W + 2 * conv3_in_elems(MT)) * 2; }

// NT n8 tiles of output channels: 4 (32 -> 32, ReLU, BF16 out) or 1 for
// layer 4 (32 -> 1: weights of output 0 in row 0 of the n8 tile, rows 1-7
// zero; no activation, FP32 out in yout).  MT m16 tiles (output rows) per
// warp: a CTA computes 4 MT rows x 16 pixels.
template <int NT, int MT>
__global__ void __launch_bounds__(128, MT == 4 ? 3 : 4)
    k_conv3_tc(const bf16* __restrict__ in, int Hin, int Win, const bf16* __restrict__ Wt,
               const float* __restrict__ b, bf16* __restrict__ out, float* __restrict__ yout) {
  extern __shared__ __align__(16) bf16 sm3[];
  bf16* sW = sm3;
  const int Hout = Hin - 2, Wout = Win - 2;
  constexpr int R = 4 * MT, IN = conv3_in_elems(MT);
  const int ntx = (Wout + kTcCols - 1) / kTcCols, ntiles = ntx * ((Hout + R - 1) / R);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sW0 = (uint32_t)__cvta_generic_to_shared(sW);
  const uint32_t sIn0 = sW0 + (uint32_t)kC3W * 2;
  // weights: 9 x 8 NT rows of 32 channels (4 chunks of 16 bytes each), once per CTA
  for (int i = tid; i < 9 * 8 * NT * 4; i += blockDim.x) {
    const int q = i & 3, row = i >> 2;
    cp_async16(sW0 + (uint32_t)(row * kTcPad + q * 8) * 2, Wt + row * 32 + q * 8);
  }
  // input tile t (with a 1-pixel halo on the right and bottom) into buffer bi;
  // pixels outside the image are zeros
  auto fetch = [&](int t, int bi) {
    const int x0 = (t % ntx) * kTcCols, y0 = (t / ntx) * R;
    const uint32_t base = sIn0 + (uint32_t)(bi * IN) * 2;
    for (int i = tid; i < (R + 2) * (kTcCols + 2) * 4; i += blockDim.x) {
      const int q = i & 3, p = i >> 2, px = p % (kTcCols + 2), py = p / (kTcCols + 2);
      const int gy = y0 + py, gx = x0 + px;
      const uint32_t dst = base + (uint32_t)(p * kTcPad + q * 8) * 2;
      if (gy < Hin && gx < Win)
        cp_async16(dst, in + ((size_t)gy * Win + gx) * 32 + q * 8);
      else
        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0));
    }
  };
  int t = blockIdx.x, bi = 0;
  if (t < ntiles) fetch(t, 0);
  cp_async_commit();
  // ldmatrix lane roles: A rows (pixels) and column halves; B rows (out channels)
  const int a_row = (lane & 7) + 8 * ((lane >> 3) & 1), a_col = 8 * (lane >> 4);
  const int b_n = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
  const int g = lane >> 2, cp = 2 * (lane & 3);
  for (; t < ntiles; t += gridDim.x, bi ^= 1) {
    // the next tile's copies run while this one is computed
    if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x, bi ^ 1);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const uint32_t sIn = sIn0 + (uint32_t)(bi * IN) * 2;
    float acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[mt][nt][k] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 9; ++kk) {
      const int ky = kk / 3, kx = kk % 3;
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        uint32_t bw[NT][2];
        if constexpr (NT == 4) {
#pragma unroll
          for (int np = 0; np < 2; ++np) {
            const uint32_t addr =
                sW0 + (uint32_t)(((kk * 32 + np * 16 + b_n) * kTcPad + kb * 16 + b_k) * 2);
            ldsm_x4(addr, bw[2 * np][0], bw[2 * np][1], bw[2 * np + 1][0], bw[2 * np + 1][1]);
          }
        } else {
          // one n8 tile: lanes 0-15 address rows (lane & 7) at k offset 8 (lane >> 3)
          const uint32_t addr =
              sW0 + (uint32_t)(((kk * 8 + (lane & 7)) * kTcPad + kb * 16 + 8 * ((lane >> 3) & 1)) * 2);
          ldsm_x2(addr, bw[0][0], bw[0][1]);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int py = MT * warp + mt + ky, px = a_row + kx;
          const uint32_t addr =
              sIn + (uint32_t)(((py * (kTcCols + 2) + px) * kTcPad + kb * 16 + a_col) * 2);
          uint32_t a0, a1, a2, a3;
          ldsm_x4(addr, a0, a1, a2, a3);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, bw[nt][0], bw[nt][1]);
        }
      }
    }
    // epilogue: accumulator (row g = lane/4 and g+8, column pair 2*(lane%4))
    // of each m16 x n8 tile; bias, then ReLU and BF16 (NT 4) or channel 0 in
    // FP32 (NT 1)
    const int x0 = (t % ntx) * kTcCols, y0 = (t / ntx) * R;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int y = y0 + MT * warp + mt;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int x = x0 + g + 8 * half;
        if (y >= Hout || x >= Wout) continue;
        if constexpr (NT == 1) {
          if (cp == 0) yout[(size_t)y * Wout + x] = acc[mt][0][2 * half] + b[0];
        } else {
          __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + ((size_t)y * Wout + x) * 32);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int c = nt * 8 + cp;
            const float v0 = fmaxf(acc[mt][nt][2 * half] + b[c], 0.f);
            const float v1 = fmaxf(acc[mt][nt][2 * half + 1] + b[c + 1], 0.f);
            o[c / 2] = __floats2bfloat162_rn(v0, v1);
          }
        }
      }
    }
    // every warp is done with this buffer before it is refilled
    __syncthreads();
  }
  cp_async_wait_all();
}

// ------------------------------- 5th-generation tensor cores: 3x3, 32 -> 32
// The 32 -> 32 layers as an implicit GEMM on tcgen05.  A tile is 4 output
// rows x 128 pixels; each row is one M = 128, N = 32 accumulator in TMEM,
// summed over K = 9 kernel offsets x 2 blocks of 16 channels by 18 MMAs
// (BF16 operands from shared memory, FP32 accumulation), issued with the
// rows interleaved so that consecutive MMAs write different accumulators.
// An input row (130 pixels x all 32 channels, 64 bytes a pixel) arrives in
// one TMA copy with the 64-byte swizzle, which is the K-major SWIZZLE_64B
// operand layout (a pixel is a row of 64 bytes, 8-row groups 512 bytes
// apart): the A operand of kernel offset (ky, kx) and channel block kb for
// output row j starts at input row j + ky, pixel kx, byte 32 kb (the
// swizzle follows the absolute shared-memory address, so the shifts need no
// base offset).  The weights use the no-swizzle layout [ky kx][block of 16]
// [half][out][8 in].  One persistent CTA an SM, warp-specialised:
//   warp 0 (one lane): TMA copies of each tile's 6 input rows (zeros outside
//     the image) into a ring of kWsStages buffers;
//   warp 1 (one lane): the MMAs of a tile into one of two TMEM accumulator
//     sets; tcgen05.commit frees the input buffer and hands the set on;
//   warps 2-9: each reads its 32 TMEM lanes (pixels) of two of the set's
//     rows (two warps share a lane quarter), stores bias + ReLU in BF16, then
//     frees its part of the set.
// Copies, MMAs and stores of different tiles overlap.  Every wait is
// bounded: on a timeout a role stops, the kernel raises an error flag, frees
// its TMEM and returns.  Measured on the 16384^2 floor's 2054^2 images: 133
// us a layer against 207 us for the mma.sync kernel.
constexpr int kUmRows = 4, kUmCols = 128, kUmInPx = kUmCols + 2, kUmInRows = kUmRows + 2;
// one input row: 130 pixels x 64 bytes (all 32 channels), one TMA copy with
// the 64-byte swizzle, in a 512-byte aligned slot
constexpr int kUmRowBytes = (kUmInPx * 64 + 511) / 512 * 512;
constexpr int kUmA = kUmInRows * kUmRowBytes;       // bytes of one input tile buffer
constexpr int kUmB = 9 * 2 * 2 * 32 * 16;           // bytes of the weights
constexpr int kWsStages = 4, kWsThreads = 320;  // warps 0, 1 and 8 store warps
constexpr int kUmTmemCols = 256;                    // 2 accumulators x kUmRows x 32 columns
constexpr size_t kUmSmem = (size_t)kWsStages * kUmA + kUmB + (2 * kWsStages + 4) * 8 + 16 + 512;
constexpr uint32_t kUmTx = (uint32_t)(kUmInRows * kUmInPx * 64);  // TMA bytes a tile
constexpr uint32_t kUmIdesc =                       // kind::f16 instruction descriptor
    (1u << 4) |                                     // D: FP32
    (1u << 7) | (1u << 10) |                        // A, B: BF16 (both K-major)
    ((uint32_t)(32 >> 3) << 17) |                   // N = 32
    ((uint32_t)(128 >> 4) << 24);                   // M = 128
static_assert(kUmRowBytes % 512 == 0 && kUmA % 512 == 0 && kUmB % 16 == 0,
              "TMA destinations and operands must stay aligned");
static_assert(2 * kUmRows * 32 <= kUmTmemCols, "accumulators exceed the TMEM allocation");
static_assert(kUmSmem <= 227 * 1024, "shared memory of the tcgen05 convolution");

// shared-memory matrix descriptor, no swizzle: start, K-direction (leading)
// and M/N-direction (stride) byte offsets between core matrices
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// the same with the 64-byte swizzle (K-major rows of 64 bytes, 8-row groups
// 512 bytes apart; the leading offset is unused)
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) |
         (1ull << 46) | (4ull << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// bounded wait for the mbarrier phase `parity`; false on a timeout.  The
// bound is about one second of the global timer (checked every 256 tries,
// each of which may suspend the thread for a short, system-defined time),
// with an iteration cap behind it.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint64_t t0 = 0;
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255) {
      uint64_t now;
      asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(now));
      if (t0 == 0)
        t0 = now;
      else if (now - t0 > 1000000000ull)
        return false;
    }
  }
  return false;
}

__global__ void __launch_bounds__(kWsThreads, 1)
    k_conv3_umma(const __grid_constant__ CUtensorMap tmap, int Hin, int Win,
                 const bf16* __restrict__ Wu, const float* __restrict__ b, bf16* __restrict__ out,
                 int* __restrict__ err, int stop_after) {
  extern __shared__ __align__(1024) uint8_t smu_raw[];
  // the swizzled buffers start on a 512-byte boundary (512 bytes allocated spare)
  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smu_raw);
  const uint32_t sA0 = (raw + 511u) & ~511u;
  uint8_t* smu = smu_raw + (sA0 - raw);
  const uint32_t sB = sA0 + kWsStages * kUmA, bar = sB + kUmB;
  // mbarriers: full[s], empty[s] (input ring), accf[a], acce[a] (accumulators)
  const uint32_t tslot = bar + (2 * kWsStages + 4) * 8;
  // after the TMEM address: the last iteration whose copies the producer
  // issued and the last one whose MMAs were committed (-1: none), which the
  // drain after a failed wait needs
  volatile int* last_issued = reinterpret_cast<volatile int*>(smu + (tslot - sA0) + 4);
  auto full = [&](int st) { return bar + 8 * st; };
  auto empty = [&](int st) { return bar + 8 * (kWsStages + st); };
  auto accf = [&](int ac) { return bar + 8 * (2 * kWsStages + ac); };
  auto acce = [&](int ac) { return bar + 8 * (2 * kWsStages + 2 + ac); };
  const int Hout = Hin - 2, Wout = Win - 2;
  const int ntx = (Wout + kUmCols - 1) / kUmCols, ntiles = ntx * ((Hout + kUmRows - 1) / kUmRows);
  const int my = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // weights once per CTA (already in the core-matrix layout, 16-byte chunks)
  for (int i = tid; i < kUmB / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smu + kWsStages * kUmA)[i] = reinterpret_cast<const uint4*>(Wu)[i];
  if (tid == 0) {
    last_issued[0] = -1;
    last_issued[1] = -1;
    for (int st = 0; st < kWsStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full(st)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(st)));
    }
    for (int ac = 0; ac < 2; ++ac) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(accf(ac)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(acce(ac)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tslot),
                 "r"(kUmTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  uint32_t tmem;
  asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem) : "r"(tslot));
  bool failed = false;
  if (warp == 0) {
    // producer: TMA copies into the ring
    if (lane == 0) {
      for (int it = 0; it < my; ++it) {
        const int t = blockIdx.x + it * gridDim.x, st = it % kWsStages;
        const uint32_t ph = (uint32_t)(it / kWsStages) & 1u;
        // test hook: stop issuing, so that the consumers' waits run out
        if (stop_after >= 0 && it >= stop_after) break;
        if (!mbar_wait(empty(st), ph ^ 1u)) {
          failed = true;
          break;
        }
        const int x0 = (t % ntx) * kUmCols, y0 = (t / ntx) * kUmRows;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full(st)), "r"(kUmTx)
                     : "memory");
        const uint32_t base = sA0 + (uint32_t)(st * kUmA);
        for (int r = 0; r < kUmInRows; ++r)
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
              "%4}], [%5];\n" ::"r"(base + (uint32_t)(r * kUmRowBytes)),
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(x0), "r"(y0 + r), "r"(full(st))
              : "memory");
        last_issued[0] = it;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // MMA issue
    if (lane == 0) {
      for (int it = 0; it < my; ++it) {
        const int st = it % kWsStages, ac = it & 1;
        const uint32_t ph = (uint32_t)(it / kWsStages) & 1u, pa = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(full(st), ph) || !mbar_wait(acce(ac), pa ^ 1u)) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // the rows' accumulations interleaved: consecutive MMAs write
        // different accumulators; every descriptor is a base plus a
        // compile-time offset (addresses stay below 256 KB, so the 14-bit
        // start field takes the sum without a carry)
        const uint64_t a0 = umma_desc_sw64(sA0 + (uint32_t)(st * kUmA));
        const uint64_t b0 = umma_desc(sB, 512, 128);
        const uint32_t d0 = tmem + (uint32_t)(ac * kUmRows * 32);
#pragma unroll
        for (int kk = 0; kk < 9; ++kk) {
#pragma unroll
          for (int kb = 0; kb < 2; ++kb) {
            const uint64_t bd = b0 + (uint64_t)(((kk * 2 + kb) * 1024) >> 4);
#pragma unroll
            for (int j = 0; j < kUmRows; ++j) {
              const uint64_t ad =
                  a0 + (uint64_t)(((j + kk / 3) * kUmRowBytes + (kk % 3) * 64 + kb * 32) >> 4);
              umma_f16(d0 + (uint32_t)(j * 32), ad, bd, kUmIdesc, (kk | kb) != 0);
            }
          }
        }
        umma_commit(empty(st));
        umma_commit(accf(ac));
        last_issued[1] = it;
      }
    }
    __syncwarp();
  } else {
    // stores: warp w reads TMEM lanes 32 (w % 4) .. + 31 (pixels) of rows
    // jh, jh + 2 (two warps share a lane quarter)
    const int sp = warp & 3, jh = (warp - 2) >> 2;
    float bias[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) bias[c] = b[c];
    for (int it = 0; it < my; ++it) {
      const int t = blockIdx.x + it * gridDim.x, ac = it & 1;
      const uint32_t pa = (uint32_t)(it >> 1) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(accf(ac), pa))) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int x0 = (t % ntx) * kUmCols, y0 = (t / ntx) * kUmRows;
      const int px = x0 + 32 * sp + lane;
      // this warp's two rows (64 values in registers), then its part of the
      // accumulator set is freed
      {
        uint32_t v[2][32];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
              "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
              "%28, %29, %30, %31}, [%32];\n"
              : "=r"(v[jj][0]), "=r"(v[jj][1]), "=r"(v[jj][2]), "=r"(v[jj][3]), "=r"(v[jj][4]),
                "=r"(v[jj][5]), "=r"(v[jj][6]), "=r"(v[jj][7]), "=r"(v[jj][8]), "=r"(v[jj][9]),
                "=r"(v[jj][10]), "=r"(v[jj][11]), "=r"(v[jj][12]), "=r"(v[jj][13]), "=r"(v[jj][14]),
                "=r"(v[jj][15]), "=r"(v[jj][16]), "=r"(v[jj][17]), "=r"(v[jj][18]), "=r"(v[jj][19]),
                "=r"(v[jj][20]), "=r"(v[jj][21]), "=r"(v[jj][22]), "=r"(v[jj][23]), "=r"(v[jj][24]),
                "=r"(v[jj][25]), "=r"(v[jj][26]), "=r"(v[jj][27]), "=r"(v[jj][28]), "=r"(v[jj][29]),
                "=r"(v[jj][30]), "=r"(v[jj][31])
              : "r"(tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)((ac * kUmRows + jh + 2 * jj) * 32)));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int y = y0 + jh + 2 * jj;
          if (px < Wout && y < Hout) {
            uint32_t o[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const float a0 = fmaxf(__uint_as_float(v[jj][2 * c]) + bias[2 * c], 0.f);
              const float a1 = fmaxf(__uint_as_float(v[jj][2 * c + 1]) + bias[2 * c + 1], 0.f);
              const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
              o[c] = *reinterpret_cast<const uint32_t*>(&h);
            }
            uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)y * Wout + px) * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acce(ac)) : "memory");
    }
  }
  if (failed) atomicExch(err, 1);
  // Every role has stopped (all waits are bounded).  After a failure the
  // copies and MMAs still in flight are waited for, bounded, before TMEM is
  // freed and the CTA exits: for each ring stage the phase of full(st) that
  // the last copies issued into it complete (iteration i lands phase
  // i / stages of stage i % stages), and the phase of the accumulator
  // barrier that the last commit completes (a tcgen05.commit tracks every
  // MMA this thread issued before it).
  if (__syncthreads_or(failed ? 1 : 0) && tid == 0) {
    const int li = last_issued[0], lm = last_issued[1];
    for (int st = 0; st < kWsStages; ++st) {
      if (li < st) continue;
      const int i = li - (li - st) % kWsStages;
      mbar_wait(full(st), (uint32_t)(i / kWsStages) & 1u);
    }
    if (lm >= 0) mbar_wait(accf(lm & 1), (uint32_t)(lm >> 1) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kUmTmemCols));
}

// BF16 weights of a 3x3 32->32 layer in the tcgen05 operand layout:
// [ky kx][block of 16 inputs][half][out][8 inputs], from the internal
// [ky][kx][in][out] floats.
__global__ void k_pack_wum(const float* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * 32 * 32) return;
  const int e = i % 8, o = (i / 8) % 32, h = (i / 256) % 2, kb = (i / 512) % 2, kk = i / 1024;
  const int c = kb * 16 + h * 8 + e;
  wt[i] = __float2bfloat16(w[(kk * 32 + c) * 32 + o]);
}

// BF16 weights of a 3x3 32->32 layer for the tensor-core kernel:
// [ky][kx][out][in] from the internal [ky][kx][in][out] floats.
__global__ void k_pack_w3(const float* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * 32 * 32) return;
  const int c = i % 32, o = (i / 32) % 32, kk = i / 1024;
  wt[i] = __float2bfloat16(w[(kk * 32 + c) * 32 + o]);
}

// BF16 weights of layer 4 (3x3, 32 -> 1) as one n8 tile: [ky][kx][8][in],
// row 0 the output's weights, rows 1-7 zero.
__global__ void k_pack_w4(const float* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * 8 * 32) return;
  const int c = i % 32, o = (i / 32) % 8, kk = i / 256;
  wt[i] = __float2bfloat16(o == 0 ? w[kk * 32 + c] : 0.f);
}

// ------------------------------------------- tensor-core 5x5, 3 -> 32
// Layer 1 as an implicit GEMM, one k16 step per kernel row ky: the K entries
// of row ky are (kx, c), 15 of them plus a zero, which for output pixel px
// are the 15 consecutive input elements from pixel px of input row py + ky
// (channel-last).  The CTA stages its 12 x 20-pixel input tile, expands each
// of its 12 x 16 (row, pixel) starts to such a 16-element run (rows padded
// to 24 elements, 48 bytes, so the ldmatrix row fetches hit distinct banks;
// a 5x expansion where a full im2col is 25x) and runs 5 k16 steps of
// m16n8k16 per m16 tile with A rows from row py + ky of the runs; layout of
// warps and fragments as k_conv3_tc, and persistent CTAs as there (the next
// tile's input is prefetched into registers).  Weights: [ky][out][16].
constexpr int kC1K = 80, kC1Run = 24;
constexpr int kC1CtasPerSm = 6;
constexpr int kC1TileElems = (kTcRows + 4) * (kTcCols + 4) * 3;  // input tile, BF16 elements
constexpr int kC1PerThread = (kC1TileElems + 127) / 128;
constexpr int kC1Starts = (kTcRows + 4) * kTcCols;               // (row, pixel) run starts
static_assert(kC1TileElems % 2 == 0, "the input tile is read as 32-bit words");

__global__ void __launch_bounds__(128)
    k_conv1_tc(const bf16* __restrict__ in, int Hin, int Win, const bf16* __restrict__ Wt,
               const float* __restrict__ b, bf16* __restrict__ out) {
  constexpr int TH = kTcRows + 4, TW = kTcCols + 4;
  __shared__ __align__(16) bf16 sX[TH * TW * 3];
  __shared__ __align__(16) bf16 sR[kC1Starts * kC1Run];
  __shared__ __align__(16) bf16 sW[5 * 32 * kC1Run];
  const int Hout = Hin - 4, Wout = Win - 4;
  const int ntx = (Wout + kTcCols - 1) / kTcCols, ntiles = ntx * ((Hout + kTcRows - 1) / kTcRows);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 5 * 32 * 16; i += blockDim.x) sW[(i / 16) * kC1Run + i % 16] = Wt[i];
  // persistent CTAs take the tiles with the grid's stride; the next tile's
  // input elements are loaded into registers while the current one is computed
  bf16 pre[kC1PerThread];
  auto fetch = [&](int t) {
    const int x0 = (t % ntx) * kTcCols, y0 = (t / ntx) * kTcRows;
#pragma unroll
    for (int u = 0; u < kC1PerThread; ++u) {
      const int i = tid + 128 * u;
      const int c = i % 3, p = i / 3, px = p % TW, py = p / TW;
      const int gy = y0 + py, gx = x0 + px;
      pre[u] = (i < kC1TileElems && gy < Hin && gx < Win) ? in[((size_t)gy * Win + gx) * 3 + c]
                                                         : __float2bfloat16(0.f);
    }
  };
  if ((int)blockIdx.x < ntiles) fetch(blockIdx.x);
  const uint32_t sR0 = (uint32_t)__cvta_generic_to_shared(sR);
  const uint32_t sW0 = (uint32_t)__cvta_generic_to_shared(sW);
  const uint32_t* sXw = reinterpret_cast<const uint32_t*>(sX);
  const int a_row = (lane & 7) + 8 * ((lane >> 3) & 1), a_col = 8 * (lane >> 4);
  const int b_n = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
  const int g = lane >> 2, cp = 2 * (lane & 3);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
#pragma unroll
    for (int u = 0; u < kC1PerThread; ++u)
      if (tid + 128 * u < kC1TileElems) sX[tid + 128 * u] = pre[u];
    __syncthreads();
    if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x);
    // runs: start (py, px) holds input elements e0 .. e0 + 14, e0 = (py TW + px) 3,
    // and a zero; read as the 8 words from e0 rounded down to even
    for (int j = tid; j < kC1Starts; j += blockDim.x) {
      const int py = j / kTcCols, px = j % kTcCols;
      const int e0 = (py * TW + px) * 3, w0 = e0 >> 1;
      uint32_t w[9];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = sXw[w0 + k];
      w[8] = 0u;
      uint32_t o[8];
      if (e0 & 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __byte_perm(w[k], w[k + 1], 0x5432);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = w[k];
      }
      o[7] &= 0x0000ffffu;  // the 16th entry is zero
      uint4* dst = reinterpret_cast<uint4*>(sR + j * kC1Run);
      dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
      dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[mt][nt][k] = 0.f;
#pragma unroll
    for (int ky = 0; ky < 5; ++ky) {
      uint32_t bw[4][2];
#pragma unroll
      for (int np = 0; np < 2; ++np)
        ldsm_x4(sW0 + (uint32_t)(((ky * 32 + np * 16 + b_n) * kC1Run + b_k) * 2), bw[2 * np][0],
                bw[2 * np][1], bw[2 * np + 1][0], bw[2 * np + 1][1]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int prow = (2 * warp + mt + ky) * kTcCols + a_row;
        uint32_t a0, a1, a2, a3;
        ldsm_x4(sR0 + (uint32_t)((prow * kC1Run + a_col) * 2), a0, a1, a2, a3);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, bw[nt][0], bw[nt][1]);
      }
    }
    const int x0 = (t % ntx) * kTcCols, y0 = (t / ntx) * kTcRows;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int y = y0 + 2 * warp + mt;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int x = x0 + g + 8 * half;
        if (y >= Hout || x >= Wout) continue;
        __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + ((size_t)y * Wout + x) * 32);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int c = nt * 8 + cp;
          const float v0 = fmaxf(acc[mt][nt][2 * half] + b[c], 0.f);
          const float v1 = fmaxf(acc[mt][nt][2 * half + 1] + b[c + 1], 0.f);
          o[c / 2] = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
    // sX and sR are rewritten by the next tile
    __syncthreads();
  }
}

// BF16 layer-1 weights [ky][out][16] (entry kk = kx*3 + c, zero at 15) from
// the internal [ky][kx][in][out] floats.
__global__ void k_pack_w1(const float* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 5 * 32 * 16) return;
  const int kk = i % 16, o = (i / 16) % 32, ky = i / 512;
  wt[i] = __float2bfloat16(kk < 15 ? w[(ky * 15 + kk) * 32 + o] : 0.f);
}

// -------------------------------------------------------------- backward
// dZ of a layer output: the incoming gradient, masked by the ReLU (A > 0).
__device__ __forceinline__ float dz_at(const float* dA, const bf16* A, size_t i, bool relu) {
  return relu ? (__bfloat162float(A[i]) > 0.f ? dA[i] : 0.f) : dA[i];
}

// dIn[y][x][c] = sum_{ky,kx,o} W[ky][kx][c][o] * dZ[y-ky][x-kx][o]
template <int CIN, int COUT, int K, bool RELU>
__global__ void __launch_bounds__(kTile* kTile)
    k_conv_dx(const float* __restrict__ dA, const bf16* __restrict__ A, int Hout, int Wout,
              const float* __restrict__ Wt, float* __restrict__ dIn) {
  constexpr int TI = kTile + K - 1;
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;
  float* sD = sm + K * K * CIN * COUT;  // dZ tile: output rows y0-K+1 .. y0+kTile-1
  const int Hin = Hout + K - 1, Win = Wout + K - 1;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const int tid = threadIdx.x;
  for (int i = tid; i < K * K * CIN * COUT; i += blockDim.x) sW[i] = Wt[i];
  for (int i = tid; i < TI * TI * COUT; i += blockDim.x) {
    const int o = i % COUT, p = i / COUT, px = p % TI, py = p / TI;
    const int gy = y0 - (K - 1) + py, gx = x0 - (K - 1) + px;
    float v = 0.f;
    if (gy >= 0 && gy < Hout && gx >= 0 && gx < Wout)
      v = dz_at(dA, A, ((size_t)gy * Wout + gx) * COUT + o, RELU);
    sD[i] = v;
  }
  __syncthreads();
  const int tx = tid % kTile, ty = tid / kTile;
  const int y = y0 + ty, x = x0 + tx;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  for (int ky = 0; ky < K; ++ky)
    for (int kx = 0; kx < K; ++kx) {
      const float* d = sD + ((ty - ky + K - 1) * TI + (tx - kx + K - 1)) * COUT;
      const float* w = sW + (ky * K + kx) * CIN * COUT;
      for (int o = 0; o < COUT; ++o) {
        const float v = d[o];
#pragma unroll
        for (int c = 0; c < CIN; ++c) acc[c] = fmaf(v, w[c * COUT + o], acc[c]);
      }
    }
  if (y >= Hin || x >= Win) return;
#pragma unroll
  for (int c = 0; c < CIN; ++c) dIn[((size_t)y * Win + x) * CIN + c] = acc[c];
}

// Per-CTA partial weight and bias gradients over a 16 x 16 tile of output
// pixels: part[cta][e] for e over W (K*K*CIN*COUT entries) then b (COUT).
template <int CIN, int COUT, int K, bool RELU>
__global__ void __launch_bounds__(kTile* kTile)
    k_conv_dw(const bf16* __restrict__ in, const float* __restrict__ dA, const bf16* __restrict__ A,
              int Hout, int Wout, float* __restrict__ part) {
  constexpr int TI = kTile + K - 1;
  constexpr int NE = K * K * CIN * COUT + COUT;
  extern __shared__ __align__(16) float sm[];
  float* sIn = sm;                   // TI*TI*CIN
  float* sD = sm + TI * TI * CIN;    // kTile*kTile*COUT
  const int Win = Wout + K - 1, Hin = Hout + K - 1;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const int tid = threadIdx.x;
  for (int i = tid; i < TI * TI * CIN; i += blockDim.x) {
    const int c = i % CIN, p = i / CIN, px = p % TI, py = p / TI;
    const int gy = y0 + py, gx = x0 + px;
    sIn[i] = (gy < Hin && gx < Win) ? __bfloat162float(in[((size_t)gy * Win + gx) * CIN + c]) : 0.f;
  }
  for (int i = tid; i < kTile * kTile * COUT; i += blockDim.x) {
    const int o = i % COUT, p = i / COUT, px = p % kTile, py = p / kTile;
    const int gy = y0 + py, gx = x0 + px;
    sD[i] = (gy < Hout && gx < Wout) ? dz_at(dA, A, ((size_t)gy * Wout + gx) * COUT + o, RELU) : 0.f;
  }
  __syncthreads();
  float* dst = part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NE;
  for (int e = tid; e < NE; e += blockDim.x) {
    float s = 0.f;
    if (e < K * K * CIN * COUT) {
      const int o = e % COUT, c = (e / COUT) % CIN, kk = e / (COUT * CIN), kx = kk % K, ky = kk / K;
      for (int p = 0; p < kTile * kTile; ++p) {
        const int px = p % kTile, py = p / kTile;
        s = fmaf(sIn[((py + ky) * TI + (px + kx)) * CIN + c], sD[p * COUT + o], s);
      }
    } else {
      const int o = e - K * K * CIN * COUT;
      for (int p = 0; p < kTile * kTile; ++p) s += sD[p * COUT + o];
    }
    dst[e] = s;
  }
}

// g[e] = sum over CTAs (fixed order) of part[cta][e]
__global__ void k_reduce_parts(const float* __restrict__ part, int nparts, int ne,
                               float* __restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  float s = 0.f;
  for (int k = 0; k < nparts; ++k) s += part[(size_t)k * ne + e];
  g[e] = s;
}

// ------------------------------------------------------------------ loss
// dY = (Y - T) / N; part[cta] = sum of (Y - T)^2 over the CTA's pixels.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int n,
                      float* __restrict__ dY, float* __restrict__ part) {
  __shared__ float s[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float d = 0.f;
  if (i < n) {
    d = Y[i] - T[i];
    dY[i] = d / (float)n;
  }
  s[threadIdx.x] = d * d;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// ------------------------------------------------------------------ Adam
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 rounding of the FP32 master weights (the forward pass and the data
// gradient use BF16 weights, held here as floats).
__global__ void k_round_bf16(const float* __restrict__ p, float* __restrict__ q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = __bfloat162float(__float2bfloat16(p[i]));
}

// ----------------------------------------------------- lattice <-> coarse
__constant__ float c_hx[9] = {0.f, 1.f, 0.70710678f, 0.f, -0.70710678f, -1.f, -0.70710678f, 0.f,
                              0.70710678f};
__constant__ float c_hy[9] = {0.f, 0.f, 0.70710678f, 1.f, 0.70710678f, 0.f, -0.70710678f, -1.f,
                              -0.70710678f};

// X[i][j][0..2] over the padded coarse grid (kHalo cells around): pedestrian
// count and heading sums of the s x s cell, / s^2; wrapped or zero outside.
__global__ void k_coarse_in(Geo g, const uint8_t* __restrict__ ocls, int s, int Hc, int Wc,
                            bf16* __restrict__ X) {
  const int Wp = Wc + 2 * kHalo, Hp = Hc + 2 * kHalo;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Wp * Hp) return;
  int ci = idx / Wp - kHalo, cj = idx % Wp - kHalo;
  float n = 0.f, hx = 0.f, hy = 0.f;
  bool ok = true;
  if (ci < 0 || ci >= Hc) {
    if (g.py) ci = (ci + Hc) % Hc; else ok = false;
  }
  if (cj < 0 || cj >= Wc) {
    if (g.px) cj = (cj + Wc) % Wc; else ok = false;
  }
  if (ok && s == 8) {
    // the cell's 8 rows of 8 bytes, all loads in flight at once
    uint2 w[8];
#pragma unroll
    for (int dy = 0; dy < 8; ++dy)
      w[dy] = *reinterpret_cast<const uint2*>(ocls + (size_t)(ci * 8 + dy) * g.opitch + cj * 8);
#pragma unroll
    for (int dy = 0; dy < 8; ++dy) {
      if (!(w[dy].x | w[dy].y)) continue;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int v = (int)(((e < 4 ? w[dy].x : w[dy].y) >> (8 * (e & 3))) & 0xffu);
        if (v) {
          n += 1.f;
          hx += c_hx[v - 1];
          hy += c_hy[v - 1];
        }
      }
    }
  } else if (ok && (s & 7) == 0) {
    // 8 bytes of a cell row per load (the grid's pitch is a multiple of 128);
    // empty words are skipped, the others summed byte by byte in row order
    for (int dy = 0; dy < s; ++dy) {
      const uint2* row = reinterpret_cast<const uint2*>(ocls + (size_t)(ci * s + dy) * g.opitch + cj * s);
      for (int dw = 0; dw < s / 8; ++dw) {
        const uint2 w = row[dw];
        if (!(w.x | w.y)) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int v = (int)(((e < 4 ? w.x : w.y) >> (8 * (e & 3))) & 0xffu);
          if (v) {
            n += 1.f;
            hx += c_hx[v - 1];
            hy += c_hy[v - 1];
          }
        }
      }
    }
  } else if (ok) {
    for (int dy = 0; dy < s; ++dy) {
      const uint8_t* row = ocls + (size_t)(ci * s + dy) * g.opitch + cj * s;
      for (int dx = 0; dx < s; ++dx) {
        const int v = row[dx];
        if (v) {
          n += 1.f;
          hx += c_hx[v - 1];
          hy += c_hy[v - 1];
        }
      }
    }
  }
  const float inv = 1.f / (float)(s * s);
  X[(size_t)idx * 3 + 0] = __float2bfloat16(n * inv);
  X[(size_t)idx * 3 + 1] = __float2bfloat16(hx * inv);
  X[(size_t)idx * 3 + 2] = __float2bfloat16(hy * inv);
}

// The same inputs from the binned records, for coarsenings that divide the
// bin side: a cell lies inside one bin, whose records are in row-major order,
// so the cell's pedestrians are summed in the order of the grid scan above.
// Reads the bins' records (a few MB) instead of the whole class grid.
__global__ void k_coarse_in_rec(Geo g, const int32_t* __restrict__ bin_start,
                                const uint32_t* __restrict__ rec, int s, int Hc, int Wc,
                                bf16* __restrict__ X) {
  const int Wp = Wc + 2 * kHalo, Hp = Hc + 2 * kHalo;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Wp * Hp) return;
  int ci = idx / Wp - kHalo, cj = idx % Wp - kHalo;
  float n = 0.f, hx = 0.f, hy = 0.f;
  bool ok = true;
  if (ci < 0 || ci >= Hc) {
    if (g.py) ci = (ci + Hc) % Hc; else ok = false;
  }
  if (cj < 0 || cj >= Wc) {
    if (g.px) cj = (cj + Wc) % Wc; else ok = false;
  }
  if (ok) {
    const int x0 = cj * s, y0 = ci * s;
    const int b = (y0 / kBin) * g.nbx + x0 / kBin;
    const uint32_t cx0 = (uint32_t)(x0 % kBin), cy0 = (uint32_t)(y0 % kBin);
    const int e = bin_start[b + 1];
    for (int k = bin_start[b]; k < e; ++k) {
      const uint32_t rc = rec[k];
      if ((rc & 0xffu) - cx0 < (uint32_t)s && ((rc >> 8) & 0xffu) - cy0 < (uint32_t)s) {
        const int cls = (int)((rc >> 16) & 0xfu);
        n += 1.f;
        hx += c_hx[cls];
        hy += c_hy[cls];
      }
    }
  }
  const float inv = 1.f / (float)(s * s);
  X[(size_t)idx * 3 + 0] = __float2bfloat16(n * inv);
  X[(size_t)idx * 3 + 1] = __float2bfloat16(hx * inv);
  X[(size_t)idx * 3 + 2] = __float2bfloat16(hy * inv);
}

// T[i][j] = mean over the cell of (F - Fnear) / scale: the far part of the
// exact field (Fnear holds the static field plus the near pedestrian part).
__global__ void k_targets(const float* __restrict__ F, const float* __restrict__ Fnear, int W,
                          int s, int Hc, int Wc, float inv_scale, float* __restrict__ T) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Hc * Wc) return;
  const int ci = idx / Wc, cj = idx % Wc;
  double acc = 0.0;
  for (int dy = 0; dy < s; ++dy)
    for (int dx = 0; dx < s; ++dx) {
      const size_t c = (size_t)(ci * s + dy) * W + cj * s + dx;
      acc += (double)(F[c] - Fnear[c]);
    }
  T[idx] = (float)(acc / (s * s)) * inv_scale;
}

// number of pedestrians (live, in bin order) whose two decisions differ;
// sums of |Fa - Fb| and |Fb - Fs| over the lattice (FP64 partials per CTA)
__global__ void k_diff_choices(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                               int nbins, const uint8_t* __restrict__ a, const uint8_t* __restrict__ b,
                               unsigned long long* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool d = false;
  if (i < bin_start[nbins]) {
    const int p = rec_id[i];
    d = a[p] != b[p];
  }
  const unsigned n = __popc(__ballot_sync(0xffffffffu, d));
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(cnt, (unsigned long long)n);
}

__global__ void k_field_err(const float* __restrict__ Fa, const float* __restrict__ Fb,
                            const float* __restrict__ Fs, size_t n, double* __restrict__ part) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    a += fabs((double)Fa[i] - (double)Fb[i]);
    b += fabs((double)Fb[i] - (double)Fs[i]);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

// ------------------------------------- decisions with an exact fallback
// Decisions on the surrogate field F_sur; a pedestrian whose energy margin
// (second best - best) is not above delta plus a rounding allowance joins
// the fallback list and is decided again on the exact field at its
// candidates.  If the error F_sur - F varies by less than the margin over a
// pedestrian's admissible candidates, every other candidate's exact energy
// stays strictly above the surrogate's choice, so the choice is the exact
// one (ties included).  ref / raw_flips (optional): count decisions that differ from
// ref before the fallback.
__device__ __forceinline__ float margin_allowance(float delta, float emag, float fmag) {
  return delta * 1.0001f + 1e-6f * (emag + fmag);
}

// The surrogate field at the 9 candidates of the pedestrian at q from its
// parts, as the lattice pass composes it: (Fs + near sum) + scale *
// bilinear(Y).  The near sum walks the records within reach (rn) of the 3 x 3
// block in the gather's order (halo bins row-major, records in bin order),
// so it holds the lattice pass's terms in its order.
struct NearPart {
  const float* CT;  // near-field class tables (global memory), radius rn
  int rn, SP, TS;
};

__device__ __forceinline__ void surrogate_at_candidates(
    const Geo& g, int2 q, const int (&cx)[3], const int (&ry)[3], const int32_t* __restrict__ bin_start,
    const uint32_t* __restrict__ rec, const float* __restrict__ Fs, const NearPart& np,
    const FarPart& far, float (&f)[9]) {
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  const int rn = np.rn;
  if (rn > 0) {
    const int x0 = q.x - 1, y0 = q.y - 1;
    const int xlo = x0 - rn, xhi = x0 + 2 + rn, ylo = y0 - rn, yhi = y0 + 2 + rn;
    const int nxl = halo_count(xlo, xhi, g.W, g.px), nyl = halo_count(ylo, yhi, g.H, g.py);
    for (int ey = 0; ey < nyl; ++ey) {
      int by, yoff;
      halo_entry(ey, ylo, yhi, g.H, g.py, y0, by, yoff);
      for (int ex = 0; ex < nxl; ++ex) {
        int bx, xoff;
        halo_entry(ex, xlo, xhi, g.W, g.px, x0, bx, xoff);
        const int id = by * g.nbx + bx;
        const int s1 = bin_start[id + 1];
        for (int i = bin_start[id]; i < s1; ++i) {
          const uint32_t rc = rec[i];
          const int rx = xoff + (int)(rc & 0xffu), rry = yoff + (int)((rc >> 8) & 0xffu);
          if (rx < -rn || rx > 2 + rn || rry < -rn || rry > 2 + rn) continue;
          const int cls = (int)((rc >> 16) & 0xfu);
          const int sx = class_sx(cls), sy = class_sy(cls);
          const float* p = np.CT + class_table(cls) * np.TS + (rn + kFieldPad - sy * rry) * np.SP + rn - sx * rx;
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int ccx = move_dx(k) + 1, ccy = move_dy(k) + 1;
            if (ccx - rx >= -rn && ccx - rx <= rn && ccy - rry >= -rn && ccy - rry <= rn)
              acc[k] += __ldg(p + sy * ccy * np.SP + sx * ccx);
          }
        }
      }
    }
  }
  FarAxis fx[3], fy[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fx[d] = far_axis(cx[d], far.inv_s, far.Wc, g.px);
    fy[d] = far_axis(ry[d], far.inv_s, far.Hc, g.py);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
    f[k] = (Fs[(size_t)ry[yi] * g.W + cx[xi]] + acc[k]) + far_value(far, fy[yi], fx[xi]);
  }
}

// CAND: the surrogate field is composed at the candidates (no lattice pass);
// else it is read from Fsur.
template <bool CAND>
__global__ void k_sur_decide(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                             int nbins, Geo g, const int2* __restrict__ xy,
                             const uint8_t* __restrict__ heading, const uint8_t* __restrict__ goal,
                             const uint8_t* __restrict__ cell, const uint8_t* __restrict__ ocls,
                             const int32_t* __restrict__ D, const float* __restrict__ Fsur,
                             const uint32_t* __restrict__ rec, const float* __restrict__ Fs,
                             NearPart np, FarPart far, float beta, const float* __restrict__ own,
                             const float* __restrict__ dirdot, float delta,
                             uint8_t* __restrict__ choice, int32_t* __restrict__ flag_list,
                             int32_t* __restrict__ nflag, uint8_t* __restrict__ fb_flag,
                             int32_t* __restrict__ fb_dd, uint32_t* __restrict__ fb_info,
                             const uint8_t* __restrict__ ref,
                             unsigned long long* __restrict__ raw_flips, WalkPeriods wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool differs = false;
  const long long t = wp.period ? wp.ctr->t : 0;
  if (i < bin_start[nbins] && wp.period &&
      t % wp.period[rec_id[i]] != wp.phase[rec_id[i]]) {
    choice[rec_id[i]] = 0;  // not this pedestrian's tick (walk period): it stays
    fb_flag[i] = 0;
    differs = ref && ref[rec_id[i]] != 0;
  } else if (i < bin_start[nbins]) {
    const int p = rec_id[i];
    const int2 q = xy[p];
    int cx[3], ry[3];
    bool okx[3], oky[3];
    candidate_coords(q, g, cx, ry, okx, oky);
    float f[9], fmag = 0.f;
    if constexpr (CAND) {
      surrogate_at_candidates(g, q, cx, ry, bin_start, rec, Fs, np, far, f);
      // the candidates' other data are loaded after the field is composed
      // (fewer values live across the near walk)
      asm volatile("" ::: "memory");
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) f[k] = Fsur[(size_t)ry[move_dy(k) + 1] * g.W + cx[move_dx(k) + 1]];
    }
    int32_t dd[9];
    uint8_t oc[9];
    candidate_loads(g, ocls, D, cx, ry, dd, oc);
#pragma unroll
    for (int k = 0; k < 9; ++k) fmag = fmaxf(fmag, fabsf(f[k]));
    float margin, emag;
    const int best = pick_move<true>(f, dd, oc, okx, oky, heading[p], goal[p], beta, own,
                                     dirdot, &margin, &emag);
    choice[p] = (uint8_t)best;
    const bool fl = !(margin > margin_allowance(delta, emag, fmag));
    fb_flag[i] = fl;
    if (fl) {
      flag_list[atomicAdd(nflag, 1)] = i;
      // what the fallback's decision needs besides the field: guidance
      // distances, admissible candidates, heading and goal
      uint32_t mask = 0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        fb_dd[(size_t)i * 9 + k] = dd[k];
        const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
        if (k == 0 || (okx[xi] && oky[yi] && dd[k] != kDWall && oc[k] == 0)) mask |= 1u << k;
      }
      fb_info[i] = mask | (uint32_t)heading[p] << 9 | (uint32_t)goal[p] << 16;
    }
    differs = ref && ref[p] != best;
  }
  if (raw_flips) {
    const unsigned nd = __popc(__ballot_sync(0xffffffffu, differs));
    if ((threadIdx.x & 31) == 0 && nd) atomicAdd(raw_flips, (unsigned long long)nd);
  }
}

// Exact field at the 9 candidates of each listed pedestrian.  A warp takes
// 32 consecutive records in bin order (fb_flag marks the listed ones) and,
// for each run of them in one bin row, walks once the records in reach of
// the run's bounding box of candidate blocks, in the gather's order (halo
// bins row-major, records in bin order); each lane adds, for every record
// that reaches one of its pedestrian's candidates, the record's class-table
// entry into that candidate's sum.  Every pedestrian's halo entries are a
// subsequence of the box's, in the same order, so each sum holds the exact
// gather's terms in its order, bit for bit (its other terms are zero pads).
// With a wide table stride an out-of-reach candidate reads a zero pad, so
// only the narrow stride tests each candidate; the stride is a template
// parameter and each record's mirror signs pick one of four unrolled reads
// with immediate offsets (warp-uniform: every lane visits the same record).  The class tables are staged in shared
// memory as for the gather (one CTA of 1024 threads per SM).  Each listed
// pedestrian is then decided again with the exact path's energy on these
// values, from the guidance distances, admissibility, heading and goal that
// k_sur_decide stored for its slot (values of candidates outside the lattice
// are never used).
constexpr int kFbThreads = 1024;

// acc[k] += the class-table entry of candidate k = (cx, cy) at p + SY cy SP
// + SX cx (compile-time offsets; out-of-reach candidates read zero pads)
template <int SP, int SX, int SY>
__device__ __forceinline__ void add_candidates(const float* __restrict__ p, float (&acc)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] += p[SY * (move_dy(k) + 1) * SP + SX * (move_dx(k) + 1)];
}

constexpr int kFbRunBins = 8;  // widest run of bins whose pedestrians share one walk

template <int SP>
__global__ void __launch_bounds__(kFbThreads, 1)
    k_sur_fallback(const uint8_t* __restrict__ fb_flag, const int32_t* __restrict__ rec_id, int nbins,
                   Geo g, const int2* __restrict__ xy, const int32_t* __restrict__ bin_start,
                   const uint32_t* __restrict__ rec, const float* __restrict__ CT, int TS,
                   const float* __restrict__ Fs, const int32_t* __restrict__ fb_dd,
                   const uint32_t* __restrict__ fb_info, float beta, const float* __restrict__ own,
                   const float* __restrict__ dirdot, uint8_t* __restrict__ choice) {
  extern __shared__ __align__(16) float sm[];
  float* sT = sm + kTableGuard;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int2* scr = reinterpret_cast<int2*>(sT + 4 * TS) + w * 32;
  copy_to_shared<8>(reinterpret_cast<float2*>(sT), reinterpret_cast<const float2*>(CT), 2 * TS);
  __syncthreads();
  const int nrec = bin_start[nbins], r = g.r;
  const int nchunks = (nrec + 31) / 32;
  for (int c = blockIdx.x * nw + w; c < nchunks; c += gridDim.x * nw) {
    const int i = c * 32 + lane;
    const bool fl = i < nrec && fb_flag[i] != 0;
    unsigned todo = __ballot_sync(0xffffffffu, fl);
    if (!todo) continue;
    const int2 q = fl ? xy[rec_id[i]] : make_int2(0, 0);
    const int brow = q.y / kBin, bcol = q.x / kBin;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    while (todo) {
      // the listed lanes of the first remaining bin row within kFbRunBins bins
      // of its first listed lane (bin order keeps them contiguous)
      const int lead = __ffs(todo) - 1;
      const int row = __shfl_sync(0xffffffffu, brow, lead), col0 = __shfl_sync(0xffffffffu, bcol, lead);
      const bool mine = ((todo >> lane) & 1u) && brow == row && bcol - col0 < kFbRunBins;
      todo &= ~__ballot_sync(0xffffffffu, mine);
      const int xmin = __reduce_min_sync(0xffffffffu, mine ? q.x : INT_MAX);
      const int xmax = __reduce_max_sync(0xffffffffu, mine ? q.x : INT_MIN);
      const int ymin = __reduce_min_sync(0xffffffffu, mine ? q.y : INT_MAX);
      const int ymax = __reduce_max_sync(0xffffffffu, mine ? q.y : INT_MIN);
      // box of the candidate blocks (at most 8 bins + 2 su wide, a bin + 2
      // high), this lane's block origin inside it, and the lane's part of a
      // table address (for mirror signs sx, sy: sy oy SP + sx ox)
      const int x0 = xmin - 1, y0 = ymin - 1, ox = q.x - xmin, oy = q.y - ymin;
      const int lox = ox - r, loy = oy - r, span = 2 * r + 2;
      // item: x = the record's part of a table address (class table, row and
      // column of candidate (0, 0)), y = its box coordinates + 64 (11 bits
      // each) and its mirror bits
      walk_records_box(
          g, bin_start, rec, scr, lane, x0, y0, xmax - xmin + 3, ymax - ymin + 3,
          [&](int rx, int ry, int cls) {
            const int sx = class_sx(cls), sy = class_sy(cls);
            return make_int2(class_table(cls) * TS + (r + kFieldPad - sy * ry) * SP + r - sx * rx,
                             (rx + 64) | (ry + 64) << 11 | (sx < 0 ? 1 : 0) << 22 |
                                 (sy < 0 ? 1 : 0) << 23);
          },
          [&](const int2 it) {
            const int rxu = (it.y & 2047) - 64, ryu = ((it.y >> 11) & 2047) - 64;
            if (mine && (unsigned)(rxu - lox) <= (unsigned)span && (unsigned)(ryu - loy) <= (unsigned)span) {
              const int m = (it.y >> 22) & 3;
              const float* p = sT + it.x + ((m & 2) ? -oy * SP : oy * SP) + ((m & 1) ? -ox : ox);
              if constexpr (SP == kNarrowStride) {
                // narrow stride: fewer than 2 zero columns, so test each candidate
                const int rx = rxu - ox, ry = ryu - oy, sx = (m & 1) ? -1 : 1, sy = (m & 2) ? -1 : 1;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                  const int cx = move_dx(k) + 1, cy = move_dy(k) + 1;
                  if (cx - rx >= -r && cx - rx <= r && cy - ry >= -r && cy - ry <= r)
                    acc[k] += p[sy * cy * SP + sx * cx];
                }
              } else if (m == 0) {
                add_candidates<SP, 1, 1>(p, acc);
              } else if (m == 1) {
                add_candidates<SP, -1, 1>(p, acc);
              } else if (m == 2) {
                add_candidates<SP, 1, -1>(p, acc);
              } else {
                add_candidates<SP, -1, -1>(p, acc);
              }
            }
          });
    }
    if (fl) {
      // the decision again on the exact candidate field, by the exact path's
      // energy (pick_move) from what k_sur_decide stored for this slot
      const uint32_t info = fb_info[i];
      float f[9];
      int32_t dd[9];
      uint8_t oc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        int tx, ty;
        const bool ok = wrap_coord(q.x + move_dx(k), g.W, g.px, tx) &
                        wrap_coord(q.y + move_dy(k), g.H, g.py, ty);
        f[k] = ok ? Fs[(size_t)ty * g.W + tx] + acc[k] : 0.f;
        dd[k] = fb_dd[(size_t)i * 9 + k];
        oc[k] = (info >> k) & 1u ? 0 : 1;  // admissible iff its mask bit is set
      }
      const bool ok3[3] = {true, true, true};
      choice[rec_id[i]] = (uint8_t)pick_move<false>(f, dd, oc, ok3, ok3, (int)((info >> 9) & 15u),
                                                    (int)((info >> 16) & 255u), beta, own, dirdot,
                                                    nullptr);
    }
  }
}

// Every pedestrian listed for the exact candidate field (delta = +inf): per
// record slot i (bin order) the flag, and the guidance distances,
// admissible candidates, heading and goal k_sur_fallback decides from; no
// surrogate field is composed.  Walk-period idle pedestrians stay.
__global__ void k_list_all(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                           int nbins, Geo g, const int2* __restrict__ xy,
                           const uint8_t* __restrict__ heading, const uint8_t* __restrict__ goal,
                           const uint8_t* __restrict__ ocls, const int32_t* __restrict__ D,
                           uint8_t* __restrict__ choice, int32_t* __restrict__ nflag,
                           uint8_t* __restrict__ fb_flag, int32_t* __restrict__ fb_dd,
                           uint32_t* __restrict__ fb_info, WalkPeriods wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool listed = false;
  if (i < bin_start[nbins]) {
    const int p = rec_id[i];
    const long long t = wp.period ? wp.ctr->t : 0;
    if (wp.period && t % wp.period[p] != wp.phase[p]) {
      choice[p] = 0;  // not this pedestrian's tick (walk period): it stays
    } else {
      int cx[3], ry[3];
      bool okx[3], oky[3];
      candidate_coords(xy[p], g, cx, ry, okx, oky);
      int32_t dd[9];
      uint8_t oc[9];
      candidate_loads(g, ocls, D, cx, ry, dd, oc);
      uint32_t mask = 0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        fb_dd[(size_t)i * 9 + k] = dd[k];
        const int xi = move_dx(k) + 1, yi = move_dy(k) + 1;
        if (k == 0 || (okx[xi] && oky[yi] && dd[k] != kDWall && oc[k] == 0)) mask |= 1u << k;
      }
      fb_info[i] = mask | (uint32_t)heading[p] << 9 | (uint32_t)goal[p] << 16;
      listed = true;
    }
    fb_flag[i] = listed;
  }
  const unsigned nl = __popc(__ballot_sync(0xffffffffu, listed));
  if ((threadIdx.x & 31) == 0 && nl) atomicAdd(nflag, (int32_t)nl);
}

// running totals of listed and decided pedestrians over surrogate ticks
__global__ void k_count_fallbacks(const int32_t* __restrict__ nflag, const int32_t* __restrict__ nrec,
                                  unsigned long long* __restrict__ tot) {
  tot[0] += (unsigned long long)*nflag;
  tot[1] += (unsigned long long)*nrec;
}

// per pedestrian (bin order): the spread max - min of Fa - Fb over its
// admissible candidates, the part of the field error a decision margin has
// to absorb (an error common to all candidates cancels)
__global__ void k_sur_err(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                          int nbins, Geo g, const int2* __restrict__ xy,
                          const uint8_t* __restrict__ cell, const uint8_t* __restrict__ ocls,
                          const float* __restrict__ Fa, const float* __restrict__ Fb,
                          float* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= bin_start[nbins]) return;
  const int2 q = xy[rec_id[i]];
  float lo = __int_as_float(0x7f800000), hi = -lo;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    int tx, ty;
    const bool ok = wrap_coord(q.x + move_dx(k), g.W, g.px, tx) &
                    wrap_coord(q.y + move_dy(k), g.H, g.py, ty);
    if (ok && (k == 0 || (cell[(size_t)ty * g.W + tx] != kWall && ocls[(size_t)ty * g.opitch + tx] == 0))) {
      const size_t c = (size_t)ty * g.W + tx;
      const float d = Fa[c] - Fb[c];
      lo = fminf(lo, d);
      hi = fmaxf(hi, d);
    }
  }
  err[i] = hi - lo;
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

// ======================================================================
struct sfm_surrogate {
  sfm_surrogate_cfg cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  // parameters (internal layout), BF16-rounded copies, Adam state, gradients
  float *p = nullptr, *pq = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  bf16 *wt1 = nullptr, *wt2 = nullptr, *wt3 = nullptr, *wt4 = nullptr;  // for the tensor cores
  bf16 *wu2 = nullptr, *wu3 = nullptr;  // layers 2 and 3 in the tcgen05 operand layout
  int* umma_err = nullptr;              // set by a tcgen05 convolution that timed out
  bool use_umma = true;                 // layers 2 and 3 on tcgen05 (else mma.sync)
  int test_stop_copies = -1;            // test hook: the next layer-2 launch stops issuing copies
  int adam_t = 0;
  // activations for an image of (Hc + 2 kHalo) x (Wc + 2 kHalo) coarse cells
  int Hc = 0, Wc = 0;
  bf16 *X = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr;
  float *Y = nullptr, *T = nullptr, *dY = nullptr, *dA3 = nullptr, *dA2 = nullptr,
        *dA1 = nullptr, *part = nullptr;
  size_t part_cap = 0;
  // lattice-sized buffers
  size_t nsu = 0;
  float *Fnear = nullptr, *Fsur = nullptr;
  uint8_t* choice2 = nullptr;
  int choice_cap = 0;
  float* CTnear = nullptr;  // near-field class tables
  int near_r_built = -1;
  double* red = nullptr;
  unsigned long long* cnt = nullptr;
  // decisions with the exact fallback
  float delta = __builtin_inff();  // field error bound behind the margin test
  int32_t* fb_dd = nullptr;        // per listed slot: guidance distances D at the 9 candidates
  uint32_t* fb_info = nullptr;     // per listed slot: admissible mask | heading << 9 | goal << 16
  int32_t* flag_list = nullptr;    // slots (bin order) of the listed pedestrians
  int32_t* nflag = nullptr;
  uint8_t* fb_flag = nullptr;      // per slot: listed or not
  float* perr = nullptr;           // per-pedestrian candidate error (calibration)
  int fb_cap = 0;
  long long fallbacks = 0, decided = 0;  // totals over surrogate ticks (host copies)
  unsigned long long* fb_dev = nullptr;  // [0] listed, [1] decided, summed on the device
  std::vector<void*> allocs;
};

namespace {

sfm_status sfail(sfm_surrogate* s, sfm_status st, const std::string& msg) {
  if (s) s->err = msg;
  else set_create_error(msg);
  return st;
}

#define SCU(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return sfail(S, e_ == cudaErrorMemoryAllocation ? SFM_ENOMEM : SFM_ECUDA,       \
                   std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

template <class T>
sfm_status salloc(sfm_surrogate* S, T** p, size_t n) {
  void* q = nullptr;
  SCU(cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16));
  S->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return SFM_OK;
}

void sfree(sfm_surrogate* S, void* p) {
  if (!p) return;
  for (size_t i = 0; i < S->allocs.size(); ++i)
    if (S->allocs[i] == p) {
      S->allocs.erase(S->allocs.begin() + (long)i);
      break;
    }
  cudaFree(p);
}

#define STRY(x)                  \
  do {                           \
    sfm_status s_ = (x);         \
    if (s_ != SFM_OK) return s_; \
  } while (0)

// activation buffers for a padded input of (Hc + 2h) x (Wc + 2h) cells
sfm_status ensure_image(sfm_surrogate* S, int Hc, int Wc) {
  if (S->Hc == Hc && S->Wc == Wc && S->X) return SFM_OK;
  for (void* q : {(void*)S->X, (void*)S->A1, (void*)S->A2, (void*)S->A3, (void*)S->Y, (void*)S->T,
                  (void*)S->dY, (void*)S->dA3, (void*)S->dA2, (void*)S->dA1})
    sfree(S, q);
  const size_t p0 = (size_t)(Hc + 2 * kHalo) * (Wc + 2 * kHalo);
  const size_t p1 = (size_t)(Hc + 6) * (Wc + 6), p2 = (size_t)(Hc + 4) * (Wc + 4),
               p3 = (size_t)(Hc + 2) * (Wc + 2), p4 = (size_t)Hc * Wc;
  STRY(salloc(S, &S->X, p0 * 3));
  STRY(salloc(S, &S->A1, p1 * 32));
  STRY(salloc(S, &S->A2, p2 * 32));
  STRY(salloc(S, &S->A3, p3 * 32));
  STRY(salloc(S, &S->Y, p4));
  STRY(salloc(S, &S->T, p4));
  STRY(salloc(S, &S->dY, p4));
  STRY(salloc(S, &S->dA3, p3 * 32));
  STRY(salloc(S, &S->dA2, p2 * 32));
  STRY(salloc(S, &S->dA1, p1 * 32));
  S->Hc = Hc;
  S->Wc = Wc;
  return SFM_OK;
}

template <int CIN, int COUT, int K>
size_t dx_smem() {
  return ((size_t)K * K * CIN * COUT + (size_t)(kTile + K - 1) * (kTile + K - 1) * COUT) * 4;
}
template <int CIN, int COUT, int K>
size_t dw_smem() {
  return ((size_t)(kTile + K - 1) * (kTile + K - 1) * CIN + (size_t)kTile * kTile * COUT) * 4;
}

template <int CIN, int COUT, int K, bool RELU>
void conv_dx(const float* dA, const bf16* A, int Hout, int Wout, const float* W, float* dIn,
             cudaStream_t s) {
  const size_t sm = dx_smem<CIN, COUT, K>();
  cudaFuncSetAttribute(k_conv_dx<CIN, COUT, K, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  dim3 grid(cdiv(Wout + K - 1, kTile), cdiv(Hout + K - 1, kTile));
  k_conv_dx<CIN, COUT, K, RELU><<<grid, kTile * kTile, sm, s>>>(dA, A, Hout, Wout, W, dIn);
}

template <int CIN, int COUT, int K, bool RELU>
sfm_status conv_dw(sfm_surrogate* S, const bf16* in, const float* dA, const bf16* A, int Hout,
                   int Wout, float* gW, cudaStream_t s) {
  constexpr int NE = K * K * CIN * COUT + COUT;
  dim3 grid(cdiv(Wout, kTile), cdiv(Hout, kTile));
  const size_t nparts = (size_t)grid.x * grid.y;
  if (nparts * NE > S->part_cap) {
    sfree(S, S->part);
    STRY(salloc(S, &S->part, nparts * NE));
    S->part_cap = nparts * NE;
  }
  const size_t sm = dw_smem<CIN, COUT, K>();
  cudaFuncSetAttribute(k_conv_dw<CIN, COUT, K, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  k_conv_dw<CIN, COUT, K, RELU><<<grid, kTile * kTile, sm, s>>>(in, dA, A, Hout, Wout, S->part);
  // W block then b block are adjacent in the flat gradient (W at kOffW, b right after)
  k_reduce_parts<<<cdiv(NE, 256), 256, 0, s>>>(S->part, (int)nparts, NE, gW);
  return SFM_OK;
}

// 3x3 layer on the tensor cores: 32 -> 32 into out (BF16), or with yout
// the 32 -> 1 last layer into yout (FP32; wt packed by k_pack_w4)
void conv3_tc(const bf16* in, int Hin, int Win, const bf16* wt, const float* b, bf16* out,
              cudaStream_t s, float* yout = nullptr) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  // 32 -> 32: 4 m16 tiles a warp (16 rows a CTA, 3 CTAs an SM); 32 -> 1: 2
  // (8 rows, 4 CTAs)
  constexpr int MT4 = 4, MT1 = 2;
  if (yout) {
    const int ntiles = cdiv(Win - 2, kTcCols) * cdiv(Hin - 2, 4 * MT1);
    const int grid = std::max(1, std::min(ntiles, nsm * 4));
    cudaFuncSetAttribute(k_conv3_tc<1, MT1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv3_smem(MT1));
    k_conv3_tc<1, MT1><<<grid, 128, conv3_smem(MT1), s>>>(in, Hin, Win, wt, b, nullptr, yout);
  } else {
    const int ntiles = cdiv(Win - 2, kTcCols) * cdiv(Hin - 2, 4 * MT4);
    const int grid = std::max(1, std::min(ntiles, nsm * 3));
    cudaFuncSetAttribute(k_conv3_tc<4, MT4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv3_smem(MT4));
    k_conv3_tc<4, MT4><<<grid, 128, conv3_smem(MT4), s>>>(in, Hin, Win, wt, b, out, nullptr);
  }
}

// cuTensorMapEncodeTiled from the driver (the library links the runtime only)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3x3 32 -> 32 layer on tcgen05 (one warp-specialised CTA an SM); false when
// the tensor map cannot be made (the caller uses the mma.sync kernel)
bool conv3_umma(const bf16* in, int Hin, int Win, const bf16* wu, const float* b, bf16* out,
                int* err, cudaStream_t s, int stop_after) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  // the input [Hin][Win][32] BF16 seen as [row][channel group][pixel][8
  // channels] (strides: pixel 64 bytes, group 16, row Win x 64): one box of
  // 8 channels x 130 pixels x 4 groups x 1 row lands as the 4 planes of a row
  alignas(64) CUtensorMap tm;
  const cuuint64_t dims[3] = {32, (cuuint64_t)Win, (cuuint64_t)Hin};
  const cuuint64_t strides[2] = {64, (cuuint64_t)Win * 64};
  const cuuint32_t box[3] = {32, (cuuint32_t)kUmInPx, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(in), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const int ntiles = cdiv(Win - 2, kUmCols) * cdiv(Hin - 2, kUmRows);
  const int grid = std::max(1, std::min(ntiles, nsm));
  cudaFuncSetAttribute(k_conv3_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmSmem);
  k_conv3_umma<<<grid, kWsThreads, kUmSmem, s>>>(tm, Hin, Win, wu, b, out, err, stop_after);
  return true;
}

// forward of the whole padded image currently in S->X (all four layers on
// the tensor cores, FP32 accumulation; layers 2 and 3 on tcgen05 when
// use_umma is on)
void forward(sfm_surrogate* S, cudaStream_t s) {
  const int Hp = S->Hc + 2 * kHalo, Wp = S->Wc + 2 * kHalo;
  const float* q = S->pq;
  {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = cdiv(Wp - 4, kTcCols) * cdiv(Hp - 4, kTcRows);
    const int grid = std::max(1, std::min(ntiles, std::max(nsm, 1) * kC1CtasPerSm));
    k_conv1_tc<<<grid, 128, 0, s>>>(S->X, Hp, Wp, S->wt1, q + kOffB[0], S->A1);
  }
  const int stop = S->test_stop_copies;
  S->test_stop_copies = -1;
  if (!(S->use_umma && conv3_umma(S->A1, Hp - 4, Wp - 4, S->wu2, q + kOffB[1], S->A2, S->umma_err, s, stop)))
    conv3_tc(S->A1, Hp - 4, Wp - 4, S->wt2, q + kOffB[1], S->A2, s);
  if (!(S->use_umma && conv3_umma(S->A2, Hp - 6, Wp - 6, S->wu3, q + kOffB[2], S->A3, S->umma_err, s, -1)))
    conv3_tc(S->A2, Hp - 6, Wp - 6, S->wt3, q + kOffB[2], S->A3, s);
  conv3_tc(S->A3, Hp - 8, Wp - 8, S->wt4, q + kOffB[3], nullptr, s, S->Y);
}

// loss and gradients (into S->g) for the image in S->X and targets in S->T
sfm_status backward(sfm_surrogate* S, float* loss_out, cudaStream_t s) {
  const int Hc = S->Hc, Wc = S->Wc, n = Hc * Wc;
  const int nb = cdiv(n, 256);
  if ((size_t)nb > S->part_cap) {
    sfree(S, S->part);
    STRY(salloc(S, &S->part, (size_t)nb));
    S->part_cap = nb;
  }
  k_mse<<<nb, 256, 0, s>>>(S->Y, S->T, n, S->dY, S->part);
  std::vector<float> hp(nb);
  SCU(cudaMemcpyAsync(hp.data(), S->part, nb * sizeof(float), cudaMemcpyDeviceToHost, s));
  SCU(cudaStreamSynchronize(s));
  double L = 0.0;
  for (float x : hp) L += x;
  if (loss_out) *loss_out = (float)(0.5 * L / n);
  const float* q = S->pq;
  // layer 4 (linear), 3, 2, 1
  STRY((conv_dw<32, 1, 3, false>(S, S->A3, S->dY, nullptr, Hc, Wc, S->g + kOffW[3], s)));
  conv_dx<32, 1, 3, false>(S->dY, nullptr, Hc, Wc, q + kOffW[3], S->dA3, s);
  STRY((conv_dw<32, 32, 3, true>(S, S->A2, S->dA3, S->A3, Hc + 2, Wc + 2, S->g + kOffW[2], s)));
  conv_dx<32, 32, 3, true>(S->dA3, S->A3, Hc + 2, Wc + 2, q + kOffW[2], S->dA2, s);
  STRY((conv_dw<32, 32, 3, true>(S, S->A1, S->dA2, S->A2, Hc + 4, Wc + 4, S->g + kOffW[1], s)));
  conv_dx<32, 32, 3, true>(S->dA2, S->A2, Hc + 4, Wc + 4, q + kOffW[1], S->dA1, s);
  STRY((conv_dw<3, 32, 5, true>(S, S->X, S->dA1, S->A1, Hc + 6, Wc + 6, S->g + kOffW[0], s)));
  SCU(cudaGetLastError());
  return SFM_OK;
}

// layout conversions between the public order (per layer: W[o][c][ky][kx], b[o])
// and the internal one (W[ky][kx][c][o], b[o])
void to_internal(const float* pub, float* in) {
  const int dims[4][3] = {{3, 32, 5}, {32, 32, 3}, {32, 32, 3}, {32, 1, 3}};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    const int C = dims[l][0], O = dims[l][1], K = dims[l][2];
    for (int o = 0; o < O; ++o)
      for (int c = 0; c < C; ++c)
        for (int ky = 0; ky < K; ++ky)
          for (int kx = 0; kx < K; ++kx)
            in[kOffW[l] + ((ky * K + kx) * C + c) * O + o] = pub[off++];
    for (int o = 0; o < O; ++o) in[kOffB[l] + o] = pub[off++];
  }
}

void to_public(const float* in, float* pub) {
  const int dims[4][3] = {{3, 32, 5}, {32, 32, 3}, {32, 32, 3}, {32, 1, 3}};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    const int C = dims[l][0], O = dims[l][1], K = dims[l][2];
    for (int o = 0; o < O; ++o)
      for (int c = 0; c < C; ++c)
        for (int ky = 0; ky < K; ++ky)
          for (int kx = 0; kx < K; ++kx)
            pub[off++] = in[kOffW[l] + ((ky * K + kx) * C + c) * O + o];
    for (int o = 0; o < O; ++o) pub[off++] = in[kOffB[l] + o];
  }
}

sfm_status check_ctx(sfm_surrogate* S, sfm_ctx* ctx) {
  if (!ctx || ctx->batch) return sfail(S, SFM_EINVAL, "needs a single-lattice context");
  if (!ctx->placed) return sfail(S, SFM_ESTATE, "context has no pedestrians placed");
  if (ctx->bands > 1) return sfail(S, SFM_ESTATE, "context is banded (no full field)");
  const int s = S->cfg.coarsen;
  if (ctx->geo.W % s || ctx->geo.H % s)
    return sfail(S, SFM_EINVAL, "lattice sides must be multiples of the coarsening factor");
  if (ctx->geo.W / s < 1 || ctx->geo.H / s < 1) return sfail(S, SFM_EINVAL, "lattice too small");
  if (S->cfg.near_radius > ctx->geo.r)
    return sfail(S, SFM_EINVAL, "near radius larger than the field radius");
  if (!ctx->CT)
    return sfail(S, SFM_EINVAL, "field radius beyond the class-table gather (r > 50)");
  if (ctx->sized) return sfail(S, SFM_EINVAL, "multi-su pedestrians are not supported here");
  return SFM_OK;
}

// lattice buffers and near-field tables for ctx
sfm_status ensure_lattice(sfm_surrogate* S, sfm_ctx* ctx) {
  const size_t nsu = (size_t)ctx->geo.W * ctx->geo.H;
  if (nsu != S->nsu) {
    sfree(S, S->Fnear);
    sfree(S, S->Fsur);
    S->Fnear = S->Fsur = nullptr;
    STRY(salloc(S, &S->Fnear, nsu));
    STRY(salloc(S, &S->Fsur, nsu));
    S->nsu = nsu;
  }
  if (ctx->cap > S->choice_cap) {
    sfree(S, S->choice2);
    STRY(salloc(S, &S->choice2, (size_t)ctx->cap));
    S->choice_cap = ctx->cap;
  }
  if (ctx->cap > S->fb_cap) {
    sfree(S, S->fb_dd);
    sfree(S, S->fb_info);
    sfree(S, S->flag_list);
    sfree(S, S->fb_flag);
    sfree(S, S->perr);
    STRY(salloc(S, &S->fb_dd, (size_t)ctx->cap * 9));
    STRY(salloc(S, &S->fb_info, (size_t)ctx->cap));
    STRY(salloc(S, &S->flag_list, (size_t)ctx->cap));
    STRY(salloc(S, &S->fb_flag, (size_t)ctx->cap));
    STRY(salloc(S, &S->perr, (size_t)ctx->cap));
    S->fb_cap = ctx->cap;
  }
  const int rn = S->cfg.near_radius;
  if (S->near_r_built != rn || !S->CTnear) {
    sfree(S, S->CTnear);
    S->CTnear = nullptr;
    const size_t n = class_table_floats(rn);
    if (n) {
      STRY(salloc(S, &S->CTnear, n));
      launch_class_tables(rn, ctx->prm, S->CTnear, S->stream, S->cfg.taper_inner);
    }
    S->near_r_built = rn;
  }
  return SFM_OK;
}

// Fnear = Fs + pedestrian field within rn of the context's current state
// (bins must be current)
void near_field(sfm_surrogate* S, sfm_ctx* ctx) {
  Geo gn = ctx->geo;
  gn.r = S->cfg.near_radius;
  Tables tb = ctx->tables();
  tb.CT = S->CTnear;
  tb.CT3 = nullptr;  // the near part runs on the 16-row gathers and their tables
  launch_field(gn, ctx->bin_start, ctx->rec, tb, ctx->Fs, S->Fnear, 0, 0, gn.H, ctx->ctr,
               ctx->stream);
}

// the network's inputs for ctx's current state (bins must be current)
void coarse_inputs(sfm_surrogate* S, sfm_ctx* ctx) {
  const int Hp = S->Hc + 2 * kHalo, Wp = S->Wc + 2 * kHalo;
  if (kBin % S->cfg.coarsen == 0)
    k_coarse_in_rec<<<cdiv(Hp * Wp, 256), 256, 0, ctx->stream>>>(
        ctx->geo, ctx->bin_start, ctx->rec, S->cfg.coarsen, S->Hc, S->Wc, S->X);
  else
    k_coarse_in<<<cdiv(Hp * Wp, 256), 256, 0, ctx->stream>>>(ctx->geo, ctx->ocls, S->cfg.coarsen,
                                                              S->Hc, S->Wc, S->X);
}

FarPart far_part(const sfm_surrogate* S) {
  FarPart far;
  far.Y = S->Y;
  far.s = S->cfg.coarsen;
  far.Hc = S->Hc;
  far.Wc = S->Wc;
  far.scale = S->cfg.target_scale;
  far.inv_s = 1.f / (float)S->cfg.coarsen;
  return far;
}

// The network's output Y (the far part on the coarse grid) for ctx's current
// state.  Bins must be current.
void surrogate_far(sfm_surrogate* S, sfm_ctx* ctx) {
  coarse_inputs(S, ctx);
  forward(S, ctx->stream);
}

// Fsur = (Fs + pedestrian field within rn) + scale * bilinear(Y) over the
// whole lattice: the network runs first and the near-field gather adds its
// interpolated output in its epilogue, so the lattice is written once.  Bins
// must be current.
void surrogate_field(sfm_surrogate* S, sfm_ctx* ctx) {
  surrogate_far(S, ctx);
  Geo gn = ctx->geo;
  gn.r = S->cfg.near_radius;
  Tables tb = ctx->tables();
  tb.CT = S->CTnear;
  tb.CT3 = nullptr;  // the near part runs on the 16-row gathers and their tables
  launch_field(gn, ctx->bin_start, ctx->rec, tb, ctx->Fs, S->Fsur, 0, 0, gn.H, ctx->ctr,
               ctx->stream, far_part(S));
}

// Decisions of ctx's live pedestrians into `choice` on the surrogate field,
// then the exact fallback for the pedestrians within the margin.  cand: the
// surrogate field is composed at each pedestrian's candidates from Y (which
// surrogate_far must have computed) and the near tables; else it is read
// from Fsur (surrogate_field).  ref/raw_flips as k_sur_decide.
// The exact candidate field and decision of every listed pedestrian
// (k_sur_fallback on the context's class tables).
void surrogate_fallback(sfm_surrogate* S, sfm_ctx* ctx, uint8_t* choice);

void surrogate_decide(sfm_surrogate* S, sfm_ctx* ctx, uint8_t* choice, const uint8_t* ref,
                      unsigned long long* raw_flips, bool cand) {
  const Geo& g = ctx->geo;
  const Tables tb = ctx->tables();
  const int nbins = g.nbx * g.nby;
  cudaStream_t st = ctx->stream;
  cudaMemsetAsync(S->nflag, 0, sizeof(int32_t), st);
  if (ctx->n <= 0) return;
  if (cand && std::isinf(S->delta) && !ref) {
    // delta = +inf: every pedestrian falls back, so neither the network's
    // output nor the surrogate composition is needed -- the exact tick with
    // the field computed at the candidates only
    k_list_all<<<cdiv(ctx->n, 256), 256, 0, st>>>(ctx->rec_id, ctx->bin_start, nbins, g, ctx->xy,
                                                  ctx->heading, ctx->goal, ctx->ocls, ctx->D, choice,
                                                  S->nflag, S->fb_flag, S->fb_dd, S->fb_info,
                                                  ctx->walk());
    surrogate_fallback(S, ctx, choice);
    return;
  }
  NearPart np;
  np.CT = S->CTnear;
  np.rn = S->cfg.near_radius;
  np.SP = class_table_stride(np.rn);
  np.TS = (2 * np.rn + 1 + 2 * kFieldPadRows) * np.SP;
  auto dk = cand ? k_sur_decide<true> : k_sur_decide<false>;
  dk<<<cdiv(ctx->n, 256), 256, 0, st>>>(
      ctx->rec_id, ctx->bin_start, nbins, g, ctx->xy, ctx->heading, ctx->goal, ctx->cell, ctx->ocls,
      ctx->D, S->Fsur, ctx->rec, ctx->Fs, np, far_part(S), ctx->prm.beta, tb.own, tb.dirdot,
      S->delta, choice, S->flag_list, S->nflag, S->fb_flag, S->fb_dd, S->fb_info, ref, raw_flips,
      ctx->walk());
  surrogate_fallback(S, ctx, choice);
}

void surrogate_fallback(sfm_surrogate* S, sfm_ctx* ctx, uint8_t* choice) {
  const Geo& g = ctx->geo;
  const Tables tb = ctx->tables();
  const int nbins = g.nbx * g.nby;
  cudaStream_t st = ctx->stream;
  const int SP = class_table_stride(g.r);
  const int TS = (2 * g.r + 1 + 2 * kFieldPadRows) * SP;
  const size_t smem = (kTableGuard + 4 * (size_t)TS) * sizeof(float) +
                      (size_t)kFbThreads / 32 * 32 * sizeof(int2);
  void (*fb)(const uint8_t*, const int32_t*, int, Geo, const int2*, const int32_t*, const uint32_t*,
             const float*, int, const float*, const int32_t*, const uint32_t*, float, const float*,
             const float*, uint8_t*);
  switch (SP) {
    case 34: fb = k_sur_fallback<34>; break;
    case 50: fb = k_sur_fallback<50>; break;
    case 66: fb = k_sur_fallback<66>; break;
    case 82: fb = k_sur_fallback<82>; break;
    case 98: fb = k_sur_fallback<98>; break;
    case 114: fb = k_sur_fallback<114>; break;
    default: fb = k_sur_fallback<kNarrowStride>; break;
  }
  cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  fb<<<nsm > 0 ? nsm : 1, kFbThreads, smem, st>>>(
      S->fb_flag, ctx->rec_id, nbins, g, ctx->xy, ctx->bin_start, ctx->rec, ctx->CT, TS, ctx->Fs,
      S->fb_dd, S->fb_info, ctx->prm.beta, tb.own, tb.dirdot, choice);
}

void round_params(sfm_surrogate* S) {
  k_round_bf16<<<cdiv(kNParams, 256), 256, 0, S->stream>>>(S->p, S->pq, kNParams);
  k_pack_w1<<<cdiv(5 * 32 * 16, 256), 256, 0, S->stream>>>(S->pq + kOffW[0], S->wt1);
  k_pack_w3<<<cdiv(9 * 32 * 32, 256), 256, 0, S->stream>>>(S->pq + kOffW[1], S->wt2);
  k_pack_w3<<<cdiv(9 * 32 * 32, 256), 256, 0, S->stream>>>(S->pq + kOffW[2], S->wt3);
  k_pack_w4<<<cdiv(9 * 8 * 32, 256), 256, 0, S->stream>>>(S->pq + kOffW[3], S->wt4);
  k_pack_wum<<<cdiv(9 * 32 * 32, 256), 256, 0, S->stream>>>(S->pq + kOffW[1], S->wu2);
  k_pack_wum<<<cdiv(9 * 32 * 32, 256), 256, 0, S->stream>>>(S->pq + kOffW[2], S->wu3);
}

// Status of the tcgen05 convolutions (synchronising): a timeout switches
// layers 2 and 3 to the mma.sync kernel for good and is reported once.
sfm_status umma_check(sfm_surrogate* S) {
  int h = 0;
  SCU(cudaMemcpyAsync(&h, S->umma_err, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
  SCU(cudaStreamSynchronize(S->stream));
  if (h) {
    S->use_umma = false;
    SCU(cudaMemsetAsync(S->umma_err, 0, sizeof(int), S->stream));
    return sfail(S, SFM_ETIMEOUT, "a tcgen05 convolution timed out; layers 2-3 now run on mma.sync");
  }
  return SFM_OK;
}

// channel-planar FP32 image [3][Hin][Win] (host) into S->X (channel-last BF16)
sfm_status upload_image(sfm_surrogate* S, int Hin, int Win, const float* X) {
  std::vector<bf16> hx((size_t)Hin * Win * 3);
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < Hin * Win; ++i) hx[(size_t)i * 3 + c] = __float2bfloat16(X[(size_t)c * Hin * Win + i]);
  SCU(cudaMemcpyAsync(S->X, hx.data(), hx.size() * sizeof(bf16), cudaMemcpyHostToDevice, S->stream));
  SCU(cudaStreamSynchronize(S->stream));
  return SFM_OK;
}

}  // namespace

extern "C" {

int32_t sfm_surrogate_nparams(void) { return kNParams; }

sfm_status sfm_surrogate_forward(sfm_surrogate* S, int32_t Hin, int32_t Win, const float* X,
                                 float* Y, int32_t tcgen05) {
  if (!S || !X || !Y) return SFM_EINVAL;
  if (Hin <= 2 * kHalo || Win <= 2 * kHalo) return sfail(S, SFM_EINVAL, "image too small");
  const int Hc = Hin - 2 * kHalo, Wc = Win - 2 * kHalo;
  STRY(ensure_image(S, Hc, Wc));
  STRY(upload_image(S, Hin, Win, X));
  const bool saved = S->use_umma;
  S->use_umma = saved && tcgen05 != 0;
  forward(S, S->stream);
  S->use_umma = saved;
  SCU(cudaMemcpyAsync(Y, S->Y, (size_t)Hc * Wc * sizeof(float), cudaMemcpyDeviceToHost, S->stream));
  SCU(cudaStreamSynchronize(S->stream));
  SCU(cudaGetLastError());
  return umma_check(S);
}

sfm_status sfm_surrogate_create(const sfm_surrogate_cfg* cfg, void* stream, sfm_surrogate** out) {
  if (out) *out = nullptr;
  if (!cfg || !out) return sfail(nullptr, SFM_EINVAL, "NULL argument");
  if (cfg->coarsen < 1 || cfg->coarsen > 64 || cfg->near_radius < 0 ||
      cfg->near_radius > kMaxTableRadius || !(cfg->target_scale > 0.f) ||
      !(cfg->taper_inner >= 0.f))
    return sfail(nullptr, SFM_EINVAL, "bad surrogate configuration");
  sfm_surrogate* S = new sfm_surrogate;
  S->cfg = *cfg;
  S->stream = static_cast<cudaStream_t>(stream);
  auto bail = [&](sfm_status st) {
    set_create_error(S->err);
    sfm_surrogate_destroy(S);
    return st;
  };
  sfm_status st;
  if ((st = salloc(S, &S->p, kNParams)) != SFM_OK || (st = salloc(S, &S->pq, kNParams)) != SFM_OK ||
      (st = salloc(S, &S->m, kNParams)) != SFM_OK || (st = salloc(S, &S->v, kNParams)) != SFM_OK ||
      (st = salloc(S, &S->g, kNParams)) != SFM_OK || (st = salloc(S, &S->red, 2 * 1024)) != SFM_OK ||
      (st = salloc(S, &S->wt1, 32 * kC1K)) != SFM_OK ||
      (st = salloc(S, &S->wt2, 9 * 32 * 32)) != SFM_OK ||
      (st = salloc(S, &S->fb_dev, 2)) != SFM_OK || (st = salloc(S, &S->nflag, 1)) != SFM_OK ||
      (st = salloc(S, &S->wt3, 9 * 32 * 32)) != SFM_OK ||
      (st = salloc(S, &S->wt4, 9 * 8 * 32)) != SFM_OK ||
      (st = salloc(S, &S->wu2, 9 * 32 * 32)) != SFM_OK ||
      (st = salloc(S, &S->wu3, 9 * 32 * 32)) != SFM_OK ||
      (st = salloc(S, &S->umma_err, 1)) != SFM_OK ||
      (st = salloc(S, &S->cnt, 2)) != SFM_OK)
    return bail(st);
  cudaMemsetAsync(S->p, 0, kNParams * sizeof(float), S->stream);
  cudaMemsetAsync(S->m, 0, kNParams * sizeof(float), S->stream);
  cudaMemsetAsync(S->v, 0, kNParams * sizeof(float), S->stream);
  cudaMemsetAsync(S->fb_dev, 0, 2 * sizeof(unsigned long long), S->stream);
  cudaMemsetAsync(S->umma_err, 0, sizeof(int), S->stream);
  round_params(S);
  if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
    S->err = "surrogate set-up failed";
    return bail(SFM_ECUDA);
  }
  *out = S;
  return SFM_OK;
}

void sfm_surrogate_destroy(sfm_surrogate* S) {
  if (!S) return;
  cudaStreamSynchronize(S->stream);
  for (void* p : S->allocs) cudaFree(p);
  delete S;
}

const char* sfm_surrogate_last_error(const sfm_surrogate* S) { return S ? S->err.c_str() : ""; }

sfm_status sfm_surrogate_set_params(sfm_surrogate* S, const float* params) {
  if (!S || !params) return SFM_EINVAL;
  std::vector<float> in(kNParams);
  to_internal(params, in.data());
  SCU(cudaMemcpyAsync(S->p, in.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice, S->stream));
  SCU(cudaMemsetAsync(S->m, 0, kNParams * sizeof(float), S->stream));
  SCU(cudaMemsetAsync(S->v, 0, kNParams * sizeof(float), S->stream));
  S->adam_t = 0;
  round_params(S);
  SCU(cudaStreamSynchronize(S->stream));
  return SFM_OK;
}

sfm_status sfm_surrogate_get_params(sfm_surrogate* S, float* params) {
  if (!S || !params) return SFM_EINVAL;
  std::vector<float> in(kNParams);
  SCU(cudaMemcpyAsync(in.data(), S->p, kNParams * sizeof(float), cudaMemcpyDeviceToHost, S->stream));
  SCU(cudaStreamSynchronize(S->stream));
  to_public(in.data(), params);
  return SFM_OK;
}

sfm_status sfm_surrogate_grad(sfm_surrogate* S, int32_t Hin, int32_t Win, const float* X,
                              const float* T, float* loss, float* grads) {
  if (!S || !X || !T) return SFM_EINVAL;
  if (Hin <= 2 * kHalo || Win <= 2 * kHalo) return sfail(S, SFM_EINVAL, "image too small");
  const int Hc = Hin - 2 * kHalo, Wc = Win - 2 * kHalo;
  STRY(ensure_image(S, Hc, Wc));
  STRY(upload_image(S, Hin, Win, X));
  SCU(cudaMemcpyAsync(S->T, T, (size_t)Hc * Wc * sizeof(float), cudaMemcpyHostToDevice, S->stream));
  forward(S, S->stream);
  STRY(backward(S, loss, S->stream));
  if (grads) {
    std::vector<float> in(kNParams);
    SCU(cudaMemcpyAsync(in.data(), S->g, kNParams * sizeof(float), cudaMemcpyDeviceToHost, S->stream));
    SCU(cudaStreamSynchronize(S->stream));
    to_public(in.data(), grads);
  }
  SCU(cudaStreamSynchronize(S->stream));
  return umma_check(S);
}

sfm_status sfm_surrogate_train(sfm_surrogate* S, sfm_ctx* ctx, int32_t iters, float* loss_curve) {
  if (!S) return SFM_EINVAL;
  STRY(check_ctx(S, ctx));
  STRY(ensure_lattice(S, ctx));
  const int s = S->cfg.coarsen;
  STRY(ensure_image(S, ctx->geo.H / s, ctx->geo.W / s));
  cudaStream_t st = ctx->stream;
  if (st != S->stream) {
    SCU(cudaStreamSynchronize(S->stream));
  }
  S->stream = st;
  const float b1 = S->cfg.beta1, b2 = S->cfg.beta2;
  for (int it = 0; it < iters; ++it) {
    // exact field of the current state, its near part, inputs and targets
    ctx_run_bins(ctx);
    ctx_field_rows(ctx, ctx->F, 0, ctx->geo.H, 0, false);
    near_field(S, ctx);
    coarse_inputs(S, ctx);
    k_targets<<<cdiv(S->Hc * S->Wc, 256), 256, 0, st>>>(ctx->F, S->Fnear, ctx->geo.W, s, S->Hc,
                                                        S->Wc, 1.f / S->cfg.target_scale, S->T);
    forward(S, st);
    float L = 0.f;
    STRY(backward(S, &L, st));
    if (loss_curve) loss_curve[it] = L;
    ++S->adam_t;
    const float c1 = 1.f - powf(b1, (float)S->adam_t), c2 = 1.f - powf(b2, (float)S->adam_t);
    k_adam<<<cdiv(kNParams, 256), 256, 0, st>>>(S->p, S->m, S->v, S->g, kNParams, S->cfg.lr, b1, b2,
                                                S->cfg.eps, c1, c2);
    round_params(S);
    // the crowd moves on: a tick of the exact path gives the next sample
    const sfm_status ss = sfm_step(ctx, 1);
    if (ss != SFM_OK) return sfail(S, ss, std::string("training tick: ") + ctx->err);
  }
  SCU(cudaStreamSynchronize(st));
  SCU(cudaGetLastError());
  return umma_check(S);
}

// set-up shared by the calls below
sfm_status surrogate_ready(sfm_surrogate* S, sfm_ctx* ctx) {
  if (!S) return SFM_EINVAL;
  STRY(check_ctx(S, ctx));
  STRY(ensure_lattice(S, ctx));
  const int s = S->cfg.coarsen;
  STRY(ensure_image(S, ctx->geo.H / s, ctx->geo.W / s));
  S->stream = ctx->stream;
  return SFM_OK;
}

sfm_status sfm_surrogate_field(sfm_surrogate* S, sfm_ctx* ctx, float* out, int32_t on_device) {
  if (!S || !out) return SFM_EINVAL;
  STRY(surrogate_ready(S, ctx));
  ctx_run_bins(ctx);
  surrogate_field(S, ctx);
  SCU(cudaMemcpyAsync(out, S->Fsur, S->nsu * sizeof(float),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  SCU(cudaStreamSynchronize(ctx->stream));
  SCU(cudaGetLastError());
  return umma_check(S);
}

sfm_status sfm_surrogate_set_delta(sfm_surrogate* S, float delta) {
  if (!S || !(delta >= 0.f)) return SFM_EINVAL;
  S->delta = delta;
  return SFM_OK;
}

sfm_status sfm_surrogate_calibrate(sfm_surrogate* S, sfm_ctx* ctx, double quantile,
                                   float* delta_out) {
  if (!(quantile >= 0.0 && quantile <= 1.0)) return sfail(S, SFM_EINVAL, "quantile outside [0, 1]");
  STRY(surrogate_ready(S, ctx));
  cudaStream_t st = ctx->stream;
  const Geo& g = ctx->geo;
  const int nbins = g.nbx * g.nby;
  ctx_run_bins(ctx);
  ctx_field_rows(ctx, ctx->F, 0, g.H, 0, false);
  surrogate_field(S, ctx);
  if (ctx->n > 0)
    k_sur_err<<<cdiv(ctx->n, 256), 256, 0, st>>>(ctx->rec_id, ctx->bin_start, nbins, g, ctx->xy,
                                                 ctx->cell, ctx->ocls, S->Fsur, ctx->F, S->perr);
  int nrec = 0;
  SCU(cudaMemcpyAsync(&nrec, ctx->bin_start + nbins, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCU(cudaStreamSynchronize(st));
  std::vector<float> e((size_t)nrec);
  if (nrec > 0) {
    SCU(cudaMemcpyAsync(e.data(), S->perr, (size_t)nrec * sizeof(float), cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
  }
  SCU(cudaGetLastError());
  float d = 0.f;
  if (nrec > 0) {
    size_t k = (size_t)(quantile * (double)(nrec - 1) + 0.5);
    if (k >= (size_t)nrec) k = (size_t)nrec - 1;
    std::nth_element(e.begin(), e.begin() + (long)k, e.end());
    d = e[k];
  }
  S->delta = d;
  if (delta_out) *delta_out = d;
  return umma_check(S);
}

sfm_status sfm_surrogate_step(sfm_surrogate* S, sfm_ctx* ctx, int32_t nsteps) {
  if (nsteps < 0) return sfail(S, SFM_EINVAL, "nsteps < 0");
  STRY(surrogate_ready(S, ctx));
  cudaStream_t st = ctx->stream;
  const Geo& g = ctx->geo;
  for (int i = 0; i < nsteps; ++i) {
    launch_clear_dead(ctx->n, ctx->alive, ctx->choice, ctx->won, st);
    ctx_run_bins(ctx);
    if (!std::isinf(S->delta)) surrogate_far(S, ctx);  // delta = +inf: no network (exact tick)
    surrogate_decide(S, ctx, ctx->choice, nullptr, nullptr, true);
    k_count_fallbacks<<<1, 1, 0, st>>>(S->nflag, ctx->bin_start + g.nbx * g.nby, S->fb_dev);
    launch_vote(ctx->n, ctx->rec_id, ctx->bin_start, ctx->xy, ctx->choice, ctx->occ, g,
                ctx->prm.seed, ctx->ctr, ctx->won, st, Sizes(), ctx->ids());
    launch_commit(ctx->n, ctx->rec_id, ctx->bin_start, ctx->xy, ctx->alive, ctx->heading,
                  ctx->choice, ctx->won, ctx->cell, ctx->occ, ctx->ocls, g, ctx->ctr, st);
    ++ctx->t;
  }
  SCU(cudaGetLastError());
  return SFM_OK;
}

sfm_status sfm_surrogate_test_stop_copies(sfm_surrogate* S, int32_t after) {
  if (!S || after < 0) return SFM_EINVAL;
  S->test_stop_copies = after;
  return SFM_OK;
}

sfm_status sfm_surrogate_counts(sfm_surrogate* S, int64_t* fallbacks, int64_t* decided) {
  if (!S) return SFM_EINVAL;
  unsigned long long h[2] = {0, 0};
  SCU(cudaMemcpyAsync(h, S->fb_dev, sizeof(h), cudaMemcpyDeviceToHost, S->stream));
  SCU(cudaStreamSynchronize(S->stream));
  if (fallbacks) *fallbacks = (int64_t)h[0];
  if (decided) *decided = (int64_t)h[1];
  return umma_check(S);
}

sfm_status sfm_surrogate_eval(sfm_surrogate* S, sfm_ctx* ctx, sfm_surrogate_report* rep) {
  if (!rep) return SFM_EINVAL;
  STRY(surrogate_ready(S, ctx));
  cudaStream_t st = ctx->stream;
  const Geo& g = ctx->geo;
  const Tables tb = ctx->tables();
  const int nbins = g.nbx * g.nby;
  cudaEvent_t e0, e1, e2, e3;
  SCU(cudaEventCreate(&e0));
  SCU(cudaEventCreate(&e1));
  SCU(cudaEventCreate(&e2));
  SCU(cudaEventCreate(&e3));
  // exact: bins, field, decisions (into ctx->choice)
  SCU(cudaEventRecord(e0, st));
  ctx_run_bins(ctx);
  ctx_field_rows(ctx, ctx->F, 0, g.H, 0, false);
  launch_decide(ctx->n, ctx->rec_id, ctx->bin_start, 0, nbins, ctx->xy, ctx->heading, ctx->goal,
                ctx->cell, ctx->ocls, ctx->D, ctx->F, 0, -1, -1, 0, 0, g.H, g, ctx->prm.beta, tb,
                ctx->choice, st, ctx->walk());
  SCU(cudaEventRecord(e1, st));
  // surrogate tick's decisions: bins, network, decisions on the surrogate
  // field at the candidates with the fallback (into choice2)
  SCU(cudaMemsetAsync(S->cnt, 0, 2 * sizeof(unsigned long long), st));
  SCU(cudaEventRecord(e1, st));
  ctx_run_bins(ctx);
  surrogate_far(S, ctx);
  surrogate_decide(S, ctx, S->choice2, ctx->choice, S->cnt + 1, true);
  SCU(cudaEventRecord(e2, st));
  // the surrogate field over the whole lattice (network and lattice pass)
  surrogate_field(S, ctx);
  SCU(cudaEventRecord(e3, st));
  if (ctx->n > 0)
    k_diff_choices<<<cdiv(ctx->n, 256), 256, 0, st>>>(ctx->rec_id, ctx->bin_start, nbins,
                                                      ctx->choice, S->choice2, S->cnt);
  k_field_err<<<1024, 256, 0, st>>>(S->Fsur, ctx->F, ctx->Fs, S->nsu, S->red);
  std::vector<double> red(2048);
  unsigned long long cnt[2] = {0, 0};
  int nrec = 0, nfl = 0;
  SCU(cudaMemcpyAsync(red.data(), S->red, red.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SCU(cudaMemcpyAsync(cnt, S->cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
  SCU(cudaMemcpyAsync(&nrec, ctx->bin_start + nbins, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCU(cudaMemcpyAsync(&nfl, S->nflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCU(cudaStreamSynchronize(st));
  SCU(cudaGetLastError());
  double a = 0.0, b = 0.0;
  for (int i = 0; i < 1024; ++i) {
    a += red[2 * i];
    b += red[2 * i + 1];
  }
  float t_ex = 0.f, t_su = 0.f, t_sf = 0.f;
  cudaEventElapsedTime(&t_ex, e0, e1);
  cudaEventElapsedTime(&t_su, e1, e2);
  cudaEventElapsedTime(&t_sf, e2, e3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  cudaEventDestroy(e3);
  const double nd = nrec > 0 ? (double)nrec : 1.0;
  rep->field_rel_err = b > 0 ? a / b : 0.0;
  rep->flip_rate = (double)cnt[0] / nd;
  rep->flip_rate_raw = (double)cnt[1] / nd;
  rep->fallback_rate = (double)nfl / nd;
  rep->ms_surrogate = t_su;
  rep->ms_exact = t_ex;
  rep->ms_surrogate_field = t_sf;
  rep->delta = S->delta;
  rep->decided = nrec;
  return umma_check(S);
}

}  // extern "C"
