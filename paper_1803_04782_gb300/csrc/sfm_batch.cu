// sfm_batch.cu -- a batch of independent lattices stepped together: one
// persistent (cooperative) kernel per tick runs every stage of the tick for
// every lattice, separated by grid-wide barriers with bounded waits.  The
// field stage walks a work list of (lattice, footprint chunk) items sorted by
// cost; the footprint height of each radius class is chosen by timing
// (sfm_batch_autotune).  A tick launch is captured once in a CUDA graph and
// replayed.  Each lattice evolves exactly as it would in its own context.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "sfm_ctx.h"
#include "sfm_gather.cuh"

using namespace sfm;

namespace sfm {

// Geometry and offsets of one lattice of a batch.
struct BatchScene {
  Geo g;
  long long su_off;    // first su in the concatenated lattice arrays
  long long ocls_off;  // first byte in the concatenated class grids
  long long ct_off;    // first float of the lattice's class tables
  unsigned long long seed;
  int bin_off;  // first bin
  int grp_off;  // first bin group (4 bins x 32 rows)
  int ped_off;  // first pedestrian
  int n;        // pedestrians
  int sp;       // class-table row stride
  int ts;       // floats per class table
  float beta;
  int pad;
};

// A field work item: footprints [f0, f0 + 32) (one per warp) of lattice
// scene; shape 0 = 16 x 16 su footprints, 1 = 32 x 16.
struct BatchChunk {
  int scene, f0, shape, pad;
};

struct BatchArgs {
  const BatchScene* scenes;
  const uint16_t* grp_scene;
  const BatchChunk* chunks;
  const uint16_t* ped_scene;
  const uint8_t* cell;
  const float* Fs;
  float* F;
  const int32_t* D;
  int32_t* occ;
  uint8_t* ocls;
  const float* own;
  const float* dirdot;
  const float* CT;
  int32_t* bin_count;
  int32_t* bin_start;
  int32_t* scan_tmp;
  uint32_t* rec;
  int32_t* rec_id;
  int2* xy;
  uint8_t* heading;
  const uint8_t* goal;
  uint8_t* alive;
  uint8_t* choice;
  uint8_t* won;
  Counters* ctr;
  unsigned int* bar;
  int* work;
  int n;             // pedestrians (all lattices)
  int total_groups;  // bin groups (all lattices)
  int total_bins;
  int total_chunks;
  int expect_blocks;  // CTAs the grid barrier waits for
  int field_only;     // 1: bins + field only (no decisions, nobody moves)
  int max_ts;         // class-table capacity of shared memory (floats per table)
};

struct BatchState {
  int nscenes = 0;
  std::vector<BatchScene> hs;
  BatchScene* scenes = nullptr;
  uint16_t* grp_scene = nullptr;
  uint16_t* ped_scene = nullptr;
  BatchChunk* chunks = nullptr;
  int total_chunks = 0, chunk_cap = 0;
  int total_groups = 0, total_bins = 0;
  long long total_ocls = 0;
  float *own = nullptr, *dirdot = nullptr, *CT = nullptr;
  unsigned int* bar = nullptr;
  int* work = nullptr;
  int max_ts = 0;
  int shape_of_sp[kNumStrideClasses] = {};  // footprint shape per class-table stride
  int missing = 0;  // test hook: CTAs the barrier expects beyond those launched
  int grid = 0;
  std::vector<int> order;  // lattices by decreasing field cost
  cudaGraphExec_t graph = nullptr;
  int graph_field_only = -1;
};

}  // namespace sfm

namespace {

constexpr int kBatchThreads = 1024;
constexpr long long kSpinLimit = 1ll << 23;  // ~1 s of 100 ns naps

// Grid-wide barrier for a co-resident (cooperative) grid, reusable across
// barriers and launches: every CTA adds 1 except CTA 0, which adds
// 2^31 - (expect - 1); the high bit flips exactly when all have arrived.  The
// wait gives up after kSpinLimit naps and flags kErrTimeout.
__device__ bool grid_sync(unsigned int* bar, int expect, Counters* ctr) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned int inc = (blockIdx.x == 0) ? (0x80000000u - (unsigned)(expect - 1)) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, inc);
    long long it = 0;
    while (((old ^ *(volatile unsigned int*)bar) & 0x80000000u) == 0u) {
      if (++it > kSpinLimit) {
        atomicOr(&ctr->err, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

__device__ int block_scan_excl(int v, int* sWarp, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sWarp[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? sWarp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < nw) sWarp[lane] = s;
  }
  __syncthreads();
  total = sWarp[nw - 1];
  const int excl = inc - v + (w > 0 ? sWarp[w - 1] : 0);
  __syncthreads();
  return excl;
}

// footprint counts per row of a lattice for each shape
__host__ __device__ inline int shape_w(int shape) { return shape ? 32 : 16; }
__host__ __device__ inline int shape_nf(const Geo& g, int shape) {
  return ((g.W + shape_w(shape) - 1) / shape_w(shape)) * ((g.H + 15) / 16);
}

template <int SP>
__device__ __forceinline__ void batch_footprint(const BatchArgs& a, const BatchScene& sc,
                                                const float* sT, int2* scr, int lane, int f,
                                                int shape) {
  const Geo& g = sc.g;
  const int fw = shape_w(shape);
  const int nfx = (g.W + fw - 1) / fw;
  const int x0 = (f % nfx) * fw, y0 = (f / nfx) * 16;
  if (shape == 0) {
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    gather_footprint16<SP>(g, a.bin_start + sc.bin_off, a.rec, sT, sc.ts, scr, lane, x0, y0, acc);
    const int x = x0 + (lane & 15), yl = y0 + (lane >> 4) * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int y = yl + j;
      if (x < g.W && y < g.H) {
        const size_t c = (size_t)sc.su_off + (size_t)y * g.W + x;
        a.F[c] = a.Fs[c] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
      }
    }
  } else {
    float2 acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
    gather_footprint32<SP>(g, a.bin_start + sc.bin_off, a.rec, sT, sc.ts, scr, lane, x0, y0, acc);
    const int x = x0 + lane;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int y = y0 + j;
      if (x < g.W && y < g.H) {
        const size_t c = (size_t)sc.su_off + (size_t)y * g.W + x;
        a.F[c] = a.Fs[c] + ((j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
      }
    }
  }
}

__device__ __forceinline__ void batch_footprint_sp(const BatchArgs& a, const BatchScene& sc,
                                                   const float* sT, int2* scr, int lane, int f,
                                                   int shape) {
  switch (sc.sp) {
    case 34: batch_footprint<34>(a, sc, sT, scr, lane, f, shape); break;
    case 50: batch_footprint<50>(a, sc, sT, scr, lane, f, shape); break;
    case 66: batch_footprint<66>(a, sc, sT, scr, lane, f, shape); break;
    case 82: batch_footprint<82>(a, sc, sT, scr, lane, f, shape); break;
    case 98: batch_footprint<98>(a, sc, sT, scr, lane, f, shape); break;
    case 114: batch_footprint<114>(a, sc, sT, scr, lane, f, shape); break;
    default: batch_footprint<kNarrowStride>(a, sc, sT, scr, lane, f, shape); break;
  }
}

constexpr int kScanChunk = kBatchThreads * 4;

__global__ void __launch_bounds__(kBatchThreads, 1) k_tick_batch(BatchArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* sT = sm + kTableGuard;  // class tables after a zero guard
  __shared__ int sWarp[32];
  __shared__ int s_chunk, s_loaded;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + tid;
  const int gwarp = gtid >> 5, nwarps = nthreads >> 5;
  int2* scr = reinterpret_cast<int2*>(sT + 4 * a.max_ts) + warp * 32;
  // tick counter of this launch, read before the first barrier: thread 0 of
  // CTA 0 advances it after the last one
  const long long t = a.ctr->t;

  // S0: decisions of pedestrians that are not alive read as "stay"; reset the
  // field work counter
  for (int p = gtid; p < a.n; p += nthreads)
    if (!a.alive[p]) {
      a.choice[p] = 0;
      a.won[p] = 0;
    }
  if (gtid == 0) *a.work = 0;
  // S1: bins -- counts, exclusive scan over all lattices' bins, fill
  for (int w = gwarp; w < a.total_groups; w += nwarps) {
    const BatchScene& sc = a.scenes[a.grp_scene[w]];
    const int lg = w - sc.grp_off, ngx = (sc.g.nbx + 3) >> 2;
    bin_count_group(sc.g, a.ocls + sc.ocls_off, a.bin_count + sc.bin_off, lg % ngx, lg / ngx, lane);
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  const int nsc = (a.total_bins + kScanChunk - 1) / kScanChunk;
  for (int c = blockIdx.x; c < nsc; c += gridDim.x) {
    const int i0 = c * kScanChunk + tid * 4;
    int s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k < a.total_bins) s += a.bin_count[i0 + k];
    int total;
    block_scan_excl(s, sWarp, total);
    if (tid == 0) a.scan_tmp[c] = total;
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  if (blockIdx.x == 0) {
    int carry = 0;
    for (int base = 0; base < nsc; base += kBatchThreads) {
      const int i = base + tid;
      const int v = i < nsc ? a.scan_tmp[i] : 0;
      int total;
      const int e = block_scan_excl(v, sWarp, total);
      if (i < nsc) a.scan_tmp[i] = e + carry;
      carry += total;
    }
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  for (int c = blockIdx.x; c < nsc; c += gridDim.x) {
    const int i0 = c * kScanChunk + tid * 4;
    int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = (i0 + k < a.total_bins) ? a.bin_count[i0 + k] : 0;
      s += v[k];
    }
    int total;
    int e = block_scan_excl(s, sWarp, total) + a.scan_tmp[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i0 + k < a.total_bins) a.bin_start[i0 + k] = e;
      e += v[k];
    }
    if (c == nsc - 1 && tid == kBatchThreads - 1) a.bin_start[a.total_bins] = e;
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  for (int w = gwarp; w < a.total_groups; w += nwarps) {
    const BatchScene& sc = a.scenes[a.grp_scene[w]];
    const int lg = w - sc.grp_off, ngx = (sc.g.nbx + 3) >> 2;
    bin_fill_group(sc.g, a.ocls + sc.ocls_off, a.occ + sc.su_off, a.bin_start + sc.bin_off, a.rec,
                   a.rec_id, lg % ngx, lg / ngx, lane);
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;

  // S2: field -- chunks of 32 footprints (one per warp) from the cost-sorted
  // work list; a lattice's class tables are loaded when the CTA switches to it
  if (tid == 0) s_loaded = -1;
  if (tid < kTableGuard) sm[tid] = 0.f;
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(a.work, 1);
    __syncthreads();
    const int c = s_chunk;
    if (c >= a.total_chunks) break;
    const BatchChunk ch = a.chunks[c];
    const BatchScene& sc = a.scenes[ch.scene];
    if (s_loaded != ch.scene) {
      const float2* src = reinterpret_cast<const float2*>(a.CT + sc.ct_off);
      float2* dst = reinterpret_cast<float2*>(sT);
      copy_to_shared<4>(dst, src, 2 * sc.ts);  // 4*ts floats
      __syncthreads();
      if (tid == 0) s_loaded = ch.scene;
    }
    const int f = ch.f0 + warp;
    if (f < shape_nf(sc.g, ch.shape)) batch_footprint_sp(a, sc, sT, scr, lane, f, ch.shape);
    __syncthreads();
  }
  if (a.field_only) return;
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;

  // S3-S5: decisions, vote, commit over every live pedestrian in bin order
  const int nrec = a.bin_start[a.total_bins];
  for (int i = gtid; i < nrec; i += nthreads) {
    const int p = a.rec_id[i];
    const BatchScene& sc = a.scenes[a.ped_scene[p]];
    a.choice[p] = decide_one(p, sc.g, a.xy, a.heading, a.goal, a.cell + sc.su_off,
                             a.ocls + sc.ocls_off, a.D + sc.su_off, a.F + sc.su_off, 0, -1, -1,
                             0, 0, sc.g.H, sc.beta, a.own + 81 * a.ped_scene[p],
                             a.dirdot + 81 * a.ped_scene[p]);
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  for (int i = gtid; i < nrec; i += nthreads) {
    const int p = a.rec_id[i];
    const BatchScene& sc = a.scenes[a.ped_scene[p]];
    const int regs = vote_one(p, sc.ped_off, sc.g, a.xy, a.choice, a.occ + sc.su_off, sc.seed, t,
                              a.won);
    if (regs > 2) atomicMax(&a.ctr->max_registrants, regs);
    if (regs > 8) atomicOr(&a.ctr->err, kErrEnroll);
  }
  if (!grid_sync(a.bar, a.expect_blocks, a.ctr)) return;
  for (int i0 = blockIdx.x * blockDim.x; i0 < nrec; i0 += nthreads) {
    const int i = i0 + tid;
    bool moved = false, left = false;
    if (i < nrec) {
      const int p = a.rec_id[i];
      const BatchScene& sc = a.scenes[a.ped_scene[p]];
      commit_one(p, sc.g, a.xy, a.alive, a.heading, a.choice, a.won, a.cell + sc.su_off,
                 a.occ + sc.su_off, a.ocls + sc.ocls_off, moved, left);
    }
    const unsigned nm = __popc(__ballot_sync(0xffffffffu, moved));
    const unsigned nl = __popc(__ballot_sync(0xffffffffu, left));
    if (lane == 0) {
      if (nm) atomicAdd(&a.ctr->moved, (unsigned long long)nm);
      if (nl) atomicAdd(&a.ctr->exited, (unsigned long long)nl);
    }
  }
  if (gtid == 0) a.ctr->t = t + 1;
}

// per-lattice placement into the concatenated grids (pedestrian indices global)
__global__ void k_batch_clear(int n, const int2* __restrict__ xy, const uint8_t* __restrict__ alive,
                              const uint16_t* __restrict__ ped_scene,
                              const BatchScene* __restrict__ scenes, int32_t* __restrict__ occ,
                              uint8_t* __restrict__ ocls) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive[p]) return;
  const BatchScene& sc = scenes[ped_scene[p]];
  const int2 q = xy[p];
  occ[sc.su_off + (size_t)q.y * sc.g.W + q.x] = -1;
  ocls[sc.ocls_off + (size_t)q.y * sc.g.opitch + q.x] = 0;
}

__global__ void k_batch_scatter(int n, const int2* __restrict__ xy,
                                const uint8_t* __restrict__ heading,
                                const uint8_t* __restrict__ goal, const uint8_t* __restrict__ alive,
                                const uint16_t* __restrict__ ped_scene,
                                const BatchScene* __restrict__ scenes,
                                const uint8_t* __restrict__ cell, int32_t* __restrict__ occ,
                                uint8_t* __restrict__ ocls, Counters* ctr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (heading[p] > 8 || goal[p] > 8) atomicOr(&ctr->err, kErrPlaceRange);
  if (!alive[p]) return;
  const BatchScene& sc = scenes[ped_scene[p]];
  const int2 q = xy[p];
  if (q.x < 0 || q.x >= sc.g.W || q.y < 0 || q.y >= sc.g.H) {
    atomicOr(&ctr->err, kErrPlaceRange);
    return;
  }
  const size_t c = sc.su_off + (size_t)q.y * sc.g.W + q.x;
  if (cell[c] != kFree) atomicOr(&ctr->err, kErrPlaceConflict);
  if (atomicCAS(&occ[c], -1, p) != -1) {
    atomicOr(&ctr->err, kErrPlaceConflict);
    return;
  }
  ocls[sc.ocls_off + (size_t)q.y * sc.g.opitch + q.x] = (uint8_t)(1 + (heading[p] > 8 ? 0 : heading[p]));
}

sfm_status bfail(sfm_ctx* c, sfm_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    set_create_error(msg);
  return st;
}

#define BCU(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail(ctx, e_ == cudaErrorMemoryAllocation ? SFM_ENOMEM : SFM_ECUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

template <class T>
sfm_status balloc(sfm_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  const cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess)
    return bfail(ctx, SFM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  ctx->allocs.push_back(q);
  ctx->device_bytes += (int64_t)bytes;
  *p = static_cast<T*>(q);
  return SFM_OK;
}

#define BTRY(x)                  \
  do {                           \
    sfm_status s_ = (x);         \
    if (s_ != SFM_OK) return s_; \
  } while (0)


// Work list of the field stage: lattices by decreasing cost per footprint,
// each cut into chunks of 32 footprints of its radius class's height.  When
// only_sp > 0, only lattices of that row stride are listed.
void build_chunks(BatchState* B, std::vector<BatchChunk>& out, int only_sp) {
  out.clear();
  for (int s : B->order) {
    const BatchScene& sc = B->hs[s];
    if (only_sp > 0 && sc.sp != only_sp) continue;
    const int shape = B->shape_of_sp[class_of_stride(sc.sp)];
    const int nf = shape_nf(sc.g, shape);
    for (int f0 = 0; f0 < nf; f0 += 32) out.push_back(BatchChunk{s, f0, shape, 0});
  }
}

sfm_status upload_chunks(sfm_ctx* ctx, const std::vector<BatchChunk>& v) {
  BatchState* B = ctx->batch;
  if ((int)v.size() > B->chunk_cap) {
    return bfail(ctx, SFM_ESTATE, "work list larger than its buffer");
  }
  if (!v.empty())
    BCU(cudaMemcpyAsync(B->chunks, v.data(), v.size() * sizeof(BatchChunk), cudaMemcpyHostToDevice,
                        ctx->stream));
  BCU(cudaStreamSynchronize(ctx->stream));
  B->total_chunks = (int)v.size();
  return SFM_OK;
}

BatchArgs make_args(sfm_ctx* ctx, int field_only) {
  BatchState* B = ctx->batch;
  BatchArgs a{};
  a.scenes = B->scenes;
  a.grp_scene = B->grp_scene;
  a.chunks = B->chunks;
  a.ped_scene = B->ped_scene;
  a.cell = ctx->cell;
  a.Fs = ctx->Fs;
  a.F = ctx->F;
  a.D = ctx->D;
  a.occ = ctx->occ;
  a.ocls = ctx->ocls;
  a.own = B->own;
  a.dirdot = B->dirdot;
  a.CT = B->CT;
  a.bin_count = ctx->bin_count;
  a.bin_start = ctx->bin_start;
  a.scan_tmp = ctx->scan_tmp;
  a.rec = ctx->rec;
  a.rec_id = ctx->rec_id;
  a.xy = ctx->xy;
  a.heading = ctx->heading;
  a.goal = ctx->goal;
  a.alive = ctx->alive;
  a.choice = ctx->choice;
  a.won = ctx->won;
  a.ctr = ctx->ctr;
  a.bar = B->bar;
  a.work = B->work;
  a.n = ctx->n;
  a.total_groups = B->total_groups;
  a.total_bins = B->total_bins;
  a.total_chunks = B->total_chunks;
  a.expect_blocks = B->grid + B->missing;
  a.field_only = field_only;
  a.max_ts = B->max_ts;
  return a;
}

size_t batch_smem(const BatchState* B) {
  return (size_t)(kTableGuard + 4 * B->max_ts) * sizeof(float) +
         (size_t)kBatchThreads / 32 * 32 * sizeof(int2);
}

cudaError_t launch_tick(sfm_ctx* ctx, int field_only, cudaStream_t s) {
  BatchState* B = ctx->batch;
  BatchArgs a = make_args(ctx, field_only);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(B->grid);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = batch_smem(B);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tick_batch, a);
}

sfm_status check_batch(sfm_ctx* ctx) {
  BCU(cudaStreamSynchronize(ctx->stream));
  Counters h;
  BCU(cudaMemcpy(&h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.err & kErrTimeout) {
    // the barrier word is left mid-count: clear it and the flag so the
    // context can tick again
    h.err &= ~kErrTimeout;
    BCU(cudaMemcpy(ctx->ctr, &h, sizeof(h), cudaMemcpyHostToDevice));
    BCU(cudaMemset(ctx->batch->bar, 0, sizeof(unsigned int)));
    return bfail(ctx, SFM_ETIMEOUT, "a grid barrier of the batched tick timed out");
  }
  return SFM_OK;
}

}  // namespace

namespace sfm {

void batch_destroy(sfm_ctx* ctx) {
  if (!ctx || !ctx->batch) return;
  if (ctx->batch->graph) cudaGraphExecDestroy(ctx->batch->graph);
  delete ctx->batch;
  ctx->batch = nullptr;
}

sfm_status batch_tick(sfm_ctx* ctx, int nsteps, int field_only) {
  BatchState* B = ctx->batch;
  if (!ctx->placed) return bfail(ctx, SFM_ESTATE, "sfm_step before a successful sfm_batch_place");
  if (B->missing) {
    // test hook: one direct launch whose barrier waits for CTAs that do not
    // exist; the bounded wait gives up and the tick reports SFM_ETIMEOUT
    BCU(launch_tick(ctx, field_only, ctx->stream));
    ctx->launches += 1;
    B->missing = 0;
    return check_batch(ctx);
  }
  if (!B->graph || B->graph_field_only != field_only) {
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    cudaStream_t cs;
    BCU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = launch_tick(ctx, field_only, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      B->graph = nullptr;
      cudaGetLastError();
      return bfail(ctx, SFM_ECUDA, std::string("tick graph: ") + cudaGetErrorString(e));
    }
    B->graph_field_only = field_only;
  }
  for (int i = 0; i < nsteps; ++i) {
    if (ctx->timing) {
      cudaEvent_t a0, b0;
      cudaEventCreate(&a0);
      cudaEventCreate(&b0);
      cudaEventRecord(a0, ctx->stream);
      BCU(cudaGraphLaunch(B->graph, ctx->stream));
      cudaEventRecord(b0, ctx->stream);
      ctx->recs.push_back({field_only ? SFM_STAGE_FIELD : SFM_STAGE_STEP, a0, b0});
    } else {
      BCU(cudaGraphLaunch(B->graph, ctx->stream));
    }
    ctx->launches += 1;
    if (!field_only) ++ctx->t;
  }
  if (ctx->timing && !field_only) ctx->timed_ticks += nsteps;
  return SFM_OK;
}

sfm_status batch_sync(sfm_ctx* ctx) { return check_batch(ctx); }

}  // namespace sfm

extern "C" {

sfm_status sfm_batch_create(int32_t nscenes, const sfm_lattice* lats, const uint8_t* const* cells,
                            const sfm_params* prms, void* stream, sfm_ctx** out) {
  sfm_ctx* ctx = nullptr;
  if (out) *out = nullptr;
  if (nscenes <= 0 || nscenes > 65535 || !lats || !cells || !prms || !out)
    return bfail(nullptr, SFM_EINVAL, "bad batch arguments (1..65535 lattices)");
  for (int s = 0; s < nscenes; ++s) {
    const sfm_lattice& L = lats[s];
    const sfm_params& p = prms[s];
    if (!cells[s] || L.W < 3 || L.H < 3 || (int64_t)L.W * L.H > ((int64_t)1 << 31))
      return bfail(nullptr, SFM_EINVAL, "lattice " + std::to_string(s) + ": bad size or cells");
    if (p.r < 0 || p.r > kMaxTableRadius)
      return bfail(nullptr, SFM_EINVAL, "lattice " + std::to_string(s) + ": radius outside [0, 50]");
    if ((L.periodic_x && L.W < 2 * p.r + 1) || (L.periodic_y && L.H < 2 * p.r + 1))
      return bfail(nullptr, SFM_EINVAL,
                   "lattice " + std::to_string(s) + ": a periodic extent must be >= 2r+1");
    if (p.bin != 0 && p.bin != kBin)
      return bfail(nullptr, SFM_EINVAL, "lattice " + std::to_string(s) + ": bin side must be 0 or 32");
  }
  ctx = new sfm_ctx;
  ctx->batch = new BatchState;
  BatchState* B = ctx->batch;
  B->nscenes = nscenes;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->lat = lats[0];
  ctx->prm = prms[0];
  ctx->prm.bin = kBin;
  auto bail = [&](sfm_status st) {
    set_create_error(ctx->err);
    sfm_destroy(ctx);
    return st;
  };
  // offsets
  long long su = 0, oc = 0, ct = 0;
  int bins = 0, grps = 0;
  B->hs.resize(nscenes);
  for (int s = 0; s < nscenes; ++s) {
    BatchScene& sc = B->hs[s];
    memset(&sc, 0, sizeof(sc));
    Geo& g = sc.g;
    g.W = lats[s].W;
    g.H = lats[s].H;
    g.px = lats[s].periodic_x ? 1 : 0;
    g.py = lats[s].periodic_y ? 1 : 0;
    g.r = prms[s].r;
    g.nbx = (g.W + kBin - 1) / kBin;
    g.nby = (g.H + kBin - 1) / kBin;
    g.opitch = (g.W + 127) / 128 * 128;
    sc.su_off = su;
    sc.ocls_off = oc;
    sc.bin_off = bins;
    sc.grp_off = grps;
    sc.sp = class_table_stride(g.r);
    sc.ts = (int)(class_table_floats(g.r) / 4);
    sc.ct_off = ct;
    sc.seed = prms[s].seed;
    sc.beta = prms[s].beta;
    su += (long long)g.W * g.H;
    oc += (long long)g.opitch * g.H;
    ct += 4LL * sc.ts;
    bins += g.nbx * g.nby;
    grps += ((g.nbx + 3) / 4) * g.nby;
    B->max_ts = std::max(B->max_ts, sc.ts);
  }
  if (su > ((long long)1 << 31) || bins > (1 << 30)) {
    ctx->err = "batch larger than 2^31 su";
    return bail(SFM_EINVAL);
  }
  B->total_bins = bins;
  B->total_groups = grps;
  B->total_ocls = oc;
  sfm_status st;
#define BALLOC(p, n)                               \
  if ((st = balloc(ctx, &(p), (n))) != SFM_OK) \
    return bail(st);
  BALLOC(ctx->cell, (size_t)su);
  BALLOC(ctx->Fs, (size_t)su);
  BALLOC(ctx->F, (size_t)su);
  BALLOC(ctx->D, (size_t)su);
  BALLOC(ctx->occ, (size_t)su);
  BALLOC(ctx->ocls, (size_t)oc);
  BALLOC(B->own, (size_t)81 * nscenes);
  BALLOC(B->dirdot, (size_t)81 * nscenes);
  BALLOC(B->CT, (size_t)ct);
  BALLOC(ctx->bin_count, (size_t)bins);
  BALLOC(ctx->bin_start, (size_t)bins + 1);
  BALLOC(ctx->scan_tmp, (size_t)bins / kScanChunk + 64);
  BALLOC(B->scenes, (size_t)nscenes);
  BALLOC(B->grp_scene, (size_t)grps);
  BALLOC(B->bar, 1);
  BALLOC(B->work, 1);
  BALLOC(ctx->ctr, 1);
  // field work list capacity: chunks of 32 footprints of the smaller shape
  {
    long long cap = 0;
    for (const BatchScene& sc : B->hs) cap += ((long long)shape_nf(sc.g, 0) + 31) / 32;
    B->chunk_cap = (int)cap;
    BALLOC(B->chunks, (size_t)cap);
  }
#undef BALLOC
  ctx->nsu_total = su;
  cudaStream_t s = ctx->stream;
  // per-lattice tables, static field and guidance (set-up, lattice by lattice)
  int maxS = 1;
  for (const BatchScene& sc : B->hs) maxS = std::max(maxS, 2 * sc.g.r + 1);
  float *T0, *TX, *TY, *KO, *KE;
  float2* hvec;
  if ((st = balloc(ctx, &T0, (size_t)maxS * maxS)) != SFM_OK ||
      (st = balloc(ctx, &TX, (size_t)maxS * maxS)) != SFM_OK ||
      (st = balloc(ctx, &TY, (size_t)maxS * maxS)) != SFM_OK ||
      (st = balloc(ctx, &KO, (size_t)maxS * maxS)) != SFM_OK ||
      (st = balloc(ctx, &KE, (size_t)maxS * maxS)) != SFM_OK || (st = balloc(ctx, &hvec, 9)) != SFM_OK)
    return bail(st);
  std::vector<uint16_t> gs(grps);
  for (int sidx = 0; sidx < nscenes; ++sidx) {
    const BatchScene& sc = B->hs[sidx];
    const size_t nsu = (size_t)sc.g.W * sc.g.H;
    if (cudaMemcpyAsync(ctx->cell + sc.su_off, cells[sidx], nsu, cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
      ctx->err = "copy cells";
      return bail(SFM_ECUDA);
    }
    launch_tables(sc.g.r, prms[sidx], T0, TX, TY, KO, KE, B->own + 81 * sidx,
                  B->dirdot + 81 * sidx, hvec, s);
    launch_class_tables(sc.g.r, prms[sidx], B->CT + sc.ct_off, s);
    Tables tb{};
    tb.KO = KO;
    tb.KE = KE;
    launch_static_field(sc.g, ctx->cell + sc.su_off, tb, ctx->Fs + sc.su_off, s);
    st = compute_guidance(sc.g, ctx->cell + sc.su_off, ctx->D + sc.su_off, s, &ctx->err);
    if (st != SFM_OK) return bail(st);
    const int ng = ((sc.g.nbx + 3) / 4) * sc.g.nby;
    for (int k = 0; k < ng; ++k) gs[sc.grp_off + k] = (uint16_t)sidx;
  }
  cudaMemsetAsync(ctx->occ, 0xff, (size_t)su * sizeof(int32_t), s);
  cudaMemsetAsync(ctx->ocls, 0, (size_t)oc, s);
  cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), s);
  cudaMemsetAsync(B->bar, 0, sizeof(unsigned int), s);
  cudaMemcpyAsync(B->grp_scene, gs.data(), gs.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(B->scenes, B->hs.data(), B->hs.size() * sizeof(BatchScene), cudaMemcpyHostToDevice,
                  s);
  // persistent grid: one 1024-thread CTA per SM, if the shared memory allows
  {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = batch_smem(B);
    cudaFuncSetAttribute(k_tick_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tick_batch, kBatchThreads, smem);
    if (per_sm < 1) {
      ctx->err = "batched tick does not fit an SM";
      return bail(SFM_ECUDA);
    }
    B->grid = sms * per_sm;
  }
  B->order.resize(nscenes);
  std::iota(B->order.begin(), B->order.end(), 0);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("batch set-up: ") + cudaGetErrorString(e);
    return bail(SFM_ECUDA);
  }
  *out = ctx;
  return SFM_OK;
}

sfm_status sfm_batch_place(sfm_ctx* ctx, const int32_t* counts, const int32_t* xy,
                           const uint8_t* heading, const uint8_t* goal, const uint8_t* alive,
                           int32_t on_device) {
  if (!ctx || !ctx->batch || !counts) return SFM_EINVAL;
  BatchState* B = ctx->batch;
  cudaStream_t s = ctx->stream;
  int64_t n64 = 0;
  for (int i = 0; i < B->nscenes; ++i) {
    if (counts[i] < 0) return bfail(ctx, SFM_EINVAL, "negative pedestrian count");
    n64 += counts[i];
  }
  if (n64 > (1 << 30)) return bfail(ctx, SFM_EINVAL, "more than 2^30 pedestrians");
  const int n = (int)n64;
  if (n > 0 && !xy) return bfail(ctx, SFM_EINVAL, "NULL positions");
  if (ctx->placed && ctx->n > 0) {
    k_batch_clear<<<(ctx->n + 255) / 256, 256, 0, s>>>(ctx->n, ctx->xy, ctx->alive, B->ped_scene,
                                                       B->scenes, ctx->occ, ctx->ocls);
    ctx->launches += 1;
  }
  BCU(cudaStreamSynchronize(s));
  if (n > ctx->cap || ctx->cap == 0) {
    for (void* p : {(void*)ctx->xy, (void*)ctx->heading, (void*)ctx->goal, (void*)ctx->alive,
                    (void*)ctx->choice, (void*)ctx->won, (void*)ctx->rec, (void*)ctx->rec_id,
                    (void*)B->ped_scene}) {
      if (!p) continue;
      for (size_t i = 0; i < ctx->allocs.size(); ++i)
        if (ctx->allocs[i] == p) {
          ctx->allocs.erase(ctx->allocs.begin() + (long)i);
          break;
        }
      cudaFree(p);
    }
    const size_t cap = n > 0 ? (size_t)n : 1;
    BTRY(balloc(ctx, &ctx->xy, cap));
    BTRY(balloc(ctx, &ctx->heading, cap));
    BTRY(balloc(ctx, &ctx->goal, cap));
    BTRY(balloc(ctx, &ctx->alive, cap));
    BTRY(balloc(ctx, &ctx->choice, cap));
    BTRY(balloc(ctx, &ctx->won, cap));
    BTRY(balloc(ctx, &ctx->rec, cap));
    BTRY(balloc(ctx, &ctx->rec_id, cap));
    BTRY(balloc(ctx, &B->ped_scene, cap));
    ctx->cap = (int)cap;
    if (B->graph) {
      cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
  }
  ctx->placed = false;
  ctx->n = n;
  std::vector<uint16_t> ps((size_t)n);
  {
    int64_t off = 0;
    for (int i = 0; i < B->nscenes; ++i) {
      B->hs[i].ped_off = (int)off;
      B->hs[i].n = counts[i];
      for (int k = 0; k < counts[i]; ++k) ps[(size_t)off + k] = (uint16_t)i;
      off += counts[i];
    }
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0) {
    BCU(cudaMemcpyAsync(B->ped_scene, ps.data(), ps.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                        s));
    BCU(cudaMemcpyAsync(ctx->xy, xy, (size_t)n * sizeof(int2), kind, s));
    if (heading) BCU(cudaMemcpyAsync(ctx->heading, heading, n, kind, s));
    else BCU(cudaMemsetAsync(ctx->heading, 0, n, s));
    if (goal) BCU(cudaMemcpyAsync(ctx->goal, goal, n, kind, s));
    else BCU(cudaMemsetAsync(ctx->goal, 0, n, s));
    if (alive) BCU(cudaMemcpyAsync(ctx->alive, alive, n, kind, s));
    else BCU(cudaMemsetAsync(ctx->alive, 1, n, s));
    BCU(cudaMemsetAsync(ctx->choice, 0, n, s));
    BCU(cudaMemsetAsync(ctx->won, 0, n, s));
  }
  BCU(cudaMemcpyAsync(B->scenes, B->hs.data(), B->hs.size() * sizeof(BatchScene),
                      cudaMemcpyHostToDevice, s));
  BCU(cudaStreamSynchronize(s));
  Counters h;
  BCU(cudaMemcpy(&h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost));
  h.moved = 0;
  h.exited = 0;
  h.max_registrants = 0;
  h.err = 0;
  BCU(cudaMemcpy(ctx->ctr, &h, sizeof(h), cudaMemcpyHostToDevice));
  if (n > 0) {
    k_batch_scatter<<<(n + 255) / 256, 256, 0, s>>>(n, ctx->xy, ctx->heading, ctx->goal, ctx->alive,
                                                    B->ped_scene, B->scenes, ctx->cell, ctx->occ,
                                                    ctx->ocls, ctx->ctr);
    ctx->launches += 1;
  }
  BCU(cudaStreamSynchronize(s));
  BCU(cudaGetLastError());
  BCU(cudaMemcpy(&h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.err) {
    const uint32_t flags = h.err;
    cudaMemsetAsync(ctx->occ, 0xff, (size_t)ctx->nsu_total * sizeof(int32_t), s);
    cudaMemsetAsync(ctx->ocls, 0, (size_t)B->total_ocls, s);
    h.err = 0;
    cudaMemcpyAsync(ctx->ctr, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return bfail(ctx, (flags & kErrPlaceRange) ? SFM_EINVAL : SFM_ECONFLICT,
                 "placement rejected: overlapping pedestrians, a pedestrian on a WALL/EXIT su, "
                 "off-lattice positions or classes > 8");
  }
  // work list: lattices by decreasing field cost per footprint (crowd density
  // times window area)
  {
    std::vector<double> cost(B->nscenes);
    for (int i = 0; i < B->nscenes; ++i) {
      const BatchScene& sc = B->hs[i];
      const double area = (double)sc.g.W * sc.g.H;
      cost[i] = (sc.n / area) * (2.0 * sc.g.r + 1) * (2.0 * sc.g.r + 1);
    }
    std::stable_sort(B->order.begin(), B->order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<BatchChunk> v;
    build_chunks(B, v, 0);
    BTRY(upload_chunks(ctx, v));
  }
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  ctx->placed = true;
  return SFM_OK;
}

sfm_status sfm_batch_offsets(const sfm_ctx* ctx, int64_t* su_off, int64_t* ped_off) {
  if (!ctx || !ctx->batch) return SFM_EINVAL;
  const BatchState* B = ctx->batch;
  for (int i = 0; i <= B->nscenes; ++i) {
    const bool end = i == B->nscenes;
    if (su_off) su_off[i] = end ? ctx->nsu_total : B->hs[i].su_off;
    if (ped_off) ped_off[i] = end ? ctx->n : B->hs[i].ped_off;
  }
  return SFM_OK;
}

sfm_status sfm_batch_autotune(sfm_ctx* ctx, int32_t* shape_per_class) {
  if (!ctx || !ctx->batch) return SFM_EINVAL;
  if (!ctx->placed) return bfail(ctx, SFM_ESTATE, "autotune needs placed pedestrians");
  BatchState* B = ctx->batch;
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  BCU(cudaEventCreate(&e0));
  BCU(cudaEventCreate(&e1));
  for (int ci = 0; ci < kNumStrideClasses; ++ci) {
    const int sp = stride_of_class(ci);
    bool present = false;
    for (const BatchScene& sc : B->hs) present |= sc.sp == sp;
    if (!present) continue;
    float best = 1e30f;
    int best_shape = 0;
    for (int shape : {0, 1}) {
      B->shape_of_sp[ci] = shape;
      std::vector<BatchChunk> v;
      build_chunks(B, v, sp);
      BTRY(upload_chunks(ctx, v));
      float tot = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        BCU(cudaEventRecord(e0, s));
        BCU(launch_tick(ctx, 1, s));
        BCU(cudaEventRecord(e1, s));
        BCU(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;  // first run warms up
        ctx->launches += 1;
      }
      BTRY(check_batch(ctx));
      if (tot < best) {
        best = tot;
        best_shape = shape;
      }
    }
    B->shape_of_sp[ci] = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<BatchChunk> v;
  build_chunks(B, v, 0);
  BTRY(upload_chunks(ctx, v));
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  if (shape_per_class)
    for (int ci = 0; ci < kNumStrideClasses; ++ci) shape_per_class[ci] = B->shape_of_sp[ci];
  return SFM_OK;
}

sfm_status sfm_batch_test_missing_ctas(sfm_ctx* ctx, int32_t missing) {
  if (!ctx || !ctx->batch || missing < 0) return SFM_EINVAL;
  ctx->batch->missing = missing;
  return SFM_OK;
}

}  // extern "C"
