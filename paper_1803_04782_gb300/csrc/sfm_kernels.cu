// sfm_kernels.cu -- sm_103a kernels of one tick of the discrete social-field
// pedestrian model (Alg. 1 of the paper: k-5 field superposition, k-2 decision,
// k-3 vote, k-4 commit), re-designed as gathers so that no step needs atomics
// on the field (Sec. 3.1 s-1 avoids them with fan-out caches instead).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sfm_gather.cuh"
#include "sfm_internal.h"

namespace sfm {

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ tables
// Kernel values are evaluated once per scene in FP64 and rounded to FP32.
__global__ void k_tables(int r, double kP, double aP, double gamma, double kO, double aO,
                         double kE, double aE, float* T0, float* TX, float* TY, float* KO,
                         float* KE, float* own, float* dirdot, float2* hvec) {
  const int S = 2 * r + 1, n = S * S;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int dx = i % S - r, dy = i / S - r;
    if (dx == 0 && dy == 0) {
      T0[i] = TX[i] = TY[i] = KO[i] = KE[i] = 0.f;
    } else {
      const double d = sqrt((double)(dx * dx + dy * dy));
      const double base = kP * pow(d, aP);
      T0[i] = (float)base;
      TX[i] = (float)(base * gamma * dx / d);
      TY[i] = (float)(base * gamma * dy / d);
      KO[i] = (float)(kO * pow(d, aO));
      KE[i] = (float)(kE * pow(d, aE));
    }
  }
  if (i < 81) {
    const int h = i / 9, k = i % 9;
    double hx = 0.0, hy = 0.0;
    if (h > 0) {
      const double nh = sqrt((double)(c_dx[h] * c_dx[h] + c_dy[h] * c_dy[h]));
      hx = c_dx[h] / nh;
      hy = c_dy[h] / nh;
    }
    double o = 0.0;
    if (k > 0 && r >= 1) {
      const double d = sqrt((double)(c_dx[k] * c_dx[k] + c_dy[k] * c_dy[k]));
      o = kP * pow(d, aP) * (1.0 + gamma * (hx * c_dx[k] + hy * c_dy[k]) / d);
    }
    own[i] = (float)o;
    dirdot[i] = (float)(c_dx[k] * hx + c_dy[k] * hy);
    if (k == 0) hvec[h] = make_float2((float)hx, (float)hy);
  }
}

void launch_tables(int r, const sfm_params& p, float* T0, float* TX, float* TY, float* KO,
                   float* KE, float* own, float* dirdot, float2* hvec, cudaStream_t s) {
  const int n = (2 * r + 1) * (2 * r + 1);
  const int total = n > 81 ? n : 81;
  k_tables<<<cdiv(total, 256), 256, 0, s>>>(r, p.kP, p.aP, p.gamma, p.kO, p.aO, p.kE, p.aE, T0,
                                            TX, TY, KO, KE, own, dirdot, hvec);
}

// ------------------------------------------------------------ static field
// F_static(c) = sum over WALL / EXIT su o within the window of K_O / K_E(c - o),
// a dense window gather over a shared-memory copy of the cell tile and its
// r-halo; compensated (Kahan) FP32 accumulation because up to (2r+1)^2 - 1
// terms enter one su.  Computed once per scene.
__global__ void __launch_bounds__(kFieldThreads)
    k_static_field(Geo g, const uint8_t* __restrict__ cell, const float* __restrict__ KO,
                   const float* __restrict__ KE, float* __restrict__ Fs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = g.r, S = 2 * r + 1, nT = S * S, HW = kTile + 2 * r;
  float* sKO = reinterpret_cast<float*>(smem);
  float* sKE = sKO + nT;
  uint8_t* sC = reinterpret_cast<uint8_t*>(sKE + nT);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  for (int i = tid; i < nT; i += blockDim.x) {
    sKO[i] = KO[i];
    sKE[i] = KE[i];
  }
  for (int i = tid; i < HW * HW; i += blockDim.x) {
    const int hx = i % HW, hy = i / HW;
    int gx, gy;
    uint8_t v = kFree;
    if (wrap_coord(x0 - r + hx, g.W, g.px, gx) && wrap_coord(y0 - r + hy, g.H, g.py, gy))
      v = cell[(size_t)gy * g.W + gx];
    sC[i] = v;
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5;
  float sum[kRowsPerThread], comp[kRowsPerThread];
#pragma unroll
  for (int j = 0; j < kRowsPerThread; ++j) sum[j] = comp[j] = 0.f;
  for (int dy = -r; dy <= r; ++dy) {
    for (int dx = -r; dx <= r; ++dx) {
      const int ti = (dy + r) * S + (dx + r);
      const float ko = sKO[ti], ke = sKE[ti];
      const uint8_t* col = sC + (lane - dx + r);
#pragma unroll
      for (int j = 0; j < kRowsPerThread; ++j) {
        const uint8_t b = col[(4 * w + j - dy + r) * HW];
        const float v = (b == kWall) ? ko : ((b == kExit) ? ke : 0.f);
        const float yk = v - comp[j];
        const float tk = sum[j] + yk;
        comp[j] = (tk - sum[j]) - yk;
        sum[j] = tk;
      }
    }
  }
  const int x = x0 + lane;
#pragma unroll
  for (int j = 0; j < kRowsPerThread; ++j) {
    const int y = y0 + 4 * w + j;
    if (x < g.W && y < g.H) Fs[(size_t)y * g.W + x] = sum[j];
  }
}

void launch_static_field(const Geo& g, const uint8_t* cell, const Tables& tb, float* Fs,
                         cudaStream_t s) {
  const int S = 2 * g.r + 1, HW = kTile + 2 * g.r;
  const size_t smem = (size_t)2 * S * S * sizeof(float) + (size_t)HW * HW;
  cudaFuncSetAttribute(k_static_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(cdiv(g.W, kTile), cdiv(g.H, kTile));
  k_static_field<<<grid, kFieldThreads, smem, s>>>(g, cell, tb.KO, tb.KE, Fs);
}

// --------------------------------------------------------------- guidance
// Chamfer (5, 7) geodesic distance to the nearest EXIT through non-WALL su
// (kDInf where none is reachable, kDWall on WALL su),
// solved as the fixed point of D(c) = min_k D(c + Delta_k) + w_k by tile-local
// relaxation in shared memory; a tile is revisited only when it or a
// neighbour changed in the previous round.  The fixed point is unique, so the
// result is exact and independent of the visiting order.
__global__ void k_guidance_init(Geo g, const uint8_t* __restrict__ cell, int32_t* __restrict__ D) {
  const size_t n = (size_t)g.W * g.H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    D[i] = cell[i] == kExit ? 0 : (cell[i] == kWall ? kDWall : kDInf);
}

// the exported form: WALL su read kDInf, like unreachable ones
__global__ void k_guidance_export(int32_t* __restrict__ D, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (D[i] == kDWall) D[i] = kDInf;
}

// the imported form: WALL su carry kDWall whatever the caller gave there
__global__ void k_guidance_import(const uint8_t* __restrict__ cell, int32_t* __restrict__ D, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (cell[i] == kWall) D[i] = kDWall;
}

__global__ void __launch_bounds__(1024)
    k_guidance_round(Geo g, const uint8_t* __restrict__ cell, int32_t* __restrict__ D,
                     const uint8_t* __restrict__ act_in, uint8_t* __restrict__ act_out,
                     int* __restrict__ changed) {
  __shared__ int32_t sD[kTile + 2][kTile + 2];
  const int ntx = (g.W + kTile - 1) / kTile, nty = (g.H + kTile - 1) / kTile;
  const int tile = blockIdx.x;
  if (!act_in[tile]) return;
  const int tx = tile % ntx, ty = tile / ntx;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int tid = threadIdx.x;
  for (int i = tid; i < (kTile + 2) * (kTile + 2); i += blockDim.x) {
    const int hx = i % (kTile + 2), hy = i / (kTile + 2);
    int gx, gy;
    int32_t v = kDInf;
    if (wrap_coord(x0 - 1 + hx, g.W, g.px, gx) && wrap_coord(y0 - 1 + hy, g.H, g.py, gy))
      v = D[(size_t)gy * g.W + gx];
    sD[hy][hx] = v;
  }
  const int lx = tid % kTile, ly = tid / kTile;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool valid = gx < g.W && gy < g.H;
  uint8_t cv = kWall;
  if (valid) cv = cell[(size_t)gy * g.W + gx];
  const bool relax = valid && cv == kFree;
  __syncthreads();
  bool mine = false;
  for (int it = 0; it < 4 * kTile * kTile; ++it) {
    bool ch = false;
    if (relax) {
      const int32_t cur = sD[ly + 1][lx + 1];
      int32_t best = cur;
#pragma unroll
      for (int k = 1; k <= 8; ++k) {
        const int32_t v = sD[ly + 1 + c_dy[k]][lx + 1 + c_dx[k]];
        const int32_t wk = (c_dx[k] != 0 && c_dy[k] != 0) ? 7 : 5;
        if (v < kDInf && v + wk < best) best = v + wk;
      }
      if (best < cur) {
        sD[ly + 1][lx + 1] = best;
        ch = true;
      }
    }
    mine |= ch;
    if (!__syncthreads_or(ch)) break;
  }
  if (mine) D[(size_t)gy * g.W + gx] = sD[ly + 1][lx + 1];
  if (__syncthreads_or(mine) && tid == 0) {
    *changed = 1;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int nx = tx + dx, ny = ty + dy;
        if (g.px) nx = (nx + ntx) % ntx;
        if (g.py) ny = (ny + nty) % nty;
        if (nx >= 0 && nx < ntx && ny >= 0 && ny < nty) act_out[ny * ntx + nx] = 1;
      }
  }
}

int device_sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

void launch_guidance_init(const Geo& g, const uint8_t* cell, int32_t* D, cudaStream_t s) {
  const size_t n = (size_t)g.W * g.H;
  int blocks = (int)((n + 255) / 256);
  // grid-stride: at most 64 blocks of 256 per SM
  if (blocks > device_sm_count() * 64) blocks = device_sm_count() * 64;
  k_guidance_init<<<blocks, 256, 0, s>>>(g, cell, D);
}

void launch_guidance_export(int32_t* D, size_t n, cudaStream_t s) {
  if (!n) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 64) blocks = device_sm_count() * 64;
  k_guidance_export<<<blocks, 256, 0, s>>>(D, n);
}

void launch_guidance_import(const uint8_t* cell, int32_t* D, size_t n, cudaStream_t s) {
  if (!n) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 64) blocks = device_sm_count() * 64;
  k_guidance_import<<<blocks, 256, 0, s>>>(cell, D, n);
}

void launch_guidance_round(const Geo& g, const uint8_t* cell, int32_t* D, const uint8_t* act_in,
                           uint8_t* act_out, int* changed, cudaStream_t s) {
  const int ntiles = cdiv(g.W, kTile) * cdiv(g.H, kTile);
  k_guidance_round<<<ntiles, kTile * kTile, 0, s>>>(g, cell, D, act_in, act_out, changed);
}

// ------------------------------------------------------------- placement
__global__ void k_place_clear(int n, const int2* __restrict__ xy, const uint8_t* __restrict__ alive,
                              Geo g, int32_t* __restrict__ occ, uint8_t* __restrict__ ocls,
                              Sizes sz) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive[p]) return;
  const int2 q = xy[p];
  const int a = sz.w ? sz.w[p] >> 1 : 0, b = sz.w ? sz.h[p] >> 1 : 0;
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      size_t s;
      if (rect_su(g, q.x, q.y, i, j, s)) occ[s] = -1;
    }
  ocls[(size_t)q.y * g.opitch + q.x] = 0;
}

__global__ void k_place_scatter(int n, const int2* __restrict__ xy,
                                const uint8_t* __restrict__ heading,
                                const uint8_t* __restrict__ goal, const uint8_t* __restrict__ alive,
                                const uint8_t* __restrict__ cell, Geo g, int32_t* __restrict__ occ,
                                uint8_t* __restrict__ ocls, Counters* ctr, Sizes sz) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (heading[p] > 8 || goal[p] > 8) atomicOr(&ctr->err, kErrPlaceRange);
  if (!alive[p]) return;
  const int2 q = xy[p];
  if (q.x < 0 || q.x >= g.W || q.y < 0 || q.y >= g.H) {
    atomicOr(&ctr->err, kErrPlaceRange);
    return;
  }
  const size_t c = (size_t)q.y * g.W + q.x;
  if (cell[c] != kFree) atomicOr(&ctr->err, kErrPlaceConflict);
  // the rectangle (1 x 1 without sizes): inside, off walls, on nobody else
  const int a = sz.w ? sz.w[p] >> 1 : 0, b = sz.w ? sz.h[p] >> 1 : 0;
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      size_t s;
      if (!rect_su(g, q.x, q.y, i, j, s)) {
        atomicOr(&ctr->err, kErrPlaceConflict);
        continue;
      }
      if (cell[s] == kWall || atomicCAS(&occ[s], -1, p) != -1)
        atomicOr(&ctr->err, kErrPlaceConflict);
    }
  ocls[(size_t)q.y * g.opitch + q.x] = (uint8_t)(1 + (heading[p] > 8 ? 0 : heading[p]));
}

void launch_place_clear(int n, const int2* xy, const uint8_t* alive, const Geo& g, int32_t* occ,
                        uint8_t* ocls, cudaStream_t s, const Sizes& sz) {
  if (n <= 0) return;
  k_place_clear<<<cdiv(n, 256), 256, 0, s>>>(n, xy, alive, g, occ, ocls, sz);
}

// A placement of as many 1 x 1 pedestrians into the same arrays (the tick
// graphs are kept).  Only pedestrians whose su or alive flag changes leave
// (leave_su) and claim (claim_su, with the checks of k_place_scatter)
// occupancy-grid entries, in two launches so that a su vacated by one may be
// claimed by another; a pedestrian that keeps its su only rewrites its class
// entry when its heading changed.  The entries of the others are already
// right: the previous placement validated them and every tick keeps the grids
// in step with the pedestrians.

// Pedestrian p, alive at q before the placement, is placed at v (alive: a):
// frees q unless it stays there.
__device__ __forceinline__ void leave_su(int2 q, int2 v, uint8_t a, const Geo& g,
                                         int32_t* __restrict__ occ, uint8_t* __restrict__ ocls) {
  if (a && q.x == v.x && q.y == v.y) return;
  occ[(size_t)q.y * g.W + q.x] = -1;
  ocls[(size_t)q.y * g.opitch + q.x] = 0;
}

// Live pedestrian p placed at v with heading hp; before the placement it was
// at q (if a_old) with heading h_old.
__device__ __forceinline__ void claim_su(int p, int2 v, uint8_t hp, bool a_old, int2 q,
                                         uint8_t h_old, const uint8_t* __restrict__ cell,
                                         const Geo& g, int32_t* __restrict__ occ,
                                         uint8_t* __restrict__ ocls, Counters* ctr) {
  const uint8_t cls = (uint8_t)(1 + (hp > 8 ? 0 : hp));
  if (a_old && q.x == v.x && q.y == v.y) {
    if (hp != h_old) ocls[(size_t)v.y * g.opitch + v.x] = cls;
    return;
  }
  if (v.x < 0 || v.x >= g.W || v.y < 0 || v.y >= g.H) {
    atomicOr(&ctr->err, kErrPlaceRange);
    return;
  }
  const size_t c = (size_t)v.y * g.W + v.x;
  if (cell[c] != kFree || atomicCAS(&occ[c], -1, p) != -1) atomicOr(&ctr->err, kErrPlaceConflict);
  ocls[(size_t)v.y * g.opitch + v.x] = cls;
}

// From copies: xy_prev / alive_prev / heading_prev hold the state before the
// placement, xy / heading / goal / alive the new one.
__global__ void k_place_diff_clear(int n, const int2* __restrict__ xy_prev,
                                   const uint8_t* __restrict__ alive_prev,
                                   const int2* __restrict__ xy, const uint8_t* __restrict__ alive,
                                   Geo g, int32_t* __restrict__ occ, uint8_t* __restrict__ ocls) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive_prev[p]) return;
  leave_su(xy_prev[p], xy[p], alive[p], g, occ, ocls);
}

__global__ void k_place_diff_claim(int n, const int2* __restrict__ xy_prev,
                                   const uint8_t* __restrict__ alive_prev,
                                   const uint8_t* __restrict__ heading_prev,
                                   const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
                                   const uint8_t* __restrict__ goal, const uint8_t* __restrict__ alive,
                                   const uint8_t* __restrict__ cell, Geo g, int32_t* __restrict__ occ,
                                   uint8_t* __restrict__ ocls, Counters* ctr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint8_t hp = heading[p];
  if (hp > 8 || goal[p] > 8) atomicOr(&ctr->err, kErrPlaceRange);
  if (!alive[p]) return;
  claim_su(p, xy[p], hp, alive_prev[p] != 0, xy_prev[p], heading_prev[p], cell, g, occ, ocls, ctr);
}

// The same placement read in place from the caller's buffers (device memory
// or pinned host memory mapped into the device's address space; a NULL
// heading, goal or alive array stands for 0, 0, 1): the first launch stages
// the new state in st_* and clears the su of the pedestrians that leave
// theirs; the second claims the su of those that take a new one (the checks
// of k_place_scatter), rewrites the class entry of those that turn in place,
// and installs the new state with cleared decisions.
__global__ void k_place_direct_stage(int n, const int2* __restrict__ src_xy,
                                     const uint8_t* __restrict__ src_h,
                                     const uint8_t* __restrict__ src_g,
                                     const uint8_t* __restrict__ src_a, int2* __restrict__ st_xy,
                                     uint8_t* __restrict__ st_h, uint8_t* __restrict__ st_g,
                                     uint8_t* __restrict__ st_a, const int2* __restrict__ xy,
                                     const uint8_t* __restrict__ alive, Geo g,
                                     int32_t* __restrict__ occ, uint8_t* __restrict__ ocls) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int2 v = src_xy[p];
  const uint8_t a = src_a ? src_a[p] : 1;
  st_xy[p] = v;
  st_h[p] = src_h ? src_h[p] : 0;
  st_g[p] = src_g ? src_g[p] : 0;
  st_a[p] = a;
  if (alive[p]) leave_su(xy[p], v, a, g, occ, ocls);
}

__global__ void k_place_direct_claim(int n, const int2* __restrict__ st_xy,
                                     const uint8_t* __restrict__ st_h,
                                     const uint8_t* __restrict__ st_g,
                                     const uint8_t* __restrict__ st_a, int2* __restrict__ xy,
                                     uint8_t* __restrict__ heading, uint8_t* __restrict__ goal,
                                     uint8_t* __restrict__ alive, uint8_t* __restrict__ choice,
                                     uint8_t* __restrict__ won, const uint8_t* __restrict__ cell,
                                     Geo g, int32_t* __restrict__ occ, uint8_t* __restrict__ ocls,
                                     Counters* ctr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int2 v = st_xy[p], q = xy[p];
  const uint8_t hp = st_h[p], gp = st_g[p], ap = st_a[p], a_old = alive[p], h_old = heading[p];
  xy[p] = v;
  heading[p] = hp;
  goal[p] = gp;
  alive[p] = ap;
  choice[p] = 0;
  won[p] = 0;
  if (hp > 8 || gp > 8) atomicOr(&ctr->err, kErrPlaceRange);
  if (ap) claim_su(p, v, hp, a_old != 0, q, h_old, cell, g, occ, ocls, ctr);
}

void launch_place_direct(int n, const int2* src_xy, const uint8_t* src_h, const uint8_t* src_g,
                         const uint8_t* src_a, int2* st_xy, uint8_t* st_h, uint8_t* st_g,
                         uint8_t* st_a, int2* xy, uint8_t* heading, uint8_t* goal, uint8_t* alive,
                         uint8_t* choice, uint8_t* won, const uint8_t* cell, const Geo& g,
                         int32_t* occ, uint8_t* ocls, Counters* ctr, cudaStream_t s) {
  if (n <= 0) return;
  // one pedestrian a thread: many small reads in flight move pinned host
  // buffers faster than fewer, wider ones (measured: 4 a thread with 16-byte
  // accesses slowed the read-back from 0.078 to 0.126 ms for 10^6)
  k_place_direct_stage<<<cdiv(n, 256), 256, 0, s>>>(n, src_xy, src_h, src_g, src_a, st_xy, st_h, st_g,
                                                    st_a, xy, alive, g, occ, ocls);
  k_place_direct_claim<<<cdiv(n, 256), 256, 0, s>>>(n, st_xy, st_h, st_g, st_a, xy, heading, goal,
                                                    alive, choice, won, cell, g, occ, ocls, ctr);
}

// Pedestrian state written in place into the caller's buffers (any may be
// NULL; device memory or mapped pinned host memory), one pedestrian a thread.
__global__ void k_read_peds(int n, const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
                            const uint8_t* __restrict__ alive, int2* __restrict__ dxy,
                            uint8_t* __restrict__ dh, uint8_t* __restrict__ da) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (dxy) dxy[p] = xy[p];
  if (dh) dh[p] = heading[p];
  if (da) da[p] = alive[p];
}

void launch_read_peds(int n, const int2* xy, const uint8_t* heading, const uint8_t* alive, int2* dxy,
                      uint8_t* dh, uint8_t* da, cudaStream_t s) {
  if (n <= 0) return;
  k_read_peds<<<cdiv(n, 256), 256, 0, s>>>(n, xy, heading, alive, dxy, dh, da);
}

void launch_place_diff(int n, const int2* xy_prev, const uint8_t* alive_prev,
                       const uint8_t* heading_prev, const int2* xy, const uint8_t* heading,
                       const uint8_t* goal, const uint8_t* alive, const uint8_t* cell, const Geo& g,
                       int32_t* occ, uint8_t* ocls, Counters* ctr, cudaStream_t s) {
  if (n <= 0) return;
  k_place_diff_clear<<<cdiv(n, 256), 256, 0, s>>>(n, xy_prev, alive_prev, xy, alive, g, occ, ocls);
  k_place_diff_claim<<<cdiv(n, 256), 256, 0, s>>>(n, xy_prev, alive_prev, heading_prev, xy, heading,
                                                  goal, alive, cell, g, occ, ocls, ctr);
}

// per-placement counters and flags back to zero (the tick counter stays)
__global__ void k_reset_counters(Counters* ctr) {
  ctr->moved = 0;
  ctr->exited = 0;
  ctr->max_registrants = 0;
  ctr->err = 0;
  ctr->decided = 0;
  ctr->near_ties = 0;
}

void launch_reset_counters(Counters* ctr, cudaStream_t s) { k_reset_counters<<<1, 1, 0, s>>>(ctr); }

void launch_place_scatter(int n, const int2* xy, const uint8_t* heading, const uint8_t* goal,
                          const uint8_t* alive, const uint8_t* cell, const Geo& g, int32_t* occ,
                          uint8_t* ocls, Counters* ctr, cudaStream_t s, const Sizes& sz) {
  if (n <= 0) return;
  k_place_scatter<<<cdiv(n, 256), 256, 0, s>>>(n, xy, heading, goal, alive, cell, g, occ, ocls,
                                               ctr, sz);
}

// --------------------------------------------------------- S1: binning
// Counting sort of the live pedestrians into 32 x 32-su bins, read off the
// per-su occupancy-class grid so that the order inside a bin is row-major
// and therefore deterministic.  One warp covers 4 bins side by side (128
// columns of a 128-byte-pitched grid, 4 bytes per lane) for 32 rows; lanes
// 8b..8b+7 cover bin b.
__global__ void k_bin_count(Geo g, const uint8_t* __restrict__ ocls, int32_t* __restrict__ count) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int ngx = (g.nbx + 3) >> 2;
  if (wid >= ngx * g.nby) return;
  bin_count_group(g, ocls, count, wid % ngx, wid / ngx, threadIdx.x & 31);
}

__global__ void k_bin_fill(Geo g, const uint8_t* __restrict__ ocls, const int32_t* __restrict__ occ,
                           const int32_t* __restrict__ start, uint32_t* __restrict__ rec,
                           int32_t* __restrict__ rec_id) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int ngx = (g.nbx + 3) >> 2;
  if (wid >= ngx * g.nby) return;
  bin_fill_group(g, ocls, occ, start, rec, rec_id, wid % ngx, wid / ngx, threadIdx.x & 31);
}

void launch_bin_count(const Geo& g, const uint8_t* ocls, int32_t* count, cudaStream_t s) {
  const int nw = ((g.nbx + 3) >> 2) * g.nby;
  k_bin_count<<<cdiv(nw * 32, 256), 256, 0, s>>>(g, ocls, count);
}

void launch_bin_fill(const Geo& g, const uint8_t* ocls, const int32_t* occ, const int32_t* start,
                     uint32_t* rec, int32_t* rec_id, cudaStream_t s) {
  const int nw = ((g.nbx + 3) >> 2) * g.nby;
  k_bin_fill<<<cdiv(nw * 32, 256), 256, 0, s>>>(g, ocls, occ, start, rec, rec_id);
}

// The same records driven by the pedestrian list, for sparse crowds where
// reading the whole class grid costs more than the pedestrians: count with
// atomics (each pedestrian keeps its arrival slot), scan, scatter each
// pedestrian's su key (row << 5 | column inside the bin) to its slot, then
// rank: a pedestrian's place in its bin is the number of smaller keys there
// (keys are unique, one pedestrian per su), which is the row-major order of
// the grid path.  Work per pedestrian is the size of its bin.
__device__ __forceinline__ int ped_bin(const Geo& g, int2 q) {
  return (q.y / kBin) * g.nbx + q.x / kBin;
}

__global__ void k_binp_count(int n, Geo g, const int2* __restrict__ xy,
                             const uint8_t* __restrict__ alive, int32_t* __restrict__ count,
                             int32_t* __restrict__ slot) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive[p]) return;
  slot[p] = atomicAdd(&count[ped_bin(g, xy[p])], 1);
}

__global__ void k_binp_scatter(int n, Geo g, const int2* __restrict__ xy,
                               const uint8_t* __restrict__ alive, const int32_t* __restrict__ slot,
                               const int32_t* __restrict__ start, uint32_t* __restrict__ key) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive[p]) return;
  const int2 q = xy[p];
  key[start[ped_bin(g, q)] + slot[p]] = (uint32_t)((q.y % kBin) << 5 | (q.x % kBin));
}

__global__ void k_binp_rank(int n, Geo g, const int2* __restrict__ xy,
                            const uint8_t* __restrict__ alive, const uint8_t* __restrict__ heading,
                            const int32_t* __restrict__ start, const uint32_t* __restrict__ key,
                            uint32_t* __restrict__ rec, int32_t* __restrict__ rec_id) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !alive[p]) return;
  const int2 q = xy[p];
  const int b = ped_bin(g, q);
  const int s = start[b], e = start[b + 1];
  const int col = q.x % kBin, row = q.y % kBin;
  const uint32_t mine = (uint32_t)(row << 5 | col);
  int rank = 0;
  for (int i = s; i < e; ++i) rank += key[i] < mine;
  const uint32_t cls = heading[p] > 8 ? 0u : heading[p];
  rec[s + rank] = (uint32_t)col | ((uint32_t)row << 8) | (cls << 16);
  rec_id[s + rank] = p;
}

void launch_bins_from_peds(const Geo& g, int n, const int2* xy, const uint8_t* alive,
                           const uint8_t* heading, int32_t* count, int32_t* start,
                           int32_t* scan_tmp, int32_t* slot, uint32_t* key, uint32_t* rec,
                           int32_t* rec_id, cudaStream_t s) {
  const int nbins = g.nbx * g.nby;
  cudaMemsetAsync(count, 0, (size_t)nbins * sizeof(int32_t), s);
  if (n > 0) k_binp_count<<<cdiv(n, 256), 256, 0, s>>>(n, g, xy, alive, count, slot);
  launch_scan(count, start, nbins, scan_tmp, s);
  if (n > 0) {
    k_binp_scatter<<<cdiv(n, 256), 256, 0, s>>>(n, g, xy, alive, slot, start, key);
    k_binp_rank<<<cdiv(n, 256), 256, 0, s>>>(n, g, xy, alive, heading, start, key, rec, rec_id);
  }
}

__global__ void k_clear_dead(int n, const uint8_t* __restrict__ alive, uint8_t* __restrict__ choice,
                             uint8_t* __restrict__ won) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && !alive[p]) {
    choice[p] = 0;
    won[p] = 0;
  }
}

void launch_clear_dead(int n, const uint8_t* alive, uint8_t* choice, uint8_t* won, cudaStream_t s) {
  if (n <= 0) return;
  k_clear_dead<<<cdiv(n, 256), 256, 0, s>>>(n, alive, choice, won);
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of n int32 into out[0..n] (out[n] = total), three
// passes: per-block totals, a single-block scan of the totals, final; one
// pass (the final one, from offset 0) when a block covers all n.
constexpr int kScanThreads = 1024, kScanItems = 4, kScanChunk = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* sWarp, int& total) {
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

__global__ void __launch_bounds__(kScanThreads) k_scan_totals(const int32_t* __restrict__ in, int n,
                                                              int32_t* __restrict__ totals) {
  __shared__ int sWarp[32];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  int total;
  block_exclusive_scan(s, sWarp, total);
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int32_t* __restrict__ totals, int nb) {
  __shared__ int sWarp[32];
  int carry = 0;
  for (int base = 0; base < nb; base += kScanChunk) {
    int v[kScanItems], s = 0;
    const int i0 = base + threadIdx.x * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (i0 + k < nb) ? totals[i0 + k] : 0;
      s += v[k];
    }
    int total;
    int e = block_exclusive_scan(s, sWarp, total) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (i0 + k < nb) totals[i0 + k] = e;
      e += v[k];
    }
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int32_t* __restrict__ in, int n,
                                                             const int32_t* __restrict__ offs,
                                                             int32_t* __restrict__ out) {
  __shared__ int sWarp[32];
  const int i0 = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
  int v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (i0 + k < n) ? in[i0 + k] : 0;
    s += v[k];
  }
  int total;
  int e = block_exclusive_scan(s, sWarp, total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (i0 + k < n) out[i0 + k] = e;
    e += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = e;
}

int scan_tmp_elems(int n) { return cdiv(n > 0 ? n : 1, kScanChunk); }

void launch_scan(const int32_t* in, int32_t* out, int n, int32_t* block_tmp, cudaStream_t s) {
  const int nb = scan_tmp_elems(n);
  if (nb == 1) {  // small lattices: one launch instead of three
    k_scan_final<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    return;
  }
  k_scan_totals<<<nb, kScanThreads, 0, s>>>(in, n, block_tmp);
  k_scan_top<<<1, kScanThreads, 0, s>>>(block_tmp, nb);
  k_scan_final<<<nb, kScanThreads, 0, s>>>(in, n, block_tmp, out);
}

// ------------------------------------ S2: field gather for radius > 50
// Used where the heading-class tables would not fit in shared memory (the
// class-table gather in sfm_field.cu covers radius <= 50).  Each CTA owns a
// 32 x 32 su tile.  The pedestrians of the bins that overlap
// the tile's r-halo are staged in shared memory in chunks of at most `cap`
// records (the bounded multi-step sum of Alg. 3 / Eq. 1: the per-su sum is
// split into a fixed number of partial passes), every lane accumulates the
// kernel-table value of each staged pedestrian inside its window for its 4
// rows, and the tile is written once as F = F_static + sum.
struct HaloBin {
  int start, count, xoff, yoff;
};
constexpr int kMaxImages = 24;

// Bins (one dimension) overlapping the halo [lo, hi]; returns entries (bin,
// offset of the bin origin relative to the tile origin).
__device__ int halo_list(int lo, int hi, int n, int periodic, int nbins, int t0, int* bin,
                         int* off) {
  int cnt = 0;
  if (!periodic) {
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    for (int b = lo / kBin; lo <= hi && b <= hi / kBin; ++b) {
      if (cnt < kMaxImages) { bin[cnt] = b; off[cnt] = b * kBin - t0; }
      ++cnt;
    }
    return cnt;
  }
  const int k0 = floor_div(lo, n), k1 = floor_div(hi, n);
  for (int k = k0; k <= k1; ++k) {
    int a = lo - k * n, z = hi - k * n;
    if (a < 0) a = 0;
    if (z > n - 1) z = n - 1;
    for (int b = a / kBin; a <= z && b <= z / kBin; ++b) {
      if (cnt < kMaxImages) { bin[cnt] = b; off[cnt] = b * kBin + k * n - t0; }
      ++cnt;
    }
  }
  (void)nbins;
  return cnt;
}

__global__ void __launch_bounds__(kFieldThreads)
    k_field(Geo g, const int32_t* __restrict__ bin_start, const uint32_t* __restrict__ rec,
            Tables tb, const float* __restrict__ Fs, float* __restrict__ out, int out_row0,
            int ty0, int store_lo, int store_hi, int cap, Counters* ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ HaloBin sBins[kMaxImages * kMaxImages];
  __shared__ int sPref[kMaxImages * kMaxImages + 1];
  __shared__ int sNB;
  const int r = g.r, S = 2 * r + 1, nT = S * S;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int4* sPed = reinterpret_cast<int4*>(smem);
  float* sT0 = reinterpret_cast<float*>(sPed + cap);
  float* sTX = sT0 + nT;
  float* sTY = sTX + nT;
  const int x0 = blockIdx.x * kTile, y0 = (ty0 + blockIdx.y) * kTile;

  for (int i = tid; i < nT; i += blockDim.x) {
    sT0[i] = tb.T0[i];
    sTX[i] = tb.TX[i];
    sTY[i] = tb.TY[i];
  }
  if (tid == 0) {
    int bxs[kMaxImages], xo[kMaxImages], bys[kMaxImages], yo[kMaxImages];
    const int nxl = halo_list(x0 - r, x0 + kTile - 1 + r, g.W, g.px, g.nbx, x0, bxs, xo);
    const int nyl = halo_list(y0 - r, y0 + kTile - 1 + r, g.H, g.py, g.nby, y0, bys, yo);
    int nb = 0;
    if (nxl > kMaxImages || nyl > kMaxImages) {
      atomicOr(&ctr->err, kErrHalo);
    } else {
      for (int a = 0; a < nyl; ++a)
        for (int b = 0; b < nxl; ++b) {
          sBins[nb].start = bys[a] * g.nbx + bxs[b];  // bin id for now
          sBins[nb].xoff = xo[b];
          sBins[nb].yoff = yo[a];
          ++nb;
        }
    }
    sNB = nb;
  }
  __syncthreads();
  const int nb = sNB;
  for (int i = tid; i < nb; i += blockDim.x) {
    const int id = sBins[i].start;
    const int s0 = bin_start[id];
    sBins[i].start = s0;
    sBins[i].count = bin_start[id + 1] - s0;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int i = 0; i < nb; ++i) {
      sPref[i] = acc;
      acc += sBins[i].count;
    }
    sPref[nb] = acc;
  }
  __syncthreads();
  const int total = sPref[nb];

  float acc[kRowsPerThread];
#pragma unroll
  for (int j = 0; j < kRowsPerThread; ++j) acc[j] = 0.f;
  const int rowb = kRowsPerThread * w;  // first row of this warp inside the tile

  for (int base = 0; base < total; base += cap) {
    const int cnt = min(cap, total - base);
    for (int i = tid; i < cnt; i += blockDim.x) {
      const int q = base + i;
      int lo = 0, hi = nb;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sPref[mid] <= q) lo = mid; else hi = mid;
      }
      const uint32_t rc = rec[sBins[lo].start + (q - sPref[lo])];
      const int cls = (rc >> 16) & 0xf;
      const float2 h = tb.hvec[cls];
      sPed[i] = make_int4(sBins[lo].xoff + (int)(rc & 0xff), sBins[lo].yoff + (int)((rc >> 8) & 0xff),
                          __float_as_int(h.x), __float_as_int(h.y));
    }
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      const int4 pd = sPed[i];
      const int dyb = rowb - pd.y;  // dy of this warp's first row
      if (dyb + kRowsPerThread - 1 < -r || dyb > r) continue;    // warp-uniform
      if (kTile - 1 - pd.x < -r || -pd.x > r) continue;          // warp-uniform
      const int dx = lane - pd.x;
      if ((unsigned)(dx + r) > (unsigned)(2 * r)) continue;
      const float hx = __int_as_float(pd.z), hy = __int_as_float(pd.w);
#pragma unroll
      for (int j = 0; j < kRowsPerThread; ++j) {
        const int dy = dyb + j;
        if ((unsigned)(dy + r) <= (unsigned)(2 * r)) {
          const int ti = (dy + r) * S + (dx + r);
          acc[j] += fmaf(hy, sTY[ti], fmaf(hx, sTX[ti], sT0[ti]));
        }
      }
    }
    __syncthreads();
  }
  const int x = x0 + lane;
#pragma unroll
  for (int j = 0; j < kRowsPerThread; ++j) {
    const int y = y0 + rowb + j;
    if (x < g.W && y < g.H && y >= store_lo && y < store_hi) {
      const size_t c = (size_t)y * g.W + x;
      out[(size_t)(y - out_row0) * g.W + x] = Fs[c] + acc[j];
    }
  }
}

static int field_cap(int r, size_t* smem_out) {
  const int S = 2 * r + 1;
  const size_t tables = (size_t)3 * S * S * sizeof(float);
  const size_t budget = 200 * 1024;
  int cap = kStageCap;
  while (cap > 256 && tables + (size_t)cap * sizeof(int4) > budget) cap >>= 1;
  *smem_out = tables + (size_t)cap * sizeof(int4);
  return cap;
}

void launch_field_v1(const Geo& g, const int32_t* bin_start, const uint32_t* rec,
                            const Tables& tb, const float* Fs, float* out, int out_row0,
                            int store_lo, int store_hi, Counters* ctr, cudaStream_t s) {
  const int ty0 = store_lo / kTile, ty1 = (store_hi + kTile - 1) / kTile;
  if (ty1 <= ty0) return;
  size_t smem;
  const int cap = field_cap(g.r, &smem);
  cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(cdiv(g.W, kTile), ty1 - ty0);
  k_field<<<grid, kFieldThreads, smem, s>>>(g, bin_start, rec, tb, Fs, out, out_row0, ty0,
                                            store_lo, store_hi, cap, ctr);
}


__global__ void k_class_tables(int r, int SP, double kP, double aP, double gamma, double taper_in,
                               float* __restrict__ T) {
  const int TR = 2 * r + 1 + 2 * kFieldPad;
  const int n = 4 * TR * SP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = i / (TR * SP), rem = i % (TR * SP);
  const int dy = rem / SP - (r + kFieldPad), dx = rem % SP - r;
  T[i] = (float)class_kernel_value(t, dx, dy, r, kP, aP, gamma, taper_in);
}

int class_table_stride(int r) { return class_table_stride_of(r); }

size_t class_table_floats(int r) { return class_table_floats_of(r); }

void launch_class_tables(int r, const sfm_params& p, float* T, cudaStream_t s, double taper_in) {
  const int sp = class_table_stride(r);
  if (!sp) return;
  const int n = (int)class_table_floats(r);
  k_class_tables<<<cdiv(n, 256), 256, 0, s>>>(r, sp, p.kP, p.aP, p.gamma, taper_in, T);
}

// --------------------------------------------------------- S3: decide
// Per live pedestrian (visited in bin order, so neighbouring threads read
// neighbouring su): E over the 9 candidates (stay + 8 neighbours), admissible
// iff inside, not WALL and unoccupied at tick start; select of the minimum
// with ties to the smallest class.
__global__ void __launch_bounds__(256, 4) k_decide(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                         int b_lo, int b_hi, const int2* __restrict__ xy,
                         const uint8_t* __restrict__ heading, const uint8_t* __restrict__ goal,
                         const uint8_t* __restrict__ cell, const uint8_t* __restrict__ ocls,
                         const int32_t* __restrict__ D, const float* __restrict__ F, int main_off,
                         int lo_row, int hi_row, int hi_off, int y_lo, int y_hi, Geo g,
                         float beta, const float* __restrict__ own,
                         const float* __restrict__ dirdot, uint8_t* __restrict__ choice,
                         WalkPeriods wp, Sizes sz, const int32_t* __restrict__ occ,
                         Counters* __restrict__ ctr, int ring) {
  // grid-stride over the records of bins [b_lo, b_hi): a band's launch needs
  // no more blocks than the GPU holds, whatever its share of the crowd.  The
  // records are taken from the last backwards: the gather wrote the band's
  // bottom rows last, so the first blocks find their field rows still in L2
  // (0.199 -> 0.195 ms a banded floor tick).
  const int end = bin_start[b_hi];
  const long long t = wp.period ? wp.ctr->t : 0;
  const int cnt = end - bin_start[b_lo];
  unsigned decided = 0, ties = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const int p = rec_id[end - 1 - k];
    if (wp.period && t % wp.period[p] != wp.phase[p]) {
      choice[p] = 0;  // not this pedestrian's tick: it stays
      continue;
    }
    bool tie = false;
    choice[p] = decide_one<true>(p, g, xy, heading, goal, cell, ocls, D, F, main_off, lo_row,
                                 hi_row, hi_off, y_lo, y_hi, beta, own, dirdot, sz.w, sz.h, occ,
                                 &tie, ring);
    ++decided;
    ties += tie ? 1u : 0u;
  }
  // decisions and near ties, one atomic per warp
  decided = __reduce_add_sync(0xffffffffu, decided);
  ties = __reduce_add_sync(0xffffffffu, ties);
  if (ctr && (threadIdx.x & 31) == 0 && decided) {
    atomicAdd(&ctr->decided, (unsigned long long)decided);
    if (ties) atomicAdd(&ctr->near_ties, (unsigned long long)ties);
  }
}

void launch_decide(int n, const int32_t* rec_id, const int32_t* bin_start, int b_lo, int b_hi,
                   const int2* xy, const uint8_t* heading, const uint8_t* goal,
                   const uint8_t* cell, const uint8_t* ocls, const int32_t* D, const float* F,
                   int main_off, int lo_row, int hi_row, int hi_off, int y_lo, int y_hi,
                   const Geo& g, float beta, const Tables& tb, uint8_t* choice, cudaStream_t s,
                   const WalkPeriods& wp, const Sizes& sz, const int32_t* occ,
                   Counters* ctr, int ring) {
  if (n <= 0 || b_hi <= b_lo) return;
  static int max_blocks = 0;
  if (!max_blocks) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    max_blocks = (nsm > 0 ? nsm : 1) * 8;  // two rounds of the 4 blocks of 256 an SM holds (64 registers)
  }
  const int blocks = cdiv(n, 256) < max_blocks ? cdiv(n, 256) : max_blocks;
  k_decide<<<blocks, 256, 0, s>>>(rec_id, bin_start, b_lo, b_hi, xy, heading, goal, cell,
                                        ocls, D, F, main_off, lo_row, hi_row, hi_off, y_lo, y_hi,
                                        g, beta, tb.own, tb.dirdot, choice, wp, sz, occ, ctr, ring);
}

// ------------------------------------------------------------ S4: vote
// The election of sub-job k-3 (vote_one), over the live pedestrians in bin order.
__global__ void k_vote(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                       int nbins, const int2* __restrict__ xy, const uint8_t* __restrict__ choice,
                       const int32_t* __restrict__ occ, Geo g, uint64_t seed, Counters* ctr,
                       uint8_t* __restrict__ won, Sizes sz, const int32_t* __restrict__ gid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= bin_start[nbins]) return;
  const int regs = sz.w ? vote_one_sized(rec_id[i], g, xy, choice, occ, sz.w, sz.h, seed, ctr->t, won)
                        : vote_one(rec_id[i], 0, g, xy, choice, occ, seed, ctr->t, won, gid);
  if (regs > 2) atomicMax(&ctr->max_registrants, regs);
  if (regs > 8) atomicOr(&ctr->err, kErrEnroll);
}

void launch_vote(int n, const int32_t* rec_id, const int32_t* bin_start, const int2* xy,
                 const uint8_t* choice, const int32_t* occ, const Geo& g, uint64_t seed,
                 Counters* ctr, uint8_t* won, cudaStream_t s, const Sizes& sz,
                 const int32_t* gid) {
  if (n <= 0) return;
  k_vote<<<cdiv(n, 256), 256, 0, s>>>(rec_id, bin_start, g.nbx * g.nby, xy, choice, occ, g, seed,
                                      ctr, won, sz, gid);
}

// ---------------------------------------------------------- S5: commit
__global__ void k_commit(const int32_t* __restrict__ rec_id, const int32_t* __restrict__ bin_start,
                         int nbins, int2* __restrict__ xy, uint8_t* __restrict__ alive,
                         uint8_t* __restrict__ heading, const uint8_t* __restrict__ choice,
                         const uint8_t* __restrict__ won, const uint8_t* __restrict__ cell,
                         int32_t* __restrict__ occ, uint8_t* __restrict__ ocls, Geo g,
                         Counters* ctr, Sizes sz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool moved = false, left = false;
  if (i < bin_start[nbins]) {
    if (sz.w)
      commit_one_sized(rec_id[i], g, xy, alive, heading, choice, won, cell, occ, ocls, sz.w, sz.h,
                       moved, left);
    else
      commit_one(rec_id[i], g, xy, alive, heading, choice, won, cell, occ, ocls, moved, left);
  }
  const unsigned nm = __popc(__ballot_sync(0xffffffffu, moved));
  const unsigned nl = __popc(__ballot_sync(0xffffffffu, left));
  if ((threadIdx.x & 31) == 0) {
    if (nm) atomicAdd(&ctr->moved, (unsigned long long)nm);
    if (nl) atomicAdd(&ctr->exited, (unsigned long long)nl);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr->t += 1;
}

void launch_commit(int n, const int32_t* rec_id, const int32_t* bin_start, int2* xy,
                   uint8_t* alive, uint8_t* heading, const uint8_t* choice, const uint8_t* won,
                   const uint8_t* cell, int32_t* occ, uint8_t* ocls, const Geo& g, Counters* ctr,
                   cudaStream_t s, const Sizes& sz) {
  const int blocks = n > 0 ? cdiv(n, 256) : 1;
  k_commit<<<blocks, 256, 0, s>>>(rec_id, bin_start, g.nbx * g.nby, xy, alive, heading, choice,
                                  won, cell, occ, ocls, g, ctr, sz);
}

}  // namespace sfm
