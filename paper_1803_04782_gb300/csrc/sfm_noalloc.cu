// sfm_noalloc.cu -- pedestrian-field superposition without any device
// allocation, for callers that cannot call cudaMalloc: for example a host
// application or framework that reserves all device memory up front in its
// own pool and forbids (or cannot afford the synchronisation of) further
// allocations while it runs.
//
// The working memory of this entry point (bin counts, bin starts, scan
// temporaries, bin records, kernel tables) lives in one file-scope device
// array of fixed size, g_noalloc_scratch, which every GPU that loads the
// library holds until the process exits.  The caller passes inputs and the
// output; nothing else is allocated.  All calls share the array: calls that
// overlap on the GPU (on different streams, or from different host threads)
// race and must not be issued.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "sfm_internal.h"

using namespace sfm;

namespace {

// Layout of the scratch array, in 32-bit words.
constexpr int kNaBins = SFM_NOALLOC_MAX_BINS;
constexpr int kNaPeds = SFM_NOALLOC_MAX_PEDS;
constexpr size_t kNaCount = 0;                          // per-bin counts
constexpr size_t kNaCursor = kNaCount + kNaBins;        // per-bin fill cursors
constexpr size_t kNaStart = kNaCursor + kNaBins;        // bin starts (kNaBins + 1)
constexpr size_t kNaScanTmp = kNaStart + kNaBins + 64;  // scan block totals
constexpr size_t kNaErr = kNaScanTmp + 64;              // error word
constexpr size_t kNaRec = kNaErr + 64;                  // bin records
constexpr size_t kNaTables = kNaRec + kNaPeds;          // heading-class tables
constexpr size_t kNaTableFloats = max_class_table_floats(SFM_NOALLOC_MAX_RADIUS);
constexpr size_t kNaWords = (kNaTables + kNaTableFloats + 63) / 64 * 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
uint32_t* g_na_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device (the first call on a device does it).
sfm_status na_scratch(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SFM_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return SFM_ECUDA;
    g_na_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_na_ptr[dev];
  return SFM_OK;
}

__device__ __forceinline__ bool na_valid(const int2 q, const Geo& g, const uint8_t* heading, int p,
                                         uint32_t* err) {
  const bool ok = q.x >= 0 && q.x < g.W && q.y >= 0 && q.y < g.H &&
                  (heading == nullptr || heading[p] <= 8);
  if (!ok) atomicOr(err, 1u);
  return ok;
}

__global__ void k_na_count(int n, const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
                           const uint8_t* __restrict__ alive, Geo g, int32_t* __restrict__ count,
                           uint32_t* __restrict__ err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || (alive && !alive[p])) return;
  const int2 q = xy[p];
  if (!na_valid(q, g, heading, p, err)) return;
  atomicAdd(&count[(q.y / kBin) * g.nbx + q.x / kBin], 1);
}

// Records in arrival order inside a bin: the sum over a bin's pedestrians is
// then taken in an unspecified order (equal to the context path's up to
// rounding).
__global__ void k_na_fill(int n, const int2* __restrict__ xy, const uint8_t* __restrict__ heading,
                          const uint8_t* __restrict__ alive, Geo g,
                          const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                          uint32_t* __restrict__ rec, uint32_t* __restrict__ err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || (alive && !alive[p])) return;
  const int2 q = xy[p];
  if (!na_valid(q, g, heading, p, err)) return;
  const int b = (q.y / kBin) * g.nbx + q.x / kBin;
  const int slot = atomicAdd(&cursor[b], 1);
  const uint32_t cls = heading ? heading[p] : 0u;
  rec[start[b] + slot] = (uint32_t)(q.x % kBin) | ((uint32_t)(q.y % kBin) << 8) | (cls << 16);
}

}  // namespace

extern "C" sfm_status sfm_field_noalloc(const sfm_lattice* lat, const sfm_params* prm, int32_t n,
                                        const int32_t* xy, const uint8_t* heading,
                                        const uint8_t* alive, const float* base, float* field,
                                        void* stream) {
  if (!lat || !prm || !base || !field || (n > 0 && !xy)) return SFM_EINVAL;
  if (lat->W < 3 || lat->H < 3) return SFM_EINVAL;
  if ((int64_t)lat->W * lat->H > ((int64_t)1 << 31)) return SFM_EINVAL;
  if (prm->r < 0 || prm->r > SFM_NOALLOC_MAX_RADIUS) return SFM_EINVAL;
  if ((lat->periodic_x && lat->W < 2 * prm->r + 1) || (lat->periodic_y && lat->H < 2 * prm->r + 1))
    return SFM_EINVAL;
  if (n < 0 || n > SFM_NOALLOC_MAX_PEDS) return SFM_EINVAL;
  Geo g{};
  g.W = lat->W;
  g.H = lat->H;
  g.px = lat->periodic_x ? 1 : 0;
  g.py = lat->periodic_y ? 1 : 0;
  g.r = prm->r;
  g.nbx = (g.W + kBin - 1) / kBin;
  g.nby = (g.H + kBin - 1) / kBin;
  g.opitch = (g.W + 127) / 128 * 128;
  const int nbins = g.nbx * g.nby;
  if (nbins > SFM_NOALLOC_MAX_BINS) return SFM_EINVAL;

  uint32_t* S = nullptr;
  sfm_status st = na_scratch(&S);
  if (st != SFM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* count = reinterpret_cast<int32_t*>(S + kNaCount);
  int32_t* cursor = reinterpret_cast<int32_t*>(S + kNaCursor);
  int32_t* start = reinterpret_cast<int32_t*>(S + kNaStart);
  int32_t* scan_tmp = reinterpret_cast<int32_t*>(S + kNaScanTmp);
  uint32_t* err = S + kNaErr;
  uint32_t* rec = S + kNaRec;
  float* tables = reinterpret_cast<float*>(S + kNaTables);

  // what must start at zero: counts, cursors and the error word
  if (cudaMemsetAsync(count, 0, sizeof(int32_t) * 2 * (size_t)kNaBins, s) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess)
    return SFM_ECUDA;
  const int2* pxy = reinterpret_cast<const int2*>(xy);
  if (n > 0) k_na_count<<<(n + 255) / 256, 256, 0, s>>>(n, pxy, heading, alive, g, count, err);
  launch_scan(count, start, nbins, scan_tmp, s);
  if (n > 0)
    k_na_fill<<<(n + 255) / 256, 256, 0, s>>>(n, pxy, heading, alive, g, start, cursor, rec, err);
  launch_class_tables(g.r, *prm, tables, s);
  Tables tb{};
  tb.CT = tables;
  tb.shape = default_field_shape(g.r);
  launch_field(g, start, rec, tb, base, field, 0, 0, g.H, nullptr, s);

  uint32_t h_err = 0;
  cudaError_t e = cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return SFM_ECUDA;
  if (h_err) return SFM_ECONFLICT;  // a live pedestrian off-lattice or with a class > 8
  return SFM_OK;
}
