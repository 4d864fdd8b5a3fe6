// sfm_ctx.h -- host-side context of the C ABI (one lattice, or a batch of
// independent lattices stepped by one persistent launch per tick).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sfm_internal.h"

struct sfm_ctx;
namespace sfm {
struct BatchState;  // sfm_batch.cu
sfm_status compute_guidance(const Geo& g, const uint8_t* cell, int32_t* D, cudaStream_t s,
                            std::string* err);
// message returned by sfm_last_error(NULL) on this thread
void set_create_error(const std::string& msg);
// bins of the context's current state (S1), field rows (S2) into `out`
void ctx_run_bins(sfm_ctx* c);
void ctx_field_rows(sfm_ctx* c, float* out, int ya, int yb, int main_off, bool halos);
// batched lattices (sfm_batch.cu)
sfm_status batch_tick(sfm_ctx* ctx, int nsteps, int field_only);
sfm_status batch_sync(sfm_ctx* ctx);
void batch_destroy(sfm_ctx* ctx);
}  // namespace sfm

struct sfm_ctx {
  sfm_lattice lat{};
  sfm_params prm{};
  cudaStream_t stream = nullptr;
  sfm::Geo geo{};
  std::string err;
  int64_t device_bytes = 0;
  int64_t nsu_total = 0;  // su of all lattice arrays (W*H, or the batch's sum)
  int64_t launches = 0;  // kernels launched by this context
  std::vector<void*> allocs;

  // lattice arrays
  uint8_t* cell = nullptr;
  float* Fs = nullptr;
  float* F = nullptr;  // full-lattice field (unbanded mode only)
  int32_t* D = nullptr;
  int32_t* occ = nullptr;
  uint8_t* ocls = nullptr;
  // tables
  float *T0 = nullptr, *TX = nullptr, *TY = nullptr, *KO = nullptr, *KE = nullptr;
  float *own = nullptr, *dirdot = nullptr;
  float2* hvec = nullptr;
  float* CT = nullptr;  // heading-class tables of the v2 gather
  float* CT3 = nullptr;  // the same in the row-trimmed gather's layout (radius 1..48)
  int field_shape = 0;  // footprint of the class-table gather (0: 16x16, 1: 32x16)
  // bins
  int32_t *bin_count = nullptr, *bin_start = nullptr, *scan_tmp = nullptr;
  uint32_t* rec = nullptr;
  int32_t* rec_id = nullptr;  // pedestrian of each bin record
  int32_t* bin_slot = nullptr;  // pedestrian-list binning: arrival slot in the bin
  uint32_t* bin_key = nullptr;  // pedestrian-list binning: su keys in slot order
  int binning = 0;              // 0 automatic, 1 class grid, 2 pedestrian list
  sfm::Counters* ctr = nullptr;
  // pedestrians
  int n = 0, cap = 0;
  int2* xy = nullptr;
  uint8_t *heading = nullptr, *goal = nullptr, *alive = nullptr, *choice = nullptr, *won = nullptr;
  uint8_t *period = nullptr, *phase = nullptr;  // walk periods (used when walk_periods)
  bool walk_periods = false;
  int32_t* gid = nullptr;  // caller's pedestrian numbers for the election (used when has_ids)
  bool has_ids = false;
  uint8_t *pw = nullptr, *ph = nullptr;  // multi-su pedestrians' widths / heights (when sized)
  // placement scratch (place_impl): the state before a placement that keeps
  // the tick graphs, or the new state staged from the caller's buffers
  int2* pl_xy = nullptr;
  uint8_t *pl_alive = nullptr, *pl_heading = nullptr, *pl_goal = nullptr;
  bool sized = false;
  bool placed = false;
  int64_t t = 0;
  // banded mode
  int bands = 1;
  int band_rows = 0;  // lattice rows per band (multiple of the tile height)
  float* band_buf = nullptr;
  // timing: stage events on every timing_every-th tick (0: none); `timing`
  // says whether the tick being launched records them
  bool timing = false;
  int timing_every = 0;
  int64_t timing_phase = 0;  // ticks since the last timed one, mod timing_every
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t timed_ticks = 0;
  // one timed tick captured as a CUDA graph whose stage events are event
  // record nodes; before each replay the nodes are pointed at fresh events
  struct TimedNode {
    int stage;
    cudaGraphNode_t a, b;
  };
  bool capturing_timed = false;  // StageScope records capture-external events
  cudaGraph_t timed_tmpl = nullptr;  // kept: the event nodes belong to it
  cudaGraphExec_t timed_graph = nullptr;
  int64_t timed_launches = 0;
  std::vector<TimedNode> timed_nodes;
  std::vector<cudaEvent_t> timed_placeholders;  // events recorded during the capture
  // one tick captured as a CUDA graph (single lattice, untimed ticks)
  cudaGraphExec_t tick_graph = nullptr;
  int64_t graph_launches = 0;  // kernels in one replay of tick_graph
  cudaGraphExec_t block_graph = nullptr;  // kBlockTicks ticks in one graph
  int64_t block_launches = 0;
  int64_t direct_ticks = 0;    // ticks launched stage by stage since placement
  // batch of independent lattices (nullptr for a single lattice)
  sfm::BatchState* batch = nullptr;

  sfm::Tables tables() const {
    sfm::Tables tb;
    tb.T0 = T0;
    tb.TX = TX;
    tb.TY = TY;
    tb.KO = KO;
    tb.KE = KE;
    tb.own = own;
    tb.dirdot = dirdot;
    tb.hvec = hvec;
    tb.CT = CT;
    tb.CT3 = CT3;
    tb.shape = field_shape;
    return tb;
  }
  sfm::Sizes sizes() const {
    sfm::Sizes sz;
    if (sized) {
      sz.w = pw;
      sz.h = ph;
    }
    return sz;
  }
  const int32_t* ids() const { return has_ids ? gid : nullptr; }
  sfm::WalkPeriods walk() const {
    sfm::WalkPeriods wp;
    if (walk_periods) {
      wp.period = period;
      wp.phase = phase;
      wp.ctr = ctr;
    }
    return wp;
  }
};

