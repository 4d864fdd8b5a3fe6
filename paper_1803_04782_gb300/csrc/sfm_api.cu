// sfm_api.cu -- C ABI (include/sfm.h): context lifetime, validation, device
// memory, and the per-tick launch sequence of Alg. 1 (bins, field gather,
// decision, vote, commit), with the banded divide-and-conquer mode of Sec. 3.3.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sfm_ctx.h"

using namespace sfm;

namespace {

thread_local std::string g_create_err;

sfm_status fail(sfm_ctx* c, sfm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_err = buf;
  return st;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SFM_ENOMEM : SFM_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                        \
  } while (0)

template <class T>
sfm_status dalloc(sfm_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess)
    return fail(ctx, SFM_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  ctx->allocs.push_back(q);
  ctx->device_bytes += (int64_t)bytes;
  *p = static_cast<T*>(q);
  return SFM_OK;
}

void dfree(sfm_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->allocs.size(); ++i)
    if (ctx->allocs[i] == p) {
      ctx->allocs.erase(ctx->allocs.begin() + (long)i);
      break;
    }
  cudaFree(p);
}

#define TRY(x)                     \
  do {                             \
    sfm_status s_ = (x);           \
    if (s_ != SFM_OK) return s_;   \
  } while (0)

cudaEvent_t pool_get(sfm_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct StageScope {
  sfm_ctx* c;
  int stage;
  cudaEvent_t a = nullptr;
  StageScope(sfm_ctx* c_, int s_) : c(c_), stage(s_) {
    if (c->timing) {
      a = pool_get(c);
      record(a);
    }
  }
  ~StageScope() {
    if (c->timing) {
      cudaEvent_t b = pool_get(c);
      record(b);
      c->recs.push_back({stage, a, b});
    }
  }
  // under the capture of the timed tick graph an event becomes a record node
  void record(cudaEvent_t e) {
    if (c->capturing_timed)
      cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, c->stream);
  }
};

sfm_status check_flags(sfm_ctx* ctx) {
  CU(cudaStreamSynchronize(ctx->stream));
  Counters h;
  CU(cudaMemcpy(&h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.err & kErrTimeout) return fail(ctx, SFM_ETIMEOUT, "a bounded device wait gave up");
  if (h.err) return fail(ctx, SFM_ECUDA, "device error flags 0x%x", h.err);
  return SFM_OK;
}

// Field of the current pedestrian state for lattice rows [ya, yb) stored in
// out with row ya at out row `main_off`; optionally the single halo rows
// ya-1 and yb (wrapped in periodic y) at out rows 0 and yb-ya+1.  Uses whole
// tiles so every su is summed in the same order in every mode.
void field_rows(sfm_ctx* c, float* out, int ya, int yb, int main_off, bool halos) {
  const Geo& g = c->geo;
  const Tables tb = c->tables();
  if (!halos) {
    launch_field(g, c->bin_start, c->rec, tb, c->Fs, out, ya - main_off, ya, yb, c->ctr,
                 c->stream);
    ++c->launches;
    return;
  }
  // one launch for the band and its in-lattice halo rows ya-1 and yb (out rows
  // 0 and yb-ya+1 follow from the same row mapping, main_off == 1)
  const int lo = ya - 1 >= 0 ? ya - 1 : 0, hi = yb + 1 <= g.H ? yb + 1 : g.H;
  launch_field(g, c->bin_start, c->rec, tb, c->Fs, out, ya - main_off, lo, hi, c->ctr,
               c->stream);
  ++c->launches;
  // halo rows that wrap around a periodic y boundary
  if (g.py && ya == 0) {
    launch_field(g, c->bin_start, c->rec, tb, c->Fs, out, g.H - 1, g.H - 1, g.H, c->ctr,
                 c->stream);
    ++c->launches;
  }
  if (g.py && yb == g.H) {
    launch_field(g, c->bin_start, c->rec, tb, c->Fs, out, -(yb - ya + 1), 0, 1, c->ctr,
                 c->stream);
    ++c->launches;
  }
}

// Pedestrian-list binning when the crowd is sparse: its cost follows the
// pedestrians (tens of bytes each), the grid scan's the area (2 bytes per su).
bool bins_from_peds(const sfm_ctx* c) {
  if (c->binning) return c->binning == 2;
  return (int64_t)c->n * 64 < (int64_t)c->geo.W * c->geo.H;
}

void run_bins(sfm_ctx* c) {
  StageScope sc(c, SFM_STAGE_BIN);
  const Geo& g = c->geo;
  // the bin scan: three passes, or one when a block covers every bin
  const int scan_launches = scan_tmp_elems(g.nbx * g.nby) == 1 ? 1 : 3;
  if (bins_from_peds(c)) {
    launch_bins_from_peds(g, c->n, c->xy, c->alive, c->heading, c->bin_count, c->bin_start,
                          c->scan_tmp, c->bin_slot, c->bin_key, c->rec, c->rec_id, c->stream);
    c->launches += (c->n > 0 ? 3 : 0) + scan_launches;  // count, scan, scatter, rank
    return;
  }
  launch_bin_count(g, c->ocls, c->bin_count, c->stream);
  launch_scan(c->bin_count, c->bin_start, g.nbx * g.nby, c->scan_tmp, c->stream);
  launch_bin_fill(g, c->ocls, c->occ, c->bin_start, c->rec, c->rec_id, c->stream);
  c->launches += 2 + scan_launches;  // count, scan, fill
}

void run_tick(sfm_ctx* c) {
  StageScope whole(c, SFM_STAGE_STEP);
  const Geo& g = c->geo;
  const Tables tb = c->tables();
  const int nbins = g.nbx * g.nby;
  {
    StageScope sc(c, SFM_STAGE_BIN);
    launch_clear_dead(c->n, c->alive, c->choice, c->won, c->stream);
    if (c->n > 0) ++c->launches;
  }
  run_bins(c);
  if (c->bands <= 1) {
    {
      StageScope sc(c, SFM_STAGE_FIELD);
      field_rows(c, c->F, 0, g.H, 0, false);
    }
    StageScope sc(c, SFM_STAGE_DECIDE);
    launch_decide(c->n, c->rec_id, c->bin_start, 0, nbins, c->xy, c->heading, c->goal, c->cell,
                  c->ocls, c->D, c->F, 0, -1, -1, 0, 0, g.H, g, c->prm.beta, tb, c->choice,
                  c->stream, c->walk(), c->sizes(), c->occ, c->ctr);
    if (c->n > 0) ++c->launches;
  } else if (!g.py && field3_shape_ok(tb.shape, g.r) && tb.CT3) {
    // The band buffer as a ring of R = band rows + 33 rows, lattice row y at
    // ring row y mod R.  Band b's launch stores the rows no earlier launch
    // stored, through the first tile row of band b + 1 (the lower halo row
    // yb and the 32 rows the next band's decisions start on); the upper halo
    // row ya - 1 and the band's first tile row come from band b - 1's
    // launch.  So every tile row of the lattice is gathered once a tick, and
    // the rows that band b's decisions read, [ya - 1, yb], are all in the
    // ring: band b's launch overwrites the rows before ya - 1 only.
    const int R = c->band_rows + kBandExtraRows;
    for (int b = 0; b < c->bands; ++b) {
      const int ya = b * c->band_rows;
      const int yb = ya + c->band_rows < g.H ? ya + c->band_rows : g.H;
      const int s_lo = b == 0 ? 0 : (ya + kTile < g.H ? ya + kTile : g.H);
      const int s_hi = yb + kTile < g.H ? yb + kTile : g.H;
      if (s_hi > s_lo) {
        StageScope sc(c, SFM_STAGE_FIELD);
        launch_field(g, c->bin_start, c->rec, tb, c->Fs, c->band_buf, s_lo - s_lo % R, s_lo, s_hi,
                     c->ctr, c->stream, FarPart(), R);
        ++c->launches;
      }
      const int y_lo = ya > 0 ? ya - 1 : 0, y_hi = yb + 1 < g.H ? yb + 1 : g.H;
      StageScope sc(c, SFM_STAGE_DECIDE);
      launch_decide(c->n, c->rec_id, c->bin_start, (ya / kBin) * g.nbx,
                    ((yb + kBin - 1) / kBin) * g.nbx, c->xy, c->heading, c->goal, c->cell, c->ocls,
                    c->D, c->band_buf, y_lo % R, -1, -1, 0, y_lo, y_hi, g, c->prm.beta, tb,
                    c->choice, c->stream, c->walk(), c->sizes(), c->occ, c->ctr, R);
      if (c->n > 0) ++c->launches;
    }
  } else {
    for (int b = 0; b < c->bands; ++b) {
      const int ya = b * c->band_rows;
      const int yb = ya + c->band_rows < g.H ? ya + c->band_rows : g.H;
      {
        StageScope sc(c, SFM_STAGE_FIELD);
        field_rows(c, c->band_buf, ya, yb, 1, true);
      }
      int lo = ya - 1, hi = yb;
      if (lo < 0) lo = g.py ? lo + g.H : -1;
      if (hi >= g.H) hi = g.py ? hi - g.H : -1;
      StageScope sc(c, SFM_STAGE_DECIDE);
      launch_decide(c->n, c->rec_id, c->bin_start, (ya / kBin) * g.nbx,
                    ((yb + kBin - 1) / kBin) * g.nbx, c->xy, c->heading, c->goal, c->cell, c->ocls,
                    c->D, c->band_buf, 1, lo, hi, yb - ya + 1, ya, yb, g, c->prm.beta, tb,
                    c->choice, c->stream, c->walk(), c->sizes(), c->occ, c->ctr);
      if (c->n > 0) ++c->launches;
    }
  }
  {
    StageScope sc(c, SFM_STAGE_VOTE);
    launch_vote(c->n, c->rec_id, c->bin_start, c->xy, c->choice, c->occ, g, c->prm.seed, c->ctr,
                c->won, c->stream, c->sizes(), c->ids());
    if (c->n > 0) ++c->launches;
  }
  StageScope sc(c, SFM_STAGE_COMMIT);
  launch_commit(c->n, c->rec_id, c->bin_start, c->xy, c->alive, c->heading, c->choice, c->won,
                c->cell, c->occ, c->ocls, g, c->ctr, c->stream, c->sizes());
  ++c->launches;
}

void drop_graph(sfm_ctx* c) {
  if (c->tick_graph) cudaGraphExecDestroy(c->tick_graph);
  c->tick_graph = nullptr;
  if (c->block_graph) cudaGraphExecDestroy(c->block_graph);
  c->block_graph = nullptr;
  if (c->timed_graph) cudaGraphExecDestroy(c->timed_graph);
  c->timed_graph = nullptr;
  if (c->timed_tmpl) cudaGraphDestroy(c->timed_tmpl);
  c->timed_tmpl = nullptr;
  c->timed_nodes.clear();
  for (cudaEvent_t e : c->timed_placeholders) cudaEventDestroy(e);
  c->timed_placeholders.clear();
  c->direct_ticks = 0;
}

// Capture one tick (all its launches, on a private stream) into a graph.
// Runs of at least this many ticks replay one graph holding that many ticks
// (fewer launches for small lattices, where launching dominates).
constexpr int kBlockTicks = 8;

// Capture `ticks` ticks (all their launches, on a private stream) into a graph.
cudaError_t build_tick_graph(sfm_ctx* c, int ticks, cudaGraphExec_t* exec, int64_t* launches) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaStream_t saved = c->stream;
  const int64_t l0 = c->launches;
  cudaGraph_t graph = nullptr;
  c->stream = cs;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int i = 0; i < ticks; ++i) run_tick(c);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    e = e2;
  }
  c->stream = saved;
  *launches = c->launches - l0;
  c->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) *exec = nullptr;
  return e;
}

// Capture one tick with its stage events as event record nodes (the timed
// tick graph), and find each stage's pair of nodes.
cudaError_t build_timed_graph(sfm_ctx* c) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaStream_t saved = c->stream;
  const int64_t l0 = c->launches;
  const size_t r0 = c->recs.size();
  cudaGraph_t graph = nullptr;
  c->stream = cs;
  c->capturing_timed = true;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    run_tick(c);
    e = cudaStreamEndCapture(cs, &graph);
  }
  c->capturing_timed = false;
  c->stream = saved;
  c->timed_launches = c->launches - l0;
  c->launches = l0;
  // the capture's events stay with the graph (its nodes name them until the
  // first replay points them elsewhere)
  std::vector<sfm_ctx::Rec> cap(c->recs.begin() + (long)r0, c->recs.end());
  c->recs.resize(r0);
  for (const auto& r : cap) {
    c->timed_placeholders.push_back(r.a);
    c->timed_placeholders.push_back(r.b);
  }
  if (e == cudaSuccess) {
    size_t nn = 0;
    e = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
    std::vector<std::pair<cudaEvent_t, cudaGraphNode_t>> ev;
    for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      cudaEvent_t x = nullptr;
      if (e == cudaSuccess && t == cudaGraphNodeTypeEventRecord) {
        e = cudaGraphEventRecordNodeGetEvent(nodes[i], &x);
        ev.push_back({x, nodes[i]});
      }
    }
    auto node_of = [&](cudaEvent_t x) -> cudaGraphNode_t {
      for (const auto& p : ev)
        if (p.first == x) return p.second;
      return nullptr;
    };
    for (const auto& r : cap) {
      const cudaGraphNode_t na = node_of(r.a), nb = node_of(r.b);
      if (!na || !nb) {
        if (e == cudaSuccess) e = cudaErrorInvalidValue;
        break;
      }
      c->timed_nodes.push_back({r.stage, na, nb});
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->timed_graph, graph, 0);
  if (e == cudaSuccess) {
    c->timed_tmpl = graph;
  } else {
    if (graph) cudaGraphDestroy(graph);
    c->timed_graph = nullptr;
    c->timed_nodes.clear();
  }
  cudaStreamDestroy(cs);
  return e;
}

// Every graph sfm_step replays, built together the first time one is needed
// after a placement: the one-tick and kBlockTicks-tick graphs and, with
// timing on, the timed one-tick graph; so no capture happens in the middle
// of a run of replays that someone is timing.
sfm_status ensure_graphs(sfm_ctx* c) {
  const bool saved = c->timing;
  cudaError_t e = cudaSuccess;
  c->timing = false;
  if (!c->tick_graph) e = build_tick_graph(c, 1, &c->tick_graph, &c->graph_launches);
  if (e == cudaSuccess && !c->block_graph)
    e = build_tick_graph(c, kBlockTicks, &c->block_graph, &c->block_launches);
  c->timing = true;
  if (e == cudaSuccess && c->timing_every > 0 && !c->timed_graph) e = build_timed_graph(c);
  c->timing = saved;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SFM_ECUDA, "tick graph: %s", cudaGetErrorString(e));
  }
  return SFM_OK;
}

// One replay of the timed tick graph, its stage nodes on fresh events.
cudaError_t replay_timed_tick(sfm_ctx* c) {
  for (const auto& n : c->timed_nodes) {
    const cudaEvent_t a = pool_get(c), b = pool_get(c);
    cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(c->timed_graph, n.a, a);
    if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(c->timed_graph, n.b, b);
    if (e != cudaSuccess) {
      c->pool.push_back(a);
      c->pool.push_back(b);
      return e;
    }
    c->recs.push_back({n.stage, a, b});
  }
  return cudaGraphLaunch(c->timed_graph, c->stream);
}

// Address under which the device reads or writes a caller's buffer in place:
// the pointer itself for device memory, the mapped address of pinned host
// memory (cudaHostAlloc / cudaMallocHost / cudaHostRegister with unified
// addressing); NULL for pageable host memory, which is copied instead.
void* device_view(const void* p, int on_device) {
  if (!p) return nullptr;
  if (on_device) return const_cast<void*>(p);
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer: not an error of this context
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

sfm_status copy_out(sfm_ctx* ctx, void* dst, const void* src, size_t bytes, int on_device) {
  CU(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  return check_flags(ctx);
}

}  // namespace

void sfm::set_create_error(const std::string& msg) { g_create_err = msg; }
void sfm::ctx_run_bins(sfm_ctx* c) { run_bins(c); }
void sfm::ctx_field_rows(sfm_ctx* c, float* out, int ya, int yb, int main_off, bool halos) {
  field_rows(c, out, ya, yb, main_off, halos);
}

// Guidance distances of one lattice: relaxation rounds until no tile changes
// (at most 4 * tiles + 256 rounds, then SFM_ETIMEOUT).
sfm_status sfm::compute_guidance(const Geo& g, const uint8_t* cell, int32_t* D, cudaStream_t s,
                                 std::string* err) {
  const int ntiles = ((g.W + kTile - 1) / kTile) * ((g.H + kTile - 1) / kTile);
  uint8_t *a0 = nullptr, *a1 = nullptr;
  int* changed = nullptr;
  if (cudaMalloc(&a0, ntiles) != cudaSuccess || cudaMalloc(&a1, ntiles) != cudaSuccess ||
      cudaMalloc(&changed, sizeof(int)) != cudaSuccess) {
    cudaFree(a0);
    cudaFree(a1);
    if (err) *err = "guidance scratch allocation failed";
    return SFM_ENOMEM;
  }
  launch_guidance_init(g, cell, D, s);
  cudaMemsetAsync(a0, 1, ntiles, s);
  int h_changed = 1, rounds = 0;
  const int max_rounds = 4 * ntiles + 256;
  while (h_changed && rounds < max_rounds) {
    cudaMemsetAsync(a1, 0, ntiles, s);
    cudaMemsetAsync(changed, 0, sizeof(int), s);
    launch_guidance_round(g, cell, D, a0, a1, changed, s);
    cudaMemcpyAsync(&h_changed, changed, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    uint8_t* tmp = a0;
    a0 = a1;
    a1 = tmp;
    ++rounds;
  }
  cudaFree(a0);
  cudaFree(a1);
  cudaFree(changed);
  if (h_changed) {
    if (err) *err = "guidance relaxation did not converge";
    return SFM_ETIMEOUT;
  }
  return SFM_OK;
}

extern "C" {

int32_t sfm_abi_version(void) { return SFM_ABI_VERSION; }

uint64_t sfm_resident_bytes(const sfm_lattice* lat) {
  if (!lat || lat->W <= 0 || lat->H <= 0) return 0;
  const uint64_t nsu = (uint64_t)lat->W * lat->H;
  const uint64_t opitch = ((uint64_t)lat->W + 127) / 128 * 128;
  return nsu * (1 + 4 + 4 + 4) + opitch * lat->H;
}

const char* sfm_last_error(const sfm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

sfm_status sfm_create(const sfm_lattice* lat, const uint8_t* cell, int32_t cell_on_device,
                      const sfm_params* prm, void* stream, sfm_ctx** out) {
  if (out) *out = nullptr;
  if (!lat || !cell || !prm || !out) return fail(nullptr, SFM_EINVAL, "NULL argument");
  if (lat->W < 3 || lat->H < 3) return fail(nullptr, SFM_EINVAL, "lattice must be >= 3x3");
  if ((int64_t)lat->W * lat->H > (int64_t)1 << 31)
    return fail(nullptr, SFM_EINVAL, "lattice larger than 2^31 su");
  if (prm->r < 0 || prm->r > SFM_MAX_RADIUS)
    return fail(nullptr, SFM_EINVAL, "radius %d outside [0, %d]", prm->r, SFM_MAX_RADIUS);
  if ((lat->periodic_x && lat->W < 2 * prm->r + 1) || (lat->periodic_y && lat->H < 2 * prm->r + 1))
    return fail(nullptr, SFM_EINVAL, "a periodic extent must be >= 2r+1");
  if (prm->bin != 0 && prm->bin != kBin)
    return fail(nullptr, SFM_EINVAL, "bin side must be 0 or %d", kBin);

  sfm_ctx* ctx = new sfm_ctx;
  ctx->lat = *lat;
  ctx->nsu_total = (int64_t)lat->W * lat->H;
  ctx->field_shape = default_field_shape(prm->r);
  ctx->prm = *prm;
  ctx->prm.bin = kBin;
  ctx->stream = static_cast<cudaStream_t>(stream);
  Geo& g = ctx->geo;
  g.W = lat->W;
  g.H = lat->H;
  g.px = lat->periodic_x ? 1 : 0;
  g.py = lat->periodic_y ? 1 : 0;
  g.r = prm->r;
  g.nbx = (g.W + kBin - 1) / kBin;
  g.nby = (g.H + kBin - 1) / kBin;
  g.opitch = (g.W + 127) / 128 * 128;
  const size_t nsu = (size_t)g.W * g.H;
  const int nbins = g.nbx * g.nby;
  const int S = 2 * g.r + 1;

  auto bail = [&](sfm_status st) {
    g_create_err = ctx->err;
    sfm_destroy(ctx);
    return st;
  };
  // resident lattice arrays: cell, static field, guidance, occupancy, class grid
  const uint64_t resident = sfm_resident_bytes(lat);
  const uint64_t budget = prm->hbm_budget_bytes;
  if (budget && resident + (uint64_t)nsu * 4 > budget) {
    // banded: rows per band from what the budget leaves for the band buffer
    if (resident >= budget) {
      fail(ctx, SFM_EBUDGET, "resident arrays need %llu bytes > budget %llu",
           (unsigned long long)resident, (unsigned long long)budget);
      return bail(SFM_EBUDGET);
    }
    int64_t rows = (int64_t)((budget - resident) / ((uint64_t)g.W * 4)) - kBandExtraRows;
    rows = rows / kTile * kTile;
    if (rows < kTile) {
      fail(ctx, SFM_EBUDGET, "budget leaves room for fewer than %d field rows", kTile);
      return bail(SFM_EBUDGET);
    }
    ctx->band_rows = (int)rows;
    ctx->bands = (int)((g.H + rows - 1) / rows);
  }
  sfm_status st;
#define ALLOC(p, n)                              \
  if ((st = dalloc(ctx, &(p), (n))) != SFM_OK) \
    return bail(st);
  ALLOC(ctx->cell, nsu);
  ALLOC(ctx->Fs, nsu);
  ALLOC(ctx->D, nsu);
  ALLOC(ctx->occ, nsu);
  ALLOC(ctx->ocls, (size_t)g.opitch * g.H);
  if (ctx->bands <= 1) {
    ALLOC(ctx->F, nsu);
  } else {
    ALLOC(ctx->band_buf, (size_t)(ctx->band_rows + kBandExtraRows) * g.W);
  }
  ALLOC(ctx->T0, (size_t)S * S);
  ALLOC(ctx->TX, (size_t)S * S);
  ALLOC(ctx->TY, (size_t)S * S);
  ALLOC(ctx->KO, (size_t)S * S);
  ALLOC(ctx->KE, (size_t)S * S);
  ALLOC(ctx->own, 81);
  ALLOC(ctx->dirdot, 81);
  ALLOC(ctx->hvec, 9);
  if (class_table_floats(g.r)) ALLOC(ctx->CT, class_table_floats(g.r));
  if (field3_table_floats(g.r)) ALLOC(ctx->CT3, field3_table_floats(g.r));
  ALLOC(ctx->bin_count, (size_t)nbins);
  ALLOC(ctx->bin_start, (size_t)nbins + 1);
  ALLOC(ctx->scan_tmp, (size_t)scan_tmp_elems(nbins));
  ALLOC(ctx->ctr, 1);
#undef ALLOC

  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(ctx->cell, cell, nsu,
                                  cell_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    fail(ctx, SFM_ECUDA, "copy cell: %s", cudaGetErrorString(e));
    return bail(SFM_ECUDA);
  }
  cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), s);
  cudaMemsetAsync(ctx->occ, 0xff, nsu * sizeof(int32_t), s);
  cudaMemsetAsync(ctx->ocls, 0, (size_t)g.opitch * g.H, s);
  launch_tables(g.r, ctx->prm, ctx->T0, ctx->TX, ctx->TY, ctx->KO, ctx->KE, ctx->own, ctx->dirdot,
                ctx->hvec, s);
  if (ctx->CT) launch_class_tables(g.r, ctx->prm, ctx->CT, s);
  if (ctx->CT3) launch_class_tables3(g.r, ctx->prm, ctx->CT3, s);
  launch_static_field(g, ctx->cell, ctx->tables(), ctx->Fs, s);

  {
    const sfm_status gst = compute_guidance(g, ctx->cell, ctx->D, s, &ctx->err);
    if (gst != SFM_OK) return bail(gst);
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    fail(ctx, SFM_ECUDA, "scene set-up: %s", cudaGetErrorString(e));
    return bail(SFM_ECUDA);
  }
  *out = ctx;
  return SFM_OK;
}

void sfm_destroy(sfm_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  batch_destroy(ctx);
  for (void* p : ctx->allocs) cudaFree(p);
  for (auto& r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

static sfm_status place_impl(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                             const uint8_t* goal, const uint8_t* alive, const uint8_t* w,
                             const uint8_t* h, int32_t on_device);

sfm_status sfm_place(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                     const uint8_t* goal, const uint8_t* alive, int32_t on_device) {
  return place_impl(ctx, n, xy, heading, goal, alive, nullptr, nullptr, on_device);
}

sfm_status sfm_place_sized(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                           const uint8_t* goal, const uint8_t* alive, const uint8_t* width,
                           const uint8_t* height, int32_t on_device) {
  if (!width || !height) return fail(ctx, SFM_EINVAL, "width and height arrays are required");
  return place_impl(ctx, n, xy, heading, goal, alive, width, height, on_device);
}

static sfm_status place_impl(sfm_ctx* ctx, int32_t n, const int32_t* xy, const uint8_t* heading,
                             const uint8_t* goal, const uint8_t* alive, const uint8_t* w,
                             const uint8_t* h, int32_t on_device) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_ESTATE, "a batch is placed with sfm_batch_place");
  // The tick graphs hold the pedestrian count and array pointers as launch
  // parameters; they stay valid for a new placement of as many pedestrians
  // into the same arrays with the same options (no walk periods, the same
  // sizing), so a place / step / read loop keeps replaying them.
  const bool keep_graphs = ctx->placed && n == ctx->n && n <= ctx->cap && !ctx->walk_periods &&
                           !ctx->has_ids && (w != nullptr) == ctx->sized;
  if (!keep_graphs) drop_graph(ctx);
  if (n < 0 || (n > 0 && !xy)) return fail(ctx, SFM_EINVAL, "bad pedestrian arrays");
  // multi-su pedestrians: odd sides in [1, kMaxPedSide]; a periodic extent of
  // at least 2 * side + 3, so minimum-image offsets stay unambiguous
  std::vector<uint8_t> hw, hh;
  if (w) {
    hw.resize((size_t)n);
    hh.resize((size_t)n);
    if (n > 0) {
      const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
      CU(cudaMemcpy(hw.data(), w, (size_t)n, k));
      CU(cudaMemcpy(hh.data(), h, (size_t)n, k));
    }
    int mw = 1, mh = 1;
    for (int p = 0; p < n; ++p) {
      if (!(hw[p] & 1) || !(hh[p] & 1) || hw[p] > kMaxPedSide || hh[p] > kMaxPedSide)
        return fail(ctx, SFM_EINVAL, "pedestrian %d: size %dx%d (odd sides, at most %d)", p,
                    (int)hw[p], (int)hh[p], kMaxPedSide);
      mw = std::max(mw, (int)hw[p]);
      mh = std::max(mh, (int)hh[p]);
    }
    if ((ctx->geo.px && ctx->geo.W < 2 * mw + 3) || (ctx->geo.py && ctx->geo.H < 2 * mh + 3))
      return fail(ctx, SFM_EINVAL, "periodic extent below 2 * pedestrian side + 3");
  }
  cudaStream_t s = ctx->stream;
  const Geo& g = ctx->geo;
  // as many 1 x 1 pedestrians into the same arrays: touch the grid entries of
  // the pedestrians that change only (a place / step / read loop that hands
  // back what it read changes none).  Buffers the device can read in place
  // (device memory, mapped pinned host memory) are read by the placement
  // kernels themselves; otherwise the previous state is kept and the new one
  // copied in.
  const bool diff = keep_graphs && !w && n > 0;
  const int2* src_xy = nullptr;
  const uint8_t *src_h = nullptr, *src_g = nullptr, *src_a = nullptr;
  bool direct = false;
  if (diff) {
    src_xy = static_cast<const int2*>(device_view(xy, on_device));
    src_h = static_cast<const uint8_t*>(device_view(heading, on_device));
    src_g = static_cast<const uint8_t*>(device_view(goal, on_device));
    src_a = static_cast<const uint8_t*>(device_view(alive, on_device));
    direct = src_xy && (!heading || src_h) && (!goal || src_g) && (!alive || src_a);
  }
  if (direct) {
    // nothing to copy: the staging launch reads the caller's buffers
  } else if (diff) {
    CU(cudaMemcpyAsync(ctx->pl_xy, ctx->xy, (size_t)n * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(ctx->pl_alive, ctx->alive, (size_t)n, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(ctx->pl_heading, ctx->heading, (size_t)n, cudaMemcpyDeviceToDevice, s));
  } else if (ctx->placed && ctx->n > 0) {
    launch_place_clear(ctx->n, ctx->xy, ctx->alive, g, ctx->occ, ctx->ocls, s, ctx->sizes());
    ++ctx->launches;
  }
  if (n > ctx->cap) {
    CU(cudaStreamSynchronize(s));
    dfree(ctx, ctx->xy);
    dfree(ctx, ctx->heading);
    dfree(ctx, ctx->goal);
    dfree(ctx, ctx->alive);
    dfree(ctx, ctx->choice);
    dfree(ctx, ctx->won);
    dfree(ctx, ctx->rec);
    dfree(ctx, ctx->rec_id);
    dfree(ctx, ctx->bin_slot);
    dfree(ctx, ctx->bin_key);
    dfree(ctx, ctx->period);
    dfree(ctx, ctx->phase);
    dfree(ctx, ctx->gid);
    dfree(ctx, ctx->pw);
    dfree(ctx, ctx->ph);
    dfree(ctx, ctx->pl_xy);
    dfree(ctx, ctx->pl_alive);
    dfree(ctx, ctx->pl_heading);
    dfree(ctx, ctx->pl_goal);
    ctx->xy = nullptr;
    ctx->cap = 0;
    TRY(dalloc(ctx, &ctx->xy, (size_t)n));
    TRY(dalloc(ctx, &ctx->heading, (size_t)n));
    TRY(dalloc(ctx, &ctx->goal, (size_t)n));
    TRY(dalloc(ctx, &ctx->alive, (size_t)n));
    TRY(dalloc(ctx, &ctx->choice, (size_t)n));
    TRY(dalloc(ctx, &ctx->won, (size_t)n));
    TRY(dalloc(ctx, &ctx->rec, (size_t)n));
    TRY(dalloc(ctx, &ctx->rec_id, (size_t)n));
    TRY(dalloc(ctx, &ctx->bin_slot, (size_t)n));
    TRY(dalloc(ctx, &ctx->bin_key, (size_t)n));
    TRY(dalloc(ctx, &ctx->period, (size_t)n));
    TRY(dalloc(ctx, &ctx->phase, (size_t)n));
    TRY(dalloc(ctx, &ctx->gid, (size_t)n));
    TRY(dalloc(ctx, &ctx->pw, (size_t)n));
    TRY(dalloc(ctx, &ctx->ph, (size_t)n));
    TRY(dalloc(ctx, &ctx->pl_xy, (size_t)n));
    TRY(dalloc(ctx, &ctx->pl_alive, (size_t)n));
    TRY(dalloc(ctx, &ctx->pl_heading, (size_t)n));
    TRY(dalloc(ctx, &ctx->pl_goal, (size_t)n));
    ctx->cap = n;
  }
  if (ctx->cap == 0) {
    TRY(dalloc(ctx, &ctx->xy, 1));
    TRY(dalloc(ctx, &ctx->heading, 1));
    TRY(dalloc(ctx, &ctx->goal, 1));
    TRY(dalloc(ctx, &ctx->alive, 1));
    TRY(dalloc(ctx, &ctx->choice, 1));
    TRY(dalloc(ctx, &ctx->won, 1));
    TRY(dalloc(ctx, &ctx->rec, 1));
    TRY(dalloc(ctx, &ctx->rec_id, 1));
    TRY(dalloc(ctx, &ctx->bin_slot, 1));
    TRY(dalloc(ctx, &ctx->bin_key, 1));
    TRY(dalloc(ctx, &ctx->period, 1));
    TRY(dalloc(ctx, &ctx->phase, 1));
    TRY(dalloc(ctx, &ctx->gid, 1));
    TRY(dalloc(ctx, &ctx->pw, 1));
    TRY(dalloc(ctx, &ctx->ph, 1));
    TRY(dalloc(ctx, &ctx->pl_xy, 1));
    TRY(dalloc(ctx, &ctx->pl_alive, 1));
    TRY(dalloc(ctx, &ctx->pl_heading, 1));
    TRY(dalloc(ctx, &ctx->pl_goal, 1));
    ctx->cap = 1;
  }
  ctx->placed = false;
  ctx->walk_periods = false;  // a placement starts with every pedestrian active
  ctx->has_ids = false;       // and numbers its pedestrians by index
  ctx->n = n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0 && !direct) {
    CU(cudaMemcpyAsync(ctx->xy, xy, (size_t)n * sizeof(int2), kind, s));
    if (heading) CU(cudaMemcpyAsync(ctx->heading, heading, n, kind, s));
    else CU(cudaMemsetAsync(ctx->heading, 0, n, s));
    if (goal) CU(cudaMemcpyAsync(ctx->goal, goal, n, kind, s));
    else CU(cudaMemsetAsync(ctx->goal, 0, n, s));
    if (alive) CU(cudaMemcpyAsync(ctx->alive, alive, n, kind, s));
    else CU(cudaMemsetAsync(ctx->alive, 1, n, s));
    CU(cudaMemsetAsync(ctx->choice, 0, n, s));
    CU(cudaMemsetAsync(ctx->won, 0, n, s));
    if (w) {
      CU(cudaMemcpyAsync(ctx->pw, hw.data(), n, cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(ctx->ph, hh.data(), n, cudaMemcpyHostToDevice, s));
    }
  }
  ctx->sized = w != nullptr;
  // reset per-placement counters and flags on the stream, keep the tick counter
  launch_reset_counters(ctx->ctr, s);
  ++ctx->launches;
  if (direct) {
    launch_place_direct(n, src_xy, src_h, src_g, src_a, ctx->pl_xy, ctx->pl_heading, ctx->pl_goal,
                        ctx->pl_alive, ctx->xy, ctx->heading, ctx->goal, ctx->alive, ctx->choice,
                        ctx->won, ctx->cell, g, ctx->occ, ctx->ocls, ctx->ctr, s);
    ctx->launches += 2;
  } else if (diff) {
    launch_place_diff(n, ctx->pl_xy, ctx->pl_alive, ctx->pl_heading, ctx->xy, ctx->heading,
                      ctx->goal, ctx->alive, ctx->cell, g, ctx->occ, ctx->ocls, ctx->ctr, s);
    ctx->launches += 2;
  } else {
    launch_place_scatter(n, ctx->xy, ctx->heading, ctx->goal, ctx->alive, ctx->cell, g, ctx->occ,
                         ctx->ocls, ctx->ctr, s, ctx->sizes());
    if (n > 0) ++ctx->launches;
  }
  Counters hc;
  CU(cudaMemcpyAsync(&hc, ctx->ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  CU(cudaGetLastError());
  if (hc.err) {
    drop_graph(ctx);
    const uint32_t flags = hc.err;
    const size_t nsu = (size_t)g.W * g.H;
    cudaMemsetAsync(ctx->occ, 0xff, nsu * sizeof(int32_t), s);
    cudaMemsetAsync(ctx->ocls, 0, (size_t)g.opitch * g.H, s);
    ctx->sized = false;
    hc.err = 0;
    cudaMemcpyAsync(ctx->ctr, &hc, sizeof(hc), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return fail(ctx, (flags & kErrPlaceRange) ? SFM_EINVAL : SFM_ECONFLICT,
                "placement rejected: overlapping pedestrians, a pedestrian on a WALL/EXIT su, "
                "off-lattice positions or classes > 8");
  }
  ctx->placed = true;
  return SFM_OK;
}

sfm_status sfm_set_time(sfm_ctx* ctx, int64_t t) {
  if (!ctx) return SFM_EINVAL;
  CU(cudaStreamSynchronize(ctx->stream));
  long long tv = t;
  CU(cudaMemcpy(&ctx->ctr->t, &tv, sizeof(tv), cudaMemcpyHostToDevice));
  ctx->t = t;
  return SFM_OK;
}

sfm_status sfm_step(sfm_ctx* ctx, int32_t nsteps) {
  if (!ctx) return SFM_EINVAL;
  if (nsteps < 0) return fail(ctx, SFM_EINVAL, "nsteps < 0");
  if (ctx->batch) return batch_tick(ctx, nsteps, 0);
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "sfm_step before a successful sfm_place");
  const int every = ctx->timing_every;
  // after `done` ticks: the phase of the timing sample
  auto advance = [&](int done) {
    if (every > 0) ctx->timing_phase = (ctx->timing_phase + done) % every;
  };
  struct Restore {  // whatever happens, the flag means "timing on" again
    sfm_ctx* c;
    ~Restore() { c->timing = c->timing_every > 0; }
  } restore{ctx};
  for (int i = 0; i < nsteps;) {
    // Timed ticks (every `every`-th) record stage events.  The first tick
    // after placement runs directly (stage by stage); the rest replay graphs:
    // a timed tick its own graph, with event record nodes between the stages;
    // untimed ticks kBlockTicks ticks at a time while that many remain before
    // the end or the next timed tick, else one.
    const bool timed = every > 0 && ctx->timing_phase == 0;
    ctx->timing = timed;
    if (ctx->direct_ticks < 1) {
      run_tick(ctx);
      ++ctx->direct_ticks;
      ++ctx->t;
      ++i;
      if (timed) ++ctx->timed_ticks;
      advance(1);
      continue;
    }
    if (timed) {
      if (!ctx->timed_graph) TRY(ensure_graphs(ctx));
      const cudaError_t re = replay_timed_tick(ctx);
      if (re != cudaSuccess) return fail(ctx, SFM_ECUDA, "timed tick: %s", cudaGetErrorString(re));
      ctx->launches += ctx->timed_launches;
      ++ctx->t;
      ++i;
      ++ctx->timed_ticks;
      advance(1);
      continue;
    }
    int room = nsteps - i;
    if (every > 0 && every - ctx->timing_phase < room) room = (int)(every - ctx->timing_phase);
    const bool block = room >= kBlockTicks;
    cudaGraphExec_t* exec = block ? &ctx->block_graph : &ctx->tick_graph;
    int64_t* nl = block ? &ctx->block_launches : &ctx->graph_launches;
    if (!*exec) TRY(ensure_graphs(ctx));
    CU(cudaGraphLaunch(*exec, ctx->stream));
    ctx->launches += *nl;
    const int done = block ? kBlockTicks : 1;
    ctx->t += done;
    i += done;
    advance(done);
  }
  CU(cudaGetLastError());
  return SFM_OK;
}

sfm_status sfm_compute_field(sfm_ctx* ctx) {
  if (!ctx) return SFM_EINVAL;
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "no pedestrians placed");
  if (ctx->batch) return batch_tick(ctx, 1, 1);
  if (ctx->bands > 1) return fail(ctx, SFM_ESTATE, "banded mode keeps no full-lattice field");
  run_bins(ctx);
  {
    StageScope sc(ctx, SFM_STAGE_FIELD);
    field_rows(ctx, ctx->F, 0, ctx->geo.H, 0, false);
  }
  CU(cudaGetLastError());
  return SFM_OK;
}

sfm_status sfm_compute_field_into(sfm_ctx* ctx, float* dst, int32_t on_device) {
  if (!ctx || !dst) return SFM_EINVAL;
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "no pedestrians placed");
  if (ctx->batch) return fail(ctx, SFM_ESTATE, "use sfm_compute_field and sfm_read_field on a batch");
  const Geo& g = ctx->geo;
  run_bins(ctx);
  if (on_device) {
    field_rows(ctx, dst, 0, g.H, 0, false);
    CU(cudaGetLastError());
    return check_flags(ctx);
  }
  float* buf = ctx->bands > 1 ? ctx->band_buf : ctx->F;
  const int rows = ctx->bands > 1 ? ctx->band_rows : g.H;
  for (int ya = 0; ya < g.H; ya += rows) {
    const int yb = ya + rows < g.H ? ya + rows : g.H;
    field_rows(ctx, buf, ya, yb, 0, false);
    CU(cudaMemcpyAsync(dst + (size_t)ya * g.W, buf, (size_t)(yb - ya) * g.W * sizeof(float),
                       cudaMemcpyDeviceToHost, ctx->stream));
  }
  CU(cudaGetLastError());
  return check_flags(ctx);
}

sfm_status sfm_autotune(sfm_ctx* ctx, int32_t* shape_out) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "use sfm_batch_autotune on a batch");
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "autotune needs placed pedestrians");
  if (!ctx->CT) {
    if (shape_out) *shape_out = ctx->field_shape;
    return SFM_OK;  // radius beyond the class-table gather: nothing to choose
  }
  const Geo& g = ctx->geo;
  float* out = ctx->bands > 1 ? ctx->band_buf : ctx->F;
  const int rows = ctx->bands > 1 ? ctx->band_rows : g.H;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  run_bins(ctx);
  float best = 1e30f;
  int best_shape = ctx->field_shape;
  for (int shape : {kShape16x16, kShape32x16, kShape32x32}) {
    if (shape >= kShape32x32 && !(ctx->CT3 && field3_shape_ok(shape, g.r))) continue;
    ctx->field_shape = shape;
    float tot = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      CU(cudaEventRecord(e0, ctx->stream));
      field_rows(ctx, out, 0, rows, 0, false);
      CU(cudaEventRecord(e1, ctx->stream));
      CU(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;  // the first run warms up
    }
    if (tot < best) {
      best = tot;
      best_shape = shape;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->field_shape = best_shape;
  drop_graph(ctx);
  if (shape_out) *shape_out = best_shape;
  return check_flags(ctx);
}

sfm_status sfm_set_walk_periods(sfm_ctx* ctx, const uint8_t* period, const uint8_t* phase,
                                int32_t on_device) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "walk periods are per single lattice");
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "walk periods need placed pedestrians");
  drop_graph(ctx);
  if (!period) {
    ctx->walk_periods = false;
    return SFM_OK;
  }
  if (!phase) return fail(ctx, SFM_EINVAL, "phase array missing");
  const int n = ctx->n;
  std::vector<uint8_t> hp((size_t)n), hf((size_t)n);
  if (n > 0) {
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    CU(cudaMemcpy(hp.data(), period, (size_t)n, k));
    CU(cudaMemcpy(hf.data(), phase, (size_t)n, k));
  }
  for (int p = 0; p < n; ++p)
    if (hp[p] < 1 || hf[p] >= hp[p])
      return fail(ctx, SFM_EINVAL, "pedestrian %d: period %d, phase %d (need 1 <= period, phase < period)",
                  p, (int)hp[p], (int)hf[p]);
  if (n > 0) {
    CU(cudaMemcpyAsync(ctx->period, hp.data(), (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->phase, hf.data(), (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  ctx->walk_periods = true;
  return SFM_OK;
}

sfm_status sfm_set_ids(sfm_ctx* ctx, const int32_t* ids, int32_t on_device) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "pedestrian numbers are per single lattice");
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "pedestrian numbers need placed pedestrians");
  if (ctx->sized) return fail(ctx, SFM_EINVAL, "pedestrian numbers with multi-su pedestrians");
  drop_graph(ctx);
  if (!ids) {
    ctx->has_ids = false;
    return SFM_OK;
  }
  const int n = ctx->n;
  std::vector<int32_t> h((size_t)n);
  if (n > 0)
    CU(cudaMemcpy(h.data(), ids, (size_t)n * sizeof(int32_t),
                  on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  {
    std::vector<int32_t> sorted(h);
    std::sort(sorted.begin(), sorted.end());
    for (int p = 0; p < n; ++p) {
      if (sorted[p] < 0) return fail(ctx, SFM_EINVAL, "pedestrian number %d < 0", sorted[p]);
      if (p && sorted[p] == sorted[p - 1])
        return fail(ctx, SFM_EINVAL, "pedestrian number %d given twice", sorted[p]);
    }
  }
  if (n > 0) {
    CU(cudaMemcpyAsync(ctx->gid, h.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  ctx->has_ids = true;
  return SFM_OK;
}

sfm_status sfm_set_guidance(sfm_ctx* ctx, const int32_t* D, int32_t on_device) {
  if (!ctx || !D) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "guidance is set per single lattice");
  const size_t n = (size_t)ctx->geo.W * ctx->geo.H;
  std::vector<int32_t> h(n);
  CU(cudaMemcpy(h.data(), D, n * sizeof(int32_t),
                on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  for (size_t i = 0; i < n; ++i)
    if (h[i] < 0 || h[i] > kDInf)
      return fail(ctx, SFM_EINVAL, "guidance value %d at su %zu outside [0, 2^23]", h[i], i);
  CU(cudaMemcpyAsync(ctx->D, h.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  launch_guidance_import(ctx->cell, ctx->D, n, ctx->stream);  // WALL su: kDWall
  ++ctx->launches;
  return check_flags(ctx);
}

sfm_status sfm_set_binning(sfm_ctx* ctx, int32_t mode) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "a batch bins from its class grids");
  if (mode < 0 || mode > 2) return fail(ctx, SFM_EINVAL, "binning mode must be 0, 1 or 2");
  if (ctx->binning != mode) {
    ctx->binning = mode;
    drop_graph(ctx);
  }
  return SFM_OK;
}

sfm_status sfm_set_field_footprint(sfm_ctx* ctx, int32_t shape) {
  if (!ctx) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "a batch tunes its footprints per radius class");
  if (shape < kShape16x16 || shape > kShape32x32)
    return fail(ctx, SFM_EINVAL, "footprint must be 0, 1 or 2");
  if (ctx->field_shape != shape) {
    ctx->field_shape = shape;
    drop_graph(ctx);
  }
  return SFM_OK;
}

sfm_status sfm_sync(sfm_ctx* ctx) {
  if (!ctx) return SFM_EINVAL;
  CU(cudaGetLastError());
  if (ctx->batch) {
    const sfm_status bs = batch_sync(ctx);
    if (bs != SFM_OK) return bs;
  }
  return check_flags(ctx);
}

sfm_status sfm_read_field(sfm_ctx* ctx, float* dst, int32_t on_device) {
  if (!ctx || !dst) return SFM_EINVAL;
  if (ctx->bands > 1) return fail(ctx, SFM_ESTATE, "banded mode keeps no full-lattice field");
  return copy_out(ctx, dst, ctx->F, (size_t)ctx->nsu_total * sizeof(float), on_device);
}

sfm_status sfm_read_static_field(sfm_ctx* ctx, float* dst, int32_t on_device) {
  if (!ctx || !dst) return SFM_EINVAL;
  return copy_out(ctx, dst, ctx->Fs, (size_t)ctx->nsu_total * sizeof(float), on_device);
}

sfm_status sfm_read_guidance(sfm_ctx* ctx, int32_t* dst, int32_t on_device) {
  if (!ctx || !dst) return SFM_EINVAL;
  const size_t n = (size_t)ctx->nsu_total;
  if (on_device) {
    CU(cudaMemcpyAsync(dst, ctx->D, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    launch_guidance_export(dst, n, ctx->stream);  // WALL su: kDWall -> kDInf
    return check_flags(ctx);
  }
  TRY(copy_out(ctx, dst, ctx->D, n * sizeof(int32_t), 0));
  for (size_t i = 0; i < n; ++i)
    if (dst[i] == kDWall) dst[i] = kDInf;
  return SFM_OK;
}

sfm_status sfm_read_peds(sfm_ctx* ctx, int32_t* xy, uint8_t* heading, uint8_t* alive,
                         int32_t on_device) {
  if (!ctx) return SFM_EINVAL;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = (size_t)ctx->n;
  // pinned host buffers are written in place by one launch, without copies
  void* dxy = on_device ? nullptr : device_view(xy, 0);
  void* dh = on_device ? nullptr : device_view(heading, 0);
  void* da = on_device ? nullptr : device_view(alive, 0);
  if (n && (xy || heading || alive) && (!xy || dxy) && (!heading || dh) && (!alive || da)) {
    launch_read_peds((int)n, ctx->xy, ctx->heading, ctx->alive, static_cast<int2*>(dxy),
                     static_cast<uint8_t*>(dh), static_cast<uint8_t*>(da), ctx->stream);
    ++ctx->launches;
  } else if (n) {
    if (xy) CU(cudaMemcpyAsync(xy, ctx->xy, n * sizeof(int2), kind, ctx->stream));
    if (heading) CU(cudaMemcpyAsync(heading, ctx->heading, n, kind, ctx->stream));
    if (alive) CU(cudaMemcpyAsync(alive, ctx->alive, n, kind, ctx->stream));
  }
  return check_flags(ctx);
}

// ---------------------------------------------------------- checkpoints
namespace {

struct SnapHeader {
  char magic[8];
  uint32_t version, flags;  // flags: 1 walk periods, 2 multi-su sizes
  int32_t W, H, px, py, r, pad_;
  uint64_t params_fp;  // fingerprint of the model parameters
  int64_t t, n;
  uint64_t exited, moved;
};
constexpr char kSnapMagic[8] = {'S', 'F', 'M', 'S', 'N', 'A', 'P', '1'};
constexpr uint32_t kSnapPeriods = 1u, kSnapSizes = 2u;

// FNV-1a over the parameters that decide a trajectory (not the HBM budget)
uint64_t params_fingerprint(const sfm_params& p) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void* d, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(d);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  mix(&p.r, sizeof p.r);
  mix(&p.kP, sizeof p.kP);
  mix(&p.aP, sizeof p.aP);
  mix(&p.gamma, sizeof p.gamma);
  mix(&p.kO, sizeof p.kO);
  mix(&p.aO, sizeof p.aO);
  mix(&p.kE, sizeof p.kE);
  mix(&p.aE, sizeof p.aE);
  mix(&p.beta, sizeof p.beta);
  mix(&p.seed, sizeof p.seed);
  return h;
}

size_t snap_bytes(int64_t n, uint32_t flags) {
  size_t per = 8 + 3;  // xy, heading, goal, alive
  if (flags & kSnapPeriods) per += 2;
  if (flags & kSnapSizes) per += 2;
  return sizeof(SnapHeader) + (size_t)n * per;
}

}  // namespace

sfm_status sfm_snapshot(sfm_ctx* ctx, void* buf, size_t* len) {
  if (!ctx || !len) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "snapshots are per single lattice");
  if (!ctx->placed) return fail(ctx, SFM_ESTATE, "nothing placed");
  const uint32_t flags = (ctx->walk_periods ? kSnapPeriods : 0u) | (ctx->sized ? kSnapSizes : 0u);
  const int64_t n = ctx->n;
  const size_t need = snap_bytes(n, flags);
  if (!buf) {
    *len = need;
    return SFM_OK;
  }
  if (*len < need) {
    *len = need;
    return fail(ctx, SFM_EINVAL, "snapshot buffer of %zu bytes, %zu needed", *len, need);
  }
  CU(cudaStreamSynchronize(ctx->stream));
  Counters hc;
  CU(cudaMemcpy(&hc, ctx->ctr, sizeof(hc), cudaMemcpyDeviceToHost));
  SnapHeader hd{};
  memcpy(hd.magic, kSnapMagic, 8);
  hd.version = 1;
  hd.flags = flags;
  hd.W = ctx->geo.W;
  hd.H = ctx->geo.H;
  hd.px = ctx->geo.px;
  hd.py = ctx->geo.py;
  hd.r = ctx->geo.r;
  hd.params_fp = params_fingerprint(ctx->prm);
  hd.t = hc.t;
  hd.n = n;
  hd.exited = hc.exited;
  hd.moved = hc.moved;
  unsigned char* o = static_cast<unsigned char*>(buf);
  memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  auto take = [&](const void* src, size_t bytes) -> cudaError_t {
    const cudaError_t e = bytes ? cudaMemcpy(o, src, bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
    o += bytes;
    return e;
  };
  CU(take(ctx->xy, (size_t)n * 8));
  CU(take(ctx->heading, (size_t)n));
  CU(take(ctx->goal, (size_t)n));
  CU(take(ctx->alive, (size_t)n));
  if (flags & kSnapPeriods) {
    CU(take(ctx->period, (size_t)n));
    CU(take(ctx->phase, (size_t)n));
  }
  if (flags & kSnapSizes) {
    CU(take(ctx->pw, (size_t)n));
    CU(take(ctx->ph, (size_t)n));
  }
  *len = need;
  return SFM_OK;
}

sfm_status sfm_restore(sfm_ctx* ctx, const void* buf, size_t len) {
  if (!ctx || !buf) return SFM_EINVAL;
  if (ctx->batch) return fail(ctx, SFM_EINVAL, "snapshots are per single lattice");
  SnapHeader hd;
  if (len < sizeof hd) return fail(ctx, SFM_EINVAL, "snapshot shorter than its header");
  memcpy(&hd, buf, sizeof hd);
  if (memcmp(hd.magic, kSnapMagic, 8) != 0 || hd.version != 1)
    return fail(ctx, SFM_EINVAL, "not a snapshot of this library (magic or version)");
  if (hd.n < 0 || hd.n > INT32_MAX || (hd.flags & ~(kSnapPeriods | kSnapSizes)) ||
      len != snap_bytes(hd.n, hd.flags))
    return fail(ctx, SFM_EINVAL, "snapshot length or flags do not match its header");
  if (hd.W != ctx->geo.W || hd.H != ctx->geo.H || hd.px != ctx->geo.px || hd.py != ctx->geo.py ||
      hd.r != ctx->geo.r || hd.params_fp != params_fingerprint(ctx->prm))
    return fail(ctx, SFM_EINVAL, "snapshot of another lattice or other model parameters");
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof hd;
  const int32_t n = (int32_t)hd.n;
  const int32_t* xy = reinterpret_cast<const int32_t*>(in);
  const uint8_t* heading = in + (size_t)n * 8;
  const uint8_t* goal = heading + n;
  const uint8_t* alive = goal + n;
  const uint8_t* extra = alive + n;
  const uint8_t *period = nullptr, *phase = nullptr, *w = nullptr, *h = nullptr;
  if (hd.flags & kSnapPeriods) {
    period = extra;
    phase = extra + n;
    extra += 2 * (size_t)n;
  }
  if (hd.flags & kSnapSizes) {
    w = extra;
    h = extra + n;
  }
  // xy may be unaligned inside the buffer: copy to aligned storage
  std::vector<int32_t> xya((size_t)n * 2);
  if (n) memcpy(xya.data(), xy, (size_t)n * 8);
  sfm_status st = place_impl(ctx, n, xya.data(), heading, goal, alive, w, h, 0);
  if (st != SFM_OK) return st;
  if (period) {
    st = sfm_set_walk_periods(ctx, period, phase, 0);
    if (st != SFM_OK) return st;
  }
  CU(cudaStreamSynchronize(ctx->stream));
  Counters hc;
  CU(cudaMemcpy(&hc, ctx->ctr, sizeof(hc), cudaMemcpyDeviceToHost));
  hc.t = hd.t;
  hc.exited = hd.exited;
  hc.moved = hd.moved;
  CU(cudaMemcpy(ctx->ctr, &hc, sizeof(hc), cudaMemcpyHostToDevice));
  ctx->t = hd.t;
  return SFM_OK;
}

sfm_status sfm_read_decisions(sfm_ctx* ctx, uint8_t* choice, uint8_t* won, int32_t on_device) {
  if (!ctx) return SFM_EINVAL;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = (size_t)ctx->n;
  if (n) {
    if (choice) CU(cudaMemcpyAsync(choice, ctx->choice, n, kind, ctx->stream));
    if (won) CU(cudaMemcpyAsync(won, ctx->won, n, kind, ctx->stream));
  }
  return check_flags(ctx);
}

sfm_status sfm_stats(sfm_ctx* ctx, sfm_stats_t* out) {
  if (!ctx || !out) return SFM_EINVAL;
  CU(cudaStreamSynchronize(ctx->stream));
  Counters h;
  CU(cudaMemcpy(&h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->t = h.t;
  out->n = ctx->n;
  out->exited = (int64_t)h.exited;
  out->moved_total = (int64_t)h.moved;
  out->max_registrants = h.max_registrants;
  out->bands = ctx->bands;
  out->error_flags = h.err;
  out->device_bytes = ctx->device_bytes;
  out->kernel_launches = ctx->launches;
  out->decided = (int64_t)h.decided;
  out->near_ties = (int64_t)h.near_ties;
  // alive = placed live pedestrians minus those that left since placement
  int64_t alive0 = 0;
  if (ctx->n) {
    std::vector<uint8_t> a((size_t)ctx->n);
    CU(cudaMemcpy(a.data(), ctx->alive, a.size(), cudaMemcpyDeviceToHost));
    for (uint8_t v : a) alive0 += v ? 1 : 0;
  }
  out->alive = alive0;
  return SFM_OK;
}

sfm_status sfm_set_timing(sfm_ctx* ctx, int32_t every) {
  if (!ctx) return SFM_EINVAL;
  if (every < 0) return fail(ctx, SFM_EINVAL, "timing period %d < 0", every);
  ctx->timing_every = every;
  ctx->timing_phase = 0;
  ctx->timing = every > 0;
  return SFM_OK;
}

sfm_status sfm_stage_times(sfm_ctx* ctx, double* ms, int64_t* ticks) {
  if (!ctx || !ms) return SFM_EINVAL;
  CU(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < SFM_NSTAGES; ++i) ms[i] = 0.0;
  for (auto& r : ctx->recs) {
    float v = 0.f;
    if (cudaEventElapsedTime(&v, r.a, r.b) == cudaSuccess) ms[r.stage] += v;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  if (ticks) *ticks = ctx->timed_ticks;
  ctx->timed_ticks = 0;
  return SFM_OK;
}

}  // extern "C"
