// Host side of the batch API (many grids advanced together): tile lists,
// the three launch forms, the autotuner.  Device memory comes from the
// caller's batch workspace; nothing here allocates device memory.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch_kernels.cuh"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr size_t kBatchAlign = 256;
constexpr long long kDefaultBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kAutoMinSteps = 96;

size_t up(size_t v) { return (v + kBatchAlign - 1) / kBatchAlign * kBatchAlign; }

long long tiles_for(const std::vector<lbm_elastic_t *> &shots, int R) {
  long long t = 0;
  for (const lbm_elastic_t *h : shots)
    t += (long long)((h->cfg.nx + 31) / 32) * ((h->cfg.ny + R - 1) / R);
  return t;
}

// Two-step tiles of a shot: 30 x 14 cells, or 28 x 12 with the
// density-gradient force.
void tile2_size(const lbm_elastic_t *h, int *W, int *H) {
  *W = h->lambda_nonzero ? kL2Cols : kF2Cols;
  *H = h->lambda_nonzero ? kL2Rows : kF2Rows;
}

// Two-step tiles of the batch if every shot took the smaller (gradient-force)
// tile: an upper bound whatever the material.
long long tiles2_max(const std::vector<lbm_elastic_t *> &shots) {
  long long t = 0;
  for (const lbm_elastic_t *h : shots)
    t += (long long)((h->cfg.nx + kL2Cols - 1) / kL2Cols) * ((h->cfg.ny + kL2Rows - 1) / kL2Rows);
  return t;
}

struct Offsets {
  size_t hdr = 0, shots = 0, dyn = 0, tiles = 0, tiles2 = 0, total = 0;
};

Offsets offsets(int n, long long max_tiles, long long max_tiles2) {
  Offsets o;
  size_t off = 0;
  o.hdr = off;
  off = up(off + sizeof(BatchHdr));
  o.shots = off;
  off = up(off + (size_t)n * sizeof(BatchShot));
  o.dyn = off;
  off = up(off + (size_t)n * sizeof(BatchDyn));
  o.tiles = off;
  off = up(off + (size_t)max_tiles * sizeof(int4));
  o.tiles2 = off;
  off = up(off + (size_t)max_tiles2 * sizeof(int4));
  o.total = off;
  return o;
}

Offsets offsets_for(const std::vector<lbm_elastic_t *> &v) {
  return offsets((int)v.size(), std::max(tiles_for(v, 4), tiles_for(v, 8)), tiles2_max(v));
}

// per thread: calls without a handle on different threads must not race on it
thread_local std::string g_batch_create_error;

}  // namespace

struct lbm_batch {
  std::vector<lbm_elastic_t *> shots;
  int storage = 0;
  bool u64 = false;
  char *ws = nullptr;
  Offsets off;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private stream the graphs are captured on
  int nsm = 0;
  lbm_batch_launch launch;
  bool tuned = false;
  // tile lists on the device: one-step tiles, and two-step tiles (their
  // geometry depends on each shot's Lambda, kept in tiles2_lam)
  int ntiles = 0, tiles_rows = 0, tiles_order = -1;
  int ntiles2 = 0, tiles2_order = -1;
  std::vector<char> tiles2_lam;
  // captured graph of graph_steps launches for the current tile list of
  // graph_tps time steps per tile
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0, graph_tps = 0;
  long long launches = 0;
  std::vector<BatchShot> shot_host;
  std::vector<BatchDyn> dyn_host;
  std::vector<int4> tile_host;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch_t *b, lbm_status s, const std::string &m) {
  if (b) b->err = m;
  else g_batch_create_error = m;
  return s;
}

lbm_status bcuda(lbm_batch_t *b, cudaError_t e, const char *what) {
  return bfail(b, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BATCH_CUDA(b, call)                                 \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return bcuda((b), e_, #call);    \
  } while (0)

BatchHdr *hdr_of(lbm_batch_t *b) { return (BatchHdr *)(b->ws + b->off.hdr); }

BatchArgs args_of(lbm_batch_t *b, int tps) {
  BatchArgs a;
  a.shots = (const BatchShot *)(b->ws + b->off.shots);
  a.dyn = (const BatchDyn *)(b->ws + b->off.dyn);
  a.tiles = (const int4 *)(b->ws + (tps == 2 ? b->off.tiles2 : b->off.tiles));
  a.ntiles = tps == 2 ? b->ntiles2 : b->ntiles;
  a.hdr = hdr_of(b);
  a.barrier_count = 0;
  a.barrier_cycles =
      b->launch.barrier_cycles > 0 ? b->launch.barrier_cycles : kDefaultBarrierCycles;
  return a;
}

bool launch_ok(const lbm_batch_launch &l) {
  return l.mode >= LBM_BATCH_AUTO && l.mode <= LBM_BATCH_PERSISTENT &&
         (l.rows == 4 || l.rows == 8) && (l.order == 0 || l.order == 1) && l.graph_steps >= 1 &&
         l.steps_per_launch >= 1 && l.ctas_per_sm >= 0 && l.barrier_cycles >= 0 &&
         l.barrier_extra >= 0 && (l.steps_per_tile == 1 || l.steps_per_tile == 2);
}

// Whether tile (x0, y0) of W x R cells of shot h is likely to take the
// general path (near an edge, a source footprint or a receiver).
bool tile_is_edge(const lbm_elastic_t *h, int x0, int y0, int W, int R) {
  const int nx = h->cfg.nx, ny = h->cfg.ny, m = 2;
  if (x0 < m || x0 + W > nx - m || y0 < m || y0 + R > ny - m) return true;
  auto hit = [&](const int *bx) {
    return bx[1] >= bx[0] && x0 <= bx[1] && x0 + W - 1 >= bx[0] && y0 <= bx[3] &&
           y0 + R - 1 >= bx[2];
  };
  return (h->nsrc > 0 && hit(h->src_box)) || (h->nrec > 0 && hit(h->rec_box));
}

void drop_graph(lbm_batch_t *b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Tiles of W x R cells of every shot (W, R from size(h)), shot by shot in
// row-major order, or (order 1) those likely to take the general path first.
template <class F>
void list_tiles(lbm_batch_t *b, int order, F size) {
  std::vector<int4> &t = b->tile_host;
  t.clear();
  for (int pass = 0; pass < (order == 1 ? 2 : 1); ++pass) {
    for (int s = 0; s < (int)b->shots.size(); ++s) {
      const lbm_elastic_t *h = b->shots[s];
      int W, R;
      size(h, &W, &R);
      const int gx = (h->cfg.nx + W - 1) / W, gy = (h->cfg.ny + R - 1) / R;
      for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
          if (order == 1 && tile_is_edge(h, bx * W, by * R, W, R) != (pass == 0)) continue;
          t.push_back(make_int4(s, bx, by, 0));
        }
    }
  }
}

lbm_status upload_tiles(lbm_batch_t *b, int R, int order) {
  if (b->tiles_rows == R && b->tiles_order == order) return LBM_OK;
  list_tiles(b, order, [R](const lbm_elastic_t *, int *W, int *H) {
    *W = 32;
    *H = R;
  });
  b->ntiles = (int)b->tile_host.size();
  BATCH_CUDA(b, cudaMemcpyAsync(b->ws + b->off.tiles, b->tile_host.data(),
                                b->tile_host.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                b->stream));
  b->tiles_rows = R;
  b->tiles_order = order;
  if (b->graph_tps == 1) drop_graph(b);
  return LBM_OK;
}

lbm_status upload_tiles2(lbm_batch_t *b, int order) {
  std::vector<char> lam(b->shots.size());
  for (size_t s = 0; s < b->shots.size(); ++s) lam[s] = b->shots[s]->lambda_nonzero ? 1 : 0;
  if (b->tiles2_order == order && b->tiles2_lam == lam) return LBM_OK;
  if (order == 1) {
    // every shot's slower tiles first (its own launch order: near an edge or
    // seam, a source or a receiver), then the others
    std::vector<int4> &t = b->tile_host;
    t.clear();
    for (int pass = 0; pass < 2; ++pass)
      for (int s = 0; s < (int)b->shots.size(); ++s) {
        const lbm_elastic_t *h = b->shots[s];
        const size_t base = h->lambda_nonzero ? (size_t)h->L.ntiles2 : 0;
        const size_t count = h->lambda_nonzero ? (size_t)h->L.ntiles2l : (size_t)h->L.ntiles2;
        const size_t first = h->lambda_nonzero ? h->order2l_first : h->order2_first;
        const size_t a = pass == 0 ? 0 : first, e = pass == 0 ? first : count;
        for (size_t k = a; k < e; ++k) {
          const int2 q = h->order_host[base + k];
          t.push_back(make_int4(s, q.x, q.y, 0));
        }
      }
  } else {
    list_tiles(b, order, [](const lbm_elastic_t *h, int *W, int *H) { tile2_size(h, W, H); });
  }
  b->ntiles2 = (int)b->tile_host.size();
  BATCH_CUDA(b, cudaMemcpyAsync(b->ws + b->off.tiles2, b->tile_host.data(),
                                b->tile_host.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                b->stream));
  b->tiles2_order = order;
  b->tiles2_lam = lam;
  if (b->graph_tps == 2) drop_graph(b);
  return LBM_OK;
}

// Uploads every shot's parameters and state, and zeroes the call counters.
lbm_status prepare_call(lbm_batch_t *b) {
  const int n = (int)b->shots.size();
  for (int s = 0; s < n; ++s) {
    lbm_elastic_t *h = b->shots[s];
    BatchShot &bs = b->shot_host[s];
    memset(&bs, 0, sizeof(bs));
    bs.p = handle_step_params(h);
    bs.p.blk_near = nullptr;  // laid out for the shot's own one-step launches
    bs.f[0] = h->ws + h->L.f[0];
    bs.f[1] = h->ws + h->L.f[1];
    bs.lam = h->lambda_nonzero ? 1 : 0;
    bs.trace_max = h->cfg.max_steps_traced;
    BatchDyn &d = b->dyn_host[s];
    d.n0 = h->step;
    d.cur0 = h->cur;
    d.traced0 = h->traced;
  }
  BATCH_CUDA(b, cudaMemcpyAsync(b->ws + b->off.shots, b->shot_host.data(),
                                n * sizeof(BatchShot), cudaMemcpyHostToDevice, b->stream));
  BATCH_CUDA(b, cudaMemcpyAsync(b->ws + b->off.dyn, b->dyn_host.data(), n * sizeof(BatchDyn),
                                cudaMemcpyHostToDevice, b->stream));
  // queue, arrive, kbase (err stays until lbm_batch_sync reads it)
  BATCH_CUDA(b, cudaMemsetAsync(hdr_of(b), 0, offsetof(BatchHdr, err), b->stream));
  return LBM_OK;
}

// The shots' host state after nlaunch batched launches of tps time steps
// each (one buffer swap per launch).
void advance_shots(lbm_batch_t *b, int nlaunch, int tps) {
  const long long nsteps = (long long)nlaunch * tps;
  for (lbm_elastic_t *h : b->shots) {
    h->step += nsteps;
    h->cur ^= (nlaunch & 1);
    if (h->nrec > 0)
      h->traced = (int)std::min<long long>((long long)h->traced + nsteps, h->cfg.max_steps_traced);
  }
}

cudaError_t launch_form(lbm_batch_t *b, int tps, bool persistent, const BatchArgs &a, int count,
                        int grid, bool pdl, cudaStream_t s) {
  const int R = b->launch.rows;
  if (b->storage == LBM_F64) return batch_launch_f64(R, tps, persistent, a, count, grid, pdl, s);
  if (b->storage == LBM_F32)
    return batch_launch_f32(b->u64, R, tps, persistent, a, count, grid, pdl, s);
  return batch_launch_16(b->storage == LBM_BF16, b->u64, R, tps, persistent, a, count, grid, pdl,
                         s);
}

int occupancy(lbm_batch_t *b, int tps) {
  const int R = b->launch.rows;
  if (b->storage == LBM_F64) return batch_occupancy_f64(R, tps);
  if (b->storage == LBM_F32) return batch_occupancy_f32(b->u64, R, tps);
  return batch_occupancy_16(b->storage == LBM_BF16, b->u64, R, tps);
}

lbm_status counted(lbm_batch_t *b, cudaError_t e, const char *what) {
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(b, e, what);
  b->launches++;
  return LBM_OK;
}

// n launches of tps time steps each, one per launch.
lbm_status run_stream(lbm_batch_t *b, int n, int tps) {
  const BatchArgs a = args_of(b, tps);
  for (int k = 0; k < n; ++k)
    if (lbm_status st = counted(b, launch_form(b, tps, false, a, k, a.ntiles, true, b->stream),
                                "batch step"))
      return st;
  return LBM_OK;
}

// Captures G launches of tps time steps each and the kbase advance into a
// graph.  The launches carry the programmatic-dependent-launch attribute
// when the capture accepts it, else they are captured plainly.
cudaError_t capture_graph(lbm_batch_t *b, int G, int tps, bool pdl, cudaGraphExec_t *out) {
  const BatchArgs a = args_of(b, tps);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < G && e == cudaSuccess; ++k)
    e = launch_form(b, tps, false, a, k, a.ntiles, pdl, b->capture);
  if (e == cudaSuccess) {
    batch_advance_kernel<<<1, 1, 0, b->capture>>>(hdr_of(b), G);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

lbm_status build_graph(lbm_batch_t *b, int G, int tps) {
  if (b->graph && b->graph_steps == G && b->graph_tps == tps) return LBM_OK;
  drop_graph(b);
  // captured on a private stream (the legacy default stream cannot be
  // captured); the graph is launched on the batch's stream
  if (!b->capture) BATCH_CUDA(b, cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  cudaGraphExec_t x = nullptr;
  cudaError_t e = capture_graph(b, G, tps, true, &x);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear, and capture without the attribute
    x = nullptr;
    e = capture_graph(b, G, tps, false, &x);
  }
  if (e != cudaSuccess) return bcuda(b, e, "batch graph capture");
  b->graph = x;
  b->graph_steps = G;
  b->graph_tps = tps;
  return LBM_OK;
}

lbm_status run_graph(lbm_batch_t *b, int n, int tps) {
  const int G = b->launch.graph_steps;
  if (n >= G) {
    if (lbm_status st = build_graph(b, G, tps)) return st;
    for (int r = 0; r + G <= n; r += G) {
      BATCH_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
      b->launches += G + 1;
    }
  }
  // the remainder: plain launches after the graphs' launches (kbase holds them)
  const BatchArgs a = args_of(b, tps);
  for (int k = 0; k < n % G; ++k)
    if (lbm_status st = counted(b, launch_form(b, tps, false, a, k, a.ntiles, true, b->stream),
                                "batch step"))
      return st;
  return LBM_OK;
}

// n steps (tps 1) or two-step phases (tps 2) in cooperative launches of at
// most steps_per_launch time steps each.
lbm_status run_persistent(lbm_batch_t *b, int n, int tps) {
  const int occ = occupancy(b, tps);
  if (occ < 1) return bfail(b, LBM_ERR_CUDA, "batch persistent kernel: no resident block fits");
  const int per_sm = b->launch.ctas_per_sm > 0 ? std::min(b->launch.ctas_per_sm, occ) : occ;
  const int grid = b->nsm * per_sm;
  BatchArgs a = args_of(b, tps);
  a.barrier_count = (unsigned)(grid + b->launch.barrier_extra);
  const int per_launch = std::max(1, b->launch.steps_per_launch / tps);
  for (int done = 0; done < n;) {
    const int m = std::min(per_launch, n - done);
    // queue and arrival counters restart with each launch
    BATCH_CUDA(b, cudaMemsetAsync(hdr_of(b), 0, offsetof(BatchHdr, kbase), b->stream));
    if (lbm_status st = counted(b, launch_form(b, tps, true, a, m, grid, false, b->stream),
                                   "batch persistent"))
      return st;
    batch_advance_kernel<<<1, 1, 0, b->stream>>>(hdr_of(b), m);
    if (lbm_status st = counted(b, cudaSuccess, "batch advance")) return st;
    done += m;
  }
  return LBM_OK;
}

// n launches of tps time steps each in the given form, from the shots'
// current state.
lbm_status run_launches(lbm_batch_t *b, int n, int tps, int mode) {
  if (n == 0) return LBM_OK;
  if (lbm_status st = tps == 2 ? upload_tiles2(b, b->launch.order)
                               : upload_tiles(b, b->launch.rows, b->launch.order))
    return st;
  if (lbm_status st = prepare_call(b)) return st;
  lbm_status st;
  if (mode == LBM_BATCH_STREAM) st = run_stream(b, n, tps);
  else if (mode == LBM_BATCH_PERSISTENT) st = run_persistent(b, n, tps);
  else st = run_graph(b, n, tps);
  if (st) return st;
  advance_shots(b, n, tps);
  return LBM_OK;
}

// nsteps time steps: with two steps per tile, nsteps / 2 two-step launches
// and, for an odd count, one one-step launch.
lbm_status run(lbm_batch_t *b, int nsteps, int mode) {
  if (b->launch.steps_per_tile == 2) {
    if (lbm_status st = run_launches(b, nsteps / 2, 2, mode)) return st;
    return run_launches(b, nsteps % 2, 1, mode);
  }
  return run_launches(b, nsteps, 1, mode);
}

// Times every launch candidate on the batch itself: per candidate two
// untimed steps (tile upload, graph capture) and trial steps (rounded up to
// even) timed.  Advances the shots by 18 (2 + trial) steps.
lbm_status tune(lbm_batch_t *b, int trial, double *best_us) {
  const lbm_batch_launch keep = b->launch;
  struct Cand {
    int mode, rows, order, tps;
  };
  trial += trial & 1;
  std::vector<Cand> cands;
  for (int mode : {LBM_BATCH_STREAM, LBM_BATCH_GRAPH, LBM_BATCH_PERSISTENT}) {
    for (int rows : {8, 4})
      for (int order : {1, 0}) cands.push_back({mode, rows, order, 1});
    for (int order : {1, 0}) cands.push_back({mode, 8, order, 2});
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BATCH_CUDA(b, cudaEventCreate(&e0));
  BATCH_CUDA(b, cudaEventCreate(&e1));
  double best = 1e300;
  Cand win = cands[0];
  lbm_status st = LBM_OK;
  for (const Cand &c : cands) {
    b->launch.mode = c.mode;
    b->launch.rows = c.rows;
    b->launch.order = c.order;
    b->launch.steps_per_tile = c.tps;
    b->launch.graph_steps = trial / c.tps;
    b->launch.steps_per_launch = std::max(keep.steps_per_launch, trial);
    if ((st = run(b, 2, c.mode))) break;
    if (c.mode == LBM_BATCH_GRAPH && (st = build_graph(b, trial / c.tps, c.tps))) break;
    cudaEventRecord(e0, b->stream);
    if ((st = run(b, trial, c.mode))) break;
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = bcuda(b, cudaGetLastError(), "batch autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = 1e3 * ms / trial;
    if (us < best) {
      best = us;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->launch = keep;
  if (st) return st;
  b->launch.mode = win.mode;
  b->launch.rows = win.rows;
  b->launch.order = win.order;
  b->launch.steps_per_tile = win.tps;
  b->tuned = true;
  if (best_us) *best_us = best;
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(lbm_elastic_t *const *shots, int n) {
  if (!shots || n < 1) return 0;
  std::vector<lbm_elastic_t *> v(shots, shots + n);
  for (lbm_elastic_t *h : v)
    if (!h) return 0;
  return offsets_for(v).total;
}

lbm_status lbm_batch_create(lbm_elastic_t *const *shots, int n, void *d_workspace, size_t bytes,
                            void *cuda_stream, lbm_batch_t **out) {
  if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!shots || n < 1) return bfail(nullptr, LBM_ERR_ARG, "need at least one shot");
  for (int s = 0; s < n; ++s)
    if (!shots[s]) return bfail(nullptr, LBM_ERR_ARG, "null shot handle");
  for (int s = 1; s < n; ++s)
    if (shots[s]->cfg.storage != shots[0]->cfg.storage ||
        (shots[s]->L.usize == 8) != (shots[0]->L.usize == 8))
      return bfail(nullptr, LBM_ERR_ARG, "shots differ in storage type or u_fp64");
  const size_t need = lbm_batch_workspace_bytes(shots, n);
  if (!d_workspace || bytes < need)
    return bfail(nullptr, LBM_ERR_WORKSPACE, "batch workspace too small");
  if ((uintptr_t)d_workspace % kBatchAlign)
    return bfail(nullptr, LBM_ERR_WORKSPACE, "batch workspace not 256-byte aligned");
  {
    const std::vector<lbm_elastic_t *> v(shots, shots + n);
    if (tiles_for(v, 4) >= (1LL << 31) || tiles2_max(v) >= (1LL << 31))
      return bfail(nullptr, LBM_ERR_ARG, "too many tiles");
  }
  lbm_batch_t *b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ERR_ARG, "out of host memory");
  b->shots.assign(shots, shots + n);
  b->storage = shots[0]->cfg.storage;
  b->u64 = shots[0]->L.usize == 8 && b->storage != LBM_F64;
  b->ws = (char *)d_workspace;
  b->off = offsets_for(b->shots);
  b->stream = (cudaStream_t)cuda_stream;
  b->shot_host.resize(n);
  b->dyn_host.resize(n);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (b->nsm < 1) b->nsm = 1;
  b->launch.mode = LBM_BATCH_AUTO;
  b->launch.rows = 8;
  b->launch.order = 1;
  b->launch.graph_steps = 50;
  b->launch.steps_per_launch = 500;
  b->launch.ctas_per_sm = 0;
  b->launch.barrier_cycles = 0;
  b->launch.barrier_extra = 0;
  b->launch.steps_per_tile = 1;
  if (cudaMemsetAsync(d_workspace, 0, sizeof(BatchHdr), b->stream) != cudaSuccess) {
    delete b;
    return bfail(nullptr, LBM_ERR_CUDA, "batch workspace clear failed");
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch_t *b, const lbm_batch_launch *l) {
  if (!b) return LBM_ERR_ARG;
  if (!l || !launch_ok(*l)) return bfail(b, LBM_ERR_ARG, "invalid launch configuration");
  b->launch = *l;
  b->tuned = l->mode != LBM_BATCH_AUTO;
  return LBM_OK;
}

lbm_status lbm_batch_get_launch(const lbm_batch_t *b, lbm_batch_launch *l) {
  if (!b || !l) return LBM_ERR_ARG;
  *l = b->launch;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch_t *b, int steps_per_trial, double *us_per_step) {
  if (!b) return LBM_ERR_ARG;
  if (steps_per_trial < 1) return bfail(b, LBM_ERR_ARG, "steps_per_trial < 1");
  return tune(b, steps_per_trial, us_per_step);
}

lbm_status lbm_batch_step(lbm_batch_t *b, int nsteps) {
  if (!b) return LBM_ERR_ARG;
  if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps < 0");
  if (b->launch.mode == LBM_BATCH_AUTO && !b->tuned) {
    // 18 candidates x (2 + 2) steps
    if (nsteps >= kAutoMinSteps) {
      if (lbm_status st = tune(b, 2, nullptr)) return st;
      nsteps -= 72;
    } else {
      return run(b, nsteps, LBM_BATCH_GRAPH);
    }
  }
  const int mode = b->launch.mode == LBM_BATCH_AUTO ? LBM_BATCH_GRAPH : b->launch.mode;
  return run(b, nsteps, mode);
}

lbm_status lbm_batch_sync(lbm_batch_t *b) {
  if (!b) return LBM_ERR_ARG;
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  int err = 0;
  BATCH_CUDA(b, cudaMemcpy(&err, &hdr_of(b)->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    BATCH_CUDA(b, cudaMemset(&hdr_of(b)->err, 0, sizeof(int)));
    return bfail(b, LBM_ERR_TIMEOUT, "a grid barrier of the persistent batch kernel gave up");
  }
  for (size_t s = 0; s < b->shots.size(); ++s) {
    lbm_elastic_t *h = b->shots[s];
    int flags = 0;
    BATCH_CUDA(b, cudaMemcpy(&flags, h->ws + h->L.flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (flags & 1)
      return bfail(b, LBM_ERR_NONFINITE,
                   "shot " + std::to_string(s) + " met a non-finite value (unstable run)");
  }
  return LBM_OK;
}

long long lbm_batch_kernel_launches(const lbm_batch_t *b) { return b ? b->launches : -1; }

long long lbm_batch_cells(const lbm_batch_t *b) {
  if (!b) return -1;
  long long c = 0;
  for (const lbm_elastic_t *h : b->shots) c += (long long)h->cfg.nx * h->cfg.ny;
  return c;
}

lbm_status lbm_batch_destroy(lbm_batch_t *b) {
  if (!b) return LBM_ERR_ARG;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
  return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch_t *b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
