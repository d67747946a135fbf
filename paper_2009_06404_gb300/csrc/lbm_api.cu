// Host side of the C ABI declared in include/lbm_elastic.h, plus the small
// set-up, conversion and reduction kernels.  All device memory comes from the
// caller's workspace; this file never allocates device memory.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "step_fused.cuh"
#include "step2_lam.cuh"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed so sums are reproducible
constexpr int kRedThreads = 256;
constexpr int kStageCells = 1 << 18;
constexpr unsigned kMagic = 0x4c424d45u;  // checkpoint header tag

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }


bool config_ok(const lbm_elastic_config *c, std::string *why) {
  auto bad = [&](const char *m) {
    if (why) *why = m;
    return false;
  };
  if (!c) return bad("config is NULL");
  if (c->nx < 3 || c->ny < 3) return bad("nx and ny must be >= 3");
  {
    // 32-bit element offsets inside the kernels: 9 planes of the padded grid
    const long long per_line =
        c->storage == LBM_F64 ? 16 : (c->storage == LBM_F32 ? 32 : 64);
    const long long pitch = (c->nx + per_line - 1) / per_line * per_line;
    if (c->ny > 500000 || 9 * pitch * c->ny >= (1LL << 31)) return bad("grid too large");
  }
  if (c->storage < LBM_F64 || c->storage > LBM_BF16) return bad("unknown storage type");
  if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return bad("tau must be finite and > 0.5");
  const int bcs[4] = {c->bc_top, c->bc_bottom, c->bc_left, c->bc_right};
  for (int b : bcs)
    if (b < LBM_BC_PERIODIC || b > LBM_BC_RIGID) return bad("unknown boundary kind");
  if ((c->bc_top == LBM_BC_PERIODIC) != (c->bc_bottom == LBM_BC_PERIODIC))
    return bad("periodic top/bottom must be paired");
  if ((c->bc_left == LBM_BC_PERIODIC) != (c->bc_right == LBM_BC_PERIODIC))
    return bad("periodic left/right must be paired");
  const int sp[4] = {c->sponge_top, c->sponge_bottom, c->sponge_left, c->sponge_right};
  for (int s : sp)
    if (s < 0) return bad("sponge thickness must be >= 0");
  if (c->sponge_top + c->sponge_bottom > c->ny || c->sponge_left + c->sponge_right > c->nx)
    return bad("absorbing layers larger than the grid");
  if (!std::isfinite(c->sponge_amax)) return bad("sponge_amax must be finite");
  if (c->free_surface_order != 0 && c->free_surface_order != 1)
    return bad("free_surface_order must be 0 or 1");
  if (c->max_sources < 0 || c->max_receivers < 0 || c->max_steps_traced < 0)
    return bad("capacities must be >= 0");
  if (c->kernel_variant < 0 || c->kernel_variant > 1) return bad("unknown kernel_variant");
  if (c->store_scale_log2 < -60 || c->store_scale_log2 > 60)
    return bad("store_scale_log2 must lie in [-60, 60]");
  return true;
}

Layout make_layout(const lbm_elastic_config *c) {
  Layout L;
  L.tsize = c->storage == LBM_F64 ? 8 : (c->storage == LBM_F32 ? 4 : 2);
  L.csize = c->storage == LBM_F64 ? 8 : 4;
  L.usize = (c->storage == LBM_F64 || c->u_fp64) ? 8 : 4;
  const int per_line = (int)(128 / L.tsize);
  L.pitch = (c->nx + per_line - 1) / per_line * per_line;
  L.plane = (long long)L.pitch * c->ny;
  L.finter = 1;
  L.fplane = L.finter ? L.pitch : L.plane;
  L.frow = L.finter ? 9LL * L.pitch : L.pitch;
  L.rec_tiles_x = (c->nx + kRecTileX - 1) / kRecTileX;
  L.rec_tiles = L.rec_tiles_x * ((c->ny + kRecTileY - 1) / kRecTileY);
  L.mat_count = c->material_per_cell ? L.plane : c->ny;
  L.stage_rows = kStageCells / c->nx;
  if (L.stage_rows < 1) L.stage_rows = 1;
  if (L.stage_rows > c->ny) L.stage_rows = c->ny;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, kAlign);
    return o;
  };
  L.f[0] = take(9 * (size_t)L.plane * L.tsize);
  L.f[1] = take(9 * (size_t)L.plane * L.tsize);
  L.u = take(2 * (size_t)L.plane * L.usize);
  L.lam = take((size_t)L.mat_count * L.csize);
  L.irho = take((size_t)L.mat_count * L.csize);
  L.src = take((size_t)c->max_sources * sizeof(SourceDev) + 8);
  L.srcb = take((size_t)c->max_sources * sizeof(int4) + 16);
  L.rec_ptr = take(((size_t)L.rec_tiles + 1) * sizeof(int));
  L.rec_xy = take((size_t)c->max_receivers * 2 * sizeof(int) + 8);
  L.rec_id = take((size_t)c->max_receivers * sizeof(int) + 8);
  L.traces = take((size_t)c->max_steps_traced * c->max_receivers * 4 * sizeof(double) + 8);
  L.partials = take((size_t)(kRedBlocks + 1) * 8 * sizeof(double));
  L.flags = take(64);
  L.ntiles2 = (long long)((c->nx + kF2Cols - 1) / kF2Cols) * ((c->ny + kF2Rows - 1) / kF2Rows);
  L.ntiles2l = (long long)((c->nx + kL2Cols - 1) / kL2Cols) * ((c->ny + kL2Rows - 1) / kL2Rows);
  L.order2 = take((size_t)L.ntiles2 * sizeof(int2));
  L.order2l = take((size_t)L.ntiles2l * sizeof(int2));
  L.nblk1 = (long long)((c->nx + 31) / 32) * ((c->ny + 7) / 8);
  L.blk1 = take((size_t)L.nblk1 + 16);
  size_t stage = (size_t)L.stage_rows * c->nx * 11 * sizeof(double);
  size_t mat_stage = (size_t)3 * c->ny * sizeof(double);
  L.stage = take(stage > mat_stage ? stage : mat_stage);
  L.total = off;
  return L;
}

// ------------------------------------------------------------ small kernels

// Lambda = (mu - lambda)/(rho0 b^2) and 1/rho0 (Eqs. 9 and 32) from FP64
// material arrays; flags: 1 = some Lambda != 0, 2 = mu/(rho0 b^2) != 1,
// 4 = invalid value.
template <class C>
__global__ void material_kernel(const double *rho0, const double *lam, const double *mu,
                                long long count, int per_cell, int nx, int pitch, long long off,
                                C *lam_out, C *irho_out, int *flags) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const double r = rho0[k], l = lam[k], m = mu[k];
    long long dst = off + k;
    if (per_cell) {
      const long long g = off + k;  // dense index of the cell
      dst = (g / nx) * pitch + g % nx;
    }
    int fl = 0;
    if (!(r > 0.0) || !isfinite(r) || !isfinite(l) || !isfinite(m)) {
      fl |= 4;
      lam_out[dst] = C(0);
      irho_out[dst] = C(1);
    } else {
      const double L = (m - l) / (r * (1.0 / 3.0));
      lam_out[dst] = C(L);
      irho_out[dst] = C(1.0 / r);
      if (C(L) != C(0)) fl |= 1;
      if (fabs(m / (r * (1.0 / 3.0)) - 1.0) > 1e-9) fl |= 2;
    }
    if (fl) atomicOr(flags, fl);
  }
}

template <class C>
__global__ void fill_kernel(C *p, long long n, C v) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    p[k] = v;
}

template <class T> __device__ __forceinline__ double to_d(T v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__half>(__half v) {
  return (double)__half2float(v);
}
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <class T> __device__ __forceinline__ T from_d(double v) { return T(v); }
template <> __device__ __forceinline__ __half from_d<__half>(double v) {
  return __double2half(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}

// State <-> dense FP64 rows [row0, row0 + nrows).  dst/src planes are
// [nplanes][rows][nx] with a plane stride of dplane elements.
template <class T>
__global__ void to_f64_kernel(const T *s, long long splane, int pitch, int nx, int row0,
                              int nrows, int nplanes, double *d, long long dplane,
                              double scale) {
  const long long n = (long long)nrows * nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * nplanes;
       k += (long long)gridDim.x * blockDim.x) {
    const int pl = (int)(k / n);
    const long long r = k % n;
    const long long y = row0 + r / nx, x = r % nx;
    d[pl * dplane + r] = to_d<T>(s[pl * splane + y * pitch + x]) * scale;
  }
}

template <class T>
__global__ void from_f64_kernel(T *s, long long splane, int pitch, int nx, int row0, int nrows,
                                int nplanes, const double *d, long long dplane, double scale) {
  const long long n = (long long)nrows * nx;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * nplanes;
       k += (long long)gridDim.x * blockDim.x) {
    const int pl = (int)(k / n);
    const long long r = k % n;
    const long long y = row0 + r / nx, x = r % nx;
    s[pl * splane + y * pitch + x] = from_d<T>(d ? d[pl * dplane + r] * scale : 0.0);
  }
}

// Deterministic FP64 block reduction of seven per-cell sums.
__device__ void block_reduce7(double *v, double *out) {
  __shared__ double sm[kRedThreads / 32][7];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sm[w][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int i = 0; i < kRedThreads / 32; ++i) t += sm[i][threadIdx.x];
    out[threadIdx.x] = t;
  }
}

template <class T, class U>
__global__ void __launch_bounds__(kRedThreads)
    moments_partial_kernel(const T *f, const U *u, long long plane, int pitch, long long fplane,
                           long long frow, int nx, int ny, double *partials,
                           double fscale = 1.0) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const long long n = (long long)nx * ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long c = (k / nx) * pitch + k % nx;
    const long long cf = (k / nx) * frow + k % nx;
    double q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = to_d<T>(f[i * fplane + cf]) * fscale;
    v[0] += q[0] + q[1] + q[2] + q[3] + q[4] + q[5] + q[6] + q[7] + q[8];
    v[1] += q[1] - q[3] + q[5] - q[6] - q[7] + q[8];
    v[2] += q[2] - q[4] + q[5] + q[6] - q[7] - q[8];
    v[3] += q[1] + q[3] + q[5] + q[6] + q[7] + q[8];
    v[4] += q[5] - q[6] + q[7] - q[8];
    v[5] += q[2] + q[4] + q[5] + q[6] + q[7] + q[8];
    const double ux = (double)u[c], uy = (double)u[plane + c];
    v[6] += ux * ux + uy * uy;
  }
  block_reduce7(v, partials + 8 * blockIdx.x);
}

__global__ void __launch_bounds__(kRedThreads) moments_final_kernel(const double *partials,
                                                                    int nblocks, double *out) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] += partials[8 * b + k];
  block_reduce7(v, out);
}

}  // namespace

// ------------------------------------------------------------ the handle

namespace {

// per thread: calls without a handle on different threads must not race on it
thread_local std::string g_create_error;

lbm_status fail(lbm_elastic_t *h, lbm_status s, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

lbm_status cuda_fail(lbm_elastic_t *h, cudaError_t e, const char *what) {
  return fail(h, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

template <class X> X *at(lbm_elastic_t *h, size_t off) { return (X *)(h->ws + off); }

int grid1d(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

lbm_status check_launch(lbm_elastic_t *h, const char *what) {
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  return LBM_OK;
}

// Reads the device error flag (synchronises the stream).
lbm_status sync_flags(lbm_elastic_t *h) {
  int flags[2] = {0, 0};
  LBM_CUDA(h, cudaMemcpyAsync(flags, at<int>(h, h->L.flags), sizeof(flags),
                              cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (flags[0] & 2)
    return fail(h, LBM_ERR_TIMEOUT, "a bounded wait in the step kernel gave up");
  if (flags[0] & 1)
    return fail(h, LBM_ERR_NONFINITE, "a step met a non-finite value (unstable run)");
  return LBM_OK;
}

double store_scale(const lbm_elastic_config &c) {
  return (c.storage == LBM_F16 || c.storage == LBM_BF16) ? std::ldexp(1.0, c.store_scale_log2)
                                                         : 1.0;
}

// The indices of the tiles (or blocks) of size T along one axis of n cells
// that hold a cell of [lo, hi], each once: cells wrapped on a periodic axis
// (the last tile may be partial, so a range across the seam continues at
// cell 0, not at a whole tile), dropped beyond a non-periodic edge.
static void tile_span(long long lo, long long hi, int T, int n, bool per, std::vector<int> &v) {
  v.clear();
  auto add = [&](long long a, long long b) {  // cells a..b, 0 <= a <= b < n
    for (long long k = a / T; k <= b / T; ++k) {
      bool seen = false;
      for (int e : v) seen |= e == (int)k;
      if (!seen) v.push_back((int)k);
    }
  };
  if (per) {
    if (hi - lo + 1 >= n) {
      add(0, n - 1);
    } else {
      const long long a = ((lo % n) + n) % n, b = a + (hi - lo);
      if (b < n) {
        add(a, b);
      } else {
        add(a, n - 1);
        add(0, b - n);
      }
    }
  } else {
    lo = std::max(lo, 0LL);
    hi = std::min(hi, (long long)n - 1);
    if (lo <= hi) add(lo, hi);
  }
}

// The two-step tiles of one geometry (W x H cells; m: the distance to an
// edge or seam within which a tile takes a slower path) in launch order:
// the tiles near an edge or seam, that a source footprint reaches, or that
// hold a receiver first, then the others, each group in row-major order.
// Appends to out; returns the size of the first group.  The first group
// holds every tile a source footprint (widened by m + 1) or a receiver can
// reach: the single-grid kernels skip the source and receiver lookups of
// the other tiles (their edge and seam tests stay in the kernel), so the
// list is rebuilt whenever sources or receivers change.
int order_tiles(const lbm_elastic_t *h, int W, int H, int m, std::vector<int2> &out) {
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  const bool perx = h->cfg.bc_left == LBM_BC_PERIODIC, pery = h->cfg.bc_top == LBM_BC_PERIODIC;
  const int gx = (nx + W - 1) / W, gy = (ny + H - 1) / H;
  std::vector<char> slow((size_t)gx * gy, 0);
  for (int by = 0; by < gy; ++by)
    for (int bx = 0; bx < gx; ++bx) {
      const int x0 = bx * W, y0 = by * H;
      if (x0 < m || x0 + W > nx - m || y0 < m || y0 + H > ny - m) slow[(size_t)by * gx + bx] = 1;
    }
  std::vector<int> xs, ys;
  for (const SourceDev &q : h->src_host) {
    tile_span((long long)q.xc - q.rb - m - 1, (long long)q.xc + q.rb + m + 1, W, nx, perx, xs);
    tile_span((long long)q.yc - q.rb - m - 1, (long long)q.yc + q.rb + m + 1, H, ny, pery, ys);
    for (int ty : ys)
      for (int tx : xs) slow[(size_t)ty * gx + tx] = 1;
  }
  for (size_t r = 0; 2 * r + 1 < h->rec_host.size(); ++r)
    slow[(size_t)(h->rec_host[2 * r + 1] / H) * gx + h->rec_host[2 * r] / W] = 1;
  int first = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int by = 0; by < gy; ++by)
      for (int bx = 0; bx < gx; ++bx)
        if ((slow[(size_t)by * gx + bx] != 0) == (pass == 0)) {
          out.push_back(make_int2(bx, by));
          if (pass == 0) ++first;
        }
  return first;
}

// Builds both tile order lists and copies them into the workspace on the
// handle's stream (the host copy stays in the handle).
lbm_status upload_tile_order(lbm_elastic_t *h) {
  std::vector<int2> &o = h->order_host;
  o.clear();
  h->order2_first = order_tiles(h, kF2Cols, kF2Rows, 2, o);
  h->order2l_first = order_tiles(h, kL2Cols, kL2Rows, 4, o);
  const Layout &L = h->L;
  if ((long long)o.size() != L.ntiles2 + L.ntiles2l)
    return fail(h, LBM_ERR_CUDA, "internal: tile order lists of the wrong size");
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.order2, o.data(), (size_t)L.ntiles2 * sizeof(int2),
                              cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.order2l, o.data() + L.ntiles2,
                              (size_t)L.ntiles2l * sizeof(int2), cudaMemcpyHostToDevice,
                              h->stream));
  // one-step blocks (32 x 8) that a source footprint widened by three cells
  // (the kernel's test reaches two) or a receiver can reach
  const int nx = h->cfg.nx, ny = h->cfg.ny, gx = (nx + 31) / 32;
  const bool perx = h->cfg.bc_left == LBM_BC_PERIODIC, pery = h->cfg.bc_top == LBM_BC_PERIODIC;
  std::vector<unsigned char> near((size_t)L.nblk1, 0);
  std::vector<int> xs, ys;
  for (const SourceDev &q : h->src_host) {
    tile_span((long long)q.xc - q.rb - 3, (long long)q.xc + q.rb + 3, 32, nx, perx, xs);
    tile_span((long long)q.yc - q.rb - 3, (long long)q.yc + q.rb + 3, 8, ny, pery, ys);
    for (int ty : ys)
      for (int tx : xs) near[(size_t)ty * gx + tx] = 1;
  }
  for (size_t r = 0; 2 * r + 1 < h->rec_host.size(); ++r)
    near[(size_t)(h->rec_host[2 * r + 1] / 8) * gx + h->rec_host[2 * r] / 32] = 1;
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.blk1, near.data(), near.size(), cudaMemcpyHostToDevice,
                              h->stream));
  // (pageable source: the copy has left the host buffer when the call returns)
  return LBM_OK;
}

StepParams base_params(lbm_elastic_t *h) {
  const lbm_elastic_config &c = h->cfg;
  const Layout &L = h->L;
  StepParams p;
  memset(&p, 0, sizeof(p));
  p.fin = h->ws + L.f[h->cur];
  p.fout = h->ws + L.f[1 - h->cur];
  p.u = h->ws + L.u;
  p.plane = (int)L.plane;
  p.fplane = (int)L.fplane;
  p.frow = (int)L.frow;
  p.finter = L.finter;
  p.nx = c.nx;
  p.ny = c.ny;
  p.pitch = L.pitch;
  p.bc_top = c.bc_top;
  p.bc_bottom = c.bc_bottom;
  p.bc_left = c.bc_left;
  p.bc_right = c.bc_right;
  p.sp_top = c.sponge_top;
  p.sp_bottom = c.sponge_bottom;
  p.sp_left = c.sponge_left;
  p.sp_right = c.sponge_right;
  p.fs_order = c.free_surface_order;
  const int Ls[4] = {c.sponge_top, c.sponge_bottom, c.sponge_left, c.sponge_right};
  for (int s = 0; s < 4; ++s) {
    double a = 0.0;
    if (Ls[s] > 0) {
      const double amax = c.sponge_amax > 0.0 ? c.sponge_amax : 12.8 / Ls[s];
      a = amax / ((double)Ls[s] * Ls[s]);
    }
    p.spA[s] = a;
    p.spA_f[s] = (float)a;
  }
  p.scale_f = (float)store_scale(c);
  p.iscale_f = (float)(1.0 / store_scale(c));
  p.omega = 1.0 / c.tau;
  p.fcoef = 1.0 - 1.0 / (2.0 * c.tau);
  p.omega_f = (float)p.omega;
  p.fcoef_f = (float)p.fcoef;
  p.lam = h->ws + L.lam;
  p.irho = h->ws + L.irho;
  p.mat_per_cell = c.material_per_cell;
  p.src = at<SourceDev>(h, L.src);
  p.nsrc = h->nsrc;
  p.srcb = at<int4>(h, L.srcb);
  p.n = h->step;
  p.trace_slot = -1;
  p.trace_end = h->cfg.max_steps_traced;
  p.tiles2 = at<int2>(h, L.order2);
  p.tiles2l = at<int2>(h, L.order2l);
  p.tiles2_first = h->order2_first;
  p.tiles2l_first = h->order2l_first;
  p.blk_near = at<unsigned char>(h, L.blk1);
  p.rec_tile_ptr = at<int>(h, L.rec_ptr);
  p.rec_xy = at<int>(h, L.rec_xy);
  p.rec_id = at<int>(h, L.rec_id);
  p.rec_tiles_x = L.rec_tiles_x;
  p.nrec = h->nrec;
  p.traces = at<double>(h, L.traces);
  p.err = at<int>(h, L.flags);
  p.src_x0 = h->src_box[0];
  p.src_x1 = h->src_box[1];
  p.src_y0 = h->src_box[2];
  p.src_y1 = h->src_box[3];
  p.rec_x0 = h->rec_box[0];
  p.rec_x1 = h->rec_box[1];
  p.rec_y0 = h->rec_box[2];
  p.rec_y1 = h->rec_box[3];
  p.reverse = (int)(h->step & 1);
  return p;
}

constexpr int kBX = 32, kBY = 8;

lbm_status launch_step(lbm_elastic_t *h, const StepParams &p, int mode, int rows) {
  const int by = h->lambda_nonzero ? kLamRows : kBY;
  dim3 block(kBX, by);
  dim3 grid((h->cfg.nx + kBX - 1) / kBX, (rows + by - 1) / by);
  if (h->cfg.storage == LBM_F64)
    launch_step_f64(p, h->lambda_nonzero, mode, grid, block, h->stream);
  else if (h->cfg.storage == LBM_F32)
    launch_step_f32(p, h->lambda_nonzero, h->cfg.u_fp64 != 0, mode, grid, block, h->stream);
  else
    launch_step_16(p, h->cfg.storage == LBM_BF16, h->lambda_nonzero, h->cfg.u_fp64 != 0, mode,
                   grid, block, h->stream);
  return check_launch(h, "step kernel launch");
}

template <class T>
lbm_status state_io(lbm_elastic_t *h, T *planes, long long splane, int srow, int nplanes,
                    double *dst, const double *src, int on_device, long long dense_plane,
                    double scale = 1.0) {
  // dst receives stored values / scale; src values are stored times scale
  const double iscale = 1.0 / scale;
  // dst (to f64) or src (from f64): [nplanes][ny][nx]
  const lbm_elastic_config &c = h->cfg;
  const Layout &L = h->L;
  if (on_device) {
    const long long n = (long long)c.nx * c.ny * nplanes;
    if (dst)
      to_f64_kernel<T><<<grid1d(n, 256), 256, 0, h->stream>>>(planes, splane, srow, c.nx, 0,
                                                               c.ny, nplanes, dst, dense_plane,
                                                               iscale);
    else
      from_f64_kernel<T><<<grid1d(n, 256), 256, 0, h->stream>>>(planes, splane, srow, c.nx, 0,
                                                                 c.ny, nplanes, src, dense_plane,
                                                                 scale);
    return check_launch(h, "state conversion launch");
  }
  double *stage = at<double>(h, L.stage);
  for (int r0 = 0; r0 < c.ny; r0 += L.stage_rows) {
    const int nr = (r0 + L.stage_rows <= c.ny) ? L.stage_rows : c.ny - r0;
    const long long chunk = (long long)nr * c.nx;
    const long long n = chunk * nplanes;
    if (dst) {
      to_f64_kernel<T><<<grid1d(n, 256), 256, 0, h->stream>>>(planes, splane, srow, c.nx, r0,
                                                               nr, nplanes, stage, chunk, iscale);
      lbm_status s = check_launch(h, "state conversion launch");
      if (s) return s;
      for (int pl = 0; pl < nplanes; ++pl)
        LBM_CUDA(h, cudaMemcpyAsync(dst + pl * dense_plane + (long long)r0 * c.nx,
                                    stage + pl * chunk, chunk * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream));
    } else {
      if (src)
        for (int pl = 0; pl < nplanes; ++pl)
          LBM_CUDA(h, cudaMemcpyAsync(stage + pl * chunk,
                                      src + pl * dense_plane + (long long)r0 * c.nx,
                                      chunk * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      from_f64_kernel<T><<<grid1d(n, 256), 256, 0, h->stream>>>(
          planes, splane, srow, c.nx, r0, nr, nplanes, src ? stage : nullptr, chunk, scale);
      lbm_status s = check_launch(h, "state conversion launch");
      if (s) return s;
    }
    // the staging area is reused by the next chunk: wait for this one
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

lbm_status f_io(lbm_elastic_t *h, double *dst, const double *src, int on_device) {
  void *f = h->ws + h->L.f[h->cur];
  const long long dp = (long long)h->cfg.nx * h->cfg.ny;
  const double sc = store_scale(h->cfg);
  if (h->cfg.storage == LBM_F16)
    return state_io<__half>(h, (__half *)f, h->L.fplane, (int)h->L.frow, 9, dst, src, on_device,
                            dp, sc);
  if (h->cfg.storage == LBM_BF16)
    return state_io<__nv_bfloat16>(h, (__nv_bfloat16 *)f, h->L.fplane, (int)h->L.frow, 9, dst,
                                   src, on_device, dp, sc);
  if (h->cfg.storage == LBM_F64)
    return state_io<double>(h, (double *)f, h->L.fplane, (int)h->L.frow, 9, dst, src, on_device,
                            dp);
  return state_io<float>(h, (float *)f, h->L.fplane, (int)h->L.frow, 9, dst, src, on_device, dp);
}

lbm_status u_io(lbm_elastic_t *h, double *dst, const double *src, int on_device) {
  void *u = h->ws + h->L.u;
  const long long dp = (long long)h->cfg.nx * h->cfg.ny;
  if (h->L.usize == 8)
    return state_io<double>(h, (double *)u, h->L.plane, h->L.pitch, 2, dst, src, on_device, dp);
  return state_io<float>(h, (float *)u, h->L.plane, h->L.pitch, 2, dst, src, on_device, dp);
}

lbm_status clear_state(lbm_elastic_t *h) {
  const Layout &L = h->L;
  LBM_CUDA(h, cudaMemsetAsync(h->ws + L.f[0], 0, 9 * (size_t)L.plane * L.tsize, h->stream));
  LBM_CUDA(h, cudaMemsetAsync(h->ws + L.f[1], 0, 9 * (size_t)L.plane * L.tsize, h->stream));
  LBM_CUDA(h, cudaMemsetAsync(h->ws + L.u, 0, 2 * (size_t)L.plane * L.usize, h->stream));
  LBM_CUDA(h, cudaMemsetAsync(h->ws + L.flags, 0, 64, h->stream));
  h->cur = 0;
  h->step = 0;
  h->traced = 0;
  return LBM_OK;
}

}  // namespace

// ------------------------------------------------------------ C ABI

StepParams lbm::handle_step_params(lbm_elastic_t *h) { return base_params(h); }

lbm_status lbm::handle_step(lbm_elastic_t *h, void *grad_out) {
  StepParams p = base_params(h);
  if (h->nrec > 0 && h->traced < h->cfg.max_steps_traced) p.trace_slot = h->traced;
  lbm_status st;
  if (grad_out) {
    // the gradient-force path, whatever Lambda is, storing grad rho
    p.grad_out = grad_out;
    const bool keep = h->lambda_nonzero;
    h->lambda_nonzero = true;
    st = launch_step(h, p, 0, h->cfg.ny);
    h->lambda_nonzero = keep;
  } else {
    st = launch_step(h, p, 0, h->cfg.ny);
  }
  if (st) return st;
  if (p.trace_slot >= 0) h->traced++;
  h->cur ^= 1;
  h->step++;
  return LBM_OK;
}

// Steps n and n + 1 of the handle in one launch of the two-step kernel.
static lbm_status handle_step2(lbm_elastic_t *h) {
  StepParams p = base_params(h);
  // consecutive launches visit the tiles in opposite orders
  p.reverse = (int)((h->step >> 1) & 1);
  const int tmax = h->cfg.max_steps_traced;
  if (h->nrec > 0 && h->traced < tmax) p.trace_slot = h->traced;
  const bool u64 = h->cfg.u_fp64 != 0, bf16 = h->cfg.storage == LBM_BF16;
  if (h->lambda_nonzero) {
    if (h->cfg.storage == LBM_F64) launch_step2_lam_f64(p, h->stream);
    else if (h->cfg.storage == LBM_F32) launch_step2_lam_f32(p, u64, h->stream);
    else launch_step2_lam_16(p, bf16, u64, h->stream);
  } else {
    if (h->cfg.storage == LBM_F64) launch_step2_f64(p, h->stream);
    else if (h->cfg.storage == LBM_F32) launch_step2_f32(p, u64, h->stream);
    else launch_step2_16(p, bf16, u64, h->stream);
  }
  if (lbm_status st = check_launch(h, "two-step kernel launch")) return st;
  if (p.trace_slot >= 0) h->traced += p.trace_slot + 1 < tmax ? 2 : 1;
  h->cur ^= 1;
  h->step += 2;
  return LBM_OK;
}

extern "C" {

size_t lbm_elastic_workspace_bytes(const lbm_elastic_config *cfg) {
  if (!config_ok(cfg, nullptr)) return 0;
  return make_layout(cfg).total;
}

lbm_status lbm_elastic_create(const lbm_elastic_config *cfg, void *d_workspace,
                              size_t workspace_bytes, void *cuda_stream, lbm_elastic_t **out) {
  std::string why;
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!config_ok(cfg, &why)) return fail(nullptr, LBM_ERR_ARG, why);
  Layout L = make_layout(cfg);
  if (!d_workspace) return fail(nullptr, LBM_ERR_WORKSPACE, "workspace is NULL");
  if ((uintptr_t)d_workspace % kAlign)
    return fail(nullptr, LBM_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(nullptr, LBM_ERR_WORKSPACE,
                "workspace too small: need " + std::to_string(L.total) + " bytes");
  lbm_elastic_t *h = new (std::nothrow) lbm_elastic();
  if (!h) return fail(nullptr, LBM_ERR_ARG, "out of host memory");
  h->cfg = *cfg;
  h->L = L;
  h->ws = (char *)d_workspace;
  h->stream = (cudaStream_t)cuda_stream;
  lbm_status s = clear_state(h);
  if (s == LBM_OK) {
    // default material: homogeneous Poisson solid, rho0 = 1 (Lambda = 0)
    if (L.csize == 8) {
      fill_kernel<double><<<grid1d(L.mat_count, 256), 256, 0, h->stream>>>(
          at<double>(h, L.lam), L.mat_count, 0.0);
      fill_kernel<double><<<grid1d(L.mat_count, 256), 256, 0, h->stream>>>(
          at<double>(h, L.irho), L.mat_count, 1.0);
    } else {
      fill_kernel<float><<<grid1d(L.mat_count, 256), 256, 0, h->stream>>>(
          at<float>(h, L.lam), L.mat_count, 0.0f);
      fill_kernel<float><<<grid1d(L.mat_count, 256), 256, 0, h->stream>>>(
          at<float>(h, L.irho), L.mat_count, 1.0f);
    }
    s = check_launch(h, "material fill launch");
  }
  if (s == LBM_OK) s = upload_tile_order(h);
  if (s == LBM_OK) {
    cudaError_t e = cudaMemsetAsync(h->ws + L.rec_ptr, 0, ((size_t)L.rec_tiles + 1) * sizeof(int),
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = cuda_fail(h, e, "create");
  }
  if (s != LBM_OK) {
    g_create_error = h->err;
    delete h;
    return s;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_elastic_set_material(lbm_elastic_t *h, const double *rho0, const double *lambda,
                                    const double *mu, int on_device) {
  if (!h) return LBM_ERR_ARG;
  if (!rho0 || !lambda || !mu) return fail(h, LBM_ERR_ARG, "material pointer is NULL");
  const lbm_elastic_config &c = h->cfg;
  const Layout &L = h->L;
  int *flags = at<int>(h, L.flags) + 1;
  LBM_CUDA(h, cudaMemsetAsync(flags, 0, sizeof(int), h->stream));
  const long long total = c.material_per_cell ? (long long)c.nx * c.ny : c.ny;
  const long long chunk = c.material_per_cell ? (long long)L.stage_rows * c.nx : c.ny;
  double *stage = at<double>(h, L.stage);
  for (long long off = 0; off < total; off += chunk) {
    const long long n = off + chunk <= total ? chunk : total - off;
    const double *r = rho0 + off, *l = lambda + off, *m = mu + off;
    if (!on_device) {
      LBM_CUDA(h, cudaMemcpyAsync(stage, r, n * 8, cudaMemcpyHostToDevice, h->stream));
      LBM_CUDA(h, cudaMemcpyAsync(stage + n, l, n * 8, cudaMemcpyHostToDevice, h->stream));
      LBM_CUDA(h, cudaMemcpyAsync(stage + 2 * n, m, n * 8, cudaMemcpyHostToDevice, h->stream));
      r = stage;
      l = stage + n;
      m = stage + 2 * n;
    }
    if (L.csize == 8)
      material_kernel<double><<<grid1d(n, 256), 256, 0, h->stream>>>(
          r, l, m, n, c.material_per_cell, c.nx, L.pitch, off, at<double>(h, L.lam),
          at<double>(h, L.irho), flags);
    else
      material_kernel<float><<<grid1d(n, 256), 256, 0, h->stream>>>(
          r, l, m, n, c.material_per_cell, c.nx, L.pitch, off, at<float>(h, L.lam),
          at<float>(h, L.irho), flags);
    lbm_status s = check_launch(h, "material kernel launch");
    if (s) return s;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  int fl = 0;
  LBM_CUDA(h, cudaMemcpyAsync(&fl, flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->lambda_nonzero = (fl & 1) != 0;
  if (fl & 4) return fail(h, LBM_ERR_ARG, "material: rho0 <= 0 or a non-finite value");
  if (fl & 2) {
    h->err = "material: mu/rho0 differs from b^2 = 1/3; v_S stays 1/sqrt(3)";
    return LBM_WARN_VS_NOT_B;
  }
  return LBM_OK;
}

lbm_status lbm_elastic_set_sources(lbm_elastic_t *h, const lbm_source *src, int n) {
  if (!h) return LBM_ERR_ARG;
  if (n < 0 || (n > 0 && !src)) return fail(h, LBM_ERR_ARG, "invalid source list");
  if (n > h->cfg.max_sources)
    return fail(h, LBM_ERR_CAPACITY, "more sources than max_sources");
  std::vector<SourceDev> v((size_t)n);
  for (int k = 0; k < n; ++k) {
    const lbm_source &s = src[k];
    const double vals[9] = {s.x, s.y, s.sigma, s.dir_x, s.dir_y, s.amplitude, s.f_peak, s.t0, s.r_cut};
    for (double d : vals)
      if (!std::isfinite(d)) return fail(h, LBM_ERR_ARG, "source value not finite");
    if (!(s.sigma > 0.0) || s.r_cut < 0.0) return fail(h, LBM_ERR_ARG, "sigma <= 0 or r_cut < 0");
    SourceDev &q = v[k];
    q.x = s.x;
    q.y = s.y;
    q.inv2s2 = 1.0 / (2.0 * s.sigma * s.sigma);
    q.rcut2 = s.r_cut * s.r_cut;
    if (std::fabs(s.x) > 1e9 || std::fabs(s.y) > 1e9 || s.r_cut > 1e9)
      return fail(h, LBM_ERR_ARG, "source position or r_cut out of range");
    q.xc = (int)std::floor(s.x + 0.5);
    q.yc = (int)std::floor(s.y + 0.5);
    q.rb = (int)std::ceil(s.r_cut) + 1;
    q.pad = 0;
    q.ax = s.amplitude * s.dir_x;
    q.ay = s.amplitude * s.dir_y;
    q.dirx = s.dir_x;
    q.diry = s.dir_y;
    q.pif2 = M_PI * M_PI * s.f_peak * s.f_peak;
    q.t0 = s.t0;
    q.inv2s2_f = (float)q.inv2s2;
    q.pif2_f = (float)q.pif2;
    q.ax_f = (float)q.ax;
    q.ay_f = (float)q.ay;
  }
  // bounding box of every footprint: clipped to the grid on a non-periodic
  // axis, the whole axis when it wraps around a periodic one
  int bx0 = h->cfg.nx, bx1 = -1, by0 = h->cfg.ny, by1 = -1;
  const bool perx = h->cfg.bc_left == LBM_BC_PERIODIC, pery = h->cfg.bc_top == LBM_BC_PERIODIC;
  for (const SourceDev &q : v) {
    const long long lo_x = (long long)q.xc - q.rb, hi_x = (long long)q.xc + q.rb;
    const long long lo_y = (long long)q.yc - q.rb, hi_y = (long long)q.yc + q.rb;
    if (perx && (lo_x < 0 || hi_x >= h->cfg.nx)) {
      bx0 = 0;
      bx1 = h->cfg.nx - 1;
    } else {
      bx0 = (int)std::min<long long>(bx0, std::max<long long>(lo_x, 0));
      bx1 = (int)std::max<long long>(bx1, std::min<long long>(hi_x, h->cfg.nx - 1));
    }
    if (pery && (lo_y < 0 || hi_y >= h->cfg.ny)) {
      by0 = 0;
      by1 = h->cfg.ny - 1;
    } else {
      by0 = (int)std::min<long long>(by0, std::max<long long>(lo_y, 0));
      by1 = (int)std::max<long long>(by1, std::min<long long>(hi_y, h->cfg.ny - 1));
    }
  }
  h->src_box[0] = bx0;
  h->src_box[1] = bx1;
  h->src_box[2] = by0;
  h->src_box[3] = by1;
  h->src_host = v;
  std::vector<int4> bounds((size_t)n);
  for (int k = 0; k < n; ++k) bounds[k] = make_int4(v[k].xc, v[k].yc, v[k].rb, 0);
  if (n) {
    LBM_CUDA(h, cudaMemcpyAsync(h->ws + h->L.src, h->src_host.data(), n * sizeof(SourceDev),
                                cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->ws + h->L.srcb, bounds.data(), n * sizeof(int4),
                                cudaMemcpyHostToDevice, h->stream));
  }
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->nsrc = n;
  return upload_tile_order(h);
}

lbm_status lbm_elastic_set_sponges(lbm_elastic_t *h, int top, int bottom, int left, int right,
                                   double amax) {
  if (!h) return LBM_ERR_ARG;
  lbm_elastic_config c = h->cfg;
  c.sponge_top = top;
  c.sponge_bottom = bottom;
  c.sponge_left = left;
  c.sponge_right = right;
  c.sponge_amax = amax;
  std::string why;
  if (!config_ok(&c, &why)) return fail(h, LBM_ERR_ARG, why);
  h->cfg = c;
  return LBM_OK;
}

lbm_status lbm_elastic_set_receivers(lbm_elastic_t *h, const int *xy, int n) {
  if (!h) return LBM_ERR_ARG;
  if (n < 0 || (n > 0 && !xy)) return fail(h, LBM_ERR_ARG, "invalid receiver list");
  if (n > h->cfg.max_receivers)
    return fail(h, LBM_ERR_CAPACITY, "more receivers than max_receivers");
  const Layout &L = h->L;
  for (int r = 0; r < n; ++r)
    if (xy[2 * r] < 0 || xy[2 * r] >= h->cfg.nx || xy[2 * r + 1] < 0 || xy[2 * r + 1] >= h->cfg.ny)
      return fail(h, LBM_ERR_ARG, "receiver outside the grid");
  // CSR by receiver tile (counting sort)
  std::vector<int> ptr((size_t)L.rec_tiles + 1, 0), sxy(2 * (size_t)n + 2), sid((size_t)n + 1);
  auto tile_of = [&](int r) {
    return (xy[2 * r + 1] / kRecTileY) * L.rec_tiles_x + xy[2 * r] / kRecTileX;
  };
  for (int r = 0; r < n; ++r) ptr[tile_of(r) + 1]++;
  for (int t = 0; t < L.rec_tiles; ++t) ptr[t + 1] += ptr[t];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int r = 0; r < n; ++r) {
    const int k = fill[tile_of(r)]++;
    sxy[2 * k] = xy[2 * r];
    sxy[2 * k + 1] = xy[2 * r + 1];
    sid[k] = r;
  }
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.rec_ptr, ptr.data(), ptr.size() * sizeof(int),
                              cudaMemcpyHostToDevice, h->stream));
  if (n) {
    LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.rec_xy, sxy.data(), 2 * (size_t)n * sizeof(int),
                                cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->ws + L.rec_id, sid.data(), (size_t)n * sizeof(int),
                                cudaMemcpyHostToDevice, h->stream));
  }
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));  // host vectors die here
  h->rec_box[0] = h->cfg.nx;
  h->rec_box[1] = -1;
  h->rec_box[2] = h->cfg.ny;
  h->rec_box[3] = -1;
  for (int r = 0; r < n; ++r) {
    h->rec_box[0] = std::min(h->rec_box[0], xy[2 * r]);
    h->rec_box[1] = std::max(h->rec_box[1], xy[2 * r]);
    h->rec_box[2] = std::min(h->rec_box[2], xy[2 * r + 1]);
    h->rec_box[3] = std::max(h->rec_box[3], xy[2 * r + 1]);
  }
  h->nrec = n;
  h->traced = 0;
  h->rec_host.assign(xy, xy + 2 * (size_t)n);
  return upload_tile_order(h);
}

lbm_status lbm_elastic_reset(lbm_elastic_t *h) {
  if (!h) return LBM_ERR_ARG;
  return clear_state(h);
}

lbm_status lbm_elastic_step(lbm_elastic_t *h, int nsteps) {
  if (!h) return LBM_ERR_ARG;
  if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
  int spl = h->steps_per_launch;
  if (spl < 0) {
    // FP64 steps are bound by the FP64 pipe, not by memory; with the
    // density-gradient force the 16-bit step is issue-bound and the larger
    // two-step window costs more than the bytes it saves
    const bool b16 = h->cfg.storage == LBM_F16 || h->cfg.storage == LBM_BF16;
    spl = (h->cfg.storage == LBM_F64 || (b16 && h->lambda_nonzero)) ? 1 : 2;
  }
  int s = 0;
  if (spl == 2)
    for (; s + 2 <= nsteps; s += 2)
      if (lbm_status st = handle_step2(h)) return st;
  for (; s < nsteps; ++s)
    if (lbm_status st = handle_step(h, nullptr)) return st;
  return LBM_OK;
}

lbm_status lbm_elastic_set_steps_per_launch(lbm_elastic_t *h, int steps) {
  if (!h) return LBM_ERR_ARG;
  if (steps < 1 || steps > 2) return fail(h, LBM_ERR_ARG, "steps per launch must be 1 or 2");
  h->steps_per_launch = steps;
  return LBM_OK;
}

long long lbm_elastic_step_index(const lbm_elastic_t *h) { return h ? h->step : -1; }

lbm_status lbm_elastic_read_fields(lbm_elastic_t *h, double *ux, double *uy, double *vx,
                                   double *vy, double *rho, double *pxx, double *pxy,
                                   double *pyy, int on_device) {
  if (!h) return LBM_ERR_ARG;
  const lbm_elastic_config &c = h->cfg;
  const Layout &L = h->L;
  double *outs[8] = {ux, uy, vx, vy, rho, pxx, pxy, pyy};
  StepParams p = base_params(h);
  if (on_device) {
    p.row0 = 0;
    p.nrows = c.ny;
    for (int k = 0; k < 8; ++k) p.out[k] = outs[k];
    lbm_status s = launch_step(h, p, 1, c.ny);
    if (s) return s;
  } else {
    double *stage = at<double>(h, L.stage);
    for (int r0 = 0; r0 < c.ny; r0 += L.stage_rows) {
      const int nr = (r0 + L.stage_rows <= c.ny) ? L.stage_rows : c.ny - r0;
      const long long chunk = (long long)nr * c.nx;
      p.row0 = r0;
      p.nrows = nr;
      for (int k = 0; k < 8; ++k) p.out[k] = outs[k] ? stage + k * chunk : nullptr;
      lbm_status s = launch_step(h, p, 1, nr);
      if (s) return s;
      for (int k = 0; k < 8; ++k)
        if (outs[k])
          LBM_CUDA(h, cudaMemcpyAsync(outs[k] + (long long)r0 * c.nx, stage + k * chunk,
                                      chunk * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    }
  }
  return sync_flags(h);
}

int lbm_elastic_traces_recorded(const lbm_elastic_t *h) { return h ? h->traced : 0; }

lbm_status lbm_elastic_read_traces(lbm_elastic_t *h, double *out, int on_device) {
  if (!h) return LBM_ERR_ARG;
  const size_t bytes = (size_t)h->traced * h->nrec * 4 * sizeof(double);
  if (bytes) {
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    LBM_CUDA(h, cudaMemcpyAsync(out, h->ws + h->L.traces, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
  }
  return sync_flags(h);
}

lbm_status lbm_elastic_set_state(lbm_elastic_t *h, const double *f9, const double *u2,
                                 long long step, int on_device) {
  if (!h) return LBM_ERR_ARG;
  if (!f9) return fail(h, LBM_ERR_ARG, "f9 is NULL");
  if (step < 0) return fail(h, LBM_ERR_ARG, "step < 0");
  lbm_status s = f_io(h, nullptr, f9, on_device);
  if (s) return s;
  s = u_io(h, nullptr, u2, on_device);
  if (s) return s;
  LBM_CUDA(h, cudaMemsetAsync(h->ws + h->L.flags, 0, 64, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->step = step;
  h->traced = 0;
  return LBM_OK;
}

lbm_status lbm_elastic_get_state(lbm_elastic_t *h, double *f9, double *u2, int on_device) {
  if (!h) return LBM_ERR_ARG;
  if (f9) {
    lbm_status s = f_io(h, f9, nullptr, on_device);
    if (s) return s;
  }
  if (u2) {
    lbm_status s = u_io(h, u2, nullptr, on_device);
    if (s) return s;
  }
  return sync_flags(h);
}

size_t lbm_elastic_checkpoint_bytes(const lbm_elastic_t *h) {
  if (!h) return 0;
  return 256 + align_up(9 * (size_t)h->L.plane * h->L.tsize, kAlign) +
         2 * (size_t)h->L.plane * h->L.usize;
}

lbm_status lbm_elastic_save(lbm_elastic_t *h, void *buf, int on_device) {
  if (!h) return LBM_ERR_ARG;
  if (!buf) return fail(h, LBM_ERR_ARG, "buffer is NULL");
  long long hdr[8] = {(long long)kMagic, h->cfg.nx, h->cfg.ny, h->cfg.storage,
                      (long long)h->L.usize, h->step, h->cfg.store_scale_log2, 0};
  char *b = (char *)buf;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t fb = 9 * (size_t)h->L.plane * h->L.tsize;
  if (on_device)
    LBM_CUDA(h, cudaMemcpyAsync(b, hdr, sizeof(hdr), cudaMemcpyHostToDevice, h->stream));
  else
    memcpy(b, hdr, sizeof(hdr));
  LBM_CUDA(h, cudaMemcpyAsync(b + 256, h->ws + h->L.f[h->cur], fb, k, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(b + 256 + align_up(fb, kAlign), h->ws + h->L.u,
                              2 * (size_t)h->L.plane * h->L.usize, k, h->stream));
  return sync_flags(h);
}

lbm_status lbm_elastic_load(lbm_elastic_t *h, const void *buf, int on_device) {
  if (!h) return LBM_ERR_ARG;
  if (!buf) return fail(h, LBM_ERR_ARG, "buffer is NULL");
  long long hdr[8];
  const char *b = (const char *)buf;
  if (on_device) {
    LBM_CUDA(h, cudaMemcpyAsync(hdr, b, sizeof(hdr), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  } else {
    memcpy(hdr, b, sizeof(hdr));
  }
  if (hdr[0] != (long long)kMagic || hdr[1] != h->cfg.nx || hdr[2] != h->cfg.ny ||
      hdr[3] != h->cfg.storage || hdr[4] != (long long)h->L.usize || hdr[5] < 0 ||
      hdr[6] != h->cfg.store_scale_log2)
    return fail(h, LBM_ERR_ARG, "checkpoint does not match this configuration");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t fb = 9 * (size_t)h->L.plane * h->L.tsize;
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + h->L.f[h->cur], b + 256, fb, k, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(h->ws + h->L.u, b + 256 + align_up(fb, kAlign),
                              2 * (size_t)h->L.plane * h->L.usize, k, h->stream));
  LBM_CUDA(h, cudaMemsetAsync(h->ws + h->L.flags, 0, 64, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->step = hdr[5];
  h->traced = 0;
  return LBM_OK;
}

lbm_status lbm_elastic_moment_sums(lbm_elastic_t *h, double out[7]) {
  if (!h) return LBM_ERR_ARG;
  if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
  const Layout &L = h->L;
  double *partials = at<double>(h, L.partials);
  const void *f = h->ws + L.f[h->cur];
  const void *u = h->ws + L.u;
  const double isc = 1.0 / store_scale(h->cfg);
  if (h->cfg.storage == LBM_F16 || h->cfg.storage == LBM_BF16) {
    if (h->cfg.storage == LBM_F16 && L.usize == 8)
      moments_partial_kernel<__half, double><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
          (const __half *)f, (const double *)u, L.plane, L.pitch, L.fplane, L.frow, h->cfg.nx,
          h->cfg.ny, partials, isc);
    else if (h->cfg.storage == LBM_F16)
      moments_partial_kernel<__half, float><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
          (const __half *)f, (const float *)u, L.plane, L.pitch, L.fplane, L.frow, h->cfg.nx,
          h->cfg.ny, partials, isc);
    else if (L.usize == 8)
      moments_partial_kernel<__nv_bfloat16, double><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
          (const __nv_bfloat16 *)f, (const double *)u, L.plane, L.pitch, L.fplane, L.frow,
          h->cfg.nx, h->cfg.ny, partials, isc);
    else
      moments_partial_kernel<__nv_bfloat16, float><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
          (const __nv_bfloat16 *)f, (const float *)u, L.plane, L.pitch, L.fplane, L.frow,
          h->cfg.nx, h->cfg.ny, partials, isc);
  } else if (h->cfg.storage == LBM_F64)
    moments_partial_kernel<double, double><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
        (const double *)f, (const double *)u, L.plane, L.pitch, L.fplane, L.frow, h->cfg.nx,
        h->cfg.ny, partials);
  else if (L.usize == 8)
    moments_partial_kernel<float, double><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
        (const float *)f, (const double *)u, L.plane, L.pitch, L.fplane, L.frow, h->cfg.nx,
        h->cfg.ny, partials);
  else
    moments_partial_kernel<float, float><<<kRedBlocks, kRedThreads, 0, h->stream>>>(
        (const float *)f, (const float *)u, L.plane, L.pitch, L.fplane, L.frow, h->cfg.nx,
        h->cfg.ny, partials);
  lbm_status s = check_launch(h, "moment sums launch");
  if (s) return s;
  moments_final_kernel<<<1, kRedThreads, 0, h->stream>>>(partials, kRedBlocks,
                                                          partials + 8 * kRedBlocks);
  s = check_launch(h, "moment sums launch");
  if (s) return s;
  LBM_CUDA(h, cudaMemcpyAsync(out, partials + 8 * kRedBlocks, 7 * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
  return sync_flags(h);
}

lbm_status lbm_elastic_sync(lbm_elastic_t *h) {
  if (!h) return LBM_ERR_ARG;
  return sync_flags(h);
}

lbm_status lbm_elastic_destroy(lbm_elastic_t *h) {
  if (!h) return LBM_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  delete h;
  return LBM_OK;
}

const char *lbm_elastic_last_error(const lbm_elastic_t *h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

const char *lbm_elastic_status_string(int s) {
  switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_WARN_VS_NOT_B: return "LBM_WARN_VS_NOT_B";
    case LBM_ERR_ARG: return "LBM_ERR_ARG";
    case LBM_ERR_UNSUPPORTED: return "LBM_ERR_UNSUPPORTED";
    case LBM_ERR_WORKSPACE: return "LBM_ERR_WORKSPACE";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_CAPACITY: return "LBM_ERR_CAPACITY";
    default: return "unknown status";
  }
}

long long lbm_elastic_kernel_launches(const lbm_elastic_t *h) { return h ? h->launches : 0; }

}  // extern "C"

// ------------------------------------------------------------ no-allocation entry point
//
// A handle needs a workspace from its caller.  Some callers cannot provide
// one and cannot let the library allocate either: code whose device memory
// is all pre-reserved by another allocator (a framework's caching pool, a
// fixed arena), or code running where a cudaMalloc would fail, or would stall
// the whole device at a bad moment.  For them the moment sums are also
// available without any workspace: the per-block partial sums go to the
// file-scope array below instead.  The array is part of the library image, so
// every GPU that loads the library holds its 19,520 bytes until the process
// exits.
namespace {

constexpr int kNoAllocScratchDoubles = (kRedBlocks + 1) * 8;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static_assert(kNoAllocScratchDoubles * sizeof(double) == LBM_NOALLOC_SCRATCH_BYTES,
              "scratch size stated in lbm_elastic.h");
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace

extern "C" lbm_status lbm_elastic_moment_sums_noalloc(const void *f9, const void *u2,
                                                       int storage, int u_fp64, int nx, int ny,
                                                       int pitch, double *out7, int out_on_device,
                                                       void *cuda_stream) {
  if (!f9 || !u2 || !out7) return fail(nullptr, LBM_ERR_ARG, "noalloc: NULL pointer");
  if (storage != LBM_F64 && storage != LBM_F32)
    return fail(nullptr, LBM_ERR_UNSUPPORTED, "noalloc: storage must be LBM_F64 or LBM_F32");
  if (nx < 1 || ny < 1 || pitch < nx) return fail(nullptr, LBM_ERR_ARG, "noalloc: bad sizes");
  if (9LL * pitch * ny > LBM_NOALLOC_MAX_ELEMENTS)
    return fail(nullptr, LBM_ERR_ARG, "noalloc: grid beyond the maximum of this entry point");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(nullptr, LBM_ERR_UNSUPPORTED, "noalloc: device index too large");
  double *scratch = nullptr;
  {
    // once per device, with that device current: the array's device address
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
      g_noalloc_ptr[dev] = (double *)ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long plane = (long long)pitch * ny;
  // every partial slot read by the final pass is written by this call first,
  // so nothing left from an earlier call needs clearing
  if (storage == LBM_F64)
    moments_partial_kernel<double, double><<<kRedBlocks, kRedThreads, 0, s>>>(
        (const double *)f9, (const double *)u2, plane, pitch, plane, pitch, nx, ny, scratch);
  else if (u_fp64)
    moments_partial_kernel<float, double><<<kRedBlocks, kRedThreads, 0, s>>>(
        (const float *)f9, (const double *)u2, plane, pitch, plane, pitch, nx, ny, scratch);
  else
    moments_partial_kernel<float, float><<<kRedBlocks, kRedThreads, 0, s>>>(
        (const float *)f9, (const float *)u2, plane, pitch, plane, pitch, nx, ny, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  moments_final_kernel<<<1, kRedThreads, 0, s>>>(scratch, kRedBlocks, scratch + 8 * kRedBlocks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  e = cudaMemcpyAsync(out7, scratch + 8 * kRedBlocks, 7 * sizeof(double),
                      out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !out_on_device) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
