// Host side of the adjoint API: forward run with checkpoints, reverse sweep
// that recomputes each segment's forward steps (storing their density
// gradients) and runs the adjoint steps backwards, gradients.  Device memory
// comes from the caller's adjoint workspace.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "adjoint_kernels.cuh"
#include "lbm_internal.h"
#include "step2_lam.cuh"

using namespace lbm;

namespace {

constexpr size_t kAdjAlign = 256;
// steps whose Lambda-gradient shares are summed in the compute type before
// they are added to the FP64 sum (step 0 always flushes)
#ifndef LBM_ADJ_FLUSH_STEPS
#define LBM_ADJ_FLUSH_STEPS 16
#endif
constexpr int kFlushSteps = LBM_ADJ_FLUSH_STEPS;

size_t aup(size_t v) { return (v + kAdjAlign - 1) / kAdjAlign * kAdjAlign; }

struct AdjLayout {
  size_t abar[2] = {0, 0}, gbar = 0, wbar = 0, rbar = 0, ubar = 0, jrec = 0, glam = 0, gpart = 0,
         gamp = 0, grad = 0, ckpt = 0, total = 0;
  size_t state_f = 0, state_u = 0, ckpt_bytes = 0, csize = 0;
  int nck = 0;
};

AdjLayout adj_layout(const lbm_elastic_t *h, int nsteps, int K) {
  AdjLayout A;
  const Layout &L = h->L;
  A.csize = L.csize;
  const size_t pl = (size_t)L.plane;
  A.state_f = 9 * pl * L.tsize;
  A.state_u = 2 * pl * L.usize;
  A.ckpt_bytes = aup(A.state_f) + aup(A.state_u);
  A.nck = (nsteps + K - 1) / K;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = aup(off + b);
    return o;
  };
  A.abar[0] = take(9 * pl * A.csize);
  A.abar[1] = take(9 * pl * A.csize);
  A.gbar = take(9 * pl * A.csize);
  A.wbar = take(2 * pl * A.csize);
  A.rbar = take(pl * A.csize);
  A.ubar = take(2 * pl * A.csize);
  const size_t nr = (size_t)std::max(1, h->cfg.max_receivers);
  A.jrec = take((size_t)nsteps * nr * 2 * A.csize);
  A.glam = take(pl * sizeof(double));
  A.gpart = take(pl * A.csize);
  A.gamp = take((size_t)std::max(1, h->cfg.max_sources) * sizeof(double));
  A.grad = take((size_t)K * 2 * pl * A.csize);
  A.ckpt = take((size_t)(A.nck + 1) * A.ckpt_bytes);  // + the final state
  A.total = off;
  return A;
}

// per thread: calls without a handle on different threads must not race on it
thread_local std::string g_adj_create_error;

// Dense FP64 [n][ny][nx] planes <-> padded planes of type C with the given
// row and plane strides.
template <class C>
__global__ void dense_in_kernel(const double *d, int n, int nx, int ny, C *o, long long oplane,
                                long long orow) {
  const long long tot = (long long)n * nx * ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
       k += (long long)gridDim.x * blockDim.x) {
    const long long pl = k / ((long long)nx * ny), r = k % ((long long)nx * ny);
    o[pl * oplane + (r / nx) * orow + r % nx] = d ? C(d[k]) : C(0);
  }
}

template <class C>
__global__ void dense_out_kernel(const C *o, long long oplane, long long orow, int n, int nx,
                                 int ny, double *d) {
  const long long tot = (long long)n * nx * ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
       k += (long long)gridDim.x * blockDim.x) {
    const long long pl = k / ((long long)nx * ny), r = k % ((long long)nx * ny);
    d[k] = (double)o[pl * oplane + (r / nx) * orow + r % nx];
  }
}

// g_Lambda [ny][pitch] -> dense dJ/dLambda, dJ/dlambda = -g / (rho0 b^2),
// dJ/dmu = g / (rho0 b^2) (Lambda = (mu - lambda)/(rho0 b^2), Eq. 32).
template <class C>
__global__ void grad_out_kernel(const double *g, const C *irho, int per_cell, int nx, int ny,
                                int pitch, double *gL, double *gl, double *gm) {
  const long long tot = (long long)nx * ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
       k += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(k / nx), x = (int)(k % nx);
    const double v = g[(long long)y * pitch + x];
    const double ir = (double)(per_cell ? irho[(long long)y * pitch + x] : irho[y]);
    if (gL) gL[k] = v;
    if (gl) gl[k] = -3.0 * ir * v;
    if (gm) gm[k] = 3.0 * ir * v;
  }
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max(1LL, std::min(b, 152LL * 16));
}

}  // namespace

struct lbm_adjoint {
  lbm_elastic_t *h = nullptr;
  int nsteps = 0, K = 1;
  char *ws = nullptr;
  AdjLayout A;
  bool f64 = false;
  bool forward_done = false;
  long long n_start = 0;  // step index of the handle when forward began
  int traced_start = 0;
  int cur_a = 0;          // adjoint buffer holding the current adjoint state
  bool fused = true;      // one fused kernel per adjoint step (else three)
  int grads_seg = -1;     // segment whose density gradients the slots hold
  long long launches = 0;
  std::string err;
};

namespace {

lbm_status afail(lbm_adjoint_t *a, lbm_status s, const std::string &m) {
  if (a) a->err = m;
  else g_adj_create_error = m;
  return s;
}

#define ADJ_CUDA(a, call)                                                           \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return afail((a), LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

AdjParams params_of(lbm_adjoint_t *a, long long n) {
  AdjParams P;
  memset(&P, 0, sizeof(P));
  P.p = handle_step_params(a->h);
  P.p.n = n;
  P.abar = a->ws + a->A.abar[a->cur_a];
  P.abar_out = a->ws + a->A.abar[a->cur_a ^ 1];
  P.gbar = a->ws + a->A.gbar;
  P.wbar = a->ws + a->A.wbar;
  P.rbar = a->ws + a->A.rbar;
  P.ufield = nullptr;
  P.jrec = a->ws + a->A.jrec;
  P.grad = nullptr;
  P.g_lam = (double *)(a->ws + a->A.glam);
  P.g_part = a->ws + a->A.gpart;
  P.flush = 0;
  P.g_amp = nullptr;
  P.lam_any = a->h->lambda_nonzero ? 1 : 0;
  return P;
}

lbm_status adj_launch(lbm_adjoint_t *a, const AdjParams &P) {
  const cudaError_t e = a->f64 ? adj_step_f64(P, a->fused, a->h->stream)
                               : adj_step_f32(P, a->fused, a->h->stream);
  if (e != cudaSuccess)
    return afail(a, LBM_ERR_CUDA, std::string("adjoint step: ") + cudaGetErrorString(e));
  a->launches += a->fused ? 1 : (P.lam_any ? 3 : 2);
  a->cur_a ^= 1;
  return LBM_OK;
}

// Copies the handle's current state into (save) or out of (!save) slot k.
lbm_status ckpt_io(lbm_adjoint_t *a, int k, bool save) {
  lbm_elastic_t *h = a->h;
  char *slot = a->ws + a->A.ckpt + (size_t)k * a->A.ckpt_bytes;
  char *f = h->ws + h->L.f[h->cur], *u = h->ws + h->L.u;
  char *sf = slot, *su = slot + aup(a->A.state_f);
  ADJ_CUDA(a, cudaMemcpyAsync(save ? sf : f, save ? f : sf, a->A.state_f,
                              cudaMemcpyDeviceToDevice, h->stream));
  ADJ_CUDA(a, cudaMemcpyAsync(save ? su : u, save ? u : su, a->A.state_u,
                              cudaMemcpyDeviceToDevice, h->stream));
  return LBM_OK;
}

char *grad_slot(lbm_adjoint_t *a, int k) {
  return a->ws + a->A.grad + (size_t)k * 2 * a->h->L.plane * a->A.csize;
}

lbm_status capture_step(lbm_adjoint_t *a, int slot) {
  if (lbm_status st = handle_step(a->h, grad_slot(a, slot)))
    return afail(a, st, std::string("forward step: ") + a->h->err);
  return LBM_OK;
}

// FP32 states: steps n and n + 1 in one launch of the two-step
// gradient-force kernel, storing both steps' density gradients into records
// slot and slot + 1 (the states and records of two capture_step calls, bit
// for bit).  FP64 states keep one step per launch (FP64-arithmetic bound).
bool two_step_capture(const lbm_adjoint_t *a) { return !a->f64; }

lbm_status capture_two(lbm_adjoint_t *a, int slot) {
  lbm_elastic_t *h = a->h;
  StepParams p = handle_step_params(h);
  p.reverse = (int)((h->step >> 1) & 1);
  p.grad_out = grad_slot(a, slot);
  const int tmax = h->cfg.max_steps_traced;
  if (h->nrec > 0 && h->traced < tmax) p.trace_slot = h->traced;
  launch_step2_lam_f32(p, h->cfg.u_fp64 != 0, h->stream);
  h->launches++;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return afail(a, LBM_ERR_CUDA, std::string("forward steps: ") + cudaGetErrorString(e));
  if (p.trace_slot >= 0) h->traced += p.trace_slot + 1 < tmax ? 2 : 1;
  h->cur ^= 1;
  h->step += 2;
  return LBM_OK;
}

// Steps n0 .. n1 - 1 of a segment, recording their gradients in slots
// 0 .. n1 - n0 - 1.
lbm_status capture_segment(lbm_adjoint_t *a, int n0, int n1) {
  for (int n = n0; n < n1;) {
    if (two_step_capture(a) && n + 1 < n1) {
      if (lbm_status st = capture_two(a, n - n0)) return st;
      n += 2;
    } else {
      if (lbm_status st = capture_step(a, n - n0)) return st;
      n += 1;
    }
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_adjoint_workspace_bytes(const lbm_elastic_t *h, int nsteps, int checkpoint_every) {
  if (!h || nsteps < 1 || checkpoint_every < 1) return 0;
  return adj_layout(h, nsteps, checkpoint_every).total;
}

lbm_status lbm_adjoint_create(lbm_elastic_t *h, int nsteps, int checkpoint_every,
                              void *d_workspace, size_t bytes, lbm_adjoint_t **out) {
  if (!out) return afail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!h || nsteps < 1 || checkpoint_every < 1)
    return afail(nullptr, LBM_ERR_ARG, "need a handle, nsteps >= 1 and checkpoint_every >= 1");
  if (h->cfg.storage != LBM_F32 && h->cfg.storage != LBM_F64)
    return afail(nullptr, LBM_ERR_UNSUPPORTED, "the adjoint needs FP32 or FP64 storage");
  if (h->cfg.storage == LBM_F32 && h->cfg.u_fp64)
    return afail(nullptr, LBM_ERR_UNSUPPORTED, "the adjoint needs u in the storage precision");
  const AdjLayout A = adj_layout(h, nsteps, checkpoint_every);
  if (!d_workspace || bytes < A.total)
    return afail(nullptr, LBM_ERR_WORKSPACE, "adjoint workspace too small");
  if ((uintptr_t)d_workspace % kAdjAlign)
    return afail(nullptr, LBM_ERR_WORKSPACE, "adjoint workspace not 256-byte aligned");
  lbm_adjoint_t *a = new (std::nothrow) lbm_adjoint();
  if (!a) return afail(nullptr, LBM_ERR_ARG, "out of host memory");
  a->h = h;
  a->nsteps = nsteps;
  a->K = checkpoint_every;
  a->ws = (char *)d_workspace;
  a->A = A;
  a->f64 = h->cfg.storage == LBM_F64;
  *out = a;
  return LBM_OK;
}

lbm_status lbm_adjoint_forward(lbm_adjoint_t *a) {
  if (!a) return LBM_ERR_ARG;
  lbm_elastic_t *h = a->h;
  a->n_start = h->step;
  a->traced_start = h->traced;
  const int last = a->A.nck - 1;  // the segment whose gradients the sweep starts with
  for (int seg = 0; seg <= last; ++seg) {
    const int n0 = seg * a->K, n1 = std::min(a->nsteps, n0 + a->K);
    if (lbm_status st = ckpt_io(a, seg, true)) return st;
    if (seg < last) {
      // only checkpoints are kept: the handle's own stepping (two steps per
      // launch where it applies; the same states bit for bit)
      if (lbm_status st = lbm_elastic_step(h, n1 - n0))
        return afail(a, st, std::string("forward steps: ") + h->err);
    } else {
      if (lbm_status st = capture_segment(a, n0, n1)) return st;
    }
  }
  if (lbm_status st = ckpt_io(a, a->A.nck, true)) return st;
  a->forward_done = true;
  a->grads_seg = a->A.nck - 1;  // the forward run just stored the last segment's
  return LBM_OK;
}

lbm_status lbm_adjoint_backward(lbm_adjoint_t *a, const double *d_dtraces) {
  if (!a) return LBM_ERR_ARG;
  if (!a->forward_done) return afail(a, LBM_ERR_ARG, "lbm_adjoint_forward has not run");
  lbm_elastic_t *h = a->h;
  if (h->nrec > 0 && !d_dtraces) return afail(a, LBM_ERR_ARG, "trace adjoint is NULL");
  const size_t pl = (size_t)h->L.plane;
  cudaStream_t s = h->stream;
  a->cur_a = 0;
  ADJ_CUDA(a, cudaMemsetAsync(a->ws + a->A.abar[0], 0, 9 * pl * a->A.csize, s));
  if (h->nrec > 0) {
    const int *rid = (const int *)(h->ws + h->L.rec_id);
    const cudaError_t e =
        a->f64 ? adj_jrec_f64(d_dtraces, rid, h->nrec, a->nsteps, a->ws + a->A.jrec, s)
               : adj_jrec_f32(d_dtraces, rid, h->nrec, a->nsteps, a->ws + a->A.jrec, s);
    if (e != cudaSuccess)
      return afail(a, LBM_ERR_CUDA, std::string("receiver adjoints: ") + cudaGetErrorString(e));
    a->launches++;
  }
  ADJ_CUDA(a, cudaMemsetAsync(a->ws + a->A.glam, 0, pl * sizeof(double), s));
  ADJ_CUDA(a, cudaMemsetAsync(a->ws + a->A.gpart, 0, pl * a->A.csize, s));
  ADJ_CUDA(a, cudaMemsetAsync(a->ws + a->A.gamp, 0,
                              std::max(1, h->cfg.max_sources) * sizeof(double), s));
  const int traced_keep = h->traced;
  h->traced = h->cfg.max_steps_traced;  // the recomputation records no traces
  lbm_status st = LBM_OK;
  for (int seg = a->A.nck - 1; seg >= 0 && !st; --seg) {
    const int n0 = seg * a->K, n1 = std::min(a->nsteps, n0 + a->K);
    if (seg != a->grads_seg) {
      // recompute the segment from its checkpoint, storing its gradients
      if ((st = ckpt_io(a, seg, false))) break;
      h->step = a->n_start + n0;
      st = capture_segment(a, n0, n1);
      a->grads_seg = seg;
    }
    for (int n = n1 - 1; n >= n0 && !st; --n) {
      AdjParams P = params_of(a, a->n_start + n);
      P.jrec = a->ws + a->A.jrec + (size_t)n * h->nrec * 2 * a->A.csize;
      P.grad = grad_slot(a, n - n0);
      // the compute-type partial sum spans at most kFlushSteps steps
      P.flush = (n % kFlushSteps == 0) ? 1 : 0;
      P.g_amp = (double *)(a->ws + a->A.gamp);
      st = adj_launch(a, P);
    }
  }
  // the handle returns to the state the forward run ended in
  if (!st) st = ckpt_io(a, a->A.nck, false);
  h->step = a->n_start + a->nsteps;
  h->traced = traced_keep;
  return st;
}

lbm_status lbm_adjoint_gradients(lbm_adjoint_t *a, double *d_g_lambda, double *d_g_mu,
                                 double *d_g_Lambda, double *d_g_amp) {
  if (!a) return LBM_ERR_ARG;
  lbm_elastic_t *h = a->h;
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  const int g = grid_for((long long)nx * ny);
  if (a->f64)
    grad_out_kernel<double><<<g, 256, 0, h->stream>>>(
        (const double *)(a->ws + a->A.glam), (const double *)(h->ws + h->L.irho),
        h->cfg.material_per_cell, nx, ny, h->L.pitch, d_g_Lambda, d_g_lambda, d_g_mu);
  else
    grad_out_kernel<float><<<g, 256, 0, h->stream>>>(
        (const double *)(a->ws + a->A.glam), (const float *)(h->ws + h->L.irho),
        h->cfg.material_per_cell, nx, ny, h->L.pitch, d_g_Lambda, d_g_lambda, d_g_mu);
  ADJ_CUDA(a, cudaGetLastError());
  a->launches++;
  if (d_g_amp && h->nsrc > 0)
    ADJ_CUDA(a, cudaMemcpyAsync(d_g_amp, a->ws + a->A.gamp, h->nsrc * sizeof(double),
                                cudaMemcpyDeviceToDevice, h->stream));
  ADJ_CUDA(a, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_adjoint_set_state(lbm_adjoint_t *a, const double *d_abar9, const double *d_ubar2) {
  if (!a) return LBM_ERR_ARG;
  lbm_elastic_t *h = a->h;
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  const Layout &L = h->L;
  const int g = grid_for(9LL * nx * ny);
  char *ab = a->ws + a->A.abar[a->cur_a];
  if (a->f64) {
    dense_in_kernel<double><<<g, 256, 0, h->stream>>>(d_abar9, 9, nx, ny, (double *)ab, L.fplane, L.frow);
    dense_in_kernel<double><<<g, 256, 0, h->stream>>>(d_ubar2, 2, nx, ny, (double *)(a->ws + a->A.ubar), L.plane, L.pitch);
  } else {
    dense_in_kernel<float><<<g, 256, 0, h->stream>>>(d_abar9, 9, nx, ny, (float *)ab, L.fplane, L.frow);
    dense_in_kernel<float><<<g, 256, 0, h->stream>>>(d_ubar2, 2, nx, ny, (float *)(a->ws + a->A.ubar), L.plane, L.pitch);
  }
  ADJ_CUDA(a, cudaGetLastError());
  a->launches += 2;
  return LBM_OK;
}

lbm_status lbm_adjoint_get_state(lbm_adjoint_t *a, double *d_abar9, double *d_ubar2) {
  if (!a) return LBM_ERR_ARG;
  lbm_elastic_t *h = a->h;
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  const Layout &L = h->L;
  const int g = grid_for(9LL * nx * ny);
  const char *ab = a->ws + a->A.abar[a->cur_a];
  if (a->f64) {
    if (d_abar9) dense_out_kernel<double><<<g, 256, 0, h->stream>>>((const double *)ab, L.fplane, L.frow, 9, nx, ny, d_abar9);
    if (d_ubar2) dense_out_kernel<double><<<g, 256, 0, h->stream>>>((const double *)(a->ws + a->A.ubar), L.plane, L.pitch, 2, nx, ny, d_ubar2);
  } else {
    if (d_abar9) dense_out_kernel<float><<<g, 256, 0, h->stream>>>((const float *)ab, L.fplane, L.frow, 9, nx, ny, d_abar9);
    if (d_ubar2) dense_out_kernel<float><<<g, 256, 0, h->stream>>>((const float *)(a->ws + a->A.ubar), L.plane, L.pitch, 2, nx, ny, d_ubar2);
  }
  ADJ_CUDA(a, cudaGetLastError());
  ADJ_CUDA(a, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_adjoint_step_linear(lbm_adjoint_t *a) {
  if (!a) return LBM_ERR_ARG;
  AdjParams P = params_of(a, a->h->step);
  P.p.nsrc = 0;
  P.ufield = a->ws + a->A.ubar;
  return adj_launch(a, P);
}

lbm_status lbm_adjoint_set_fused(lbm_adjoint_t *a, int fused) {
  if (!a) return LBM_ERR_ARG;
  a->fused = fused != 0;
  return LBM_OK;
}

long long lbm_adjoint_kernel_launches(const lbm_adjoint_t *a) { return a ? a->launches : -1; }

lbm_status lbm_adjoint_destroy(lbm_adjoint_t *a) {
  if (!a) return LBM_ERR_ARG;
  delete a;
  return LBM_OK;
}

const char *lbm_adjoint_last_error(const lbm_adjoint_t *a) {
  return a ? a->err.c_str() : g_adj_create_error.c_str();
}

}  // extern "C"
