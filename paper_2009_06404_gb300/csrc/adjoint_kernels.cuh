// Reverse-time (adjoint) step: the exact transpose of the linear part of
// one step (pull streaming with the wall rules of Sec. 6, moments, the
// centred density gradient of Eq. 10 with its wall ghosts, the implicit
// absorbing layer of Eq. 44, the BGK collision with forcing of Eqs. 11-18,
// and u += j / rho0), plus the accumulation of the gradients with respect to
// Lambda = (mu - lambda)/(rho0 b^2) per cell and to each source amplitude.
//
// Per cell x the step maps the pulled populations g_i(x), the force
// H(x) = G(x) + F(x) (G = Lambda b^2 grad rho, F the body force) and u(x) to
//   j   = sigma (m + H/2),                  sigma = 1 / (1 + A/2)
//   S   = sigma H - A sigma m
//   f*_i = (1 - w) g_i + w f^eq_i(rho, j, P) + (1 - w/2) 3 w_i c_i.S,  w = 1/tau
//   u'  = u + j / rho0.
// Its transpose, given the adjoint a_i of f*_i and jb of j, is
//   rho_b = w sum_i a_i w_i (2 - 1.5 |c_i|^2)
//   j_b  += w sum_i a_i 3 w_i c_i,   S_b = (1 - w/2) sum_i a_i 3 w_i c_i
//   P_b   = w sum_i a_i 4.5 w_i (c_i c_i - b^2 I)     (off-diagonal counted twice)
//   H_b   = sigma S_b + sigma/2 j_b,   m_b = sigma j_b - A sigma S_b
//   g_b,i = (1 - w) a_i + rho_b + c_i.m_b + c_i c_i : P_b,
// then H_b feeds the density-gradient adjoint (a divergence of
// Lambda b^2 H_b / 2 with the same wall ghosts), and the pull transposes to
// a push: the adjoint of f*_j(y) is the adjoint of the pulled population j
// at y + c_j, or, where that link leaves through a wall, the wall rule's
// transpose at y (with the anti-bounce-back's extrapolated rho and
// tangential stress spread back over the moments of y and, for the linear
// rule, of the cell inside it).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct AdjParams {
  StepParams p;        // grid, boundaries, layers, material, sources, step n
  const void *abar;    // adjoint of f* of step n, population layout of p
  void *abar_out;      // adjoint of f* of step n - 1
  void *gbar;          // adjoint of the pulled populations (scratch, same layout)
  void *wbar;          // Lambda b^2 H_b / 2, 2 planes (scratch)
  void *rbar;          // adjoint of the streamed density, 1 plane (scratch)
  const void *ufield;  // adjoint of u as 2 full planes (transpose tests), or null
  const void *jrec;    // else: per receiver (sorted order), the adjoint of j/rho0 there
  const void *grad;    // the forward's centred density gradient of step n, 2 planes
  double *g_lam;       // dJ/dLambda, one plane (FP64)
  double *g_amp;       // dJ/d amplitude, per source (FP64)
  int lam_any;         // some Lambda != 0
};

template <class C>
__device__ __forceinline__ const C *cp(const void *v) { return (const C *)v; }

// Local transpose of the collision, forcing, sponge and displacement update,
// and the gradient accumulation.  Blocks of 32 x 8 cells; inactive lanes of
// ragged blocks take part in the warp-wide source culling only.
template <class C>
__global__ void __launch_bounds__(256) adj_local_kernel(const AdjParams a) {
  const StepParams &p = a.p;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  const bool active = x < p.nx && y < p.ny;
  const int xc = x < p.nx ? x : p.nx - 1, yc = y < p.ny ? y : p.ny - 1;
  const int c = yc * p.pitch + xc;
  const long long cf = (long long)yc * p.frow + xc;
  C av[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) av[i] = cp<C>(a.abar)[cf + i * p.fplane];
  const C irho = mat_at<C>(p.irho, p.mat_per_cell, xc, yc, p.pitch);
  // adjoint of j from u' = u + j/rho0 and v = j/rho0
  C jbx0 = C(0), jby0 = C(0);
  if (a.ufield) {
    jbx0 = cp<C>(a.ufield)[c] * irho;
    jby0 = cp<C>(a.ufield)[p.plane + c] * irho;
  } else if (p.nrec > 0 && active && x >= p.rec_x0 && x <= p.rec_x1 && y >= p.rec_y0 &&
             y <= p.rec_y1) {
    const int tile = (y / kRecTileY) * p.rec_tiles_x + x / kRecTileX;
    for (int r = p.rec_tile_ptr[tile]; r < p.rec_tile_ptr[tile + 1]; ++r)
      if (p.rec_xy[2 * r] == x && p.rec_xy[2 * r + 1] == y) {
        jbx0 += cp<C>(a.jrec)[2 * r];
        jby0 += cp<C>(a.jrec)[2 * r + 1];
      }
    jbx0 *= irho;
    jby0 *= irho;
  }
  const C om = par<C>(p.omega, p.omega_f), kap = par<C>(p.fcoef, p.fcoef_f);
  const C A = sponge_A<C>(p, xc, yc);
  const C sig = C(1) / (C(1) + C(0.5) * A);
  C rs = C(0), jx = C(0), jy = C(0), pxx = C(0), pyy = C(0), pxy = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = cxd(i), cy = cyd(i), cc = cx * cx + cy * cy;
    const C wa = wd<C>(i) * av[i];
    rs += wa * (C(2) - C(1.5) * C(cc));
    jx += wa * C(cx);
    jy += wa * C(cy);
    pxx += wa * (C(cx * cx) - C(1.0 / 3.0));
    pyy += wa * (C(cy * cy) - C(1.0 / 3.0));
    pxy += wa * C(cx * cy);
  }
  const C rho_b = om * rs;
  const C jbx = jbx0 + om * C(3) * jx, jby = jby0 + om * C(3) * jy;
  const C sbx = kap * C(3) * jx, sby = kap * C(3) * jy;
  const C pbxx = om * C(4.5) * pxx, pbyy = om * C(4.5) * pyy, pbxy = om * C(9) * pxy;
  const C hbx = sig * sbx + C(0.5) * sig * jbx, hby = sig * sby + C(0.5) * sig * jby;
  const C mbx = sig * jbx - A * sig * sbx, mby = sig * jby - A * sig * sby;
  if (active) {
    C *gb = (C *)a.gbar;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int cx = cxd(i), cy = cyd(i);
      gb[cf + i * p.fplane] = (C(1) - om) * av[i] + rho_b + C(cx) * mbx + C(cy) * mby +
                              C(cx * cx) * pbxx + C(cy * cy) * pbyy + C(cx * cy) * pbxy;
    }
    const C lam = mat_at<C>(p.lam, p.mat_per_cell, xc, yc, p.pitch);
    if (a.lam_any) {
      C *wb = (C *)a.wbar;
      wb[c] = lam * C(1.0 / 3.0) * C(0.5) * hbx;
      wb[p.plane + c] = lam * C(1.0 / 3.0) * C(0.5) * hby;
    }
    if (a.grad) {
      // dG/dLambda = b^2 grad rho of the forward step
      const double gx = (double)cp<C>(a.grad)[c], gy = (double)cp<C>(a.grad)[p.plane + c];
      a.g_lam[c] += ((double)hbx * gx + (double)hby * gy) * (1.0 / 3.0);
    }
  }
  // amplitude gradient: dF/dA_s = dir_s g_s(x) r_s(n); warps cull sources
  // like the forward's body force (all lanes of a warp share one row)
  if (a.g_amp == nullptr || p.nsrc == 0) return;
  const int lane = threadIdx.x;
  const int xmid = blockIdx.x * 32 + 16;
  for (int s0 = 0; s0 < p.nsrc; s0 += 32) {
    bool hit = false;
    const int s = s0 + lane;
    if (s < p.nsrc) {
      const SourceDev &q = p.src[s];
      int dy = yc - q.yc, dx = xmid - q.xc;
      if (p.bc_top == BC_PERIODIC) {
        if (dy > p.ny / 2) dy -= p.ny;
        else if (dy < -(p.ny / 2)) dy += p.ny;
      }
      if (p.bc_left == BC_PERIODIC) {
        if (dx > p.nx / 2) dx -= p.nx;
        else if (dx < -(p.nx / 2)) dx += p.nx;
      }
      hit = abs(dy) <= q.rb && abs(dx) <= q.rb + 17;
    }
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const SourceDev &q = p.src[s0 + b];
      double v = 0.0;
      if (active)
        v = ((double)hbx * q.dirx + (double)hby * q.diry) *
            source_shape(q, xc, yc, p.n, p.nx, p.ny, p.bc_left == BC_PERIODIC,
                         p.bc_top == BC_PERIODIC);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0 && v != 0.0) atomicAdd(&a.g_amp[s0 + b], v);
    }
  }
}

// Adjoint of the density through the centred gradient (Eq. 10) and its wall
// ghosts.
template <class C>
__device__ __forceinline__ C div_axis(const C *w, int n, int k, int stride, bool per, int bc_lo,
                                      int bc_hi, int fs_order) {
  const bool lin_lo = bc_lo == BC_FREE && fs_order == 1;
  const bool lin_hi = bc_hi == BC_FREE && fs_order == 1;
  C r = C(0);
  if (k > 0 || per) {  // this cell is the + neighbour of k - 1
    const int km = k > 0 ? k - 1 : n - 1;
    const C v = w[(long long)(km - k) * stride];
    r += v;
    if (!per && km == 0 && lin_lo) r += v;  // its linear ghost uses this density too
  }
  if (k < n - 1 || per) {  // this cell is the - neighbour of k + 1
    const int kp = k < n - 1 ? k + 1 : 0;
    const C v = w[(long long)(kp - k) * stride];
    r -= v;
    if (!per && kp == n - 1 && lin_hi) r -= v;
  }
  if (!per) {
    const C v = w[0];
    if (k == 0) r += lin_lo ? C(-2) * v : -v;
    if (k == n - 1) r += lin_hi ? C(2) * v : v;
  }
  return r;
}

template <class C>
__global__ void __launch_bounds__(256) adj_div_kernel(const AdjParams a) {
  const StepParams &p = a.p;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = y * p.pitch + x;
  const C *wx = cp<C>(a.wbar) + c, *wy = cp<C>(a.wbar) + p.plane + c;
  ((C *)a.rbar)[c] =
      div_axis<C>(wx, p.nx, x, 1, p.bc_left == BC_PERIODIC, p.bc_left, p.bc_right, p.fs_order) +
      div_axis<C>(wy, p.ny, y, p.pitch, p.bc_top == BC_PERIODIC, p.bc_top, p.bc_bottom,
                  p.fs_order);
}

// The adjoint of pulled population i at cell (x, y): its local part plus
// the density adjoint (rho = sum of the pulled populations).
template <class C>
__device__ __forceinline__ C gtot(const AdjParams &a, int x, int y, int i) {
  const StepParams &p = a.p;
  C g = cp<C>(a.gbar)[(long long)y * p.frow + x + i * p.fplane];
  if (a.lam_any) g += cp<C>(a.rbar)[y * p.pitch + x];
  return g;
}

// Which wall, if any, supplies population i = opp(j) at (x, y): the link
// from (x + c_j, y + c_j) (the forward's rule: the y axis first, then x).
__device__ __forceinline__ bool link_wall(const StepParams &p, int x, int y, int j, int &tx,
                                          int &ty, int &bc, int &hz) {
  tx = x + cxd(j);
  ty = y + cyd(j);
  if (ty < 0 || ty >= p.ny) {
    if (p.bc_top == BC_PERIODIC) {
      ty = ty < 0 ? ty + p.ny : ty - p.ny;
    } else {
      bc = ty < 0 ? p.bc_top : p.bc_bottom;
      hz = 1;
      return true;
    }
  }
  if (tx < 0 || tx >= p.nx) {
    if (p.bc_left == BC_PERIODIC) {
      tx = tx < 0 ? tx + p.nx : tx - p.nx;
    } else {
      bc = tx < 0 ? p.bc_left : p.bc_right;
      hz = 0;
      return true;
    }
  }
  return false;
}

// Adjoint of rho_air and of the tangential stress of one anti-bounce-back
// link whose pulled-population adjoint is gb and whose outgoing population
// is k (the value is -f*_k + 2 w_k (rho_air + 4.5 h), Eqs. 37-42).
template <class C>
__device__ __forceinline__ void abb_moments(C gb, int k, int hz, C &rb, C &tb) {
  const int cx = cxd(k), cy = cyd(k), cc = cx * cx + cy * cy;
  const C w2 = C(2) * wd<C>(k);
  rb = gb * w2 * (C(2) - C(1.5) * C(cc));
  tb = gb * w2 * C(4.5) * (hz ? (C(cx * cx) - C(1.0 / 3.0)) : (C(cy * cy) - C(1.0 / 3.0)));
}

// Adds the moment adjoints (rb on rho, tb on the tangential stress P_xx for
// a horizontal wall, P_yy for a vertical one), times s, to the populations.
template <class C>
__device__ __forceinline__ void spread_moments(C *out, C rb, C tb, int hz, C s) {
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    const int cm = hz ? cxd(m) : cyd(m);
    out[m] += s * (rb + (cm != 0 ? tb : C(0)));
  }
}

// The pulled-population adjoint of the walls of boundary cell (xb, yb) whose
// inner cell is (xi, yi), summed as moment adjoints onto out (weight s): the
// anti-bounce-back links at (xb, yb) whose wall has normal (xb - xi, yb - yi).
template <class C>
__device__ __forceinline__ void inner_contrib(const AdjParams &a, int xb, int yb, int hz, C *out) {
  const StepParams &p = a.p;
  for (int j = 1; j < 9; ++j) {
    int tx, ty, bc, h;
    if (!link_wall(p, xb, yb, j, tx, ty, bc, h)) continue;
    // only the links through the wall between (xb, yb) and the inner cell
    if (bc != BC_FREE || h != hz) continue;
    C rb, tb;
    abb_moments<C>(gtot<C>(a, xb, yb, oppd(j)), j, hz, rb, tb);
    spread_moments<C>(out, rb, tb, hz, C(-0.5));
  }
}

// Transpose of the pull streaming with the wall rules.
template <class C>
__global__ void __launch_bounds__(256) adj_pull_kernel(const AdjParams a) {
  const StepParams &p = a.p;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long cf = (long long)y * p.frow + x;
  const bool lin = p.fs_order == 1;
  C out[9];
  bool wall_cell = false;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int tx, ty, bc, hz;
    if (!link_wall(p, x, y, j, tx, ty, bc, hz)) {
      out[j] = gtot<C>(a, tx, ty, j);
    } else {
      wall_cell = true;
      const C gi = gtot<C>(a, x, y, oppd(j));
      out[j] = bc == BC_RIGID ? gi : -gi;
    }
  }
  if (wall_cell) {
    // moments of this cell in its own anti-bounce-back links
    for (int j = 1; j < 9; ++j) {
      int tx, ty, bc, hz;
      if (!link_wall(p, x, y, j, tx, ty, bc, hz) || bc != BC_FREE) continue;
      C rb, tb;
      abb_moments<C>(gtot<C>(a, x, y, oppd(j)), j, hz, rb, tb);
      spread_moments<C>(out, rb, tb, hz, lin ? C(1.5) : C(1));
    }
  }
  if (lin) {
    // moments of this cell as the inner cell of a free-surface boundary cell
    if (p.bc_top == BC_FREE && y == 1) inner_contrib<C>(a, x, 0, 1, out);
    if (p.bc_bottom == BC_FREE && y == p.ny - 2) inner_contrib<C>(a, x, p.ny - 1, 1, out);
    if (p.bc_left == BC_FREE && x == 1) inner_contrib<C>(a, 0, y, 0, out);
    if (p.bc_right == BC_FREE && x == p.nx - 2) inner_contrib<C>(a, p.nx - 1, y, 0, out);
  }
  C *o = (C *)a.abar_out + cf;
#pragma unroll
  for (int j = 0; j < 9; ++j) o[j * p.fplane] = out[j];
}

// Receiver adjoints of step n (receivers in the sorted order of the
// receiver table): ubar_r += du (the adjoint of u^{n+1}, carried by every
// later u), jrec_r = ubar_r + dv (with dv the adjoint of v^n; both enter as
// j / rho0).  d: [nrec][4] of this step by original receiver index.
template <class C>
__global__ void adj_inject_kernel(C *ubar_r, C *jrec, const int *rec_id, int nrec,
                                  const double *d) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
    const double *q = d + 4 * (long long)rec_id[r];
    const C ux = ubar_r[2 * r] + C(q[0]), uy = ubar_r[2 * r + 1] + C(q[1]);
    ubar_r[2 * r] = ux;
    ubar_r[2 * r + 1] = uy;
    jrec[2 * r] = ux + C(q[2]);
    jrec[2 * r + 1] = uy + C(q[3]);
  }
}

// Launchers (one translation unit per compute type).
cudaError_t adj_step_f32(const AdjParams &a, cudaStream_t s);
cudaError_t adj_step_f64(const AdjParams &a, cudaStream_t s);
cudaError_t adj_inject_f32(void *ubar_r, void *jrec, const int *rec_id, int nrec,
                           const double *d, cudaStream_t s);
cudaError_t adj_inject_f64(void *ubar_r, void *jrec, const int *rec_id, int nrec,
                           const double *d, cudaStream_t s);

template <class C>
cudaError_t adj_step_t(const AdjParams &a, cudaStream_t s) {
  const dim3 block(32, 8), grid((a.p.nx + 31) / 32, (a.p.ny + 7) / 8);
  adj_local_kernel<C><<<grid, block, 0, s>>>(a);
  if (a.lam_any) adj_div_kernel<C><<<grid, block, 0, s>>>(a);
  adj_pull_kernel<C><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <class C>
cudaError_t adj_inject_t(void *ubar_r, void *jrec, const int *rec_id, int nrec, const double *d,
                         cudaStream_t s) {
  adj_inject_kernel<C><<<(nrec + 127) / 128, 128, 0, s>>>((C *)ubar_r, (C *)jrec, rec_id, nrec, d);
  return cudaGetLastError();
}

}  // namespace lbm
