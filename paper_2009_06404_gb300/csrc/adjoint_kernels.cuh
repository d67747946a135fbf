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
  void *g_part;        // the last steps' share of dJ/dLambda, one plane (compute type)
  int flush;           // 1: move g_part into g_lam after this step's share
  double *g_amp;       // dJ/d amplitude, per source (FP64)
  int lam_any;         // some Lambda != 0
};

template <class C>
__device__ __forceinline__ const C *cp(const void *v) { return (const C *)v; }

// dJ/dLambda += H_b . b^2 grad rho at plane index c: the product and a
// partial sum over a few steps in the compute type, moved into the FP64
// sum when a.flush is set (keeps FP64 arithmetic, slow on this GPU, off
// most steps).
template <class C>
__device__ __forceinline__ void add_lambda_grad(const AdjParams &a, int c, C hbx, C hby) {
  const C gx = cp<C>(a.grad)[c], gy = cp<C>(a.grad)[a.p.plane + c];
  C *part = (C *)a.g_part;
  const C v = part[c] + (hbx * gx + hby * gy) * C(1.0 / 3.0);
  if (a.flush) {
    a.g_lam[c] += (double)v;
    part[c] = C(0);
  } else {
    part[c] = v;
  }
}

// Adjoint of j / rho0 at cell (x, y) (in the grid): from the full u-adjoint
// planes (transpose tests) or from the receivers there.
template <class C>
__device__ __forceinline__ void jbar_at(const AdjParams &a, int x, int y, C irho, C &jx, C &jy) {
  const StepParams &p = a.p;
  jx = C(0);
  jy = C(0);
  if (a.ufield) {
    const int c = y * p.pitch + x;
    jx = cp<C>(a.ufield)[c] * irho;
    jy = cp<C>(a.ufield)[p.plane + c] * irho;
  } else if (p.nrec > 0 && x >= p.rec_x0 && x <= p.rec_x1 && y >= p.rec_y0 && y <= p.rec_y1) {
    const int tile = (y / kRecTileY) * p.rec_tiles_x + x / kRecTileX;
    for (int r = p.rec_tile_ptr[tile]; r < p.rec_tile_ptr[tile + 1]; ++r)
      if (p.rec_xy[2 * r] == x && p.rec_xy[2 * r + 1] == y) {
        jx += cp<C>(a.jrec)[2 * r];
        jy += cp<C>(a.jrec)[2 * r + 1];
      }
    jx *= irho;
    jy *= irho;
  }
}

// The local transpose at one cell: from the adjoint av of its post-collision
// populations and jb0 of j, the adjoint g of its pulled populations (without
// the density-gradient part) and hb of the force H = G + F.
template <class C>
__device__ __forceinline__ void local_transpose(const StepParams &p, const C *av, C jbx0, C jby0,
                                                C A, C *g, C &hbx, C &hby) {
  const C om = par<C>(p.omega, p.omega_f), kap = par<C>(p.fcoef, p.fcoef_f);
  const C sig = C(1) / (C(1) + C(0.5) * A);
  // weighted moments of the adjoint, sum_i w_i a_i (.), with w = 4/9, 1/9,
  // 1/36 written out (no products with zero lattice components)
  const C s13 = av[1] + av[3], s24 = av[2] + av[4];
  const C d13 = av[1] - av[3], d24 = av[2] - av[4];
  const C s58 = (av[5] + av[7]) + (av[6] + av[8]);
  const C d5768x = (av[5] - av[7]) + (av[8] - av[6]);  // sum c_x a over 5..8
  const C d5768y = (av[5] - av[7]) + (av[6] - av[8]);  // sum c_y a over 5..8
  const C d5768xy = (av[5] + av[7]) - (av[6] + av[8]); // sum c_x c_y a over 5..8
  // rho: w_i (2 - 1.5 |c_i|^2) = 8/9, 1/18, -1/36
  const C rs = C(8.0 / 9.0) * av[0] + C(1.0 / 18.0) * (s13 + s24) - C(1.0 / 36.0) * s58;
  const C jx = C(1.0 / 9.0) * d13 + C(1.0 / 36.0) * d5768x;
  const C jy = C(1.0 / 9.0) * d24 + C(1.0 / 36.0) * d5768y;
  // w_i (c_x^2 - 1/3): -4/27, 2/27 (x links), -1/27 (y links), 1/54 (diagonals)
  const C pxx = C(-4.0 / 27.0) * av[0] + C(2.0 / 27.0) * s13 - C(1.0 / 27.0) * s24 +
                C(1.0 / 54.0) * s58;
  const C pyy = C(-4.0 / 27.0) * av[0] + C(2.0 / 27.0) * s24 - C(1.0 / 27.0) * s13 +
                C(1.0 / 54.0) * s58;
  const C pxy = C(1.0 / 36.0) * d5768xy;
  const C rho_b = om * rs;
  const C jbx = jbx0 + om * C(3) * jx, jby = jby0 + om * C(3) * jy;
  const C sbx = kap * C(3) * jx, sby = kap * C(3) * jy;
  const C pbxx = om * C(4.5) * pxx, pbyy = om * C(4.5) * pyy, pbxy = om * C(9) * pxy;
  hbx = sig * sbx + C(0.5) * sig * jbx;
  hby = sig * sby + C(0.5) * sig * jby;
  const C mbx = sig * jbx - A * sig * sbx, mby = sig * jby - A * sig * sby;
  const C k1 = C(1) - om;
  const C dd = rho_b + pbxx + pbyy;  // diagonal links: rho, P_xx and P_yy
  g[0] = k1 * av[0] + rho_b;
  g[1] = k1 * av[1] + (rho_b + pbxx) + mbx;
  g[3] = k1 * av[3] + (rho_b + pbxx) - mbx;
  g[2] = k1 * av[2] + (rho_b + pbyy) + mby;
  g[4] = k1 * av[4] + (rho_b + pbyy) - mby;
  g[5] = k1 * av[5] + (dd + pbxy) + (mbx + mby);
  g[7] = k1 * av[7] + (dd + pbxy) - (mbx + mby);
  g[6] = k1 * av[6] + (dd - pbxy) + (mby - mbx);
  g[8] = k1 * av[8] + (dd - pbxy) - (mby - mbx);
}

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
  C jbx0, jby0;
  jbar_at<C>(a, xc, yc, irho, jbx0, jby0);
  if (!active) jbx0 = jby0 = C(0);
  C g[9], hbx, hby;
  local_transpose<C>(p, av, jbx0, jby0, sponge_A<C>(p, xc, yc), g, hbx, hby);
  if (active) {
    C *gb = (C *)a.gbar;
#pragma unroll
    for (int i = 0; i < 9; ++i) gb[cf + i * p.fplane] = g[i];
    const C lam = mat_at<C>(p.lam, p.mat_per_cell, xc, yc, p.pitch);
    if (a.lam_any) {
      C *wb = (C *)a.wbar;
      wb[c] = lam * C(1.0 / 3.0) * C(0.5) * hbx;
      wb[p.plane + c] = lam * C(1.0 / 3.0) * C(0.5) * hby;
    }
    // dG/dLambda = b^2 grad rho of the forward step
    if (a.grad) add_lambda_grad<C>(a, c, hbx, hby);
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
      const int4 qb = src_bound(p, s);
      int dy = yc - qb.y, dx = xmid - qb.x;
      if (p.bc_top == BC_PERIODIC) {
        if (dy > p.ny / 2) dy -= p.ny;
        else if (dy < -(p.ny / 2)) dy += p.ny;
      }
      if (p.bc_left == BC_PERIODIC) {
        if (dx > p.nx / 2) dx -= p.nx;
        else if (dx < -(p.nx / 2)) dx += p.nx;
      }
      hit = abs(dy) <= qb.z && abs(dx) <= qb.z + 17;
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

// ------------------------------------------------------------ fused form
//
// The whole adjoint step in one kernel: a block of 32 x 8 cells computes the
// local transposes of its cells and of a two-cell ring around them (36 x 12
// cells; periodic axes wrapped, cells beyond a non-periodic edge zero) into
// shared memory, then the density adjoint of the inner 34 x 10 cells, then
// the push of its own cells.  Each population adjoint is read once from
// HBM by its own block (the ring comes from L2) and written once.
#ifndef LBM_ADJ_TH
#define LBM_ADJ_TH 8
#endif
constexpr int kAdjTW = 32, kAdjTH = LBM_ADJ_TH;
constexpr int kAdjThreads = 32 * kAdjTH;
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS (2048 / (2 * kAdjThreads))
#endif
constexpr int kAdjW2 = kAdjTW + 4, kAdjH2 = kAdjTH + 4;
constexpr int kAdjW1 = kAdjTW + 2, kAdjH1 = kAdjTH + 2;

// div_axis on a shared-memory row or column: the neighbours sit at +-stride
// (the ring holds the wrapped cells of periodic axes); k is the global index.
template <class C>
__device__ __forceinline__ C div_axis_s(const C *w, int stride, int n, int k, bool per, int bc_lo,
                                        int bc_hi, int fs_order) {
  const bool lin_lo = bc_lo == BC_FREE && fs_order == 1;
  const bool lin_hi = bc_hi == BC_FREE && fs_order == 1;
  C r = C(0);
  if (k > 0 || per) {
    const C v = w[-stride];
    r += v;
    if (!per && k == 1 && lin_lo) r += v;
  }
  if (k < n - 1 || per) {
    const C v = w[stride];
    r -= v;
    if (!per && k == n - 2 && lin_hi) r -= v;
  }
  if (!per) {
    const C v = w[0];
    if (k == 0) r += lin_lo ? C(-2) * v : -v;
    if (k == n - 1) r += lin_hi ? C(2) * v : v;
  }
  return r;
}

template <class C>
struct AdjSmem {
  C g[9][kAdjH1][kAdjW1];  // local adjoint of the pulled populations
  C r[kAdjH1][kAdjW1];     // density adjoint
  C w[2][kAdjH2][kAdjW2];  // Lambda b^2 H_b / 2
};

// Total adjoint of pulled population i at tile-relative cell (hx, hy),
// -1 <= hx <= 32, -1 <= hy <= 8.
template <class C>
__device__ __forceinline__ C gtot_s(const AdjSmem<C> &S, bool lam_any, int hx, int hy, int i) {
  C g = S.g[i][hy + 1][hx + 1];
  if (lam_any) g += S.r[hy + 1][hx + 1];
  return g;
}

// Block b of a gx x gy grid of blocks, the blocks on the grid's edge first
// (their cells take the wall rules and hold the receivers: they run longer,
// and started last they would trail the launch), then the interior ones in
// row-major order.
__device__ __forceinline__ void edge_blocks_first(int b, int gx, int gy, int &bx, int &by) {
  if (gx < 3 || gy < 3) {
    bx = b % gx;
    by = b / gx;
    return;
  }
  const int side = gy - 2, per = 2 * gx + 2 * side;
  if (b < gx) {
    bx = b;
    by = 0;
  } else if (b < 2 * gx) {
    bx = b - gx;
    by = gy - 1;
  } else if (b < 2 * gx + side) {
    bx = 0;
    by = 1 + (b - 2 * gx);
  } else if (b < per) {
    bx = gx - 1;
    by = 1 + (b - 2 * gx - side);
  } else {
    const int i = b - per;
    bx = 1 + i % (gx - 2);
    by = 1 + i / (gx - 2);
  }
}

template <class C>
__global__ void __launch_bounds__(kAdjThreads, LBM_ADJ_MIN_BLOCKS) adj_fused_kernel(const AdjParams a) {
#if LBM_PDL
  // programmatic dependent launch: wait for the previous kernel (the
  // adjoint of the step after this one, or the recomputation) to complete,
  // then let the next adjoint step's blocks be scheduled as SMs free up
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  const StepParams &p = a.p;
  __shared__ AdjSmem<C> S;
  const int t = threadIdx.y * 32 + threadIdx.x;
  int bxi, byi;
  edge_blocks_first(blockIdx.x, (p.nx + kAdjTW - 1) / kAdjTW, (p.ny + kAdjTH - 1) / kAdjTH, bxi,
                    byi);
  const int x0 = bxi * kAdjTW, y0 = byi * kAdjTH;
  const bool perx = p.bc_left == BC_PERIODIC, pery = p.bc_top == BC_PERIODIC;
  const bool src_blk = a.g_amp != nullptr && p.nsrc > 0 && x0 <= p.src_x1 &&
                       x0 + kAdjTW - 1 >= p.src_x0 && y0 <= p.src_y1 &&
                       y0 + kAdjTH - 1 >= p.src_y0;
  // ---- local transposes of the block and its two-cell ring
  for (int k = t; k < kAdjW2 * kAdjH2; k += kAdjThreads) {
    const int hx = k % kAdjW2 - 2, hy = k / kAdjW2 - 2;
    int gx = x0 + hx, gy = y0 + hy;
    bool ex = true;
    if (gx < 0 || gx >= p.nx) {
      if (perx) gx = ((gx % p.nx) + p.nx) % p.nx;
      else ex = false;
    }
    if (gy < 0 || gy >= p.ny) {
      if (pery) gy = ((gy % p.ny) + p.ny) % p.ny;
      else ex = false;
    }
    C g[9], hbx = C(0), hby = C(0), lam = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = C(0);
    if (ex) {
      const long long cf = (long long)gy * p.frow + gx;
      C av[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) av[i] = cp<C>(a.abar)[cf + i * p.fplane];
      const C irho = mat_at<C>(p.irho, p.mat_per_cell, gx, gy, p.pitch);
      lam = mat_at<C>(p.lam, p.mat_per_cell, gx, gy, p.pitch);
      C jbx0, jby0;
      jbar_at<C>(a, gx, gy, irho, jbx0, jby0);
      local_transpose<C>(p, av, jbx0, jby0, sponge_A<C>(p, gx, gy), g, hbx, hby);
      // the block's own cells (unwrapped, inside the grid): gradient sums
      const bool own = hx >= 0 && hx < kAdjTW && hy >= 0 && hy < kAdjTH &&
                       x0 + hx < p.nx && y0 + hy < p.ny;
      if (own && a.grad) add_lambda_grad<C>(a, gy * p.pitch + gx, hbx, hby);
      if (own && src_blk) {
        // dF/dA_s = dir_s g_s(x) r_s(n) (integer footprint test first)
        for (int s = 0; s < p.nsrc; ++s) {
          const int4 qb = src_bound(p, s);
          int dy = gy - qb.y, dx = gx - qb.x;
          if (pery) {
            if (dy > p.ny / 2) dy -= p.ny;
            else if (dy < -(p.ny / 2)) dy += p.ny;
          }
          if (perx) {
            if (dx > p.nx / 2) dx -= p.nx;
            else if (dx < -(p.nx / 2)) dx += p.nx;
          }
          if (abs(dy) > qb.z || abs(dx) > qb.z) continue;
          const SourceDev &q = p.src[s];
          const double v = ((double)hbx * q.dirx + (double)hby * q.diry) *
                           source_shape(q, gx, gy, p.n, p.nx, p.ny, perx, pery);
          if (v != 0.0) atomicAdd(&a.g_amp[s], v);
        }
      }
    }
    S.w[0][hy + 2][hx + 2] = lam * C(1.0 / 3.0) * C(0.5) * hbx;
    S.w[1][hy + 2][hx + 2] = lam * C(1.0 / 3.0) * C(0.5) * hby;
    if (hx >= -1 && hx <= kAdjTW && hy >= -1 && hy <= kAdjTH) {
#pragma unroll
      for (int i = 0; i < 9; ++i) S.g[i][hy + 1][hx + 1] = g[i];
    }
  }
  __syncthreads();
  // ---- density adjoint of the block and its one-cell ring
  if (a.lam_any) {
    for (int k = t; k < kAdjW1 * kAdjH1; k += kAdjThreads) {
      const int hx = k % kAdjW1 - 1, hy = k / kAdjW1 - 1;
      int gx = x0 + hx, gy = y0 + hy;
      bool ex = true;
      if (gx < 0 || gx >= p.nx) {
        if (perx) gx = ((gx % p.nx) + p.nx) % p.nx;
        else ex = false;
      }
      if (gy < 0 || gy >= p.ny) {
        if (pery) gy = ((gy % p.ny) + p.ny) % p.ny;
        else ex = false;
      }
      C r = C(0);
      if (ex) {
        r = div_axis_s<C>(&S.w[0][hy + 2][hx + 2], 1, p.nx, gx, perx, p.bc_left, p.bc_right,
                          p.fs_order) +
            div_axis_s<C>(&S.w[1][hy + 2][hx + 2], kAdjW2, p.ny, gy, pery, p.bc_top,
                          p.bc_bottom, p.fs_order);
      }
      S.r[hy + 1][hx + 1] = r;
    }
  }
  __syncthreads();
  // ---- the push, gathered per own cell
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= p.nx || y >= p.ny) return;
  const bool lin = p.fs_order == 1;
  const bool la = a.lam_any != 0;
  C out[9];
  if (x0 >= 2 && x0 + kAdjTW <= p.nx - 2 && y0 >= 2 && y0 + kAdjTH <= p.ny - 2) {
    // no cell of the block is within two cells of an edge: every link is a
    // plain pull and no wall rule involves the block
#pragma unroll
    for (int j = 0; j < 9; ++j) out[j] = gtot_s<C>(S, la, tx + cxd(j), ty + cyd(j), j);
    C *o = (C *)a.abar_out + (long long)y * p.frow + x;
#pragma unroll
    for (int j = 0; j < 9; ++j) o[j * p.fplane] = out[j];
    return;
  }
  bool wall_cell = false;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int wx, wy, bc, hz;
    if (!link_wall(p, x, y, j, wx, wy, bc, hz)) {
      out[j] = gtot_s<C>(S, la, tx + cxd(j), ty + cyd(j), j);
    } else {
      wall_cell = true;
      const C gi = gtot_s<C>(S, la, tx, ty, oppd(j));
      out[j] = bc == BC_RIGID ? gi : -gi;
    }
  }
  if (wall_cell) {
    for (int j = 1; j < 9; ++j) {
      int wx, wy, bc, hz;
      if (!link_wall(p, x, y, j, wx, wy, bc, hz) || bc != BC_FREE) continue;
      C rb, tb;
      abb_moments<C>(gtot_s<C>(S, la, tx, ty, oppd(j)), j, hz, rb, tb);
      spread_moments<C>(out, rb, tb, hz, lin ? C(1.5) : C(1));
    }
  }
  if (lin) {
    // this cell as the inner cell of a free-surface boundary cell
    auto inner = [&](int xb, int yb, int rx, int ry, int hzw) {
      for (int j = 1; j < 9; ++j) {
        int wx, wy, bc, h;
        if (!link_wall(p, xb, yb, j, wx, wy, bc, h)) continue;
        if (bc != BC_FREE || h != hzw) continue;
        C rb, tb;
        abb_moments<C>(gtot_s<C>(S, la, rx, ry, oppd(j)), j, hzw, rb, tb);
        spread_moments<C>(out, rb, tb, hzw, C(-0.5));
      }
    };
    if (p.bc_top == BC_FREE && y == 1) inner(x, 0, tx, ty - 1, 1);
    if (p.bc_bottom == BC_FREE && y == p.ny - 2) inner(x, p.ny - 1, tx, ty + 1, 1);
    if (p.bc_left == BC_FREE && x == 1) inner(0, y, tx - 1, ty, 0);
    if (p.bc_right == BC_FREE && x == p.nx - 2) inner(p.nx - 1, y, tx + 1, ty, 0);
  }
  C *o = (C *)a.abar_out + (long long)y * p.frow + x;
#pragma unroll
  for (int j = 0; j < 9; ++j) o[j * p.fplane] = out[j];
}

// The receiver adjoints of every step at once, in the sorted receiver order:
// jrec[n][r] = sum_{m >= n} du[m][r] + dv[n][r], the adjoint of j / rho0 of
// step n at receiver r (u^{m+1} carries j^n for every m >= n).  d:
// [T][nrec][4] by original receiver index.  One thread per receiver.
template <class C>
__global__ void adj_jrec_kernel(const double *d, const int *rec_id, int nrec, int T, C *jrec) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrec) return;
  const long long id = rec_id[r];
  double ux = 0.0, uy = 0.0;
  for (int n = T - 1; n >= 0; --n) {
    const double *q = d + ((long long)n * nrec + id) * 4;
    ux += q[0];
    uy += q[1];
    jrec[((long long)n * nrec + r) * 2] = C(ux + q[2]);
    jrec[((long long)n * nrec + r) * 2 + 1] = C(uy + q[3]);
  }
}

// Launchers (one translation unit per compute type).
cudaError_t adj_step_f32(const AdjParams &a, bool fused, cudaStream_t s);
cudaError_t adj_step_f64(const AdjParams &a, bool fused, cudaStream_t s);
cudaError_t adj_jrec_f32(const double *d, const int *rec_id, int nrec, int T, void *jrec,
                         cudaStream_t s);
cudaError_t adj_jrec_f64(const double *d, const int *rec_id, int nrec, int T, void *jrec,
                         cudaStream_t s);

template <class C>
cudaError_t adj_step_t(const AdjParams &a, bool fused, cudaStream_t s) {
  const dim3 block(32, 8), grid((a.p.nx + 31) / 32, (a.p.ny + 7) / 8);
  if (fused) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid.x * ((a.p.ny + kAdjTH - 1) / kAdjTH));
    cfg.blockDim = dim3(32, kAdjTH);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = LBM_PDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, adj_fused_kernel<C>, a);
  } else {
    adj_local_kernel<C><<<grid, block, 0, s>>>(a);
    if (a.lam_any) adj_div_kernel<C><<<grid, block, 0, s>>>(a);
    adj_pull_kernel<C><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class C>
cudaError_t adj_jrec_t(const double *d, const int *rec_id, int nrec, int T, void *jrec,
                       cudaStream_t s) {
  adj_jrec_kernel<C><<<(nrec + 127) / 128, 128, 0, s>>>(d, rec_id, nrec, T, (C *)jrec);
  return cudaGetLastError();
}

}  // namespace lbm
