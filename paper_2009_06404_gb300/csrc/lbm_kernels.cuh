// Device code of the elastic-solid D2Q9 LBM step (arXiv 2009.06404) for
// sm_103a.  The per-cell update is, in order:
//   pull streaming with wall rules        (Eq. 18 left side; Eqs. 36-42)
//   moments rho, m, P                      (Eq. 12 applied to f)
//   centred density gradient               (Eq. 10)
//   source and physical flux               (Eqs. 9, 44, half-force shift)
//   equilibrium, BGK and forcing           (Eqs. 11, 14, 15, 18)
//   displacement u += j / rho0 and receivers.
// Lattice: c_0 = (0,0); c_1..4 = (1,0),(0,1),(-1,0),(0,-1);
// c_5..8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36; b^2 = 1/3.
// Rows are stored top (y = 0) to bottom; population plane i starts at
// i * plane elements; a row is `pitch` elements long.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

enum { BC_PERIODIC = 0, BC_FREE = 1, BC_RIGID = 2 };

// Cells per receiver tile (the receiver lookup table is per tile).
constexpr int kRecTileX = 64;
constexpr int kRecTileY = 4;

// Rows of the 32-wide blocks of the single-grid step with the
// density-gradient force (the others have 8).
#ifndef LBM_LAM_ROWS
#define LBM_LAM_ROWS 8
#endif
constexpr int kLamRows = LBM_LAM_ROWS;
static_assert(64 + 2 * kLamRows <= 32 * kLamRows, "one ring cell per thread at most");

// One body-force source, prepared on the host from an lbm_source.
struct SourceDev {
  double x, y;      // position (cells)
  double inv2s2;    // 1 / (2 sigma^2)
  double rcut2;     // r_cut^2
  double ax, ay;    // amplitude * direction
  double pif2;      // pi^2 f_peak^2
  double t0;
  int xc, yc;       // nearest cell of the position
  int rb;           // integer bound: ceil(r_cut) + 1 cells around (xc, yc)
  int pad;
  double dirx, diry;  // direction (the force per unit amplitude)
  // single-precision copies for the FP32-arithmetic kernels
  float inv2s2_f, pif2_f, ax_f, ay_f;
};

struct StepParams {
  const void *fin;   // post-collision populations of step n-1 (9 planes)
  void *fout;        // post-collision populations of step n
  void *u;           // displacement: u_x plane then u_y plane
  int plane;         // displacement / per-cell material: elements between planes
  int nx, ny, pitch; // pitch: elements between rows of those arrays
  int fplane, frow;  // populations: elements between planes i and i+1, rows y and y+1
  int finter;        // 1: rows of the nine planes interleaved (frow = 9 fplane)
  float scale_f, iscale_f;  // 16-bit storage keeps populations times scale_f (2^k)
  int bc_top, bc_bottom, bc_left, bc_right;
  int sp_top, sp_bottom, sp_left, sp_right;
  int fs_order;      // free-surface extrapolation: 1 linear, 0 constant
  double spA[4];     // A_max / L^2 per layer: top, bottom, left, right
  float spA_f[4];    // the same in FP32
  double omega;      // 1 / tau
  double fcoef;      // 1 - 1 / (2 tau)
  float omega_f, fcoef_f;
  const void *lam;   // Lambda = (mu - lambda)/(rho0 b^2), per row or per cell
  const void *irho;  // 1 / rho0, same layout
  int mat_per_cell;
  const SourceDev *src;
  int nsrc;
  // (xc, yc, rb, 0) of every source, packed: the per-block and per-cell
  // source tests read one 16-byte entry per source (one coalesced load per
  // warp) instead of three fields of each full record
  const int4 *srcb;
  long long n;       // index of this step (force time t = n)
  int trace_slot;    // >= 0: record receivers into this slot
  int trace_end;     // two-step launches: trace slots below this exist
  const int *rec_tile_ptr;  // [tiles + 1] CSR over receiver tiles
  const int *rec_xy;        // [nrec][2]  sorted by tile
  const int *rec_id;        // [nrec]     original receiver index
  int rec_tiles_x;
  int nrec;
  double *traces;           // [slots][nrec][4]
  int *err;                 // bit 0: non-finite value met
  // bounding boxes (inclusive, in cells) of every receiver and of every
  // source footprint; blocks outside them skip the per-block lookups
  int rec_x0, rec_x1, rec_y0, rec_y1;
  int src_x0, src_x1, src_y0, src_y1;
  int reverse;              // 1: blocks visit the grid in reverse order
  // when set (gradient-force path only): the centred density gradient of
  // every cell is stored here, x component then y component plane
  // ([2][ny][pitch], compute type)
  void *grad_out;
  // two-step launches: each block's tile from a list in launch order -- the
  // [first] tiles that take a slower path (near an edge or seam, a source or
  // a receiver) first, then the others in row-major order, reversed when
  // reverse is set; one list per tile geometry (without and with the
  // density-gradient force)
  const int2 *tiles2, *tiles2l;
  int tiles2_first, tiles2l_first;
  // one-step launches of the single grid: per 32 x 8 block (row-major), 0
  // when no source footprint and no receiver can reach the block, so that
  // its source and receiver lookups are skipped; null: every block looks
  const unsigned char *blk_near;
  // fields mode only
  int row0, nrows;
  double *out[8];           // ux uy vx vy rho pxx pxy pyy, [nrows][nx] each
};

// (xc, yc, rb) of source s in x, y, z.
__device__ __forceinline__ int4 src_bound(const StepParams &p, int s) { return p.srcb[s]; }

// ------------------------------------------------------------ lattice

__host__ __device__ constexpr int cxd(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cyd(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int oppd(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <class C>
__host__ __device__ constexpr C wd(int i) {
  return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// ------------------------------------------------------------ storage I/O

template <class T, class C> __device__ __forceinline__ C ld(const T *p) { return C(*p); }
template <> __device__ __forceinline__ float ld<__half, float>(const __half *p) {
  return __half2float(*p);
}
template <> __device__ __forceinline__ float ld<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
template <class T, class C> __device__ __forceinline__ void st(T *p, C v) { *p = T(v); }
template <> __device__ __forceinline__ void st<__half, float>(__half *p, float v) {
  *p = __float2half_rn(v);
}
template <> __device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) {
  *p = __float2bfloat16_rn(v);
}

// Population loads and stores.  16-bit storage keeps f * 2^k; the step works
// on those scaled values throughout (the step is linear and 2^k is exact, so
// every rounding is the unscaled one times 2^k): only the body force enters
// times 2^k, and 1/rho0 (for u += j / rho0) and the fields read out carry
// 2^-k (see force_scale, irho_at).
//
// Global loads of populations and displacements go to L2 directly (ld.cg):
// within a step no cell's value is loaded twice by one block, and a kernel
// that advances several steps with blocks waiting on one another (the
// persistent batched kernel) must not read a stale line from the SM's L1.
template <class T, class C> __device__ __forceinline__ C ldg(const T *p) { return C(__ldcg(p)); }
template <> __device__ __forceinline__ float ldg<__half, float>(const __half *p) {
  return __half2float(__ldcg(p));
}
template <> __device__ __forceinline__ float ldg<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldcg(p));
}
template <class T, class C>
__device__ __forceinline__ C ldp(const T *ptr, const StepParams &) {
  return ldg<T, C>(ptr);
}
template <class T, class C>
__device__ __forceinline__ void stp(T *ptr, C v, const StepParams &) {
  st<T, C>(ptr, v);
}

// 2^k for 16-bit storage (the body force in the populations' units), else 1.
template <class T, class C>
__device__ __forceinline__ C force_scale(const StepParams &p) {
  return sizeof(T) == 2 ? C(p.scale_f) : C(1);
}
// 2^-k for 16-bit storage (back to physical units), else 1.
template <class T, class C>
__device__ __forceinline__ C unit_scale(const StepParams &p) {
  return sizeof(T) == 2 ? C(p.iscale_f) : C(1);
}

// Product rounded on its own (never fused with a following addition), and a
// fused multiply-add, so that every path of the step rounds these
// expressions the same way whatever the compiler would contract.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------------ wall rules

// Where the wall rules read post-collision populations: a whole grid in
// global memory (periodic axes wrapped), or a window of cells around a block
// held in shared memory, which stores the periodic images of cells beyond a
// seam at their unwrapped coordinates (no wrap).
template <class T>
struct GridPops {
  const T *f;
  int fplane, frow;
  static constexpr bool kWrap = true;
  template <class C>
  __device__ __forceinline__ C load(int i, int x, int y) const {
    return ldg<T, C>(f + (i * fplane + (y * frow + x)));
  }
};

// Moments rho and the diagonal stress components of the post-collision
// populations at one in-domain cell (the collision conserves rho and P, so
// these equal the moments at time t of Eqs. 39-42).
// rho and the diagonal stress components of nine populations (the sums in
// one fixed order on every path).
template <class C>
__device__ __forceinline__ void rho_pdiag(const C *v, C &rho, C &pxx, C &pyy) {
  rho = v[0] + v[1] + v[2] + v[3] + v[4] + v[5] + v[6] + v[7] + v[8];
  pxx = v[1] + v[3] + v[5] + v[6] + v[7] + v[8];
  pyy = v[2] + v[4] + v[5] + v[6] + v[7] + v[8];
}

template <class T, class C, class A>
__device__ void cell_rho_pdiag(const StepParams &p, const A &a, int x, int y, C &rho, C &pxx,
                               C &pyy) {
  C v[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = a.template load<C>(i, x, y);
  rho_pdiag<C>(v, rho, pxx, pyy);
}

// The air state of a free-surface wall with outward normal (nxo, nyo)
// (Eqs. 37-42): rho_air and P^n_air = P_air - rho_air b^2 I, P_air keeping
// only the tangential stress (P_xx on a horizontal wall, P_yy on a vertical
// one), from the moments of the boundary cell (b) and, for the linear
// extrapolation half a cell out (Eq. 39), of the cell inside it (i).
template <class C>
struct AirState {
  C rho_air, pnxx, pnyy;
};
template <class C>
__device__ __forceinline__ AirState<C> air_state(const StepParams &p, int nyo, C rb, C pxxb,
                                                 C pyyb, C ri, C pxxi, C pyyi) {
  // The products and sums are rounded in a fixed order (explicit fused
  // multiply-adds), so the value does not depend on how the compiler
  // contracts the expression where the link is a constant (an unrolled
  // caller) or a run-time value.
  AirState<C> s;
  C ptan;  // tangential stress: P_xx on a horizontal wall, P_yy on a vertical one
  if (p.fs_order == 1) {
    // 0.5 x is exact
    s.rho_air = fma_rn(C(1.5), rb, C(-0.5) * ri);
    ptan = nyo != 0 ? fma_rn(C(1.5), pxxb, C(-0.5) * pxxi) : fma_rn(C(1.5), pyyb, C(-0.5) * pyyi);
  } else {
    // constant extrapolation: the boundary cell's own values
    s.rho_air = rb;
    ptan = nyo != 0 ? pxxb : pyyb;
  }
  const C third = C(1.0 / 3.0);
  s.pnxx = fma_rn(-s.rho_air, third, nyo != 0 ? ptan : C(0));
  s.pnyy = fma_rn(-s.rho_air, third, nyo != 0 ? C(0) : ptan);
  return s;
}

// Anti-bounce-back value of the population entering opposite to k, whose
// outgoing post-collision population is fk: -f*_k + 2 w_k (rho_air +
// P^n_air : H_k / (2 b^4)) (Eq. 38).
template <class C>
__device__ __forceinline__ C abb_value(const AirState<C> &s, int k, C fk) {
  const C third = C(1.0 / 3.0);
  const int cx = cxd(k), cy = cyd(k);
  const C h = fma_rn(C(cx * cx) - third, s.pnxx, mul_rn(C(cy * cy) - third, s.pnyy));
  return fma_rn(C(2) * wd<C>(k), fma_rn(C(4.5), h, s.rho_air), -fk);
}

// Population i entering boundary cell (x, y) through a wall of kind bc with
// outward normal (nxo, nyo).  Rigid: half-way bounce-back (Eq. 36).  Free
// surface: anti-bounce-back with rho_air and the tangential stress
// extrapolated from x_b and x_in = x_b - n; P_air has no other component
// (Eqs. 37-42).
template <class T, class C, class A>
__device__ C wall_value(const StepParams &p, const A &a, int bc, int nxo, int nyo, int i, int x,
                        int y) {
  const int k = oppd(i);
  const C fk = a.template load<C>(k, x, y);
  if (bc == BC_RIGID) return fk;
  C rb, pxxb, pyyb, ri = C(0), pxxi = C(0), pyyi = C(0);
  cell_rho_pdiag<T, C>(p, a, x, y, rb, pxxb, pyyb);
  if (p.fs_order == 1) cell_rho_pdiag<T, C>(p, a, x - nxo, y - nyo, ri, pxxi, pyyi);
  return abb_value<C>(air_state<C>(p, nyo, rb, pxxb, pyyb, ri, pxxi, pyyi), k, fk);
}

// Pull of population i into (x, y) on a boundary cell (general path): the
// upstream cell, or the wall rule where the link crosses a non-periodic
// edge (top and bottom first: a corner link crosses two edges).
template <class T, class C, class A>
__device__ __forceinline__ C pull_general_a(const StepParams &p, const A &a, int i, int x, int y) {
  int sx = x - cxd(i), sy = y - cyd(i);
  if (sy < 0 || sy >= p.ny) {
    if (p.bc_top == BC_PERIODIC) {
      if (A::kWrap) sy = sy < 0 ? sy + p.ny : sy - p.ny;
    } else if (sy < 0) {
      return wall_value<T, C>(p, a, p.bc_top, 0, -1, i, x, y);
    } else {
      return wall_value<T, C>(p, a, p.bc_bottom, 0, 1, i, x, y);
    }
  }
  if (sx < 0 || sx >= p.nx) {
    if (p.bc_left == BC_PERIODIC) {
      if (A::kWrap) sx = sx < 0 ? sx + p.nx : sx - p.nx;
    } else if (sx < 0) {
      return wall_value<T, C>(p, a, p.bc_left, -1, 0, i, x, y);
    } else {
      return wall_value<T, C>(p, a, p.bc_right, 1, 0, i, x, y);
    }
  }
  return a.template load<C>(i, sx, sy);
}

template <class T, class C>
__device__ __noinline__ C pull_general(const StepParams &p, const T *f, int i, int x, int y) {
  return pull_general_a<T, C>(p, GridPops<T>{f, p.fplane, p.frow}, i, x, y);
}

// pull_general_a out of line, for any population source.
template <class T, class C, class A>
__device__ __noinline__ C pull_link(const StepParams &p, const A a, int i, int x, int y) {
  return pull_general_a<T, C>(p, a, i, x, y);
}

// All nine streamed populations of the in-grid cell (x, y) by the rules of
// pull_general_a (wrapped pulls across periodic seams, the wall rule for
// links that cross a non-periodic edge), with every load issued before any
// wall value is formed: a cell on one wall loads its own nine post-collision
// populations (and, for the linear free-surface rule, those of the cell
// inside it) once and forms the air state once for its three wall links.
// The values are those of pull_general_a, bit for bit.  A cell on two walls
// (a corner) takes the per-link rule.  Out of line: the register budget of
// the step kernels' bulk paths stays the budget of this function too.
template <class T, class C, class A>
__device__ __noinline__ void pull_cell(const StepParams &p, const A a, int x, int y, C *f) {
  const bool wt = y == 0 && p.bc_top != BC_PERIODIC;
  const bool wb = y == p.ny - 1 && p.bc_bottom != BC_PERIODIC;
  const bool wl = x == 0 && p.bc_left != BC_PERIODIC;
  const bool wr = x == p.nx - 1 && p.bc_right != BC_PERIODIC;
  const int nw = (int)wt + (int)wb + (int)wl + (int)wr;
  if (nw > 1) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = pull_link<T, C, A>(p, a, i, x, y);
    return;
  }
  // pulls that cross no wall (wrapped across periodic seams)
  const int nxo = wl ? -1 : (wr ? 1 : 0), nyo = wt ? -1 : (wb ? 1 : 0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (cxd(i) * nxo + cyd(i) * nyo < 0) continue;  // crosses the wall
    int sx = x - cxd(i), sy = y - cyd(i);
    if (A::kWrap) {
      sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
      sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
    }
    f[i] = a.template load<C>(i, sx, sy);
  }
  if (nw == 0) return;
  // the three links through the wall
  const int bc = wt ? p.bc_top : (wb ? p.bc_bottom : (wl ? p.bc_left : p.bc_right));
  C own[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) own[k] = a.template load<C>(k, x, y);
  if (bc == BC_RIGID) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (cxd(i) * nxo + cyd(i) * nyo < 0) f[i] = own[oppd(i)];
    return;
  }
  C rb, pxxb, pyyb, ri = C(0), pxxi = C(0), pyyi = C(0);
  if (p.fs_order == 1) {
    C inn[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) inn[k] = a.template load<C>(k, x - nxo, y - nyo);
    rho_pdiag<C>(inn, ri, pxxi, pyyi);
  }
  rho_pdiag<C>(own, rb, pxxb, pyyb);
  const AirState<C> air = air_state<C>(p, nyo, rb, pxxb, pyyb, ri, pxxi, pyyi);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (cxd(i) * nxo + cyd(i) * nyo < 0) f[i] = abb_value<C>(air, oppd(i), own[oppd(i)]);
}

// Whether no pull of the in-grid cell (x, y) crosses a non-periodic edge
// (its nine pulls are plain loads, wrapped across periodic seams).
__device__ __forceinline__ bool off_walls(const StepParams &p, int x, int y) {
  return (p.bc_left == BC_PERIODIC || (x > 0 && x < p.nx - 1)) &&
         (p.bc_top == BC_PERIODIC || (y > 0 && y < p.ny - 1));
}

// All nine streamed populations of the in-grid cell (x, y).
template <class T, class C>
__device__ __forceinline__ void gather(const StepParams &p, const T *f, int x, int y, C *fo) {
  if (x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1) {
    const T *b = f + (y * p.frow + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) fo[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  } else if (off_walls(p, x, y)) {
    // a cell on a periodic seam: the pulls wrapped, inline
    const int xs[3] = {x > 0 ? x - 1 : p.nx - 1, x, x < p.nx - 1 ? x + 1 : 0};
    const int ys[3] = {y > 0 ? y - 1 : p.ny - 1, y, y < p.ny - 1 ? y + 1 : 0};
#pragma unroll
    for (int i = 0; i < 9; ++i)
      fo[i] = ldp<T, C>(f + (i * p.fplane + (ys[1 - cyd(i)] * p.frow + xs[1 - cxd(i)])), p);
  } else {
    pull_cell<T, C>(p, GridPops<T>{f, p.fplane, p.frow}, x, y, fo);
  }
}

template <class T, class C>
__device__ __forceinline__ C rho_at(const StepParams &p, const T *f, int x, int y) {
  C v[9];
  gather<T, C>(p, f, x, y, v);
  return v[0] + v[1] + v[2] + v[3] + v[4] + v[5] + v[6] + v[7] + v[8];
}

// v wrapped into [0, n) (one period either way by an add, further by a
// remainder).
__device__ __forceinline__ int wrap_any(int v, int n) {
  if (v >= -n && v < 2 * n) return v < 0 ? v + n : (v >= n ? v - n : v);
  return ((v % n) + n) % n;
}

// Streamed density at grid coordinate (x, y) with periodic axes wrapped;
// zero beyond a non-periodic edge (the wall rules below replace it there).
// Inline, so the loads of a caller's own pulls and these are in flight
// together.
template <class T, class C>
__device__ __forceinline__ C rho_wrapped(const StepParams &p, const T *f, int x, int y) {
  if (x < 0 || x >= p.nx) {
    if (p.bc_left != BC_PERIODIC) return C(0);
    x = wrap_any(x, p.nx);
  }
  if (y < 0 || y >= p.ny) {
    if (p.bc_top != BC_PERIODIC) return C(0);
    y = wrap_any(y, p.ny);
  }
  return rho_at<T, C>(p, f, x, y);
}

// The input populations around a general tile or block, staged in shared memory by
// one pass of copies so that the general rules (wrapped pulls, wall rules,
// ring densities) read them from there instead of making a round trip to
// memory per branch.  Layout [SH][9][SW], the global row-interleaved order:
// element (0, 0) of plane i is grid cell (ox, oy); cells beyond a periodic
// seam hold the image's populations at their unwrapped coordinates, cells
// beyond a non-periodic edge are not copied (the wall rules never read
// them).
template <class T, int SW, int SH>
struct StagePops {
  const T *f;
  int ox, oy;
  static constexpr bool kWrap = false;
  __device__ __forceinline__ const T *at(int i, int x, int y) const {
    return f + (((y - oy) * 9 + i) * SW + (x - ox));
  }
  template <class C>
  __device__ __forceinline__ C load(int i, int x, int y) const {
    return ld<T, C>(at(i, x, y));
  }
};

// 16-byte chunks of the staged rows: elements per chunk, the columns a
// region of width w with margin m needs (its origin rounded down to a
// chunk), rounded up to whole chunks.
template <class T>
constexpr int stage_chunk() { return 16 / (int)sizeof(T); }
template <class T>
constexpr int stage_width(int w, int m) {
  return (w + 2 * m + stage_chunk<T>() - 1 + stage_chunk<T>() - 1) / stage_chunk<T>() *
         stage_chunk<T>();
}
// The origin column of a staged region: x0 - m rounded down to a chunk
// (floor for negative values too).
template <class T>
__device__ __forceinline__ int stage_origin(int x0, int m) {
  constexpr int E = stage_chunk<T>();
  const int v = x0 - m;
  return v >= 0 ? v / E * E : -((-v + E - 1) / E * E);
}

// Stages SH grid rows from oy (each with its nine planes) of SW columns from
// ox (a multiple of the chunk) of fin into st (16-byte aligned), by every
// thread of an NT-thread block: whole chunks inside the grid by 16-byte
// asynchronous copies to shared memory through L2 (cp.async.cg, no
// registers held), chunks across an edge element by element (wrapped on a
// periodic axis, skipped beyond a non-periodic one).  The caller waits with
// stage_wait() and a block barrier.  With a layout other than the row
// interleaved one, every chunk goes element by element.
template <class T, int SW, int SH, int NT>
__device__ __forceinline__ void stage_rows(const StepParams &p, const T *fin, int ox, int oy,
                                           T *st) {
  constexpr int E = stage_chunk<T>(), NC = SW / E, N = SH * 9 * NC;
  static_assert(SW % E == 0, "whole chunks per staged row");
  const bool inter = p.frow == 9 * p.fplane;
  for (int q = threadIdx.y * 32 + threadIdx.x; q < N; q += NT) {
    const int R = q / NC, c = q - R * NC;
    const int r = R / 9, i = R - 9 * r;
    int gy = oy + r;
    if (gy < 0 || gy >= p.ny) {
      if (p.bc_top != BC_PERIODIC) continue;
      gy = wrap_any(gy, p.ny);
    }
    const int gx = ox + c * E;
    T *dst = st + (R * SW + c * E);
    const T *src = fin + ((long long)gy * p.frow + (long long)i * p.fplane);
    // a chunk wholly beyond a periodic seam is copied from its image (whole
    // and aligned when nx is a multiple of the chunk)
    int wx = gx;
    if ((wx < 0 || wx >= p.nx) && p.bc_left == BC_PERIODIC) wx = wrap_any(wx, p.nx);
    if (inter && wx >= 0 && wx + E <= p.nx && wx % E == 0) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + wx)
                   : "memory");
    } else {
      // across an edge or seam: element by element, every load issued
      // before the first shared store
      T v[E];
      unsigned okm = 0u;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        int x = gx + e;
        if (x < 0 || x >= p.nx) {
          if (p.bc_left != BC_PERIODIC) continue;
          x = wrap_any(x, p.nx);
        }
        v[e] = __ldcg(src + x);
        okm |= 1u << e;
      }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (okm & (1u << e)) dst[e] = v[e];
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// All nine streamed populations of the in-grid cell (x, y) (unwrapped on
// periodic axes) from a staged region: plain pulls off the walls, the wall
// rules otherwise (the values of gather, bit for bit).
template <class T, class C, class A>
__device__ __forceinline__ void pull_staged(const StepParams &p, const A &a, int x, int y,
                                            C *f) {
  if (off_walls(p, x, y)) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = a.template load<C>(i, x - cxd(i), y - cyd(i));
  } else {
    pull_cell<T, C>(p, a, x, y, f);
  }
}

// Whether the general tiles of storage type T stage their inputs (the
// staged region of 8-byte populations would pass the 48 KB of static shared
// memory; FP64 keeps per-cell global pulls).
template <class T>
constexpr bool stages() { return sizeof(T) <= 4; }

// Ghost densities of the centred gradient (Eq. 10) on a non-periodic edge of
// one axis: free surface 2 rho_b - rho_in (linear extrapolation) or rho_b
// (constant), rigid wall rho_b.  lo / hi: the cell is the first / last of
// the axis; rm, rp: the neighbours' densities (zero beyond the edge).
__device__ __forceinline__ bool edge_linear(const StepParams &p, int bc) {
  return bc == BC_FREE && p.fs_order == 1;
}
template <class C>
__device__ __forceinline__ void wall_ghosts(const StepParams &p, bool lo, bool hi, int bc_lo,
                                            int bc_hi, C rho, C &rm, C &rp) {
  if (bc_lo == BC_PERIODIC) return;
  if (lo) rm = edge_linear(p, bc_lo) ? C(2) * rho - rp : rho;
  if (hi) rp = edge_linear(p, bc_hi) ? C(2) * rho - rm : rho;
}

// Centred density gradient (Eq. 10) of one cell from its neighbours'
// streamed densities, with the wall ghosts on non-periodic edges.
template <class T, class C>
__device__ void grad_rho(const StepParams &p, const T *f, int x, int y, C rho, C &gx, C &gy) {
  C rxm = rho_wrapped<T, C>(p, f, x - 1, y), rxp = rho_wrapped<T, C>(p, f, x + 1, y);
  C rym = rho_wrapped<T, C>(p, f, x, y - 1), ryp = rho_wrapped<T, C>(p, f, x, y + 1);
  wall_ghosts<C>(p, x == 0, x == p.nx - 1, p.bc_left, p.bc_right, rho, rxm, rxp);
  wall_ghosts<C>(p, y == 0, y == p.ny - 1, p.bc_top, p.bc_bottom, rho, rym, ryp);
  gx = C(0.5) * (rxp - rxm);
  gy = C(0.5) * (ryp - rym);
}


// Scalar parameter in the compute type (FP32 kernels read the FP32 copy, so
// no FP64 conversion runs per cell).
template <class C> __device__ __forceinline__ C par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

// Absorbing-layer coefficient A(x) = A_max (d/L)^2, d = depth into the layer
// (0 on the first interior cell); the largest value where layers overlap.
template <class C>
__device__ __forceinline__ C sponge_A(const StepParams &p, int x, int y) {
  C a = C(0);
  int d;
  d = p.sp_top - y;
  if (d > 0) a = max(a, par<C>(p.spA[0], p.spA_f[0]) * C(d * d));
  d = y - (p.ny - 1 - p.sp_bottom);
  if (d > 0) a = max(a, par<C>(p.spA[1], p.spA_f[1]) * C(d * d));
  d = p.sp_left - x;
  if (d > 0) a = max(a, par<C>(p.spA[2], p.spA_f[2]) * C(d * d));
  d = x - (p.nx - 1 - p.sp_right);
  if (d > 0) a = max(a, par<C>(p.spA[3], p.spA_f[3]) * C(d * d));
  return a;
}

// Body force of step n at (x, y) (Sec. 5): sum over sources of
// amplitude * dir * exp(-r^2/(2 sigma^2)) * ricker(n), r <= r_cut, with
// minimum-image distances on periodic axes.  Sources are culled per warp
// (one lane per source tests the warp's row segment), and only the few
// cells near a source evaluate it.

// Squared minimum-image distance from (x, y) to the source position, in
// FP64 (the r <= r_cut test is exact, as in the definition).  The periodic
// image shift floor(d / n + 0.5) is zero whenever |d| < 0.49 n, so the
// division is only carried out near half a period.
__device__ __forceinline__ double source_r2(const SourceDev &q, int x, int y, int nx, int ny,
                                            int wrap_x, int wrap_y) {
  double dx = (double)x - q.x, dy = (double)y - q.y;
  if (wrap_x && !(fabs(dx) < 0.49 * nx)) dx -= nx * floor(dx / nx + 0.5);
  if (wrap_y && !(fabs(dy) < 0.49 * ny)) dy -= ny * floor(dy / ny + 0.5);
  return dx * dx + dy * dy;
}

// Gaussian x Ricker factor of one source at (x, y) for step n, in FP64
// (zero beyond r_cut).
__device__ __forceinline__ double source_shape(const SourceDev &q, int x, int y, long long n,
                                               int nx, int ny, int wrap_x, int wrap_y) {
  const double r2 = source_r2(q, x, y, nx, ny, wrap_x, wrap_y);
  if (!(r2 <= q.rcut2)) return 0.0;
  const double tt = (double)n - q.t0;
  const double a = q.pif2 * tt * tt;
  return exp(-r2 * q.inv2s2) * (1.0 - 2.0 * a) * exp(-a);
}

// Force of one source at (x, y) for step n in the kernel's arithmetic: FP64
// for the FP64 kernel; for the FP32-arithmetic kernels the distance test in
// FP64 and the two exponentials in FP32 (the FP64 pipe of this GPU is a
// small fraction of the FP32 one, and a warp near a source would otherwise
// spend most of the step there).  Out of line, so the path every cell takes
// carries none of it.
static __device__ __noinline__ double2 source_term(const SourceDev &q, int x, int y, long long n,
                                                   int nx, int ny, int wrap_x, int wrap_y,
                                                   double) {
  const double g = source_shape(q, x, y, n, nx, ny, wrap_x, wrap_y);
  return make_double2(q.ax * g, q.ay * g);
}
static __device__ __noinline__ float2 source_term(const SourceDev &q, int x, int y, long long n,
                                                  int nx, int ny, int wrap_x, int wrap_y, float) {
  const double r2 = source_r2(q, x, y, nx, ny, wrap_x, wrap_y);
  if (!(r2 <= q.rcut2)) return make_float2(0.0f, 0.0f);
  const float tt = (float)((double)n - q.t0);
  const float a = q.pif2_f * tt * tt;
  const float g = expf(-(float)r2 * q.inv2s2_f) * (1.0f - 2.0f * a) * expf(-a);
  return make_float2(q.ax_f * g, q.ay_f * g);
}

template <class C>
__device__ void body_force(const StepParams &p, int x, int y, C &Fx, C &Fy) {
  Fx = C(0);
  Fy = C(0);
  if (p.nsrc == 0) return;
  const int lane = threadIdx.x & 31;
  // the row segment this warp covers (all lanes share y when blockDim.x % 32 == 0);
  // the cull test uses integers only
  const int xmid = x - lane + 16;
  for (int s0 = 0; s0 < p.nsrc; s0 += 32) {
    bool hit = false;
    const int s = s0 + lane;
    if (s < p.nsrc) {
      const int4 qb = src_bound(p, s);
      int dy = y - qb.y, dx = xmid - qb.x;
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
      const auto F = source_term(p.src[s0 + b], x, y, p.n, p.nx, p.ny,
                                 p.bc_left == BC_PERIODIC, p.bc_top == BC_PERIODIC, C(0));
      Fx += C(F.x);
      Fy += C(F.y);
    }
  }
}

// Sources that may reach the cells within hx columns and hy rows of
// (cx, cy): bit s is set when source s's integer bound (|dx|, |dy| <= rb,
// minimum image on periodic axes) can contain such a cell; every bit when
// there are more than 32 sources.  Warp-wide: every lane of the warp calls
// it, and blocks are 32 threads wide (threadIdx.x is the lane).
__device__ __forceinline__ unsigned source_mask(const StepParams &p, int cx, int cy, int hx,
                                                int hy) {
  if (p.nsrc > 32) return 0xffffffffu;
  bool hit = false;
  if ((int)threadIdx.x < p.nsrc) {
    const int4 qb = src_bound(p, threadIdx.x);
    int dx = cx - qb.x, dy = cy - qb.y;
    if (p.bc_left == BC_PERIODIC) {
      if (dx > p.nx / 2) dx -= p.nx;
      else if (dx < -(p.nx / 2)) dx += p.nx;
    }
    if (p.bc_top == BC_PERIODIC) {
      if (dy > p.ny / 2) dy -= p.ny;
      else if (dy < -(p.ny / 2)) dy += p.ny;
    }
    hit = abs(dx) <= qb.z + hx && abs(dy) <= qb.z + hy;
  }
  return __ballot_sync(0xffffffffu, hit);
}

// Source s's share of the body force at (x, y), step n, if its integer
// bound contains the cell.
template <class C>
__device__ __forceinline__ void add_source(const StepParams &p, int s, int x, int y, long long n,
                                           C &Fx, C &Fy) {
  const int4 qb = src_bound(p, s);
  int dy = y - qb.y, dx = x - qb.x;
  if (p.bc_top == BC_PERIODIC) {
    if (dy > p.ny / 2) dy -= p.ny;
    else if (dy < -(p.ny / 2)) dy += p.ny;
  }
  if (p.bc_left == BC_PERIODIC) {
    if (dx > p.nx / 2) dx -= p.nx;
    else if (dx < -(p.nx / 2)) dx += p.nx;
  }
  if (abs(dy) <= qb.z && abs(dx) <= qb.z) {
    const auto F = source_term(p.src[s], x, y, n, p.nx, p.ny, p.bc_left == BC_PERIODIC,
                               p.bc_top == BC_PERIODIC, C(0));
    Fx += C(F.x);
    Fy += C(F.y);
  }
}

// The body force of step n at (x, y) computed by one thread alone (no warp
// cooperation): the sources whose integer bound contains the cell, in
// ascending order, among those of `mask` (a superset of them, e.g. from
// source_mask).  Every source that body_force adds and this one skips
// contributes an exact zero, so the two agree bit for bit.  The sum is out
// of line (its registers stay out of the general paths' budget) and only
// called inside the bounding box of the footprints.
template <class C>
struct ForcePair {
  C x, y;
};
template <class C>
__device__ __noinline__ ForcePair<C> body_force_sum(const StepParams &p, int x, int y,
                                                    long long n, unsigned mask) {
  C Fx = C(0), Fy = C(0);
  if (p.nsrc > 32) {
    for (int s = 0; s < p.nsrc; ++s) add_source<C>(p, s, x, y, n, Fx, Fy);
  } else {
    for (unsigned m = mask; m != 0u; m &= m - 1u) add_source<C>(p, __ffs(m) - 1, x, y, n, Fx, Fy);
  }
  return ForcePair<C>{Fx, Fy};
}

template <class C>
__device__ __forceinline__ void body_force_cell(const StepParams &p, int x, int y, long long n,
                                                C &Fx, C &Fy, unsigned mask = 0xffffffffu) {
  Fx = C(0);
  Fy = C(0);
  // outside the bounding box of every footprint no source contributes
  if (mask == 0u || x < p.src_x0 || x > p.src_x1 || y < p.src_y0 || y > p.src_y1) return;
  const ForcePair<C> F = body_force_sum<C>(p, x, y, n, mask);
  Fx = F.x;
  Fy = F.y;
}

template <class C>
__device__ __forceinline__ C mat_at(const void *tab, int per_cell, int x, int y, int pitch) {
  const C *t = (const C *)tab;
  return per_cell ? t[y * pitch + x] : t[y];
}

// 1/rho0 at (x, y) times the populations' unit scale (u and v come out in
// physical units from j in the populations' units).
template <class T, class C>
__device__ __forceinline__ C irho_at(const StepParams &p, int x, int y) {
  return mat_at<C>(p.irho, p.mat_per_cell, x, y, p.pitch) * unit_scale<T, C>(p);
}

// ------------------------------------------------------------ the step

// Density of the streamed populations at an interior cell whose nine
// upstream cells all lie inside the grid (direct loads only).
template <class T, class C>
__device__ __forceinline__ C rho_direct(const StepParams &p, const T *f, int x, int y) {
  const T *b = f + (y * p.frow + x);
  C r = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) r += ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  return r;
}

// Raw moments of the streamed populations, summed pairwise over opposite
// links: rho, m, P (Eq. 12 applied to f) and the three higher moments
// Q_xxy = sum f c_x^2 c_y, Q_xyy = sum f c_x c_y^2, R = sum f c_x^2 c_y^2.
template <class C>
struct Moments {
  C rho, mx, my, pxx, pxy, pyy, qxxy, qxyy, r;
};

template <class C>
__device__ __forceinline__ Moments<C> cell_moments(const C *f) {
  const C s13 = f[1] + f[3], d13 = f[1] - f[3];
  const C s24 = f[2] + f[4], d24 = f[2] - f[4];
  const C s57 = f[5] + f[7], d57 = f[5] - f[7];
  const C s68 = f[6] + f[8], d68 = f[6] - f[8];
  Moments<C> M;
  M.r = s57 + s68;
  M.pxy = s57 - s68;
  M.qxxy = d57 + d68;
  M.qxyy = d57 - d68;
  M.pxx = s13 + M.r;
  M.pyy = s24 + M.r;
  M.rho = (f[0] + s13) + (s24 + M.r);
  M.mx = d13 + M.qxyy;
  M.my = d24 + M.qxxy;
  return M;
}

// Physical flux with the half-force shift and the source; the absorbing term
// -A j is taken implicitly (Eq. 44 treated as a forcing, Eqs. 9, 12, 22).
template <class C>
__device__ __forceinline__ void flux_and_source(C mx, C my, C Gx, C Gy, C Fx, C Fy, C A, C &jx,
                                                C &jy, C &Sx, C &Sy) {
  const C inv = C(1) / (C(1) + C(0.5) * A);
  jx = (mx + C(0.5) * (Gx + Fx)) * inv;
  jy = (my + C(0.5) * (Gy + Fy)) * inv;
  Sx = Gx + Fx - A * jx;
  Sy = Gy + Fy - A * jy;
}

// BGK collision with forcing (Eqs. 11, 14, 15, 18), carried out on the raw
// moments.  The map f -> (rho, m, P, Q_xxy, Q_xyy, R) is one to one on D2Q9,
// so f* = f - w (f - f^eq) + (1 - 1/(2 tau)) S_i is equivalent to:
//   rho* = rho, P* = P                    (conserved: Eqs. 12, 22)
//   m*   = m + S                          (Guo forcing with j = m + S/2)
//   Q*_xxy = (1 - w) Q_xxy + b^2 (w j_y + (1 - 1/(2 tau)) S_y)
//   Q*_xyy = (1 - w) Q_xyy + b^2 (w j_x + (1 - 1/(2 tau)) S_x)
//   R*   = (1 - w) R + w (b^2 (P_xx + P_yy) - b^4 rho)
// using the moments of f^eq (Q^eq_xxy = b^2 j_y, R^eq = b^2 tr P - b^4 rho) and
// of S_i (sum S_i c_x^2 c_y = b^2 S_y).  The populations follow from the
// inverse map, whose coefficients (1/2, 1/4) are exact in binary, so the
// conserved moments pass through unchanged apart from the final rounding.
template <class C>
__device__ __forceinline__ void collide_cell(const Moments<C> &M, C jx, C jy, C Sx, C Sy, C om,
                                             C fc, C *fs) {
  // (explicit fused multiply-adds: a sum of two products can be contracted
  // either way, and the compiler's choice may depend on the caller)
  const C k1 = C(1) - om, b2 = C(1.0 / 3.0);
  const C mxs = M.mx + Sx, mys = M.my + Sy;
  const C qxxy = fma_rn(k1, M.qxxy, b2 * fma_rn(om, jy, fc * Sy));
  const C qxyy = fma_rn(k1, M.qxyy, b2 * fma_rn(om, jx, fc * Sx));
  const C r = fma_rn(k1, M.r, om * fma_rn(b2, M.pxx + M.pyy, C(-1.0 / 9.0) * M.rho));
  const C rp = r + M.pxy, rm = r - M.pxy, qp = qxxy + qxyy, qm = qxxy - qxyy;
  fs[5] = C(0.25) * (rp + qp);   // ( 1,  1)
  fs[7] = C(0.25) * (rp - qp);   // (-1, -1)
  fs[6] = C(0.25) * (rm + qm);   // (-1,  1)
  fs[8] = C(0.25) * (rm - qm);   // ( 1, -1)
  const C ax = M.pxx - r, ay = M.pyy - r, bx = mxs - qxyy, by = mys - qxxy;
  fs[1] = C(0.5) * (ax + bx);
  fs[3] = C(0.5) * (ax - bx);
  fs[2] = C(0.5) * (ay + by);
  fs[4] = C(0.5) * (ay - by);
  fs[0] = (M.rho - (M.pxx + M.pyy)) + r;
}

// Writes (u^{n+1}, v^n) into trace slot `slot` of the receiver at (x, y),
// if any.
template <class U>
__device__ __forceinline__ void record_receiver(const StepParams &p, int slot, int x, int y,
                                                U ux, U uy, U vx, U vy) {
  // no table lookup outside the bounding box of the receivers
  if (x < p.rec_x0 || x > p.rec_x1 || y < p.rec_y0 || y > p.rec_y1) return;
  const int tile = (y / kRecTileY) * p.rec_tiles_x + x / kRecTileX;
  const int r0 = p.rec_tile_ptr[tile], r1 = p.rec_tile_ptr[tile + 1];
  for (int r = r0; r < r1; ++r) {
    if (p.rec_xy[2 * r] == x && p.rec_xy[2 * r + 1] == y) {
      double *t = p.traces + ((long long)slot * p.nrec + p.rec_id[r]) * 4;
      t[0] = (double)ux;
      t[1] = (double)uy;
      t[2] = (double)vx;
      t[3] = (double)vy;
    }
  }
}

// Everything after streaming and the density gradient: moments, source and
// physical flux, equilibrium/BGK/forcing, stores, displacement, receivers.
// MODE 0: full step.  MODE 1: fields of the current state (no state change).
// With UIN the current displacement comes in (ux0, uy0) instead of being read
// from global memory.
template <class T, class C, class U, bool LAM, int MODE, bool UIN = false>
__device__ __forceinline__ void finish_cell(const StepParams &p, const C *f, C gx, C gy, C Fx,
                                            C Fy, int x, int y, int xc, int yc, bool active,
                                            U ux0 = U(0), U uy0 = U(0)) {
  const Moments<C> M = cell_moments<C>(f);
  C Gx = C(0), Gy = C(0);
  if (LAM) {
    // elastic force (mu - lambda)/rho0 grad rho = Lambda b^2 grad rho (Eq. 9)
    // (products rounded on their own: Gx + Fx is never contracted, so cells
    // near a source round alike on every path)
    const C lb2 = mat_at<C>(p.lam, p.mat_per_cell, xc, yc, p.pitch) * C(1.0 / 3.0);
    Gx = mul_rn(lb2, gx);
    Gy = mul_rn(lb2, gy);
  }
  const C A = sponge_A<C>(p, xc, yc);
  C jx, jy, Sx, Sy;
  flux_and_source<C>(M.mx, M.my, Gx, Gy, Fx, Fy, A, jx, jy, Sx, Sy);
  const C irho = irho_at<T, C>(p, xc, yc);

  if (MODE == 1) {
    if (!active) return;
    const long long o = (long long)(y - p.row0) * p.nx + x;
    const int c = y * p.pitch + x;
    const U *u = (const U *)p.u;
    if (p.out[0]) p.out[0][o] = (double)u[c];
    if (p.out[1]) p.out[1][o] = (double)u[p.plane + c];
    if (p.out[2]) p.out[2][o] = (double)mul_rn(jx, irho);
    if (p.out[3]) p.out[3][o] = (double)mul_rn(jy, irho);
    const C us = unit_scale<T, C>(p);
    if (p.out[4]) p.out[4][o] = (double)(M.rho * us);
    if (p.out[5]) p.out[5][o] = (double)(M.pxx * us);
    if (p.out[6]) p.out[6][o] = (double)(M.pxy * us);
    if (p.out[7]) p.out[7][o] = (double)(M.pyy * us);
    return;
  }

  C fs[9];
  collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f), fs);
  if (!active) return;
  const int c = y * p.pitch + x;
  T *fout = (T *)p.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  U *u = (U *)p.u;
  const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
  const U ux = (UIN ? ux0 : __ldcg(u + c)) + vx;
  const U uy = (UIN ? uy0 : __ldcg(u + p.plane + c)) + vy;
  u[c] = ux;
  u[p.plane + c] = uy;
  // non-finite guard: x * 0 == 0 fails exactly for NaN and +-Inf
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
  if (p.trace_slot >= 0) record_receiver<U>(p, p.trace_slot, x, y, ux, uy, vx, vy);
}

// Cells near a wall or a periodic seam: every pull goes through the general
// path with the wall rules, and so do the neighbours' densities.  Kept out
// of line so that the interior path carries none of this code.
template <class T, class C, class U, bool LAM, int MODE>
__device__ __noinline__ void boundary_cell(const StepParams &p, C Fx, C Fy, int x, int y, int xc,
                                           int yc, bool active) {
  const T *fin = (const T *)p.fin;
  C f[9];
#pragma unroll
  pull_cell<T, C>(p, GridPops<T>{fin, p.fplane, p.frow}, xc, yc, f);
  C gx = C(0), gy = C(0);
  if (LAM) {
    const C rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    grad_rho<T, C>(p, fin, xc, yc, rho, gx, gy);
  }
  finish_cell<T, C, U, LAM, MODE>(p, f, gx, gy, Fx, Fy, x, y, xc, yc, active);
}

// Whether the block's cells [x0, x0 + W) x [y0, y0 + h) need anything
// beyond the bulk update: a wall or periodic seam within m cells, a source
// reaching the block widened by `halo` cells on every side, or (when
// recording) a receiver in the block.  Warp-wide (all 32 lanes call it);
// every lane gets the same answer.  near (optional): the host's flag of the
// block (StepParams::blk_near); 0 skips the source and receiver lookups.
template <int W = 32>
__device__ __forceinline__ bool block_is_special(const StepParams &p, int x0, int y0, int h,
                                                 int m, int halo = 0,
                                                 const unsigned char *near = nullptr) {
  static_assert(W == 32 || W == kRecTileX, "a block spans one receiver tile column");
  if (x0 < m || x0 + W > p.nx - m || y0 < m || y0 + h > p.ny - m) return true;
  const bool near_src = p.nsrc > 0 && x0 - halo <= p.src_x1 && x0 + W - 1 + halo >= p.src_x0 &&
                        y0 - halo <= p.src_y1 && y0 + h - 1 + halo >= p.src_y0;
  const bool near_rec = p.trace_slot >= 0 && x0 <= p.rec_x1 && x0 + W - 1 >= p.rec_x0 &&
                        y0 <= p.rec_y1 && y0 + h - 1 >= p.rec_y0;
  if (!near_src && !near_rec) return false;
  if (near != nullptr && *near == 0) return false;
  if (p.nsrc > 32) return true;
  const int lane = threadIdx.x & 31;
  bool hit = false;
  if (near_src && lane < p.nsrc) {
    const int4 qb = src_bound(p, lane);
    int dx = x0 + W / 2 - qb.x, dy = y0 + h / 2 - qb.y;
    if (p.bc_left == BC_PERIODIC) {
      if (dx > p.nx / 2) dx -= p.nx;
      else if (dx < -(p.nx / 2)) dx += p.nx;
    }
    if (p.bc_top == BC_PERIODIC) {
      if (dy > p.ny / 2) dy -= p.ny;
      else if (dy < -(p.ny / 2)) dy += p.ny;
    }
    hit = abs(dx) <= qb.z + W / 2 + 1 + halo && abs(dy) <= qb.z + h / 2 + 1 + halo;
  }
  if (near_rec && lane >= 30) {
    // receiver tiles are 64 x 4; this block spans one tile column, and rows
    // y0 / 4 .. (y0 + h - 1) / 4
    for (int ty = y0 / kRecTileY + (lane - 30); ty * kRecTileY < y0 + h && ty * kRecTileY < p.ny;
         ty += 2) {
      const int t = ty * p.rec_tiles_x + x0 / kRecTileX;
      hit |= p.rec_tile_ptr[t + 1] > p.rec_tile_ptr[t];
    }
  }
  return __ballot_sync(0xffffffffu, hit) != 0u;
}

// Full update of one cell without the gradient force but with every other
// feature (walls, sources, receivers): the path of blocks that are special,
// kept out of line so the bulk path carries none of its registers.
template <class T, class C, class U, int MODE>
__device__ __noinline__ void general_cell(const StepParams &p, int x, int y, int yend) {
  const bool active = x < p.nx && y < yend;
  const int xc = x < p.nx ? x : p.nx - 1;
  const int yc = y < yend ? y : yend - 1;
  C Fx, Fy;
  body_force<C>(p, xc, yc, Fx, Fy);  // all lanes of the warp take part
  Fx *= force_scale<T, C>(p);
  Fy *= force_scale<T, C>(p);
  if (!(xc >= 1 && xc < p.nx - 1 && yc >= 1 && yc < p.ny - 1)) {
    boundary_cell<T, C, U, false, MODE>(p, Fx, Fy, x, y, xc, yc, active);
    return;
  }
  const T *fin = (const T *)p.fin;
  C f[9];
  {
    const T *b = fin + (yc * p.frow + xc);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  }
  const U *u = (const U *)p.u;
  const int c = yc * p.pitch + xc;
  const U ux0 = __ldcg(u + c), uy0 = __ldcg(u + p.plane + c);  // before any store
  finish_cell<T, C, U, false, MODE, true>(p, f, C(0), C(0), Fx, Fy, x, y, xc, yc, active, ux0,
                                          uy0);
}

// Flux, source and collision of a bulk cell (no wall, no body force): the
// absorbing layer where the block overlaps one (spg), else j = m + G/2,
// S = G.
template <class C>
__device__ __forceinline__ void bulk_collide(const StepParams &p, const Moments<C> &M, C Gx, C Gy,
                                             bool spg, int x, int y, C *fs, C &jx, C &jy) {
  C Sx, Sy;
  if (spg) {
    flux_and_source<C>(M.mx, M.my, Gx, Gy, C(0), C(0), sponge_A<C>(p, x, y), jx, jy, Sx, Sy);
  } else {
    jx = M.mx + C(0.5) * Gx;
    jy = M.my + C(0.5) * Gy;
    Sx = Gx;
    Sy = Gy;
  }
  collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f), fs);
}

// Ring cell t (0 <= t < 64 + 2 R) around a block of 32 x R cells, as an
// offset from the block's first cell: the rows above and below (64 cells),
// then the columns left and right (2 R).
template <int R>
__device__ __forceinline__ void ring_cell(int t, int &hx, int &hy) {
  if (t < 64) {
    hx = t & 31;
    hy = t < 32 ? -1 : R;
  } else {
    hx = (t & 1) ? 32 : -1;
    hy = (t - 64) >> 1;
  }
}

// Update of a block of 32 x R cells with the density-gradient force that
// needs the general path (walls, periodic seams, sources, receivers).  The
// streamed densities of the block and of the ring around it (periodic axes
// wrapped) go to shared memory first, so a cell pulls its populations once
// rather than once for itself and once per neighbour; the wall rules then
// supply the ghosts on non-periodic edges.  Every thread of the block calls
// it (one barrier).
template <class T, class C, class U, int MODE, int R>
__device__ __noinline__ void general_block_lam(const StepParams &p, int x0, int y0, int yend) {
  __shared__ C rho_s[R + 2][34];
  // the input populations of the block widened by two cells (the pulls of
  // its cells and of the density ring), staged by one pass of copies; only
  // for blocks of 8 rows or more (4-row blocks, many per SM, would give up
  // most of the L1 cache to it: the batched 4-row form measured 9 % slower)
  constexpr bool STAGE = stages<T>() && R >= 8;
  constexpr int SW = stage_width<T>(32, 2), SH = R + 4;
  __shared__ __align__(16) T stage[STAGE ? 9 * SH * SW : 8];
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < p.nx && y < yend;
  const int xc = x < p.nx ? x : p.nx - 1;
  const int yc = y < yend ? y : yend - 1;
  const T *fin = (const T *)p.fin;
  const int sox = stage_origin<T>(x0, 2);
  if constexpr (STAGE) stage_rows<T, SW, SH, 32 * R>(p, fin, sox, y0 - 2, stage);
  C Fx, Fy;
  body_force<C>(p, xc, yc, Fx, Fy);  // all lanes of the warp take part
  Fx *= force_scale<T, C>(p);
  Fy *= force_scale<T, C>(p);
  if constexpr (STAGE) {
    stage_wait();
    __syncthreads();
  }
  const StagePops<T, SW, SH> sg{stage, sox, y0 - 2};
  C f[9];
  if constexpr (STAGE) pull_staged<T, C>(p, sg, xc, yc, f);
  else gather<T, C>(p, fin, xc, yc, f);
  const C rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  // a cell of the block outside the updated range holds the density of its
  // own (wrapped) coordinate, as a neighbour of the cells that are updated
  rho_s[ty + 1][tx + 1] = active ? rho : rho_wrapped<T, C>(p, fin, x, y);
  if (t < 64 + 2 * R) {
    int hx, hy;
    ring_cell<R>(t, hx, hy);
    const int rx = x0 + hx, ry = y0 + hy;
    C r = C(0);
    if constexpr (STAGE) {
      // zero beyond a non-periodic edge, as rho_wrapped gives
      if ((p.bc_left == BC_PERIODIC || (rx >= 0 && rx < p.nx)) &&
          (p.bc_top == BC_PERIODIC || (ry >= 0 && ry < p.ny))) {
        C v[9];
        pull_staged<T, C>(p, sg, rx, ry, v);
        r = v[0] + v[1] + v[2] + v[3] + v[4] + v[5] + v[6] + v[7] + v[8];
      }
    } else {
      r = rho_wrapped<T, C>(p, fin, rx, ry);
    }
    rho_s[hy + 1][hx + 1] = r;
  }
  __syncthreads();
  C rxm = rho_s[ty + 1][tx], rxp = rho_s[ty + 1][tx + 2];
  C rym = rho_s[ty][tx + 1], ryp = rho_s[ty + 2][tx + 1];
  wall_ghosts<C>(p, xc == 0, xc == p.nx - 1, p.bc_left, p.bc_right, rho, rxm, rxp);
  wall_ghosts<C>(p, yc == 0, yc == p.ny - 1, p.bc_top, p.bc_bottom, rho, rym, ryp);
  const C gx = C(0.5) * (rxp - rxm), gy = C(0.5) * (ryp - rym);
  if (MODE == 0 && p.grad_out && active) {
    ((C *)p.grad_out)[y * p.pitch + x] = gx;
    ((C *)p.grad_out)[p.plane + y * p.pitch + x] = gy;
  }
  finish_cell<T, C, U, true, MODE>(p, f, gx, gy, Fx, Fy, x, y, xc, yc, active);
}

// One thread per cell, blocks of 32 x 8 threads (a warp is 32 consecutive
// cells of a row).  Blocks in the bulk (no wall, source or receiver nearby)
// do only what the bulk needs: pull, moments, the absorbing layer where the
// block overlaps one, the density-gradient force when some Lambda != 0,
// collision, stores, displacement.  MODE 0: full step.  MODE 1: fields of the
// current state, rows [row0, row0 + nrows).
// LBM_PDL: launch the steps with programmatic dependent launch (the next
// step's blocks are scheduled while the previous step drains; each waits for
// the previous step to complete before reading).  LBM_ORDER 1: on reversed
// steps the top block row (free surface, receivers) is still visited first,
// so the slower wall blocks never form the last wave.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
#ifndef LBM_ORDER
#define LBM_ORDER 1
#endif

// Resident blocks per SM the compiler is asked to allow for (sets the
// register budget of the step kernel: 65536 / (256 x this)).
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 6
#endif
#ifndef LBM_STEP_MIN_BLOCKS_LAM
#define LBM_STEP_MIN_BLOCKS_LAM 8
#endif

template <class T, class C, class U, bool LAM, int MODE, int R>
__device__ __forceinline__ void step_block(const StepParams &p, int bx, int by);

template <class T, class C, class U, bool LAM, int MODE>
__global__ void __launch_bounds__(LAM ? 32 * kLamRows : 256,
                                  LAM ? LBM_STEP_MIN_BLOCKS_LAM : LBM_STEP_MIN_BLOCKS)
    step_kernel(const StepParams p) {
#if LBM_PDL
  // programmatic dependent launch: wait for the previous step to complete
  // (its populations are this step's input), then let the next step's
  // blocks be scheduled as SMs free up
  if (MODE == 0) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
  }
#endif
  // alternate steps visit the blocks in reverse order: the rows written last
  // by one step (still in L2) are the first the next step reads
  int bx = blockIdx.x, by = blockIdx.y;
  if (MODE == 0 && p.reverse) {
#if LBM_ORDER == 1
    // the top block row (walls, receivers) still goes first
    if (by > 0) by = gridDim.y - by;
    bx = gridDim.x - 1 - bx;
#else
    bx = gridDim.x - 1 - bx;
    by = gridDim.y - 1 - by;
#endif
  }
  step_block<T, C, U, LAM, MODE, LAM ? kLamRows : 8>(p, bx, by);
}

// The update of block (bx, by) of 32 x R cells by 32 x R threads.
template <class T, class C, class U, bool LAM, int MODE, int R>
__device__ __forceinline__ void step_block(const StepParams &p, int bx, int by) {
  const int x0 = bx * 32;
  const int x = x0 + threadIdx.x;
  const int y0 = by * R + (MODE == 1 ? p.row0 : 0);
  const int y = y0 + threadIdx.y;
  const int yend = MODE == 1 ? p.row0 + p.nrows : p.ny;
  const int m = LAM ? 2 : 1;
  // the host's per-block flags are laid out for the single grid's 32 x 8
  // blocks of one-step launches; taken with the gradient force only (with
  // Lambda = 0 the flag's load made the 8192^2 step 8 % slower, with it the
  // 16-bit step 4 % faster)
  const unsigned char *near = (LAM && MODE == 0 && R == 8 && p.blk_near != nullptr)
                                  ? p.blk_near + (by * ((p.nx + 31) >> 5) + bx)
                                  : nullptr;
  if (MODE == 1 || block_is_special(p, x0, y0, R, m, 0, near)) {
    // the same for every thread of the block (block_is_special depends on
    // the block's position only)
    if (LAM) general_block_lam<T, C, U, MODE, R>(p, x0, y0, yend);
    else general_cell<T, C, U, MODE>(p, x, y, yend);
    return;
  }
  // bulk cell: every upstream cell (and every neighbour's) is inside the
  // grid.  All loads of the cell are issued before any store (the
  // displacement could otherwise not be read until the populations are
  // written).
  const T *fin = (const T *)p.fin;
  C f[9];
  {
    const T *b = fin + (y * p.frow + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  }
  // the first 64 + 2 R threads of a block with the gradient force also pull
  // the populations of one cell of the ring around the block.  They are
  // loaded together with the cell's own, so both wait for one memory
  // latency, not two.
  const int t = threadIdx.y * 32 + threadIdx.x;
  int hx = 0, hy = 0;
  C hf[LAM ? 9 : 1];
  if (LAM && t < 64 + 2 * R) {
    ring_cell<R>(t, hx, hy);
    const T *b = fin + ((y0 + hy) * p.frow + x0 + hx);
#pragma unroll
    for (int i = 0; i < (LAM ? 9 : 1); ++i)
      hf[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  }
  const int c = y * p.pitch + x;
  U *u = (U *)p.u;
  const U ux0 = __ldcg(u + c), uy0 = __ldcg(u + p.plane + c);
  const C irho = irho_at<T, C>(p, x, y);
  const Moments<C> M = cell_moments<C>(f);
  C Gx = C(0), Gy = C(0);
  if (LAM) {
    // streamed density of the block and its ring in shared memory (every
    // block in this branch is bulk: the barrier is uniform)
    // (every density that enters a gradient is the plain sum f_0 + ... + f_8
    // of the pulled populations, on every path, so the result of a cell does
    // not depend on which path its block takes)
    __shared__ C rho_s[R + 2][34];
    rho_s[threadIdx.y + 1][threadIdx.x + 1] =
        f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    if (t < 64 + 2 * R) {
      C r = C(0);
#pragma unroll
      for (int i = 0; i < (LAM ? 9 : 1); ++i) r += hf[i];
      rho_s[hy + 1][hx + 1] = r;
    }
    __syncthreads();
    // elastic force Lambda b^2 grad rho with the centred difference (Eqs. 9-10)
    const C gx = C(0.5) * (rho_s[threadIdx.y + 1][threadIdx.x + 2] - rho_s[threadIdx.y + 1][threadIdx.x]);
    const C gy = C(0.5) * (rho_s[threadIdx.y + 2][threadIdx.x + 1] - rho_s[threadIdx.y][threadIdx.x + 1]);
    if (p.grad_out) {
      ((C *)p.grad_out)[c] = gx;
      ((C *)p.grad_out)[p.plane + c] = gy;
    }
    const C lb2 = mat_at<C>(p.lam, p.mat_per_cell, x, y, p.pitch) * C(1.0 / 3.0);
    Gx = mul_rn(lb2, gx);
    Gy = mul_rn(lb2, gy);
  }
  C jx, jy, fs[9];
  const bool spg = x0 < p.sp_left || x0 + 32 > p.nx - p.sp_right || y0 < p.sp_top ||
                   y0 + R > p.ny - p.sp_bottom;
  bulk_collide<C>(p, M, Gx, Gy, spg, x, y, fs, jx, jy);
  T *fout = (T *)p.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  u[c] = ux0 + U(mul_rn(jx, irho));
  u[p.plane + c] = uy0 + U(mul_rn(jy, irho));
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
}

// Launch entry points, one translation unit per storage type.
void launch_step_f64(const StepParams &p, bool lam, int mode, dim3 grid, dim3 block,
                     cudaStream_t s);
void launch_step_f32(const StepParams &p, bool lam, bool u64, int mode, dim3 grid, dim3 block,
                     cudaStream_t s);
void launch_step_16(const StepParams &p, bool bf16, bool lam, bool u64, int mode, dim3 grid,
                    dim3 block, cudaStream_t s);

// Launches kernel k with programmatic stream serialization when LBM_PDL is
// set (the kernel then starts with griddepcontrol.wait), else plainly.
template <class K>
inline cudaError_t launch_pdl(K k, dim3 grid, dim3 block, cudaStream_t s, const StepParams &p) {
#if LBM_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, p);
#else
  k<<<grid, block, 0, s>>>(p);
  return cudaSuccess;
#endif
}


}  // namespace lbm
