// Two steps per launch with the density-gradient force (some Lambda != 0).
//
// The force of a cell needs the streamed densities of its four neighbours
// (Eq. 10), so each step reaches one cell further than without it.  A block
// owns a 28 x kL2Rows tile and computes:
//   step n on W2 = the tile widened by two cells (32 x (kL2Rows + 4), one
//     cell per thread), from the streamed densities of W3 = the tile widened
//     by three cells (W2's own plus a one-cell ring pulled from HBM);
//   its post-collision populations on W2 into shared memory;
//   the streamed densities of step n + 1 on W1 = the tile widened by one cell
//     (pulled from the shared W2 window), then step n + 1 of the tile cells.
// Per two steps the populations cross HBM once each way; every cell update
// uses the one-step arithmetic (the plain sums f_0 + ... + f_8 for every
// density that enters a gradient, the same wall ghosts), so results are
// bit-identical to one step per launch.
#pragma once

#include "step_fused.cuh"

namespace lbm {

constexpr int kL2Cols = 28;             // columns of a tile
constexpr int kL2Rows = 12;             // rows of a tile
constexpr int kL2W = kL2Cols + 4;       // W2: 32 columns, one warp per row
constexpr int kL2H = kL2Rows + 4;       // W2 rows = warps per block
constexpr int kL2RW = kL2W + 2;         // W3 columns (density buffer)
constexpr int kL2RH = kL2H + 2;         // W3 rows
constexpr int kL2Ring = 2 * kL2RW + 2 * kL2H;  // W3 cells outside W2
static_assert(kL2W == 32, "a W2 row is one warp");
// Staged region of a general tile: the tile widened by four cells (the W3
// ring's pulls), aliasing the W2 window buffer until step n's stores.
template <class T>
constexpr int l2_stage_w() { return stage_width<T>(kL2Cols, 4); }
constexpr int kL2SH = kL2Rows + 8;
template <class T>
constexpr int l2_buf() {
  return stages<T>() && 9 * kL2SH * l2_stage_w<T>() > 9 * kL2H * kL2W
             ? 9 * kL2SH * l2_stage_w<T>()
             : 9 * kL2H * kL2W;
}
static_assert(kL2Ring <= 32 * kL2H, "one ring cell per thread at most");

#ifndef LBM_STEP2L_MIN_BLOCKS
#define LBM_STEP2L_MIN_BLOCKS (2048 / (32 * kL2H))
#endif

// Ring cell t (0 <= t < kL2Ring) of W3 in W3 coordinates: the top and bottom
// rows, then the left and right columns beside W2's rows.
__device__ __forceinline__ void lam_ring_cell(int t, int &hx, int &hy) {
  if (t < 2 * kL2RW) {
    hx = t % kL2RW;
    hy = t < kL2RW ? 0 : kL2RH - 1;
  } else {
    const int q = t - 2 * kL2RW;
    hx = (q & 1) ? kL2RW - 1 : 0;
    hy = 1 + (q >> 1);
  }
}

// Whether a tile at (x0, y0) takes the general rules: an edge or seam of the
// grid within four cells (W3's pulls), a source reaching W2, or a receiver
// among the tile's cells when recording.  Warp-wide.  lookup = false skips
// the source and receiver tests (a tile the host's launch order places
// after every tile a source or receiver can reach).
__device__ __forceinline__ bool lam_tile_special(const StepParams &p, int x0, int y0,
                                                 int slot_a, bool lookup = true) {
  constexpr int W = kL2Cols, H = kL2Rows;
  if (x0 < 4 || x0 + W > p.nx - 4 || y0 < 4 || y0 + H > p.ny - 4) return true;
  if (!lookup) return false;
  const bool near_src = p.nsrc > 0 && x0 - 2 <= p.src_x1 && x0 + W + 1 >= p.src_x0 &&
                        y0 - 2 <= p.src_y1 && y0 + H + 1 >= p.src_y0;
  const bool near_rec = slot_a >= 0 && x0 <= p.rec_x1 && x0 + W - 1 >= p.rec_x0 &&
                        y0 <= p.rec_y1 && y0 + H - 1 >= p.rec_y0;
  if (!near_src && !near_rec) return false;
  if (near_src && p.nsrc > 32) return true;
  const int lane = threadIdx.x & 31;
  bool hit = false;
  if (near_src && lane < p.nsrc) {
    // W2 cells lie within W/2 + 2 columns and H/2 + 2 rows of the centre
    const int4 qb = src_bound(p, lane);
    int dx = x0 + W / 2 - qb.x, dy = y0 + H / 2 - qb.y;
    if (p.bc_left == BC_PERIODIC) {
      if (dx > p.nx / 2) dx -= p.nx;
      else if (dx < -(p.nx / 2)) dx += p.nx;
    }
    if (p.bc_top == BC_PERIODIC) {
      if (dy > p.ny / 2) dy -= p.ny;
      else if (dy < -(p.ny / 2)) dy += p.ny;
    }
    hit = abs(dx) <= qb.z + W / 2 + 3 && abs(dy) <= qb.z + H / 2 + 3;
  }
  if (near_rec) {
    const int tx0 = x0 / kRecTileX, tx1 = min((x0 + W - 1) / kRecTileX, p.rec_tiles_x - 1);
    const int ty0 = y0 / kRecTileY, ty1 = min((y0 + H - 1) / kRecTileY, (p.ny - 1) / kRecTileY);
    const int nty = ty1 - ty0 + 1;
    for (int j = lane; j < (tx1 - tx0 + 1) * nty; j += 32) {
      const int t = (ty0 + j % nty) * p.rec_tiles_x + tx0 + j / nty;
      hit |= p.rec_tile_ptr[t + 1] > p.rec_tile_ptr[t];
    }
  }
  return __ballot_sync(0xffffffffu, hit) != 0u;
}

// The W2 window in shared memory, [9][kL2H][kL2W]; element (0, 0) is grid
// cell (ox, oy) = (x0 - 2, y0 - 2); periodic images at unwrapped
// coordinates.
template <class T>
struct LamTilePops {
  const T *f;
  int ox, oy;
  static constexpr bool kWrap = false;
  __device__ __forceinline__ const T *at(int i, int x, int y) const {
    return f + ((i * kL2H + (y - oy)) * kL2W + (x - ox));
  }
  template <class C>
  __device__ __forceinline__ C load(int i, int x, int y) const {
    return ld<T, C>(at(i, x, y));
  }
};

// With p.grad_out set (the adjoint's recording runs): the centred density
// gradient of step n + k (k = 0, 1) of cell index c, into the k-th of two
// consecutive records of two planes each ([2][2][ny][pitch], compute type),
// as the one-step kernel stores it.
template <class C>
__device__ __forceinline__ void store_grad(const StepParams &p, int k, int c, C gx, C gy) {
  C *g = (C *)p.grad_out + 2LL * k * p.plane;
  g[c] = gx;
  g[p.plane + c] = gy;
}

// The plain bulk tile: no edge or seam within four cells, no source, no
// receiver.  Every thread calls it (three block barriers).
template <class T, class C, class U>
__device__ __forceinline__ void lam_bulk(const StepParams &p, const Phase2 &ph, int x0, int y0,
                                         T *tile, C (*rho_s)[kL2RW]) {
  const int lane = threadIdx.x, w = threadIdx.y, t = w * 32 + lane;
  const int x = x0 - 2 + lane, y = y0 - 2 + w;  // this thread's W2 cell
  const bool w1 = lane >= 1 && lane <= kL2W - 2 && w >= 1 && w <= kL2H - 2;
  const bool core = lane >= 2 && lane <= kL2W - 3 && w >= 2 && w <= kL2H - 3;
  const T *fin = (const T *)ph.fin;
  C f[9];
  {
    const T *b = fin + (y * p.frow + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  }
  // the ring of W3 around W2, pulled together with the cells' own
  int hx = 0, hy = 0;
  C hf[9];
  if (t < kL2Ring) {
    lam_ring_cell(t, hx, hy);
    const T *b = fin + ((y0 - 3 + hy) * p.frow + (x0 - 3 + hx));
#pragma unroll
    for (int i = 0; i < 9; ++i)
      hf[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
  }
  U *u = (U *)p.u;
  const int c = y * p.pitch + x;
  U ux = U(0), uy = U(0);
  C irho = C(0);
  if (core) {
    ux = __ldcg(u + c);
    uy = __ldcg(u + p.plane + c);
    irho = irho_at<T, C>(p, x, y);
  }
  // streamed densities of step n on W3 (the plain sums, as on every path)
  rho_s[w + 1][lane + 1] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  if (t < kL2Ring) {
    C r = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) r += hf[i];
    rho_s[hy][hx] = r;
  }
  __syncthreads();
  const bool spg = x0 - 2 < p.sp_left || x0 + kL2Cols + 2 > p.nx - p.sp_right ||
                   y0 - 2 < p.sp_top || y0 + kL2Rows + 2 > p.ny - p.sp_bottom;
  const C lb2 = mat_at<C>(p.lam, p.mat_per_cell, x, y, p.pitch) * C(1.0 / 3.0);
  {
    // step n on W2: elastic force Lambda b^2 grad rho (Eqs. 9-10)
    const C gx = C(0.5) * (rho_s[w + 1][lane + 2] - rho_s[w + 1][lane]);
    const C gy = C(0.5) * (rho_s[w + 2][lane + 1] - rho_s[w][lane + 1]);
    if (core && p.grad_out) store_grad<C>(p, 0, c, gx, gy);
    const Moments<C> M = cell_moments<C>(f);
    C jx, jy, fs[9];
    bulk_collide<C>(p, M, mul_rn(lb2, gx), mul_rn(lb2, gy), spg, x, y, fs, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) st<T, C>(tile + ((i * kL2H + w) * kL2W + lane), fs[i]);
    if (core) {
      ux += U(mul_rn(jx, irho));
      uy += U(mul_rn(jy, irho));
    }
  }
  __syncthreads();
  // streamed densities of step n + 1 on W1, pulled from the window
  if (w1) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      f[i] = ld<T, C>(tile + ((i * kL2H + w - cyd(i)) * kL2W + lane - cxd(i)));
    rho_s[w + 1][lane + 1] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  }
  __syncthreads();
  if (!core) return;
  // step n + 1 of the tile cell
  const C gx = C(0.5) * (rho_s[w + 1][lane + 2] - rho_s[w + 1][lane]);
  const C gy = C(0.5) * (rho_s[w + 2][lane + 1] - rho_s[w][lane + 1]);
  if (p.grad_out) store_grad<C>(p, 1, c, gx, gy);
  const Moments<C> M = cell_moments<C>(f);
  C jx, jy, fs[9];
  bulk_collide<C>(p, M, mul_rn(lb2, gx), mul_rn(lb2, gy), spg, x, y, fs, jx, jy);
  T *fout = (T *)ph.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  u[c] = ux + U(mul_rn(jx, irho));
  u[p.plane + c] = uy + U(mul_rn(jy, irho));
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
}

// Tiles near an edge or seam, a source or receivers: every cell at its
// wrapped coordinate, cells beyond a non-periodic edge skipped (density 0,
// as rho_wrapped gives; the wall ghosts replace it), the wall rules for the
// pulls (in step n from the input populations of the tile widened by four
// cells, staged in shared memory by one pass of loads; in step n + 1 from
// the window), the body force per cell and the receivers.  Out of line;
// every thread calls it (four barriers).
//
// Register budget: the body force of each step is summed (out of line, in
// the sources' bounding box) before that step's pulls, when little else is
// live, and the displacement after step n goes through global memory (u +
// v^n stored, reloaded for + v^{n+1}: the same two roundings).
template <class T, class C, class U>
__device__ __noinline__ void lam_general(const StepParams &p, const Phase2 &ph, int x0, int y0,
                                         T *tile, C (*rho_s)[kL2RW]) {
  const int lane = threadIdx.x, w = threadIdx.y, t = w * 32 + lane;
  const int x = x0 - 2 + lane, y = y0 - 2 + w;  // W2 cell, unwrapped
  int wx = x, wy = y;
  bool valid = true;
  if (x < 0 || x >= p.nx) {
    if (p.bc_left == BC_PERIODIC) wx = wrap_any(x, p.nx);
    else valid = false;
  }
  if (y < 0 || y >= p.ny) {
    if (p.bc_top == BC_PERIODIC) wy = wrap_any(y, p.ny);
    else valid = false;
  }
  const bool w1 = lane >= 1 && lane <= kL2W - 2 && w >= 1 && w <= kL2H - 2;
  const bool core = lane >= 2 && lane <= kL2W - 3 && w >= 2 && w <= kL2H - 3;
  const bool active = core && x < p.nx && y < p.ny;
  // W2 cells lie within kL2Cols/2 + 2 columns and kL2Rows/2 + 2 rows of the
  // centre
  const unsigned smask = source_mask(p, x0 + kL2Cols / 2, y0 + kL2Rows / 2, kL2Cols / 2 + 3,
                                     kL2Rows / 2 + 3);
  C Fx = C(0), Fy = C(0);
  if (valid) body_force_cell<C>(p, wx, wy, ph.n, Fx, Fy, smask);
  // the input populations of every pull of step n (W2's and the W3 ring's),
  // staged in the window buffer, which step n's stores overwrite only after
  // the barrier that follows the pulls
  constexpr int SW = l2_stage_w<T>();
  const int sox = stage_origin<T>(x0, 4);
  if constexpr (stages<T>()) {
    stage_rows<T, SW, kL2SH, 32 * kL2H>(p, (const T *)ph.fin, sox, y0 - 4, tile);
    stage_wait();
  }
  __syncthreads();
  const StagePops<T, SW, kL2SH> sg{tile, sox, y0 - 4};
  C f[9];
  C rho = C(0);
  if (valid) {
    if constexpr (stages<T>()) pull_staged<T, C>(p, sg, x, y, f);
    else gather<T, C>(p, (const T *)ph.fin, wx, wy, f);
  }
  // the ring's densities (zero beyond a non-periodic edge), by the block's
  // last threads (W2 rows away from a top wall, or beyond a bottom wall)
  const int tr = 32 * kL2H - 1 - t;
  if (tr < kL2Ring) {
    int hx, hy;
    lam_ring_cell(tr, hx, hy);
    const int rx = x0 - 3 + hx, ry = y0 - 3 + hy;
    C r = C(0);
    if constexpr (stages<T>()) {
      if ((p.bc_left == BC_PERIODIC || (rx >= 0 && rx < p.nx)) &&
          (p.bc_top == BC_PERIODIC || (ry >= 0 && ry < p.ny))) {
        C v[9];
        pull_staged<T, C>(p, sg, rx, ry, v);
        r = v[0] + v[1] + v[2] + v[3] + v[4] + v[5] + v[6] + v[7] + v[8];
      }
    } else {
      r = rho_wrapped<T, C>(p, (const T *)ph.fin, rx, ry);
    }
    rho_s[hy][hx] = r;
  }
  if (valid) rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  rho_s[w + 1][lane + 1] = rho;
  __syncthreads();
  U *u = (U *)p.u;
  const int c = y * p.pitch + x;
  if (valid) {
    // step n on W2
    C rxm = rho_s[w + 1][lane], rxp = rho_s[w + 1][lane + 2];
    C rym = rho_s[w][lane + 1], ryp = rho_s[w + 2][lane + 1];
    wall_ghosts<C>(p, wx == 0, wx == p.nx - 1, p.bc_left, p.bc_right, rho, rxm, rxp);
    wall_ghosts<C>(p, wy == 0, wy == p.ny - 1, p.bc_top, p.bc_bottom, rho, rym, ryp);
    const C gx = C(0.5) * (rxp - rxm), gy = C(0.5) * (ryp - rym);
    if (active && p.grad_out) store_grad<C>(p, 0, c, gx, gy);
    const C lb2 = mat_at<C>(p.lam, p.mat_per_cell, wx, wy, p.pitch) * C(1.0 / 3.0);
    Fx *= force_scale<T, C>(p);
    Fy *= force_scale<T, C>(p);
    const Moments<C> M = cell_moments<C>(f);
    C jx, jy, Sx, Sy, fs[9];
    flux_and_source<C>(M.mx, M.my, mul_rn(lb2, gx), mul_rn(lb2, gy), Fx, Fy,
                       sponge_A<C>(p, wx, wy), jx, jy, Sx, Sy);
    collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f),
                    fs);
#pragma unroll
    for (int i = 0; i < 9; ++i) st<T, C>(tile + ((i * kL2H + w) * kL2W + lane), fs[i]);
    if (active) {
      const C irho = irho_at<T, C>(p, x, y);
      const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
      const U ux = __ldcg(u + c) + vx, uy = __ldcg(u + p.plane + c) + vy;
      u[c] = ux;
      u[p.plane + c] = uy;
      if (ph.slot_a >= 0) record_receiver<U>(p, ph.slot_a, x, y, ux, uy, vx, vy);
    }
  }
  __syncthreads();
  Fx = C(0);
  Fy = C(0);
  if (active) body_force_cell<C>(p, x, y, ph.n + 1, Fx, Fy, smask);
  // streamed densities of step n + 1 on W1 (0 beyond a non-periodic edge)
  if (w1) {
    rho = C(0);
    if (valid) {
      if (off_walls(p, wx, wy)) {
        // the window holds the periodic images at unwrapped coordinates
#pragma unroll
        for (int i = 0; i < 9; ++i)
          f[i] = ld<T, C>(tile + ((i * kL2H + w - cyd(i)) * kL2W + lane - cxd(i)));
      } else {
        pull_cell<T, C>(p, LamTilePops<T>{tile, x0 - 2, y0 - 2}, x, y, f);
      }
      rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    }
    rho_s[w + 1][lane + 1] = rho;
  }
  __syncthreads();
  if (!active) return;
  // step n + 1 of the tile cell (x, y)
  C rxm = rho_s[w + 1][lane], rxp = rho_s[w + 1][lane + 2];
  C rym = rho_s[w][lane + 1], ryp = rho_s[w + 2][lane + 1];
  wall_ghosts<C>(p, x == 0, x == p.nx - 1, p.bc_left, p.bc_right, rho, rxm, rxp);
  wall_ghosts<C>(p, y == 0, y == p.ny - 1, p.bc_top, p.bc_bottom, rho, rym, ryp);
  const C gx = C(0.5) * (rxp - rxm), gy = C(0.5) * (ryp - rym);
  if (p.grad_out) store_grad<C>(p, 1, c, gx, gy);
  const C lb2 = mat_at<C>(p.lam, p.mat_per_cell, x, y, p.pitch) * C(1.0 / 3.0);
  Fx *= force_scale<T, C>(p);
  Fy *= force_scale<T, C>(p);
  const Moments<C> M = cell_moments<C>(f);
  C jx, jy, Sx, Sy, fs[9];
  flux_and_source<C>(M.mx, M.my, mul_rn(lb2, gx), mul_rn(lb2, gy), Fx, Fy, sponge_A<C>(p, x, y),
                     jx, jy, Sx, Sy);
  collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f), fs);
  T *fout = (T *)ph.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  const C irho = irho_at<T, C>(p, x, y);
  const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
  const U ux = u[c] + vx, uy = u[p.plane + c] + vy;
  u[c] = ux;
  u[p.plane + c] = uy;
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
  if (ph.slot_b >= 0) record_receiver<U>(p, ph.slot_b, x, y, ux, uy, vx, vy);
}

// Steps n = p.n and n + 1 of the tile (bx, by) with the density-gradient
// force, by the 32 x kL2H threads of a block (tile, rho_s: its shared
// memory).  Every thread calls it; it holds three block barriers.
// lookup: as for lam_tile_special.
template <class T, class C, class U>
__device__ __forceinline__ void step2_lam_tile(const StepParams &p, int bx, int by, T *tile,
                                               C (*rho_s)[kL2RW], bool lookup = true) {
  const Phase2 ph = phase2(p);
  const int x0 = bx * kL2Cols, y0 = by * kL2Rows;
  if (lam_tile_special(p, x0, y0, ph.slot_a, lookup)) {
    lam_general<T, C, U>(p, ph, x0, y0, tile, rho_s);
    return;
  }
  lam_bulk<T, C, U>(p, ph, x0, y0, tile, rho_s);
}

// Steps n = p.n and n + 1 from p.fin to p.fout with the density-gradient
// force, one block of 32 x kL2H threads per 28 x kL2Rows tile (the tiles in
// the order of p.tiles2l).
template <class T, class C, class U>
__global__ void __launch_bounds__(32 * kL2H, LBM_STEP2L_MIN_BLOCKS)
    step2_lam_kernel(const StepParams p) {
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  __shared__ __align__(16) T tile[l2_buf<T>()];
  __shared__ C rho_s[kL2RH][kL2RW];
  const int2 t = tile_of_block(p.tiles2l, p.tiles2l_first, gridDim.x, blockIdx.x, p.reverse);
  // the tiles after the list's first part are out of every source's and
  // receiver's reach (the edge and seam tests stay)
  step2_lam_tile<T, C, U>(p, t.x, t.y, tile, rho_s, (int)blockIdx.x < p.tiles2l_first);
}

inline dim3 step2_lam_grid(int nx, int ny) {
  return dim3(((nx + kL2Cols - 1) / kL2Cols) * ((ny + kL2Rows - 1) / kL2Rows), 1, 1);
}
inline dim3 step2_lam_block() { return dim3(32, kL2H, 1); }

// Launch entry points, one translation unit per storage type.
void launch_step2_lam_f64(const StepParams &p, cudaStream_t s);
void launch_step2_lam_f32(const StepParams &p, bool u64, cudaStream_t s);
void launch_step2_lam_16(const StepParams &p, bool bf16, bool u64, cudaStream_t s);

}  // namespace lbm
