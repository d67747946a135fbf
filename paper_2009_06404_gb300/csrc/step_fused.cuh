// Two steps of the elastic-solid D2Q9 LBM per launch (temporal blocking of
// the step of lbm_kernels.cuh, for grids without the density-gradient force).
//
// A block owns an output tile of kF2Cols x kF2Rows cells.  Step n is
// computed on the tile's window, the tile widened by one cell on every side
// (kF2W x kF2H cells), from the populations of step n - 1 in global memory;
// its post-collision populations go to shared memory, not to HBM.  Step n + 1 of
// the tile's cells then pulls from shared memory and writes the populations
// and the displacement once.  Per two steps each population crosses HBM
// once each way instead of twice; the window's halo (the neighbour tiles'
// cells) is recomputed, and its loads are mostly L2 hits.
//
// Every cell update uses the arithmetic of the one-step kernel (the same
// moments, flux, source, collision and wall functions, and 16-bit rounding
// of the intermediate populations in shared memory), so two-step and
// one-step launches give bit-identical states, traces and displacements.
//
// Non-finite values are tested in step n + 1 only: a non-finite population
// of step n reaches the step n + 1 moments of some tile cell in the same
// launch (its own cell's rest population if the density is non-finite, the
// neighbours' otherwise; a window's halo cell is also a tile cell of the
// block that owns it, which recomputes it the same way).
//
// Warps (LBM_STEP2_COLS = 30, the default): a tile is 30 columns wide, so a
// window row is 32 cells and each of the kF2H warps computes one window row
// in step n; in step n + 1 lanes 1..30 of the warps of the tile's rows
// update their own cells.  LBM_STEP2_COLS = 32: 32-wide tiles, kF2H warps
// for the 32 columns above the tile's and one more warp for the two side
// columns (2 kF2H = 32 cells).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

#ifndef LBM_STEP2_COLS
#define LBM_STEP2_COLS 30
#endif
#ifndef LBM_STEP2_ROWS
#define LBM_STEP2_ROWS 14
#endif
constexpr int kF2Cols = LBM_STEP2_COLS;             // columns of a block's output tile
constexpr int kF2Rows = LBM_STEP2_ROWS;             // rows of a block's output tile
constexpr bool kF2Side = kF2Cols == 32;             // a separate warp for the side columns
constexpr int kF2H = kF2Rows + 2;                   // rows of its window
constexpr int kF2W = kF2Cols + 2;                   // columns of its window
constexpr int kF2Warps = kF2H + (kF2Side ? 1 : 0);  // threads per block: 32 x kF2Warps
static_assert(kF2Cols == 30 || kF2Cols == 32, "tiles are 30 or 32 columns wide");
static_assert(!kF2Side || 2 * kF2H == 32, "the two side columns of the window fill one warp");
static_assert(kF2Warps <= 32, "at most 1024 threads per block");

// Resident blocks per SM the register budget is set for.
#ifndef LBM_STEP2_MIN_BLOCKS
#define LBM_STEP2_MIN_BLOCKS (2048 / (32 * kF2Warps))
#endif

// The window in shared memory, [9][kF2H][kF2W]; element (0, 0) is grid cell
// (ox, oy) = (x0 - 1, y0 - 1).  Cells beyond a periodic seam hold the
// image's populations at their unwrapped coordinates.
template <class T>
struct TilePops {
  const T *f;
  int ox, oy;
  static constexpr bool kWrap = false;
  __device__ __forceinline__ const T *at(int i, int x, int y) const {
    return f + ((i * kF2H + (y - oy)) * kF2W + (x - ox));
  }
  template <class C>
  __device__ __forceinline__ C load(int i, int x, int y) const {
    return ld<T, C>(at(i, x, y));
  }
};


// Staged region of a Lambda = 0 general tile: the tile widened by two cells
// (the window's pulls), aliasing the window buffer until step n's stores.
template <class T>
constexpr int f2_stage_w() { return stage_width<T>(kF2Cols, 2); }
constexpr int kF2SH = kF2Rows + 4;
template <class T>
constexpr int f2_buf() {
  return stages<T>() && 9 * kF2SH * f2_stage_w<T>() > 9 * kF2H * kF2W
             ? 9 * kF2SH * f2_stage_w<T>()
             : 9 * kF2H * kF2W;
}

// The two steps of a launch: steps n = p.n and n + 1 read p.fin and write
// p.fout; they record into trace slots trace_slot and trace_slot + 1 while
// those exist (below trace_end).
struct Phase2 {
  const void *fin;
  void *fout;
  long long n;
  int slot_a, slot_b;
};
__device__ __forceinline__ Phase2 phase2(const StepParams &p) {
  Phase2 q;
  q.fin = p.fin;
  q.fout = p.fout;
  q.n = p.n;
  const int s = p.trace_slot;
  q.slot_a = (s >= 0 && s < p.trace_end) ? s : -1;
  q.slot_b = (s >= 0 && s + 1 < p.trace_end) ? s + 1 : -1;
  return q;
}

// Window cell of this thread: column ex, row ey; core: the cell is one of
// the tile's.
__device__ __forceinline__ void window_cell(int lane, int w, int &ex, int &ey, bool &core) {
  if (!kF2Side) {
    ex = lane;
    ey = w;
    core = w >= 1 && w <= kF2Rows && lane >= 1 && lane <= kF2Cols;
  } else if (w < kF2H) {
    ex = lane + 1;
    ey = w;
    core = w >= 1 && w <= kF2Rows;
  } else {
    ex = (lane & 1) ? kF2W - 1 : 0;
    ey = lane >> 1;
    core = false;
  }
}

// Origin along one axis of the cells a tile computes.  A partial tile (the
// last along an axis of n cells that is not a multiple of the tile size T)
// on a periodic axis at least two tiles long computes the full tile that
// ends at the seam, n - T, and stores only its own cells (from t0 on): the
// cells below t0 are the previous tile's, computed again the same way.
__device__ __forceinline__ int tile_origin(int t0, int T, int n, bool periodic) {
  return periodic && t0 + T > n && n >= 2 * T ? n - T : t0;
}

// Kinds of tile (origin x0, y0), from its position only (every lane of
// every warp gets the same answer).  kTileGeneral: the general rules -- a
// non-periodic edge within two cells (step n reaches one cell beyond the
// tile and pulls from one more), a partial tile on a non-periodic axis, or
// a periodic axis shorter than two tiles.  Otherwise any of: kTileWrap, the
// window or its pulls cross a periodic seam (every partial tile on a
// periodic axis, whose cells are computed from tile_origin); kTileSrc, a
// source reaches the window; kTileRec, a receiver is among the cells
// computed (when recording).  0: the plain bulk update.  lookup = false
// skips the source and receiver tests (a tile the host's launch order
// places after every tile a source or receiver can reach).
enum { kTileGeneral = 1, kTileWrap = 2, kTileSrc = 4, kTileRec = 8 };

__device__ __forceinline__ int tile_kind(const StepParams &p, int x0, int y0, int slot_a,
                                         bool lookup = true) {
  constexpr int W = kF2Cols, H = kF2Rows;
  int kind = 0;
  if (p.bc_left == BC_PERIODIC) {
    if (p.nx < 2 * W) return kTileGeneral;
    if (x0 + W > p.nx) x0 = p.nx - W;
    if (x0 < 2 || x0 + W > p.nx - 2) kind |= kTileWrap;
  } else if (x0 < 2 || x0 + W > p.nx - 2) {
    return kTileGeneral;
  }
  if (p.bc_top == BC_PERIODIC) {
    if (p.ny < 2 * H) return kTileGeneral;
    if (y0 + H > p.ny) y0 = p.ny - H;
    if (y0 < 2 || y0 + H > p.ny - 2) kind |= kTileWrap;
  } else if (y0 < 2 || y0 + H > p.ny - 2) {
    return kTileGeneral;
  }
  if (!lookup) return kind;
  const bool near_src = p.nsrc > 0 && x0 - 1 <= p.src_x1 && x0 + W >= p.src_x0 &&
                        y0 - 1 <= p.src_y1 && y0 + H >= p.src_y0;
  const bool near_rec = slot_a >= 0 && x0 <= p.rec_x1 && x0 + W - 1 >= p.rec_x0 &&
                        y0 <= p.rec_y1 && y0 + H - 1 >= p.rec_y0;
  if (!near_src && !near_rec) return kind;
  const int lane = threadIdx.x & 31;
  bool hit_src = near_src && p.nsrc > 32;
  if (near_src && p.nsrc <= 32 && lane < p.nsrc) {
    // window cells lie within W/2 + 1 columns and H/2 + 1 rows of the centre
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
    hit_src = abs(dx) <= qb.z + W / 2 + 2 && abs(dy) <= qb.z + H / 2 + 2;
  }
  bool hit_rec = false;
  if (near_rec) {
    // receiver tiles (kRecTileX x kRecTileY) touched by the tile's cells
    const int tx0 = x0 / kRecTileX, tx1 = min((x0 + W - 1) / kRecTileX, p.rec_tiles_x - 1);
    const int ty0 = y0 / kRecTileY, ty1 = min((y0 + H - 1) / kRecTileY, (p.ny - 1) / kRecTileY);
    const int nty = ty1 - ty0 + 1;
    for (int j = lane; j < (tx1 - tx0 + 1) * nty; j += 32) {
      const int t = (ty0 + j % nty) * p.rec_tiles_x + tx0 + j / nty;
      hit_rec |= p.rec_tile_ptr[t + 1] > p.rec_tile_ptr[t];
    }
  }
  if (__ballot_sync(0xffffffffu, hit_src)) kind |= kTileSrc;
  if (__ballot_sync(0xffffffffu, hit_rec)) kind |= kTileRec;
  return kind;
}

// Blocks within reach of a wall, seam, source or receiver: every cell runs
// the general rules.  Step n is evaluated at each window cell (cells beyond
// a non-periodic edge are never read: the wall rules replace them), its
// pulls read from the input populations of the tile widened by two cells,
// staged in the window buffer by one pass of copies (FP64: per-cell global
// pulls); step n + 1 at the tile's cells.  Out of line so the bulk path
// carries none of its registers.  Every thread calls it (three barriers:
// inputs staged, staged region read, window written).
//
// Register budget: the body force of each step is summed (out of line, in
// the sources' bounding box) before that step's pulls, and the displacement
// after step n goes through global memory (u + v^n stored, reloaded for
// + v^{n+1}: the same two roundings).
template <class T, class C, class U>
__device__ __noinline__ void step2_general(const StepParams &p, int x0, int y0, T *tile) {
  // window cells lie within kF2Cols/2 + 1 columns and kF2Rows/2 + 1 rows of
  // the centre
  const unsigned smask = source_mask(p, x0 + kF2Cols / 2, y0 + kF2Rows / 2, kF2Cols / 2 + 2,
                                     kF2Rows / 2 + 2);
  // the input populations of the window's pulls, staged in the window
  // buffer (dead until step n's stores, after the second barrier)
  constexpr int SW = f2_stage_w<T>();
  const int sox = stage_origin<T>(x0, 2);
  if constexpr (stages<T>()) {
    stage_rows<T, SW, kF2SH, 32 * kF2Warps>(p, (const T *)phase2(p).fin, sox, y0 - 2, tile);
    stage_wait();
  }
  __syncthreads();
  C fs[9];
  bool stored = false;
  {
    int ex, ey;
    bool core;
    window_cell(threadIdx.x, threadIdx.y, ex, ey, core);
    const int x = x0 - 1 + ex, y = y0 - 1 + ey;
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
    if (valid) {
      const Phase2 ph = phase2(p);
      C Fx, Fy;
      body_force_cell<C>(p, wx, wy, ph.n, Fx, Fy, smask);
      C f[9];
      if constexpr (stages<T>()) {
        pull_staged<T, C>(p, StagePops<T, SW, kF2SH>{tile, sox, y0 - 2}, x, y, f);
      } else {
        gather<T, C>(p, (const T *)ph.fin, wx, wy, f);
      }
      const Moments<C> M = cell_moments<C>(f);
      Fx *= force_scale<T, C>(p);
      Fy *= force_scale<T, C>(p);
      C jx, jy, Sx, Sy;
      flux_and_source<C>(M.mx, M.my, C(0), C(0), Fx, Fy, sponge_A<C>(p, wx, wy), jx, jy, Sx, Sy);
      collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f),
                      fs);
      stored = true;
      if (core && x < p.nx && y < p.ny) {
        const C irho = irho_at<T, C>(p, x, y);
        const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
        U *u = (U *)p.u;
        const int c = y * p.pitch + x;
        const U ux = __ldcg(u + c) + vx, uy = __ldcg(u + p.plane + c) + vy;
        u[c] = ux;
        u[p.plane + c] = uy;
        if (ph.slot_a >= 0) record_receiver<U>(p, ph.slot_a, x, y, ux, uy, vx, vy);
      }
    }
  }
  __syncthreads();  // every read of the staged region is done
  int ex, ey;
  bool core;
  window_cell(threadIdx.x, threadIdx.y, ex, ey, core);
  if (stored) {
#pragma unroll
    for (int i = 0; i < 9; ++i) st<T, C>(tile + ((i * kF2H + ey) * kF2W + ex), fs[i]);
  }
  __syncthreads();
  const int x = x0 - 1 + ex, y = y0 - 1 + ey;
  if (!(core && x < p.nx && y < p.ny)) return;
  // step n + 1 of the tile's cell (x, y)
  const Phase2 ph = phase2(p);
  C Fx, Fy;
  body_force_cell<C>(p, x, y, ph.n + 1, Fx, Fy, smask);
  C f[9];
  if (off_walls(p, x, y)) {
    // the window holds the periodic images at unwrapped coordinates
    const TilePops<T> tp{tile, x0 - 1, y0 - 1};
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ld<T, C>(tp.at(i, x - cxd(i), y - cyd(i)));
  } else {
    pull_cell<T, C>(p, TilePops<T>{tile, x0 - 1, y0 - 1}, x, y, f);
  }
  const Moments<C> M = cell_moments<C>(f);
  Fx *= force_scale<T, C>(p);
  Fy *= force_scale<T, C>(p);
  C jx, jy, Sx, Sy;
  flux_and_source<C>(M.mx, M.my, C(0), C(0), Fx, Fy, sponge_A<C>(p, x, y), jx, jy, Sx, Sy);
  collide_cell<C>(M, jx, jy, Sx, Sy, par<C>(p.omega, p.omega_f), par<C>(p.fcoef, p.fcoef_f), fs);
  T *fout = (T *)ph.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  const C irho = irho_at<T, C>(p, x, y);
  const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
  U *u = (U *)p.u;
  const int c = y * p.pitch + x;
  const U ux = u[c] + vx, uy = u[p.plane + c] + vy;
  u[c] = ux;
  u[p.plane + c] = uy;
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
  if (ph.slot_b >= 0) record_receiver<U>(p, ph.slot_b, x, y, ux, uy, vx, vy);
}

// A coordinate one period back into the grid (at most one period out).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Tiles without a non-periodic edge nearby whose window crosses a periodic
// seam, or that a source reaches, or that hold receivers: the bulk update
// with the window's cells and pulls wrapped, the body force where a source
// reaches, and the receivers recorded.  Out of line, so the plain bulk path
// carries none of its registers.  Every thread calls it (one barrier).
// (x0, y0): the cells computed; only those from (xs, ys) on are stored (a
// partial tile on a periodic axis, tile_origin).
template <class T, class C, class U, bool SRC>
__device__ __noinline__ void step2_featured(const StepParams &p, int x0, int y0, int xs, int ys,
                                            int kind, T *tile) {
  const Phase2 ph = phase2(p);
  const int lane = threadIdx.x, w = threadIdx.y;
  int ex, ey;
  bool core;
  window_cell(lane, w, ex, ey, core);
  const int x = x0 - 1 + ex, y = y0 - 1 + ey;  // tile cells: inside the grid
  core = core && x >= xs && y >= ys;           // the cells this tile stores
  const int wx = wrap1(x, p.nx), wy = wrap1(y, p.ny);
  constexpr bool src = SRC;  // kind & kTileSrc
  const bool spg = (kind & kTileWrap) || x0 - 1 < p.sp_left || x0 + kF2Cols + 1 > p.nx - p.sp_right ||
                   y0 - 1 < p.sp_top || y0 + kF2Rows + 1 > p.ny - p.sp_bottom;
  const C om = par<C>(p.omega, p.omega_f), fc = par<C>(p.fcoef, p.fcoef_f);
  // the body force of step n first (an out-of-line sum inside the sources'
  // bounding box), before the pulls fill the registers
  const unsigned smask = src ? source_mask(p, x0 + kF2Cols / 2, y0 + kF2Rows / 2,
                                           kF2Cols / 2 + 2, kF2Rows / 2 + 2)
                             : 0u;
  C Fx = C(0), Fy = C(0);
  if (src) body_force_cell<C>(p, wx, wy, ph.n, Fx, Fy, smask);
  // step n on the window
  const T *fin = (const T *)ph.fin;
  C f[9];
  {
    const int xs[3] = {wrap1(wx - 1, p.nx), wx, wrap1(wx + 1, p.nx)};
    const int ys[3] = {wrap1(wy - 1, p.ny), wy, wrap1(wy + 1, p.ny)};
#pragma unroll
    for (int i = 0; i < 9; ++i)
      f[i] = ldp<T, C>(fin + (i * p.fplane + (ys[1 - cyd(i)] * p.frow + xs[1 - cxd(i)])), p);
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
  {
    const Moments<C> M = cell_moments<C>(f);
    C jx, jy, fs[9];
    if (src) {  // (a compile-time branch)
      C Sx, Sy;
      Fx *= force_scale<T, C>(p);
      Fy *= force_scale<T, C>(p);
      flux_and_source<C>(M.mx, M.my, C(0), C(0), Fx, Fy, sponge_A<C>(p, wx, wy), jx, jy, Sx, Sy);
      collide_cell<C>(M, jx, jy, Sx, Sy, om, fc, fs);
    } else {
      bulk_collide<C>(p, M, C(0), C(0), spg, wx, wy, fs, jx, jy);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) st<T, C>(tile + ((i * kF2H + ey) * kF2W + ex), fs[i]);
    if (core) {
      const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
      ux += vx;
      uy += vy;
      if ((kind & kTileRec) && ph.slot_a >= 0)
        record_receiver<U>(p, ph.slot_a, x, y, ux, uy, vx, vy);
    }
  }
  __syncthreads();
  if (!core) return;
  if (src) body_force_cell<C>(p, x, y, ph.n + 1, Fx, Fy, smask);
  // step n + 1 of the tile's cell, pulled from the window
#pragma unroll
  for (int i = 0; i < 9; ++i)
    f[i] = ld<T, C>(tile + ((i * kF2H + ey - cyd(i)) * kF2W + ex - cxd(i)));
  const Moments<C> M = cell_moments<C>(f);
  C jx, jy, fs[9];
  if (src) {
    C Sx, Sy;
    Fx *= force_scale<T, C>(p);
    Fy *= force_scale<T, C>(p);
    flux_and_source<C>(M.mx, M.my, C(0), C(0), Fx, Fy, sponge_A<C>(p, x, y), jx, jy, Sx, Sy);
    collide_cell<C>(M, jx, jy, Sx, Sy, om, fc, fs);
  } else {
    bulk_collide<C>(p, M, C(0), C(0), spg, x, y, fs, jx, jy);
  }
  T *fout = (T *)ph.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
  ux += vx;
  uy += vy;
  u[c] = ux;
  u[p.plane + c] = uy;
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
  if ((kind & kTileRec) && ph.slot_b >= 0)
    record_receiver<U>(p, ph.slot_b, x, y, ux, uy, vx, vy);
}

// Steps p.n and p.n + 1 of the tile (bx, by), by the 32 x kF2Warps threads
// of the block (tile: the block's shared-memory window).  Every thread
// calls it; it holds one block barrier (three on the general path).
// lookup: as for tile_kind.
template <class T, class C, class U>
__device__ __forceinline__ void step2_tile(const StepParams &p, int bx, int by, T *tile,
                                           bool lookup = true) {
  const Phase2 ph = phase2(p);
  const int x0 = bx * kF2Cols, y0 = by * kF2Rows;
  const int kind = tile_kind(p, x0, y0, ph.slot_a, lookup);
  if (kind & kTileGeneral) {
    step2_general<T, C, U>(p, x0, y0, tile);
    return;
  }
  if (kind) {
    const int cx = tile_origin(x0, kF2Cols, p.nx, p.bc_left == BC_PERIODIC);
    const int cy = tile_origin(y0, kF2Rows, p.ny, p.bc_top == BC_PERIODIC);
    if (kind & kTileSrc) step2_featured<T, C, U, true>(p, cx, cy, x0, y0, kind, tile);
    else step2_featured<T, C, U, false>(p, cx, cy, x0, y0, kind, tile);
    return;
  }
  const int lane = threadIdx.x, w = threadIdx.y;
  int ex, ey;
  bool core;
  window_cell(lane, w, ex, ey, core);
  const int x = x0 - 1 + ex, y = y0 - 1 + ey;
  // step n on the window: every upstream cell is inside the grid
  const T *fin = (const T *)ph.fin;
  C f[9];
  {
    const T *b = fin + (y * p.frow + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ldp<T, C>(b + (i * p.fplane - cyd(i) * p.frow - cxd(i)), p);
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
  const bool spg = x0 - 1 < p.sp_left || x0 + kF2Cols + 1 > p.nx - p.sp_right ||
                   y0 - 1 < p.sp_top || y0 + kF2Rows + 1 > p.ny - p.sp_bottom;
  {
    const Moments<C> M = cell_moments<C>(f);
    C jx, jy, fs[9];
    bulk_collide<C>(p, M, C(0), C(0), spg, x, y, fs, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) st<T, C>(tile + ((i * kF2H + ey) * kF2W + ex), fs[i]);
    if (core) {
      ux += U(mul_rn(jx, irho));
      uy += U(mul_rn(jy, irho));
    }
  }
  __syncthreads();
  if (!core) return;
  // step n + 1 of the tile's cell, pulled from the window
#pragma unroll
  for (int i = 0; i < 9; ++i)
    f[i] = ld<T, C>(tile + ((i * kF2H + ey - cyd(i)) * kF2W + ex - cxd(i)));
  const Moments<C> M = cell_moments<C>(f);
  C jx, jy, fs[9];
  bulk_collide<C>(p, M, C(0), C(0), spg, x, y, fs, jx, jy);
  T *fout = (T *)ph.fout + (y * p.frow + x);
#pragma unroll
  for (int i = 0; i < 9; ++i) stp<T, C>(fout + i * p.fplane, fs[i], p);
  u[c] = ux + U(mul_rn(jx, irho));
  u[p.plane + c] = uy + U(mul_rn(jy, irho));
  if (!((M.rho + jx + jy) * C(0) == C(0))) atomicOr(p.err, 1);
}

// The tile of block b of a two-step launch: list[b] for the first `first`
// blocks (the tiles that take a slower path start first, so their longer
// run overlaps the bulk instead of trailing the launch), then the rest of
// the list in order, or in reverse order when `reverse` is set (alternate
// launches: the rows written last by one launch, still in L2, are the first
// the next one reads).  One block per tile (n blocks).
__device__ __forceinline__ int2 tile_of_block(const int2 *list, int first, int n, int b,
                                              int reverse) {
  if (reverse && b >= first) b = first + (n - 1 - b);
  return list[b];
}

// Steps n = p.n and n + 1 from p.fin to p.fout, one block per kF2Cols x
// kF2Rows tile (the tiles in the order of p.tiles2); blocks of 32 x
// kF2Warps threads.
template <class T, class C, class U>
__global__ void __launch_bounds__(32 * kF2Warps, LBM_STEP2_MIN_BLOCKS)
    step2_kernel(const StepParams p) {
  // the tile list is written only by host copies ordered before the
  // previous launch, so its entry is read before the wait for that launch
  const int2 t = tile_of_block(p.tiles2, p.tiles2_first, gridDim.x, blockIdx.x, p.reverse);
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  __shared__ __align__(16) T tile[f2_buf<T>()];
  // the tiles after the list's first part are out of every source's and
  // receiver's reach (the edge and seam tests stay)
  step2_tile<T, C, U>(p, t.x, t.y, tile, (int)blockIdx.x < p.tiles2_first);
}

// Launch configuration of the two-step kernel for an nx x ny grid: one
// block per tile.
inline dim3 step2_grid(int nx, int ny) {
  return dim3(((nx + kF2Cols - 1) / kF2Cols) * ((ny + kF2Rows - 1) / kF2Rows), 1, 1);
}
inline dim3 step2_block() { return dim3(32, kF2Warps, 1); }

// Launch entry points, one translation unit per storage type.
void launch_step2_f64(const StepParams &p, cudaStream_t s);
void launch_step2_f32(const StepParams &p, bool u64, cudaStream_t s);
void launch_step2_16(const StepParams &p, bool bf16, bool u64, cudaStream_t s);

}  // namespace lbm
