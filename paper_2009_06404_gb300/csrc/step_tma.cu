// TMA-staged step kernel (sm_103a) for FP32 and 16-bit population storage.
//
// Persistent CTAs walk the grid in tiles of 128 x TH cells.  For each tile
// one 3-D tensor copy (cp.async.bulk.tensor) brings the nine population planes
// of the previous step into shared memory, with a halo of H rows above and
// below and 16 bytes left and right (TMA boxes must start on 16-byte x
// boundaries, so the +-1 x shifts of the pull are taken from the halo), and a
// second copy brings the displacement.  An mbarrier per stage tracks the
// bytes; three stages keep two tiles in flight while one is computed.  Cells
// within H of an edge (walls, periodic seams) take the general path of
// lbm_kernels.cuh with plain global loads; all others pull from shared memory.
// With a density gradient (H = 2) the streamed density of the tile and a
// one-cell ring is first built in shared memory (Eq. 10 needs it).
//
// Every wait on an mbarrier is bounded (about one second of clock); on
// expiry the kernel sets bit 1 of the error word (LBM_ERR_TIMEOUT), waits a
// bounded time for its own copies in flight and returns.
#include <cuda.h>

#include "lbm_kernels.cuh"
#include "step_tma.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <class T, class U, int TH, int H>
struct TileGeom;

// Offset of plane i, tile row r (0 = first halo row) in a stage: the smem
// tile keeps the order of the global layout ([row][plane] when the rows of
// the nine planes are interleaved, [plane][row] otherwise).
template <class G>
__device__ __forceinline__ int sidx(int inter, int i, int r) {
  return (inter ? (r * 9 + i) : (i * G::kRows + r)) * G::kRowLen;
}

template <class T, class U, int TH, int H>
struct TileGeom {
  static constexpr int kHalo = 16 / (int)sizeof(T);  // x halo: one 16-byte unit
  static constexpr int kRowLen = kTileW + 2 * kHalo; // smem row of one plane
  static constexpr int kRows = TH + 2 * H;
  static constexpr int kFBytes = 9 * kRows * kRowLen * (int)sizeof(T);
  static constexpr int kUBytes = 2 * TH * kTileW * (int)sizeof(U);
  static constexpr int kFBytesAl = (kFBytes + 1023) / 1024 * 1024;
  static constexpr int kUBytesAl = (kUBytes + 1023) / 1024 * 1024;
  static constexpr int kStage = kFBytesAl + kUBytesAl;
  static constexpr int kRhoLen = kTileW + 2;          // density ring row
  static constexpr int kRhoBytes = H == 2 ? (TH + 2) * kRhoLen * 4 : 0;
};

}  // namespace

// Bits of the first 32 sources whose disk may reach the tile
// [x0, x0 + 128) x [y0, y0 + th) (integer test, minimum image on periodic
// axes).  Called by all 32 lanes of a warp; every lane gets the same mask.
__device__ __forceinline__ unsigned tile_source_mask(const StepParams &p, int x0, int y0, int th) {
  const int lane = threadIdx.x & 31;
  bool hit = false;
  if (lane < p.nsrc) {
    const SourceDev &q = p.src[lane];
    int dx = x0 + kTileW / 2 - q.xc, dy = y0 + th / 2 - q.yc;
    if (p.bc_left == BC_PERIODIC) {
      if (dx > p.nx / 2) dx -= p.nx;
      else if (dx < -(p.nx / 2)) dx += p.nx;
    }
    if (p.bc_top == BC_PERIODIC) {
      if (dy > p.ny / 2) dy -= p.ny;
      else if (dy < -(p.ny / 2)) dy += p.ny;
    }
    hit = abs(dx) <= q.rb + kTileW / 2 + 1 && abs(dy) <= q.rb + th / 2 + 1;
  }
  return __ballot_sync(0xffffffffu, hit);
}

// Whether any receiver lies in the tile (its 2 x 2 receiver tiles of 64 x 4
// cells; x0 is a multiple of 128 and y0 of 8).  Warp-wide, same on all lanes.
__device__ __forceinline__ bool tile_has_receiver(const StepParams &p, int x0, int y0) {
  const int lane = threadIdx.x & 31;
  bool any = false;
  if (lane < 4) {
    const int ty = y0 / kRecTileY + (lane >> 1), tx = x0 / kRecTileX + (lane & 1);
    if (ty * kRecTileY < p.ny && tx * kRecTileX < p.nx) {
      const int t = ty * p.rec_tiles_x + tx;
      any = p.rec_tile_ptr[t + 1] > p.rec_tile_ptr[t];
    }
  }
  return __ballot_sync(0xffffffffu, any) != 0u;
}

#ifndef LBM_TMA_MIN_BLOCKS
#define LBM_TMA_MIN_BLOCKS 3
#endif

template <class T, class U, bool LAM, int TH, int STAGES>
__global__ void __launch_bounds__(kTmaThreads, LBM_TMA_MIN_BLOCKS)
    step_tma_kernel(const StepParams p, const __grid_constant__ CUtensorMap fmap,
                    const __grid_constant__ CUtensorMap umap, int ntx, int nty) {
  constexpr int H = LAM ? 2 : 1;
  constexpr int kWarpsPerRow = kTmaThreads / 32 / TH;
  constexpr int kCellsPerLane = kTileW / 32 / kWarpsPerRow;
  using G = TileGeom<T, U, TH, H>;
  static_assert(kWarpsPerRow * TH * 32 == kTmaThreads, "whole warps per tile row");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // stages start on 1024-byte boundaries (the launch reserves 1 KB of slack)
  unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint64_t *bar = (uint64_t *)(smem + STAGES * G::kStage + G::kRhoBytes);
  float *rho_s = (float *)(smem + STAGES * G::kStage);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int row = w / kWarpsPerRow, seg = w % kWarpsPerRow;
  const int ntiles = ntx * nty;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](int t, int s) {
    const int x0 = (t % ntx) * kTileW, y0 = (t / ntx) * TH;
    unsigned char *st = smem + s * G::kStage;
    mbar_expect_tx(&bar[s], (uint32_t)(G::kFBytes + G::kUBytes));
    if (p.finter)
      tma_load_3d(st, &fmap, x0 - G::kHalo, 0, y0 - H, &bar[s]);
    else
      tma_load_3d(st, &fmap, x0 - G::kHalo, y0 - H, 0, &bar[s]);
    tma_load_3d(st + G::kFBytesAl, &umap, x0, y0, 0, &bar[s]);
  };

  if (tid == 0) {
    for (int j = 0; j < STAGES; ++j) {
      const int t = blockIdx.x + j * gridDim.x;
      if (t < ntiles) issue(t, j);
    }
  }

  const int m = LAM ? 2 : 1;  // cells closer than m to an edge take the general path
  const float om = p.omega_f, fc = p.fcoef_f;
  int iter = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++iter) {
    const int s = iter % STAGES;
    const bool ok = mbar_wait(&bar[s], (uint32_t)((iter / STAGES) & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.err, 2);
        // let this CTA's copies still in flight land before it exits
        for (int j = 1; j < STAGES; ++j) {
          const int it2 = iter + j;
          if (blockIdx.x + it2 * gridDim.x < ntiles)
            mbar_wait(&bar[it2 % STAGES], (uint32_t)((it2 / STAGES) & 1));
        }
      }
      return;
    }
    const T *sf = (const T *)(smem + s * G::kStage);
    const U *su = (const U *)(smem + s * G::kStage + G::kFBytesAl);
    const int x0 = (t % ntx) * kTileW, y0 = (t / ntx) * TH;

    // what this tile needs (uniform across the CTA)
    const bool edge = x0 < m || x0 + kTileW > p.nx - m || y0 < m || y0 + TH > p.ny - m;
    const bool spg = x0 < p.sp_left || x0 + kTileW > p.nx - p.sp_right || y0 < p.sp_top ||
                     y0 + TH > p.ny - p.sp_bottom;
    const unsigned smask =
        p.nsrc == 0 ? 0u : (p.nsrc <= 32 ? tile_source_mask(p, x0, y0, TH) : 0xffffffffu);
    const bool rec = p.trace_slot >= 0 && tile_has_receiver(p, x0, y0);

    if (LAM) {
      // streamed density of the tile plus a one-cell ring (Eq. 10 needs it)
      for (int k = tid; k < (TH + 2) * G::kRhoLen; k += kTmaThreads) {
        const int r = k / G::kRhoLen - 1, c = k % G::kRhoLen - 1;
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
          acc += ld<T, float>(sf + sidx<G>(p.finter, i, r + H - cyd(i)) + (c + G::kHalo - cxd(i)));
        rho_s[k] = acc;
      }
      __syncthreads();
    }

    const int y = y0 + row;
    const int yc = y < p.ny ? y : p.ny - 1;
    const float lam_row = (LAM && !p.mat_per_cell) ? ((const float *)p.lam)[yc] : 0.f;
    const float irho_row = p.mat_per_cell ? 0.f : ((const float *)p.irho)[yc];
#pragma unroll
    for (int k = 0; k < kCellsPerLane; ++k) {
      const int lx = seg * (kTileW / kWarpsPerRow) + lane + 32 * k;
      const int x = x0 + lx;
      const int xc = x < p.nx ? x : p.nx - 1;
      float Fx = 0.f, Fy = 0.f;
      if (smask) {
        if (p.nsrc <= 32) {
          unsigned mk = smask;
          while (mk) {
            const int b = __ffs(mk) - 1;
            mk &= mk - 1;
            const float2 F = source_term(p.src[b], xc, yc, p.n, p.nx, p.ny,
                                         p.bc_left == BC_PERIODIC, p.bc_top == BC_PERIODIC,
                                         0.0f);
            Fx += F.x;
            Fy += F.y;
          }
        } else {
          body_force<float>(p, xc, yc, Fx, Fy);  // whole warp: one row, 32 consecutive x
        }
      }
      if (edge && !(xc >= m && xc < p.nx - m && yc >= m && yc < p.ny - m)) {
        boundary_cell<T, float, U, LAM, 0>(p, Fx, Fy, x, y, xc, yc, x < p.nx && y < p.ny);
        continue;
      }
      // interior cell: everything from shared memory
      float f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i)
        f[i] = ld<T, float>(sf + sidx<G>(p.finter, i, row + H - cyd(i)) + (lx + G::kHalo - cxd(i)));
      const Moments<float> M = cell_moments<float>(f);
      const int c = y * p.pitch + x;
      float Gx = 0.f, Gy = 0.f;
      if (LAM) {
        const float *rr = rho_s + (row + 1) * G::kRhoLen + (lx + 1);
        const float lam = p.mat_per_cell ? ((const float *)p.lam)[c] : lam_row;
        // elastic force Lambda b^2 grad rho with the centred difference (Eqs. 9-10)
        const float lb2 = lam * (1.0f / 3.0f);
        Gx = mul_rn(lb2, 0.5f * (rr[1] - rr[-1]));
        Gy = mul_rn(lb2, 0.5f * (rr[G::kRhoLen] - rr[-G::kRhoLen]));
      }
      const float A = spg ? sponge_A<float>(p, x, y) : 0.f;
      float jx, jy, Sx, Sy;
      flux_and_source<float>(M.mx, M.my, Gx, Gy, Fx, Fy, A, jx, jy, Sx, Sy);
      float fs[9];
      collide_cell<float>(M, jx, jy, Sx, Sy, om, fc, fs);
      T *fout = (T *)p.fout + (y * p.frow + x);
#pragma unroll
      for (int i = 0; i < 9; ++i) st<T, float>(fout + i * p.fplane, fs[i]);
      const float irho = p.mat_per_cell ? ((const float *)p.irho)[c] : irho_row;
      const U vx = U(mul_rn(jx, irho)), vy = U(mul_rn(jy, irho));
      const U ux = su[row * kTileW + lx] + vx, uy = su[(TH + row) * kTileW + lx] + vy;
      U *u = (U *)p.u;
      u[c] = ux;
      u[p.plane + c] = uy;
      if (!((M.rho + jx + jy) * 0.f == 0.f)) atomicOr(p.err, 1);
      if (rec) record_receiver<U>(p, p.trace_slot, x, y, ux, uy, vx, vy);
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0) {
      const int tn = t + STAGES * gridDim.x;
      if (tn < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(tn, s);
      }
    }
  }
}

// Three stages where they fit in 227 KB of shared memory, else two.
template <class T, class U, bool LAM>
constexpr int stages_of() {
  using G = TileGeom<T, U, kTileH, LAM ? 2 : 1>;
  return (kTmaStages * G::kStage + G::kRhoBytes + kTmaStages * 8 + 1024 <= 227 * 1024)
             ? kTmaStages
             : 2;
}

template <class T, class U, bool LAM>
static int smem_bytes() {
  constexpr int H = LAM ? 2 : 1;
  using G = TileGeom<T, U, kTileH, H>;
  constexpr int S = stages_of<T, U, LAM>();
  return S * G::kStage + G::kRhoBytes + S * 8 + 1024;
}

template <class T, class U, bool LAM>
static int ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, step_tma_kernel<T, U, LAM, kTileH, stages_of<T, U, LAM>()>, kTmaThreads,
          smem_bytes<T, U, LAM>()) != cudaSuccess)
    n = 1;
  return n < 1 ? 1 : n;
}

template <class T, class U, bool LAM>
static cudaError_t launch_one(const StepParams &p, const TmaMaps &maps, int cur, int nsm,
                              cudaStream_t s) {
  auto kern = step_tma_kernel<T, U, LAM, kTileH, stages_of<T, U, LAM>()>;
  const int bytes = smem_bytes<T, U, LAM>();
  static int per_sm = 0;  // resident CTAs per SM, queried once per variant
  if (per_sm == 0) per_sm = ctas_per_sm<T, U, LAM>();
  const int ntx = (p.nx + kTileW - 1) / kTileW, nty = (p.ny + kTileH - 1) / kTileH;
  const int ntiles = ntx * nty;
  const int grid = ntiles < nsm * per_sm ? ntiles : nsm * per_sm;
  kern<<<grid, kTmaThreads, bytes, s>>>(p, maps.f[cur][LAM ? 1 : 0], maps.u, ntx, nty);
  return cudaGetLastError();
}

cudaError_t launch_step_tma(const StepParams &p, const TmaMaps &maps, int cur, int storage,
                            bool u64, bool lam, int nsm, cudaStream_t s) {
  if (storage == 1) {  // FP32
    if (u64) return lam ? launch_one<float, double, true>(p, maps, cur, nsm, s)
                        : launch_one<float, double, false>(p, maps, cur, nsm, s);
    return lam ? launch_one<float, float, true>(p, maps, cur, nsm, s)
               : launch_one<float, float, false>(p, maps, cur, nsm, s);
  }
  return cudaErrorNotSupported;
}

template <class T, class U, bool LAM>
static cudaError_t prepare_one() {
  return cudaFuncSetAttribute(step_tma_kernel<T, U, LAM, kTileH, stages_of<T, U, LAM>()>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes<T, U, LAM>());
}

cudaError_t tma_prepare(int storage, bool u64) {
  if (storage != 1) return cudaErrorNotSupported;
  cudaError_t e = u64 ? prepare_one<float, double, false>() : prepare_one<float, float, false>();
  if (e == cudaSuccess)
    e = u64 ? prepare_one<float, double, true>() : prepare_one<float, float, true>();
  return e;
}

int tma_ctas_per_sm(int storage, bool u64, bool lam) {
  if (storage == 1) {
    if (u64) return lam ? ctas_per_sm<float, double, true>() : ctas_per_sm<float, double, false>();
    return lam ? ctas_per_sm<float, float, true>() : ctas_per_sm<float, float, false>();
  }
  return 0;
}

int tma_stages(int storage, bool u64, bool lam) {
  if (storage == 1) {
    if (u64) return lam ? stages_of<float, double, true>() : stages_of<float, double, false>();
    return lam ? stages_of<float, float, true>() : stages_of<float, float, false>();
  }
  return 0;
}

int tma_smem_bytes(int storage, bool u64, bool lam) {
  if (storage == 1) {
    if (u64) return lam ? smem_bytes<float, double, true>() : smem_bytes<float, double, false>();
    return lam ? smem_bytes<float, float, true>() : smem_bytes<float, float, false>();
  }
  return 0;
}

}  // namespace lbm
