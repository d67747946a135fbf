// Batched step: many independent grids ("shots") advanced together.  The
// work of one launch is a flat list of tiles (shot, block column, block row);
// each tile runs the same block update as the single-grid kernels, with its
// shot's parameters staged in shared memory.  Tiles come in two kinds: one
// time step on 32 x R cells (the one-step block update), or two time steps
// on the tile of the two-step kernels (30 x 14 cells without the
// density-gradient force, 28 x 12 with it; the intermediate populations stay
// in shared memory).  Two launch forms share them: one launch per step (or
// per two steps) over all tiles, as stream launches or a CUDA graph, and a
// persistent cooperative launch that claims tiles from an atomic queue and
// separates the steps with a grid barrier.
#pragma once

#include "lbm_kernels.cuh"
#include "step2_lam.cuh"

namespace lbm {

// Step-independent parameters of one shot (buffers and step index are
// filled in per step).
struct BatchShot {
  StepParams p;
  const void *f[2];  // the two population buffers
  int lam;           // some Lambda != 0: the gradient path
  int trace_max;     // trace slots of the shot (max_steps_traced)
};

// Shot state at the start of a batched call.
struct BatchDyn {
  long long n0;  // index of the next step
  int cur0;      // buffer holding the latest post-collision state
  int traced0;   // trace slots used
};

// Device-side control block of a batch.
struct BatchHdr {
  unsigned long long queue;   // tile claims of the persistent kernel
  unsigned long long arrive;  // grid-barrier arrivals
  long long kbase;            // steps of this call done by earlier launches
  int err;                    // bit 1: a grid barrier gave up waiting
  int pad;
};

struct BatchArgs {
  const BatchShot *shots;
  const BatchDyn *dyn;
  const int4 *tiles;  // (shot, bx, by, 0) in processing order
  int ntiles;
  BatchHdr *hdr;
  // persistent form: arrivals each grid barrier waits for (the grid size;
  // tests raise it to exercise the time-out) and the wait limit in cycles
  unsigned barrier_count;
  long long barrier_cycles;
};

// Whether 32-bit word w of StepParams belongs to a field that changes from
// phase to phase (buffers, step index, trace slot and its end), which
// load_shot2 writes itself.
__device__ __forceinline__ bool per_step_word(int w) {
  constexpr int fin = (int)(offsetof(StepParams, fin) / 4);
  constexpr int fout = (int)(offsetof(StepParams, fout) / 4);
  constexpr int n = (int)(offsetof(StepParams, n) / 4);
  constexpr int ts = (int)(offsetof(StepParams, trace_slot) / 4);
  constexpr int te = (int)(offsetof(StepParams, trace_end) / 4);
  return w == fin || w == fin + 1 || w == fout || w == fout + 1 || w == n || w == n + 1 ||
         w == ts || w == te;
}

// Stages the parameters of shot s for step hdr->kbase + k of this call in
// shared memory (every thread of the block calls it).
template <int NT>
__device__ __forceinline__ void load_shot(const BatchArgs &a, int s, int k, StepParams &sp,
                                          int &lam) {
  const int t = threadIdx.y * 32 + threadIdx.x;
  const int *src = (const int *)&a.shots[s].p;
  int *dst = (int *)&sp;
  for (int w = t; w < (int)(sizeof(StepParams) / 4); w += NT) dst[w] = src[w];
  __syncthreads();
  if (t == 0) {
    const BatchShot &b = a.shots[s];
    const BatchDyn d = a.dyn[s];
    const long long step = a.hdr->kbase + k;
    const int cur = (int)((d.cur0 + step) & 1);
    sp.fin = b.f[cur];
    sp.fout = (void *)b.f[cur ^ 1];
    sp.n = d.n0 + step;
    const long long slot = d.traced0 + step;
    sp.trace_slot = (sp.nrec > 0 && slot < b.trace_max) ? (int)slot : -1;
    lam = b.lam;
  }
  __syncthreads();
}

// Stages the parameters of shot s for the two steps of phase hdr->kbase + k
// of this call (steps n0 + 2 phase and n0 + 2 phase + 1; one buffer swap per
// phase) in shared memory (every thread of the block calls it): the threads
// copy the step-independent words while thread 0 forms the per-step fields,
// so the staging costs one memory round trip and one barrier (for the
// two-step tiles 5 % faster than copying first and patching after a
// barrier; the short one-step tiles measured 1 % slower that way, and keep
// the two barriers).
template <int NT>
__device__ __forceinline__ void load_shot2(const BatchArgs &a, int s, int k, StepParams &sp,
                                           int &lam) {
  const int t = threadIdx.y * 32 + threadIdx.x;
  const BatchShot &b = a.shots[s];
  const int *src = (const int *)&b.p;
  int *dst = (int *)&sp;
  for (int w = t; w < (int)(sizeof(StepParams) / 4); w += NT)
    if (!per_step_word(w)) dst[w] = src[w];
  if (t == 0) {
    // every load issued before any is used (one round trip)
    const BatchDyn d = a.dyn[s];
    const long long ph = a.hdr->kbase + k;
    const void *f0 = b.f[0], *f1 = b.f[1];
    const int cur = (int)((d.cur0 + ph) & 1);
    sp.fin = cur ? f1 : f0;
    sp.fout = (void *)(cur ? f0 : f1);
    sp.n = d.n0 + 2 * ph;
    const long long slot = d.traced0 + 2 * ph;
    // phase2() checks each of the two slots against trace_end
    sp.trace_slot = (b.p.nrec > 0 && slot < b.trace_max) ? (int)slot : -1;
    sp.trace_end = b.trace_max;
    lam = b.lam;
  }
  __syncthreads();
}

// One-step tile: 32 x R cells, one per thread.
template <class T, class C, class U, int R>
__device__ __forceinline__ void batch_tile(const StepParams &sp, int lam, int bx, int by) {
  if (lam) step_block<T, C, U, true, 0, R>(sp, bx, by);
  else step_block<T, C, U, false, 0, R>(sp, bx, by);
}

// Two-step tiles: both kinds are blocks of 32 x 16 threads.
static_assert(kF2Warps == kL2H && kF2W == kL2W && kF2H == kL2H,
              "the two kinds of two-step tile share one block shape");
constexpr int kBatch2Threads = 32 * kF2Warps;

// Shared memory of a two-step tile: the window of either kind (large enough
// for the staged inputs of a general tile, which it holds first), and the
// density buffer of the density-gradient kind behind it.
template <class T, class C>
struct Batch2Smem {
  static constexpr int kWin = l2_buf<T>() > f2_buf<T>() ? l2_buf<T>() : f2_buf<T>();
  static constexpr size_t kBytes = kWin * sizeof(T) + sizeof(C) * kL2RH * kL2RW;
};

template <class T, class C, class U>
__device__ __forceinline__ void batch_tile2(const StepParams &sp, int lam, int bx, int by,
                                            char *smem) {
  T *win = (T *)smem;
  if (lam)
    step2_lam_tile<T, C, U>(sp, bx, by, win,
                            (C(*)[kL2RW])(smem + Batch2Smem<T, C>::kWin * sizeof(T)));
  else
    step2_tile<T, C, U>(sp, bx, by, win);
}

// Resident blocks per SM the register budget of a tile kind is set for.
template <int R> constexpr int batch_min_blocks() { return 48 / R; }

// One step (index hdr->kbase + k of this call) over every tile.
template <class T, class C, class U, int R>
__global__ void __launch_bounds__(32 * R, (batch_min_blocks<R>()))
    batch_step_kernel(const BatchArgs a, int k) {
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  __shared__ StepParams sp;
  __shared__ int lam;
  const int4 tl = a.tiles[blockIdx.x];
  load_shot<32 * R>(a, tl.x, k, sp, lam);
  batch_tile<T, C, U, R>(sp, lam, tl.y, tl.z);
}

// Two steps (phase hdr->kbase + k of this call) over every two-step tile.
template <class T, class C, class U>
__global__ void __launch_bounds__(kBatch2Threads, LBM_STEP2_MIN_BLOCKS)
    batch_step2_kernel(const BatchArgs a, int k) {
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  __shared__ StepParams sp;
  __shared__ int lam;
  __shared__ __align__(16) char smem[Batch2Smem<T, C>::kBytes];
  const int4 tl = a.tiles[blockIdx.x];
  load_shot2<kBatch2Threads>(a, tl.x, k, sp, lam);
  batch_tile2<T, C, U>(sp, lam, tl.y, tl.z, smem);
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier k of a persistent launch, by thread 0 of each block: arrive,
// then wait (bounded by barrier_cycles; past it bit 1 of hdr->err is set and
// the block is told to quit).  Every thread calls it; it holds one block
// barrier.  Returns whether the block must quit.
__device__ __forceinline__ bool batch_grid_barrier(const BatchArgs &a, int k, int *quit) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    *quit = 0;
    __threadfence();  // this block's stores before its arrival
    atomicAdd(&a.hdr->arrive, 1ULL);
    const unsigned long long target = (unsigned long long)(k + 1) * a.barrier_count;
    const long long t0 = clock64();
    while (load_acquire(&a.hdr->arrive) < target) {
      if (clock64() - t0 > a.barrier_cycles) {
        atomicOr(&a.hdr->err, 2);
        *quit = 1;
        break;
      }
    }
    __threadfence();  // the other blocks' stores before this block's loads
  }
  __syncthreads();
  return *quit != 0;
}

// nsteps steps (TPS = 1) or two-step phases (TPS = 2) in one launch.  Blocks
// claim tiles from hdr->queue (each block makes exactly one failing claim
// per step, so the claims of step k start at k (ntiles + gridDim.x)) and meet
// at a grid barrier after each step.  The barrier wait is bounded: past
// barrier_cycles it sets bit 1 of hdr->err and the block returns.  Needs a
// cooperative launch (all blocks resident).
template <class T, class C, class U, int R, int TPS>
__global__ void __launch_bounds__(TPS == 2 ? kBatch2Threads : 32 * R,
                                  TPS == 2 ? LBM_STEP2_MIN_BLOCKS : batch_min_blocks<R>())
    batch_persistent_kernel(const BatchArgs a, int nsteps) {
  __shared__ StepParams sp;
  __shared__ int lam, tile, quit;
  __shared__ __align__(16) char smem[TPS == 2 ? Batch2Smem<T, C>::kBytes : 16];
  constexpr int NT = TPS == 2 ? kBatch2Threads : 32 * R;
  const int t = threadIdx.y * 32 + threadIdx.x;
  const unsigned long long per_step = (unsigned long long)a.ntiles + gridDim.x;
  for (int k = 0; k < nsteps; ++k) {
    for (;;) {
      if (t == 0)
        tile = (int)(atomicAdd(&a.hdr->queue, 1ULL) - (unsigned long long)k * per_step);
      __syncthreads();
      const int ti = tile;
      if (ti >= a.ntiles) break;  // the same for the whole block
      const int4 tl = a.tiles[ti];
      if constexpr (TPS == 2) {
        load_shot2<NT>(a, tl.x, k, sp, lam);
        batch_tile2<T, C, U>(sp, lam, tl.y, tl.z, smem);
      } else {
        load_shot<NT>(a, tl.x, k, sp, lam);
        batch_tile<T, C, U, R>(sp, lam, tl.y, tl.z);
      }
      __syncthreads();  // every thread is done with sp and smem before the next claim
    }
    if (batch_grid_barrier(a, k, &quit)) return;
  }
}

// Advances hdr->kbase by g (the last node of a captured group of steps).
__global__ void batch_advance_kernel(BatchHdr *h, int g);

// Launch entry points, one translation unit per storage type.  tps: time
// steps per tile, 1 (tiles of 32 x R cells, R = 4 or 8) or 2 (the two-step
// tiles; R unused).
cudaError_t batch_launch_f64(int R, int tps, bool persistent, const BatchArgs &a, int count,
                             int grid, bool pdl, cudaStream_t s);
cudaError_t batch_launch_f32(bool u64, int R, int tps, bool persistent, const BatchArgs &a,
                             int count, int grid, bool pdl, cudaStream_t s);
cudaError_t batch_launch_16(bool bf16, bool u64, int R, int tps, bool persistent,
                            const BatchArgs &a, int count, int grid, bool pdl, cudaStream_t s);
int batch_occupancy_f64(int R, int tps);
int batch_occupancy_f32(bool u64, int R, int tps);
int batch_occupancy_16(bool bf16, bool u64, int R, int tps);

// Launches one form of the batched kernel: persistent (count = steps or
// phases, grid = resident blocks, cooperative) or one step / phase (count =
// its index k, grid = tiles).
template <class T, class C, class U, int R, int TPS>
cudaError_t batch_launch_t(bool persistent, const BatchArgs &a, int count, int grid, bool pdl,
                           cudaStream_t s) {
  const dim3 block = TPS == 2 ? dim3(32, kF2Warps) : dim3(32, R);
  if (persistent) {
    void *args[] = {(void *)&a, (void *)&count};
    return cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel<T, C, U, R, TPS>,
                                       dim3(grid), block, args, 0, s);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = block;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl && LBM_PDL) ? 1 : 0;
  if constexpr (TPS == 2) return cudaLaunchKernelEx(&cfg, batch_step2_kernel<T, C, U>, a, count);
  else return cudaLaunchKernelEx(&cfg, batch_step_kernel<T, C, U, R>, a, count);
}

template <class T, class C, class U, int R, int TPS>
int batch_occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, batch_persistent_kernel<T, C, U, R, TPS>, TPS == 2 ? kBatch2Threads : 32 * R,
          0) != cudaSuccess)
    return 0;
  return n;
}

template <class T, class C, class U>
cudaError_t batch_launch_r(int R, int tps, bool persistent, const BatchArgs &a, int count,
                           int grid, bool pdl, cudaStream_t s) {
  if (tps == 2) return batch_launch_t<T, C, U, 8, 2>(persistent, a, count, grid, pdl, s);
  if (R == 4) return batch_launch_t<T, C, U, 4, 1>(persistent, a, count, grid, pdl, s);
  return batch_launch_t<T, C, U, 8, 1>(persistent, a, count, grid, pdl, s);
}

template <class T, class C, class U>
int batch_occupancy_r(int R, int tps) {
  if (tps == 2) return batch_occupancy_t<T, C, U, 8, 2>();
  return R == 4 ? batch_occupancy_t<T, C, U, 4, 1>() : batch_occupancy_t<T, C, U, 8, 1>();
}

}  // namespace lbm
