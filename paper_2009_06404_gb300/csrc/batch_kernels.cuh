// Batched step: many independent grids ("shots") advanced together.  The
// work of one step is a flat list of tiles (shot, block column, block row)
// of 32 x R cells (64 x R with two cells per thread); each tile runs the
// same block update as the single-grid kernel, with its shot's parameters
// staged in shared memory.  Two launch forms share it: one launch per step
// over all tiles (stream launches or a CUDA graph), and a persistent
// cooperative launch that claims tiles from an atomic queue and separates
// the steps with a grid barrier.
#pragma once

#include "lbm_kernels.cuh"

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

// One tile: 32 x R cells, one per thread (CPT 1), or 64 x R cells, two
// horizontally adjacent cells per thread (CPT 2, paired loads and stores).
template <class T, class C, class U, int R, int CPT>
__device__ __forceinline__ void batch_tile(const StepParams &sp, int lam, int bx, int by) {
  if constexpr (CPT == 2) {
    if (lam) step_block_pair<T, C, U, true, R>(sp, bx, by);
    else step_block_pair<T, C, U, false, R>(sp, bx, by);
  } else {
    if (lam) step_block<T, C, U, true, 0, R>(sp, bx, by);
    else step_block<T, C, U, false, 0, R>(sp, bx, by);
  }
}

// Resident blocks per SM the register budget of a tile kind is set for.
template <int R, int CPT> constexpr int batch_min_blocks() { return CPT == 2 ? 4 : 48 / R; }

// One step (index hdr->kbase + k of this call) over every tile.
template <class T, class C, class U, int R, int CPT>
__global__ void __launch_bounds__(32 * R, (batch_min_blocks<R, CPT>()))
    batch_step_kernel(const BatchArgs a, int k) {
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
#endif
  __shared__ StepParams sp;
  __shared__ int lam;
  const int4 tl = a.tiles[blockIdx.x];
  load_shot<32 * R>(a, tl.x, k, sp, lam);
  batch_tile<T, C, U, R, CPT>(sp, lam, tl.y, tl.z);
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// nsteps steps in one launch.  Blocks claim tiles from hdr->queue (each
// block makes exactly one failing claim per step, so the claims of step k
// start at k (ntiles + gridDim.x)) and meet at a grid barrier after each
// step.  The barrier wait is bounded: past barrier_cycles it sets bit 1 of
// hdr->err and the block returns.  Needs a cooperative launch (all blocks
// resident).
template <class T, class C, class U, int R, int CPT>
__global__ void __launch_bounds__(32 * R, (batch_min_blocks<R, CPT>()))
    batch_persistent_kernel(const BatchArgs a, int nsteps) {
  __shared__ StepParams sp;
  __shared__ int lam, tile, quit;
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
      load_shot<32 * R>(a, tl.x, k, sp, lam);
      batch_tile<T, C, U, R, CPT>(sp, lam, tl.y, tl.z);
      __syncthreads();  // every thread is done with sp before the next claim
    }
    if (t == 0) {
      quit = 0;
      __threadfence();  // this block's stores before its arrival
      atomicAdd(&a.hdr->arrive, 1ULL);
      const unsigned long long target = (unsigned long long)(k + 1) * a.barrier_count;
      const long long t0 = clock64();
      while (load_acquire(&a.hdr->arrive) < target) {
        if (clock64() - t0 > a.barrier_cycles) {
          atomicOr(&a.hdr->err, 2);
          quit = 1;
          break;
        }
      }
      __threadfence();  // the other blocks' stores before this block's loads
    }
    __syncthreads();
    if (quit) return;
  }
}

// Advances hdr->kbase by g (the last node of a captured group of steps).
__global__ void batch_advance_kernel(BatchHdr *h, int g);

// Launch entry points, one translation unit per storage type.  R: 4 or 8;
// cpt: cells per thread, 1 or 2 (2 with R = 8 only).
cudaError_t batch_launch_f64(int R, int cpt, bool persistent, const BatchArgs &a, int count,
                             int grid, bool pdl, cudaStream_t s);
cudaError_t batch_launch_f32(bool u64, int R, int cpt, bool persistent, const BatchArgs &a,
                             int count, int grid, bool pdl, cudaStream_t s);
cudaError_t batch_launch_16(bool bf16, bool u64, int R, int cpt, bool persistent,
                            const BatchArgs &a, int count, int grid, bool pdl, cudaStream_t s);
int batch_occupancy_f64(int R, int cpt);
int batch_occupancy_f32(bool u64, int R, int cpt);
int batch_occupancy_16(bool bf16, bool u64, int R, int cpt);

// Launches one form of the batched kernel: persistent (count = steps, grid
// = resident blocks, cooperative) or one step (count = k, grid = tiles).
template <class T, class C, class U, int R, int CPT>
cudaError_t batch_launch_t(bool persistent, const BatchArgs &a, int count, int grid, bool pdl,
                           cudaStream_t s) {
  if (persistent) {
    void *args[] = {(void *)&a, (void *)&count};
    return cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel<T, C, U, R, CPT>,
                                       dim3(grid), dim3(32, R), args, 0, s);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32, R);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl && LBM_PDL) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, batch_step_kernel<T, C, U, R, CPT>, a, count);
}

template <class T, class C, class U, int R, int CPT>
int batch_occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_persistent_kernel<T, C, U, R, CPT>,
                                                    32 * R, 0) != cudaSuccess)
    return 0;
  return n;
}

template <class T, class C, class U>
cudaError_t batch_launch_r(int R, int cpt, bool persistent, const BatchArgs &a, int count,
                           int grid, bool pdl, cudaStream_t s) {
  if (cpt == 2) return batch_launch_t<T, C, U, 8, 2>(persistent, a, count, grid, pdl, s);
  if (R == 4) return batch_launch_t<T, C, U, 4, 1>(persistent, a, count, grid, pdl, s);
  return batch_launch_t<T, C, U, 8, 1>(persistent, a, count, grid, pdl, s);
}

template <class T, class C, class U>
int batch_occupancy_r(int R, int cpt) {
  if (cpt == 2) return batch_occupancy_t<T, C, U, 8, 2>();
  return R == 4 ? batch_occupancy_t<T, C, U, 4, 1>() : batch_occupancy_t<T, C, U, 8, 1>();
}

}  // namespace lbm
