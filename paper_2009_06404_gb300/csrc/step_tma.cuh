// Shared declarations of the TMA-staged step kernel (step_tma.cu) and its
// host-side set-up (lbm_api.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbm {

#ifndef LBM_TMA_TILE_H
#define LBM_TMA_TILE_H 4
#endif
#ifndef LBM_TMA_STAGES
#define LBM_TMA_STAGES 2
#endif
#ifndef LBM_TMA_L2_PROMOTION
#define LBM_TMA_L2_PROMOTION 2   // 0 none, 1 128 B, 2 256 B
#endif
constexpr int kTileW = 128;        // tile width in cells (one warp covers 32 of them)
constexpr int kTileH = LBM_TMA_TILE_H;  // tile height
#ifndef LBM_TMA_THREADS
#define LBM_TMA_THREADS 256
#endif
constexpr int kTmaThreads = LBM_TMA_THREADS;  // warps per CTA / kTileH per tile row
constexpr int kTmaStages = LBM_TMA_STAGES;  // tiles in flight per CTA (several CTAs share an SM)
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz: bound of every wait

// Tensor maps of one handle: the two population buffers, each with a halo of
// one row (no density gradient) and of two rows (with it), and the
// displacement.
struct TmaMaps {
  CUtensorMap f[2][2];  // [buffer][halo rows - 1]
  CUtensorMap u;
};

// x halo of the shared-memory tile of a storage type: one 16-byte unit.
inline int tma_halo_x(int elem_bytes) { return 16 / elem_bytes; }

// Launches the TMA-staged step (MODE 0) reading buffer `cur`.  Returns
// cudaErrorNotSupported for storage types it does not cover.
cudaError_t launch_step_tma(const StepParams &p, const TmaMaps &maps, int cur, int storage,
                            bool u64, bool lam, int nsm, cudaStream_t s);

// Resident CTAs per SM of the variant (after tma_prepare).
int tma_ctas_per_sm(int storage, bool u64, bool lam);

// Sets the dynamic shared memory limit of the kernel variants for one storage
// type on the current device (call once per handle, before launching).
cudaError_t tma_prepare(int storage, bool u64);

// Dynamic shared memory the kernel needs (0 if not covered).
int tma_smem_bytes(int storage, bool u64, bool lam);

// Number of pipeline stages the variant uses.
int tma_stages(int storage, bool u64, bool lam);

}  // namespace lbm
