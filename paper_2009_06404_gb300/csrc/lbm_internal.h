// Internals shared by the host files of the library: the workspace layout
// of one grid and the handle.  Not part of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "lbm_elastic.h"
#include "lbm_kernels.cuh"

namespace lbm {

// Offsets (bytes) of the regions of one grid's workspace, and strides.
struct Layout {
  int pitch = 0;
  long long plane = 0;
  int finter = 1;                 // population rows interleaved ([y][i][x])
  long long fplane = 0, frow = 0; // population strides (elements)
  size_t tsize = 0, usize = 0, csize = 0;
  size_t f[2] = {0, 0}, u = 0, lam = 0, irho = 0, src = 0, srcb = 0, rec_ptr = 0, rec_xy = 0,
         rec_id = 0, traces = 0, partials = 0, flags = 0, stage = 0, total = 0;
  int rec_tiles_x = 0, rec_tiles = 0, stage_rows = 0;
  size_t order2 = 0, order2l = 0; // two-step tiles in launch order (int2), both geometries
  long long ntiles2 = 0, ntiles2l = 0;
  size_t blk1 = 0;                // one-step blocks (32 x 8) a source or receiver reaches (bytes)
  long long nblk1 = 0;
  long long mat_count = 0;
};

}  // namespace lbm

// One grid: configuration, workspace layout and host-side state.
struct lbm_elastic {
  int nsm = 0;                 // multiprocessors of the device
  lbm_elastic_config cfg;
  lbm::Layout L;
  char *ws = nullptr;
  cudaStream_t stream = nullptr;
  int cur = 0;                 // buffer holding the latest post-collision state
  long long step = 0;
  int traced = 0;
  int nsrc = 0, nrec = 0;
  bool lambda_nonzero = false;
  int steps_per_launch = -1;   // lbm_elastic_step: 1, 2, -1 auto
  long long launches = 0;
  std::vector<lbm::SourceDev> src_host;
  std::vector<int> rec_host;        // receivers (x, y), as set
  std::vector<int2> order_host;     // the tile order lists last uploaded
  int order2_first = 0, order2l_first = 0;
  int src_box[4] = {0, -1, 0, -1};  // x0, x1, y0, y1 of all source footprints
  int rec_box[4] = {0, -1, 0, -1};  // x0, x1, y0, y1 of all receivers
  std::string err;
};

namespace lbm {
// Step parameters of the handle's next step (current buffers, step index,
// no trace slot).
StepParams handle_step_params(lbm_elastic_t *h);
// One step of the handle.  With grad_out set, the step takes the
// gradient-force path (whatever Lambda is; the result is the same) and
// stores the centred density gradient of every cell there.
lbm_status handle_step(lbm_elastic_t *h, void *grad_out);
}  // namespace lbm
