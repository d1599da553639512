// Batched estimator kernels for bf16 storage of X (batches of independent posteriors): one
// instantiation per compiled tile shape, the same tiles as est_bf16.cu. A translation unit of
// its own so that the library's sources compile in parallel.
#include "estimator.cuh"

namespace subsmc {
namespace {
using XT = __nv_bfloat16;
}  // namespace

int est_launch_batch_bf16(int op, int tile, const BatchArgs &b, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile_batch<XT, 1, 8, 3, 4>(op, b, s);
    case 1: return launch_tile_batch<XT, 2, 8, 3, 4>(op, b, s);
    case 2: return launch_tile_batch<XT, 4, 8, 2, 4>(op, b, s);
    case 3: return launch_tile_batch<XT, 2, 16, 2, 4>(op, b, s);
    case 4: return launch_tile_batch<XT, 4, 16, 2, 4>(op, b, s);
    case 5: return launch_tile_batch<XT, 8, 8, 2, 4>(op, b, s);
    case 6: return launch_tile_batch<XT, 8, 8, 3, 4>(op, b, s);
    case 7: return launch_tile_batch<XT, 8, 16, 2, 4>(op, b, s);
    case 8: return launch_tile_batch<XT, 16, 8, 2, 4>(op, b, s);
    case 9: return launch_tile_batch<XT, 4, 8, 3, 4, true>(op, b, s);
    case 10: return launch_tile_batch<XT, 4, 16, 3, 4, true>(op, b, s);
    case 11: return launch_tile_batch<XT, 8, 8, 3, 4, true>(op, b, s);
    default: return -1;
  }
}

}  // namespace subsmc
