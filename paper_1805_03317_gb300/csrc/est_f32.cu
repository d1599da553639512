// Estimator kernels for f32 storage of X: one instantiation per compiled tile shape.
#include "estimator.cuh"

namespace subsmc {
namespace {
using XT = float;
const Tile kTiles[] = {{1, 8, 2, 4}, {1, 24, 1, 4}, {2, 16, 1, 4}, {4, 8, 2, 4}, {4, 16, 1, 4}, {8, 16, 1, 4}};
}  // namespace

int est_tiles_f32(Tile *out, int cap) {
  const int n = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kTiles[i];
  return n;
}

int est_launch_f32(int op, int tile, const EstArgs &a, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile<XT, 1, 8, 2, 4>(op, a, s);
    case 1: return launch_tile<XT, 1, 24, 1, 4>(op, a, s);
    case 2: return launch_tile<XT, 2, 16, 1, 4>(op, a, s);
    case 3: return launch_tile<XT, 4, 8, 2, 4>(op, a, s);
    case 4: return launch_tile<XT, 4, 16, 1, 4>(op, a, s);
    case 5: return launch_tile<XT, 8, 16, 1, 4>(op, a, s);
    default: return -1;
  }
}

}  // namespace subsmc
