// Estimator kernels for f64 storage of X: one instantiation per compiled tile shape.
#include "estimator.cuh"

namespace subsmc {
namespace {
using XT = double;
const Tile kTiles[] = {{1, 8, 1, 4}, {4, 8, 1, 4}, {8, 16, 1, 4}};
}  // namespace

int est_tiles_f64(Tile *out, int cap) {
  const int n = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kTiles[i];
  return n;
}

int est_launch_f64(int op, int tile, const EstArgs &a, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile<XT, 1, 8, 1, 4>(op, a, s);
    case 1: return launch_tile<XT, 4, 8, 1, 4>(op, a, s);
    case 2: return launch_tile<XT, 8, 16, 1, 4>(op, a, s);
    default: return -1;
  }
}

}  // namespace subsmc
