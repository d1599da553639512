// Estimator kernels for f32 storage of X: one instantiation per compiled tile shape.
#include "estimator.cuh"
#include "resident.cuh"

namespace subsmc {
namespace {
using XT = float;
const Tile kTiles[] = {{1, 4, 3, 4, 0}, {2, 4, 3, 4, 0}, {4, 4, 2, 4, 0}, {2, 8, 2, 4, 0},
                       {8, 4, 2, 4, 0}, {4, 8, 2, 4, 0}, {8, 8, 2, 4, 0}, {16, 8, 2, 4, 0}};
}  // namespace

int est_tiles_f32(Tile *out, int cap) {
  const int n = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kTiles[i];
  return n;
}

int est_launch_f32(int op, int tile, const EstArgs &a, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile<XT, 1, 4, 3, 4>(op, a, s);
    case 1: return launch_tile<XT, 2, 4, 3, 4>(op, a, s);
    case 2: return launch_tile<XT, 4, 4, 2, 4>(op, a, s);
    case 3: return launch_tile<XT, 2, 8, 2, 4>(op, a, s);
    case 4: return launch_tile<XT, 8, 4, 2, 4>(op, a, s);
    case 5: return launch_tile<XT, 4, 8, 2, 4>(op, a, s);
    case 6: return launch_tile<XT, 8, 8, 2, 4>(op, a, s);
    case 7: return launch_tile<XT, 16, 8, 2, 4>(op, a, s);
    default: return -1;
  }
}

namespace {
const Tile kResTiles[] = {{1, 8, 1, 4, 0}, {1, 16, 1, 4, 0}, {1, 24, 1, 4, 0}, {1, 32, 1, 4, 0},
                          {1, 16, 1, 8, 0}, {1, 24, 1, 8, 0}, {1, 20, 1, 4, 0}, {1, 12, 1, 4, 0}};
}  // namespace

int res_tiles_f32(Tile *out, int cap) {
  const int n = (int)(sizeof(kResTiles) / sizeof(kResTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kResTiles[i];
  return n;
}

int res_launch_f32(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 0: return launch_res<XT, 8, 4>(a, s, sms, dry);
    case 1: return launch_res<XT, 16, 4>(a, s, sms, dry);
    case 2: return launch_res<XT, 24, 4>(a, s, sms, dry);
    case 3: return launch_res<XT, 32, 4>(a, s, sms, dry);
    case 4: return launch_res<XT, 16, 8>(a, s, sms, dry);
    case 5: return launch_res<XT, 24, 8>(a, s, sms, dry);
    case 6: return launch_res<XT, 20, 4>(a, s, sms, dry);
    case 7: return launch_res<XT, 12, 4>(a, s, sms, dry);
    default: return -1;
  }
}

}  // namespace subsmc
