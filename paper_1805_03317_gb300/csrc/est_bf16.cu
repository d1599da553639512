// Estimator kernels for bf16 storage of X: one instantiation per compiled tile shape.
#include "estimator.cuh"

namespace subsmc {
namespace {
using XT = __nv_bfloat16;
const Tile kTiles[] = {{1, 8, 3, 4, 0}, {2, 8, 3, 4, 0}, {4, 8, 2, 4, 0}, {2, 16, 2, 4, 0},
                       {4, 16, 2, 4, 0}, {8, 8, 2, 4, 0}, {8, 8, 3, 4, 0}, {8, 16, 2, 4, 0},
                       {16, 8, 2, 4, 0}, {4, 8, 3, 4, 1}, {4, 16, 3, 4, 1}, {8, 8, 3, 4, 1}};
}  // namespace

int est_tiles_bf16(Tile *out, int cap) {
  const int n = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kTiles[i];
  return n;
}

int est_launch_bf16(int op, int tile, const EstArgs &a, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile<XT, 1, 8, 3, 4>(op, a, s);
    case 1: return launch_tile<XT, 2, 8, 3, 4>(op, a, s);
    case 2: return launch_tile<XT, 4, 8, 2, 4>(op, a, s);
    case 3: return launch_tile<XT, 2, 16, 2, 4>(op, a, s);
    case 4: return launch_tile<XT, 4, 16, 2, 4>(op, a, s);
    case 5: return launch_tile<XT, 8, 8, 2, 4>(op, a, s);
    case 6: return launch_tile<XT, 8, 8, 3, 4>(op, a, s);
    case 7: return launch_tile<XT, 8, 16, 2, 4>(op, a, s);
    case 8: return launch_tile<XT, 16, 8, 2, 4>(op, a, s);
    case 9: return launch_tile<XT, 4, 8, 3, 4, true>(op, a, s);
    case 10: return launch_tile<XT, 4, 16, 3, 4, true>(op, a, s);
    case 11: return launch_tile<XT, 8, 8, 3, 4, true>(op, a, s);
    default: return -1;
  }
}

int est_warp_smem_bf16(int tile, int p) {
  switch (tile) {
    case 0: return warp_smem_bytes<XT, 1, 8, 3>(p);
    case 1: return warp_smem_bytes<XT, 2, 8, 3>(p);
    case 2: return warp_smem_bytes<XT, 4, 8, 2>(p);
    case 3: return warp_smem_bytes<XT, 2, 16, 2>(p);
    case 4: return warp_smem_bytes<XT, 4, 16, 2>(p);
    case 5: return warp_smem_bytes<XT, 8, 8, 2>(p);
    case 6: return warp_smem_bytes<XT, 8, 8, 3>(p);
    case 7: return warp_smem_bytes<XT, 8, 16, 2>(p);
    case 8: return warp_smem_bytes<XT, 16, 8, 2>(p);
    case 9: return warp_smem_bytes<XT, 4, 8, 3>(p);
    case 10: return warp_smem_bytes<XT, 4, 16, 3>(p);
    case 11: return warp_smem_bytes<XT, 8, 8, 3>(p);
    default: return 0;
  }
}

}  // namespace subsmc
