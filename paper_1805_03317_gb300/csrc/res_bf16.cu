// Resident-trajectory HMC kernels for bf16 storage of X: one instantiation per compiled tile.
// A translation unit of its own so that the library's sources compile in parallel.
#include "resident.cuh"
#include "resident_tc.cuh"

namespace subsmc {
namespace {
using XT = __nv_bfloat16;
// T = 0 marks the tensor-core trajectory kernel (resident_tc.cuh: p <= 32, 8 warps); the 40-slot
// tiles hold two columns per lane. Tiles 10..16 are the two-warp CTAs (res_bf16_w2.cu) and 17..23
// the one-warp CTAs (res_bf16_w1.cu) for small subsamples, where the per-pass work that every
// warp repeats outweighs the rows.
const Tile kResTiles[] = {{1, 8, 1, 4},  {1, 16, 1, 4}, {1, 24, 1, 4}, {1, 32, 1, 4}, {1, 16, 1, 8},
                          {1, 24, 1, 8}, {1, 20, 1, 4}, {1, 12, 1, 4}, {0, 32, 1, 8}, {1, 40, 1, 4},
                          {1, 8, 1, 2},  {1, 12, 1, 2}, {1, 16, 1, 2}, {1, 20, 1, 2}, {1, 24, 1, 2},
                          {1, 32, 1, 2}, {1, 40, 1, 2}, {1, 8, 1, 1},  {1, 12, 1, 1}, {1, 16, 1, 1},
                          {1, 20, 1, 1}, {1, 24, 1, 1}, {1, 32, 1, 1}, {1, 40, 1, 1}};
}  // namespace

int res_tiles_bf16(Tile *out, int cap) {
  const int n = (int)(sizeof(kResTiles) / sizeof(kResTiles[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kResTiles[i];
  return n;
}

int res_launch_bf16(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 0: return launch_res<XT, 8, 4>(a, s, sms, dry);
    case 1: return launch_res<XT, 16, 4>(a, s, sms, dry);
    case 2: return launch_res<XT, 24, 4>(a, s, sms, dry);
    case 3: return launch_res<XT, 32, 4>(a, s, sms, dry);
    case 4: return launch_res<XT, 16, 8>(a, s, sms, dry);
    case 5: return launch_res<XT, 24, 8>(a, s, sms, dry);
    case 6: return launch_res<XT, 20, 4>(a, s, sms, dry);
    case 7: return launch_res<XT, 12, 4>(a, s, sms, dry);
    case 8: return launch_res_tc(a, s, sms, dry);
    case 9: return launch_res<XT, 40, 4>(a, s, sms, dry);
    default: return tile >= 17 ? res_launch_bf16_w1(tile, a, s, sms, dry)
                               : res_launch_bf16_w2(tile, a, s, sms, dry);
  }
}

int res_launch_batch_bf16(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                          cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 0: return launch_res_batch<XT, 8, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 1: return launch_res_batch<XT, 16, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 2: return launch_res_batch<XT, 24, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 3: return launch_res_batch<XT, 32, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 6: return launch_res_batch<XT, 20, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 7: return launch_res_batch<XT, 12, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 9: return launch_res_batch<XT, 40, 4>(b, p_max, m_max, G_max, s, sms, dry);
    case 4:
    case 5:
    case 8: return -1;  // the 8-warp and tensor-core tiles have no batched form
    default:
      return tile >= 17 ? res_launch_batch_bf16_w1(tile, b, p_max, m_max, G_max, s, sms, dry)
                        : res_launch_batch_bf16_w2(tile, b, p_max, m_max, G_max, s, sms, dry);
  }
}

}  // namespace subsmc
