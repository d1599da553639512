// One-warp resident-trajectory tiles for BF16 storage of X (tiles 17..23 of the table in
// res_bf16.cu): for subsamples of at most a few warps' rows, one warp carries the whole trajectory.
// A translation unit of its own so that the library's sources compile in parallel.
#include "resident.cuh"

namespace subsmc {
namespace {
using XT = __nv_bfloat16;
}  // namespace

int res_launch_bf16_w1(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 17: return launch_res<XT, 8, 1>(a, s, sms, dry);
    case 18: return launch_res<XT, 12, 1>(a, s, sms, dry);
    case 19: return launch_res<XT, 16, 1>(a, s, sms, dry);
    case 20: return launch_res<XT, 20, 1>(a, s, sms, dry);
    case 21: return launch_res<XT, 24, 1>(a, s, sms, dry);
    case 22: return launch_res<XT, 32, 1>(a, s, sms, dry);
    case 23: return launch_res<XT, 40, 1>(a, s, sms, dry);
    default: return -1;
  }
}

int res_launch_batch_bf16_w1(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                             cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 17: return launch_res_batch<XT, 8, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 18: return launch_res_batch<XT, 12, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 19: return launch_res_batch<XT, 16, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 20: return launch_res_batch<XT, 20, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 21: return launch_res_batch<XT, 24, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 22: return launch_res_batch<XT, 32, 1>(b, p_max, m_max, G_max, s, sms, dry);
    case 23: return launch_res_batch<XT, 40, 1>(b, p_max, m_max, G_max, s, sms, dry);
    default: return -1;
  }
}

}  // namespace subsmc
