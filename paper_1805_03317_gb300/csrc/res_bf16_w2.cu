// Two-warp resident-trajectory tiles for BF16 storage of X (tiles 10..16 of the table in
// res_bf16.cu). A translation unit of its own so that the library's sources compile in parallel.
#include "resident.cuh"

namespace subsmc {
namespace {
using XT = __nv_bfloat16;
}  // namespace

int res_launch_bf16_w2(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 10: return launch_res<XT, 8, 2>(a, s, sms, dry);
    case 11: return launch_res<XT, 12, 2>(a, s, sms, dry);
    case 12: return launch_res<XT, 16, 2>(a, s, sms, dry);
    case 13: return launch_res<XT, 20, 2>(a, s, sms, dry);
    case 14: return launch_res<XT, 24, 2>(a, s, sms, dry);
    case 15: return launch_res<XT, 32, 2>(a, s, sms, dry);
    case 16: return launch_res<XT, 40, 2>(a, s, sms, dry);
    default: return -1;
  }
}

int res_launch_batch_bf16_w2(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                             cudaStream_t s, int sms, bool dry) {
  switch (tile) {
    case 10: return launch_res_batch<XT, 8, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 11: return launch_res_batch<XT, 12, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 12: return launch_res_batch<XT, 16, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 13: return launch_res_batch<XT, 20, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 14: return launch_res_batch<XT, 24, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 15: return launch_res_batch<XT, 32, 2>(b, p_max, m_max, G_max, s, sms, dry);
    case 16: return launch_res_batch<XT, 40, 2>(b, p_max, m_max, G_max, s, sms, dry);
    default: return -1;
  }
}

}  // namespace subsmc
