// fvna_net.h -- internals of the correction network shared by fvna_net.cu
// and the solver runtime (which appends the network to the step graph).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fvna.h"

namespace fvna {

// offsets of the parameter blocks in the flat FP32 parameter vector
constexpr int NET_OFF_W1 = 0;                       // 32 x 3 x 3 x 3
constexpr int NET_OFF_B1 = NET_OFF_W1 + 32 * 3 * 9;  // 32
constexpr int NET_OFF_W2 = NET_OFF_B1 + 32;         // 32 x 32 x 3 x 3
constexpr int NET_OFF_B2 = NET_OFF_W2 + 32 * 32 * 9;  // 32
constexpr int NET_OFF_W3 = NET_OFF_B2 + 32;         // 3 x 32 x 3 x 3
constexpr int NET_OFF_B3 = NET_OFF_W3 + 3 * 32 * 9;  // 3
static_assert(NET_OFF_B3 + 3 == FVNA_NET_PARAMS, "parameter layout");

struct NetConvArgs {
  int h, w;
  const float *in;                 // FP32 input planes (first layer)
  long long in_pstride, in_bstride;
  int in_pitch;
  float in_scale;
  const __nv_bfloat16 *hin;        // BF16 hidden input (pixel-major, 32 channels)
  const __nv_bfloat16 *wmat;       // packed weights [n][k]
  const float *bias;
  __nv_bfloat16 *hout;             // BF16 hidden output
  float *out;                      // FP32 output planes (last layer)
  long long out_pstride, out_bstride;
  int out_pitch;
  int apply;                       // 1: out += out_scale * y
  float out_scale;
  const int *done;                 // if not NULL and *done != 0: do nothing
  const long long *step;           // if not NULL: apply only when (*step + 1) % every == 0
  int every;
  int band;                        // apply: leave cells within `band` of any edge unchanged
};

cudaError_t net_forward_launch(const fvna_net *n, int B, int H, int W, const float *in,
                               long long in_pstride, int in_pitch, long long in_bstride,
                               float in_scale, float *out, long long out_pstride, int out_pitch,
                               long long out_bstride, int apply, float out_scale,
                               __nv_bfloat16 *h1, __nv_bfloat16 *h2, cudaStream_t s,
                               const int *done = nullptr, const long long *step = nullptr,
                               int every = 1, int band = 0);

}  // namespace fvna
