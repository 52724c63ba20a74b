// fvna_net.cu -- the learned sub-grid correction (not in the paper): three
// 3x3 convolutions with zero padding, 3 -> 32 -> 32 -> 3 channels, ReLU after
// the first two,
//     y[o,i,j] = b[o] + sum_c sum_{u,v} w[o,c,u,v] x[c, i+u-1, j+v-1].
//
// Forward: BF16 tensor-core implicit GEMM (mma.sync m16n8k16, FP32
// accumulation).  A CTA owns an 8 x 32 pixel tile; each warp one 32-pixel row
// (two m-tiles of 16 pixels).  The input tile plus a 1-pixel halo sits in
// shared memory channel-innermost (pixel stride 40 bf16 = 80 bytes, so the
// eight rows an ldmatrix reads fall in distinct bank groups); K runs over the
// nine taps times the input channels.  The 3-channel first layer builds its
// (pixels x 32) im2col tile in shared memory instead.  Hidden activations are
// stored as BF16, pixel-major with 32 channels; network input and output are
// FP32 channel planes.
// Backward (training): FP32 CUDA-core kernels for the input and weight
// gradients, then Adam on FP32 master weights, which are re-packed to BF16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "../../include/fvna.h"
#include "fvna_net.h"

namespace fvna {

constexpr int NET_TH = 8;             // tile rows (one warp per row)
constexpr int NET_TW = 32;            // tile columns
constexpr int NET_PIX = NET_TH * NET_TW;
constexpr int NET_HALO_W = NET_TW + 2;
constexpr int NET_HALO_H = NET_TH + 2;
constexpr int CH = 32;                // hidden channels
constexpr int CPAD = 40;              // padded channel stride of shared tiles
constexpr int KH = 9 * CH;            // K of the hidden layers (288)
constexpr int KPAD = KH + 8;          // padded K stride of shared weights (296)
constexpr int K1 = 32;                // K of the first layer (27 taps x channels, padded)

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                        unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned &r0, unsigned &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float d[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Forward convolution on tensor cores.
//   MODE 0: input = FP32 planes (3 channels) times in_scale, output BF16 hidden + ReLU
//   MODE 1: input = BF16 hidden, output BF16 hidden + ReLU
//   MODE 2: input = BF16 hidden, output FP32 planes (3 channels); if apply,
//           the planes receive += out_scale * y instead of y
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_net_conv(NetConvArgs a) {
  constexpr int NT = MODE == 2 ? 1 : 4;           // n-tiles of 8 output channels
  constexpr int KS = MODE == 0 ? K1 / 16 : KH / 16;  // k-steps of 16
  constexpr int WROWS = NT * 8;
  constexpr int WSTRIDE = MODE == 0 ? K1 + 8 : KPAD;
  __shared__ __align__(16) __nv_bfloat16 s_in[NET_HALO_H * NET_HALO_W * CPAD];  // also im2col
  __shared__ __align__(16) __nv_bfloat16 s_w[WROWS * WSTRIDE];
  if (a.done && *a.done) return;   // the step of this domain was not taken
  if (a.step && a.every > 1 && (*a.step + 1) % a.every != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * NET_TH, j0 = blockIdx.x * NET_TW;
  const int H = a.h, W = a.w;

  // weights: [n][k] rows of the packed BF16 matrix
  {
    const int kk = MODE == 0 ? K1 : KH;
    for (int e = tid; e < WROWS * kk / 8; e += 256) {
      int n = e / (kk / 8), k8 = e - n * (kk / 8);
      uint4 v = reinterpret_cast<const uint4 *>(a.wmat + (size_t)n * kk)[k8];
      *reinterpret_cast<uint4 *>(&s_w[n * WSTRIDE + k8 * 8]) = v;
    }
  }
  if (MODE == 0) {
    // 3-channel FP32 input tile -> BF16, then the im2col tile (pixels x 32)
    __shared__ __nv_bfloat16 s_x3[NET_HALO_H * NET_HALO_W * 4];
    for (int e = tid; e < NET_HALO_H * NET_HALO_W; e += 256) {
      int r = e / NET_HALO_W, cc = e - r * NET_HALO_W;
      int gi = i0 + r - 1, gj = j0 + cc - 1;
      float v[3] = {0.f, 0.f, 0.f};
      if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
        size_t off = (size_t)b * a.in_bstride + (size_t)gi * a.in_pitch + gj;
        for (int c = 0; c < 3; c++) v[c] = a.in[off + (size_t)c * a.in_pstride] * a.in_scale;
      }
      for (int c = 0; c < 3; c++) s_x3[e * 4 + c] = __float2bfloat16_rn(v[c]);
      s_x3[e * 4 + 3] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int e = tid; e < NET_PIX * K1; e += 256) {
      int p = e / K1, k = e - p * K1;
      int r = p / NET_TW, cc = p - r * NET_TW;
      __nv_bfloat16 v = __float2bfloat16_rn(0.f);
      if (k < 27) {
        int t = k / 3, c = k - t * 3;
        v = s_x3[((r + t / 3) * NET_HALO_W + cc + t % 3) * 4 + c];
      }
      s_in[p * CPAD + k] = v;
    }
  } else {
    // BF16 hidden input tile with halo (zero outside the image)
    for (int e = tid; e < NET_HALO_H * NET_HALO_W * 4; e += 256) {
      int pix = e >> 2, q = e & 3;
      int r = pix / NET_HALO_W, cc = pix - r * NET_HALO_W;
      int gi = i0 + r - 1, gj = j0 + cc - 1;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gi >= 0 && gi < H && gj >= 0 && gj < W)
        v = reinterpret_cast<const uint4 *>(a.hin + (((size_t)b * H + gi) * W + gj) * CH)[q];
      *reinterpret_cast<uint4 *>(&s_in[pix * CPAD + q * 8]) = v;
    }
  }
  __syncthreads();

  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[mt][nt][q] = 0.f;

  const int mi = lane >> 3, mr = lane & 7;
#pragma unroll 2
  for (int ks = 0; ks < KS; ks++) {
    unsigned af[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      int m = mt * 16 + mr + (mi & 1) * 8;      // pixel within the warp's 32
      int kof = (mi >> 1) * 8;
      const __nv_bfloat16 *src;
      if (MODE == 0) {
        src = &s_in[(warp * NET_TW + m) * CPAD + ks * 16 + kof];
      } else {
        int tap = ks >> 1, half = ks & 1;
        int u = tap / 3, v = tap - u * 3;
        src = &s_in[((warp + u) * NET_HALO_W + m + v) * CPAD + half * 16 + kof];
      }
      ldsm_x4(smem_u32(src), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
      unsigned b0, b1;
      const __nv_bfloat16 *src = &s_w[(nt * 8 + mr) * WSTRIDE + ks * 16 + (mi & 1) * 8];
      ldsm_x2(smem_u32(src), b0, b1);
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
        mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
    }
  }

  // epilogue: bias, ReLU, store
  const int g = lane >> 2, tig = lane & 3;
  const int gi = i0 + warp;
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      int gj = j0 + mt * 16 + g + hh * 8;
      if (gi >= H || gj >= W) continue;
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        int ch = nt * 8 + tig * 2;
        if (MODE == 2 && ch >= 3) continue;
        float y0 = acc[mt][nt][hh * 2] + a.bias[ch];
        float y1 = acc[mt][nt][hh * 2 + 1] + (MODE == 2 && ch + 1 >= 3 ? 0.f : a.bias[ch + 1]);
        if (MODE != 2) {
          y0 = fmaxf(y0, 0.f);
          y1 = fmaxf(y1, 0.f);
          __nv_bfloat162 v = __floats2bfloat162_rn(y0, y1);
          *reinterpret_cast<__nv_bfloat162 *>(a.hout + (((size_t)b * H + gi) * W + gj) * CH + ch) = v;
        } else {
          if (a.apply && (gj < a.band || gj >= W - a.band || gi < a.band || gi >= H - a.band))
            continue;
          size_t off = (size_t)b * a.out_bstride + (size_t)gi * a.out_pitch + gj;
          if (ch < 3) {
            float *o = a.out + off + (size_t)ch * a.out_pstride;
            *o = a.apply ? *o + a.out_scale * y0 : y0;
          }
          if (ch + 1 < 3) {
            float *o = a.out + off + (size_t)(ch + 1) * a.out_pstride;
            *o = a.apply ? *o + a.out_scale * y1 : y1;
          }
        }
      }
    }
}

// ---------------------------------------------------------------------------
// Parameter packing: FP32 master parameters (w[o][c][u][v] per layer, then
// biases) -> BF16 matrices [n][k], k = tap*CIN + c (first layer: tap*3 + c,
// padded to 32), rows beyond the output channels zero (last layer: 8 rows).
// ---------------------------------------------------------------------------
__global__ void k_net_pack(const float *params, __nv_bfloat16 *w1, __nv_bfloat16 *w2,
                           __nv_bfloat16 *w3) {
  const float *p1 = params + NET_OFF_W1, *p2 = params + NET_OFF_W2, *p3 = params + NET_OFF_W3;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 32 * K1 + 32 * KH + 8 * KH;
       e += gridDim.x * blockDim.x) {
    if (e < 32 * K1) {
      int n = e / K1, k = e - n * K1;
      float v = 0.f;
      if (k < 27) { int t = k / 3, c = k - t * 3; v = p1[(n * 3 + c) * 9 + t]; }
      w1[e] = __float2bfloat16_rn(v);
    } else if (e < 32 * K1 + 32 * KH) {
      int f = e - 32 * K1, n = f / KH, k = f - n * KH;
      int t = k / CH, c = k - t * CH;
      w2[f] = __float2bfloat16_rn(p2[(n * CH + c) * 9 + t]);
    } else {
      int f = e - 32 * K1 - 32 * KH, n = f / KH, k = f - n * KH;
      int t = k / CH, c = k - t * CH;
      w3[f] = __float2bfloat16_rn(n < 3 ? p3[(n * CH + c) * 9 + t] : 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// Training kernels (FP32 CUDA cores)
// ---------------------------------------------------------------------------
// loss = mean over the pixels at least `margin` from the image edge of
// (y - t)^2, g = 2 (y - t) / N there and 0 elsewhere
// edges (device, batch x 4: top, bottom, left, right margins) overrides the
// uniform margin per image side: 0 where a crop side is an edge of the field.
__global__ void k_net_count(int B, int H, int W, int margin, const int *edges, long long *nin) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long s = 0;
  for (int b = 0; b < B; b++) {
    int t = edges ? edges[4 * b] : margin, bo = edges ? edges[4 * b + 1] : margin;
    int l = edges ? edges[4 * b + 2] : margin, r = edges ? edges[4 * b + 3] : margin;
    s += (long long)(H - t - bo) * (W - l - r);
  }
  *nin = s;
}

__global__ void k_net_mse(const float *y, const float *t, float *g, long long n, int H, int W,
                          int margin, const int *edges, const long long *nin_p, double *loss) {
  const long long nin = *nin_p;
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int j = (int)(e % W), i = (int)((e / W) % H);
    int b = (int)(e / (3LL * H * W));
    int mt = edges ? edges[4 * b] : margin, mb = edges ? edges[4 * b + 1] : margin;
    int ml = edges ? edges[4 * b + 2] : margin, mr = edges ? edges[4 * b + 3] : margin;
    bool in = i >= mt && i < H - mb && j >= ml && j < W - mr;
    float d = in ? y[e] - t[e] : 0.f;
    g[e] = 2.f * d / (float)nin;
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (double)nin);
}

// Gradient w.r.t. a hidden activation: gin[b][c][i][j] = [h[b][i][j][c] > 0] *
// sum_o sum_{u,v} w[o][c][u][v] g[b][o][i-u+1][j-v+1], with w read from the
// packed BF16 matrix (k = tap*CH + c) that the forward used.
template <int CO>
__global__ void k_net_bwd_input(const float *g, const __nv_bfloat16 *wmat,
                                const __nv_bfloat16 *h, float *gin, int B, int H, int W) {
  const long long n = (long long)B * CH * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int j = (int)(e % W);
    long long r = e / W;
    int i = (int)(r % H);
    r /= H;
    int c = (int)(r % CH);
    int b = (int)(r / CH);
    float hv = __bfloat162float(h[(((size_t)b * H + i) * W + j) * CH + c]);
    float s = 0.f;
    if (hv > 0.f) {
      for (int o = 0; o < CO; o++) {
        const float *go = g + ((size_t)b * CO + o) * H * W;
        for (int u = 0; u < 3; u++) {
          int ii = i - u + 1;
          if (ii < 0 || ii >= H) continue;
          for (int v = 0; v < 3; v++) {
            int jj = j - v + 1;
            if (jj < 0 || jj >= W) continue;
            s += __bfloat162float(wmat[(size_t)o * KH + (u * 3 + v) * CH + c]) *
                 go[(size_t)ii * W + jj];
          }
        }
      }
    }
    gin[e] = s;
  }
}

// Weight and bias gradient of one layer: one block per (o, c) pair,
//   gw[o][c][u][v] = sum_{b,i,j} g[b][o][i][j] x[b][c][i+u-1][j+v-1],
// x being the layer input: BF16 hidden (pixel-major) or, for the first
// layer, the FP32 planes times in_scale rounded to BF16 as the forward did.
template <int CI, int CO, bool FIRST>
__global__ void k_net_bwd_weight(const float *g, const __nv_bfloat16 *xh, const float *x3,
                                 float in_scale, float *gw, float *gb, int B, int H, int W) {
  const int o = blockIdx.x / CI, c = blockIdx.x - o * CI;
  float s[9];
  for (int t = 0; t < 9; t++) s[t] = 0.f;
  float sb = 0.f;
  const long long n = (long long)B * H * W;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    int j = (int)(e % W);
    long long r = e / W;
    int i = (int)(r % H);
    int b = (int)(r / H);
    float gv = g[((size_t)b * CO + o) * H * W + (size_t)i * W + j];
    sb += gv;
    for (int u = 0; u < 3; u++) {
      int ii = i + u - 1;
      if (ii < 0 || ii >= H) continue;
      for (int v = 0; v < 3; v++) {
        int jj = j + v - 1;
        if (jj < 0 || jj >= W) continue;
        float xv;
        if (FIRST)
          xv = __bfloat162float(__float2bfloat16_rn(
              x3[((size_t)b * 3 + c) * H * W + (size_t)ii * W + jj] * in_scale));
        else
          xv = __bfloat162float(xh[(((size_t)b * H + ii) * W + jj) * CH + c]);
        s[u * 3 + v] += gv * xv;
      }
    }
  }
  __shared__ float red[10][32];
  for (int t = 0; t < 10; t++) {
    float v = t < 9 ? s[t] : sb;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[threadIdx.x][w];
    if (threadIdx.x < 9) gw[(o * CI + c) * 9 + threadIdx.x] = v;
    else if (c == 0) gb[o] = v;
  }
}

__global__ void k_net_adam(float *p, const float *g, float *m, float *v, int n, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float gg = g[e];
  float mm = b1 * m[e] + (1.f - b1) * gg;
  float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace fvna

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using namespace fvna;

struct fvna_net {
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, Adam
  __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;            // packed BF16
  __nv_bfloat16 *h1 = nullptr, *h2 = nullptr;                           // activations
  float *y = nullptr, *g3 = nullptr, *gh2 = nullptr, *gh1 = nullptr;
  double *loss = nullptr;
  long long *nin = nullptr;
  long long cap_pix = 0;  // capacity of the activation buffers (B*H*W)
  int adam_t = 0;
};

namespace {

int cerr(cudaError_t e) {
  if (e == cudaSuccess) return FVNA_OK;
  return e == cudaErrorMemoryAllocation ? FVNA_ERR_OOM : FVNA_ERR_CUDA;
}
#define NCK(x)                          \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return cerr(e_); \
  } while (0)

void net_free_buffers(fvna_net *n) {
  cudaFree(n->h1); cudaFree(n->h2); cudaFree(n->y); cudaFree(n->g3);
  cudaFree(n->gh2); cudaFree(n->gh1);
  n->h1 = n->h2 = nullptr;
  n->y = n->g3 = n->gh2 = n->gh1 = nullptr;
  n->cap_pix = 0;
}

int net_reserve(fvna_net *n, long long pix) {
  if (pix <= n->cap_pix) return FVNA_OK;
  net_free_buffers(n);
  NCK(cudaMalloc(&n->h1, (size_t)pix * CH * sizeof(__nv_bfloat16)));
  NCK(cudaMalloc(&n->h2, (size_t)pix * CH * sizeof(__nv_bfloat16)));
  NCK(cudaMalloc(&n->y, (size_t)pix * 3 * sizeof(float)));
  NCK(cudaMalloc(&n->g3, (size_t)pix * 3 * sizeof(float)));
  NCK(cudaMalloc(&n->gh2, (size_t)pix * CH * sizeof(float)));
  NCK(cudaMalloc(&n->gh1, (size_t)pix * CH * sizeof(float)));
  n->cap_pix = pix;
  return FVNA_OK;
}

}  // namespace

namespace fvna {

cudaError_t net_pack(fvna_net *n, cudaStream_t s) {
  k_net_pack<<<64, 256, 0, s>>>(n->params, n->w1, n->w2, n->w3);
  return cudaGetLastError();
}

// The three forward launches.  in: FP32 planes (plane stride, pitch, batch
// stride in elements); out: FP32 planes (or the same planes with apply).
cudaError_t net_forward_launch(const fvna_net *n, int B, int H, int W, const float *in,
                               long long in_pstride, int in_pitch, long long in_bstride,
                               float in_scale, float *out, long long out_pstride, int out_pitch,
                               long long out_bstride, int apply, float out_scale,
                               __nv_bfloat16 *h1, __nv_bfloat16 *h2, cudaStream_t s,
                               const int *done, const long long *step, int every,
                               int band) {
  dim3 grid((W + NET_TW - 1) / NET_TW, (H + NET_TH - 1) / NET_TH, B);
  NetConvArgs a;
  std::memset(&a, 0, sizeof a);
  a.h = H; a.w = W;
  a.in = in; a.in_pstride = in_pstride; a.in_pitch = in_pitch; a.in_bstride = in_bstride;
  a.in_scale = in_scale;
  a.done = done;
  a.step = step;
  a.every = every;
  a.band = band;
  a.wmat = n->w1; a.bias = n->params + NET_OFF_B1; a.hout = h1;
  k_net_conv<0><<<grid, 256, 0, s>>>(a);
  a.hin = h1; a.wmat = n->w2; a.bias = n->params + NET_OFF_B2; a.hout = h2;
  k_net_conv<1><<<grid, 256, 0, s>>>(a);
  a.hin = h2; a.wmat = n->w3; a.bias = n->params + NET_OFF_B3;
  a.out = out; a.out_pstride = out_pstride; a.out_pitch = out_pitch; a.out_bstride = out_bstride;
  a.apply = apply; a.out_scale = out_scale;
  k_net_conv<2><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fvna

extern "C" {

int fvna_net_create(const float *params, fvna_net **out) {
  if (!out || !params) return FVNA_ERR_ARG;
  *out = nullptr;
  fvna_net *n = new (std::nothrow) fvna_net();
  if (!n) return FVNA_ERR_OOM;
  cudaError_t e = cudaMalloc(&n->params, 4 * FVNA_NET_PARAMS * sizeof(float));
  if (e == cudaSuccess) {
    n->grads = n->params + FVNA_NET_PARAMS;
    n->m = n->grads + FVNA_NET_PARAMS;
    n->v = n->m + FVNA_NET_PARAMS;
    e = cudaMalloc(&n->w1, (size_t)(32 * K1 + 32 * KH + 8 * KH) * sizeof(__nv_bfloat16));
  }
  if (e == cudaSuccess) {
    n->w2 = n->w1 + 32 * K1;
    n->w3 = n->w2 + 32 * KH;
    e = cudaMalloc(&n->loss, sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc(&n->nin, sizeof(long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(n->params, params, FVNA_NET_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, 2 * FVNA_NET_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = net_pack(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fvna_net_destroy(n);
    return cerr(e);
  }
  *out = n;
  return FVNA_OK;
}

void fvna_net_destroy(fvna_net *n) {
  if (!n) return;
  cudaDeviceSynchronize();
  net_free_buffers(n);
  cudaFree(n->params);
  cudaFree(n->w1);
  cudaFree(n->loss);
  cudaFree(n->nin);
  delete n;
}

int fvna_net_params(fvna_net *n, float *dst, const float *src) {
  if (!n || (!dst && !src)) return FVNA_ERR_ARG;
  if (src) {
    NCK(cudaMemcpy(n->params, src, FVNA_NET_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    NCK(net_pack(n, 0));
  }
  if (dst) NCK(cudaMemcpy(dst, n->params, FVNA_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
  NCK(cudaDeviceSynchronize());
  return FVNA_OK;
}

int fvna_net_forward(fvna_net *n, int B, int H, int W, const float *x, float in_scale, float *y,
                     unsigned short *h1_out, unsigned short *h2_out, void *stream) {
  if (!n || !x || !y || B < 1 || H < 1 || W < 1) return FVNA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = net_reserve(n, (long long)B * H * W);
  if (rc != FVNA_OK) return rc;
  long long hw = (long long)H * W;
  NCK(net_forward_launch(n, B, H, W, x, hw, W, 3 * hw, in_scale, y, hw, W, 3 * hw, 0, 1.f, n->h1,
                         n->h2, s));
  size_t hb = (size_t)B * hw * CH * sizeof(__nv_bfloat16);
  if (h1_out) NCK(cudaMemcpyAsync(h1_out, n->h1, hb, cudaMemcpyDeviceToDevice, s));
  if (h2_out) NCK(cudaMemcpyAsync(h2_out, n->h2, hb, cudaMemcpyDeviceToDevice, s));
  NCK(cudaStreamSynchronize(s));
  return FVNA_OK;
}

int fvna_net_backward(fvna_net *n, int B, int H, int W, const float *x, float in_scale,
                      const float *gy, float *grads, void *stream) {
  if (!n || !x || !gy || B < 1 || H < 1 || W < 1) return FVNA_ERR_ARG;
  if ((long long)B * H * W > n->cap_pix) return FVNA_ERR_ARG;  // needs the forward's activations
  cudaStream_t s = (cudaStream_t)stream;
  float *g = n->grads;
  long long tot = (long long)B * CH * H * W;
  int blocks = (int)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
  k_net_bwd_weight<CH, 3, false><<<3 * CH, 256, 0, s>>>(gy, n->h2, nullptr, 1.f,
                                                       g + NET_OFF_W3, g + NET_OFF_B3, B, H, W);
  k_net_bwd_input<3><<<blocks, 256, 0, s>>>(gy, n->w3, n->h2, n->gh2, B, H, W);
  k_net_bwd_weight<CH, CH, false><<<CH * CH, 256, 0, s>>>(n->gh2, n->h1, nullptr, 1.f,
                                                          g + NET_OFF_W2, g + NET_OFF_B2, B, H, W);
  k_net_bwd_input<CH><<<blocks, 256, 0, s>>>(n->gh2, n->w2, n->h1, n->gh1, B, H, W);
  k_net_bwd_weight<3, CH, true><<<CH * 3, 256, 0, s>>>(n->gh1, nullptr, x, in_scale,
                                                       g + NET_OFF_W1, g + NET_OFF_B1, B, H, W);
  NCK(cudaGetLastError());
  if (grads) NCK(cudaMemcpyAsync(grads, g, FVNA_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice, s));
  NCK(cudaStreamSynchronize(s));
  return FVNA_OK;
}

int fvna_net_train_step(fvna_net *n, int B, int H, int W, const float *x, float in_scale,
                        const float *target, int margin, const int *edges, float lr, double *loss,
                        void *stream) {
  if (!n || !x || !target || B < 1 || H < 1 || W < 1 || !(lr > 0.f)) return FVNA_ERR_ARG;
  if (margin < 0 || 2 * margin >= H || 2 * margin >= W) return FVNA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = net_reserve(n, (long long)B * H * W);
  if (rc != FVNA_OK) return rc;
  long long hw = (long long)H * W;
  NCK(net_forward_launch(n, B, H, W, x, hw, W, 3 * hw, in_scale, n->y, hw, W, 3 * hw, 0, 1.f,
                         n->h1, n->h2, s));
  NCK(cudaMemsetAsync(n->loss, 0, sizeof(double), s));
  long long ny = 3LL * B * hw;
  k_net_count<<<1, 32, 0, s>>>(B, H, W, margin, edges, n->nin);
  k_net_mse<<<(int)((ny + 255) / 256 < 2048 ? (ny + 255) / 256 : 2048), 256, 0, s>>>(
      n->y, target, n->g3, ny, H, W, margin, edges, n->nin, n->loss);
  NCK(cudaGetLastError());
  rc = fvna_net_backward(n, B, H, W, x, in_scale, n->g3, nullptr, stream);
  if (rc != FVNA_OK) return rc;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
  k_net_adam<<<(FVNA_NET_PARAMS + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->m, n->v,
                                                           FVNA_NET_PARAMS, lr, b1, b2, 1e-8f, c1, c2);
  NCK(cudaGetLastError());
  NCK(net_pack(n, s));
  if (loss) NCK(cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  NCK(cudaStreamSynchronize(s));
  return FVNA_OK;
}

}  // extern "C"
