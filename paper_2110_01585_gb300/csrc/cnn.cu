// Learned warm start: the building blocks of a small fully convolutional network
// (3x3 convolutions on the torus with bias and ReLU, their backward pass, the
// Adam step, the training loss) and nothing else.  The paper has no
// counterpart; its EP sweeps correct whatever the network's output gets wrong.
//
// Arrays are float32 NCHW.  The convolution is a direct one on CUDA cores: a
// block computes a 16 x 16 pixel tile of one image for all (up to 32) output
// channels, staging 8 input channels at a time with a one-pixel circular halo
// in shared memory; each input value is reused for every output channel from
// registers, and the weights of a (channel, tap) are read as float4 broadcasts.
// The weight gradient is a per-tile partial sum over pixels, reduced over tiles
// in a fixed order (no atomics), so training is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace eptv {

namespace {

constexpr int kT = 16;        // tile side (pixels)
constexpr int kHalo = kT + 2;
constexpr int kCC = 8;        // input channels staged per pass
constexpr int kMaxOut = 32;   // output channels per launch
constexpr int kThreads = kT * kT;
constexpr int kWarmOut = 6;   // network outputs: mean residual, five site log-precisions

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// y[n, o] = b[o] + sum_c sum_tap w[o, c, tap] x[n, c, shifted by tap], ReLU optional.
__global__ void __launch_bounds__(kThreads) conv3x3_fwd_kernel(int cin, int cout, int H, int W,
                                                                const float* __restrict__ x,
                                                                const float* __restrict__ w,
                                                                const float* __restrict__ b,
                                                                int relu, float* __restrict__ y) {
  __shared__ float xs[kCC][kHalo][kHalo];
  __shared__ __align__(16) float ws[kCC][9][kMaxOut];
  const int n = blockIdx.z;
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  float acc[kMaxOut];
#pragma unroll
  for (int o = 0; o < kMaxOut; ++o) acc[o] = (b && o < cout) ? b[o] : 0.0f;
  const long long plane = (long long)H * W;
  for (int c0 = 0; c0 < cin; c0 += kCC) {
    const int cc = min(kCC, cin - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cc * kHalo * kHalo; i += kThreads) {
      const int c = i / (kHalo * kHalo), r = (i / kHalo) % kHalo, q = i % kHalo;
      const int gr = wrapi(y0 - 1 + r, H), gq = wrapi(x0 - 1 + q, W);
      xs[c][r][q] = x[((long long)n * cin + c0 + c) * plane + (long long)gr * W + gq];
    }
    for (int i = threadIdx.x; i < kCC * 9 * kMaxOut; i += kThreads) {
      const int c = i / (9 * kMaxOut), tap = (i / kMaxOut) % 9, o = i % kMaxOut;
      ws[c][tap][o] = (c < cc && o < cout) ? w[((long long)o * cin + c0 + c) * 9 + tap] : 0.0f;
    }
    __syncthreads();
    for (int c = 0; c < cc; ++c) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float xv = xs[c][ty + tap / 3][tx + tap % 3];
        const float4* wv = reinterpret_cast<const float4*>(ws[c][tap]);
#pragma unroll
        for (int o4 = 0; o4 < kMaxOut / 4; ++o4) {
          const float4 q = wv[o4];
          acc[4 * o4 + 0] = fmaf(q.x, xv, acc[4 * o4 + 0]);
          acc[4 * o4 + 1] = fmaf(q.y, xv, acc[4 * o4 + 1]);
          acc[4 * o4 + 2] = fmaf(q.z, xv, acc[4 * o4 + 2]);
          acc[4 * o4 + 3] = fmaf(q.w, xv, acc[4 * o4 + 3]);
        }
      }
    }
  }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= W || gy >= H) return;
#pragma unroll
  for (int o = 0; o < kMaxOut; ++o) {
    if (o < cout) {
      const float v = relu ? fmaxf(acc[o], 0.0f) : acc[o];
      y[((long long)n * cout + o) * plane + (long long)gy * W + gx] = v;
    }
  }
}

// g = dy, masked by y > 0 when the layer had a ReLU (y = max(z, 0) > 0 iff z > 0).
__global__ void relu_mask_kernel(long long count, const float* dy, const float* y, float* g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    g[i] = (y == nullptr || y[i] > 0.0f) ? dy[i] : 0.0f;
}

// Weights of the input gradient: dx = conv3x3(g, wt) with wt[c, o, 8 - tap] = w[o, c, tap].
__global__ void transpose_weights_kernel(int cin, int cout, const float* w, float* wt) {
  const int total = cin * cout * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int c = i / (cout * 9), o = (i / 9) % cout, tap = i % 9;
    wt[i] = w[((long long)o * cin + c) * 9 + (8 - tap)];
  }
}

// Partial weight and bias gradients of one 16 x 16 tile of one image:
// part[blk][o][c][tap] = sum_p g[o, p] x[c, p shifted by tap], part[blk][cout*cin*9 + o] = sum_p g[o, p].
__global__ void __launch_bounds__(kThreads) conv3x3_dw_kernel(int cin, int cout, int H, int W,
                                                               const float* __restrict__ x,
                                                               const float* __restrict__ g,
                                                               float* __restrict__ part) {
  __shared__ float gs[kMaxOut][kThreads + 1];
  __shared__ float xs[kCC][kHalo][kHalo];
  const int n = blockIdx.z;
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  const int blk = (n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const long long plane = (long long)H * W;
  const long long stride = (long long)cout * cin * 9 + cout;
  float* out = part + blk * stride;
  // the tile's output gradient (zero outside the image)
  for (int i = threadIdx.x; i < kMaxOut * kThreads; i += kThreads) {
    const int o = i / kThreads, p = i % kThreads;
    const int gx = x0 + p % kT, gy = y0 + p / kT;
    gs[o][p] = (o < cout && gx < W && gy < H) ? g[((long long)n * cout + o) * plane + (long long)gy * W + gx]
                                              : 0.0f;
  }
  __syncthreads();
  const int o = threadIdx.x % kMaxOut, cg = threadIdx.x / kMaxOut;  // 32 outputs x 8 channels
  if (cg == 0 && o < cout) {
    float s = 0.0f;
    for (int p = 0; p < kThreads; ++p) s += gs[o][p];
    out[(long long)cout * cin * 9 + o] = s;
  }
  for (int c0 = 0; c0 < cin; c0 += kCC) {
    const int cc = min(kCC, cin - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cc * kHalo * kHalo; i += kThreads) {
      const int c = i / (kHalo * kHalo), r = (i / kHalo) % kHalo, q = i % kHalo;
      const int gr = wrapi(y0 - 1 + r, H), gq = wrapi(x0 - 1 + q, W);
      xs[c][r][q] = x[((long long)n * cin + c0 + c) * plane + (long long)gr * W + gq];
    }
    __syncthreads();
    if (cg < cc && o < cout) {
      float acc[9] = {};
      for (int p = 0; p < kThreads; ++p) {
        const float gv = gs[o][p];
        const int px = p % kT, py = p / kT;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) acc[tap] = fmaf(gv, xs[cg][py + tap / 3][px + tap % 3], acc[tap]);
      }
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) out[((long long)o * cin + c0 + cg) * 9 + tap] = acc[tap];
    }
  }
}

// dst[i] = sum over blocks of part[blk][i], in block order.
__global__ void reduce_parts_kernel(const float* part, long long stride, int nblk, float* dw,
                                    float* db, int nw) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k * stride + i];
    if (i < nw) dw[i] = (float)s;
    else db[i - nw] = (float)s;
  }
}

__global__ void adam_kernel(long long count, float* p, const float* g, float* m, float* v,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Targets of the warm start from a labelled EP state: out0 -> mean - y and
// out[1 + s] -> log(tau_s) + log(xi) for the five sites s.  dout = dL/dout of
// L = mean over images and pixels of w_mu (out0 - t0)^2 + (1/5) sum_s (out[1+s] - t[1+s])^2;
// loss += block sums.
__global__ void warmstart_loss_kernel(int n, long long hw, const float* out, const float* y,
                                      const float* mean, const float* tau, const float* log_xi,
                                      float w_mu, float* dout, double* loss) {
  const double inv = 1.0 / ((double)n * hw);
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * hw;
       i += (long long)gridDim.x * blockDim.x) {
    const long long img = i / hw, p = i - img * hw;
    const float* o = out + img * kWarmOut * hw + p;
    float* d = dout + img * kWarmOut * hw + p;
    const float r0 = o[0] - (mean[i] - y[i]);
    d[0] = (float)(2.0 * w_mu * r0 * inv);
    double acc = (double)w_mu * r0 * r0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float t = logf(tau[(img * 5 + k) * hw + p]) + log_xi[img];
      const float r = o[(1 + k) * hw] - t;
      d[(1 + k) * hw] = (float)(0.4 * r * inv);
      acc += 0.2 * (double)r * r;
    }
    s += acc;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

inline int ew_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

bool conv_args_ok(int n, int cin, int cout, int h, int w) {
  return n >= 1 && cin >= 1 && cout >= 1 && cout <= kMaxOut && h >= 1 && w >= 1 &&
         (long long)n * (cin > cout ? cin : cout) * h * w < (1ll << 40);
}

inline ep_tv_status launch_status() {
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

long long tiles(int h, int w) { return (long long)((w + kT - 1) / kT) * ((h + kT - 1) / kT); }

}  // namespace
}  // namespace eptv

using namespace eptv;

extern "C" {

ep_tv_status ep_tv_conv3x3_forward(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                   int32_t width, const float* x, const float* weight,
                                   const float* bias, int32_t relu, float* y, void* cuda_stream) {
  if (!conv_args_ok(n, cin, cout, height, width) || !x || !weight || !y || x == y) return EP_TV_ERR_ARG;
  if (n > 65535) return EP_TV_ERR_ARG;
  dim3 grid((width + kT - 1) / kT, (height + kT - 1) / kT, n);
  conv3x3_fwd_kernel<<<grid, kThreads, 0, (cudaStream_t)cuda_stream>>>(cin, cout, height, width, x,
                                                                        weight, bias, relu != 0, y);
  return launch_status();
}

size_t ep_tv_conv3x3_backward_work(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                   int32_t width) {
  if (!conv_args_ok(n, cin, cout, height, width)) return 0;
  const long long nblk = tiles(height, width) * n;
  const long long stride = (long long)cout * cin * 9 + cout;
  return sizeof(float) * ((long long)n * cout * height * width + (long long)cin * cout * 9 + nblk * stride);
}

ep_tv_status ep_tv_conv3x3_backward(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                    int32_t width, const float* x, const float* weight,
                                    const float* y, const float* dy, float* dx, float* dweight,
                                    float* dbias, void* work, size_t work_bytes, void* cuda_stream) {
  if (!conv_args_ok(n, cin, cout, height, width) || !x || !weight || !dy || !dweight || !dbias || !work)
    return EP_TV_ERR_ARG;
  if (n > 65535 || (dx && cin > kMaxOut)) return EP_TV_ERR_ARG;
  if (work_bytes < ep_tv_conv3x3_backward_work(n, cin, cout, height, width)) return EP_TV_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long count = (long long)n * cout * height * width;
  float* g = (float*)work;
  float* wt = g + count;
  float* part = wt + (long long)cin * cout * 9;
  relu_mask_kernel<<<ew_grid(count), 256, 0, s>>>(count, dy, y, g);
  dim3 grid((width + kT - 1) / kT, (height + kT - 1) / kT, n);
  conv3x3_dw_kernel<<<grid, kThreads, 0, s>>>(cin, cout, height, width, x, g, part);
  const long long stride = (long long)cout * cin * 9 + cout;
  const int nblk = (int)(tiles(height, width) * n);
  reduce_parts_kernel<<<ew_grid(stride), 256, 0, s>>>(part, stride, nblk, dweight, dbias,
                                                      cout * cin * 9);
  if (dx) {
    transpose_weights_kernel<<<ew_grid((long long)cin * cout * 9), 256, 0, s>>>(cin, cout, weight, wt);
    conv3x3_fwd_kernel<<<grid, kThreads, 0, s>>>(cout, cin, height, width, g, wt, nullptr, 0, dx);
  }
  return launch_status();
}

ep_tv_status ep_tv_adam_step(int64_t count, float* param, const float* grad, float* m, float* v,
                             int32_t t, float lr, float beta1, float beta2, float eps,
                             void* cuda_stream) {
  if (count < 1 || !param || !grad || !m || !v || t < 1) return EP_TV_ERR_ARG;
  const float c1 = (float)(1.0 - pow((double)beta1, t)), c2 = (float)(1.0 - pow((double)beta2, t));
  adam_kernel<<<ew_grid(count), 256, 0, (cudaStream_t)cuda_stream>>>(count, param, grad, m, v, lr,
                                                                       beta1, beta2, eps, c1, c2);
  return launch_status();
}

ep_tv_status ep_tv_warmstart_loss(int32_t n, int32_t height, int32_t width, const float* out,
                                  const float* y, const float* mean, const float* tau,
                                  const float* log_xi, float w_mean, float* dout, double* loss,
                                  void* cuda_stream) {
  if (n < 1 || height < 1 || width < 1 || !out || !y || !mean || !tau || !log_xi || !dout || !loss)
    return EP_TV_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return EP_TV_ERR_CUDA;
  const long long hw = (long long)height * width;
  warmstart_loss_kernel<<<ew_grid(n * hw), 256, 0, s>>>(n, hw, out, y, mean, tau, log_xi, w_mean,
                                                        dout, loss);
  return launch_status();
}

}  // extern "C"
