// Elementwise kernels: site initialisation (Algorithm 1) and the recombination
// of the five sites into the posterior (Eq. Q_x_final).
#include "internal.cuh"

namespace eptv {

namespace {

constexpr int kEwThreads = 256;

inline int ew_blocks(long long n) {
  long long b = (n + kEwThreads - 1) / kEwThreads;
  if (b > (1ll << 20)) b = 1ll << 20;
  return (int)(b < 1 ? 1 : b);
}

// q_{x,0} = N(mu0, xi I) and q_{x,k} = N(0, var_cap I), in natural parameters.
__global__ void init_sites_kernel(float* tau0, float* nu0, float* tp, float* np,
                                  const float* mu0, long long n, float inv_xi, float min_tau) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    tau0[p] = inv_xi;
    nu0[p] = mu0[p] * inv_xi;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      tp[s * n + p] = min_tau;
      np[s * n + p] = 0.0f;
    }
  }
}

// Option 1 of the EM statistic (Sec. IV, Eq. ax): a_x = E_{Q(x)} sum_{(i,j) in V}
// |x_i - x_j| under the diagonal Gaussian Q(x) of Eq. Q_x_final, i.e. the sum over
// all edges of the folded-normal mean of N(mu_i - mu_j, s_i^2 + s_j^2).  Pixel p
// takes the edge to its right neighbour (V1 or V2) and the one below it (V3 or
// V4); on the free boundary the wrap-around edges do not exist.  One FP64 partial
// per block, summed in a fixed order by the E|u| reduction.
__device__ __forceinline__ void moments_at(const float* tau0, const float* nu0, const float* tp,
                                           const float* np, long long n, long long p, float& m,
                                           float& v) {
  float t = tau0[p], s = nu0[p];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    t += tp[k * n + p];
    s += np[k * n + p];
  }
  v = 1.0f / t;
  m = s * v;
}

__device__ __forceinline__ double folded_mean_edge(float mi, float vi, float mj, float vj) {
  const double m = (double)mi - (double)mj, v = (double)vi + (double)vj;
  const double s = sqrt(v);
  return s * 0.79788456080286536 * exp(-0.5 * m * m / v) + m * erf(m / (1.4142135623730951 * s));
}

// Rows [row_lo, row_hi) take their right and lower edges; periodic_rows: the
// last row's lower edge wraps to row 0 (a row block of a sharded image: no wrap,
// its lower halo rows are in the block).
__global__ void ax_kernel(const float* tau0, const float* nu0, const float* tp, const float* np,
                          int height, int width, int periodic, int periodic_rows, int row_lo,
                          int row_hi, double* partial) {
  const long long n = (long long)height * width;
  const long long p_lo = (long long)row_lo * width, p_hi = (long long)row_hi * width;
  double acc = 0.0;
  for (long long p = p_lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; p < p_hi;
       p += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(p / width), c = (int)(p - (long long)r * width);
    float m, v, mq, vq;
    moments_at(tau0, nu0, tp, np, n, p, m, v);
    if (c + 1 < width || (periodic && width > 1)) {
      const long long q = (long long)r * width + (c + 1 < width ? c + 1 : 0);
      moments_at(tau0, nu0, tp, np, n, q, mq, vq);
      acc += folded_mean_edge(m, v, mq, vq);
    }
    if (r + 1 < height || (periodic_rows && height > 1)) {
      const long long q = (long long)(r + 1 < height ? r + 1 : 0) * width + c;
      moments_at(tau0, nu0, tp, np, n, q, mq, vq);
      acc += folded_mean_edge(m, v, mq, vq);
    }
  }
  __shared__ double red[kEwThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEwThreads / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// Convergence check of the inner EP run of EP-EM: the posterior mean replaces
// prev, and out[0] / out[1] receive max |mean - prev| and max |mean| as float
// bits (non-negative floats order like their bit patterns, so atomicMax is exact
// and independent of the order of the blocks).  out starts at zero.
__global__ void mean_change_kernel(const float* __restrict__ tau0, const float* __restrict__ nu0,
                                   const float* __restrict__ tp, const float* __restrict__ np,
                                   long long n, float* prev, unsigned* out) {
  float dmax = 0.f, mmax = 0.f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float t = tau0[p], v = nu0[p];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      t += tp[s * n + p];
      v += np[s * n + p];
    }
    const float m = v / t;
    dmax = fmaxf(dmax, fabsf(m - prev[p]));
    mmax = fmaxf(mmax, fabsf(m));
    prev[p] = m;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
    mmax = fmaxf(mmax, __shfl_down_sync(0xffffffffu, mmax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(dmax));
    atomicMax(out + 1, __float_as_uint(mmax));
  }
}

// Denoising with a diagonal noise covariance: site 0 = (1 / xi_p, y_p / xi_p),
// the exact likelihood site (Eq. tilted_P_1 with H = I).
__global__ void site0_noise_kernel(float* tau0, float* nu0, const float* y, const float* xi,
                                   long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float t = 1.0f / xi[p];
    tau0[p] = t;
    nu0[p] = y[p] * t;
  }
}

// mean = (sum_s nu_s) / (sum_s tau_s), var = 1 / (sum_s tau_s)
__global__ void posterior_kernel(const float* __restrict__ tau0, const float* __restrict__ nu0,
                                 const float* __restrict__ tp, const float* __restrict__ np,
                                 long long n, float* mean, float* var) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float t = tau0[p], v = nu0[p];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      t += tp[s * n + p];
      v += np[s * n + p];
    }
    const float sig = 1.0f / t;
    if (mean) mean[p] = v * sig;
    if (var) var[p] = sig;
  }
}

// Warm start: sites from the warm-start network's output for the observation y:
// the predicted posterior mean is y + out[0] and site s gets the precision
// exp(out[1 + s] - log(xi)) (prior sites capped below at min_tau) and the mean of
// the prediction, nu_s = tau_s * mean.  keep_site0: site 0 is exact from the
// start (denoising) and stays.  site0_only: the prior sites keep their values
// and only site 0 is set; keep_site0 and not site0_only: only the prior sites.
__global__ void warm_start_kernel(float* tau0, float* nu0, float* tp, float* np, const float* out,
                                  const float* y, float log_xi, long long n, float min_tau,
                                  int keep_site0, int site0_only) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float mean = y[p] + out[p];
    if (!keep_site0) {
      const float t0 = expf(out[n + p] - log_xi);
      tau0[p] = t0;
      nu0[p] = t0 * mean;
    }
    if (site0_only) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float t = expf(out[(2 + s) * n + p] - log_xi);
      if (!(t >= min_tau)) t = min_tau;
      tp[s * n + p] = t;
      np[s * n + p] = t * mean;
    }
  }
}

}  // namespace

void launch_warm_start(float* tau0, float* nu0, float* tp, float* np, const float* out,
                       const float* y, float log_xi, long long n, float min_tau, bool keep_site0,
                       bool site0_only, cudaStream_t s) {
  warm_start_kernel<<<ew_blocks(n), kEwThreads, 0, s>>>(tau0, nu0, tp, np, out, y, log_xi, n,
                                                        min_tau, keep_site0 ? 1 : 0,
                                                        site0_only ? 1 : 0);
}

void launch_init_sites(float* tau0, float* nu0, float* tp, float* np, const float* mu0, long long n,
                       float inv_xi, float min_tau, cudaStream_t s) {
  init_sites_kernel<<<ew_blocks(n), kEwThreads, 0, s>>>(tau0, nu0, tp, np, mu0, n, inv_xi, min_tau);
}

void launch_posterior(const float* tau0, const float* nu0, const float* tp, const float* np,
                      long long n, float* mean, float* var, cudaStream_t s) {
  posterior_kernel<<<ew_blocks(n), kEwThreads, 0, s>>>(tau0, nu0, tp, np, n, mean, var);
}

void launch_ax(const float* tau0, const float* nu0, const float* tp, const float* np, int height,
               int width, int periodic, double* partial, int n_partial, cudaStream_t s) {
  ax_kernel<<<n_partial, kEwThreads, 0, s>>>(tau0, nu0, tp, np, height, width, periodic, periodic,
                                             0, height, partial);
}

void launch_ax_block(const float* tau0, const float* nu0, const float* tp, const float* np,
                     int height, int width, int periodic, int row_lo, int row_hi, double* partial,
                     int n_partial, cudaStream_t s) {
  ax_kernel<<<n_partial, kEwThreads, 0, s>>>(tau0, nu0, tp, np, height, width, periodic, 0, row_lo,
                                             row_hi, partial);
}

void launch_mean_change(const float* tau0, const float* nu0, const float* tp, const float* np,
                        long long n, float* prev, unsigned* out, cudaStream_t s) {
  mean_change_kernel<<<ew_blocks(n) < 1024 ? ew_blocks(n) : 1024, kEwThreads, 0, s>>>(tau0, nu0, tp,
                                                                                      np, n, prev, out);
}

void launch_site0_noise(float* tau0, float* nu0, const float* y, const float* xi, long long n,
                        cudaStream_t s) {
  site0_noise_kernel<<<ew_blocks(n), kEwThreads, 0, s>>>(tau0, nu0, y, xi, n);
}

}  // namespace eptv
