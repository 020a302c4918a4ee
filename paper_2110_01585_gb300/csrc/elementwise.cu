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

}  // namespace eptv
