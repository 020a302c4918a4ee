// Likelihood-site (q_{x,0}) update for non-diagonal H^T H: interface between
// the C ABI and the operator-specific kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/ep_tv.h"

namespace eptv {

struct Tracer;

struct LikelihoodConfig {
  const ep_tv_operator* op;
  const ep_tv_params* p;
  int height, width;
  long long n;
  int m;
  const float* y;  // device copy owned by the context
};

struct LikelihoodState;

// Builds operator data and solver buffers; writes the initial mean of site 0
// (Algorithm 1: y; H^T y when y is shorter than x) into mu0 (device, n floats).
ep_tv_status likelihood_create(const LikelihoodConfig& cfg, cudaStream_t s, LikelihoodState** out,
                               float* mu0);
void likelihood_destroy(LikelihoodState* L);
// Clears solver warm starts (called on init/reset).
ep_tv_status likelihood_reset(LikelihoodState* L, cudaStream_t s);
ep_tv_status likelihood_set_probes(LikelihoodState* L, const float* eps1, const float* eps2,
                                   int n_samples, cudaStream_t s);
// Diagonal noise covariance (dense operator; EP_TV_ERR_UNSUPPORTED otherwise).
ep_tv_status likelihood_set_noise(LikelihoodState* L, const float* xi_m, cudaStream_t s);
// Whether the last update ran as a graph replay (device-driven solver loops).
bool likelihood_graph_last(const LikelihoodState* L);
// One q_{x,0} update: cavity from sites 1..4, tilted moments of P_0
// (Eq. tilted_P_1), site update (Eq. update_q0_x) with cap and damping.
// tau0, nu0: likelihood site (updated in place); tp, np: prior sites, [4][N].
ep_tv_status likelihood_update(LikelihoodState* L, float* tau0, float* nu0, const float* tp,
                               const float* np, unsigned* status, unsigned long long* counters,
                               Tracer* tr, cudaStream_t s);
// Algorithmic DRAM bytes per unit of the traced likelihood kernels.
double likelihood_bytes_per_unit(const LikelihoodState* L, int kernel);
int likelihood_systems(const LikelihoodState* L);
int likelihood_last_iters(const LikelihoodState* L);
// Outer refinement passes and final relative residuals of the last update.
void likelihood_report(const LikelihoodState* L, int* outer, double* relres_mean,
                       double* relres_probe);
size_t likelihood_state_bytes(const LikelihoodState* L);
ep_tv_status likelihood_state_export(LikelihoodState* L, void* host, cudaStream_t s);
ep_tv_status likelihood_state_import(LikelihoodState* L, const void* host, cudaStream_t s);

// Dense sensing matrix (compressive sensing): Woodbury form in FP64 (cs.cu).
struct CsState;
ep_tv_status cs_create(const LikelihoodConfig& cfg, cudaStream_t s, CsState** out, float* mu0);
void cs_destroy(CsState* S);
// Diagonal noise covariance: K = diag(xi_m) + A C A^T (xi_m DEVICE, M floats, copied).
ep_tv_status cs_set_noise(CsState* S, const float* xi_m, cudaStream_t s);
ep_tv_status cs_update(CsState* S, float* tau0, float* nu0, const float* tp, const float* np,
                       unsigned* status, unsigned long long* counters, Tracer* tr, cudaStream_t s);
double cs_flops(const CsState* S);      // FP64 CUDA-core flops of the last update
double cs_mma_flops(const CsState* S);  // BF16 tensor flops of the last update

}  // namespace eptv
