// C ABI of libeptv: context management, argument checking, the sweep driver
// (Algorithm 1) and the EM step (Algorithm 2).  Compute runs in the kernels of
// the other translation units; this file only orders their launches.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "likelihood.cuh"

using namespace eptv;

struct ep_tv_ctx {
  ep_tv_operator op;
  ep_tv_params p;
  int height = 0, width = 0;
  long long n = 0;
  int m = 0;
  cudaStream_t stream = nullptr;
  int device = 0;

  float* tau0 = nullptr;      // [N] likelihood site
  float* nu0 = nullptr;
  float* ptau[2] = {nullptr, nullptr};  // [4][N] prior sites, two buffers
  float* pnu[2] = {nullptr, nullptr};
  int cur = 0;                // buffer holding the current prior sites
  float* y = nullptr;         // [M]
  float* mu0 = nullptr;       // initial mean of site 0 (y, or H^T y for DENSE)
  double* dscal = nullptr;    // DS_*
  double* abar_partial = nullptr;
  int n_partial = 0;
  unsigned* status = nullptr;
  unsigned long long* counters = nullptr;
  LikelihoodState* lik = nullptr;  // CONV_PERIODIC / DENSE
  Tracer tracer;
  unsigned long long cnt_base[DC_COUNT] = {};  // counters when tracing was enabled
  bool failed = false;
  long long sweeps = 0;
  // Sweeps of a context without a likelihood solver replayed from a captured
  // graph: one per starting buffer parity, for the EM period it was captured with.
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_em[2] = {-1, -1};
  int graph_len[2] = {0, 0};
  long long graph_sweeps = 0;  // sweeps run from graph replays (this context or its batch)
  float* xi_plane = nullptr;  // [M] noise variances of a diagonal noise covariance, or NULL
  // Row block of a sharded image (ep_tv_init_block); rows = 0 for a whole image.
  int blk_rows = 0, blk_top = 0, blk_bottom = 0;  // own rows, halo rows above and below
  // EP-EM convergence checks (allocated on the first ep_tv_ep_em call)
  float* mu_prev = nullptr;     // [N] posterior mean after the previous sweep
  unsigned* d_change = nullptr; // max |change|, max |mean| (float bits)
  unsigned* h_change = nullptr; // pinned copy
};

namespace {

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return EP_TV_ERR_CUDA;  \
  } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

namespace eptv {
// The edge factor's parameters (Sec. II-B): beta for l1-TV (checked by the
// callers), omega in (0, 1) and positive component variances for the mixtures.
bool prior_params_ok(const ep_tv_params* p) {
  if (p->em_option < 1 || p->em_option > 3) return false;
  switch (p->prior) {
    case EP_TV_PRIOR_L1: return true;
    case EP_TV_PRIOR_MOG2:
      return p->omega > 0.0 && p->omega < 1.0 && finite_pos(p->s1_sq) && finite_pos(p->s2_sq);
    case EP_TV_PRIOR_BG: return p->omega > 0.0 && p->omega < 1.0 && finite_pos(p->s1_sq);
  }
  return false;
}

void set_prior_args(SweepArgs& a, const ep_tv_params* p) {
  a.prior = p->prior;
  a.em_option = p->em_option;
  a.mix_logit = 0.f;
  a.mix_v1 = a.mix_v2 = 0.f;
  if (p->prior != EP_TV_PRIOR_L1) {
    a.mix_logit = (float)std::log((1.0 - p->omega) / p->omega);
    a.mix_v1 = (float)p->s1_sq;
    a.mix_v2 = p->prior == EP_TV_PRIOR_MOG2 ? (float)p->s2_sq : 0.f;
  }
}
}  // namespace eptv

namespace {

ep_tv_status check_params(const ep_tv_operator* op, const ep_tv_params* p) {
  if (!op || !p) return EP_TV_ERR_ARG;
  if (op->height < 1 || op->width < 1) return EP_TV_ERR_ARG;
  if ((long long)op->height * op->width > (1ll << 31)) return EP_TV_ERR_ARG;
  if (!finite_pos(p->xi)) return EP_TV_ERR_ARG;
  if (!(std::isfinite(p->beta) && p->beta >= 0.0)) return EP_TV_ERR_ARG;
  if (!(p->damping > 0.0 && p->damping <= 1.0)) return EP_TV_ERR_ARG;
  if (!finite_pos(p->var_cap)) return EP_TV_ERR_ARG;
  if (p->periodic != 0 && p->periodic != 1) return EP_TV_ERR_ARG;
  if (p->periodic && ((op->height % 2) || (op->width % 2))) return EP_TV_ERR_ARG;
  if (p->order_mode != 0 && p->order_mode != 1) return EP_TV_ERR_ARG;
  if (p->precision != 0 && p->precision != 1) return EP_TV_ERR_ARG;
  if (!prior_params_ok(p)) return EP_TV_ERR_ARG;
  const long long n = (long long)op->height * op->width;
  switch (op->op) {
    case EP_TV_OP_IDENTITY:
      if (op->m != n) return EP_TV_ERR_ARG;
      break;
    case EP_TV_OP_CONV_PERIODIC:
      if (op->m != n || !op->kernel) return EP_TV_ERR_ARG;
      if (op->kh < 1 || op->kw < 1 || !(op->kh % 2) || !(op->kw % 2)) return EP_TV_ERR_ARG;
      if (op->kh > op->height || op->kw > op->width) return EP_TV_ERR_ARG;
      if (p->rbmc_samples < 1 || p->cg_max_iter < 1 || !finite_pos(p->cg_rtol)) return EP_TV_ERR_ARG;
      break;
    case EP_TV_OP_DENSE:
      if (op->m < 1 || !op->dense) return EP_TV_ERR_ARG;
      break;
    case EP_TV_OP_HADAMARD: {
      if (op->m < 1 || op->m > n || !op->patterns) return EP_TV_ERR_ARG;
      if ((op->height & (op->height - 1)) || (op->width & (op->width - 1))) return EP_TV_ERR_ARG;
      std::vector<char> seen((size_t)n, 0);  // M distinct indices in [0, N)
      for (int i = 0; i < op->m; ++i) {
        const int32_t q = op->patterns[i];
        if (q < 0 || q >= n || seen[q]) return EP_TV_ERR_ARG;
        seen[q] = 1;
      }
      break;
    }
    default:
      return EP_TV_ERR_ARG;
  }
  return EP_TV_OK;
}

void drop_graphs(ep_tv_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    if (c->graph[b]) cudaGraphExecDestroy(c->graph[b]);
    c->graph[b] = nullptr;
    c->graph_em[b] = -1;
    c->graph_len[b] = 0;
  }
}

void free_ctx(ep_tv_ctx* c) {
  if (!c) return;
  drop_graphs(c);
  if (c->lik) likelihood_destroy(c->lik);
  cudaFree(c->tau0);
  cudaFree(c->nu0);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->ptau[b]);
    cudaFree(c->pnu[b]);
  }
  cudaFree(c->y);
  cudaFree(c->mu0);
  cudaFree(c->dscal);
  cudaFree(c->abar_partial);
  cudaFree(c->status);
  cudaFree(c->counters);
  cudaFree(c->mu_prev);
  cudaFree(c->xi_plane);
  cudaFree(c->d_change);
  if (c->h_change) cudaFreeHost(c->h_change);
  delete c;
}

ep_tv_status init_state(ep_tv_ctx* c) {
  const float inv_xi = (float)(1.0 / c->p.xi);
  const float min_tau = (float)(1.0 / c->p.var_cap);
  c->cur = 0;
  launch_init_sites(c->tau0, c->nu0, c->ptau[0], c->pnu[0], c->mu0, c->n, inv_xi, min_tau,
                    c->stream);
  if (c->xi_plane && c->op.op == EP_TV_OP_IDENTITY)
    launch_site0_noise(c->tau0, c->nu0, c->y, c->xi_plane, c->n, c->stream);
  double ds[DS_COUNT] = {c->p.beta, 0.0, 0.0, 0.0};
  CK(cudaMemcpyAsync(c->dscal, ds, sizeof(ds), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
  CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * DC_COUNT, c->stream));
  CK(cudaMemsetAsync(c->abar_partial, 0, sizeof(double) * c->n_partial, c->stream));
  if (c->lik) {
    ep_tv_status st = likelihood_reset(c->lik, c->stream);
    if (st != EP_TV_OK) return st;
  }
  CK(cudaStreamSynchronize(c->stream));
  c->failed = false;
  c->sweeps = 0;
  return EP_TV_OK;
}

ep_tv_status latched(ep_tv_ctx* c) {
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st) c->failed = true;
  if (st & ST_NONFINITE) return EP_TV_ERR_NONFINITE;
  if (st & ST_TIMEOUT) return EP_TV_ERR_TIMEOUT;
  if (st & ST_CG_NOCONV) return EP_TV_ERR_CG_NOCONV;
  return EP_TV_OK;
}

// Denoising contexts with i.i.d. noise form site 0 from y inside the prior pass;
// with a noise plane (and for the other operators) the site is stored.
bool site0_from_y(const ep_tv_ctx* c) { return c->op.op == EP_TV_OP_IDENTITY && !c->xi_plane; }

// The EM update (Sec. IV, Algorithm 2) on the device: the statistic that
// params.em_option selects, reduced in a fixed order, then beta = N / a.  Option 1
// (Eq. ax) is formed here from the sites (tp, np: the prior buffers holding the
// sweep's result); Options 2 and 3 were accumulated by the prior pass.
void launch_em(ep_tv_ctx* c, const float* tp, const float* np, cudaStream_t s) {
  if (c->p.em_option == 1)
    launch_ax(c->tau0, c->nu0, tp, np, c->height, c->width, c->p.periodic, c->abar_partial,
              c->n_partial, s);
  launch_abar_reduce(c->abar_partial, c->n_partial, c->dscal, (double)c->n, 1, s);
}

// Option 1 for a row block: the edges whose first pixel is one of its own rows.
void launch_ax_rows(ep_tv_ctx* c) {
  launch_ax_block(c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur], c->height, c->width,
                  c->p.periodic, c->blk_top, c->blk_top + c->blk_rows, c->abar_partial, c->n_partial,
                  c->stream);
}

SweepArgs sweep_args(ep_tv_ctx* c, int order) {
  SweepArgs a;
  a.tau0 = c->tau0;
  a.nu0 = c->nu0;
  a.tin = c->ptau[c->cur];
  a.nin = c->pnu[c->cur];
  a.tout = c->ptau[c->cur ^ 1];
  a.nout = c->pnu[c->cur ^ 1];
  a.y = c->y;
  a.inv_xi = (float)(1.0 / c->p.xi);
  a.height = c->height;
  a.width = c->width;
  a.n = c->n;
  a.periodic = c->p.periodic;
  a.periodic_rows = c->blk_rows ? 0 : c->p.periodic;
  a.count_lo = c->blk_rows ? c->blk_top : 0;
  a.count_hi = c->blk_rows ? c->blk_top + c->blk_rows : c->height;
  a.damping = (float)c->p.damping;
  a.min_tau = (float)(1.0 / c->p.var_cap);
  a.beta = c->dscal + DS_BETA;
  a.order = order;
  a.fp64_tail = c->p.precision == 0;
  set_prior_args(a, &c->p);
  a.abar_partial = c->abar_partial;
  a.status = c->status;
  a.counters = c->counters;
  return a;
}

// Graph of `period` sweeps (default order) of a context without a likelihood
// solver, starting from buffer parity c->cur; captured on first use and cached.
cudaGraphExec_t graph_for(ep_tv_ctx* c, int period, int em_every) {
  const int b = c->cur;
  if (c->graph[b] && c->graph_em[b] == em_every && c->graph_len[b] == period) return c->graph[b];
  if (c->graph[b]) {
    cudaGraphExecDestroy(c->graph[b]);
    c->graph[b] = nullptr;
  }
  prior_sweep_prewarm();  // occupancy queries and attributes outside the capture
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  int cur = c->cur;
  for (int t = 0; t < period; ++t) {
    SweepArgs a = sweep_args(c, 0x4321);
    a.tin = c->ptau[cur];
    a.nin = c->pnu[cur];
    a.tout = c->ptau[cur ^ 1];
    a.nout = c->pnu[cur ^ 1];
    launch_prior_sweep(a, site0_from_y(c), c->stream);
    cur ^= 1;
    if (em_every > 0 && (t + 1) % em_every == 0) launch_em(c, c->ptau[cur], c->pnu[cur], c->stream);
  }
  const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  cudaGraphExec_t exec = nullptr;
  if (e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  c->graph[b] = exec;
  c->graph_em[b] = em_every;
  c->graph_len[b] = period;
  return exec;
}

}  // namespace

extern "C" {

ep_tv_status ep_tv_default_params(ep_tv_params* p) {
  if (!p) return EP_TV_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->damping = 0.5;
  p->var_cap = 1e8;
  p->periodic = 1;
  p->order_mode = 0;
  p->rbmc_samples = 32;
  p->cg_max_iter = 1000;
  p->cg_rtol = 1e-9;
  p->precision = 0;
  p->seed = 1234;
  p->prior = EP_TV_PRIOR_L1;
  p->em_option = 3;
  return EP_TV_OK;
}

ep_tv_status ep_tv_init(const ep_tv_operator* op, const float* y, const ep_tv_params* p,
                        void* cuda_stream, ep_tv_ctx** out) {
  if (!out) return EP_TV_ERR_ARG;
  *out = nullptr;
  ep_tv_status st = check_params(op, p);
  if (st != EP_TV_OK) return st;
  if (!y) return EP_TV_ERR_ARG;
  ep_tv_ctx* c = new (std::nothrow) ep_tv_ctx();
  if (!c) return EP_TV_ERR_NOMEM;
  c->op = *op;
  c->op.patterns = nullptr;  // copied into the likelihood state below; not kept
  c->p = *p;
  c->height = op->height;
  c->width = op->width;
  c->n = (long long)op->height * op->width;
  c->m = op->m;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return EP_TV_ERR_CUDA; }
  c->n_partial = prior_sweep_blocks(c->height, c->width);
  bool ok = cudaMalloc(&c->tau0, sizeof(float) * c->n) == cudaSuccess &&
            cudaMalloc(&c->nu0, sizeof(float) * c->n) == cudaSuccess &&
            cudaMalloc(&c->ptau[0], sizeof(float) * 4 * c->n) == cudaSuccess &&
            cudaMalloc(&c->ptau[1], sizeof(float) * 4 * c->n) == cudaSuccess &&
            cudaMalloc(&c->pnu[0], sizeof(float) * 4 * c->n) == cudaSuccess &&
            cudaMalloc(&c->pnu[1], sizeof(float) * 4 * c->n) == cudaSuccess &&
            cudaMalloc(&c->y, sizeof(float) * c->m) == cudaSuccess &&
            cudaMalloc(&c->mu0, sizeof(float) * c->n) == cudaSuccess &&
            cudaMalloc(&c->dscal, sizeof(double) * DS_COUNT) == cudaSuccess &&
            cudaMalloc(&c->abar_partial, sizeof(double) * c->n_partial) == cudaSuccess &&
            cudaMalloc(&c->status, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&c->counters, sizeof(unsigned long long) * DC_COUNT) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return EP_TV_ERR_NOMEM;
  }
  if (cudaMemcpyAsync(c->y, y, sizeof(float) * c->m, cudaMemcpyDeviceToDevice, c->stream) !=
      cudaSuccess) {
    free_ctx(c);
    return EP_TV_ERR_CUDA;
  }
  if (op->op == EP_TV_OP_IDENTITY) {
    if (cudaMemcpyAsync(c->mu0, c->y, sizeof(float) * c->n, cudaMemcpyDeviceToDevice, c->stream) !=
        cudaSuccess) {
      free_ctx(c);
      return EP_TV_ERR_CUDA;
    }
  } else {
    LikelihoodConfig lc;
    lc.op = op;
    lc.p = p;
    lc.height = c->height;
    lc.width = c->width;
    lc.n = c->n;
    lc.m = c->m;
    lc.y = c->y;
    st = likelihood_create(lc, c->stream, &c->lik, c->mu0);
    if (st != EP_TV_OK) {
      free_ctx(c);
      return st;
    }
  }
  st = init_state(c);
  if (st != EP_TV_OK) {
    free_ctx(c);
    return st;
  }
  if (cudaGetLastError() != cudaSuccess) {
    free_ctx(c);
    return EP_TV_ERR_CUDA;
  }
  *out = c;
  return EP_TV_OK;
}

ep_tv_status ep_tv_init_noise(const ep_tv_operator* op, const float* y, const float* xi,
                              const ep_tv_params* p, void* cuda_stream, ep_tv_ctx** out) {
  if (!out) return EP_TV_ERR_ARG;
  *out = nullptr;
  if (!op || !p || !xi || !y) return EP_TV_ERR_ARG;
  if (op->op == EP_TV_OP_CONV_PERIODIC) return EP_TV_ERR_UNSUPPORTED;
  if (op->m < 1) return EP_TV_ERR_ARG;
  std::vector<float> h((size_t)op->m);
  CK(cudaMemcpy(h.data(), xi, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
  double sum = 0.0;
  for (float v : h) {
    if (!(std::isfinite(v) && v > 0.0f)) return EP_TV_ERR_ARG;
    sum += v;
  }
  ep_tv_params q = *p;
  q.xi = sum / (double)h.size();  // the scalar the initial site of Algorithm 1 takes for CS
  ep_tv_status st = ep_tv_init(op, y, &q, cuda_stream, out);
  if (st != EP_TV_OK) return st;
  ep_tv_ctx* c = *out;
  if (cudaMalloc(&c->xi_plane, sizeof(float) * op->m) != cudaSuccess) {
    cudaGetLastError();
    ep_tv_destroy(c);
    *out = nullptr;
    return EP_TV_ERR_NOMEM;
  }
  st = cudaMemcpyAsync(c->xi_plane, xi, sizeof(float) * op->m, cudaMemcpyDeviceToDevice, c->stream) ==
               cudaSuccess
           ? EP_TV_OK
           : EP_TV_ERR_CUDA;
  if (st == EP_TV_OK && c->lik) st = likelihood_set_noise(c->lik, c->xi_plane, c->stream);
  if (st == EP_TV_OK) st = init_state(c);
  if (st != EP_TV_OK) {
    ep_tv_destroy(c);
    *out = nullptr;
  }
  return st;
}

ep_tv_status ep_tv_init_block(const ep_tv_operator* op, const float* y, const ep_tv_params* p,
                              const ep_tv_block* blk, void* cuda_stream, ep_tv_ctx** out) {
  if (!out) return EP_TV_ERR_ARG;
  *out = nullptr;
  if (!op || !p || !blk || op->op != EP_TV_OP_IDENTITY) return EP_TV_ERR_ARG;
  const int H = blk->global_height;
  if (H < 4 || blk->row0 < 0 || (blk->row0 % 2) || blk->rows < 2 || blk->row0 + blk->rows > H ||
      blk->rows >= H)
    return EP_TV_ERR_ARG;
  if (p->periodic && (H % 2 || blk->rows % 2)) return EP_TV_ERR_ARG;
  const int top = (p->periodic || blk->row0 > 0) ? 2 : 0;
  const int bottom = (p->periodic || blk->row0 + blk->rows < H) ? 2 : 0;
  if (op->height != blk->rows + top + bottom) return EP_TV_ERR_ARG;
  // the block itself is an image whose rows do not wrap; its halo rows carry the
  // neighbours' state, so the parity of the matchings V3 and V4 is kept (row0 even)
  ep_tv_params q = *p;
  ep_tv_operator o = *op;
  const int periodic_cols = p->periodic;
  q.periodic = 0;  // the argument checks of a free-boundary image (odd widths allowed)
  if (periodic_cols && (op->width % 2)) return EP_TV_ERR_ARG;
  ep_tv_status st = ep_tv_init(&o, y, &q, cuda_stream, out);
  if (st != EP_TV_OK) return st;
  ep_tv_ctx* c = *out;
  c->p.periodic = periodic_cols;
  c->blk_rows = blk->rows;
  c->blk_top = top;
  c->blk_bottom = bottom;
  return EP_TV_OK;
}

ep_tv_status ep_tv_block_halo_out(ep_tv_ctx* c, int32_t side, float* buf) {
  if (!c || !c->blk_rows || !buf || (side != 0 && side != 1)) return EP_TV_ERR_ARG;
  const int r = side == 0 ? c->blk_top : c->blk_top + c->blk_rows - 2;
  const size_t row = (size_t)c->width, plane = (size_t)c->n;
  for (int k = 0; k < 8; ++k) {
    const float* src = (k < 4 ? c->ptau[c->cur] + k * plane : c->pnu[c->cur] + (k - 4) * plane) + r * row;
    CK(cudaMemcpyAsync(buf + k * 2 * row, src, sizeof(float) * 2 * row, cudaMemcpyDeviceToDevice,
                       c->stream));
  }
  return EP_TV_OK;
}

ep_tv_status ep_tv_block_halo_in(ep_tv_ctx* c, int32_t side, const float* buf) {
  if (!c || !c->blk_rows || !buf || (side != 0 && side != 1)) return EP_TV_ERR_ARG;
  if ((side == 0 && !c->blk_top) || (side == 1 && !c->blk_bottom)) return EP_TV_ERR_ARG;
  const int r = side == 0 ? 0 : c->blk_top + c->blk_rows;
  const size_t row = (size_t)c->width, plane = (size_t)c->n;
  for (int k = 0; k < 8; ++k) {
    float* dst = (k < 4 ? c->ptau[c->cur] + k * plane : c->pnu[c->cur] + (k - 4) * plane) + r * row;
    CK(cudaMemcpyAsync(dst, buf + k * 2 * row, sizeof(float) * 2 * row, cudaMemcpyDeviceToDevice,
                       c->stream));
  }
  return EP_TV_OK;
}

ep_tv_status ep_tv_set_probes(ep_tv_ctx* c, const float* eps1, const float* eps2,
                              int32_t n_samples) {
  if (!c || !eps1 || !eps2 || n_samples < 1) return EP_TV_ERR_ARG;
  if (!c->lik) return EP_TV_ERR_ARG;
  return likelihood_set_probes(c->lik, eps1, eps2, n_samples, c->stream);
}

ep_tv_status ep_tv_sweep(ep_tv_ctx* c, int32_t n_sweeps, const int8_t* k_order,
                         int32_t em_every) {
  if (!c || n_sweeps < 0 || em_every < 0) return EP_TV_ERR_ARG;
  if (em_every > 0 && c->blk_rows) return EP_TV_ERR_ARG;  // blocks: EM needs all blocks' a_u
  if (em_every > 0 && c->p.prior != EP_TV_PRIOR_L1) return EP_TV_ERR_ARG;  // EM: l1-TV only
  if (c->failed) return EP_TV_ERR_STATE;
  if (k_order) {
    for (int t = 0; t < n_sweeps; ++t) {
      int seen = 0;
      for (int u = 0; u < 4; ++u) {
        int k = k_order[4 * t + u];
        if (k < 1 || k > 4 || (seen & (1 << k))) return EP_TV_ERR_ARG;
        seen |= 1 << k;
      }
    }
  }
  int t0 = 0;
  if (!k_order && !c->lik && !c->tracer.on && c->stream != nullptr) {
    // Denoising: a sweep is the prior-site launch (and an E|u| reduction with EM),
    // the same launches every period of lcm(2, em_every) sweeps; replay them from
    // a graph captured once.
    const int period = em_every > 0 ? (em_every % 2 == 0 ? em_every : 2 * em_every) : 2;
    const int reps = n_sweeps / period;
    if (reps >= 2) {
      cudaGraphExec_t g = graph_for(c, period, em_every);
      if (g) {
        for (int r = 0; r < reps; ++r)
          if (cudaGraphLaunch(g, c->stream) != cudaSuccess) return EP_TV_ERR_CUDA;
        c->sweeps += (long long)reps * period;
        c->graph_sweeps += (long long)reps * period;
        t0 = reps * period;
      }
    }
  }
  for (int t = t0; t < n_sweeps; ++t) {
    int order = 0;
    for (int u = 0; u < 4; ++u) {
      int k = k_order ? k_order[4 * t + u] : u + 1;
      order |= k << (4 * u);
    }
    if (c->lik && c->p.order_mode == 1) {
      ep_tv_status st = likelihood_update(c->lik, c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur],
                                          c->status, c->counters, &c->tracer, c->stream);
      if (st != EP_TV_OK) return st;
    }
    c->tracer.begin(EP_TV_K_PRIOR_SWEEP, c->stream);
    launch_prior_sweep(sweep_args(c, order), site0_from_y(c), c->stream);
    c->tracer.end(c->stream, (double)c->n);
    c->cur ^= 1;
    if (c->lik && c->p.order_mode == 0) {
      ep_tv_status st = likelihood_update(c->lik, c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur],
                                          c->status, c->counters, &c->tracer, c->stream);
      if (st != EP_TV_OK) return st;
    }
    if (c->lik && likelihood_graph_last(c->lik)) ++c->graph_sweeps;
    ++c->sweeps;
    if (em_every > 0 && (t + 1) % em_every == 0) launch_em(c, c->ptau[c->cur], c->pnu[c->cur], c->stream);
  }
  if (cudaGetLastError() != cudaSuccess) return EP_TV_ERR_CUDA;
  return EP_TV_OK;
}

ep_tv_status ep_tv_em_beta(ep_tv_ctx* c, double* beta_out, double* abar_out) {
  if (!c) return EP_TV_ERR_ARG;
  if (c->p.prior != EP_TV_PRIOR_L1) return EP_TV_ERR_UNSUPPORTED;  // Sec. IV: l1-TV only
  if (c->failed) return EP_TV_ERR_STATE;
  if (c->sweeps == 0) return EP_TV_ERR_ARG;
  if (c->blk_rows) {
    // a row block reports the a_u of its own edges; beta is set by the caller
    if (c->p.em_option == 1)
      launch_ax_rows(c);
    launch_abar_reduce(c->abar_partial, c->n_partial, c->dscal, (double)c->n, 0, c->stream);
  } else {
    launch_em(c, c->ptau[c->cur], c->pnu[c->cur], c->stream);
  }
  if (cudaGetLastError() != cudaSuccess) return EP_TV_ERR_CUDA;
  if (beta_out || abar_out) {
    double ds[DS_COUNT];
    CK(cudaMemcpyAsync(ds, c->dscal, sizeof(ds), cudaMemcpyDeviceToHost, c->stream));
    ep_tv_status st = latched(c);
    if (st != EP_TV_OK) return st;
    if (beta_out) *beta_out = ds[DS_BETA];
    if (abar_out) *abar_out = ds[DS_ABAR];
  }
  return EP_TV_OK;
}

ep_tv_status ep_tv_ep_em(ep_tv_ctx* c, int32_t n_em, int32_t max_sweeps, double tol,
                         double* beta_out, int32_t* sweeps_out) {
  if (!c || n_em < 1 || max_sweeps < 1 || !(tol >= 0.0) || !beta_out) return EP_TV_ERR_ARG;
  if (c->p.prior != EP_TV_PRIOR_L1) return EP_TV_ERR_UNSUPPORTED;
  if (c->failed) return EP_TV_ERR_STATE;
  cudaStream_t s = c->stream;
  if (!c->mu_prev) {
    if (cudaMalloc(&c->mu_prev, sizeof(float) * c->n) != cudaSuccess ||
        cudaMalloc(&c->d_change, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaHostAlloc(&c->h_change, 2 * sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return EP_TV_ERR_NOMEM;
    }
  }
  auto change = [&]() -> ep_tv_status {
    CK(cudaMemsetAsync(c->d_change, 0, 2 * sizeof(unsigned), s));
    launch_mean_change(c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur], c->n, c->mu_prev,
                       c->d_change, s);
    return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
  };
  for (int t = 0; t < n_em; ++t) {
    ep_tv_status st = change();  // the posterior before this iteration's EP run
    if (st != EP_TV_OK) return st;
    int sw = 0;
    while (sw < max_sweeps) {
      st = ep_tv_sweep(c, 1, nullptr, 0);
      if (st != EP_TV_OK) return st;
      ++sw;
      st = change();
      if (st != EP_TV_OK) return st;
      CK(cudaMemcpyAsync(c->h_change, c->d_change, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      float dmax, mmax;
      memcpy(&dmax, c->h_change, sizeof(float));
      memcpy(&mmax, c->h_change + 1, sizeof(float));
      if (dmax <= (float)tol * mmax) break;
    }
    launch_em(c, c->ptau[c->cur], c->pnu[c->cur], s);
    double beta = 0.0;
    CK(cudaMemcpyAsync(&beta, c->dscal + DS_BETA, sizeof(double), cudaMemcpyDeviceToHost, s));
    st = latched(c);
    if (st != EP_TV_OK) return st;
    beta_out[t] = beta;
    if (sweeps_out) sweeps_out[t] = sw;
  }
  return EP_TV_OK;
}

ep_tv_status ep_tv_set_beta(ep_tv_ctx* c, double beta) {
  if (!c || !(std::isfinite(beta) && beta >= 0.0)) return EP_TV_ERR_ARG;
  CK(cudaMemcpyAsync(c->dscal + DS_BETA, &beta, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return EP_TV_OK;
}

ep_tv_status ep_tv_posterior(ep_tv_ctx* c, float* mean, float* var) {
  if (!c || (!mean && !var)) return EP_TV_ERR_ARG;
  launch_posterior(c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur], c->n, mean, var, c->stream);
  if (cudaGetLastError() != cudaSuccess) return EP_TV_ERR_CUDA;
  return EP_TV_OK;
}

ep_tv_status ep_tv_get_sites(ep_tv_ctx* c, float* tau, float* nu) {
  if (!c || !tau || !nu) return EP_TV_ERR_ARG;
  const size_t nb = sizeof(float) * c->n;
  CK(cudaMemcpyAsync(tau, c->tau0, nb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(tau + c->n, c->ptau[c->cur], 4 * nb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(nu, c->nu0, nb, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(nu + c->n, c->pnu[c->cur], 4 * nb, cudaMemcpyDeviceToDevice, c->stream));
  return EP_TV_OK;
}

ep_tv_status ep_tv_status_check(ep_tv_ctx* c) {
  if (!c) return EP_TV_ERR_ARG;
  return latched(c);
}

ep_tv_status ep_tv_stats(ep_tv_ctx* c, int32_t* cg_iters, uint64_t* n_fp64, uint64_t* n_capped) {
  if (!c) return EP_TV_ERR_ARG;
  unsigned long long cnt[DC_COUNT];
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (cg_iters) *cg_iters = c->lik ? likelihood_last_iters(c->lik) : 0;
  if (n_fp64) *n_fp64 = cnt[DC_FP64];
  if (n_capped) *n_capped = cnt[DC_CAPPED];
  return EP_TV_OK;
}

ep_tv_status ep_tv_solver_report(ep_tv_ctx* c, int32_t* passes, int32_t* iterations,
                                 double* relres_mean, double* relres_probe_max) {
  if (!c) return EP_TV_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  int outer = 0;
  double rm = 0.0, rp = 0.0;
  if (c->lik) likelihood_report(c->lik, &outer, &rm, &rp);
  if (passes) *passes = outer;
  if (iterations) *iterations = c->lik ? likelihood_last_iters(c->lik) : 0;
  if (relres_mean) *relres_mean = rm;
  if (relres_probe_max) *relres_probe_max = rp;
  return EP_TV_OK;
}

// State layout: header (magic, n, m, sweeps), dscal, tau, nu, likelihood blob.
ep_tv_status ep_tv_state_export(ep_tv_ctx* c, void* host_buf, size_t* bytes) {
  if (!c || !bytes) return EP_TV_ERR_ARG;
  const size_t lik_bytes = c->lik ? likelihood_state_bytes(c->lik) : 0;
  const size_t need = 4 * sizeof(long long) + sizeof(double) * DS_COUNT +
                      2 * sizeof(float) * 5 * (size_t)c->n + lik_bytes;
  if (!host_buf) {
    *bytes = need;
    return EP_TV_OK;
  }
  if (*bytes < need) return EP_TV_ERR_ARG;
  char* b = (char*)host_buf;
  long long hdr[4] = {0x45505456ll, c->n, c->m, c->sweeps};
  memcpy(b, hdr, sizeof(hdr));
  b += sizeof(hdr);
  CK(cudaMemcpyAsync(b, c->dscal, sizeof(double) * DS_COUNT, cudaMemcpyDeviceToHost, c->stream));
  b += sizeof(double) * DS_COUNT;
  const size_t nb = sizeof(float) * c->n;
  CK(cudaMemcpyAsync(b, c->tau0, nb, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(b + nb, c->ptau[c->cur], 4 * nb, cudaMemcpyDeviceToHost, c->stream));
  b += 5 * nb;
  CK(cudaMemcpyAsync(b, c->nu0, nb, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(b + nb, c->pnu[c->cur], 4 * nb, cudaMemcpyDeviceToHost, c->stream));
  b += 5 * nb;
  if (c->lik) {
    ep_tv_status st = likelihood_state_export(c->lik, b, c->stream);
    if (st != EP_TV_OK) return st;
  }
  *bytes = need;
  return latched(c);
}

ep_tv_status ep_tv_state_import(ep_tv_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return EP_TV_ERR_ARG;
  const size_t lik_bytes = c->lik ? likelihood_state_bytes(c->lik) : 0;
  const size_t need = 4 * sizeof(long long) + sizeof(double) * DS_COUNT +
                      2 * sizeof(float) * 5 * (size_t)c->n + lik_bytes;
  if (bytes != need) return EP_TV_ERR_ARG;
  const char* b = (const char*)host_buf;
  long long hdr[4];
  memcpy(hdr, b, sizeof(hdr));
  if (hdr[0] != 0x45505456ll || hdr[1] != c->n || hdr[2] != c->m) return EP_TV_ERR_ARG;
  b += sizeof(hdr);
  CK(cudaMemcpyAsync(c->dscal, b, sizeof(double) * DS_COUNT, cudaMemcpyHostToDevice, c->stream));
  b += sizeof(double) * DS_COUNT;
  const size_t nb = sizeof(float) * c->n;
  CK(cudaMemcpyAsync(c->tau0, b, nb, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ptau[c->cur], b + nb, 4 * nb, cudaMemcpyHostToDevice, c->stream));
  b += 5 * nb;
  CK(cudaMemcpyAsync(c->nu0, b, nb, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->pnu[c->cur], b + nb, 4 * nb, cudaMemcpyHostToDevice, c->stream));
  b += 5 * nb;
  if (c->lik) {
    ep_tv_status st = likelihood_state_import(c->lik, b, c->stream);
    if (st != EP_TV_OK) return st;
  }
  CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->sweeps = hdr[3];
  c->failed = false;
  return EP_TV_OK;
}

ep_tv_status ep_tv_reset(ep_tv_ctx* c) {
  if (!c) return EP_TV_ERR_ARG;
  return init_state(c);
}

ep_tv_status ep_tv_warm_start(ep_tv_ctx* c, const float* out, int32_t mode) {
  if (!c || !out || c->op.op == EP_TV_OP_DENSE || c->op.op == EP_TV_OP_HADAMARD) return EP_TV_ERR_ARG;
  if (mode != EP_TV_WARM_ALL_SITES && mode != EP_TV_WARM_SITE0 && mode != EP_TV_WARM_PRIOR)
    return EP_TV_ERR_ARG;
  if (c->failed) return EP_TV_ERR_STATE;
  const bool identity = c->op.op == EP_TV_OP_IDENTITY;
  if (identity && mode == EP_TV_WARM_SITE0) return EP_TV_OK;  // site 0 is exact already
  launch_warm_start(c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur], out, c->y,
                    (float)log(c->p.xi), c->n, (float)(1.0 / c->p.var_cap),
                    identity || mode == EP_TV_WARM_PRIOR, mode == EP_TV_WARM_SITE0, c->stream);
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

ep_tv_status ep_tv_solve_host(const ep_tv_operator* op, const float* y_host,
                              const ep_tv_params* p, int32_t n_sweeps, int32_t em_every,
                              float* mean_host, float* var_host, double* beta_out) {
  if (!op || !y_host || !p || !mean_host || !var_host || n_sweeps < 0) return EP_TV_ERR_ARG;
  ep_tv_status st = check_params(op, p);
  if (st != EP_TV_OK) return st;
  const long long n = (long long)op->height * op->width;
  float* d_y = nullptr;
  float* d_out = nullptr;
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  if (cudaMalloc(&d_y, sizeof(float) * op->m) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(float) * 2 * n) != cudaSuccess) {
    cudaFree(d_y);
    cudaStreamDestroy(s);
    return EP_TV_ERR_NOMEM;
  }
  ep_tv_ctx* c = nullptr;
  st = EP_TV_OK;
  if (cudaMemcpyAsync(d_y, y_host, sizeof(float) * op->m, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = EP_TV_ERR_CUDA;
  if (st == EP_TV_OK) st = ep_tv_init(op, d_y, p, s, &c);
  if (st == EP_TV_OK) st = ep_tv_sweep(c, n_sweeps, nullptr, em_every);
  if (st == EP_TV_OK) st = ep_tv_posterior(c, d_out, d_out + n);
  if (st == EP_TV_OK) {
    if (cudaMemcpyAsync(mean_host, d_out, sizeof(float) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(var_host, d_out + n, sizeof(float) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = EP_TV_ERR_CUDA;
  }
  if (st == EP_TV_OK && beta_out) {
    if (cudaMemcpyAsync(beta_out, c->dscal + DS_BETA, sizeof(double), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      st = EP_TV_ERR_CUDA;
  }
  if (st == EP_TV_OK) st = latched(c);
  ep_tv_destroy(c);
  cudaFree(d_y);
  cudaFree(d_out);
  cudaStreamDestroy(s);
  return st;
}

ep_tv_status ep_tv_trace_enable(ep_tv_ctx* c, int32_t on) {
  if (!c) return EP_TV_ERR_ARG;
  if (on) {
    if (!c->tracer.ensure()) return EP_TV_ERR_CUDA;
    CK(cudaStreamSynchronize(c->stream));
    c->tracer.reset();
    CK(cudaMemcpy(c->cnt_base, c->counters, sizeof(c->cnt_base), cudaMemcpyDeviceToHost));
  } else if (c->tracer.on) {
    c->tracer.harvest();
  }
  c->tracer.on = on != 0;
  return EP_TV_OK;
}

ep_tv_status ep_tv_trace_read(ep_tv_ctx* c, int32_t kernel, double* ms, int64_t* launches,
                              double* units, double* bytes_per_unit) {
  if (!c || kernel < 0 || kernel >= EP_TV_K_COUNT) return EP_TV_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->tracer.harvest();
  unsigned long long cnt[DC_COUNT];
  CK(cudaMemcpy(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  double u = c->tracer.host_units[kernel];
  if (kernel == EP_TV_K_CG_DIRECTION)
    u = (double)(cnt[DC_CG_DIR_UNITS] - c->cnt_base[DC_CG_DIR_UNITS]) * (double)c->n;
  if (kernel == EP_TV_K_CG_UPDATE)
    u = (double)(cnt[DC_CG_UPD_UNITS] - c->cnt_base[DC_CG_UPD_UNITS]) * (double)c->n;
  if (kernel == EP_TV_K_CG_PRECOND)
    u = (double)(cnt[DC_CG_PRE_UNITS] - c->cnt_base[DC_CG_PRE_UNITS]) * (double)c->n;
  double bpu = 0.0;
  if (kernel == EP_TV_K_PRIOR_SWEEP)
    bpu = prior_sweep_bytes_per_pixel(site0_from_y(c));
  else if (c->lik)
    bpu = likelihood_bytes_per_unit(c->lik, kernel);
  if (kernel == EP_TV_K_CS && c->n > 0) bpu /= (double)c->n;  // FP64 flops per pixel
  if (ms) *ms = c->tracer.ms[kernel];
  if (launches) *launches = c->tracer.launches[kernel];
  if (units) *units = u;
  if (bytes_per_unit) *bytes_per_unit = bpu;
  return EP_TV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many contexts advanced together.  One launch runs the prior-site
// pass of every image (a block -> image table); the likelihood-site updates of
// the contexts that have one run concurrently on worker streams, each driven by
// a host thread of a small pool (their CG loops poll their own convergence).
struct ep_tv_batch {
  std::vector<ep_tv_ctx*> ctx;
  cudaStream_t stream = nullptr;
  int device = 0;
  BatchItem* d_items[2] = {nullptr, nullptr};
  BatchItem* h_items[2] = {nullptr, nullptr};
  cudaEvent_t items_ev[2] = {nullptr, nullptr};
  int slot = 0;
  long long total_units = 0;             // prior-sweep work units of all images
  std::vector<int> lik;                 // contexts with a likelihood state
  std::vector<cudaStream_t> wstream;    // one worker stream per such context
  std::vector<cudaEvent_t> wdone;
  cudaEvent_t prior_done = nullptr;
  // pool
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_job, cv_done;
  int next_job = 0, jobs_total = 0, jobs_done = 0;
  bool stop = false;
  ep_tv_status job_err = EP_TV_OK;
  // Batches without likelihood solvers: sweeps replayed from a captured graph of
  // one persistent launch per sweep over two fixed image tables (one per parity).
  BatchItem* g_items[2] = {nullptr, nullptr};
  cudaGraphExec_t graph = nullptr;
  int graph_em = -1, graph_len = 0;
  std::vector<int> graph_cur;            // buffer parity of every context at capture
};

namespace {

// Image table of a sweep with every context's prior buffers at parity cur ^ flip.
void fill_items(ep_tv_batch* b, BatchItem* h, int flip) {
  long long unit = 0;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    ep_tv_ctx* c = b->ctx[i];
    h[i].a = sweep_args(c, 0x4321);
    if (flip) {
      h[i].a.tin = c->ptau[c->cur ^ 1];
      h[i].a.nin = c->pnu[c->cur ^ 1];
      h[i].a.tout = c->ptau[c->cur];
      h[i].a.nout = c->pnu[c->cur];
    }
    prior_sweep_prepare(h[i].a);
    h[i].site0_from_y = site0_from_y(c);
    h[i].units = prior_sweep_blocks(c->height, c->width);
    h[i].unit_begin = unit;
    unit += h[i].units;
  }
}

// Graph of `period` batch sweeps from the contexts' current parities (captured on
// first use, recaptured when the parities or the EM period differ).
cudaGraphExec_t batch_graph(ep_tv_batch* b, int period, int em_every) {
  std::vector<int> cur;
  for (ep_tv_ctx* c : b->ctx) cur.push_back(c->cur);
  if (b->graph && b->graph_em == em_every && b->graph_len == period && b->graph_cur == cur)
    return b->graph;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  const size_t n = b->ctx.size();
  for (int i = 0; i < 2; ++i)
    if (!b->g_items[i] && cudaMalloc(&b->g_items[i], sizeof(BatchItem) * n) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  std::vector<BatchItem> h(n);
  for (int f = 0; f < 2; ++f) {
    fill_items(b, h.data(), f);
    if (cudaMemcpy(b->g_items[f], h.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  prior_sweep_prewarm();
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  for (int t = 0; t < period; ++t) {
    launch_prior_sweep_batch(b->g_items[t & 1], (int)n, b->total_units, b->stream);
    if (em_every > 0 && (t + 1) % em_every == 0)
      for (ep_tv_ctx* c : b->ctx) {
        const int cur = c->cur ^ ((t + 1) & 1);  // the contexts' parity after sweep t
        launch_em(c, c->ptau[cur], c->pnu[cur], b->stream);
      }
  }
  const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  cudaGraphExec_t exec = nullptr;
  if (e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  b->graph = exec;
  b->graph_em = em_every;
  b->graph_len = period;
  b->graph_cur = cur;
  return exec;
}

void batch_worker(ep_tv_batch* b) {
  cudaSetDevice(b->device);
  for (;;) {
    int job;
    {
      std::unique_lock<std::mutex> lock(b->mu);
      b->cv_job.wait(lock, [b] { return b->stop || b->next_job < b->jobs_total; });
      if (b->stop) return;
      job = b->next_job++;
    }
    ep_tv_ctx* c = b->ctx[b->lik[job]];
    ep_tv_status st = EP_TV_OK;
    if (cudaStreamWaitEvent(b->wstream[job], b->prior_done, 0) != cudaSuccess) st = EP_TV_ERR_CUDA;
    if (st == EP_TV_OK)
      st = likelihood_update(c->lik, c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur], c->status,
                             c->counters, &c->tracer, b->wstream[job]);
    if (st == EP_TV_OK && cudaEventRecord(b->wdone[job], b->wstream[job]) != cudaSuccess)
      st = EP_TV_ERR_CUDA;
    {
      std::lock_guard<std::mutex> lock(b->mu);
      if (st != EP_TV_OK && b->job_err == EP_TV_OK) b->job_err = st;
      if (++b->jobs_done == b->jobs_total) b->cv_done.notify_one();
    }
  }
}

void batch_free(ep_tv_batch* b) {
  {
    std::lock_guard<std::mutex> lock(b->mu);
    b->stop = true;
  }
  b->cv_job.notify_all();
  for (auto& t : b->threads) t.join();
  for (int i = 0; i < 2; ++i) {
    cudaFree(b->d_items[i]);
    if (b->h_items[i]) cudaFreeHost(b->h_items[i]);
    if (b->items_ev[i]) cudaEventDestroy(b->items_ev[i]);
  }
  for (int i = 0; i < 2; ++i) cudaFree(b->g_items[i]);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto s : b->wstream) cudaStreamDestroy(s);
  for (auto e : b->wdone) cudaEventDestroy(e);
  if (b->prior_done) cudaEventDestroy(b->prior_done);
  delete b;
}

}  // namespace

extern "C" {

ep_tv_status ep_tv_batch_create(int32_t n, ep_tv_ctx* const* ctxs, ep_tv_batch** out) {
  if (!out || n < 1 || !ctxs) return EP_TV_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return EP_TV_ERR_ARG;
    if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->device != ctxs[0]->device)
      return EP_TV_ERR_ARG;
    if (ctxs[i]->p.order_mode != 0) return EP_TV_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return EP_TV_ERR_ARG;
  }
  ep_tv_batch* b = new (std::nothrow) ep_tv_batch();
  if (!b) return EP_TV_ERR_NOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  b->stream = ctxs[0]->stream;
  b->device = ctxs[0]->device;
  for (int i = 0; i < n; ++i) {
    b->total_units += prior_sweep_blocks(ctxs[i]->height, ctxs[i]->width);
    if (ctxs[i]->lik) b->lik.push_back(i);
  }
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaMalloc(&b->d_items[i], sizeof(BatchItem) * n) == cudaSuccess &&
         cudaHostAlloc(&b->h_items[i], sizeof(BatchItem) * n, cudaHostAllocDefault) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->items_ev[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->prior_done, cudaEventDisableTiming) == cudaSuccess;
  for (size_t k = 0; k < b->lik.size() && ok; ++k) {
    cudaStream_t ws;
    cudaEvent_t ev;
    ok = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->wstream.push_back(ws);
    ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->wdone.push_back(ev);
  }
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return EP_TV_ERR_NOMEM;
  }
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthreads = (int)std::min<size_t>(b->lik.size(), std::min(16u, hw));
  for (int t = 0; t < nthreads; ++t) b->threads.emplace_back(batch_worker, b);
  *out = b;
  return EP_TV_OK;
}

ep_tv_status ep_tv_batch_sweep(ep_tv_batch* b, int32_t n_sweeps, int32_t em_every) {
  if (!b || n_sweeps < 0 || em_every < 0) return EP_TV_ERR_ARG;
  if (em_every > 0)
    for (ep_tv_ctx* c : b->ctx)
      if (c->p.prior != EP_TV_PRIOR_L1) return EP_TV_ERR_ARG;  // EM: l1-TV only
  const int n = (int)b->ctx.size();
  bool tracing = false;
  for (ep_tv_ctx* c : b->ctx) {
    if (c->failed) return EP_TV_ERR_STATE;
    tracing |= c->tracer.on;
  }
  int t0 = 0;
  if (b->lik.empty() && !tracing && b->stream != nullptr) {
    // denoising only: replay one persistent launch per sweep (and the EM
    // reductions) from a captured graph, lcm(2, em_every) sweeps per replay
    const int period = em_every > 0 ? (em_every % 2 == 0 ? em_every : 2 * em_every) : 2;
    const int reps = n_sweeps / period;
    if (reps >= 2) {
      cudaGraphExec_t g = batch_graph(b, period, em_every);
      if (g) {
        for (int r = 0; r < reps; ++r) CK(cudaGraphLaunch(g, b->stream));
        for (ep_tv_ctx* c : b->ctx) {
          c->sweeps += (long long)reps * period;
          c->graph_sweeps += (long long)reps * period;
        }
        t0 = reps * period;
      }
    }
  }
  for (int t = t0; t < n_sweeps; ++t) {
    // image table of this sweep (prior buffers alternate per context)
    CK(cudaEventSynchronize(b->items_ev[b->slot]));
    BatchItem* h = b->h_items[b->slot];
    fill_items(b, h, 0);
    CK(cudaMemcpyAsync(b->d_items[b->slot], h, sizeof(BatchItem) * n, cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaEventRecord(b->items_ev[b->slot], b->stream));
    launch_prior_sweep_batch(b->d_items[b->slot], n, b->total_units, b->stream);
    b->slot ^= 1;
    for (ep_tv_ctx* c : b->ctx) {
      c->cur ^= 1;
      ++c->sweeps;
    }
    if (!b->lik.empty() && !tracing) {
      // every likelihood update is one graph replay (its solver loops run on the
      // device): enqueue them all from this thread, each on its own stream after
      // the prior pass, and join them below
      CK(cudaEventRecord(b->prior_done, b->stream));
      for (size_t k = 0; k < b->lik.size(); ++k) {
        ep_tv_ctx* c = b->ctx[b->lik[k]];
        CK(cudaStreamWaitEvent(b->wstream[k], b->prior_done, 0));
        const ep_tv_status st = likelihood_update(c->lik, c->tau0, c->nu0, c->ptau[c->cur], c->pnu[c->cur],
                                                  c->status, c->counters, &c->tracer, b->wstream[k]);
        if (st != EP_TV_OK) return st;
        if (likelihood_graph_last(c->lik)) ++c->graph_sweeps;
        CK(cudaEventRecord(b->wdone[k], b->wstream[k]));
      }
      for (size_t k = 0; k < b->lik.size(); ++k) CK(cudaStreamWaitEvent(b->stream, b->wdone[k], 0));
    } else if (!b->lik.empty()) {
      // traced: the host-driven solver loops poll convergence, one host thread each
      CK(cudaEventRecord(b->prior_done, b->stream));
      {
        std::lock_guard<std::mutex> lock(b->mu);
        b->next_job = 0;
        b->jobs_done = 0;
        b->jobs_total = (int)b->lik.size();
        b->job_err = EP_TV_OK;
      }
      b->cv_job.notify_all();
      {
        std::unique_lock<std::mutex> lock(b->mu);
        b->cv_done.wait(lock, [b] { return b->jobs_done == b->jobs_total; });
        b->jobs_total = 0;
        b->next_job = 0;
        if (b->job_err != EP_TV_OK) return b->job_err;
      }
      for (size_t k = 0; k < b->lik.size(); ++k) CK(cudaStreamWaitEvent(b->stream, b->wdone[k], 0));
    }
    if (em_every > 0 && (t + 1) % em_every == 0)
      for (ep_tv_ctx* c : b->ctx) launch_em(c, c->ptau[c->cur], c->pnu[c->cur], b->stream);
  }
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

int64_t ep_tv_graph_sweeps(const ep_tv_ctx* c) { return c ? c->graph_sweeps : -1; }

void ep_tv_batch_destroy(ep_tv_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}

void ep_tv_destroy(ep_tv_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

const char* ep_tv_status_str(ep_tv_status s) {
  switch (s) {
    case EP_TV_OK: return "ok";
    case EP_TV_ERR_ARG: return "invalid argument";
    case EP_TV_ERR_NOMEM: return "device allocation failed";
    case EP_TV_ERR_CUDA: return "CUDA runtime error";
    case EP_TV_ERR_NONFINITE: return "a site value became NaN or infinite";
    case EP_TV_ERR_CG_NOCONV: return "likelihood-site solver hit its iteration cap";
    case EP_TV_ERR_TIMEOUT: return "bounded device-side wait gave up";
    case EP_TV_ERR_STATE: return "context unusable after a device error; call ep_tv_reset";
    case EP_TV_ERR_UNSUPPORTED: return "not supported by this build";
  }
  return "unknown status";
}

}  // extern "C"
