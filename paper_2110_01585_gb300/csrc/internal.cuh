// Internal declarations shared by the CUDA translation units of libeptv.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ep_tv.h"

namespace eptv {

// Device status bits (latched with atomicOr, read by synchronising calls).
enum : unsigned {
  ST_NONFINITE = 1u,
  ST_CG_NOCONV = 2u,
  ST_TIMEOUT = 4u,
};

// Slots of the per-context FP64 device scalars.
enum : int {
  DS_BETA = 0,   // current beta (lambda)
  DS_ABAR = 1,   // a_u of the last sweep (after reduction)
  DS_COUNT = 4,
};

// Counters (uint64 on the device).
enum : int {
  DC_FP64 = 0,
  DC_CAPPED = 1,
  DC_CG_ITERS = 2,
  DC_CG_DIR_UNITS = 3,   // active systems summed over direction launches
  DC_CG_UPD_UNITS = 4,   // active systems summed over update launches
  DC_CG_PRE_UNITS = 5,   // systems transformed, summed over preconditioner applications
  DC_COUNT = 8,
};

// Host-side tracer: CUDA events around kernel launches, per kernel class.
struct Tracer {
  static constexpr int kPairs = 8192;
  bool on = false;
  std::vector<cudaEvent_t> ev;   // 2 * kPairs
  std::vector<int> kid;          // class of each recorded pair
  std::vector<double> units;     // host-known units of each pair (or -1)
  int used = 0;
  double ms[EP_TV_K_COUNT] = {};
  long long launches[EP_TV_K_COUNT] = {};
  double host_units[EP_TV_K_COUNT] = {};

  ~Tracer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  bool ensure() {
    if (!ev.empty()) return true;
    ev.resize(2 * kPairs);
    kid.resize(kPairs);
    units.resize(kPairs);
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return false;
    return true;
  }
  void reset() {
    used = 0;
    for (int i = 0; i < EP_TV_K_COUNT; ++i) { ms[i] = 0; launches[i] = 0; host_units[i] = 0; }
  }
  // Waits for the recorded pairs and folds them into the totals.
  void harvest() {
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      cudaEventSynchronize(ev[2 * i + 1]);
      if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
        ms[kid[i]] += t;
        launches[kid[i]] += 1;
        if (units[i] > 0) host_units[kid[i]] += units[i];
      }
    }
    used = 0;
  }
  void begin(int k, cudaStream_t s) {
    if (!on) return;
    if (used == kPairs) harvest();
    kid[used] = k;
    cudaEventRecord(ev[2 * used], s);
  }
  void end(cudaStream_t s, double u) {
    if (!on) return;
    units[used] = u;
    cudaEventRecord(ev[2 * used + 1], s);
    ++used;
  }
};

struct SweepArgs {
  const float* tau0;          // [N] likelihood-site precision
  const float* nu0;           // [N] likelihood-site precision-times-mean
  const float* tin;           // [4][N] prior sites k = 1..4 before the sweep (row k - 1)
  const float* nin;
  float* tout;                // [4][N] prior sites after the sweep (a different buffer:
  float* nout;                // halo tiles read while other tiles write)
  const float* y;             // identity operator: observation (site 0 = (1/xi, y/xi))
  float inv_xi;               // 1 / xi as float (identity operator)
  int height, width;
  long long n;
  int periodic;               // columns wrap (and rows, unless periodic_rows says otherwise)
  int periodic_rows;          // rows wrap (a row block of a sharded image: 0)
  int count_lo, count_hi;     // E|u| and the counters take the edges whose first pixel's
                              // row is in [count_lo, count_hi) (whole image: [0, height))
  float damping;
  float min_tau;              // 1 / var_cap
  const double* beta;         // device scalar
  int order;                  // four 4-bit k values, first update in the low nibble
  int fp64_tail;              // 1: recompute poorly conditioned edges in FP64
  int prior;                  // ep_tv_prior
  int em_option;              // 1, 2 or 3: which EM statistic the pass accumulates (2: Eq. au)
  float mix_logit;            // MoG2 / BG: log((1 - omega) / omega)
  float mix_v1, mix_v2;       // MoG2 / BG: component variances (BG: v2 = 0, the point mass)
  double* abar_partial;       // one FP64 partial sum of E|u| per work unit
  int vec2;                   // set by prior_sweep_prepare: float2 loads and stores allowed
  unsigned* status;
  unsigned long long* counters;
};

// One image of a batched prior-site launch.
struct BatchItem {
  SweepArgs a;
  int site0_from_y;
  long long units;        // work units of this image
  long long unit_begin;   // first unit of this image in the launch
};

// Whether the prior fields of p are valid, and their copy into the sweep arguments.
bool prior_params_ok(const ep_tv_params* p);
void set_prior_args(SweepArgs& a, const ep_tv_params* p);

// Prior-site sweep over V_1..V_4 for one image; site 0 implicit (identity) or stored.
void launch_prior_sweep(const SweepArgs& a, bool site0_from_y, cudaStream_t s);
// Algorithmic DRAM bytes per pixel of one prior-site pass.
double prior_sweep_bytes_per_pixel(bool site0_from_y);
// Runs the per-device set-up of the prior-pass launchers (occupancy queries and
// attributes) so that a later launch inside a stream capture makes no such calls.
void prior_sweep_prewarm();
// Fills the fields of `a` that the launch derives (vector access).
void prior_sweep_prepare(SweepArgs& a);
// Work units (and E|u| partial sums) of one image's prior-site pass.
int prior_sweep_blocks(int height, int width);
void launch_prior_sweep_batch(const BatchItem* items, int n_items, long long total_units,
                              cudaStream_t s);

// abar = sum(partials) in a fixed order; if do_em, beta = n / abar.
void launch_abar_reduce(const double* partial, int n_partial, double* dscal, double n_pixels,
                        int do_em, cudaStream_t s);

void launch_init_sites(float* tau0, float* nu0, float* tp, float* np, const float* mu0, long long n,
                       float inv_xi, float min_tau, cudaStream_t s);
void launch_warm_start(float* tau0, float* nu0, float* tp, float* np, const float* out,
                       const float* y, float log_xi, long long n, float min_tau, bool keep_site0,
                       bool site0_only, cudaStream_t s);
// Option 1 of the EM statistic (a_x) into n_partial FP64 block partials.
void launch_ax(const float* tau0, const float* nu0, const float* tp, const float* np, int height,
               int width, int periodic, double* partial, int n_partial, cudaStream_t s);
// The same over the edges whose first pixel's row is in [row_lo, row_hi), rows not wrapping.
void launch_ax_block(const float* tau0, const float* nu0, const float* tp, const float* np,
                     int height, int width, int periodic, int row_lo, int row_hi, double* partial,
                     int n_partial, cudaStream_t s);
// Posterior mean into prev, max |change| and max |mean| as float bits into out[0..1].
void launch_mean_change(const float* tau0, const float* nu0, const float* tp, const float* np,
                        long long n, float* prev, unsigned* out, cudaStream_t s);
// Site 0 of denoising with per-pixel noise variances xi: (1 / xi, y / xi).
void launch_site0_noise(float* tau0, float* nu0, const float* y, const float* xi, long long n,
                        cudaStream_t s);
void launch_posterior(const float* tau0, const float* nu0, const float* tp, const float* np,
                      long long n, float* mean, float* var, cudaStream_t s);

}  // namespace eptv
