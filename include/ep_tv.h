/*
 * ep_tv.h - C ABI of the GB300 expectation-propagation library for image
 * restoration with an anisotropic l1 total-variation prior.
 *
 * Method: Yao, McLaughlin and Altmann, "Fast Scalable Image Restoration using
 * Total Variation Priors and Expectation Propagation" (arXiv:2110.01585).
 *
 *   Observation model (Sec. II-A, Eq. likelihood): y = H x + n, n ~ N(0, xi I),
 *     x an H x W image (N = H W pixels, row-major, p = r W + c), y of length M.
 *   Prior (Sec. II-B, Eq. prior1, Eq. L1_TV): prod over the four matchings V_k of
 *     the 4-neighbour graph of exp(-beta |x_i - x_j|)  (beta is the paper's lambda).
 *   Approximation (Sec. III): Q(x) = N(mu, diag sigma^2) built from five diagonal
 *     Gaussian sites: q_{x,0} for the likelihood and q_{x,k}, k = 1..4, one per V_k.
 *   One sweep (Algorithm 1) updates the four prior sites (all edges of a V_k in
 *     parallel) and the likelihood site, with the variance cap and damping of
 *     Sec. III-C; the EM step (Sec. IV, Algorithm 2, Eq. 3rd_alternative_a0) sets
 *     beta = N / a_u, a_u the sum over all edges of the tilted E|x_i - x_j|.
 *
 * Conventions for every call:
 *   - Pointers documented as "device" must be CUDA device pointers valid on the
 *     context's device; "host" pointers are ordinary CPU memory.
 *   - Floating-point data are float32 unless stated.  Images are row-major,
 *     contiguous, H rows of W elements.
 *   - All work is enqueued on the stream given to ep_tv_init (0 = legacy default
 *     stream).  Calls return once the work is enqueued, except where stated.
 *   - The library owns all site state and scratch memory it allocates; the
 *     caller owns every buffer it passes in.  Input buffers are copied during the
 *     call that receives them, except the dense sensing matrix (see below).
 *   - Argument errors are returned synchronously and change nothing.  Errors found
 *     on the device (non-finite site values, solver failure) are latched in a
 *     device status word and returned by the next call that synchronises
 *     (ep_tv_em_beta with an output pointer, ep_tv_status_check, ep_tv_state_export,
 *     ep_tv_solve_host); after that the context refuses further sweeps with
 *     EP_TV_ERR_STATE until ep_tv_reset.  No call aborts the process.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef EP_TV_H
#define EP_TV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ep_tv_ctx ep_tv_ctx;

typedef enum {
  EP_TV_OK = 0,
  EP_TV_ERR_ARG = 1,          /* invalid argument (returned before any work) */
  EP_TV_ERR_NOMEM = 2,        /* device allocation failed */
  EP_TV_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  EP_TV_ERR_NONFINITE = 4,    /* a site value became NaN or infinite */
  EP_TV_ERR_CG_NOCONV = 5,    /* the likelihood-site solver hit its iteration cap */
  EP_TV_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  EP_TV_ERR_STATE = 7,        /* context unusable after a latched device error */
  EP_TV_ERR_UNSUPPORTED = 8   /* valid request this build does not implement */
} ep_tv_status;

/* Degradation operators (Sec. II-A): (i) identity, (ii) convolution, (iii) compressive
   sensing with a dense matrix or with subsampled 2-D Hadamard patterns. */
typedef enum {
  EP_TV_OP_IDENTITY = 0,        /* denoising, M = N */
  EP_TV_OP_CONV_PERIODIC = 1,   /* periodic convolution with a centred odd kernel, M = N */
  EP_TV_OP_DENSE = 2,           /* compressive sensing, dense M x N matrix; the likelihood
                                   site uses the Woodbury identity in FP64 */
  EP_TV_OP_HADAMARD = 3         /* compressive sensing with M rows of the 2-D Walsh-Hadamard
                                   matrix (Sec. II-A (iii), single-pixel imaging); Woodbury
                                   in FP64 with fast transforms in place of the dense products */
} ep_tv_op;

typedef struct {
  int32_t op;            /* ep_tv_op */
  int32_t height;        /* image rows H >= 1 */
  int32_t width;         /* image columns W >= 1 */
  int32_t m;             /* length of y: N for IDENTITY and CONV_PERIODIC, M for DENSE and
                            HADAMARD */
  const float* kernel;   /* CONV_PERIODIC: HOST pointer, kh x kw row-major, copied at init.
                            (H x)[r,c] = sum_{a,b} k[a,b] x[(r-a+kh/2) mod H, (c-b+kw/2) mod W] */
  int32_t kh, kw;        /* odd kernel sizes, kh <= H, kw <= W */
  const float* dense;    /* DENSE: DEVICE pointer, M x N row-major.  Borrowed: it must stay
                            valid and unchanged for the life of the context. */
  const int32_t* patterns; /* HADAMARD: HOST pointer, M distinct pattern indices, copied at
                            init.  H and W must be powers of two.  Pattern p = kr * W + kc is
                            the outer product of the Walsh functions of sequency kr (length H)
                            and kc (length W), Paley order: entry (r, c) is
                            (-1)^(popcount(r & rev(kr)) + popcount(c & rev(kc))), rev reversing
                            the log2 H (log2 W) index bits.  Row m of A is pattern p_m over
                            sqrt(M), so that A A^T = (N / M) I. */
} ep_tv_operator;

/* Edge factor phi(x_i - x_j; theta) of the prior (Sec. II-B). */
typedef enum {
  EP_TV_PRIOR_L1 = 0,    /* l1-TV, Eq. L1_TV: exp(-beta |u|) (beta is the paper's lambda) */
  EP_TV_PRIOR_MOG2 = 1,  /* MoG2-TV, Eq. MoG2_TV_prior:
                            omega N(u; 0, s1_sq) + (1 - omega) N(u; 0, s2_sq) */
  EP_TV_PRIOR_BG = 2     /* BG-TV, Eq. BG_TV: omega N(u; 0, s1_sq) + (1 - omega) delta(u) */
} ep_tv_prior;

typedef struct {
  double xi;             /* noise variance xi > 0 (Eq. likelihood) */
  double beta;           /* TV parameter (the paper's lambda) >= 0; EM start value (l1-TV) */
  double damping;        /* weight in (0, 1] on the freshly updated site when mixing
                            natural parameters: new = d * updated + (1 - d) * old */
  double var_cap;        /* site variances are capped at var_cap (the paper suggests
                            1e8, Sec. III-C): a new site precision below 1/var_cap
                            (negative or tiny) is set to 1/var_cap */
  int32_t periodic;      /* 1: torus, every pixel in one edge of each V_k; needs even
                            H and W.  0: free boundary, wrap-around edges dropped. */
  int32_t order_mode;    /* 0: the four prior-site updates, then the likelihood site
                            (uses the initial likelihood site).  1: likelihood site
                            first, as Algorithm 1 lists it. */
  int32_t rbmc_samples;  /* CONV_PERIODIC: S probes of the Rao-Blackwellised Monte Carlo
                            variance estimator (default 32) */
  int32_t cg_max_iter;   /* CONV_PERIODIC: cap on the conjugate-gradient iterations of one
                            likelihood-site update (all refinement passes together) */
  double cg_rtol;        /* CONV_PERIODIC: target of the true relative residual ||b - Q x|| /
                            ||b|| of the mean solve (probe solves: max(cg_rtol, 1e-6)).  The
                            residual is recomputed in float-float arithmetic between FP32
                            CG passes; a solve also stops when a pass no longer halves a
                            residual already below 1e-6 (the evaluation floor).  Default 1e-9. */
  int32_t precision;     /* 0: FP32 with FP64 for edges whose tilted moments lose
                            FP32 accuracy; 1: FP32 only */
  uint64_t seed;         /* seed of the library's own probe generator */
  int32_t prior;         /* ep_tv_prior (default EP_TV_PRIOR_L1) */
  double omega;          /* MoG2 / BG: mixture weight of the N(0, s1_sq) component, in (0, 1) */
  double s1_sq;          /* MoG2 / BG: variance of the first Gaussian component, > 0 */
  double s2_sq;          /* MoG2: variance of the second component, > 0 (BG: unused) */
  int32_t em_option;     /* l1-TV: the approximation of a_0 (Eq. a_0) of the EM update
                            (Sec. IV): 1 = a_x (Eq. ax), E|x_i - x_j| under Q(x) after
                            the sweep; 2 = a_u (Eq. au), E|u_n| under the Gaussian Q(u_n)
                            matched during the sweep; 3 = abar_u (Eq. 3rd_alternative_a0,
                            default), E|u_n| under the tilted P_k(u_n) */
} ep_tv_params;

/* Fills *p with defaults: damping 0.5, var_cap 1e8, periodic 1, order_mode 0,
   rbmc_samples 32, cg_max_iter 1000, cg_rtol 1e-9, precision 0, seed 1234,
   prior EP_TV_PRIOR_L1, em_option 3.  xi and beta (or, for the mixture priors, omega, s1_sq
   and s2_sq) are set to 0 and must be provided.  The mixture priors are not
   log-concave: their edge updates can ask for negative site variances, which the
   variance cap of Sec. III-C replaces.  The EM update of beta (Sec. IV) exists
   for l1-TV only. */
ep_tv_status ep_tv_default_params(ep_tv_params* p);

/* Creates a context and initialises the sites as Algorithm 1 does:
   q_{x,0} has mean y (H^T y for DENSE) and variance xi; q_{x,1..4} have mean 0
   and variance var_cap.  y: DEVICE pointer of length op->m, copied.
   cuda_stream: a cudaStream_t (or NULL) on the current device; all later work of
   this context is enqueued on it.  *out receives the context. */
ep_tv_status ep_tv_init(const ep_tv_operator* op, const float* y, const ep_tv_params* p,
                        void* cuda_stream, ep_tv_ctx** out);

/* Like ep_tv_init, with a diagonal noise covariance: y_m ~ N(h_m x, xi_m), one
   variance per measurement, which the likelihood site takes in place of xi I
   (Sec. III-C, last sentence of the discussion of Eq. tilted_P_1).  xi: DEVICE,
   op->m floats, each finite and > 0 (EP_TV_ERR_ARG otherwise), copied; p->xi is
   ignored.  Denoising: site 0 is (1/xi_p, y_p/xi_p), still exact.  Dense
   operator: K = diag(xi) + A C A^T in the Woodbury site, and the initial site 0
   of Algorithm 1 takes the mean of xi as its variance.  The periodic convolution
   is not supported with a noise plane (EP_TV_ERR_UNSUPPORTED).  Synchronises
   once (the variances are checked on the host). */
ep_tv_status ep_tv_init_noise(const ep_tv_operator* op, const float* y, const float* xi,
                              const ep_tv_params* p, void* cuda_stream, ep_tv_ctx** out);

/* ---- Row blocks of a sharded image (not in the paper) -----------------------
   One image split by rows over several processes or GPUs, denoising only.  A
   sweep (Algorithm 1) moves information across at most one row per vertical
   update (V3, V4), i.e. two rows per sweep, so a block that also holds the two
   rows above and below its own rows (its halo) computes the sweep of its own
   rows exactly as the whole image would, bit for bit.  After every sweep each
   block sends its two first and two last own rows of the prior sites to its
   neighbours' halos (ep_tv_block_halo_out / _in; the caller moves the buffers,
   e.g. with NCCL), and the EM statistic is the sum over blocks of each block's
   own edges (ep_tv_em_beta on a block returns it in abar_out and leaves beta
   alone; the caller sets beta = N / sum with ep_tv_set_beta). */
typedef struct {
  int32_t global_height;  /* rows of the whole image */
  int32_t row0;           /* first own row, even */
  int32_t rows;           /* own rows, >= 2 and < global_height (even on the torus) */
} ep_tv_block;

/* Creates the context of one row block.  op: EP_TV_OP_IDENTITY with width W and
   height = rows + halo above + halo below, the halos being 2 rows where the whole
   image has rows there (always on the torus, p->periodic = 1, which makes the
   columns wrap and the block's halo rows the torus neighbours of its own rows;
   on the free boundary none above row 0 or below the last row).  y: DEVICE, the
   observation of those rows, top halo first.  The block's own rows start at row
   2 of the context (0 if it has no top halo).  Other arguments as ep_tv_init;
   ep_tv_sweep refuses em_every > 0 on a block. */
ep_tv_status ep_tv_init_block(const ep_tv_operator* op, const float* y, const ep_tv_params* p,
                              const ep_tv_block* blk, void* cuda_stream, ep_tv_ctx** out);
/* Copies the block's first (side 0) or last (side 1) two own rows of the eight
   prior-site planes (tau_1..4, nu_1..4, each 2 x W, in that order) into buf
   (DEVICE, 16 W floats).  Asynchronous on the context's stream. */
ep_tv_status ep_tv_block_halo_out(ep_tv_ctx* ctx, int32_t side, float* buf);
/* Writes buf (as ep_tv_block_halo_out fills it, from the neighbour) into the
   block's halo rows above (side 0) or below (side 1).  Asynchronous. */
ep_tv_status ep_tv_block_halo_in(ep_tv_ctx* ctx, int32_t side, const float* buf);

/* Replaces the library-drawn probe vectors of the RBMC estimator (CONV_PERIODIC)
   by caller-drawn standard normals.  eps1: DEVICE, S x M; eps2: DEVICE, S x N;
   both copied.  The probes stay fixed across sweeps (common random numbers). */
ep_tv_status ep_tv_set_probes(ep_tv_ctx* ctx, const float* eps1, const float* eps2,
                              int32_t n_samples);

/* Runs n_sweeps sweeps of Algorithm 1.  k_order: HOST array of 4 * n_sweeps values,
   each group of four a permutation of {1,2,3,4} giving the order of the prior-site
   updates in that sweep; NULL means 1,2,3,4 every sweep.  em_every > 0 applies the
   EM update of beta after every em_every-th sweep of this call, on the device.
   Each sweep also records a_u for ep_tv_em_beta. */
ep_tv_status ep_tv_sweep(ep_tv_ctx* ctx, int32_t n_sweeps, const int8_t* k_order,
                         int32_t em_every);

/* EM M-step (Algorithm 2): beta <- N / a, with a the statistic chosen by
   params.em_option (default Option 3: a_u, the sum over all edges of E_{P_k}|u_n|
   taken during the last sweep), reduced in FP64 in a fixed order.  Enqueued on the stream.  If beta_out or abar_out is non-NULL the call
   synchronises the stream and writes the new beta / a_u there (HOST doubles).
   l1-TV prior only (EP_TV_ERR_UNSUPPORTED otherwise; ep_tv_sweep likewise
   refuses em_every > 0 for the mixture priors with EP_TV_ERR_ARG). */
ep_tv_status ep_tv_em_beta(ep_tv_ctx* ctx, double* beta_out, double* abar_out);

/* EP-EM (Algorithm 2) with the EP of Algorithm 1 run to convergence inside every
   EM iteration.  For each of n_em iterations: sweeps until the largest change of a
   posterior mean in one sweep is at most tol times the largest |posterior mean|
   (the reading of the paper's StopRule), or max_sweeps sweeps; then the EM update
   of beta with the statistic of params.em_option.  beta_out: HOST, n_em doubles,
   beta after each iteration; sweeps_out: HOST, n_em int32 (sweeps of each inner
   run), or NULL.  Synchronises after every sweep to read the change.  l1-TV only
   (EP_TV_ERR_UNSUPPORTED otherwise).  The fast variant of Sec. IV (a fixed, small
   number of sweeps per EM iteration) is ep_tv_sweep with em_every. */
ep_tv_status ep_tv_ep_em(ep_tv_ctx* ctx, int32_t n_em, int32_t max_sweeps, double tol,
                         double* beta_out, int32_t* sweeps_out);

/* Sets beta (no EM). */
ep_tv_status ep_tv_set_beta(ep_tv_ctx* ctx, double beta);

/* Posterior of Eq. Q_x_final: mean = nu_x / tau_x and var = 1 / tau_x, with
   tau_x, nu_x the sums of the five sites.  mean, var: DEVICE, N floats each. */
ep_tv_status ep_tv_posterior(ep_tv_ctx* ctx, float* mean, float* var);

/* Site natural parameters, for inspection: tau, nu DEVICE, 5 x N floats each,
   row s = site s (0 likelihood, 1..4 prior sites of V_1..V_4). */
ep_tv_status ep_tv_get_sites(ep_tv_ctx* ctx, float* tau, float* nu);

/* Synchronises the stream and returns the latched device status. */
ep_tv_status ep_tv_status_check(ep_tv_ctx* ctx);

/* Statistics of the last sweep call (HOST out-pointers may be NULL):
   cg_iters   conjugate-gradient iterations of the last likelihood-site update,
   n_fp64     number of edges whose moments were recomputed in FP64,
   n_capped   number of site updates that hit the variance cap.  Synchronises. */
ep_tv_status ep_tv_stats(ep_tv_ctx* ctx, int32_t* cg_iters, uint64_t* n_fp64,
                         uint64_t* n_capped);

/* Solver report of the last likelihood-site update (CONV_PERIODIC; zeros otherwise):
   refinement passes, conjugate-gradient iterations, and the final true relative
   residual ||b - Q x|| / ||b|| of the mean solve and the largest over the probe
   solves.  HOST out-pointers may be NULL.  Synchronises. */
ep_tv_status ep_tv_solver_report(ep_tv_ctx* ctx, int32_t* passes, int32_t* iterations,
                                 double* relres_mean, double* relres_probe_max);

/* Checkpoint: the full EP state (sites, beta, a_u, solver warm starts, counters).
   With host_buf == NULL, *bytes receives the size.  Otherwise host_buf (HOST,
   *bytes long) receives the state; synchronises.  A run resumed with
   ep_tv_state_import continues bit-identically. */
ep_tv_status ep_tv_state_export(ep_tv_ctx* ctx, void* host_buf, size_t* bytes);
ep_tv_status ep_tv_state_import(ep_tv_ctx* ctx, const void* host_buf, size_t bytes);

/* Re-initialises the sites (as ep_tv_init) and clears a latched error. */
ep_tv_status ep_tv_reset(ep_tv_ctx* ctx);

/* One complete restoration from HOST memory: copies y (HOST, op->m floats) to the
   device, runs n_sweeps sweeps with EM every em_every sweeps (0 = never), and
   copies the posterior mean and variance (HOST, N floats each) and the final beta
   (HOST, may be NULL) back.  op->kernel is HOST as in ep_tv_init; op->dense must
   be a DEVICE pointer.  Synchronous; allocates and frees its own context. */
ep_tv_status ep_tv_solve_host(const ep_tv_operator* op, const float* y_host,
                              const ep_tv_params* p, int32_t n_sweeps, int32_t em_every,
                              float* mean_host, float* var_host, double* beta_out);

/* Kernel classes reported by the tracer. */
typedef enum {
  EP_TV_K_PRIOR_SWEEP = 0,   /* fused V_1..V_4 prior-site pass, unit = pixel */
  EP_TV_K_CG_DIRECTION = 1,  /* CG direction + H^T H stencil (with 512-point FFT rows and a
                                separable blur also the previous iteration's correction
                                update), unit = pixel of one active system */
  EP_TV_K_CG_UPDATE = 2,     /* CG correction / residual update (with 512-point FFT rows: the
                                residual update fused with the preconditioner's forward row
                                pass), unit = pixel of one active system */
  EP_TV_K_CG_RESIDUAL = 3,   /* true CG residual of a refinement pass, unit = pixel of one
                                system */
  EP_TV_K_SITE0 = 4,         /* likelihood-site update, unit = pixel */
  EP_TV_K_CG_PRECOND = 5,    /* FFT circulant preconditioner (3 kernels; 2 in CG iterations whose
                                forward row pass runs with the update), unit = pixel of one
                                transformed system (pairs of stopped systems are skipped) */
  EP_TV_K_CS = 6,            /* compressive-sensing likelihood site (Woodbury, FP64-accurate)
                                except its tensor-core products, unit = pixel; its per-unit
                                figure is FP64 CUDA-core flops, not bytes */
  EP_TV_K_CG_COMMIT = 7,     /* adds a refinement pass's FP32 correction to the FP64 solution,
                                unit = pixel of one system that iterated in the pass */
  EP_TV_K_CS_MMA = 8,        /* the compressive-sensing site's products as exact BF16 slice
                                products on the tensor cores (packing included), unit = BF16
                                tensor flop (per-unit figure 1) */
  EP_TV_K_COUNT = 9
} ep_tv_kernel;

/* Tracing: with on != 0, every launch of the kernel classes above is bracketed
   by CUDA events on the context's stream.  ep_tv_trace_read synchronises and
   returns, for one class since tracing was enabled: total device milliseconds,
   number of launches, units processed, and the algorithmic DRAM bytes per unit
   (what the kernel must read and write at least once).  HOST out-pointers may
   be NULL.  Enabling resets the totals. */
ep_tv_status ep_tv_trace_enable(ep_tv_ctx* ctx, int32_t on);
ep_tv_status ep_tv_trace_read(ep_tv_ctx* ctx, int32_t kernel, double* ms, int64_t* launches,
                              double* units, double* bytes_per_unit);

/* One pass of the four prior-site updates (the kernel ep_tv_sweep runs) that
   allocates no device memory.  The paper has no counterpart: this exists for
   callers that cannot call cudaMalloc when they run a sweep, e.g. code that must
   not allocate after start-up, or runs inside an allocator or host runtime that
   owns the device memory and only hands out the buffers it was asked for.  The
   caller passes every input and output; the scratch the pass needs (one FP64
   partial sum of E|u| per work unit of 16 row pairs of a 60-column strip, a
   status word, counters) lives in a file-scope device array of 65536 + 8 doubles
   (512 KB) that every GPU loading the library holds until the process exits.
     height, width  image size; its ceil(width / 60) * ceil(((height + 1) / 2 + 1) / 16)
                    work units (about 126 M pixels at most) must not exceed 65536, and
                    height * width must not exceed 2^31, else EP_TV_ERR_ARG.
     p              uses damping, var_cap, periodic, precision (0 or 1), the prior and
                    its omega, s1_sq, s2_sq, and xi when y is given.
     beta           DEVICE pointer to the TV parameter (one double).
     y              DEVICE, N floats: denoising, site 0 = (1/xi, y/xi); or NULL and
     tau0, nu0      DEVICE, N floats each: the likelihood site.
     tau_in, nu_in  DEVICE, 4 x N floats each: prior sites k = 1..4 (row k-1) before
                    the pass.
     tau_out, nu_out DEVICE, 4 x N floats each: after the pass; must not alias the inputs.
     k_order        HOST, 4 values, a permutation of 1..4, or NULL for 1,2,3,4.
     abar_out       DEVICE, one double: a_u of this pass (sum of E|u| over all edges).
     flags_out      DEVICE, one uint32 or NULL: 1 if a site value became non-finite.
     cuda_stream    stream (cudaStream_t or NULL) the work is enqueued on.
   All calls on a device share the scratch array and it keeps the last call's
   contents: calls that overlap on the GPU race and must be serialised by the
   caller.  The first call on a device looks up the array's device address with
   that device current and keeps it; make it before any stream capture begins,
   and do not call this entry point again after cudaDeviceReset on that device
   (the kept address belongs to the reset context).  Asynchronous. */
ep_tv_status ep_tv_prior_sweep_noalloc(int32_t height, int32_t width, const ep_tv_params* p,
                                       const double* beta, const float* y, const float* tau0,
                                       const float* nu0, const float* tau_in, const float* nu_in,
                                       float* tau_out, float* nu_out, const int8_t* k_order,
                                       double* abar_out, uint32_t* flags_out, void* cuda_stream);

/* Batches (not in the paper): advance many independent problems together.  All
   contexts must live on the same device and stream and use order_mode 0; a
   context belongs to at most one batch at a time and stays usable on its own
   (posterior, sites, EM) between batch sweeps.  The batch keeps the context
   pointers (the caller still owns and frees the contexts, after the batch). */
typedef struct ep_tv_batch ep_tv_batch;
ep_tv_status ep_tv_batch_create(int32_t n, ep_tv_ctx* const* ctxs, ep_tv_batch** out);
/* n_sweeps sweeps of every context: one persistent launch runs the prior-site
   pass of all images (warps take contiguous ranges of the images' work units,
   found through a table), then the likelihood-site
   updates run concurrently on one worker stream per context, each driven by a host
   thread of a pool of up to 16; with em_every > 0 every context's beta is updated
   after each em_every-th sweep.  Returns when all work is enqueued (the likelihood
   solvers synchronise with their own streams while they run). */
ep_tv_status ep_tv_batch_sweep(ep_tv_batch* batch, int32_t n_sweeps, int32_t em_every);
/* Synchronises and frees the batch (not the contexts).  NULL is accepted. */
void ep_tv_batch_destroy(ep_tv_batch* batch);

/* CUDA graphs (not in the paper).  Contexts without a likelihood solver
   (denoising) and batches of them, on a stream other than the legacy default
   stream, with tracing off and the default update order, run ep_tv_sweep /
   ep_tv_batch_sweep calls of at least two periods of lcm(2, em_every) sweeps by
   replaying a graph of one period, captured on first use (thread-local capture
   mode) and cached per buffer parity; the remaining sweeps are launched
   directly.  The deconvolution site runs every update, with tracing off and on
   such a stream, as one graph whose refinement passes and CG iterations are
   conditional WHILE nodes driven by device-side counters (no host round trip
   inside an update), captured on first use per prior-site buffer; with tracing
   on it runs the host-driven loop.  Results are identical to direct launches.
   Returns how many of the context's sweeps ran from graph replays (-1 for NULL). */
int64_t ep_tv_graph_sweeps(const ep_tv_ctx* ctx);

/* ---- Learned warm start (not in the paper) ----------------------------------
   A small fully convolutional network predicts, from an observation, a per-pixel
   guess of the EP posterior mean and log-variance; ep_tv_warm_start turns the
   guess into sites before plain EP sweeps, which then correct its error
   (a context that is never warm-started is the cold-start fallback).  The calls
   below are the network's building blocks.  Arrays are float32 in NCHW order
   (image, channel, row, column), DEVICE pointers; every call is asynchronous on
   cuda_stream and returns EP_TV_ERR_ARG for invalid sizes or NULL pointers. */

/* y = conv3x3(x, weight) + bias on the torus (circular one-pixel padding), then a
   ReLU if relu != 0.  x: n x cin x h x w; weight: cout x cin x 3 x 3, the taps of a
   cross-correlation, y[o](i, j) = bias[o] + sum_c sum_{a,e} weight[o, c, a, e]
   x[c]((i + a - 1) mod h, (j + e - 1) mod w); bias: cout floats or NULL; y: n x cout
   x h x w, must not alias x.  1 <= cout <= 32, 1 <= n <= 65535. */
ep_tv_status ep_tv_conv3x3_forward(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                   int32_t width, const float* x, const float* weight,
                                   const float* bias, int32_t relu, float* y, void* cuda_stream);
/* Bytes of DEVICE scratch ep_tv_conv3x3_backward needs for these sizes (0 if invalid). */
size_t ep_tv_conv3x3_backward_work(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                   int32_t width);
/* Gradients through one ep_tv_conv3x3_forward call given dy = dL/dy.  y is that
   call's output when it applied the ReLU (dy is masked by y > 0), else NULL.
   Overwrites dweight (cout x cin x 3 x 3), dbias (cout) and, unless it is NULL,
   dx (n x cin x h x w; needs cin <= 32).  work: DEVICE scratch of at least
   ep_tv_conv3x3_backward_work bytes, owned by the caller.  The weight gradient
   is summed per 16 x 16 tile and then over tiles in a fixed order
   (deterministic). */
ep_tv_status ep_tv_conv3x3_backward(int32_t n, int32_t cin, int32_t cout, int32_t height,
                                    int32_t width, const float* x, const float* weight,
                                    const float* y, const float* dy, float* dx, float* dweight,
                                    float* dbias, void* work, size_t work_bytes, void* cuda_stream);
/* One Adam step (Kingma and Ba) on count parameters in place; m, v are the moment
   buffers (start at zero), t the step number from 1. */
ep_tv_status ep_tv_adam_step(int64_t count, float* param, const float* grad, float* m, float* v,
                             int32_t t, float lr, float beta1, float beta2, float eps,
                             void* cuda_stream);
/* Training loss of the warm start against converged states of plain EP.  out is
   the network output, n x 6 x h x w; y and mean are n x h x w (observation, EP
   posterior mean); tau is n x 5 x h x w (the EP site precisions, site 0 first);
   log_xi holds n floats, log of each image's noise variance.  With targets
   t0 = mean - y and t[1 + s] = log(tau_s) + log_xi, loss = mean over images and
   pixels of w_mean (out0 - t0)^2 + (1/5) sum_s (out[1 + s] - t[1 + s])^2.
   Writes dL/dout (n x 6 x h x w) and the loss (DEVICE, one double). */
ep_tv_status ep_tv_warmstart_loss(int32_t n, int32_t height, int32_t width, const float* out,
                                  const float* y, const float* mean, const float* tau,
                                  const float* log_xi, float w_mean, float* dout, double* loss,
                                  void* cuda_stream);
/* Which sites ep_tv_warm_start sets. */
typedef enum {
  EP_TV_WARM_ALL_SITES = 0,  /* all five sites from the prediction */
  EP_TV_WARM_SITE0 = 1,      /* the likelihood site only; the prior sites keep their
                                initial (capped) values, as in the cold start */
  EP_TV_WARM_PRIOR = 2       /* the four prior sites only; the likelihood site keeps
                                its initial value (y/xi, 1/xi) and is formed by the
                                first sweep from the warm prior sites */
} ep_tv_warm_mode;

/* Sets sites of a context from the warm-start network's output for its
   observation (DEVICE, 6 x N floats): the predicted posterior mean is
   y + out[0] (y and xi of the context; not for the dense operator, EP_TV_ERR_ARG),
   and site s gets the precision tau_s = exp(out[1 + s]) / xi (prior sites capped
   below at 1/var_cap) and the predicted mean, nu_s = tau_s (y + out[0]).  mode
   (ep_tv_warm_mode) selects the sites.  For denoising, site 0 is exact from the
   start and keeps (1/xi, y/xi) (EP_TV_WARM_SITE0 then changes nothing).  Call it
   after ep_tv_init (or ep_tv_reset) and before sweeping. */
ep_tv_status ep_tv_warm_start(ep_tv_ctx* ctx, const float* out, int32_t mode);

/* The FP64-accurate product of the compressive-sensing site on the BF16 tensor
   cores (Sec. III-C, the products of the Woodbury form), exposed to check it on
   its own: C = A B^T for row-major A (m x k), B (n x k) and C (m x n), all DEVICE
   pointers, on cuda_stream (NULL: the legacy stream).  Every FP64 entry is split
   into `slices` 7-bit BF16 digit slices under a power-of-two scale per row; the
   slices (slices + 1) / 2 slice products with the largest weights run as BF16
   MMAs (tcgen05) whose partial sums are exact up to a short FP32 tail.
   slices = 8 is the form of the site's operator products: |C - A B^T| <~
   2^-55 (max|A_i| sum|B_j| + max|B_j| sum|A_i|) + 2^-52 k max|A_i| max|B_j| plus one
   rounding of the result.  slices = 10 (k <= 8192) is the form of its Cholesky
   factorisation's products, about 2^-14 of that error.  Allocates and frees its
   packing buffers (about 2 slices (m + n) k bytes) and synchronises the stream.
   EP_TV_ERR_ARG for NULL pointers, sizes below 1 or another slice count,
   EP_TV_ERR_NOMEM, EP_TV_ERR_TIMEOUT if a bounded device-side wait gave up. */
ep_tv_status ep_tv_tc_gemm_f64(const double* A, const double* B, double* C, int32_t m, int32_t n,
                               int32_t k, int32_t slices, void* cuda_stream);

/* Frees the context (synchronises its stream first).  NULL is accepted. */
void ep_tv_destroy(ep_tv_ctx* ctx);

/* Static English description of a status code. */
const char* ep_tv_status_str(ep_tv_status s);

#ifdef __cplusplus
}
#endif
#endif /* EP_TV_H */
