// Likelihood site q_{x,0} for a periodic convolution H (deconvolution).
//
// Eq. tilted_P_1: the tilted P_0 is Gaussian with precision
//   Q = H^T H / xi + diag(d),  d = cavity precision of site 0 = sum_{k=1..4} tau_k,
// mean E = Q^{-1} (H^T y / xi + n), n = sum_{k=1..4} nu_k (cavity natural mean).
// Only diag(Q^{-1}) is needed (Sec. III-C).  The paper names Rao-Blackwellised
// Monte Carlo for it; the estimator here (fixed probes, so the EP map stays
// deterministic across sweeps) is
//   z_s = Q^{-1} w_s,  w_s = H^T eps1_s / sqrt(xi) + sqrt(d) eps2_s   (cov w_s = Q)
//   Var_i = 1/Q_ii + (1/S) sum_s (sum_{j != i} Q_ij z_{s,j})^2 / Q_ii^2,
// with the off-diagonal sum taken from an explicit matvec of the computed z_s
// (rb_offdiag_kernel), so that the estimate does not depend on how closely the
// probe solves met their tolerance.
// The 1 + S systems share Q and are solved together by conjugate gradients with
// a circulant (FFT) preconditioner, in FP32 with FP64 dot products inside an
// iterative refinement on a float-float true residual, warm-started from the
// previous sweep's solutions.  Then Eq. update_q0_x with cap and damping.
//
// Q p is a periodic stencil: H^T H is the autocorrelation of the kernel,
// G(a, b) = sum_{u,v} k[u,v] k[u+a, v+b], |a| <= kh-1, |b| <= kw-1.  A separable
// kernel k = u v^T gives G = autocorr(u) x autocorr(v), applied as two 1-D passes;
// otherwise H then H^T are applied in shared memory.
//
// Layout: every vector is one FP32 plane of N = H*W pixels, row-major; the
// 1 + S right-hand sides are consecutive planes ([0] = mean system).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"
#include "likelihood.cuh"

namespace eptv {

namespace {

constexpr int kTile = 32;        // stencil and update tile, kTile x kTile pixels
constexpr int kThreads = 256;
constexpr int kMaxHalf = 14;     // H^T H half-width, kernels up to 15 x 15
constexpr int kChunk = 4;        // CG iterations between convergence polls

struct ConvDesc {
  int H, W;
  long long N;
  int kh, kw;
  int hr, hc;            // H^T H half-widths: kh - 1, kw - 1
  int separable;
  const float* k;        // kh x kw
  const float* gr;       // 2 hr + 1 (separable)
  const float* gc;       // 2 hc + 1 (separable)
  const double* hd;      // forward-blur taps, FP64: separable u (kh) then v (kw), else k
  const float* hf;       // the same taps in FP32
  float inv_xi;
  double inv_xi_d;
  float g0_xi;           // diag of H^T H / xi = sum k^2 / xi
  int tiles_x, tiles_y;
};

__device__ __forceinline__ int wrapi(int v, int n) {
  if (v >= 0 && v < n) return v;  // the common cases without a division
  if (v < 0 && v >= -n) return v + n;
  if (v >= n && v < 2 * n) return v - n;
  v %= n;
  return v < 0 ? v + n : v;
}

// Wrapped global column of each region column, computed once per block
// (region columns < 64 + 2 * 28).  Rows are wrapped once per row in the loops.
__device__ __forceinline__ void column_table(int* tab, int c_first, int n_cols, int W) {
  for (int cc = threadIdx.x; cc < n_cols; cc += blockDim.x) tab[cc] = wrapi(c_first + cc, W);
}

struct StencilSmem {
  float* v;    // region (kTile + 2 hr) x (kTile + 2 hc)
  float* tmp;  // separable: (kTile + 2 hr) x kTile; otherwise (kTile + hr) x (kTile + hc)
  float* taps; // kernel taps staged in shared memory
};

// Separable H^T H with compile-time half-widths.  Row pass: each thread produces
// two adjacent outputs of a region row from one window of 2 HC + 2 inputs read as
// float2 (16 threads per row); column pass: each thread produces four consecutive
// rows of one column, so the 2 HR + 4 inputs it loads serve four outputs.  Every
// output sums its taps in the same order as a one-output loop.
template <int HR, int HC>
__device__ __forceinline__ void hth_tile_sep(StencilSmem& sm, float* out) {
  constexpr int RH = kTile + 2 * HR, RW = kTile + 2 * HC;
  const float* gr = sm.taps;
  const float* gc = sm.taps + (2 * HR + 1);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float wc[2 * HC + 1];
#pragma unroll
  for (int b = 0; b <= 2 * HC; ++b) wc[b] = gc[b];
  static_assert(RW % 2 == 0, "float2 rows");
  const int cp = threadIdx.x & 15;  // column pair 2 cp, 2 cp + 1 of the tile
  for (int rr = threadIdx.x >> 4; rr < RH; rr += kThreads / 16) {
    const float2* row2 = reinterpret_cast<const float2*>(sm.v + rr * RW + 2 * cp);
    float win[2 * HC + 2];
#pragma unroll
    for (int q = 0; q <= HC; ++q) {
      const float2 t = row2[q];
      win[2 * q] = t.x;
      win[2 * q + 1] = t.y;
    }
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int b = 0; b <= 2 * HC; ++b) {
      a0 = fmaf(wc[b], win[b], a0);
      a1 = fmaf(wc[b], win[b + 1], a1);
    }
    *reinterpret_cast<float2*>(sm.tmp + rr * kTile + 2 * cp) = make_float2(a0, a1);
  }
  __syncthreads();
  float wr[2 * HR + 1];
#pragma unroll
  for (int a = 0; a <= 2 * HR; ++a) wr[a] = gr[a];
  // 8 warps x 4 rows = 32 output rows
  const int tr0 = ty * 4;
  float in[2 * HR + 4];
#pragma unroll
  for (int i = 0; i < 2 * HR + 4; ++i) in[i] = sm.tmp[(tr0 + i) * kTile + tx];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a <= 2 * HR; ++a) acc = fmaf(wr[a], in[o + a], acc);
    out[(tr0 + o) * kTile + tx] = acc;
  }
  __syncthreads();
}

// out[tr * kTile + tc] = (H^T H v)(tile pixel) for the region staged in sm.v.
// All threads of the block participate; ends with __syncthreads().
__device__ void hth_tile(const ConvDesc& c, StencilSmem& sm, float* out) {
  if (c.separable && c.hr == c.hc) {
    switch (c.hr) {
      case 2: hth_tile_sep<2, 2>(sm, out); return;
      case 4: hth_tile_sep<4, 4>(sm, out); return;
      case 8: hth_tile_sep<8, 8>(sm, out); return;
      case 14: hth_tile_sep<14, 14>(sm, out); return;
      default: break;
    }
  }
  const int RH = kTile + 2 * c.hr, RW = kTile + 2 * c.hc;
  const int tid = threadIdx.x;
  if (c.separable) {
    const float* gr = sm.taps;
    const float* gc = sm.taps + (2 * c.hr + 1);
    // pass 1: along rows, all region rows, tile columns
    for (int idx = tid; idx < RH * kTile; idx += kThreads) {
      const int rr = idx / kTile, tc = idx - rr * kTile;
      const float* row = sm.v + rr * RW + tc;
      float acc = 0.f;
      for (int b = 0; b <= 2 * c.hc; ++b) acc = fmaf(gc[b], row[b], acc);
      sm.tmp[idx] = acc;
    }
    __syncthreads();
    // pass 2: along columns
    for (int idx = tid; idx < kTile * kTile; idx += kThreads) {
      const int tr = idx / kTile, tc = idx - tr * kTile;
      const float* col = sm.tmp + tr * kTile + tc;
      float acc = 0.f;
      for (int a = 0; a <= 2 * c.hr; ++a) acc = fmaf(gr[a], col[a * kTile], acc);
      out[idx] = acc;
    }
    __syncthreads();
  } else {
    const float* k = sm.taps;
    const int hh = c.kh / 2, hw = c.kw / 2;
    const int UH = kTile + 2 * hh, UW = kTile + 2 * hw;
    // u = H v on the tile plus a (kh/2, kw/2) halo: u(r,c) = sum k[a,b] v(r-a+hh, c-b+hw)
    for (int idx = tid; idx < UH * UW; idx += kThreads) {
      const int ur = idx / UW, uc = idx - ur * UW;
      float acc = 0.f;
      for (int a = 0; a < c.kh; ++a) {
        const float* vrow = sm.v + (ur - a + c.hr) * RW + uc + c.hc;
        const float* krow = k + a * c.kw;
        for (int b = 0; b < c.kw; ++b) acc = fmaf(krow[b], vrow[-b], acc);
      }
      sm.tmp[idx] = acc;
    }
    __syncthreads();
    // out = H^T u: out(r,c) = sum k[a,b] u(r+a-hh, c+b-hw)
    for (int idx = tid; idx < kTile * kTile; idx += kThreads) {
      const int tr = idx / kTile, tc = idx - tr * kTile;
      float acc = 0.f;
      for (int a = 0; a < c.kh; ++a) {
        const float* urow = sm.tmp + (tr + a) * UW + tc;
        const float* krow = k + a * c.kw;
        for (int b = 0; b < c.kw; ++b) acc = fmaf(krow[b], urow[b], acc);
      }
      out[idx] = acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void stage_taps(const ConvDesc& c, float* taps) {
  if (c.separable) {
    const int nr = 2 * c.hr + 1, nc = 2 * c.hc + 1;
    for (int i = threadIdx.x; i < nr + nc; i += kThreads) taps[i] = i < nr ? c.gr[i] : c.gc[i - nr];
  } else {
    for (int i = threadIdx.x; i < c.kh * c.kw; i += kThreads) taps[i] = c.k[i];
  }
}

__device__ __forceinline__ StencilSmem carve(const ConvDesc& c, float* base) {
  StencilSmem sm;
  const int RH = kTile + 2 * c.hr, RW = kTile + 2 * c.hc;
  sm.taps = base;
  sm.v = base + 512;
  sm.tmp = sm.v + RH * RW;
  return sm;
}

// FP64 block sum of up to three per-thread values, written by thread 0 (any block
// size up to 1024 threads, a multiple of 32).
__device__ __forceinline__ void block_sum3(double a, double b, double c3, double* out_a,
                                           double* out_b, double* out_c) {
  __shared__ double red[3][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
    c3 += __shfl_down_sync(0xffffffffu, c3, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c3;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0, sc = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      sa += red[0][i];
      sb += red[1][i];
      sc += red[2][i];
    }
    if (out_a) *out_a = sa;
    if (out_b) *out_b = sb;
    if (out_c) *out_c = sc;
  }
  __syncthreads();
}

// block_sum3 for per-thread FP32 partials of NV values (1..3): the sums within a
// warp run in FP32 (the CG's vectors are FP32 already), the warps' sums are added
// in FP64 in a fixed order.  GB300's FP64 pipe is narrow, and a five-level FP64
// shuffle tree per value in every block of the CG kernels kept it busy.
template <int NV>
__device__ __forceinline__ void block_sumf(float a, float b, float c3, double* out_a, double* out_b,
                                           double* out_c) {
  __shared__ double red[3][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    if (NV > 1) b += __shfl_down_sync(0xffffffffu, b, off);
    if (NV > 2) c3 += __shfl_down_sync(0xffffffffu, c3, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = (double)a;
    red[1][w] = (double)b;
    red[2][w] = (double)c3;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0, sc = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      sa += red[0][i];
      if (NV > 1) sb += red[1][i];
      if (NV > 2) sc += red[2][i];
    }
    if (out_a) *out_a = sa;
    if (NV > 1 && out_b) *out_b = sb;
    if (NV > 2 && out_c) *out_c = sc;
  }
  __syncthreads();
}

// Last-block reduction.  Every block of a group has written its partial sum (by
// thread 0, before the block barrier at the end of block_sum3); each then counts
// itself in with an atomic, and the block that arrives last returns true and
// resets the counter for the next launch.  That block sums the group's partials
// in index order (group_sum), so the result does not depend on which block it is.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned n_blocks) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial is visible before it is counted
    last = atomicAdd(counter, 1u) == n_blocks - 1;
    if (last) atomicExch(counter, 0u);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of n partials in a fixed order, by the first warp of a block (all 32 lanes
// get the result).  Loads bypass L1: the partials were written by other SMs.
__device__ __forceinline__ double group_sum(const double* part, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += __ldcg(part + i);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

struct CgArgs {
  ConvDesc c;
  int R;                 // right-hand sides (1 + S)
  int S;
  double* X;             // R planes, FP64 solutions
  float* Rr;             // R planes
  float* P;              // R planes: search directions of even iterations
  float* P2;             // R planes: search directions of odd iterations.  Two buffers
                         // because a tile reads the previous direction over its halo
                         // while neighbouring tiles write the new one.
  float* Qp;             // R planes
  const float* D;        // cavity precision
  const float* Ncav;     // cavity natural mean
  const float* Minv;     // 1 / diag(Q)
  const float* Hty;      // H^T y / xi
  const float* E1;       // S planes, H^T eps1 / sqrt(xi)
  const float* E2;       // S planes, eps2
  const float* Y0;       // observation y
  const float* Y1;       // S planes, sqrt(xi) eps1 (data-space probe)
  const double* thr;     // [R] inner-loop convergence threshold on r.r
  const double* rr0;     // [R] r.r at the start of the refinement pass
  float* Z;              // R planes, preconditioned residual (FFT preconditioner)
  float* Ec;             // R planes, FP32 correction summed over one refinement pass
  double* part_pq;       // [R][nb]
  double* part_rz;       // [R][nbz]
  double* part_rr;       // [R][nb]
  double* part_bb;       // [R][nb]
  double rtol2;
  float* scal;           // [R][4]: active flag, beta; each written by the last block
                         // of the kernel whose partial sums it needs
  double* rzs;           // [R] r.z of the current iteration
  unsigned* arrive;      // [R] block-arrival counters of the update kernel
  const int* act0;       // [R] 1 if the system iterates in the current refinement pass
  const int* it_dev;     // iteration index in device memory (graph replays), or NULL: the
                         // kernels' it argument
  int nb;                // tile blocks per system
  int nbz;               // blocks per system producing r.z partials
  int fft;               // 1: z = M^{-1} r by the circulant preconditioner, else Jacobi
  unsigned long long* counters;
  int defer_e;           // 1: the update leaves e += alpha p to the next direction kernel
                         // (or the commit), see fft512_update_rows_fwd_kernel
};

// d = sum tau_k, n = sum nu_k (k = 1..4), Minv = 1 / (sum k^2 / xi + d); block sums of d.
__global__ void __launch_bounds__(kThreads) prep_kernel(const float* __restrict__ tp,
                                                        const float* __restrict__ np, long long N,
                                                        float g0_xi, float* D, float* Ncav,
                                                        float* Minv, double* dpart) {
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const float d = tp[p] + tp[N + p] + tp[2 * N + p] + tp[3 * N + p];
    const float n = np[p] + np[N + p] + np[2 * N + p] + np[3 * N + p];
    D[p] = d;
    Ncav[p] = n;
    Minv[p] = 1.0f / (g0_xi + d);
    acc += (double)d;
  }
  block_sum3(acc, 0.0, 0.0, dpart + blockIdx.x, nullptr, nullptr);
}

// dbar = mean of d over the image (fixed-order reduction of the block sums).
__global__ void mean_kernel(const double* dpart, int n, double inv_count, double* out) {
  __shared__ double buf[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += dpart[i];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = buf[0] * inv_count;
}

// Float-float ("double-single") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// giving about 44 significant bits from FP32 operations only (GB300's FP64 rate is a
// small fraction of its FP32 rate).  TwoSum is Knuth's, TwoProduct uses the FMA
// (Dekker's splitting is not needed with a fused multiply-add).
struct ff {
  float hi, lo;
};
// The _rn intrinsics keep the compiler from fusing these products and sums into
// FMAs, which would break the error-free transformations.
__device__ __forceinline__ ff ff_from_double(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
// x as hi + lo without FP64 arithmetic (GB300's FP64 pipe retires about one
// operation per clock per SM, and the residual stages one FP64 value per region
// pixel): hi is x truncated to 24 significant bits, assembled from the bit fields;
// lo is the remaining 29 mantissa bits, converted as an integer (rounded to 24
// bits) and scaled by a power of two, so |x - hi - lo| <= 2^-47 |x|.  Zero is
// exact; magnitudes below 2^-74 or beyond float's range take ff_from_double.
__device__ __forceinline__ ff ff_split_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  if ((u << 1) == 0ull) return {0.f, 0.f};
  const int ef = (int)((u >> 52) & 0x7FFull) - 1023 + 127;  // biased float exponent of hi
  if (ef < 53 || ef > 254) return ff_from_double(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29));
  const float scale = __uint_as_float((unsigned)(ef - 52) << 23);  // 2^(ef - 127 - 52), normal
  const float lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) * scale;
  return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// acc + x * g with g = g_hi + g_lo
__device__ __forceinline__ ff ff_fma(ff acc, ff x, float g_hi, float g_lo) {
  const float p = __fmul_rn(x.hi, g_hi);
  float e = fmaf(x.hi, g_hi, -p);
  e = fmaf(x.hi, g_lo, fmaf(x.lo, g_hi, e));
  const ff s = two_sum(acc.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, acc.lo), e));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// a * b for float b
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = fmaf(a.hi, b, -p);
  return fast_two_sum(p, fmaf(a.lo, b, e));
}

// Float-float on pairs: (value of system 0, value of system 1) in each float2, with
// the packed FP32 add, multiply and FMA of sm_100-family GPUs.  Every packed
// operation rounds each lane as the scalar one does, so a pair gives what two scalar
// evaluations of the same expressions give.
struct ff2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {  // a - b, one rounding
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b) {  // |a| >= |b|
  const float2 s = f2add(a, b);
  return {s, f2sub(b, f2sub(s, a))};
}
// ff_fma on pairs: acc + x * g with the tap g = g_hi + g_lo common to both lanes,
// given as gh = (g_hi, g_hi), gl = (g_lo, g_lo) and gn = -gh.  The product is formed
// negated (x.hi * -g_hi = -p exactly), so TwoSum(acc.hi, p) is written with
// subtractions of -p; each lane's result equals ff_fma's.
__device__ __forceinline__ ff2 ff2_fma(ff2 acc, ff2 x, float2 gh, float2 gl, float2 gn) {
  const float2 pn = f2mul(x.hi, gn);
  float2 e = f2fma(x.hi, gh, pn);
  e = f2fma(x.hi, gl, f2fma(x.lo, gh, e));
  const float2 sh = f2sub(acc.hi, pn);                                   // acc.hi + p
  const float2 bb = f2sub(sh, acc.hi);
  const float2 sl = f2sub(f2sub(acc.hi, f2sub(sh, bb)), f2add(pn, bb));  // + (p - bb)
  return fast_two_sum2(sh, f2add(f2add(sl, acc.lo), e));
}
// y - acc for y exact in FP32 (lo = 0), as ff_add(ff{y, 0}, ff_neg(acc)) per lane
__device__ __forceinline__ ff2 ff2_sub_from(float2 y, ff2 acc) {
  const float2 sh = f2sub(y, acc.hi);
  const float2 bb = f2sub(sh, y);                                        // s - a, a = y
  const float2 sl = f2sub(f2sub(y, f2sub(sh, bb)), f2add(acc.hi, bb));   // (a - (s - bb)) + (-acc.hi - bb)
  return fast_two_sum2(sh, f2sub(f2add(sl, make_float2(0.f, 0.f)), acc.lo));
}

// The separable part of residual_kernel with a compile-time K x K kernel: the
// same float-float H x and FP32 H^T sums in the same order, with the region
// sizes, index divisions and tap loops resolved at compile time.
template <int K>
__device__ __forceinline__ void residual_sep_fixed(const ConvDesc& c, const float* taph,
                                                   const float* tapl, const float* xh,
                                                   const float* xl, float* ph, float* pl, float* vs,
                                                   float* tmpf, float* outb, const float* yp, int r0,
                                                   int c0) {
  constexpr int hh = K / 2, hw = K / 2;
  constexpr int RH = kTile + 2 * (K - 1), RW = RH;
  constexpr int MH = kTile + 2 * hh, MW = MH;
  float uh[K], ul[K], vh[K], vl[K];
#pragma unroll
  for (int b = 0; b < K; ++b) {
    uh[b] = taph[b];
    ul[b] = tapl[b];
    vh[b] = taph[K + b];
    vl[b] = tapl[K + b];
  }
  // Both float-float passes produce two adjacent outputs per thread from one
  // window of K + 1 inputs (the row pass reads it as float2); every output sums its
  // taps in the same order as a one-output loop.
  static_assert(K % 2 == 1 && RW % 2 == 0 && MW % 2 == 0 && MH % 2 == 0, "paired outputs");
  for (int idx = threadIdx.x; idx < RH * (MW / 2); idx += kThreads) {
    const int rr = idx / (MW / 2), mp = idx - rr * (MW / 2);
    // outputs (rr, 2 mp) and (rr, 2 mp + 1) read x[rr][2 mp .. 2 mp + K]
    const float2* h2 = reinterpret_cast<const float2*>(xh + rr * RW + 2 * mp);
    const float2* l2 = reinterpret_cast<const float2*>(xl + rr * RW + 2 * mp);
    float wh[K + 1], wl[K + 1];
#pragma unroll
    for (int q = 0; q < (K + 1) / 2; ++q) {
      const float2 th = h2[q], tl = l2[q];
      wh[2 * q] = th.x;
      wh[2 * q + 1] = th.y;
      wl[2 * q] = tl.x;
      wl[2 * q + 1] = tl.y;
    }
    ff acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
#pragma unroll
    for (int b = 0; b < K; ++b) {
      acc0 = ff_fma(acc0, ff{wh[K - 1 - b], wl[K - 1 - b]}, vh[b], vl[b]);
      acc1 = ff_fma(acc1, ff{wh[K - b], wl[K - b]}, vh[b], vl[b]);
    }
    const int o = rr * MW + 2 * mp;
    ph[o] = acc0.hi;
    pl[o] = acc0.lo;
    ph[o + 1] = acc1.hi;
    pl[o + 1] = acc1.lo;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < (MH / 2) * MW; idx += kThreads) {
    const int mp = idx / MW, mc = idx - mp * MW, mr = 2 * mp;
    // outputs (mr, mc) and (mr + 1, mc) read rows mr .. mr + K of column mc
    const int gcol = wrapi(c0 - hw + mc, c.W);
    const float y0 = yp[(long long)wrapi(r0 - hh + mr, c.H) * c.W + gcol];
    const float y1 = yp[(long long)wrapi(r0 - hh + mr + 1, c.H) * c.W + gcol];
    float wh[K + 1], wl[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      wh[j] = ph[(mr + j) * MW + mc];
      wl[j] = pl[(mr + j) * MW + mc];
    }
    ff acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
#pragma unroll
    for (int aa = 0; aa < K; ++aa) {
      acc0 = ff_fma(acc0, ff{wh[K - 1 - aa], wl[K - 1 - aa]}, uh[aa], ul[aa]);
      acc1 = ff_fma(acc1, ff{wh[K - aa], wl[K - aa]}, uh[aa], ul[aa]);
    }
    const ff v0 = ff_add(ff{y0, 0.f}, ff_neg(acc0));
    const ff v1 = ff_add(ff{y1, 0.f}, ff_neg(acc1));
    vs[mr * MW + mc] = v0.hi + v0.lo;
    vs[(mr + 1) * MW + mc] = v1.hi + v1.lo;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < MH * kTile; idx += kThreads) {
    const int mr = idx / kTile, tc = idx - mr * kTile;
    const float* row = vs + mr * MW + tc;
    float acc = 0.f;
#pragma unroll
    for (int b = 0; b < K; ++b) acc = fmaf(vh[b], row[b], acc);
    tmpf[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
    const int tr = idx / kTile, tc = idx - tr * kTile;
    const float* col = tmpf + tr * kTile + tc;
    float acc = 0.f;
#pragma unroll
    for (int aa = 0; aa < K; ++aa) acc = fmaf(uh[aa], col[aa * kTile], acc);
    outb[idx] = acc;
  }
}

// True residual of every system (blockIdx.z),
//   r = H^T (y' - H x) / xi + (n' - d x),
// y' = y, n' = n for the mean system and y' = sqrt(xi) eps1_s, n' = sqrt(d) eps2_s for
// probe s, so that r = b - Q x with the right-hand side b = H^T y / xi + n (mean) or
// b = H^T eps1_s / sqrt(xi) + sqrt(d) eps2_s (probe s).  Near the solution H^T H x / xi
// and d x are several times larger than r; evaluated in FP32 they leave an error of
// order eps |H^T y'| / xi, which the conditioning of Q (1e4..1e5) turns into
// percent-level errors in x.  So H x and n' - d x are formed in float-float from the
// FP64 solution; y' - H x is then small and its H^T / xi runs in FP32, which bounds
// the relative residual error by about 1e-10 for the mean system and 1e-7 for the
// probes, below their targets.  Partials: r.r (buffer 0), b.b, r.Minv.r (Jacobi).
__global__ void __launch_bounds__(kThreads) residual_kernel(CgArgs a) {
  extern __shared__ float smf[];
  __shared__ float taph[232], tapl[232];
  __shared__ float outb[kTile * kTile];
  __shared__ int ctab[kTile + 2 * kMaxHalf];
  const ConvDesc& c = a.c;
  const int j = blockIdx.z;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  const int hh = c.kh / 2, hw = c.kw / 2;
  const int RH = kTile + 2 * c.hr, RW = kTile + 2 * c.hc;  // x region, halo kh - 1
  const int MH = kTile + 2 * hh, MW = kTile + 2 * hw;      // y' - H x region, halo kh / 2
  float* xh = smf;                                         // RH x RW (hi)
  float* xl = xh + RH * RW;                                // RH x RW (lo)
  float* ph = xl + RH * RW;                                // RH x MW (separable, hi)
  float* pl = ph + (c.separable ? RH * MW : 0);            // RH x MW (lo)
  float* vs = pl + (c.separable ? RH * MW : 0);            // MH x MW, y' - H x (FP32)
  float* tmpf = vs + MH * MW;                              // MH x kTile (separable)
  const int ntap = c.separable ? c.kh + c.kw : c.kh * c.kw;
  for (int i = threadIdx.x; i < ntap; i += kThreads) {
    const ff t = ff_from_double(c.hd[i]);
    taph[i] = t.hi;
    tapl[i] = t.lo;
  }
  column_table(ctab, c0 - c.hc, RW, c.W);
  __syncthreads();
  const double* x = a.X + (long long)j * c.N;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  {
    // the FP64 region, kResBatch loads in flight per thread before the first split
    constexpr int kResBatch = 8;
    const int total = RH * RW;
    for (int i0 = threadIdx.x; i0 < total; i0 += kResBatch * kThreads) {
      double xv[kResBatch];
#pragma unroll
      for (int u = 0; u < kResBatch; ++u) {
        const int i = i0 + u * kThreads;
        if (i < total) {
          const int rr = i / RW, cc = i - rr * RW;
          xv[u] = x[(long long)wrapi(r0 - c.hr + rr, c.H) * c.W + ctab[cc]];
        }
      }
#pragma unroll
      for (int u = 0; u < kResBatch; ++u) {
        const int i = i0 + u * kThreads;
        if (i < total) {
          const ff t = ff_split_bits(xv[u]);
          xh[i] = t.hi;
          xl[i] = t.lo;
        }
      }
    }
  }
  __syncthreads();
  const float* yp = j == 0 ? a.Y0 : a.Y1 + (long long)(j - 1) * c.N;
  if (c.separable && c.kh == 9 && c.kw == 9) {
    residual_sep_fixed<9>(c, taph, tapl, xh, xl, ph, pl, vs, tmpf, outb, yp, r0, c0);
  } else {
    // v = y' - H x on the (kh/2, kw/2)-halo region: (H x)(r,c) = sum k[a,b] x(r-a+hh, c-b+hw)
    if (c.separable) {
      const float* uh = taph;
      const float* ul = tapl;
      const float* vh = taph + c.kh;
      const float* vl = tapl + c.kh;
      for (int idx = threadIdx.x; idx < RH * MW; idx += kThreads) {
        const int rr = idx / MW, mc = idx - rr * MW;
        const int base = rr * RW + mc + 2 * hw;
        ff acc = {0.f, 0.f};
        for (int b = 0; b < c.kw; ++b) acc = ff_fma(acc, ff{xh[base - b], xl[base - b]}, vh[b], vl[b]);
        ph[idx] = acc.hi;
        pl[idx] = acc.lo;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < MH * MW; idx += kThreads) {
        const int mr = idx / MW, mc = idx - mr * MW;
        const int base = (mr + 2 * hh) * MW + mc;
        ff acc = {0.f, 0.f};
        for (int aa = 0; aa < c.kh; ++aa)
          acc = ff_fma(acc, ff{ph[base - aa * MW], pl[base - aa * MW]}, uh[aa], ul[aa]);
        const int gr = wrapi(r0 - hh + mr, c.H), gcol = wrapi(c0 - hw + mc, c.W);
        const ff v = ff_add(ff{yp[(long long)gr * c.W + gcol], 0.f}, ff_neg(acc));
        vs[idx] = v.hi + v.lo;
      }
    } else {
      for (int idx = threadIdx.x; idx < MH * MW; idx += kThreads) {
        const int mr = idx / MW, mc = idx - mr * MW;
        ff acc = {0.f, 0.f};
        for (int aa = 0; aa < c.kh; ++aa) {
          const int base = (mr + 2 * hh - aa) * RW + mc + 2 * hw;
          for (int b = 0; b < c.kw; ++b)
            acc = ff_fma(acc, ff{xh[base - b], xl[base - b]}, taph[aa * c.kw + b], tapl[aa * c.kw + b]);
        }
        const int gr = wrapi(r0 - hh + mr, c.H), gcol = wrapi(c0 - hw + mc, c.W);
        const ff v = ff_add(ff{yp[(long long)gr * c.W + gcol], 0.f}, ff_neg(acc));
        vs[idx] = v.hi + v.lo;
      }
    }
    __syncthreads();
    // H^T v on the tile in FP32: (H^T v)(r, c) = sum k[a, b] v(r + a - hh, c + b - hw)
    if (c.separable) {
      const float* u = taph;
      const float* v = taph + c.kh;
      for (int idx = threadIdx.x; idx < MH * kTile; idx += kThreads) {
        const int mr = idx / kTile, tc = idx - mr * kTile;
        const float* row = vs + mr * MW + tc;
        float acc = 0.f;
        for (int b = 0; b < c.kw; ++b) acc = fmaf(v[b], row[b], acc);
        tmpf[idx] = acc;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
        const int tr = idx / kTile, tc = idx - tr * kTile;
        const float* col = tmpf + tr * kTile + tc;
        float acc = 0.f;
        for (int aa = 0; aa < c.kh; ++aa) acc = fmaf(u[aa], col[aa * kTile], acc);
        outb[idx] = acc;
      }
    } else {
      for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
        const int tr = idx / kTile, tc = idx - tr * kTile;
        float acc = 0.f;
        for (int aa = 0; aa < c.kh; ++aa) {
          const float* vrow = vs + (tr + aa) * MW + tc;
          const float* krow = taph + aa * c.kw;
          for (int b = 0; b < c.kw; ++b) acc = fmaf(krow[b], vrow[b], acc);
        }
        outb[idx] = acc;
      }
    }
  }
  __syncthreads();
  float rz = 0.f, rr2 = 0.f, bb = 0.f;
  // the thread's output rows: their d, n' inputs and right-hand sides loaded first,
  // all in flight together
  constexpr int kRowsPer = kTile / (kThreads / 32);
  float dv[kRowsPer], nv[kRowsPer], ev[kRowsPer];
  const int gcol = c0 + tx;
#pragma unroll
  for (int i = 0; i < kRowsPer; ++i) {
    const int gr = r0 + ty + i * (kThreads / 32);
    dv[i] = nv[i] = ev[i] = 0.f;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    dv[i] = a.D[p];
    if (j == 0) {
      nv[i] = a.Ncav[p];
      ev[i] = a.Hty[p];
    } else {
      nv[i] = a.E2[(long long)(j - 1) * c.N + p];
      ev[i] = a.E1[(long long)(j - 1) * c.N + p];
    }
  }
#pragma unroll
  for (int i = 0; i < kRowsPer; ++i) {
    const int tr = ty + i * (kThreads / 32);
    const int gr = r0 + tr;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    const int xi_ = (tr + c.hr) * RW + tx + c.hc;
    const float d = dv[i];
    // n' - d x in float-float
    ff np;
    if (j == 0) {
      np = {nv[i], 0.f};
    } else {
      const float sd = sqrtf(d), e2 = nv[i];
      const float pr = __fmul_rn(sd, e2);
      np = {pr, fmaf(sd, e2, -pr)};
    }
    const ff t = ff_add(np, ff_neg(ff_mul_f(ff{xh[xi_], xl[xi_]}, d)));
    const float r = outb[tr * kTile + tx] * c.inv_xi + (t.hi + t.lo);
    a.Rr[(long long)j * c.N + p] = r;
    // the right-hand side b
    const float b = j == 0 ? ev[i] + nv[i] : ev[i] + sqrtf(d) * nv[i];
    if (!a.fft) rz = fmaf(r * r, a.Minv[p], rz);
    rr2 = fmaf(r, r, rr2);
    bb = fmaf(b, b, bb);
  }
  const long long o = (long long)j * a.nb + blockIdx.y * c.tiles_x + blockIdx.x;
  block_sumf<3>(rz, rr2, bb, a.fft ? nullptr : a.part_rz + o,
             a.part_rr + o, a.part_bb + o);
}

// residual_kernel for the two systems 2 blockIdx.z, 2 blockIdx.z + 1 at once with a
// separable K x K blur: every region value is a (system 0, system 1) pair, so each
// float-float tap of H x and each FP32 tap of H^T is one packed operation for both
// (ff2_fma: per lane the operations of ff_fma), and the index arithmetic, tap loads
// and the loads of d are shared.  Per system and output the taps are summed in the
// order of residual_sep_fixed, and the epilogue forms r, b and the partial sums as
// residual_kernel does.  Shared memory: the x region (hi, lo) and the row-pass output
// (hi, lo); y' - H x is written over the latter's hi half once every thread has read
// it, and the H^T row pass over its lo half.
template <int K>
__global__ void __launch_bounds__(kThreads, K >= 15 ? 2 : 3) residual_pair_kernel(CgArgs a) {
  constexpr int HR = K - 1, hh = K / 2;
  constexpr int RH = kTile + 2 * HR, RW = RH;  // x region
  constexpr int MH = kTile + 2 * hh, MW = MH;  // y' - H x region
  static_assert(K % 2 == 1 && RW % 2 == 0 && MW % 2 == 0 && MH % 2 == 0, "paired outputs");
  extern __shared__ float4 smem4[];
  float2* xh = reinterpret_cast<float2*>(smem4);  // RH x RW
  float2* xl = xh + RH * RW;
  float2* ph = xl + RH * RW;                      // RH x MW
  float2* pl = ph + RH * MW;
  float2* vs = ph;                                // MH x MW, after the column pass
  float2* tmpf = pl;                              // MH x kTile, H^T row pass
  __shared__ float2 tgh[2 * K], tgl[2 * K], tgn[2 * K];  // u taps, then v taps
  __shared__ int ctab[RW];
  const ConvDesc& c = a.c;
  const int j0 = 2 * blockIdx.z, j1 = j0 + 1;
  const bool two = j1 < a.R;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < 2 * K; i += kThreads) {
    const ff t = ff_from_double(c.hd[i]);
    tgh[i] = make_float2(t.hi, t.hi);
    tgl[i] = make_float2(t.lo, t.lo);
    tgn[i] = make_float2(-t.hi, -t.hi);
  }
  column_table(ctab, c0 - HR, RW, c.W);
  __syncthreads();
  const long long N = c.N;
  const double* x0 = a.X + (long long)j0 * N;
  const double* x1 = a.X + (long long)j1 * N;
  {
    // the FP64 regions of both systems, kB positions (2 kB loads) in flight per thread
    constexpr int kB = 4, NE = RH * RW;
    for (int i0 = threadIdx.x; i0 < NE; i0 += kB * kThreads) {
      double v0[kB], v1[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int i = i0 + u * kThreads;
        v0[u] = v1[u] = 0.0;
        if (i < NE) {
          const int rr = i / RW, cc = i - rr * RW;
          const long long p = (long long)wrapi(r0 - HR + rr, c.H) * c.W + ctab[cc];
          v0[u] = x0[p];
          if (two) v1[u] = x1[p];
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int i = i0 + u * kThreads;
        if (i < NE) {
          const ff t0 = ff_split_bits(v0[u]), t1 = ff_split_bits(v1[u]);
          xh[i] = make_float2(t0.hi, t1.hi);
          xl[i] = make_float2(t0.lo, t1.lo);
        }
      }
    }
  }
  __syncthreads();
  // H x along the rows (v taps): outputs (rr, 2 mp), (rr, 2 mp + 1) from x[rr][2 mp .. 2 mp + K]
  for (int idx = threadIdx.x; idx < RH * (MW / 2); idx += kThreads) {
    const int rr = idx / (MW / 2), mp = idx - rr * (MW / 2);
    const float4* h4 = reinterpret_cast<const float4*>(xh + rr * RW + 2 * mp);
    const float4* l4 = reinterpret_cast<const float4*>(xl + rr * RW + 2 * mp);
    float2 wh[K + 1], wl[K + 1];
#pragma unroll
    for (int q = 0; q < (K + 1) / 2; ++q) {
      const float4 th = h4[q], tl = l4[q];
      wh[2 * q] = make_float2(th.x, th.y);
      wh[2 * q + 1] = make_float2(th.z, th.w);
      wl[2 * q] = make_float2(tl.x, tl.y);
      wl[2 * q + 1] = make_float2(tl.z, tl.w);
    }
    ff2 acc0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, acc1 = acc0;
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const float2 gh = tgh[K + b], gl = tgl[K + b], gn = tgn[K + b];
      acc0 = ff2_fma(acc0, ff2{wh[K - 1 - b], wl[K - 1 - b]}, gh, gl, gn);
      acc1 = ff2_fma(acc1, ff2{wh[K - b], wl[K - b]}, gh, gl, gn);
    }
    const int o = rr * MW + 2 * mp;
    *reinterpret_cast<float4*>(ph + o) = make_float4(acc0.hi.x, acc0.hi.y, acc1.hi.x, acc1.hi.y);
    *reinterpret_cast<float4*>(pl + o) = make_float4(acc0.lo.x, acc0.lo.y, acc1.lo.x, acc1.lo.y);
  }
  __syncthreads();
  // H x along the columns (u taps) and y' - H x: outputs (mr, mc), (mr + 1, mc); the
  // results wait in registers until every thread has read the row-pass output
  const float* y0p = j0 == 0 ? a.Y0 : a.Y1 + (long long)(j0 - 1) * N;
  const float* y1p = a.Y1 + (long long)(j1 - 1) * N;
  constexpr int kColItems = ((MH / 2) * MW + kThreads - 1) / kThreads;
  float2 vout[kColItems][2];
#pragma unroll
  for (int it = 0; it < kColItems; ++it) {
    const int idx = threadIdx.x + it * kThreads;
    vout[it][0] = vout[it][1] = make_float2(0.f, 0.f);
    if (idx >= (MH / 2) * MW) continue;
    const int mp = idx / MW, mc = idx - mp * MW, mr = 2 * mp;
    const int gcol = wrapi(c0 - hh + mc, c.W);
    const long long q0 = (long long)wrapi(r0 - hh + mr, c.H) * c.W + gcol;
    const long long q1 = (long long)wrapi(r0 - hh + mr + 1, c.H) * c.W + gcol;
    const float2 ya = make_float2(y0p[q0], two ? y1p[q0] : 0.f);
    const float2 yb = make_float2(y0p[q1], two ? y1p[q1] : 0.f);
    float2 wh[K + 1], wl[K + 1];
#pragma unroll
    for (int jj = 0; jj <= K; ++jj) {
      wh[jj] = ph[(mr + jj) * MW + mc];
      wl[jj] = pl[(mr + jj) * MW + mc];
    }
    ff2 acc0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, acc1 = acc0;
#pragma unroll
    for (int aa = 0; aa < K; ++aa) {
      const float2 gh = tgh[aa], gl = tgl[aa], gn = tgn[aa];
      acc0 = ff2_fma(acc0, ff2{wh[K - 1 - aa], wl[K - 1 - aa]}, gh, gl, gn);
      acc1 = ff2_fma(acc1, ff2{wh[K - aa], wl[K - aa]}, gh, gl, gn);
    }
    const ff2 v0 = ff2_sub_from(ya, acc0), v1 = ff2_sub_from(yb, acc1);
    vout[it][0] = f2add(v0.hi, v0.lo);
    vout[it][1] = f2add(v1.hi, v1.lo);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kColItems; ++it) {
    const int idx = threadIdx.x + it * kThreads;
    if (idx >= (MH / 2) * MW) continue;
    const int mp = idx / MW, mc = idx - mp * MW, mr = 2 * mp;
    vs[mr * MW + mc] = vout[it][0];
    vs[(mr + 1) * MW + mc] = vout[it][1];
  }
  __syncthreads();
  // H^T in FP32 along the rows (v taps, hi parts): two adjacent outputs per thread
  for (int idx = threadIdx.x; idx < MH * (kTile / 2); idx += kThreads) {
    const int mr = idx / (kTile / 2), tp = idx - mr * (kTile / 2);
    const float4* r4 = reinterpret_cast<const float4*>(vs + mr * MW + 2 * tp);
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
    float4 t = r4[0];
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
      const float4 u = r4[q + 1];
      const float2 w0 = tgh[K + 2 * q], w1 = tgh[K + 2 * q + 1];
      a0 = f2fma(w0, make_float2(t.x, t.y), a0);
      a1 = f2fma(w0, make_float2(t.z, t.w), a1);
      a0 = f2fma(w1, make_float2(t.z, t.w), a0);
      a1 = f2fma(w1, make_float2(u.x, u.y), a1);
      t = u;
    }
    const float2 wlast = tgh[K + K - 1];
    a0 = f2fma(wlast, make_float2(t.x, t.y), a0);
    a1 = f2fma(wlast, make_float2(t.z, t.w), a1);
    *reinterpret_cast<float4*>(tmpf + mr * kTile + 2 * tp) = make_float4(a0.x, a0.y, a1.x, a1.y);
  }
  __syncthreads();
  // H^T along the columns (u taps): rows tr0 .. tr0 + 3 of column tx, in registers
  const int tx = threadIdx.x & 31, tr0 = (threadIdx.x >> 5) * 4;
  float2 hv[4];
  {
    float2 in0 = tmpf[tr0 * kTile + tx], in1 = tmpf[(tr0 + 1) * kTile + tx],
           in2 = tmpf[(tr0 + 2) * kTile + tx];
#pragma unroll
    for (int o = 0; o < 4; ++o) hv[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < K; ++t) {
      const float2 in3 = tmpf[(tr0 + t + 3) * kTile + tx];
      const float2 wr = tgh[t];
      hv[0] = f2fma(wr, in0, hv[0]);
      hv[1] = f2fma(wr, in1, hv[1]);
      hv[2] = f2fma(wr, in2, hv[2]);
      hv[3] = f2fma(wr, in3, hv[3]);
      in0 = in1;
      in1 = in2;
      in2 = in3;
    }
  }
  // epilogue: the inputs of all four rows loaded first
  const int gcol = c0 + tx;
  float dv[4], nv0[4], ev0[4], nv1[4], ev1[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int gr = r0 + tr0 + o;
    dv[o] = nv0[o] = ev0[o] = nv1[o] = ev1[o] = 0.f;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    dv[o] = a.D[p];
    if (j0 == 0) {
      nv0[o] = a.Ncav[p];
      ev0[o] = a.Hty[p];
    } else {
      nv0[o] = a.E2[(long long)(j0 - 1) * N + p];
      ev0[o] = a.E1[(long long)(j0 - 1) * N + p];
    }
    if (two) {
      nv1[o] = a.E2[(long long)(j1 - 1) * N + p];
      ev1[o] = a.E1[(long long)(j1 - 1) * N + p];
    }
  }
  float rz0 = 0.f, rr0 = 0.f, bb0 = 0.f, rz1 = 0.f, rr1 = 0.f, bb1 = 0.f;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int tr = tr0 + o, gr = r0 + tr;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    const int xi_ = (tr + HR) * RW + tx + HR;
    const float2 xhv = xh[xi_], xlv = xl[xi_];
    const float d = dv[o];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      const int j = u ? j1 : j0;
      const float nvu = u ? nv1[o] : nv0[o], evu = u ? ev1[o] : ev0[o];
      // n' - d x in float-float, as residual_kernel forms it
      ff np;
      if (j == 0) {
        np = {nvu, 0.f};
      } else {
        const float sd = sqrtf(d);
        const float pr = __fmul_rn(sd, nvu);
        np = {pr, fmaf(sd, nvu, -pr)};
      }
      const ff xu = u ? ff{xhv.y, xlv.y} : ff{xhv.x, xlv.x};
      const ff t = ff_add(np, ff_neg(ff_mul_f(xu, d)));
      const float r = (u ? hv[o].y : hv[o].x) * c.inv_xi + (t.hi + t.lo);
      a.Rr[(long long)j * N + p] = r;
      const float b = j == 0 ? evu + nvu : evu + sqrtf(d) * nvu;
      if (u) {
        if (!a.fft) rz1 = fmaf(r * r, a.Minv[p], rz1);
        rr1 = fmaf(r, r, rr1);
        bb1 = fmaf(b, b, bb1);
      } else {
        if (!a.fft) rz0 = fmaf(r * r, a.Minv[p], rz0);
        rr0 = fmaf(r, r, rr0);
        bb0 = fmaf(b, b, bb0);
      }
    }
  }
  const int blk = blockIdx.y * c.tiles_x + blockIdx.x;
  const long long o0 = (long long)j0 * a.nb + blk, o1 = (long long)j1 * a.nb + blk;
  block_sumf<3>(rz0, rr0, bb0, a.fft ? nullptr : a.part_rz + o0, a.part_rr + o0, a.part_bb + o0);
  if (two)
    block_sumf<3>(rz1, rr1, bb1, a.fft ? nullptr : a.part_rz + o1, a.part_rr + o1,
                  a.part_bb + o1);
}

// Per system after a true residual: done if r.r <= rtol^2 b.b (threshold +inf),
// otherwise the inner loop runs until r.r <= max(eta^2 r.r, (rtol/2)^2 b.b).
// Also starts the pass's CG scalars: active flag (and act0) = not done, beta = 0,
// and for Jacobi r.z from the residual kernel's r.Minv.r partials.
__global__ void thresholds_kernel(const double* part_rr, const double* part_bb,
                                  const double* part_rz, int fft, int R, int nb,
                                  double rtol2_mean, double rtol2_probe, double eta2, double* thr,
                                  double* relres, double* prev_rr, double* rr0, int first_arg,
                                  const int* outer_dev, int* active, float* scal, int* act0,
                                  double* rzs) {
  // the first true residual of this update (graph replays: passes started = 0)
  const int first = outer_dev ? (*outer_dev == 0) : first_arg;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < R; j += blockDim.x / 32) {
    double rr = 0, bb = 0;
    for (int i = lane; i < nb; i += 32) {
      rr += part_rr[(long long)j * nb + i];
      bb += part_bb[(long long)j * nb + i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      rr += __shfl_down_sync(0xffffffffu, rr, off);
      bb += __shfl_down_sync(0xffffffffu, bb, off);
    }
    if (lane == 0) {
      const double rtol2 = j == 0 ? rtol2_mean : rtol2_probe;
      // Converged at the target, or at the floor of the FP32 inner solver: a pass
      // that failed to halve the true residual once it is below 1e-6 relative for
      // the mean (for a well-conditioned Q the floor, about 1e-8, already means an
      // accurate x) or 1e-4 for a probe (whose RBMC sample carries far larger
      // Monte Carlo error).
      const double floor2 = j == 0 ? 1e-12 : 1e-8;
      const bool floor_hit = !first && rr <= floor2 * bb && rr > 0.25 * prev_rr[j];
      const bool done = rr <= rtol2 * bb || floor_hit;
      prev_rr[j] = rr;
      rr0[j] = rr;
      relres[j] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      thr[j] = done ? INFINITY : fmax(eta2 * rr, 0.25 * rtol2 * bb);
      scal[4 * j] = done ? 0.f : 1.f;
      scal[4 * j + 1] = 0.f;
      scal[4 * j + 2] = 0.f;   // alpha of the pending correction update
      scal[4 * j + 3] = -1.f;  // its iteration (none yet)
      act0[j] = done ? 0 : 1;
      if (!done) atomicAdd(&cnt, 1);
    }
    if (!fft) {
      double rz = 0;
      for (int i = lane; i < nb; i += 32) rz += part_rz[(long long)j * nb + i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) rz += __shfl_down_sync(0xffffffffu, rz, off);
      if (lane == 0) rzs[j] = rz;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *active = cnt;
}

// Direction and product: p = Minv r + beta p, q = Q p, partial p.q.
__global__ void __launch_bounds__(kThreads, 5) direction_kernel(CgArgs a, int it_arg) {
  extern __shared__ float smem[];
  const ConvDesc& c = a.c;
  const int j = blockIdx.z;
  const int it = a.it_dev ? *a.it_dev : it_arg;
  if (a.scal[4 * j] == 0.f) return;  // this system has converged
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(&a.counters[DC_CG_DIR_UNITS], 1ull);
  const float beta = a.scal[4 * j + 1];
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  StencilSmem sm = carve(c, smem);
  __shared__ float outb[kTile * kTile];
  stage_taps(c, sm.taps);
  const int RH = kTile + 2 * c.hr, RW = kTile + 2 * c.hc;
  const float* r = a.Rr + (long long)j * c.N;
  const float* z = a.Z + (long long)j * c.N;
  const float* Pold = ((it & 1) ? a.P : a.P2) + (long long)j * c.N;
  float* P = ((it & 1) ? a.P2 : a.P) + (long long)j * c.N;
  __shared__ int ctab[kTile + 2 * kMaxHalf];
  column_table(ctab, c0 - c.hc, RW, c.W);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // Region staging: every thread issues all of its loads (up to kRegionRows4 float4
  // rows, or kDirBatch scalars per round) before it uses the first, so a tile pays
  // about one global-memory latency instead of one per element.
  if (a.fft && (c.W & 3) == 0 && (c.hc & 3) == 0 && RW <= 64 && c0 >= c.hc &&
      c0 + kTile + c.hc <= c.W) {
    // no column wraps: float4 rows, 16 threads per region row
    constexpr int kRegionRows4 = (kTile + 2 * kMaxHalf + 15) / 16;
    const int q = threadIdx.x & 15, rb = threadIdx.x >> 4;
    if (4 * q < RW) {
      float4 zv[kRegionRows4], pv[kRegionRows4];
#pragma unroll
      for (int k = 0; k < kRegionRows4; ++k) {
        const int rr_ = rb + 16 * k;
        if (rr_ < RH) {
          const long long p = (long long)wrapi(r0 - c.hr + rr_, c.H) * c.W + c0 - c.hc + 4 * q;
          zv[k] = *reinterpret_cast<const float4*>(z + p);
          if (it > 0) pv[k] = *reinterpret_cast<const float4*>(Pold + p);
        }
      }
#pragma unroll
      for (int k = 0; k < kRegionRows4; ++k) {
        const int rr_ = rb + 16 * k;
        if (rr_ < RH) {
          float4 v = zv[k];
          if (it > 0) {
            v.x = fmaf(beta, pv[k].x, v.x);
            v.y = fmaf(beta, pv[k].y, v.y);
            v.z = fmaf(beta, pv[k].z, v.z);
            v.w = fmaf(beta, pv[k].w, v.w);
          }
          *reinterpret_cast<float4*>(sm.v + rr_ * RW + 4 * q) = v;
        }
      }
    }
  } else {
    constexpr int kDirBatch = 4;
    const int total = RH * RW;
    for (int i0 = threadIdx.x; i0 < total; i0 += kDirBatch * kThreads) {
      float v[kDirBatch], po[kDirBatch];
#pragma unroll
      for (int u = 0; u < kDirBatch; ++u) {
        const int i = i0 + u * kThreads;
        if (i < total) {
          const int rr_ = i / RW, cc = i - rr_ * RW;
          const long long p = (long long)wrapi(r0 - c.hr + rr_, c.H) * c.W + ctab[cc];
          v[u] = a.fft ? z[p] : r[p] * a.Minv[p];
          po[u] = it > 0 ? Pold[p] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < kDirBatch; ++u) {
        const int i = i0 + u * kThreads;
        if (i < total) sm.v[i] = it > 0 ? fmaf(beta, po[u], v[u]) : v[u];
      }
    }
  }
  __syncthreads();
  hth_tile(c, sm, outb);
  float pq = 0.f;
  for (int tr = ty; tr < kTile; tr += kThreads / 32) {
    const int gr = r0 + tr, gcol = c0 + tx;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    const float pv = sm.v[(tr + c.hr) * RW + tx + c.hc];
    const float q = outb[tr * kTile + tx] * c.inv_xi + a.D[p] * pv;
    P[p] = pv;
    a.Qp[(long long)j * c.N + p] = q;
    pq = fmaf(pv, q, pq);
  }
  block_sumf<1>(pq, 0.f, 0.f,
             a.part_pq + (long long)j * a.nb + blockIdx.y * c.tiles_x + blockIdx.x, nullptr,
             nullptr);
}

// direction_kernel for the two systems 2 blockIdx.z, 2 blockIdx.z + 1 at once (FFT
// preconditioner, separable H^T H with equal half-widths HR).  The region holds
// (system 0, system 1) float2 pairs, so that each tap of both stencil passes is one
// packed FP32 FMA for the two systems, and the index arithmetic, the shared-memory
// addressing and the loads of d serve both.  Row pass: two adjacent outputs per thread
// from one window read as float4; column pass: four consecutive rows of one column per
// thread, whose outputs stay in registers for the epilogue.  Per system and output
// the taps are summed in the order of hth_tile_sep.  A system that has stopped is
// neither read nor written.
template <int HR>
__global__ void __launch_bounds__(kThreads, HR >= 14 ? 3 : 5) direction_pair_kernel(CgArgs a, int it_arg) {
  constexpr int RH = kTile + 2 * HR, RW = kTile + 2 * HR, NT = 2 * HR + 1;
  extern __shared__ float4 smem4[];
  float2* reg = reinterpret_cast<float2*>(smem4);  // RH x RW region pairs
  float2* tmp = reg + RH * RW;                     // RH x kTile, after the row pass
  __shared__ float2 taps2[2 * NT];                 // (g, g): row taps, then column taps
  __shared__ int ctab[RW];
  const ConvDesc& c = a.c;
  const int j0 = 2 * blockIdx.z, j1 = j0 + 1;
  const bool act0 = a.scal[4 * j0] != 0.f, act1 = j1 < a.R && a.scal[4 * j1] != 0.f;
  if (!act0 && !act1) return;
  const int it = a.it_dev ? *a.it_dev : it_arg;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(&a.counters[DC_CG_DIR_UNITS], (unsigned long long)(act0 + act1));
  const float beta0 = a.scal[4 * j0 + 1], beta1 = act1 ? a.scal[4 * j1 + 1] : 0.f;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < 2 * NT; i += kThreads) {
    const float g = i < NT ? c.gr[i] : c.gc[i - NT];
    taps2[i] = make_float2(g, g);
  }
  column_table(ctab, c0 - HR, RW, c.W);
  const long long N = c.N;
  const long long o0 = (long long)j0 * N, o1 = (long long)j1 * N;
  const float* Pold = (it & 1) ? a.P : a.P2;
  if (a.defer_e && it > 1 && threadIdx.x < 64) {
    // the tile's rows of e, read by the pending correction update at the end: fetched
    // into L2 now, while the region is staged and the stencil runs
    const int u = threadIdx.x >> 5, gr = r0 + (threadIdx.x & 31);
    if ((u ? act1 : act0) && gr < c.H)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Ec + (u ? o1 : o0) + (long long)gr * c.W + c0));
  }
  __syncthreads();
  // Region staging, all of a thread's loads issued before the first is used
  if ((c.W & 3) == 0 && (HR & 3) == 0 && c0 >= HR && c0 + kTile + HR <= c.W) {
    // no column wraps: float4 quads of each plane
    // in rounds of KQ quads per thread, all loads of a round in flight together
    constexpr int Q4 = RW / 4, NQ = RH * Q4, KQ = 2;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i0 = threadIdx.x; i0 < NQ; i0 += KQ * kThreads) {
    float4 zv0[KQ], zv1[KQ], pv0[KQ], pv1[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const int i = i0 + k * kThreads;
      zv0[k] = zv1[k] = pv0[k] = pv1[k] = zero4;
      if (i < NQ) {
        const int rr = i / Q4, q = i - rr * Q4;
        const long long p = (long long)wrapi(r0 - HR + rr, c.H) * c.W + c0 - HR + 4 * q;
        if (act0) {
          zv0[k] = *reinterpret_cast<const float4*>(a.Z + o0 + p);
          if (it > 0) pv0[k] = *reinterpret_cast<const float4*>(Pold + o0 + p);
        }
        if (act1) {
          zv1[k] = *reinterpret_cast<const float4*>(a.Z + o1 + p);
          if (it > 0) pv1[k] = *reinterpret_cast<const float4*>(Pold + o1 + p);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const int i = i0 + k * kThreads;
      if (i < NQ) {
        const int rr = i / Q4, q = i - rr * Q4;
        float4 v0 = zv0[k], v1 = zv1[k];
        if (it > 0) {
          v0.x = fmaf(beta0, pv0[k].x, v0.x);
          v0.y = fmaf(beta0, pv0[k].y, v0.y);
          v0.z = fmaf(beta0, pv0[k].z, v0.z);
          v0.w = fmaf(beta0, pv0[k].w, v0.w);
          v1.x = fmaf(beta1, pv1[k].x, v1.x);
          v1.y = fmaf(beta1, pv1[k].y, v1.y);
          v1.z = fmaf(beta1, pv1[k].z, v1.z);
          v1.w = fmaf(beta1, pv1[k].w, v1.w);
        }
        float4* dst = reinterpret_cast<float4*>(reg + rr * RW + 4 * q);
        dst[0] = make_float4(v0.x, v1.x, v0.y, v1.y);
        dst[1] = make_float4(v0.z, v1.z, v0.w, v1.w);
      }
    }
    }
  } else {
    constexpr int kBatch = 4, NE = RH * RW;
    for (int i0 = threadIdx.x; i0 < NE; i0 += kBatch * kThreads) {
      float zs0[kBatch], zs1[kBatch], ps0[kBatch], ps1[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = i0 + u * kThreads;
        zs0[u] = zs1[u] = ps0[u] = ps1[u] = 0.f;
        if (i < NE) {
          const int rr = i / RW, cc = i - rr * RW;
          const long long p = (long long)wrapi(r0 - HR + rr, c.H) * c.W + ctab[cc];
          if (act0) {
            zs0[u] = a.Z[o0 + p];
            if (it > 0) ps0[u] = Pold[o0 + p];
          }
          if (act1) {
            zs1[u] = a.Z[o1 + p];
            if (it > 0) ps1[u] = Pold[o1 + p];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = i0 + u * kThreads;
        if (i < NE)
          reg[i] = it > 0 ? make_float2(fmaf(beta0, ps0[u], zs0[u]), fmaf(beta1, ps1[u], zs1[u]))
                          : make_float2(zs0[u], zs1[u]);
      }
    }
  }
  __syncthreads();
  // row pass (column taps along the rows)
  {
    const int cp = threadIdx.x & 15;  // column pair 2 cp, 2 cp + 1 of the tile
    for (int rr = threadIdx.x >> 4; rr < RH; rr += kThreads / 16) {
      const float4* row4 = reinterpret_cast<const float4*>(reg + rr * RW + 2 * cp);
      // window columns 2 q, 2 q + 1 arrive as one float4; tap b meets columns b, b + 1
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
      float4 t = row4[0];
#pragma unroll
      for (int q = 0; q < HR; ++q) {
        const float4 u = row4[q + 1];
        const float2 w0 = taps2[NT + 2 * q], w1 = taps2[NT + 2 * q + 1];
        a0 = __ffma2_rn(w0, make_float2(t.x, t.y), a0);
        a1 = __ffma2_rn(w0, make_float2(t.z, t.w), a1);
        a0 = __ffma2_rn(w1, make_float2(t.z, t.w), a0);
        a1 = __ffma2_rn(w1, make_float2(u.x, u.y), a1);
        t = u;
      }
      const float2 wl = taps2[NT + 2 * HR];
      a0 = __ffma2_rn(wl, make_float2(t.x, t.y), a0);
      a1 = __ffma2_rn(wl, make_float2(t.z, t.w), a1);
      *reinterpret_cast<float4*>(tmp + rr * kTile + 2 * cp) = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
  }
  __syncthreads();
  // column pass: rows tr0 .. tr0 + 3 of column tx
  const int tx = threadIdx.x & 31, tr0 = (threadIdx.x >> 5) * 4;
  float2 acc[4];
  {
    // a sliding window of four inputs: tap t meets rows tr0 + t .. tr0 + t + 3
    float2 in0 = tmp[tr0 * kTile + tx], in1 = tmp[(tr0 + 1) * kTile + tx],
           in2 = tmp[(tr0 + 2) * kTile + tx];
#pragma unroll
    for (int o = 0; o < 4; ++o) acc[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float2 in3 = tmp[(tr0 + t + 3) * kTile + tx];
      const float2 wr = taps2[t];
      acc[0] = __ffma2_rn(wr, in0, acc[0]);
      acc[1] = __ffma2_rn(wr, in1, acc[1]);
      acc[2] = __ffma2_rn(wr, in2, acc[2]);
      acc[3] = __ffma2_rn(wr, in3, acc[3]);
      in0 = in1;
      in1 = in2;
      in2 = in3;
    }
  }
  float* P = (it & 1) ? a.P2 : a.P;
  float pq0 = 0.f, pq1 = 0.f;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int tr = tr0 + o, gr = r0 + tr, gcol = c0 + tx;
    if (gr >= c.H || gcol >= c.W) continue;
    const long long p = (long long)gr * c.W + gcol;
    const float2 pv = reg[(tr + HR) * RW + tx + HR];
    const float d = a.D[p];
    if (act0) {
      const float q = acc[o].x * c.inv_xi + d * pv.x;
      P[o0 + p] = pv.x;
      a.Qp[o0 + p] = q;
      pq0 = fmaf(pv.x, q, pq0);
    }
    if (act1) {
      const float q = acc[o].y * c.inv_xi + d * pv.y;
      P[o1 + p] = pv.y;
      a.Qp[o1 + p] = q;
      pq1 = fmaf(pv.y, q, pq1);
    }
  }
  const int blk = blockIdx.y * c.tiles_x + blockIdx.x;
  block_sumf<2>(pq0, pq1, 0.f, act0 ? a.part_pq + (long long)j0 * a.nb + blk : nullptr,
                act1 ? a.part_pq + (long long)j1 * a.nb + blk : nullptr, nullptr);
  if (a.defer_e && it > 0) {
    // the previous iteration's correction update on this tile, e += alpha p with that
    // iteration's alpha and direction (the update kernel left it; a system active now
    // was active then)
    const float al0 = a.scal[4 * j0 + 2], al1 = act1 ? a.scal[4 * j1 + 2] : 0.f;
    const bool e_zero = it == 1;  // the correction starts at zero: not read
    const int gr = r0 + (threadIdx.x >> 3), gc0 = c0 + (threadIdx.x & 7) * 4;
    if (gr < c.H) {
      const long long p = (long long)gr * c.W + gc0;
      if ((c.W & 3) == 0 && gc0 + 4 <= c.W) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (!(u ? act1 : act0)) continue;
          const long long q = (u ? o1 : o0) + p;
          const float al = u ? al1 : al0;
          const float4 pv = *reinterpret_cast<const float4*>(Pold + q);
          float4 ev = e_zero ? make_float4(0.f, 0.f, 0.f, 0.f)
                             : *reinterpret_cast<const float4*>(a.Ec + q);
          ev.x = fmaf(al, pv.x, ev.x);
          ev.y = fmaf(al, pv.y, ev.y);
          ev.z = fmaf(al, pv.z, ev.z);
          ev.w = fmaf(al, pv.w, ev.w);
          *reinterpret_cast<float4*>(a.Ec + q) = ev;
        }
      } else {
        for (int t = 0; t < 4 && gc0 + t < c.W; ++t) {
          if (act0) a.Ec[o0 + p + t] = fmaf(al0, Pold[o0 + p + t], e_zero ? 0.f : a.Ec[o0 + p + t]);
          if (act1) a.Ec[o1 + p + t] = fmaf(al1, Pold[o1 + p + t], e_zero ? 0.f : a.Ec[o1 + p + t]);
        }
      }
    }
  }
}

// e += alpha p, r -= alpha q (e: the FP32 correction of this refinement pass,
// added to the FP64 solution by commit_kernel when the pass ends), partials of
// the new r.r (and r.Minv.r for Jacobi).  alpha = r.z / p.q: every block sums the
// direction kernel's p.q partials of its system itself, in the same order, while
// its tile loads are in flight.  The last block of a system then sets its active
// flag for the next iteration (and, for Jacobi, beta and r.z).
// 64 threads per 32 x 32 tile: four rows of float4 per thread keep more loads in
// flight and make the block reduction a smaller share of the work.
constexpr int kUpdThreads = 64;
constexpr int kUpdRows = kTile * kTile / 4 / kUpdThreads;

__global__ void __launch_bounds__(kUpdThreads) update_kernel(CgArgs a, int it_arg) {
  const ConvDesc& c = a.c;
  const int j = blockIdx.z;
  const int it = a.it_dev ? *a.it_dev : it_arg;
  if (a.scal[4 * j] == 0.f) return;  // this system has stopped
  const int blk = blockIdx.y * c.tiles_x + blockIdx.x;
  if (blk == 0 && threadIdx.x == 0) atomicAdd(&a.counters[DC_CG_UPD_UNITS], 1ull);
  __shared__ float alpha_s;
  auto form_alpha = [&]() {
    if (threadIdx.x < 32) {
      const double pqs = group_sum(a.part_pq + (long long)j * a.nb, a.nb);
      if (threadIdx.x == 0) alpha_s = (float)(a.rzs[j] / pqs);
    }
    __syncthreads();
    return alpha_s;
  };
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  float* Ec = a.Ec + (long long)j * c.N;
  float* Rr = a.Rr + (long long)j * c.N;
  const float* P = ((it & 1) ? a.P2 : a.P) + (long long)j * c.N;
  const float* Q = a.Qp + (long long)j * c.N;
  const bool first = it == 0;  // the correction starts at zero: not read
  float rz2 = 0.f, rr2 = 0.f;
  if ((c.W & 3) == 0 && c0 + kTile <= c.W && r0 + kTile <= c.H) {
    // full tile, rows 16-byte aligned: kUpdRows float4 of each plane per thread,
    // all loads issued before the first store
    const int c4 = (threadIdx.x & 7) * 4;
    float4 pv[kUpdRows], qv[kUpdRows], rv[kUpdRows], ev[kUpdRows], mv[kUpdRows];
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int tr = (threadIdx.x >> 3) + k * (kUpdThreads >> 3);
      const long long p = (long long)(r0 + tr) * c.W + c0 + c4;
      pv[k] = *reinterpret_cast<const float4*>(P + p);
      qv[k] = *reinterpret_cast<const float4*>(Q + p);
      rv[k] = *reinterpret_cast<const float4*>(Rr + p);
      ev[k] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(Ec + p);
      if (!a.fft) mv[k] = *reinterpret_cast<const float4*>(a.Minv + p);
    }
    const float alpha = form_alpha();
#pragma unroll
    for (int k = 0; k < kUpdRows; ++k) {
      const int tr = (threadIdx.x >> 3) + k * (kUpdThreads >> 3);
      const long long p = (long long)(r0 + tr) * c.W + c0 + c4;
      float4 e = ev[k], r = rv[k];
      e.x = fmaf(alpha, pv[k].x, e.x);
      e.y = fmaf(alpha, pv[k].y, e.y);
      e.z = fmaf(alpha, pv[k].z, e.z);
      e.w = fmaf(alpha, pv[k].w, e.w);
      r.x = fmaf(-alpha, qv[k].x, r.x);
      r.y = fmaf(-alpha, qv[k].y, r.y);
      r.z = fmaf(-alpha, qv[k].z, r.z);
      r.w = fmaf(-alpha, qv[k].w, r.w);
      *reinterpret_cast<float4*>(Ec + p) = e;
      *reinterpret_cast<float4*>(Rr + p) = r;
      rr2 += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
      if (!a.fft)
        rz2 += r.x * r.x * mv[k].x + r.y * r.y * mv[k].y + r.z * r.z * mv[k].z + r.w * r.w * mv[k].w;
    }
  } else {
    const float alpha = form_alpha();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int tr = ty; tr < kTile; tr += kUpdThreads / 32) {
      const int gr = r0 + tr, gcol = c0 + tx;
      if (gr >= c.H || gcol >= c.W) continue;
      const long long p = (long long)gr * c.W + gcol;
      Ec[p] = fmaf(alpha, P[p], first ? 0.f : Ec[p]);
      const float r = fmaf(-alpha, Q[p], Rr[p]);
      Rr[p] = r;
      if (!a.fft) rz2 = fmaf(r * r, a.Minv[p], rz2);
      rr2 = fmaf(r, r, rr2);
    }
  }
  block_sumf<2>(rz2, rr2, 0.f, a.fft ? nullptr : a.part_rz + (long long)j * a.nbz + blk,
             a.part_rr + (long long)j * a.nb + blk, nullptr);
  if (arrive_last(a.arrive + j, (unsigned)a.nb) && threadIdx.x < 32) {
    const double rr = group_sum(a.part_rr + (long long)j * a.nb, a.nb);
    const double rzn = a.fft ? 0.0 : group_sum(a.part_rz + (long long)j * a.nbz, a.nbz);
    if (threadIdx.x == 0) {
      // stop at the pass target, or when the recurrence residual has grown
      // fourfold over the pass (FP32 CG losing its way on a badly conditioned
      // system): the next pass restarts from the true residual
      a.scal[4 * j] = (rr <= a.thr[j] || rr > 16.0 * a.rr0[j]) ? 0.f : 1.f;
      if (!a.fft) {
        a.scal[4 * j + 1] = (float)(rzn / a.rzs[j]);
        a.rzs[j] = rzn;
      }
    }
  }
}

// x += e for every system that iterated in the pass that just ended.
// With deferred correction updates (CgArgs::defer_e) the last iteration's e += alpha p
// of each system is still pending (scal[4 j + 2] = alpha, scal[4 j + 3] = its
// iteration, whose direction is in P or P2 by parity; e is not read if it was the
// first): it is formed here, with the operation the update kernel would have used.
__global__ void commit_kernel(double* X, const float* Ec, const int* act0, long long N,
                              const float* scal, const float* P, const float* P2) {
  const int j = blockIdx.y;
  if (!act0[j]) return;
  double* x = X + (long long)j * N;
  const float* e = Ec + (long long)j * N;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  stride = (long long)gridDim.x * blockDim.x;
  const float kp = scal ? scal[4 * j + 3] : -1.f;
  const bool pend = kp >= 0.f;
  const int k = pend ? (int)kp : 1;
  const float al = pend ? scal[4 * j + 2] : 0.f;
  const float* pk = ((k & 1) ? P2 : P) + (long long)j * N;
  if ((N & 3) == 0) {
    // four pixels per step: one float4 of e, two double2 of x (planes 32-byte aligned)
    for (long long q = t0; q < N / 4; q += stride) {
      float4 ev = k > 0 ? reinterpret_cast<const float4*>(e)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (pend) {
        const float4 pv = reinterpret_cast<const float4*>(pk)[q];
        ev.x = fmaf(al, pv.x, ev.x);
        ev.y = fmaf(al, pv.y, ev.y);
        ev.z = fmaf(al, pv.z, ev.z);
        ev.w = fmaf(al, pv.w, ev.w);
      }
      double2* x2 = reinterpret_cast<double2*>(x) + 2 * q;
      double2 a = x2[0], b = x2[1];
      a.x += (double)ev.x;
      a.y += (double)ev.y;
      b.x += (double)ev.z;
      b.y += (double)ev.w;
      x2[0] = a;
      x2[1] = b;
    }
    return;
  }
  for (long long p = t0; p < N; p += stride)
    x[p] += (double)(pend ? fmaf(al, pk[p], k > 0 ? e[p] : 0.f) : e[p]);
}


// Device-side state of the solver loops of a graph replay.
struct LoopState {
  int it;         // CG iteration within the current pass
  int outer;      // passes started
  int total;      // CG iterations of this update
  int converged;  // 1 once a true residual met every system's target
};

// ---------------------------------------------------------------------------
// Circulant preconditioner for power-of-two H and W:
//   M = H^T H / xi + dbar I,  dbar = mean(d),  M^{-1} r = F^{-1}[F r / (|h_f|^2 / xi + dbar)].
// H^T H is circulant, so M differs from Q only by d - dbar on the diagonal; CG
// on M^{-1} Q needs a few tens of iterations where Jacobi needs hundreds.
// Two real systems share one complex transform (z = r_a + i r_b): the filter is
// real and even in frequency, so the real and imaginary parts of the result are
// M^{-1} r_a and M^{-1} r_b.  Rows, then columns (forward, filter, inverse in one
// pass), then rows again; 512-point transforms are register-resident (one warp per
// row or column), other sizes run Stockham passes in shared memory.
struct FftDesc {
  int H, W;          // image
  int HP, WP;        // power-of-two transform sizes, HP >= H, WP >= W
  int R, pairs;
  int cw;            // columns per block in the column pass
  int rpb;           // rows per block in the row passes
  int nbz;           // blocks per pair in the inverse row pass
  float2* tmp;       // pairs x H x WP (rows of the padded grid beyond H are zero)
  const float* hth;  // |h_f|^2 / xi on the HP x WP grid
  const double* dbar;
  const float2* tw512;  // exp(-2 pi i m / 512), m < 512 (the 512-point kernels)
  const float2* tw1024; // exp(-2 pi i m / 1024), m < 512 (the 1024-point kernels)
  const float* act;  // CG scalars of the current iteration ([4 R], [4 j] = 1 if system j
                     // is active), or NULL: transform every system
  float* scal_w;     // the same array, written: beta of the active systems
  double* rzs;       // [R] r.z, or NULL: leave the CG scalars alone (shape tuning)
  unsigned* arrive;  // [pairs] block-arrival counters of the inverse row pass
  int first;         // 1: first application of a refinement pass (beta = 0)
  unsigned long long* counters;  // DC_CG_PRE_UNITS counts the systems transformed
  LoopState* loop;   // graph replays: the column pass also counts the CG iteration and
                     // sets the inner loop's condition (loop_step), else NULL
  cudaGraphConditionalHandle h_inner;
  int max_iter;
};

// The last block of a pair's inverse row pass sums the r.z partials of its two
// systems and sets, for each system still active, beta = r.z(new) / r.z(old)
// (0 in the first application of a refinement pass) and r.z = r.z(new).
__device__ __forceinline__ void rz_tail(const FftDesc& f, int pair, const double* part_rz) {
  if (!f.rzs) return;
  if (!arrive_last(f.arrive + pair, gridDim.x) || threadIdx.x >= 32) return;
  for (int u = 0; u < 2; ++u) {
    const int j = 2 * pair + u;
    if (j >= f.R) break;
    const double rz = group_sum(part_rz + (long long)j * f.nbz, f.nbz);
    if (threadIdx.x == 0 && f.act[4 * j] != 0.f) {
      f.scal_w[4 * j + 1] = f.first ? 0.f : (float)(rz / f.rzs[j]);
      f.rzs[j] = rz;
    }
  }
}

// Both systems of a pair have stopped in this CG iteration: their z is not used.
__device__ __forceinline__ bool pair_idle(const FftDesc& f, int pair) {
  if (!f.act) return false;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  return f.act[4 * j0] == 0.f && (j1 >= f.R || f.act[4 * j1] == 0.f);
}

// After a CG iteration's update (graph replays, by block (0, 0) of the column pass,
// which every iteration launches): count the iteration, and go on while a system is
// still active and the iteration budget lasts, as iter_kernel does.
__device__ __forceinline__ void loop_step(const FftDesc& f) {
  if (!f.loop || blockIdx.x != 0 || blockIdx.y != 0 || threadIdx.x >= 32) return;
  int cnt = 0;
  for (int j = threadIdx.x; j < f.R; j += 32) cnt += f.act[4 * j] != 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  if (threadIdx.x == 0) {
    f.loop->it += 1;
    f.loop->total += 1;
    cudaGraphSetConditional(f.h_inner, (cnt > 0 && f.loop->total < f.max_iter) ? 1u : 0u);
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// In-register forward DFTs of length 2, 4 and 8 (output in natural order).
template <int R> __device__ __forceinline__ void dft_reg(float2* v);
template <> __device__ __forceinline__ void dft_reg<2>(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <> __device__ __forceinline__ void dft_reg<4>(float2* v) {
  const float2 a0 = cadd(v[0], v[2]), a2 = csub(v[0], v[2]);
  const float2 a1 = cadd(v[1], v[3]), a3 = cmul_mi(csub(v[1], v[3]));
  v[0] = cadd(a0, a1);
  v[1] = cadd(a2, a3);
  v[2] = csub(a0, a1);
  v[3] = csub(a2, a3);
}
template <> __device__ __forceinline__ void dft_reg<8>(float2* v) {
  const float s2 = 0.70710678118654752440f;
  const float2 a0 = cadd(v[0], v[4]), a1 = cadd(v[1], v[5]), a2 = cadd(v[2], v[6]),
               a3 = cadd(v[3], v[7]);
  const float2 d4 = csub(v[0], v[4]), d5 = csub(v[1], v[5]), d6 = csub(v[2], v[6]),
               d7 = csub(v[3], v[7]);
  // twiddles exp(-2 pi i m / 8) for m = 1, 2, 3
  const float2 a5 = make_float2(s2 * (d5.x + d5.y), s2 * (d5.y - d5.x));
  const float2 a6 = cmul_mi(d6);
  const float2 a7 = make_float2(s2 * (d7.y - d7.x), -s2 * (d7.x + d7.y));
  const float2 b0 = cadd(a0, a2), b1 = cadd(a1, a3), b2 = csub(a0, a2), b3 = cmul_mi(csub(a1, a3));
  const float2 b4 = cadd(d4, a6), b5 = cadd(a5, a7), b6 = csub(d4, a6), b7 = cmul_mi(csub(a5, a7));
  v[0] = cadd(b0, b1);
  v[4] = csub(b0, b1);
  v[2] = cadd(b2, b3);
  v[6] = csub(b2, b3);
  v[1] = cadd(b4, b5);
  v[5] = csub(b4, b5);
  v[3] = cadd(b6, b7);
  v[7] = csub(b6, b7);
}

constexpr int kFftMaxItems = 2;  // work items per thread in one pass
constexpr int kFftThreads = 256; // threads per FFT block (four resident blocks per SM)

// One Stockham autosort pass of radix R: `count` transforms of length n, element i
// of transform t at s[t * tstride + i * stride]; Ns = product of earlier radices.
// Item j reads x[j + r n/R], multiplies by exp(-2 pi i r k / (Ns R)), k = j mod Ns,
// applies the length-R DFT and writes y[(j - k) R + k + q Ns].  In place: every
// item is read into registers before the barrier, written after it.
template <int R>
__device__ __forceinline__ void stockham_pass(float2* s, int n, int count, int stride, int tstride,
                                              int Ns, const float2* tw) {
  const int nq = n / R;
  const int items = nq * count;
  const int twstep = n / (Ns * R);
  float2 v[kFftMaxItems][R];
#pragma unroll
  for (int it = 0; it < kFftMaxItems; ++it) {
    const int w = threadIdx.x + it * blockDim.x;
    if (w < items) {
      int t, j;
      if (tstride == 1) { j = w / count; t = w - j * count; } else { t = w / nq; j = w - t * nq; }
      const int k = j & (Ns - 1);
      const float2* base = s + t * tstride;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 x = base[(j + r * nq) * stride];
        v[it][r] = r ? cmul(x, tw[(k * r * twstep) & (n - 1)]) : x;
      }
      dft_reg<R>(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kFftMaxItems; ++it) {
    const int w = threadIdx.x + it * blockDim.x;
    if (w < items) {
      int t, j;
      if (tstride == 1) { j = w / count; t = w - j * count; } else { t = w / nq; j = w - t * nq; }
      const int k = j & (Ns - 1);
      float2* base = s + t * tstride;
      const int ob = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) base[(ob + q * Ns) * stride] = v[it][q];
    }
  }
  __syncthreads();
}

// Forward transform (exp(-)) in natural order, radix 8 first, then one 4 or 2.
__device__ void fft_forward(float2* s, int n, int count, int stride, int tstride, const float2* tw) {
  for (int Ns = 1; Ns < n;) {
    const int rem = n / Ns;
    if (rem >= 8) {
      stockham_pass<8>(s, n, count, stride, tstride, Ns, tw);
      Ns *= 8;
    } else if (rem == 4) {
      stockham_pass<4>(s, n, count, stride, tstride, Ns, tw);
      Ns *= 4;
    } else {
      stockham_pass<2>(s, n, count, stride, tstride, Ns, tw);
      Ns *= 2;
    }
  }
}

// tw[m] = exp(-2 pi i m / n), m < n
__device__ __forceinline__ void make_table(float2* tw, int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    float sn, cs;
    sincospif(-2.0f * (float)m / (float)n, &sn, &cs);
    tw[m] = make_float2(cs, sn);
  }
}

// s[idx] = get(idx) for idx < total, four loads in flight per thread before the
// stores to shared memory.
template <typename Get>
__device__ __forceinline__ void stage_loads(float2* s, int total, Get get) {
  for (int base = 0; base < total; base += 4 * kFftThreads) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * kFftThreads + threadIdx.x;
      v[u] = idx < total ? get(idx) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * kFftThreads + threadIdx.x;
      if (idx < total) s[idx] = v[u];
    }
  }
}

// Pack two residual planes into complex rows (zero-padded to WP) and transform them.
__global__ void __launch_bounds__(kFftThreads, 4) fft_rows_fwd_kernel(FftDesc f, const float* __restrict__ Rr) {
  if (pair_idle(f, blockIdx.y)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters)
    atomicAdd(&f.counters[DC_CG_PRE_UNITS], 2 * blockIdx.y + 1 < f.R ? 2ull : 1ull);
  extern __shared__ float2 sm2[];
  float2* tw = sm2;
  float2* s = sm2 + f.WP;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const long long N = (long long)f.H * f.W;
  const int row0 = blockIdx.x * f.rpb;
  make_table(tw, f.WP);
  const float* r0p = Rr + (long long)j0 * N;
  const float* r1p = Rr + (long long)j1 * N;
  const bool two = j1 < f.R;
  stage_loads(s, f.rpb * f.WP, [&](int idx) {
    const int rr = idx / f.WP, cc = idx - rr * f.WP;
    const int row = row0 + rr;
    float2 v = make_float2(0.f, 0.f);
    if (row < f.H && cc < f.W) {
      const long long p = (long long)row * f.W + cc;
      v = make_float2(r0p[p], two ? r1p[p] : 0.f);
    }
    return v;
  });
  __syncthreads();
  fft_forward(s, f.WP, f.rpb, 1, f.WP, tw);
  float2* out = f.tmp + (long long)pair * f.H * f.WP;
  for (int rr = 0; rr < f.rpb; ++rr) {
    const int row = row0 + rr;
    if (row >= f.H) break;
    for (int cc = threadIdx.x; cc < f.WP; cc += blockDim.x)
      out[(long long)row * f.WP + cc] = s[rr * f.WP + cc];
  }
}

// Column transforms (rows beyond H are zero), the preconditioner filter and the
// inverse column transforms; only rows below H are kept.
__global__ void __launch_bounds__(kFftThreads, 4) fft_cols_filter_kernel(FftDesc f) {
  loop_step(f);
  if (pair_idle(f, blockIdx.y)) return;
  extern __shared__ float2 sm2[];
  float2* tw = sm2;
  float2* s = sm2 + f.HP;
  const int pair = blockIdx.y;
  const int c0 = blockIdx.x * f.cw;
  float2* t = f.tmp + (long long)pair * f.H * f.WP;
  make_table(tw, f.HP);
  stage_loads(s, f.HP * f.cw, [&](int idx) {
    const int i = idx / f.cw, c = idx - i * f.cw;
    return i < f.H ? t[(long long)i * f.WP + c0 + c] : make_float2(0.f, 0.f);
  });
  __syncthreads();
  fft_forward(s, f.HP, f.cw, f.cw, 1, tw);
  // filter, then the inverse column transform as conj(F(conj(.)))
  const float dbar = (float)(*f.dbar);
  for (int idx = threadIdx.x; idx < f.HP * f.cw; idx += blockDim.x) {
    const int i = idx / f.cw, c = idx - i * f.cw;
    const float g = __frcp_rn(f.hth[(long long)i * f.WP + c0 + c] + dbar);
    s[idx] = make_float2(s[idx].x * g, -s[idx].y * g);
  }
  __syncthreads();
  fft_forward(s, f.HP, f.cw, f.cw, 1, tw);
  for (int idx = threadIdx.x; idx < f.H * f.cw; idx += blockDim.x) {
    const int i = idx / f.cw, c = idx - i * f.cw;
    t[(long long)i * f.WP + c0 + c] = cconj(s[idx]);
  }
}

// Inverse row transforms, scale 1/(HP WP), crop to W, unpack into z planes,
// partial r.z per system.
__global__ void __launch_bounds__(kFftThreads, 4) fft_rows_inv_kernel(FftDesc f, const float* __restrict__ Rr,
                                                                      float* Z, double* part_rz) {
  if (pair_idle(f, blockIdx.y)) return;
  extern __shared__ float2 sm2[];
  float2* tw = sm2;
  float2* s = sm2 + f.WP;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const long long N = (long long)f.H * f.W;
  const float scale = 1.0f / ((float)f.HP * (float)f.WP);
  const int rows_per = (f.H + f.nbz - 1) / f.nbz;
  const int rbeg = blockIdx.x * rows_per, rend = min(f.H, rbeg + rows_per);
  make_table(tw, f.WP);
  double acc0 = 0.0, acc1 = 0.0;
  const float2* tin = f.tmp + (long long)pair * f.H * f.WP;
  for (int r0 = rbeg; r0 < rend; r0 += f.rpb) {
    __syncthreads();
    stage_loads(s, f.rpb * f.WP, [&](int idx) {
      const int rr = idx / f.WP, cc = idx - rr * f.WP;
      const int row = r0 + rr;
      return row < rend ? cconj(tin[(long long)row * f.WP + cc]) : make_float2(0.f, 0.f);
    });
    __syncthreads();
    fft_forward(s, f.WP, f.rpb, 1, f.WP, tw);
    float rz0 = 0.f, rz1 = 0.f;
    for (int rr = 0; rr < f.rpb; ++rr) {
      const int row = r0 + rr;
      if (row >= rend) break;
      for (int cc = threadIdx.x; cc < f.W; cc += blockDim.x) {
        const float2 v = cconj(s[rr * f.WP + cc]);
        const long long p = (long long)row * f.W + cc;
        const float z0 = v.x * scale;
        Z[(long long)j0 * N + p] = z0;
        rz0 = fmaf(Rr[(long long)j0 * N + p], z0, rz0);
        if (j1 < f.R) {
          const float z1 = v.y * scale;
          Z[(long long)j1 * N + p] = z1;
          rz1 = fmaf(Rr[(long long)j1 * N + p], z1, rz1);
        }
      }
    }
    acc0 += (double)rz0;
    acc1 += (double)rz1;
  }
  __syncthreads();
  block_sum3(acc0, acc1, 0.0, part_rz + (long long)j0 * f.nbz + blockIdx.x,
             j1 < f.R ? part_rz + (long long)j1 * f.nbz + blockIdx.x : nullptr, nullptr);
  rz_tail(f, pair, part_rz);
}

// ---- register-resident 512-point transforms
//
// When a transform length is 512 each transform is held by one warp: lane l
// keeps x[32 m + l], m = 0..15, and the transform runs as three radix-8 steps,
// 512 = 8 x 8 x 8, with the index splits n = 64 r + t, t = 8 s + u and
// k = k1 + 8 k3 + 64 k4 (w_n = exp(-2 pi i / n)):
//   B_t[k1]              = w512^(t k1) sum_r x[64 r + t] w8^(r k1)
//   C_u[k1, k3]          = w64^(u k3)  sum_s B_(8 s + u)[k1] w8^(s k3)
//   X[k1 + 8 k3 + 64 k4] = sum_u C_u[k1, k3] w8^(u k4)
// The two regroupings pass through a per-warp scratch of kXs float2 in shared
// memory, padded so that the accesses of a half-warp fall in distinct banks;
// the output X[32 m + l] lands in lane l, the layout of the input, so a forward
// transform, a pointwise filter and another transform chain in registers.
constexpr int kF = 512;
constexpr int kXs = 578;        // scratch / staged-column pitch in float2
constexpr int kF512Warps = 8;   // warps per block of the 512-point kernels
// Rows per warp of the 512-point row passes, one after another; each row's loads
// are all issued before the transform starts (prefetching the next row during the
// transform measured slower: it raises register pressure at the 128-register limit).
constexpr int kRowsPerWarp512 = 4;

// tw[m] = w512^m and tw[512 + m] = w1024^m for m < 512
__global__ void tw512_kernel(float2* tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 2 * kF) {
    float sn, cs;
    if (m < kF)
      sincospif(-2.0f * (float)m / (float)kF, &sn, &cs);
    else
      sincospif(-2.0f * (float)(m - kF) / (float)(2 * kF), &sn, &cs);
    tw[m] = make_float2(cs, sn);
  }
}

// L2 eviction priorities for the preconditioner's planes: the complex plane of
// each system pair and the residual read by both row passes are kept (evict
// last) from their first touch to their last read, which releases them (evict
// first); the streamed CG planes of the other kernels then go first.  The kept
// footprint, one complex plane per pair plus the residuals, is about 70 MB at
// 512^2 with 33 systems, inside the 129 MB L2.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_release() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float2 ld_hint(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_hint(const float* a, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint4(float2* a, float2 u, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(u.x),
               "f"(u.y), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_hint_f(float* a, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}

// Which passes take the 512-point kernels (the others take the Stockham ones).
inline bool fft512_rows(const FftDesc& f) { return f.WP == kF; }
inline bool fft512_cols(const FftDesc& f) { return f.HP == kF && f.WP >= kF512Warps; }
// and the 1024-point ones (below)
inline bool fft1024_rows(const FftDesc& f) { return f.WP == 2 * kF; }
inline bool fft1024_cols(const FftDesc& f) { return f.HP == 2 * kF && f.WP >= kF512Warps; }

__device__ __forceinline__ void fft512_warp(float2 (&v)[16], float2* xs, const float2* tw) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = l + 32 * h;
    float2 a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = v[2 * r + h];
    dft_reg<8>(a);
    xs[t * 9] = a[0];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) xs[t * 9 + k1] = cmul(a[k1], tw[(t * k1) & (kF - 1)]);
  }
  __syncwarp();
  const int k1 = l & 7;
  float2 b[2][8];
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int u = (l >> 3) + 4 * g;
#pragma unroll
    for (int s = 0; s < 8; ++s) b[g][s] = xs[(8 * s + u) * 9 + k1];
  }
  __syncwarp();
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int u = (l >> 3) + 4 * g;
    dft_reg<8>(b[g]);
    xs[u * 72 + k1] = b[g][0];
#pragma unroll
    for (int k3 = 1; k3 < 8; ++k3)
      xs[u * 72 + k1 + 8 * k3] = cmul(b[g][k3], tw[(8 * u * k3) & (kF - 1)]);
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = l + 32 * h;  // j = k1 + 8 k3
    float2 c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = xs[u * 72 + j];
    dft_reg<8>(c);
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4) v[2 * k4 + h] = c[k4];
  }
  __syncwarp();  // the scratch is free again
}

// fft_rows_fwd_kernel for WP = 512: one warp per row, rows [blockIdx.x rpb, +rpb).
__global__ void __launch_bounds__(32 * kF512Warps) fft512_rows_fwd_kernel(FftDesc f,
                                                                         const float* __restrict__ Rr,
                                                                         int rpb) {
  if (pair_idle(f, blockIdx.y)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters)
    atomicAdd(&f.counters[DC_CG_PRE_UNITS], 2 * blockIdx.y + 1 < f.R ? 2ull : 1ull);
  __shared__ float2 tw[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) tw[m] = f.tw512[m];
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const long long N = (long long)f.H * f.W;
  const float* r0p = Rr + (long long)j0 * N;
  const float* r1p = Rr + (long long)j1 * N;
  float2* out = f.tmp + (long long)pair * f.H * kF;
  const int rend = min(f.H, (blockIdx.x + 1) * rpb);
  const uint64_t keep = l2_policy_keep();
  float2 nx[16];  // the row, all loads in flight together
  auto load_row = [&](int rw) {
    const long long p0 = (long long)rw * f.W;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int c = 32 * m + l;
      nx[m] = make_float2(0.f, 0.f);
      if (c < f.W) nx[m] = make_float2(ld_hint(r0p + p0 + c, keep), two ? ld_hint(r1p + p0 + c, keep) : 0.f);
    }
  };
  for (int row = blockIdx.x * rpb + w; row < rend; row += kF512Warps) {
    load_row(row);
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = nx[m];
    fft512_warp(v, scratch[w], tw);
#pragma unroll
    for (int m = 0; m < 16; ++m) st_hint(out + (long long)row * kF + 32 * m + l, v[m], keep);
  }
}

// The CG update fused with the forward row pass (512-point rows): for each system
// of the pair that is active when the iteration starts, alpha = r.z / p.q from the
// direction kernel's partials, e += alpha p and r -= alpha q, exactly as update_kernel
// forms them; the new residual rows of the pair then go through the forward row
// transform without being read again.  A system that stopped earlier enters the
// transform as zero (its z is not used before the next pass recomputes it).  The last
// block of the pair sums its r.r partials in block order and sets the active flags,
// as update_kernel's last block does, so the column and inverse passes that follow
// skip the pairs that stopped here.  With a.defer_e (the paired direction kernel) only
// r is updated here: alpha and the iteration go to the CG scalars, and e += alpha p is
// done by the next direction kernel over its tile, where p is the direction it reads
// anyway, or by the commit after a system's last iteration; the same operation on the
// same values, so the results do not change.
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft512_update_rows_fwd_kernel(FftDesc f,
                                                                                CgArgs a,
                                                                                int it_arg,
                                                                                int rpb) {
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const bool act0 = a.scal[4 * j0] != 0.f, act1 = two && a.scal[4 * j1] != 0.f;
  if (!act0 && !act1) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters) {
    atomicAdd(&f.counters[DC_CG_PRE_UNITS], two ? 2ull : 1ull);
    atomicAdd(&f.counters[DC_CG_UPD_UNITS], (unsigned long long)(act0 + act1));
  }
  const int it = a.it_dev ? *a.it_dev : it_arg;
  const bool first = it == 0;  // the correction starts at zero: not read
  __shared__ float2 tw[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  __shared__ float alpha_s[2];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) tw[m] = f.tw512[m];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w < 2 && (w == 0 ? act0 : act1)) {
    const int j = j0 + w;
    const double pqs = group_sum(a.part_pq + (long long)j * a.nb, a.nb);
    if (l == 0) alpha_s[w] = (float)(a.rzs[j] / pqs);
  }
  __syncthreads();
  const long long N = (long long)f.H * f.W;
  float2* out = f.tmp + (long long)pair * f.H * kF;
  const int rend = min(f.H, (blockIdx.x + 1) * rpb);
  const uint64_t keep = l2_policy_keep();
  float rr0 = 0.f, rr1 = 0.f;
  for (int row = blockIdx.x * rpb + w; row < rend; row += kF512Warps) {
    const long long p0 = (long long)row * f.W;
    float2 v[16];
    if (a.defer_e) {
      // r only, both systems' loads in flight together: e += alpha p is left to the
      // next direction kernel or the commit
      const float* Q0 = a.Qp + (long long)j0 * N + p0;
      const float* Q1 = a.Qp + (long long)j1 * N + p0;
      float* R0 = a.Rr + (long long)j0 * N + p0;
      float* R1 = a.Rr + (long long)j1 * N + p0;
      float qa[16], ra[16], qb[16], rb[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int c = 32 * m + l;
        qa[m] = ra[m] = qb[m] = rb[m] = 0.f;
        if (c < f.W) {
          if (act0) {
            qa[m] = Q0[c];
            ra[m] = R0[c];
          }
          if (act1) {
            qb[m] = Q1[c];
            rb[m] = R1[c];
          }
        }
      }
      const float al0 = alpha_s[0], al1 = alpha_s[1];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int c = 32 * m + l;
        v[m] = make_float2(0.f, 0.f);
        if (c < f.W) {
          if (act0) {
            v[m].x = fmaf(-al0, qa[m], ra[m]);
            st_hint_f(R0 + c, v[m].x, keep);
            rr0 = fmaf(v[m].x, v[m].x, rr0);
          }
          if (act1) {
            v[m].y = fmaf(-al1, qb[m], rb[m]);
            st_hint_f(R1 + c, v[m].y, keep);
            rr1 = fmaf(v[m].y, v[m].y, rr1);
          }
        }
      }
    } else {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!(u ? act1 : act0)) {
#pragma unroll
        for (int m = 0; m < 16; ++m) (u ? v[m].y : v[m].x) = 0.f;
        continue;
      }
      const long long o = (long long)(j0 + u) * N + p0;
      const float* P = ((it & 1) ? a.P2 : a.P) + o;
      const float* Q = a.Qp + o;
      float* Ec = a.Ec + o;
      float* Rr = a.Rr + o;
      const float alpha = alpha_s[u];
      float pv[16], qv[16], rv[16], ev[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int c = 32 * m + l;
        pv[m] = qv[m] = rv[m] = ev[m] = 0.f;
        if (c < f.W) {
          pv[m] = P[c];
          qv[m] = Q[c];
          rv[m] = Rr[c];
          if (!first) ev[m] = Ec[c];
        }
      }
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int c = 32 * m + l;
        float r = 0.f;
        if (c < f.W) {
          Ec[c] = fmaf(alpha, pv[m], ev[m]);
          r = fmaf(-alpha, qv[m], rv[m]);
          st_hint_f(Rr + c, r, keep);
          if (u) rr1 = fmaf(r, r, rr1); else rr0 = fmaf(r, r, rr0);
        }
        (u ? v[m].y : v[m].x) = r;
      }
    }
    }
    fft512_warp(v, scratch[w], tw);
#pragma unroll
    for (int m = 0; m < 16; ++m) st_hint(out + (long long)row * kF + 32 * m + l, v[m], keep);
  }
  block_sumf<2>(rr0, rr1, 0.f, act0 ? a.part_rr + (long long)j0 * a.nb + blockIdx.x : nullptr,
                act1 ? a.part_rr + (long long)j1 * a.nb + blockIdx.x : nullptr, nullptr);
  if (arrive_last(a.arrive + j0, gridDim.x) && threadIdx.x < 32) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!(u ? act1 : act0)) continue;
      const int j = j0 + u;
      const double r2 = group_sum(a.part_rr + (long long)j * a.nb, gridDim.x);
      // the stopping rule of update_kernel
      if (threadIdx.x == 0) {
        a.scal[4 * j] = (r2 <= a.thr[j] || r2 > 16.0 * a.rr0[j]) ? 0.f : 1.f;
        if (a.defer_e) {
          a.scal[4 * j + 2] = alpha_s[u];
          a.scal[4 * j + 3] = (float)it;
        }
      }
    }
  }
}

// fft_cols_filter_kernel for HP = 512: the block takes columns c0 .. c0 + 7 of a
// pair, stages the 512 x 8 tile in shared memory (64-byte row segments from
// global memory; rows at and beyond H are zero), and each warp transforms one
// column in registers, filters it with hthT (the filter stored column-major,
// [c][i]), transforms again and leaves it in its slot for the block's store.
__global__ void __launch_bounds__(32 * kF512Warps, 3) fft512_cols_filter_kernel(FftDesc f,
                                                                            const float* __restrict__ hthT) {
  loop_step(f);
  if (pair_idle(f, blockIdx.y)) return;
  __shared__ float2 tw[kF];
  __shared__ float2 cols[kF512Warps][kXs];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) tw[m] = f.tw512[m];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int c0 = blockIdx.x * kF512Warps;
  float2* t = f.tmp + (long long)blockIdx.y * f.H * f.WP;
  const int cc = threadIdx.x & 7, ro = threadIdx.x >> 3;  // 32 rows x 8 columns per block step
  const uint64_t keep = l2_policy_keep();
  {
    float2 x[16];  // all of the thread's tile loads in flight at once
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = 32 * u + ro;
      x[u] = i < f.H ? ld_hint(t + (long long)i * f.WP + c0 + cc, keep) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) cols[cc][32 * u + ro] = x[u];
  }
  __syncthreads();
  float2* xs = cols[w];
  const float* g = hthT + (long long)(c0 + w) * kF;
  float gv[16];  // the filter column, loaded before the transform
#pragma unroll
  for (int m = 0; m < 16; ++m) gv[m] = g[32 * m + l];
  float2 v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = xs[32 * m + l];
  __syncwarp();
  fft512_warp(v, xs, tw);
  // filter, then the inverse transform as conj(F(conj(.)))
  const float dbar = (float)(*f.dbar);
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const float gi = __frcp_rn(gv[m] + dbar);
    v[m] = make_float2(v[m].x * gi, -v[m].y * gi);
  }
  fft512_warp(v, xs, tw);
#pragma unroll
  for (int m = 0; m < 16; ++m) xs[32 * m + l] = cconj(v[m]);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int i = 32 * u + ro;
    if (i < f.H) st_hint(t + (long long)i * f.WP + c0 + cc, cols[cc][i], keep);
  }
}

// fft_rows_inv_kernel for WP = 512: one warp per row of the block's range
// [blockIdx.x rows_per, +rows_per), rows_per = ceil(H / nbz).
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft512_rows_inv_kernel(FftDesc f,
                                                                         const float* __restrict__ Rr,
                                                                         float* Z, double* part_rz) {
  if (pair_idle(f, blockIdx.y)) return;
  __shared__ float2 tw[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) tw[m] = f.tw512[m];
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const long long N = (long long)f.H * f.W;
  const float scale = 1.0f / ((float)f.HP * (float)kF);
  const int rows_per = (f.H + f.nbz - 1) / f.nbz;
  const int rend = min(f.H, (blockIdx.x + 1) * rows_per);
  const float2* tin = f.tmp + (long long)pair * f.H * kF;
  const uint64_t release = l2_policy_release();
  double acc0 = 0.0, acc1 = 0.0;
  // the row's transform input and both residuals, all loads in flight together
  float2 nv[16], nr[16];
  auto load_row = [&](int rw) {
    const long long p0 = (long long)rw * f.W;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      nv[m] = cconj(ld_hint(tin + (long long)rw * kF + 32 * m + l, release));
      const int c = 32 * m + l;
      nr[m] = make_float2(0.f, 0.f);
      if (c < f.W) {
        nr[m].x = ld_hint(Rr + (long long)j0 * N + p0 + c, release);
        if (two) nr[m].y = ld_hint(Rr + (long long)j1 * N + p0 + c, release);
      }
    }
  };
  int row = blockIdx.x * rows_per + w;
  for (; row < rend; row += kF512Warps) {
    load_row(row);
    const long long p0 = (long long)row * f.W;
    float2 v[16], rr[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      v[m] = nv[m];
      rr[m] = nr[m];
    }
    fft512_warp(v, scratch[w], tw);
    float rz0 = 0.f, rz1 = 0.f;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int c = 32 * m + l;
      if (c < f.W) {
        const long long p = p0 + c;
        const float z0 = v[m].x * scale;
        Z[(long long)j0 * N + p] = z0;
        rz0 = fmaf(rr[m].x, z0, rz0);
        if (two) {
          const float z1 = -v[m].y * scale;
          Z[(long long)j1 * N + p] = z1;
          rz1 = fmaf(rr[m].y, z1, rz1);
        }
      }
    }
    acc0 += (double)rz0;
    acc1 += (double)rz1;
  }
  block_sum3(acc0, acc1, 0.0, part_rz + (long long)j0 * f.nbz + blockIdx.x,
             two ? part_rz + (long long)j1 * f.nbz + blockIdx.x : nullptr, nullptr);
  rz_tail(f, pair, part_rz);
}

// ---- register-resident 1024-point transforms
//
// A 1024-point transform held by one warp as lo[q] = x[32 q + l], hi[q] = x[512 + 32 q + l]
// (q < 16) takes one decimation-in-frequency step into two 512-point transforms:
//   a[n] = x[n] + x[n + 512],  b[n] = (x[n] - x[n + 512]) w1024^n   (n < 512),
//   X[2 k] = A[k],  X[2 k + 1] = B[k]   (A, B the 512-point transforms of a and b),
// which keeps the 512-point kernels' layout: afterwards lo[m] = X[64 m + 2 l] and
// hi[m] = X[64 m + 2 l + 1] in lane l, one float4 of the transform in natural order.
constexpr int kRowsPerWarp1024 = 2;
constexpr int kXs2 = 2 * kF + 66;  // staged-column pitch of the 1024-point column pass

__device__ __forceinline__ void fft1024_warp(float2 (&lo)[16], float2 (&hi)[16], float2* xs,
                                             const float2* tw, const float2* tw2) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float2 x0 = lo[q], x1 = hi[q];
    lo[q] = cadd(x0, x1);
    hi[q] = cmul(csub(x0, x1), tw2[32 * q + l]);
  }
  fft512_warp(lo, xs, tw);
  fft512_warp(hi, xs, tw);
}

// fft_rows_fwd_kernel for WP = 1024: one warp per row, rows [blockIdx.x rpb, +rpb).
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft1024_rows_fwd_kernel(FftDesc f,
                                                                          const float* __restrict__ Rr,
                                                                          int rpb) {
  if (pair_idle(f, blockIdx.y)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters)
    atomicAdd(&f.counters[DC_CG_PRE_UNITS], 2 * blockIdx.y + 1 < f.R ? 2ull : 1ull);
  __shared__ float2 tw[kF], tw2[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) {
    tw[m] = f.tw512[m];
    tw2[m] = f.tw1024[m];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const long long N = (long long)f.H * f.W;
  const float* r0p = Rr + (long long)j0 * N;
  const float* r1p = Rr + (long long)j1 * N;
  float2* out = f.tmp + (long long)pair * f.H * (2 * kF);
  const int rend = min(f.H, (blockIdx.x + 1) * rpb);
  const uint64_t keep = l2_policy_keep();
  for (int row = blockIdx.x * rpb + w; row < rend; row += kF512Warps) {
    const long long p0 = (long long)row * f.W;
    float2 lo[16], hi[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = 32 * q + l, c2 = c + kF;
      lo[q] = hi[q] = make_float2(0.f, 0.f);
      if (c < f.W) lo[q] = make_float2(ld_hint(r0p + p0 + c, keep), two ? ld_hint(r1p + p0 + c, keep) : 0.f);
      if (c2 < f.W) hi[q] = make_float2(ld_hint(r0p + p0 + c2, keep), two ? ld_hint(r1p + p0 + c2, keep) : 0.f);
    }
    fft1024_warp(lo, hi, scratch[w], tw, tw2);
#pragma unroll
    for (int m = 0; m < 16; ++m) st_hint4(out + (long long)row * (2 * kF) + 64 * m + 2 * l, lo[m], hi[m], keep);
  }
}

// fft512_update_rows_fwd_kernel for WP = 1024, deferred correction updates only
// (a.defer_e): r -= alpha q per active system of the pair, the new residual rows
// transformed without a re-read; the pair's last block sets the active flags, alpha
// and the iteration.  A row's loads go in four batches of eight columns per lane.
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft1024_update_rows_fwd_kernel(FftDesc f,
                                                                                 CgArgs a,
                                                                                 int it_arg,
                                                                                 int rpb) {
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const bool act0 = a.scal[4 * j0] != 0.f, act1 = two && a.scal[4 * j1] != 0.f;
  if (!act0 && !act1) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters) {
    atomicAdd(&f.counters[DC_CG_PRE_UNITS], two ? 2ull : 1ull);
    atomicAdd(&f.counters[DC_CG_UPD_UNITS], (unsigned long long)(act0 + act1));
  }
  const int it = a.it_dev ? *a.it_dev : it_arg;
  __shared__ float2 tw[kF], tw2[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  __shared__ float alpha_s[2];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) {
    tw[m] = f.tw512[m];
    tw2[m] = f.tw1024[m];
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w < 2 && (w == 0 ? act0 : act1)) {
    const int j = j0 + w;
    const double pqs = group_sum(a.part_pq + (long long)j * a.nb, a.nb);
    if (l == 0) alpha_s[w] = (float)(a.rzs[j] / pqs);
  }
  __syncthreads();
  const long long N = (long long)f.H * f.W;
  float2* out = f.tmp + (long long)pair * f.H * (2 * kF);
  const int rend = min(f.H, (blockIdx.x + 1) * rpb);
  const uint64_t keep = l2_policy_keep();
  const float al0 = alpha_s[0], al1 = alpha_s[1];
  float rr0 = 0.f, rr1 = 0.f;
  for (int row = blockIdx.x * rpb + w; row < rend; row += kF512Warps) {
    const long long p0 = (long long)row * f.W;
    const float* Q0 = a.Qp + (long long)j0 * N + p0;
    const float* Q1 = a.Qp + (long long)j1 * N + p0;
    float* R0 = a.Rr + (long long)j0 * N + p0;
    float* R1 = a.Rr + (long long)j1 * N + p0;
    float2 lo[16], hi[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      // columns 256 b + 32 qq + l, qq < 8: lo[8 b + qq] for b < 2, hi[8 (b - 2) + qq] after
      float qa[8], ra[8], qb[8], rb[8];
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        const int c = 256 * b + 32 * qq + l;
        qa[qq] = ra[qq] = qb[qq] = rb[qq] = 0.f;
        if (c < f.W) {
          if (act0) {
            qa[qq] = Q0[c];
            ra[qq] = R0[c];
          }
          if (act1) {
            qb[qq] = Q1[c];
            rb[qq] = R1[c];
          }
        }
      }
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        const int c = 256 * b + 32 * qq + l;
        float2 v = make_float2(0.f, 0.f);
        if (c < f.W) {
          if (act0) {
            v.x = fmaf(-al0, qa[qq], ra[qq]);
            st_hint_f(R0 + c, v.x, keep);
            rr0 = fmaf(v.x, v.x, rr0);
          }
          if (act1) {
            v.y = fmaf(-al1, qb[qq], rb[qq]);
            st_hint_f(R1 + c, v.y, keep);
            rr1 = fmaf(v.y, v.y, rr1);
          }
        }
        if (b < 2)
          lo[8 * b + qq] = v;
        else
          hi[8 * (b - 2) + qq] = v;
      }
    }
    fft1024_warp(lo, hi, scratch[w], tw, tw2);
#pragma unroll
    for (int m = 0; m < 16; ++m) st_hint4(out + (long long)row * (2 * kF) + 64 * m + 2 * l, lo[m], hi[m], keep);
  }
  block_sumf<2>(rr0, rr1, 0.f, act0 ? a.part_rr + (long long)j0 * a.nb + blockIdx.x : nullptr,
                act1 ? a.part_rr + (long long)j1 * a.nb + blockIdx.x : nullptr, nullptr);
  if (arrive_last(a.arrive + j0, gridDim.x) && threadIdx.x < 32) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!(u ? act1 : act0)) continue;
      const int j = j0 + u;
      const double r2 = group_sum(a.part_rr + (long long)j * a.nb, gridDim.x);
      // the stopping rule of update_kernel
      if (threadIdx.x == 0) {
        a.scal[4 * j] = (r2 <= a.thr[j] || r2 > 16.0 * a.rr0[j]) ? 0.f : 1.f;
        a.scal[4 * j + 2] = alpha_s[u];
        a.scal[4 * j + 3] = (float)it;
      }
    }
  }
}

// fft_cols_filter_kernel for HP = 1024: the block stages columns c0 .. c0 + 7 of a pair
// (rows at and beyond H are zero); each warp transforms one column, filters it with
// hthT (column-major, [c][i]), writes it back to its slot in natural order and
// transforms it again (the inverse as conj(F(conj(.)))); the block then stores rows
// below H.  Shared memory: kF512Warps x kXs2 float2, dynamic.
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft1024_cols_filter_kernel(FftDesc f,
                                                                             const float* __restrict__ hthT) {
  loop_step(f);
  if (pair_idle(f, blockIdx.y)) return;
  __shared__ float2 tw[kF], tw2[kF];
  extern __shared__ float4 colsm4[];
  float2* cols = reinterpret_cast<float2*>(colsm4);
  for (int m = threadIdx.x; m < kF; m += blockDim.x) {
    tw[m] = f.tw512[m];
    tw2[m] = f.tw1024[m];
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int c0 = blockIdx.x * kF512Warps;
  float2* t = f.tmp + (long long)blockIdx.y * f.H * f.WP;
  const int cc = threadIdx.x & 7, ro = threadIdx.x >> 3;  // 32 rows x 8 columns per block step
  const uint64_t keep = l2_policy_keep();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float2 x[16];  // half of the thread's tile loads in flight at once
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = 32 * (16 * h + u) + ro;
      x[u] = i < f.H ? ld_hint(t + (long long)i * f.WP + c0 + cc, keep) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) cols[cc * kXs2 + 32 * (16 * h + u) + ro] = x[u];
  }
  __syncthreads();
  float2* xs = cols + w * kXs2;
  float2 lo[16], hi[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    lo[q] = xs[32 * q + l];
    hi[q] = xs[kF + 32 * q + l];
  }
  __syncwarp();
  fft1024_warp(lo, hi, xs, tw, tw2);
  // filter (frequencies 64 m + 2 l and 64 m + 2 l + 1 of this lane), conjugated for the
  // inverse, and back to natural order in the slot
  const float* g = hthT + (long long)(c0 + w) * (2 * kF);
  const float dbar = (float)(*f.dbar);
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const float2 gv = *reinterpret_cast<const float2*>(g + 64 * m + 2 * l);
    const float g0 = __frcp_rn(gv.x + dbar), g1 = __frcp_rn(gv.y + dbar);
    lo[m] = make_float2(lo[m].x * g0, -lo[m].y * g0);
    hi[m] = make_float2(hi[m].x * g1, -hi[m].y * g1);
  }
#pragma unroll
  for (int m = 0; m < 16; ++m)
    *reinterpret_cast<float4*>(xs + 64 * m + 2 * l) = make_float4(lo[m].x, lo[m].y, hi[m].x, hi[m].y);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    lo[q] = xs[32 * q + l];
    hi[q] = xs[kF + 32 * q + l];
  }
  __syncwarp();
  fft1024_warp(lo, hi, xs, tw, tw2);
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const float2 a = cconj(lo[m]), b = cconj(hi[m]);
    *reinterpret_cast<float4*>(xs + 64 * m + 2 * l) = make_float4(a.x, a.y, b.x, b.y);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 32; ++u) {
    const int i = 32 * u + ro;
    if (i < f.H) st_hint(t + (long long)i * f.WP + c0 + cc, cols[cc * kXs2 + i], keep);
  }
}

// fft_rows_inv_kernel for WP = 1024: one warp per row of the block's range
// [blockIdx.x rows_per, +rows_per), rows_per = ceil(H / nbz).
__global__ void __launch_bounds__(32 * kF512Warps, 2) fft1024_rows_inv_kernel(FftDesc f,
                                                                          const float* __restrict__ Rr,
                                                                          float* Z, double* part_rz) {
  if (pair_idle(f, blockIdx.y)) return;
  __shared__ float2 tw[kF], tw2[kF];
  __shared__ float2 scratch[kF512Warps][kXs];
  for (int m = threadIdx.x; m < kF; m += blockDim.x) {
    tw[m] = f.tw512[m];
    tw2[m] = f.tw1024[m];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int pair = blockIdx.y;
  const int j0 = 2 * pair, j1 = 2 * pair + 1;
  const bool two = j1 < f.R;
  const long long N = (long long)f.H * f.W;
  const float scale = 1.0f / ((float)f.HP * (float)(2 * kF));
  const int rows_per = (f.H + f.nbz - 1) / f.nbz;
  const int rend = min(f.H, (blockIdx.x + 1) * rows_per);
  const float2* tin = f.tmp + (long long)pair * f.H * (2 * kF);
  const uint64_t release = l2_policy_release();
  const float* r0p = Rr + (long long)j0 * N;
  const float* r1p = Rr + (long long)j1 * N;
  double acc0 = 0.0, acc1 = 0.0;
  for (int row = blockIdx.x * rows_per + w; row < rend; row += kF512Warps) {
    const long long p0 = (long long)row * f.W;
    const float2* trow = tin + (long long)row * (2 * kF);
    float2 lo[16], hi[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      lo[q] = cconj(ld_hint(trow + 32 * q + l, release));
      hi[q] = cconj(ld_hint(trow + kF + 32 * q + l, release));
    }
    fft1024_warp(lo, hi, scratch[w], tw, tw2);
    // lo[m], hi[m]: columns 64 m + 2 l and 64 m + 2 l + 1; the residuals there are read
    // in two halves of eight m each
    float rz0 = 0.f, rz1 = 0.f;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      float ra[8][2], rb[8][2];
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = 64 * (8 * hf + mm) + 2 * l + e;
          ra[mm][e] = rb[mm][e] = 0.f;
          if (c < f.W) {
            ra[mm][e] = ld_hint(r0p + p0 + c, release);
            if (two) rb[mm][e] = ld_hint(r1p + p0 + c, release);
          }
        }
      }
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
        const int m = 8 * hf + mm;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = 64 * m + 2 * l + e;
          if (c < f.W) {
            const float2 v = e ? hi[m] : lo[m];
            const long long p = p0 + c;
            const float z0 = v.x * scale;
            Z[(long long)j0 * N + p] = z0;
            rz0 = fmaf(ra[mm][e], z0, rz0);
            if (two) {
              const float z1 = -v.y * scale;
              Z[(long long)j1 * N + p] = z1;
              rz1 = fmaf(rb[mm][e], z1, rz1);
            }
          }
        }
      }
    }
    acc0 += (double)rz0;
    acc1 += (double)rz1;
  }
  block_sum3(acc0, acc1, 0.0, part_rz + (long long)j0 * f.nbz + blockIdx.x,
             two ? part_rz + (long long)j1 * f.nbz + blockIdx.x : nullptr, nullptr);
  rz_tail(f, pair, part_rz);
}

// |h_f|^2 / xi on the H x W frequency grid (phases reduced exactly in integers).
// transposed: out[fc * H + fr] (column-major, the layout of the 512- and 1024-point
// column passes).
__global__ void hth_kernel(float* out, int H, int W, const float* k, int kh, int kw, float inv_xi,
                           int transposed) {
  const long long N = (long long)H * W;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const int fr = (int)(p / W), fc = (int)(p - (long long)fr * W);
    double re = 0.0, im = 0.0;
    for (int a = 0; a < kh; ++a) {
      const long long pr = ((long long)fr * a) % H;
      for (int b = 0; b < kw; ++b) {
        const long long pc = ((long long)fc * b) % W;
        // phase / pi = -2 (pr / H + pc / W)
        const double ph = -2.0 * ((double)pr / H + (double)pc / W);
        double sn, cs;
        sincospi(ph, &sn, &cs);
        re += (double)k[a * kw + b] * cs;
        im += (double)k[a * kw + b] * sn;
      }
    }
    out[transposed ? (long long)fc * H + fr : p] = (float)((re * re + im * im) * inv_xi);
  }
}

// Number of systems still active after the last update (their flags).
__global__ void check_kernel(const float* scal, int R, int* active) {
  int cnt = 0;
  for (int j = threadIdx.x; j < R; j += blockDim.x) cnt += scal[4 * j] != 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
  __shared__ int wsum[32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    *active = t;
  }
}

// ---- device-driven solver loop (CUDA graph with conditional nodes)
//
// The refinement passes and the CG iterations of a pass run as two nested WHILE
// nodes of a graph, with an IF node around each pass; their conditions are set
// by the kernels below from counters in device memory, so a likelihood-site
// update needs no host round trip.  The outer body (and the inner one with Jacobi)
// starts by clearing its own condition (cond_clear_kernel), so a body that did not
// set it again ends the loop; with the FFT preconditioner the column pass of every
// iteration sets the inner condition to 0 or 1 (loop_step).  The counters bound
// both loops (max_outer passes, max_iter iterations).
// Iterative refinement of the likelihood-site solves: a true residual in
// float-float, then FP32 preconditioned CG on the correction until its recurrence
// residual has dropped below max(eta ||r||, (rtol / 2) ||b||), repeated until
// ||r|| <= rtol ||b|| for every system.  With eta = 3.2e-5 the second term decides
// once the warm start is within about 1e-4 relative of the solution (every sweep
// after the first few), so a sweep normally needs one pass; a cold start still
// moves in steps of eta, which FP32 CG reaches before its rounding floor.
constexpr double kEta2 = 1e-9;

__global__ void cond_clear_kernel(cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
}

__global__ void loop_init_kernel(LoopState* ls) {
  if (threadIdx.x == 0) {
    ls->it = 0;
    ls->outer = 0;
    ls->total = 0;
    ls->converged = 0;
  }
}

// After a true residual and its thresholds: start another pass, or stop
// (converged, or out of passes or iterations), as the host loop does.
__global__ void pass_kernel(LoopState* ls, const int* active, int max_outer, int max_iter,
                            cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_pass,
                            cudaGraphConditionalHandle h_inner) {
  if (threadIdx.x != 0) return;
  unsigned go = 0;
  if (*active == 0) {
    ls->converged = 1;
  } else if (ls->outer < max_outer && ls->total < max_iter) {
    go = 1;
    ls->it = 0;
    ls->outer += 1;
  }
  cudaGraphSetConditional(h_pass, go);
  cudaGraphSetConditional(h_outer, go);
  cudaGraphSetConditional(h_inner, go);
}

// After a CG iteration: count it, and go on while a system is active and the
// iteration budget lasts.
__global__ void iter_kernel(LoopState* ls, const float* scal, int R, int max_iter,
                            cudaGraphConditionalHandle h_inner) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int j = threadIdx.x; j < R; j += blockDim.x) mine += scal[4 * j] != 0.f;
  if (mine) atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    ls->it += 1;
    ls->total += 1;
    cudaGraphSetConditional(h_inner, (cnt > 0 && ls->total < max_iter) ? 1u : 0u);
  }
}

__global__ void loop_finish_kernel(const LoopState* ls, unsigned* status,
                                   unsigned long long* counters) {
  if (threadIdx.x == 0) {
    if (!ls->converged) atomicOr(status, ST_CG_NOCONV);
    counters[DC_CG_ITERS] = (unsigned long long)ls->total;
  }
}

// Rao-Blackwellised terms of the probes, by an explicit matvec of each computed
// sample: with Q z = H^T H z / xi + d z and (H^T H)_ii = g0 = sum k^2, the
// off-diagonal part of row i is
//   o_s(i) = sum_{j != i} Q_ij z_{s,j} = (H^T H z_s)_i / xi - (g0 / xi) z_{s,i}
// (the d z terms cancel).  Block z = group g of kRbGroup probes; the block's
// tile sums o_s(i)^2 over its probes in order and writes acc[g][i].
constexpr int kRbGroup = 8;

__global__ void __launch_bounds__(kThreads) rb_offdiag_kernel(CgArgs a, float* acc) {
  extern __shared__ float smem[];
  const ConvDesc& c = a.c;
  const int g = blockIdx.z;
  const int s_lo = g * kRbGroup, s_hi = min(a.S, s_lo + kRbGroup);
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  StencilSmem sm = carve(c, smem);
  __shared__ float outb[kTile * kTile];
  __shared__ int ctab[kTile + 2 * kMaxHalf];
  stage_taps(c, sm.taps);
  const int RH = kTile + 2 * c.hr, RW = kTile + 2 * c.hc;
  column_table(ctab, c0 - c.hc, RW, c.W);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  constexpr int kRowsPerThread = kTile / (kThreads / 32);
  float sq[kRowsPerThread];
#pragma unroll
  for (int u = 0; u < kRowsPerThread; ++u) sq[u] = 0.f;
  for (int s = s_lo; s < s_hi; ++s) {
    const double* z = a.X + (long long)(s + 1) * c.N;
    for (int rr = ty; rr < RH; rr += kThreads / 32) {
      const long long rowp = (long long)wrapi(r0 - c.hr + rr, c.H) * c.W;
      for (int cc = tx; cc < RW; cc += 32) sm.v[rr * RW + cc] = (float)z[rowp + ctab[cc]];
    }
    __syncthreads();
    hth_tile(c, sm, outb);
#pragma unroll
    for (int u = 0; u < kRowsPerThread; ++u) {
      const int tr = ty + u * (kThreads / 32);
      const float zi = sm.v[(tr + c.hr) * RW + tx + c.hc];
      const float o = outb[tr * kTile + tx] * c.inv_xi - c.g0_xi * zi;
      sq[u] = fmaf(o, o, sq[u]);
    }
    __syncthreads();  // the next probe overwrites the staged region
  }
#pragma unroll
  for (int u = 0; u < kRowsPerThread; ++u) {
    const int gr = r0 + ty + u * (kThreads / 32), gcol = c0 + tx;
    if (gr < c.H && gcol < c.W) acc[(long long)g * c.N + (long long)gr * c.W + gcol] = sq[u];
  }
}

// Eq. update_q0_x from E = X[0] and the RBMC variance, with cap and damping.
// acc: the n_groups planes of rb_offdiag_kernel, summed in group order.
__global__ void site0_kernel(CgArgs a, const float* acc, int n_groups, float* tau0, float* nu0,
                             float min_tau, float damping, unsigned* status,
                             unsigned long long* counters) {
  const long long N = a.c.N;
  unsigned capped = 0;
  bool bad = false;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const float minv = a.Minv[p];
    float sq = 0.f;
    for (int g = 0; g < n_groups; ++g) sq += acc[(long long)g * N + p];
    const float var = minv + minv * minv * sq / (float)a.S;
    const float E = (float)a.X[p];
    const float d = a.D[p];
    float tn = 1.0f / var - d;
    if (!(tn >= min_tau)) {
      tn = min_tau;
      ++capped;
    }
    const float nn = tn * E + d * E - a.Ncav[p];  // tau E + (E - m) / c
    const float t_new = damping * tn + (1.0f - damping) * tau0[p];
    const float n_new = damping * nn + (1.0f - damping) * nu0[p];
    tau0[p] = t_new;
    nu0[p] = n_new;
    bad |= !(isfinite(t_new) && isfinite(n_new));
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  if (capped) atomicAdd(&counters[DC_CAPPED], (unsigned long long)capped);
}

// out = scale * H^T in (periodic), one plane per blockIdx.y; one-time setup.
__global__ void conv_t_kernel(const float* in, float* out, int H, int W, const float* k, int kh,
                              int kw, float scale, int planes) {
  const long long N = (long long)H * W;
  const int pl = blockIdx.y;
  if (pl >= planes) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(p / W), c = (int)(p - (long long)r * W);
    double acc = 0.0;
    for (int a = 0; a < kh; ++a)
      for (int b = 0; b < kw; ++b) {
        const int rr = wrapi(r + a - kh / 2, H), cc = wrapi(c + b - kw / 2, W);
        acc += (double)k[a * kw + b] * (double)in[(long long)pl * N + (long long)rr * W + cc];
      }
    out[(long long)pl * N + p] = (float)(acc * scale);
  }
}

// Standard normals from SplitMix64 (Steele, Lea and Flood, 2014) used as a
// counter-based generator: draw t is the output for state seed + (t+1) * golden
// gamma; two 24-bit uniforms feed the Box-Muller transform.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long t) {
  unsigned long long z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void normals_kernel(float* out, long long count, unsigned long long seed,
                               unsigned long long base) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long t = 2ull * (base + (unsigned long long)i);
    const double u1 = ((double)(splitmix64(seed, t) >> 40) + 0.5) * (1.0 / 16777216.0);
    const double u2 = ((double)(splitmix64(seed, t + 1) >> 40) + 0.5) * (1.0 / 16777216.0);
    out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

__global__ void set_status_kernel(unsigned* status, unsigned bit) { atomicOr(status, bit); }
__global__ void scale_kernel(float* out, const float* in, long long n, float scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i] * scale;
}
__global__ void store_iters_kernel(unsigned long long* counters, unsigned long long v) {
  counters[DC_CG_ITERS] = v;
}

inline int grid1d(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 1 << 20);
}

}  // namespace

struct LikelihoodState {
  CsState* cs = nullptr;    // dense operator: everything below is unused
  ConvDesc c;
  int S = 0, R = 0;
  float inv_xi = 0.f;
  double rtol2 = 0.0;
  int max_iter = 0;
  unsigned long long seed = 0;
  float damping = 0.5f, min_tau = 1e-8f;
  float* d_k = nullptr;
  float* d_g = nullptr;     // gr then gc
  float* Hty = nullptr;
  const float* Y0 = nullptr;  // the context's copy of y
  float* E1 = nullptr;
  float* E2 = nullptr;
  float* D = nullptr;
  float* Ncav = nullptr;
  float* Minv = nullptr;
  double* X = nullptr;      // FP64 solutions (warm starts across sweeps)
  float* Y1 = nullptr;      // sqrt(xi) eps1
  double* thr = nullptr;    // inner convergence thresholds
  double* d_hd = nullptr;   // forward-blur taps FP64
  float* d_hf = nullptr;    // forward-blur taps FP32
  double rtol2_true = 0.0;  // target of the true relative residual of the mean solve, squared
  double rtol2_probe = 0.0; // the same for the probe solves
  int max_outer = 24;
  float* Rr = nullptr;
  float* P = nullptr;
  float* P2 = nullptr;
  float* Qp = nullptr;
  double* part = nullptr;   // pq, rz[2], rr[2], bb
  int nbz = 0, nbmax = 0;
  // circulant FFT preconditioner (power-of-two sizes)
  bool fft = false;
  FftDesc fd;
  float2* ftmp = nullptr;
  float* Z = nullptr;
  float* hth = nullptr;
  float2* tw512 = nullptr;      // w512^m, then w1024^m (m < 512)
  double* dpart = nullptr;
  double* dbar = nullptr;
  int prep_blocks = 0;
  size_t smem_rows = 0, smem_cols = 0;
  int* d_active = nullptr;
  int* h_active = nullptr;  // pinned, 2 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int nb = 0;
  size_t smem = 0;
  size_t smem_res = 0;
  int last_iters = 0;
  float* d_scal = nullptr;      // [R][4] CG scalars: active flag, beta, alpha and iteration of
                                // a deferred correction update
  double* d_rzs = nullptr;      // [R] r.z of the current iteration
  unsigned* d_arrive = nullptr; // [R + pairs] block-arrival counters (start and stay zero)
  int* d_act0 = nullptr;        // [R] systems that iterate in the current pass
  float* Ec = nullptr;          // R planes: FP32 correction of the current pass
  // the update as a graph with conditional nodes, one per prior-site buffer
  LoopState* d_loop = nullptr;
  struct {
    const float* tp = nullptr;
    cudaGraphExec_t exec = nullptr;
  } graph[2];
  bool graph_failed = false;    // capture or instantiation refused: host-driven loop only
  bool graph_last = false;      // the last update ran from a graph
  double* d_relres = nullptr;  // [R] sqrt(r.r / b.b) after the last true residual
  double* d_prev_rr = nullptr; // [R] r.r of the previous refinement pass
  double* d_rr0 = nullptr;     // [R] r.r at the start of the current pass
  double* h_relres = nullptr;  // pinned copy
  double rep_mean = 0.0, rep_probe = 0.0;
  int rep_outer = 0;
  bool debug = false;
};

namespace {

CgArgs cg_args(LikelihoodState* L) {
  CgArgs a = {};
  a.c = L->c;
  a.R = L->R;
  a.S = L->S;
  a.X = L->X;
  a.Rr = L->Rr;
  a.P = L->P;
  a.P2 = L->P2;
  a.Qp = L->Qp;
  a.D = L->D;
  a.Ncav = L->Ncav;
  a.Minv = L->Minv;
  a.Hty = L->Hty;
  a.E1 = L->E1;
  a.E2 = L->E2;
  a.Y0 = L->Y0;
  a.Y1 = L->Y1;
  a.thr = L->thr;
  a.rr0 = L->d_rr0;
  a.scal = L->d_scal;
  a.rzs = L->d_rzs;
  a.arrive = L->d_arrive;
  a.act0 = L->d_act0;
  a.it_dev = nullptr;
  a.Z = L->Z;
  a.Ec = L->Ec;
  const long long rn = (long long)L->R * L->nbmax;
  a.part_pq = L->part;
  a.part_rz = L->part + rn;
  a.part_rr = L->part + 2 * rn;
  a.part_bb = L->part + 3 * rn;
  a.rtol2 = L->rtol2;
  a.nb = L->nb;
  a.nbz = L->nbz;
  a.fft = L->fft ? 1 : 0;
  a.counters = nullptr;
  a.defer_e = 0;
  return a;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// z = M^{-1} r; r.z partials into rz_buf ([R][nbz]).  With cg (the solver's own
// call), pairs of systems that have both stopped are skipped and the inverse row
// pass sets beta and r.z of the active systems (first: the first application of a
// refinement pass, beta = 0); without it every system is transformed and the CG
// scalars are left alone (launch-shape tuning).
// stages: 1 = the forward row pass (fused with the CG update when upd is given:
// 512-point rows only, see fused_update), 2 = the column and inverse row passes.
// step: graph replays, whose column pass then advances the inner loop and its
// condition h_step (loop_step).
void precond_apply(LikelihoodState* L, double* rz_buf, bool cg, int first,
                   unsigned long long* counters, cudaStream_t s, const CgArgs* upd = nullptr,
                   int it = 0, int stages = 3, bool step = false,
                   cudaGraphConditionalHandle h_step = 0) {
  FftDesc f = L->fd;
  f.loop = step ? L->d_loop : nullptr;
  f.h_inner = h_step;
  f.max_iter = L->max_iter;
  f.act = cg ? L->d_scal : nullptr;
  f.scal_w = cg ? L->d_scal : nullptr;
  f.rzs = cg ? L->d_rzs : nullptr;
  f.arrive = L->d_arrive + L->R;
  f.first = first;
  f.counters = counters;
  constexpr int kRows512 = kF512Warps * kRowsPerWarp512;
  constexpr int kRows1024 = kF512Warps * kRowsPerWarp1024;
  if (stages & 1) {
    if (upd && fft1024_rows(f))
      fft1024_update_rows_fwd_kernel<<<dim3((f.H + kRows1024 - 1) / kRows1024, f.pairs),
                                       32 * kF512Warps, 0, s>>>(f, *upd, it, kRows1024);
    else if (upd)
      fft512_update_rows_fwd_kernel<<<dim3((f.H + kRows512 - 1) / kRows512, f.pairs),
                                      32 * kF512Warps, 0, s>>>(f, *upd, it, kRows512);
    else if (fft512_rows(f))
      fft512_rows_fwd_kernel<<<dim3((f.H + kRows512 - 1) / kRows512, f.pairs), 32 * kF512Warps, 0,
                               s>>>(f, L->Rr, kRows512);
    else if (fft1024_rows(f))
      fft1024_rows_fwd_kernel<<<dim3((f.H + kRows1024 - 1) / kRows1024, f.pairs), 32 * kF512Warps,
                                0, s>>>(f, L->Rr, kRows1024);
    else
      fft_rows_fwd_kernel<<<dim3((f.H + f.rpb - 1) / f.rpb, f.pairs), kFftThreads, L->smem_rows,
                            s>>>(f, L->Rr);
  }
  if (!(stages & 2)) return;
  if (fft512_cols(f))
    fft512_cols_filter_kernel<<<dim3(f.WP / kF512Warps, f.pairs), 32 * kF512Warps, 0, s>>>(f, f.hth);
  else if (fft1024_cols(f))
    fft1024_cols_filter_kernel<<<dim3(f.WP / kF512Warps, f.pairs), 32 * kF512Warps,
                                 sizeof(float2) * kF512Warps * kXs2, s>>>(f, f.hth);
  else
    fft_cols_filter_kernel<<<dim3(f.WP / f.cw, f.pairs), kFftThreads, L->smem_cols, s>>>(f);
  if (fft512_rows(f))
    fft512_rows_inv_kernel<<<dim3(f.nbz, f.pairs), 32 * kF512Warps, 0, s>>>(f, L->Rr, L->Z, rz_buf);
  else if (fft1024_rows(f))
    fft1024_rows_inv_kernel<<<dim3(f.nbz, f.pairs), 32 * kF512Warps, 0, s>>>(f, L->Rr, L->Z, rz_buf);
  else
    fft_rows_inv_kernel<<<dim3(f.nbz, f.pairs), kFftThreads, L->smem_rows, s>>>(f, L->Rr, L->Z,
                                                                                rz_buf);
}

// The true residual of every system: two systems per block for a separable K x K blur,
// K = 5, 9 or 15 (residual_pair_kernel), else one (residual_kernel).
template <int K>
void launch_residual_pair(const LikelihoodState* L, const CgArgs& a, cudaStream_t s) {
  constexpr int RH = kTile + 2 * (K - 1), MW = kTile + 2 * (K / 2);
  const size_t sm = sizeof(float2) * 2 * ((size_t)RH * RH + (size_t)RH * MW);
  const ConvDesc& c = L->c;
  residual_pair_kernel<K><<<dim3(c.tiles_x, c.tiles_y, (L->R + 1) / 2), kThreads, sm, s>>>(a);
}

void launch_residual(const LikelihoodState* L, const CgArgs& a, cudaStream_t s) {
  const ConvDesc& c = L->c;
  if (c.separable && c.kh == c.kw) {
    switch (c.kh) {
      case 5: launch_residual_pair<5>(L, a, s); return;
      case 9: launch_residual_pair<9>(L, a, s); return;
      case 15: launch_residual_pair<15>(L, a, s); return;
      default: break;
    }
  }
  residual_kernel<<<dim3(c.tiles_x, c.tiles_y, L->R), kThreads, L->smem_res, s>>>(a);
}

// Whether the direction step runs two systems per block (direction_pair_kernel).
inline bool pair_direction(const LikelihoodState* L) {
  const ConvDesc& c = L->c;
  return L->fft && c.separable && c.hr == c.hc &&
         (c.hr == 2 || c.hr == 4 || c.hr == 8 || c.hr == 14);
}

void launch_direction(const LikelihoodState* L, const CgArgs& a, int it, cudaStream_t s) {
  const ConvDesc& c = L->c;
  if (pair_direction(L)) {
    const dim3 g(c.tiles_x, c.tiles_y, (L->R + 1) / 2);
    // region (RH x RW) and row-pass output (RH x kTile) pairs
    const size_t sm = sizeof(float2) * (size_t)(kTile + 2 * c.hr) * (2 * kTile + 2 * c.hr);
    switch (c.hr) {
      case 2: direction_pair_kernel<2><<<g, kThreads, sm, s>>>(a, it); return;
      case 4: direction_pair_kernel<4><<<g, kThreads, sm, s>>>(a, it); return;
      case 8: direction_pair_kernel<8><<<g, kThreads, sm, s>>>(a, it); return;
      default: direction_pair_kernel<14><<<g, kThreads, sm, s>>>(a, it); return;
    }
  }
  direction_kernel<<<dim3(c.tiles_x, c.tiles_y, L->R), kThreads, L->smem, s>>>(a, it);
}

// Whether a CG iteration runs its update inside the preconditioner's forward row
// pass (fft512_update_rows_fwd_kernel; for 1024-point rows, which take deferred
// correction updates only, fft1024_update_rows_fwd_kernel) instead of update_kernel.
inline bool fused_update(const LikelihoodState* L) {
  return L->fft && (fft512_rows(L->fd) || (fft1024_rows(L->fd) && pair_direction(L)));
}

// ---- launch-shape tuning of the FFT preconditioner
//
// Rows per block of the two row passes (rpb) and columns per block of the column
// pass (cw) trade shared memory, occupancy and the length of each block's work;
// the best pair depends on the padded size and the number of systems.  Measured
// once per (device, HP, WP, H, R) with CUDA events on the context's stream and
// cached for every later context of that shape.  Neither changes any result: a
// transform is computed the same way in any block shape, and the r.z partial sums
// are grouped by nbz, which is not tuned.
struct FftShape {
  int rpb, cw;
};
std::mutex g_tune_mu;
std::map<std::array<int, 5>, FftShape> g_tune;

float time_precond(LikelihoodState* L, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const int reps = 3;
  precond_apply(L, L->part + (size_t)L->R * L->nbmax, false, 0, nullptr, s);  // warm
  cudaEventRecord(e0, s);
  for (int i = 0; i < reps; ++i)
    precond_apply(L, L->part + (size_t)L->R * L->nbmax, false, 0, nullptr, s);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    return -1.f;
  return ms;
}

void tune_fft_shape(LikelihoodState* L, cudaStream_t s) {
  const char* env = getenv("EPTV_FFT_TUNE");
  if (env && env[0] == '0') return;
  FftDesc& f = L->fd;
  if ((fft512_rows(f) || fft1024_rows(f)) && (fft512_cols(f) || fft1024_cols(f)))
    return;  // the tuned shapes are not used
  int dev = 0;
  cudaGetDevice(&dev);
  const std::array<int, 5> key{dev, f.HP, f.WP, f.H, f.R};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      f.rpb = it->second.rpb;
      f.cw = it->second.cw;
      L->smem_rows = sizeof(float2) * ((size_t)f.WP + (size_t)f.rpb * f.WP);
      L->smem_cols = sizeof(float2) * ((size_t)f.HP + (size_t)f.HP * f.cw);
      return;
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // candidates: powers of two up to the shapes the plan allows (the defaults)
  const int rpb_max = f.rpb, cw_max = f.cw;
  auto set = [&](int rpb, int cw) {
    f.rpb = rpb;
    f.cw = cw;
    L->smem_rows = sizeof(float2) * ((size_t)f.WP + (size_t)rpb * f.WP);
    L->smem_cols = sizeof(float2) * ((size_t)f.HP + (size_t)f.HP * cw);
  };
  FftShape best{rpb_max, cw_max};
  float best_ms = time_precond(L, s, e0, e1);
  bool ok = best_ms >= 0.f;
  for (int cw = 1; ok && cw < cw_max; cw *= 2) {
    set(best.rpb, cw);
    const float ms = time_precond(L, s, e0, e1);
    if (ms < 0.f) ok = false;
    else if (ms < best_ms) { best_ms = ms; best.cw = cw; }
  }
  for (int rpb = 1; ok && rpb < rpb_max; rpb *= 2) {
    set(rpb, best.cw);
    const float ms = time_precond(L, s, e0, e1);
    if (ms < 0.f) ok = false;
    else if (ms < best_ms) { best_ms = ms; best.rpb = rpb; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) {  // keep the plan's shapes
    cudaGetLastError();
    best = FftShape{rpb_max, cw_max};
  }
  set(best.rpb, best.cw);
  if (L->debug)
    fprintf(stderr, "[eptv fft] HP %d WP %d H %d R %d: rpb %d (of %d) cw %d (of %d), %.3f ms / 3\n",
            f.HP, f.WP, f.H, f.R, best.rpb, rpb_max, best.cw, cw_max, best_ms);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
}

// E1 = H^T eps1 / sqrt(xi) from E1 holding eps1 (in place through Rr as scratch).
ep_tv_status finish_probes(LikelihoodState* L, cudaStream_t s) {
  const long long N = L->c.N;
  // Rr has R >= S planes: use it as scratch for the transform
  if (cudaMemcpyAsync(L->Rr, L->E1, sizeof(float) * L->S * N, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return EP_TV_ERR_CUDA;
  dim3 g(grid1d(N), L->S);
  conv_t_kernel<<<g, 256, 0, s>>>(L->Rr, L->E1, L->c.H, L->c.W, L->d_k, L->c.kh, L->c.kw,
                                  (float)std::sqrt((double)L->inv_xi), L->S);
  scale_kernel<<<grid1d((long long)L->S * N), 256, 0, s>>>(L->Y1, L->Rr, (long long)L->S * N,
                                                            (float)std::sqrt(1.0 / L->inv_xi));
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

}  // namespace

namespace {

// Raises the dynamic shared-memory limit of the solver kernels to the device's
// opt-in maximum minus their static shared memory (once per device).
bool raise_smem_limits() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return true;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const void* fns[] = {(const void*)direction_kernel, (const void*)residual_kernel,
                       (const void*)residual_pair_kernel<5>, (const void*)residual_pair_kernel<9>,
                       (const void*)residual_pair_kernel<15>,
                       (const void*)fft_rows_fwd_kernel, (const void*)fft_rows_inv_kernel,
                       (const void*)fft_cols_filter_kernel, (const void*)fft1024_cols_filter_kernel};
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess)
      return false;
  }
  done[dev] = true;
  return true;
}

}  // namespace

ep_tv_status likelihood_create(const LikelihoodConfig& cfg, cudaStream_t s, LikelihoodState** out,
                               float* mu0) {
  *out = nullptr;
  const ep_tv_operator* op = cfg.op;
  if (op->op == EP_TV_OP_DENSE || op->op == EP_TV_OP_HADAMARD) {
    LikelihoodState* L = new (std::nothrow) LikelihoodState();
    if (!L) return EP_TV_ERR_NOMEM;
    ep_tv_status st = cs_create(cfg, s, &L->cs, mu0);
    if (st != EP_TV_OK) {
      delete L;
      return st;
    }
    *out = L;
    return EP_TV_OK;
  }
  if (op->op != EP_TV_OP_CONV_PERIODIC) return EP_TV_ERR_UNSUPPORTED;
  if (op->kh > 2 * kMaxHalf / 2 + 1 || op->kw > 2 * kMaxHalf / 2 + 1) return EP_TV_ERR_UNSUPPORTED;
  LikelihoodState* L = new (std::nothrow) LikelihoodState();
  if (!L) return EP_TV_ERR_NOMEM;
  const int kh = op->kh, kw = op->kw;
  // host: kernel, autocorrelation factors, separability
  std::vector<double> k(kh * kw);
  double kmax = 0.0;
  int ai = 0, bi = 0;
  for (int i = 0; i < kh * kw; ++i) {
    k[i] = op->kernel[i];
    if (!std::isfinite(k[i])) { delete L; return EP_TV_ERR_ARG; }
    if (std::fabs(k[i]) > kmax) { kmax = std::fabs(k[i]); ai = i / kw; bi = i % kw; }
  }
  if (kmax == 0.0) { delete L; return EP_TV_ERR_ARG; }
  std::vector<double> u(kh), v(kw);
  for (int a = 0; a < kh; ++a) u[a] = k[a * kw + bi];
  for (int b = 0; b < kw; ++b) v[b] = k[ai * kw + b] / k[ai * kw + bi];
  bool sep = true;
  for (int a = 0; a < kh && sep; ++a)
    for (int b = 0; b < kw; ++b)
      if (std::fabs(k[a * kw + b] - u[a] * v[b]) > 1e-7 * kmax) { sep = false; break; }
  const int hr = kh - 1, hc = kw - 1;
  std::vector<float> g;
  double g0 = 0.0;
  for (int i = 0; i < kh * kw; ++i) g0 += k[i] * k[i];
  if (sep) {
    for (int a = -hr; a <= hr; ++a) {
      double acc = 0;
      for (int t = 0; t < kh; ++t)
        if (t + a >= 0 && t + a < kh) acc += u[t] * u[t + a];
      g.push_back((float)acc);
    }
    for (int b = -hc; b <= hc; ++b) {
      double acc = 0;
      for (int t = 0; t < kw; ++t)
        if (t + b >= 0 && t + b < kw) acc += v[t] * v[t + b];
      g.push_back((float)acc);
    }
  }
  L->S = cfg.p->rbmc_samples;
  L->R = 1 + L->S;
  L->inv_xi = (float)(1.0 / cfg.p->xi);
  L->rtol2 = cfg.p->cg_rtol * cfg.p->cg_rtol;
  L->rtol2_true = L->rtol2;
  // Probe solves: their right-hand sides are O(1/sqrt(xi)) noise whose residual
  // H^T (y' - H z) / xi + (n' - d z) cancels between two terms several times
  // larger, which puts their FP32 floor near 1e-7.  A relative residual of 1e-6
  // moves an RB variance term by about Q_ii / d * 1e-6 relative, below 1e-4.
  L->rtol2_probe = std::max(L->rtol2, 1e-12);
  L->max_iter = cfg.p->cg_max_iter;
  {
    const char* dbg = getenv("EPTV_DEBUG");
    L->debug = dbg && dbg[0] == '1';
  }
  L->seed = cfg.p->seed;
  L->damping = (float)cfg.p->damping;
  L->min_tau = (float)(1.0 / cfg.p->var_cap);
  ConvDesc& c = L->c;
  c.H = cfg.height;
  c.W = cfg.width;
  c.N = cfg.n;
  c.kh = kh;
  c.kw = kw;
  c.hr = hr;
  c.hc = hc;
  c.separable = sep ? 1 : 0;
  c.inv_xi = L->inv_xi;
  c.inv_xi_d = 1.0 / cfg.p->xi;
  c.g0_xi = (float)(g0 / cfg.p->xi);
  c.tiles_x = (c.W + kTile - 1) / kTile;
  c.tiles_y = (c.H + kTile - 1) / kTile;
  L->nb = c.tiles_x * c.tiles_y;
  // circulant preconditioner on the smallest power-of-two torus that holds the image
  // (padding keeps it symmetric positive definite: crop * C^-1 * pad)
  auto next_pow2 = [](int v) {
    int p2 = 2;
    while (p2 < v) p2 <<= 1;
    return p2;
  };
  const int HP = next_pow2(c.H), WP = next_pow2(c.W);
  L->fft = HP <= 8192 && WP <= 8192;
  L->nbz = L->nb;
  if (L->fft) {
    FftDesc& f = L->fd;
    f.H = c.H;
    f.W = c.W;
    f.HP = HP;
    f.WP = WP;
    f.R = L->R;
    f.pairs = (L->R + 1) / 2;
    // smallest radix of a length-n plan: 8 if log2 n is a multiple of 3, else 4 or 2
    auto rmin = [](int n) {
      const int logn = ilog2(n);
      return logn % 3 == 0 ? 8 : (logn % 3 == 2 ? 4 : 2);
    };
    // one pass handles at most kFftMaxItems * kFftThreads work items of n / R points
    const int cap = kFftMaxItems * kFftThreads;
    f.rpb = std::max(1, std::min({HP, 4096 / WP, cap * rmin(WP) / WP}));
    f.cw = std::max(1, std::min({WP, 16, cap * rmin(HP) / HP}));
    // r.z partials: one per block of the inverse row pass (kF512Warps * kRowsPerWarp512
    // rows each for 512-point rows)
    constexpr int kRowsInv512 = kF512Warps * kRowsPerWarp512;
    constexpr int kRowsInv1024 = kF512Warps * kRowsPerWarp1024;
    f.nbz = WP == kF       ? (c.H + kRowsInv512 - 1) / kRowsInv512
            : WP == 2 * kF ? (c.H + kRowsInv1024 - 1) / kRowsInv1024
                           : std::min(c.H, 64);
    L->nbz = f.nbz;
    L->smem_rows = sizeof(float2) * ((size_t)WP + (size_t)f.rpb * WP);
    L->smem_cols = sizeof(float2) * ((size_t)HP + (size_t)HP * f.cw);
  }
  L->nbmax = std::max(L->nb, L->nbz);
  L->prep_blocks = (int)std::min<long long>(std::max<long long>((c.N + 255) / 256, 1), 2048);
  const long long N = c.N;
  const size_t RN = (size_t)L->R * N;
  const size_t region = (size_t)(kTile + 2 * hr) * (kTile + 2 * hc);
  const size_t tmp = std::max((size_t)(kTile + 2 * hr) * kTile,
                              (size_t)(kTile + 2 * (kh / 2)) * (kTile + 2 * (kw / 2)));
  L->smem = sizeof(float) * (512 + region + tmp);
  {
    const size_t MH = kTile + 2 * (kh / 2), MW = kTile + 2 * (kw / 2);
    const size_t RH = kTile + 2 * hr, RW = kTile + 2 * hc;
    L->smem_res = sizeof(float) * (2 * RH * RW + (sep ? 2 * RH * MW : 0) + MH * MW +
                                   (sep ? MH * kTile : 0));
  }
  std::vector<float> kf(kh * kw);
  for (int i = 0; i < kh * kw; ++i) kf[i] = (float)k[i];
  bool ok = cudaMalloc(&L->d_k, sizeof(float) * kh * kw) == cudaSuccess &&
            cudaMalloc(&L->d_g, sizeof(float) * std::max<size_t>(g.size(), 1)) == cudaSuccess &&
            cudaMalloc(&L->Hty, sizeof(float) * N) == cudaSuccess &&
            cudaMalloc(&L->E1, sizeof(float) * L->S * N) == cudaSuccess &&
            cudaMalloc(&L->E2, sizeof(float) * L->S * N) == cudaSuccess &&
            cudaMalloc(&L->D, sizeof(float) * N) == cudaSuccess &&
            cudaMalloc(&L->Ncav, sizeof(float) * N) == cudaSuccess &&
            cudaMalloc(&L->Minv, sizeof(float) * N) == cudaSuccess &&
            cudaMalloc(&L->X, sizeof(double) * RN) == cudaSuccess &&
            cudaMalloc(&L->Y1, sizeof(float) * L->S * N) == cudaSuccess &&
            cudaMalloc(&L->thr, sizeof(double) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_hd, sizeof(double) * (kh * kw + kh + kw)) == cudaSuccess &&
            cudaMalloc(&L->d_hf, sizeof(float) * (kh * kw + kh + kw)) == cudaSuccess &&
            cudaMalloc(&L->Rr, sizeof(float) * RN) == cudaSuccess &&
            cudaMalloc(&L->P, sizeof(float) * RN) == cudaSuccess &&
            cudaMalloc(&L->P2, sizeof(float) * RN) == cudaSuccess &&
            cudaMalloc(&L->Qp, sizeof(float) * RN) == cudaSuccess &&
            cudaMalloc(&L->part, sizeof(double) * 4 * L->R * L->nbmax) == cudaSuccess &&
            cudaMalloc(&L->dpart, sizeof(double) * L->prep_blocks) == cudaSuccess &&
            cudaMalloc(&L->dbar, sizeof(double)) == cudaSuccess &&
            (!L->fft ||
             (cudaMalloc(&L->ftmp, sizeof(float2) * ((L->R + 1) / 2) * c.H * L->fd.WP) == cudaSuccess &&
              cudaMalloc(&L->Z, sizeof(float) * RN) == cudaSuccess &&
              cudaMalloc(&L->hth, sizeof(float) * L->fd.HP * L->fd.WP) == cudaSuccess &&
              cudaMalloc(&L->tw512, sizeof(float2) * 2 * kF) == cudaSuccess)) &&
            cudaMalloc(&L->d_active, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&L->d_relres, sizeof(double) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_prev_rr, sizeof(double) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_rr0, sizeof(double) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_scal, sizeof(float) * 4 * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_rzs, sizeof(double) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_arrive, sizeof(unsigned) * (L->R + (L->R + 1) / 2)) == cudaSuccess &&
            cudaMalloc(&L->d_act0, sizeof(int) * L->R) == cudaSuccess &&
            cudaMalloc(&L->d_loop, sizeof(LoopState)) == cudaSuccess &&
            cudaMalloc(&L->Ec, sizeof(float) * RN) == cudaSuccess &&
            cudaHostAlloc(&L->h_relres, sizeof(double) * L->R, cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc(&L->h_active, 2 * sizeof(int), cudaHostAllocDefault) == cudaSuccess &&
            cudaEventCreateWithFlags(&L->ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&L->ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    likelihood_destroy(L);
    return EP_TV_ERR_NOMEM;
  }
  // the block-arrival counters start at zero; every last block resets its own
  if (cudaMemsetAsync(L->d_arrive, 0, sizeof(unsigned) * (L->R + (L->R + 1) / 2), s) !=
      cudaSuccess) {
    likelihood_destroy(L);
    return EP_TV_ERR_CUDA;
  }
  c.k = L->d_k;
  c.gr = L->d_g;
  c.gc = L->d_g + (2 * hr + 1);
  c.hd = L->d_hd;
  c.hf = L->d_hf;
  L->Y0 = cfg.y;
  {
    std::vector<double> hd;
    if (sep) {
      hd.insert(hd.end(), u.begin(), u.end());
      hd.insert(hd.end(), v.begin(), v.end());
    } else {
      hd = k;
    }
    std::vector<float> hf(hd.begin(), hd.end());
    if (cudaMemcpyAsync(L->d_hd, hd.data(), sizeof(double) * hd.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(L->d_hf, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      likelihood_destroy(L);
      return EP_TV_ERR_CUDA;
    }
  }
  if (cudaMemcpyAsync(L->d_k, kf.data(), sizeof(float) * kh * kw, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      (sep && cudaMemcpyAsync(L->d_g, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice,
                              s) != cudaSuccess)) {
    likelihood_destroy(L);
    return EP_TV_ERR_CUDA;
  }
  // The dynamic shared-memory limit is a property of the kernel, shared by every
  // context: raise it once to what the device allows, never lower it per context.
  if (!raise_smem_limits()) {
    likelihood_destroy(L);
    return EP_TV_ERR_CUDA;
  }
  {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t need = std::max({L->smem + 8192, L->smem_res + 16384,
                                  L->fft ? std::max(L->smem_rows, L->smem_cols) + 1024 : (size_t)0});
    if (need > (size_t)optin) {
      likelihood_destroy(L);
      return EP_TV_ERR_UNSUPPORTED;
    }
  }
  if (L->fft) {
    L->fd.tmp = L->ftmp;
    L->fd.hth = L->hth;
    L->fd.tw512 = L->tw512;
    L->fd.tw1024 = L->tw512 + kF;
    tw512_kernel<<<(2 * kF + 255) / 256, 256, 0, s>>>(L->tw512);
    L->fd.dbar = L->dbar;
    hth_kernel<<<grid1d((long long)L->fd.HP * L->fd.WP), 256, 0, s>>>(
        L->hth, L->fd.HP, L->fd.WP, L->d_k, kh, kw, L->inv_xi,
        (fft512_cols(L->fd) || fft1024_cols(L->fd)) ? 1 : 0);
  }
  // H^T y / xi
  conv_t_kernel<<<dim3(grid1d(N), 1), 256, 0, s>>>(cfg.y, L->Hty, c.H, c.W, L->d_k, kh, kw,
                                                   L->inv_xi, 1);
  // Algorithm 1 initialises q_{x,0} at mean y (M = N here)
  if (cudaMemcpyAsync(mu0, cfg.y, sizeof(float) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    likelihood_destroy(L);
    return EP_TV_ERR_CUDA;
  }
  // library-drawn probes: eps1 then eps2 from one SplitMix64 counter stream
  normals_kernel<<<grid1d((long long)L->S * N), 256, 0, s>>>(L->E1, (long long)L->S * N, L->seed, 0);
  normals_kernel<<<grid1d((long long)L->S * N), 256, 0, s>>>(L->E2, (long long)L->S * N, L->seed,
                                                             (unsigned long long)L->S * N);
  ep_tv_status st = finish_probes(L, s);
  if (st != EP_TV_OK) {
    likelihood_destroy(L);
    return st;
  }
  if (L->fft) tune_fft_shape(L, s);
  if (cudaGetLastError() != cudaSuccess) {
    likelihood_destroy(L);
    return EP_TV_ERR_CUDA;
  }
  *out = L;
  return EP_TV_OK;
}

void likelihood_destroy(LikelihoodState* L) {
  if (!L) return;
  if (L->cs) cs_destroy(L->cs);
  cudaFree(L->d_k);
  cudaFree(L->d_g);
  cudaFree(L->Hty);
  cudaFree(L->E1);
  cudaFree(L->E2);
  cudaFree(L->D);
  cudaFree(L->Ncav);
  cudaFree(L->Minv);
  cudaFree(L->X);
  cudaFree(L->Y1);
  cudaFree(L->thr);
  cudaFree(L->d_hd);
  cudaFree(L->d_hf);
  cudaFree(L->Rr);
  cudaFree(L->P);
  cudaFree(L->P2);
  cudaFree(L->Qp);
  cudaFree(L->part);
  cudaFree(L->dpart);
  cudaFree(L->dbar);
  cudaFree(L->ftmp);
  cudaFree(L->tw512);
  cudaFree(L->Z);
  cudaFree(L->hth);
  cudaFree(L->d_active);
  cudaFree(L->d_relres);
  cudaFree(L->d_prev_rr);
  cudaFree(L->d_rr0);
  cudaFree(L->d_scal);
  cudaFree(L->d_rzs);
  cudaFree(L->d_arrive);
  cudaFree(L->d_act0);
  cudaFree(L->d_loop);
  for (auto& g : L->graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  cudaFree(L->Ec);
  if (L->h_relres) cudaFreeHost(L->h_relres);
  if (L->h_active) cudaFreeHost(L->h_active);
  if (L->ev[0]) cudaEventDestroy(L->ev[0]);
  if (L->ev[1]) cudaEventDestroy(L->ev[1]);
  delete L;
}

ep_tv_status likelihood_reset(LikelihoodState* L, cudaStream_t s) {
  if (L->cs) return EP_TV_OK;
  if (cudaMemsetAsync(L->X, 0, sizeof(double) * L->R * L->c.N, s) != cudaSuccess) return EP_TV_ERR_CUDA;
  L->last_iters = 0;
  return EP_TV_OK;
}

ep_tv_status likelihood_set_noise(LikelihoodState* L, const float* xi_m, cudaStream_t s) {
  if (!L->cs) return EP_TV_ERR_UNSUPPORTED;
  return cs_set_noise(L->cs, xi_m, s);
}

ep_tv_status likelihood_set_probes(LikelihoodState* L, const float* eps1, const float* eps2,
                                   int n_samples, cudaStream_t s) {
  if (L->cs || n_samples != L->S) return EP_TV_ERR_ARG;
  const long long N = L->c.N;
  if (cudaMemcpyAsync(L->E1, eps1, sizeof(float) * L->S * N, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(L->E2, eps2, sizeof(float) * L->S * N, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return EP_TV_ERR_CUDA;
  return finish_probes(L, s);
}

namespace {

// The likelihood-site update of likelihood_update below as one graph: the prior
// sites tp/np in, site 0 out; the refinement passes and the CG iterations are
// WHILE nodes, each pass an IF node (see LoopState).  Built by stream capture
// into the graph and its conditional bodies, one at a time; false if CUDA
// refuses any step (the caller then keeps the host-driven loop).
bool build_update_graph(LikelihoodState* L, float* tau, float* nu, const float* tp, const float* np,
                        unsigned* status, unsigned long long* counters, cudaStream_t s,
                        cudaGraphExec_t* out) {
  *out = nullptr;
  const ConvDesc& c = L->c;
  const long long N = c.N;
  CgArgs a = cg_args(L);
  a.counters = counters;
  a.it_dev = &L->d_loop->it;
  a.defer_e = fused_update(L) && pair_direction(L);
  const dim3 grid(c.tiles_x, c.tiles_y, L->R);
  const int groups = (L->S + kRbGroup - 1) / kRbGroup;
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle h_outer = 0, h_pass = 0, h_inner = 0;
  bool ok = cudaGraphConditionalHandleCreate(&h_outer, G, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h_pass, G, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h_inner, G, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  // a conditional node after the current capture dependencies of s; *body gets its graph
  auto add_cond = [&](cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                      cudaGraph_t* body) -> bool {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
      return false;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p) != cudaSuccess) return false;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies) == cudaSuccess;
  };
  auto capture = [&](cudaGraph_t g, auto&& launches) -> bool {
    if (cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      return false;
    const bool fine = launches();
    cudaGraph_t tmp = nullptr;
    const bool ended = cudaStreamEndCapture(s, &tmp) == cudaSuccess;
    return fine && ended && cudaGetLastError() == cudaSuccess;
  };
  cudaGraph_t b_outer = nullptr, b_pass = nullptr, b_inner = nullptr;
  ok = ok && capture(G, [&]() {
    prep_kernel<<<L->prep_blocks, kThreads, 0, s>>>(tp, np, N, c.g0_xi, L->D, L->Ncav, L->Minv,
                                                    L->dpart);
    mean_kernel<<<1, 1024, 0, s>>>(L->dpart, L->prep_blocks, 1.0 / (double)N, L->dbar);
    loop_init_kernel<<<1, 32, 0, s>>>(L->d_loop);
    if (!add_cond(h_outer, cudaGraphCondTypeWhile, &b_outer)) return false;
    loop_finish_kernel<<<1, 32, 0, s>>>(L->d_loop, status, counters);
    rb_offdiag_kernel<<<dim3(c.tiles_x, c.tiles_y, groups), kThreads, L->smem, s>>>(a, L->Qp);
    site0_kernel<<<grid1d(N), 256, 0, s>>>(a, L->Qp, groups, tau, nu, L->min_tau, L->damping,
                                           status, counters);
    return true;
  });
  ok = ok && capture(b_outer, [&]() {
    cond_clear_kernel<<<1, 32, 0, s>>>(h_outer);
    launch_residual(L, a, s);
    thresholds_kernel<<<1, 1024, 0, s>>>(a.part_rr, a.part_bb, a.part_rz, a.fft, L->R, L->nb,
                                         L->rtol2_true, L->rtol2_probe, kEta2, L->thr, L->d_relres,
                                         L->d_prev_rr, L->d_rr0, 0, &L->d_loop->outer, L->d_active,
                                         L->d_scal, L->d_act0, L->d_rzs);
    pass_kernel<<<1, 32, 0, s>>>(L->d_loop, L->d_active, L->max_outer, L->max_iter, h_outer, h_pass,
                                 h_inner);
    return add_cond(h_pass, cudaGraphCondTypeIf, &b_pass);
  });
  ok = ok && capture(b_pass, [&]() {
    if (L->fft) precond_apply(L, a.part_rz, true, 1, counters, s);
    if (!add_cond(h_inner, cudaGraphCondTypeWhile, &b_inner)) return false;
    commit_kernel<<<dim3(std::min(grid1d((N + 3) / 4), 1024), L->R), 256, 0, s>>>(
        L->X, L->Ec, L->d_act0, N, a.defer_e ? L->d_scal : nullptr, L->P, L->P2);
    return true;
  });
  // with the FFT preconditioner the column pass, which every iteration launches,
  // counts the iteration and sets the condition (0 or 1, and 0 once the budget is
  // spent); Jacobi keeps the clearing and counting kernels
  ok = ok && capture(b_inner, [&]() {
    if (!L->fft) cond_clear_kernel<<<1, 32, 0, s>>>(h_inner);
    launch_direction(L, a, 0, s);
    if (fused_update(L)) {
      precond_apply(L, a.part_rz, true, 0, counters, s, &a, 0, 3, true, h_inner);
    } else {
      update_kernel<<<grid, kUpdThreads, 0, s>>>(a, 0);
      if (L->fft) precond_apply(L, a.part_rz, true, 0, counters, s, nullptr, 0, 3, true, h_inner);
    }
    if (!L->fft) iter_kernel<<<1, 64, 0, s>>>(L->d_loop, L->d_scal, L->R, L->max_iter, h_inner);
    return true;
  });
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, G, 0) == cudaSuccess;
  cudaGraphDestroy(G);
  cudaGetLastError();
  *out = ok ? exec : nullptr;
  return ok;
}

}  // namespace

ep_tv_status likelihood_update(LikelihoodState* L, float* tau, float* nu, const float* tp,
                               const float* np, unsigned* status, unsigned long long* counters,
                               Tracer* tr, cudaStream_t s) {
  if (L->cs) return cs_update(L->cs, tau, nu, tp, np, status, counters, tr, s);
  // Graph replay: the whole update with device-driven loops, one launch.  Not with
  // tracing (which brackets every kernel launch) nor on the legacy default
  // stream (which cannot be captured).
  if (!tr->on && s != nullptr && !L->graph_failed) {
    int slot = L->graph[0].tp == tp ? 0 : (L->graph[1].tp == tp ? 1 : -1);
    if (slot < 0) {
      slot = L->graph[0].exec ? 1 : 0;
      if (L->graph[slot].exec) cudaGraphExecDestroy(L->graph[slot].exec);
      L->graph[slot].exec = nullptr;
      L->graph[slot].tp = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (build_update_graph(L, tau, nu, tp, np, status, counters, s, &exec)) {
        L->graph[slot].exec = exec;
        L->graph[slot].tp = tp;
      } else {
        L->graph_failed = true;
      }
    }
    if (!L->graph_failed) {
      if (cudaGraphLaunch(L->graph[slot].exec, s) != cudaSuccess) return EP_TV_ERR_CUDA;
      L->graph_last = true;
      return EP_TV_OK;
    }
  }
  L->graph_last = false;
  const ConvDesc& c = L->c;
  const long long N = c.N;
  prep_kernel<<<L->prep_blocks, kThreads, 0, s>>>(tp, np, N, c.g0_xi, L->D, L->Ncav, L->Minv,
                                                  L->dpart);
  mean_kernel<<<1, 1024, 0, s>>>(L->dpart, L->prep_blocks, 1.0 / (double)N, L->dbar);
  CgArgs a = cg_args(L);
  a.counters = counters;
  a.defer_e = fused_update(L) && pair_direction(L);
  dim3 grid(c.tiles_x, c.tiles_y, L->R);
  // Iterative refinement (see kEta2): true residual (float-float), then FP32
  // preconditioned CG on the correction, repeated until ||r|| <= rtol ||b||.
  const double eta2 = kEta2;
  int total = 0, iters = 0;
  bool converged = false;
  for (int outer = 0;; ++outer) {
    tr->begin(EP_TV_K_CG_RESIDUAL, s);
    launch_residual(L, a, s);
    tr->end(s, (double)L->R * N);
    thresholds_kernel<<<1, 1024, 0, s>>>(a.part_rr, a.part_bb, a.part_rz, a.fft, L->R, L->nb,
                                         L->rtol2_true, L->rtol2_probe, eta2, L->thr, L->d_relres,
                                         L->d_prev_rr, L->d_rr0, outer == 0, nullptr, L->d_active,
                                         L->d_scal, L->d_act0, L->d_rzs);
    if (cudaMemcpyAsync(L->h_active, L->d_active, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(L->h_relres, L->d_relres, sizeof(double) * L->R, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return EP_TV_ERR_CUDA;
    {
      double pm = 0.0;
      for (int jj = 1; jj < L->R; ++jj) pm = std::max(pm, L->h_relres[jj]);
      L->rep_mean = L->h_relres[0];
      L->rep_probe = pm;
      L->rep_outer = outer;
      if (L->debug)
        fprintf(stderr, "[eptv cg] outer %d inner-total %d relres mean %.3e probes max %.3e active %d\n",
                outer, total, L->rep_mean, pm, L->h_active[0]);
    }
    if (L->h_active[0] == 0) {
      converged = true;
      break;
    }
    if (outer >= L->max_outer || total >= L->max_iter) break;
    const int started = L->h_active[0];  // systems that iterate in this pass
    if (L->fft) {
      // z = M^{-1} r of the true residual: r.z of every active system, beta = 0
      tr->begin(EP_TV_K_CG_PRECOND, s);
      precond_apply(L, a.part_rz, true, 1, counters, s);
      tr->end(s, -1.0);
    }
    // Iterations run in chunks; the CG scalars (alpha, beta, active flags) are
    // formed on the device by the last block of each reduction, so a chunk needs
    // no host round trip.  The host reads the active count of a chunk while the
    // next one is already queued, and stops once it reaches zero.
    int launched = 0, pending = -1, slot = 0;
    while (true) {
      const int n = std::min(kChunk, L->max_iter - total - launched);
      for (int t = 0; t < n; ++t) {
        tr->begin(EP_TV_K_CG_DIRECTION, s);
        launch_direction(L, a, launched, s);
        tr->end(s, -1.0);
        if (fused_update(L)) {
          // the update with the preconditioner's forward row pass, then its other passes
          tr->begin(EP_TV_K_CG_UPDATE, s);
          precond_apply(L, a.part_rz, true, 0, counters, s, &a, launched, 1);
          tr->end(s, -1.0);
          tr->begin(EP_TV_K_CG_PRECOND, s);
          precond_apply(L, a.part_rz, true, 0, counters, s, nullptr, 0, 2);
          tr->end(s, -1.0);
        } else {
          tr->begin(EP_TV_K_CG_UPDATE, s);
          update_kernel<<<grid, kUpdThreads, 0, s>>>(a, launched);
          tr->end(s, -1.0);
          if (L->fft) {
            tr->begin(EP_TV_K_CG_PRECOND, s);
            precond_apply(L, a.part_rz, true, 0, counters, s);
            tr->end(s, -1.0);
          }
        }
        ++launched;
      }
      check_kernel<<<1, 64, 0, s>>>(L->d_scal, L->R, L->d_active);
      if (cudaMemcpyAsync(L->h_active + slot, L->d_active, sizeof(int), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaEventRecord(L->ev[slot], s) != cudaSuccess)
        return EP_TV_ERR_CUDA;
      if (pending >= 0) {
        if (cudaEventSynchronize(L->ev[pending & 1]) != cudaSuccess) return EP_TV_ERR_CUDA;
        if (L->h_active[pending & 1] == 0) break;
      }
      pending = (launched << 1) | slot;
      slot ^= 1;
      if (n == 0 || total + launched >= L->max_iter) {
        if (cudaEventSynchronize(L->ev[pending & 1]) != cudaSuccess) return EP_TV_ERR_CUDA;
        break;
      }
    }
    // the corrections of every launched iteration are final: add them to the FP64
    // solutions of the systems that iterated, then count the iterations up to the
    // poll that found all systems stopped
    tr->begin(EP_TV_K_CG_COMMIT, s);
    commit_kernel<<<dim3(std::min(grid1d((N + 3) / 4), 1024), L->R), 256, 0, s>>>(
        L->X, L->Ec, L->d_act0, N, a.defer_e ? L->d_scal : nullptr, L->P, L->P2);
    tr->end(s, (double)started * N);
    total += launched;
  }
  iters = total;
  const bool ran_out = !converged;
  L->last_iters = iters;
  if (ran_out) set_status_kernel<<<1, 1, 0, s>>>(status, ST_CG_NOCONV);
  store_iters_kernel<<<1, 1, 0, s>>>(counters, (unsigned long long)iters);
  tr->begin(EP_TV_K_SITE0, s);
  // Q p is free once the solves have finished: it holds the RB sums
  const int groups = (L->S + kRbGroup - 1) / kRbGroup;
  rb_offdiag_kernel<<<dim3(c.tiles_x, c.tiles_y, groups), kThreads, L->smem, s>>>(a, L->Qp);
  site0_kernel<<<grid1d(N), 256, 0, s>>>(a, L->Qp, groups, tau, nu, L->min_tau, L->damping, status,
                                         counters);
  tr->end(s, (double)N);
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

// What each kernel class must move at least once per unit (the method's data,
// not the implementation's intermediates), for the roofline.
double likelihood_bytes_per_unit(const LikelihoodState* L, int kernel) {
  if (L->cs) return kernel == EP_TV_K_CS ? cs_flops(L->cs) : kernel == EP_TV_K_CS_MMA ? 1.0 : 0.0;
  const double groups = (double)((L->S + kRbGroup - 1) / kRbGroup);
  // with deferred correction updates the direction kernel also does e += alpha p
  // (read and write e; p is the direction it reads anyway) and the update only r
  const bool defer = fused_update(L) && pair_direction(L);
  switch (kernel) {
    case EP_TV_K_CG_DIRECTION:               // read z, p; write p, Q p (per active system
      return defer ? 24.0 : 16.0;            // pixel); deferred: also read and write e
    case EP_TV_K_CG_UPDATE:                  // read e, r, p, Q p; write e, r (FP32
      return defer ? 12.0 : 24.0;            // correction); deferred: read r, Q p, write r
    case EP_TV_K_CG_RESIDUAL: return 24.0;   // read x (FP64), y', the probe planes; write r
    case EP_TV_K_CG_PRECOND: return 8.0;     // r in, z out (per transformed system pixel)
    case EP_TV_K_CG_COMMIT: return 20.0;     // read x (FP64) and e, write x (per committed
                                             // system pixel)
    case EP_TV_K_SITE0:                      // read the S probe solutions (FP64), write and
      return 8.0 * L->S + 8.0 * groups       // read the RB sums, read x_0 (FP64), d, n, Minv,
             + 36.0;                         // tau0, nu0; write tau0, nu0 (per pixel)
  }
  return 0.0;
}

int likelihood_systems(const LikelihoodState* L) { return L->R; }

// After a graph replay the counts and residuals live in device memory only
// (the callers have synchronised the context's stream).
bool likelihood_graph_last(const LikelihoodState* L) { return !L->cs && L->graph_last; }

int likelihood_last_iters(const LikelihoodState* L) {
  if (L->cs || !L->graph_last) return L->last_iters;
  LoopState ls;
  if (cudaMemcpy(&ls, L->d_loop, sizeof(ls), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return ls.total;
}

void likelihood_report(const LikelihoodState* L, int* outer, double* relres_mean,
                       double* relres_probe) {
  int o = L->rep_outer;
  double rm = L->rep_mean, rp = L->rep_probe;
  if (!L->cs && L->graph_last) {
    LoopState ls;
    std::vector<double> rel(L->R);
    if (cudaMemcpy(&ls, L->d_loop, sizeof(ls), cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(rel.data(), L->d_relres, sizeof(double) * L->R, cudaMemcpyDeviceToHost) ==
            cudaSuccess) {
      o = ls.outer;
      rm = rel[0];
      rp = 0.0;
      for (int j = 1; j < L->R; ++j) rp = std::max(rp, rel[j]);
    }
  }
  if (outer) *outer = o;
  if (relres_mean) *relres_mean = rm;
  if (relres_probe) *relres_probe = rp;
}

size_t likelihood_state_bytes(const LikelihoodState* L) {
  if (L->cs) return 0;
  return sizeof(double) * (size_t)L->R * L->c.N;
}

ep_tv_status likelihood_state_export(LikelihoodState* L, void* host, cudaStream_t s) {
  if (L->cs) return EP_TV_OK;
  return cudaMemcpyAsync(host, L->X, likelihood_state_bytes(L), cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess
             ? EP_TV_OK
             : EP_TV_ERR_CUDA;
}

ep_tv_status likelihood_state_import(LikelihoodState* L, const void* host, cudaStream_t s) {
  if (L->cs) return EP_TV_OK;
  return cudaMemcpyAsync(L->X, host, likelihood_state_bytes(L), cudaMemcpyHostToDevice, s) ==
                 cudaSuccess
             ? EP_TV_OK
             : EP_TV_ERR_CUDA;
}

}  // namespace eptv
