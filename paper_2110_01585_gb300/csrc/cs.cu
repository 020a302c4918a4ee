// Likelihood site q_{x,0} for a dense sensing matrix A (compressive sensing).
//
// Eq. tilted_P_1 with H = A (M x N, M < N): A^T A is low rank, and the paper takes
// the Woodbury identity (Sec. III-C).  With C = diag(c), c the cavity variances of
// site 0 (1 / sum_k tau_k) and m the cavity means,
//   K = xi I_M + A C A^T = L L^T,   W = L^{-1} A,   w_i = sum_m W_mi^2 = a_i^T K^{-1} a_i,
//   Var_i = c_i - c_i^2 w_i,        E = m + C A^T K^{-1} (y - A m) = m + c * W^T L^{-1}(y - A m).
// The site update of Eq. update_q0_x then needs 1/Var_i - 1/c_i = w_i / (1 - c_i w_i).
//
// Precision: all of it is FP64-accurate.  c spans 1e-2 .. 1e8 (prior sites at
// their variance cap), which drives cond(K) to 1e7 .. 1e8 within a few sweeps and
// c_i w_i to within 1e-4 of 1; an FP32 or plain BF16 factorisation loses every
// digit of 1 - c_i w_i there.  GB300's FP64 rate is low (1.25 TFLOP/s), so the
// large products run as exact BF16 slice products on the tensor cores instead.
//
// Subsampled 2-D Hadamard operator (Sec. II-A (iii)): A = S W / sqrt(M), W the
// N x N Walsh-Hadamard matrix in Sylvester order (entry (a, b) = (-1)^popcount(a & b),
// the Kronecker product of the row and column matrices), S the M selected rows
// s_1..s_M.  Walsh functions multiply by XOR of their indices, so
//   K[m, m'] = xi delta + (1/M) sum_i W[s_m, i] W[s_m', i] c_i = xi delta + (W c)[s_m ^ s_m'] / M:
// one fast transform of c and a gather form K, with no GEMM.  And
//   W_A = L^{-1} A = (L^{-1} S) W / sqrt(M):
// the triangular inverse L^{-1} scattered to the selected columns, then one fast
// transform per row, in place of the M x N triangular solve.  The mean uses
// A m = (W m)[s] / sqrt(M) and W_A^T.  Same FP64 precision as the dense path.
//
// Structure of one update.  The products with A (K = A C A^T and W = L^{-1} A =
// Z A, Z = L^{-1}) run on the BF16 tensor cores in the FP64-accurate split form of
// ozaki.cu.  K = L L^T and Z = L^{-1} come together from a recursion on halves
// (L21 = K21 Z11^T, K22 -= L21 L21^T, Z21 = -Z22 L21 Z11) whose large products
// run in the same split form with 10 digit slices and seven exact diagonals (as
// accurate as FP64 on these operands); blocks of 64 rows and smaller products
// stay on the FP64 CUDA cores.  The mean uses v = Z t and g = W^T v.
//
// Kernels here: an FP64 tiled GEMM (64 x 64 tiles, 4 x 4 per thread) for the
// small products; the Cholesky factor and inverse of one block of at most 64 rows
// in shared memory; column sums; matrix-vector products; the fast Walsh-Hadamard
// transform and the gathers of the Hadamard operator.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "internal.cuh"
#include "likelihood.cuh"
#include "ozaki.cuh"

namespace eptv {

namespace {

constexpr int kNb = 64;      // Cholesky / triangular-solve block size
constexpr int kGt = 64;      // GEMM tile
constexpr int kGk = 16;      // GEMM k step

// C[i, j] = alpha * C[i, j] + beta_ * sum_k A[i, k] * B(k, j) for a tile of
// (m x n); B(k, j) = B[j * ldb + k] (transposed, "NT") or B[k * ldb + j] ("NN").
// lower_only: skip tiles strictly above the diagonal (C symmetric).  a_lower: A
// is lower triangular; b_lower: the matrix stored in B is lower triangular.  A
// tile then skips the range of k where every product is zero (the sums of the
// remaining terms are formed in the same order, so the result does not change).
template <bool kNT>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int m, int n, int k, const double* A, int lda,
                                                       const double* B, int ldb, double* C, int ldc,
                                                       double alpha, double beta_, int lower_only, int a_lower,
                                                       int b_lower) {
  const int bi = blockIdx.y * kGt, bj = blockIdx.x * kGt;
  if (lower_only && bj > bi + kGt - 1) return;
  __shared__ double As[kGk][kGt + 1];
  __shared__ double Bs[kGk][kGt + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 each
  double acc[4][4] = {};
  int k_lo = 0, k_hi = k;
  if (a_lower) k_hi = min(k_hi, bi + kGt);                     // A(i, kk) = 0 for kk > i
  if (b_lower && kNT) k_hi = min(k_hi, bj + kGt);              // B(kk, j) = B_jkk = 0 for kk > j
  if (b_lower && !kNT) k_lo = bj / kGk * kGk;                  // B(kk, j) = B_kkj = 0 for kk < j
  for (int k0 = k_lo; k0 < k_hi; k0 += kGk) {
    // A tile: rows bi..bi+63, cols k0..k0+15
    for (int e = threadIdx.x; e < kGt * kGk; e += 256) {
      const int r = e / kGk, kk = e - r * kGk;
      const int gi = bi + r, gk = k0 + kk;
      As[kk][r] = (gi < m && gk < k) ? A[(long long)gi * lda + gk] : 0.0;
    }
    for (int e = threadIdx.x; e < kGt * kGk; e += 256) {
      int r, kk;
      if (kNT) {
        r = e / kGk;
        kk = e - r * kGk;
      } else {
        kk = e / kGt;
        r = e - kk * kGt;
      }
      const int gj = bj + r, gk = k0 + kk;
      double v = 0.0;
      if (gj < n && gk < k) v = kNT ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj];
      Bs[kk][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGk; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = bi + ty * 4 + u;
    if (gi >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gj = bj + tx * 4 + v;
      if (gj >= n) continue;
      double* cp = C + (long long)gi * ldc + gj;
      *cp = alpha == 0.0 ? beta_ * acc[u][v] : alpha * *cp + beta_ * acc[u][v];
    }
  }
}

// K = 0, then the diagonal gets the noise covariance: xi, or xi_v[i] for a
// diagonal (non-i.i.d.) noise covariance (the product adds G G^T with beta = 1).
__global__ void init_k_kernel(double* K, int M, double xi, const double* xi_v) {
  const long long total = (long long)M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e - (long long)i * M);
    K[e] = i == j ? (xi_v ? xi_v[i] : xi) : 0.0;
  }
}

__global__ void f32_to_f64_kernel(const float* in, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

// In-place Cholesky of the diagonal block K[k0:k0+b, k0:k0+b] (b <= 64), one block
// of threads, in shared memory; writes L (lower) back.  A non-positive pivot (K not
// numerically positive definite) raises the non-finite status bit.
__global__ void potrf_block_kernel(double* K, int ldk, int k0, int b, unsigned* status) {
  __shared__ double S[kNb][kNb + 1];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    S[i][j] = K[(long long)(k0 + i) * ldk + k0 + j];
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      const double d = S[j][j];
      if (!(d > 0.0)) atomicOr(status, ST_NONFINITE);
      S[j][j] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double djj = S[j][j];
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) S[i][j] /= djj;
    __syncthreads();
    // trailing update of the block
    for (int e = threadIdx.x; e < (b - j - 1) * (b - j - 1); e += blockDim.x) {
      const int i = j + 1 + e / (b - j - 1), l = j + 1 + e % (b - j - 1);
      if (l <= i) S[i][l] -= S[i][j] * S[l][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    K[(long long)(k0 + i) * ldk + k0 + j] = j <= i ? S[i][j] : 0.0;
  }
}

// w[i] = sum_m W[m, i]^2 (column sums, FP64)
__global__ void colsq_kernel(const double* W, int M, int N, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int m = 0; m < M; ++m) {
    const double v = W[(long long)m * N + i];
    s = fma(v, v, s);
  }
  w[i] = s;
}

// t = y - A m  (one warp per row)
__global__ void resid_vec_kernel(const float* A, const float* y, const double* m, int M, int N,
                                 double* t) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  double s = 0.0;
  for (int i = lane; i < N; i += 32) s = fma((double)A[(long long)row * N + i], m[i], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) t[row] = (double)y[row] - s;
}

// g = W^T v  (one thread per column)
__global__ void wtv_kernel(const double* W, const double* v, int M, int N, double* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int m = 0; m < M; ++m) s = fma(W[(long long)m * N + i], v[m], s);
  g[i] = s;
}

// Cavity of site 0 from the prior sites: d = sum tau_k, n = sum nu_k; c = 1/d, m = n/d.
__global__ void cs_cavity_kernel(const float* tp, const float* np, long long N, double* c,
                                 double* sqc, double* m) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const double d = (double)tp[p] + tp[N + p] + tp[2 * N + p] + tp[3 * N + p];
    const double n = (double)np[p] + np[N + p] + np[2 * N + p] + np[3 * N + p];
    c[p] = 1.0 / d;
    sqc[p] = sqrt(1.0 / d);
    m[p] = n / d;
  }
}

// Eq. update_q0_x: tau = w / (1 - c w) (= 1/Var - 1/c), cap, nu = tau E + (E - m)/c, damp.
__global__ void cs_site0_kernel(const double* w, const double* g, const double* c, const double* m,
                                long long N, float* tau0, float* nu0, float min_tau, float damping,
                                unsigned* status, unsigned long long* counters) {
  unsigned capped = 0;
  bool bad = false;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const double ci = c[p];
    const double E = m[p] + ci * g[p];
    double tn = w[p] / (1.0 - ci * w[p]);
    if (!(tn >= (double)min_tau)) {
      tn = min_tau;
      ++capped;
    }
    const double nn = tn * E + (E - m[p]) / ci;
    const float t_new = (float)(damping * tn + (1.0 - damping) * (double)tau0[p]);
    const float n_new = (float)(damping * nn + (1.0 - damping) * (double)nu0[p]);
    tau0[p] = t_new;
    nu0[p] = n_new;
    bad |= !(isfinite(t_new) && isfinite(n_new));
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  if (capped) atomicAdd(&counters[DC_CAPPED], (unsigned long long)capped);
}

// ---- Hadamard operator
//
// Fast Walsh-Hadamard transform (Sylvester order, unnormalised) of rows of n
// doubles, n a power of two: one row per block in shared memory (n <= 16384), the
// butterflies (a, b) -> (a + b, a - b) at strides 1, 2, 4, ...
constexpr int kFwhtThreads = 1024;
constexpr int kFwhtMaxSmem = 16384;

__global__ void __launch_bounds__(kFwhtThreads) fwht_rows_smem_kernel(double* rows, int n) {
  extern __shared__ double v[];
  double* row = rows + (long long)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = row[i];
  __syncthreads();
  for (int h = 1; h < n; h <<= 1) {
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int i = (t / h) * 2 * h + (t % h), j = i + h;
      const double a = v[i], b = v[j];
      v[i] = a + b;
      v[j] = a - b;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = v[i];
}

// One butterfly stage (stride h) over rows rows of n doubles in global memory.
__global__ void fwht_stage_kernel(double* rows, int n, int h, long long pairs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pairs;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / (n / 2);
    const int t = (int)(e - r * (n / 2));
    const int i = (t / h) * 2 * h + (t % h);
    double* row = rows + r * n;
    const double a = row[i], b = row[i + h];
    row[i] = a + b;
    row[i + h] = a - b;
  }
}

// K = diag(xi) + (W c)[s_m ^ s_m'] / M, from wc = W c.
__global__ void hadamard_k_kernel(double* K, int M, const int* sel, const double* wc, double xi,
                                  const double* xi_v) {
  const long long total = (long long)M * M;
  const double inv_m = 1.0 / (double)M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e - (long long)i * M);
    double v = wc[sel[i] ^ sel[j]] * inv_m;
    if (i == j) v += xi_v ? xi_v[i] : xi;
    K[e] = v;
  }
}

// G = 0, then G[m, s_j] = Z[m, j] / sqrt(M) for the lower triangle of Z (L^{-1} is lower).
__global__ void hadamard_scatter_kernel(const double* Z, int M, const int* sel, double* G, int N) {
  const long long total = (long long)M * M;
  const double scale = 1.0 / sqrt((double)M);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e - (long long)i * M);
    if (j <= i) G[(long long)i * N + sel[j]] = Z[e] * scale;
  }
}

// t = y - (W m)[s] / sqrt(M), from wm = W m.
__global__ void hadamard_resid_kernel(const float* y, const double* wm, const int* sel, int M,
                                      double* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) t[i] = (double)y[i] - wm[sel[i]] / sqrt((double)M);
}

// v[s_m] = y_m (v zeroed before): the input of the back-projection A^T y.
__global__ void hadamard_place_kernel(const float* y, const int* sel, int M, double* v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) v[sel[i]] = (double)y[i];
}
__global__ void to_f32_scaled_kernel(const double* in, float* out, int n, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(in[i] * scale);
}

// mu0 = A^T y (one thread per column, FP64 accumulation)
__global__ void aty_kernel(const float* A, const float* y, int M, int N, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int m = 0; m < M; ++m) s = fma((double)A[(long long)m * N + i], (double)y[m], s);
  out[i] = (float)s;
}

// Z = L^{-1} for the n x n (n <= 64) lower block L (leading dimension ld), zeros
// above the diagonal; forward substitution on the unit vectors, one thread per
// column (each thread reads back only the entries of Z it wrote itself).
__global__ void trinv_block_kernel(const double* L, long long ld, double* Z, long long ldz, int n) {
  __shared__ double Ls[kNb][kNb + 1];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    Ls[i][j] = j <= i ? L[(long long)i * ld + j] : 0.0;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= n) return;
  for (int i = 0; i < n; ++i) {
    double z = 0.0;
    if (i >= j) {
      double v = i == j ? 1.0 : 0.0;
      for (int l = j; l < i; ++l) v -= Ls[i][l] * Z[(long long)l * ldz + j];
      z = v / Ls[i][i];
    }
    Z[(long long)i * ldz + j] = z;
  }
}

// v = Z t for lower-triangular Z (M x M), one warp per row.
__global__ void trmv_lower_kernel(const double* Z, int M, const double* t, double* v) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  double acc = 0.0;
  for (int k = lane; k <= row; k += 32) acc = fma(Z[(long long)row * M + k], t[k], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) v[row] = acc;
}

inline int g1d(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 1 << 20);
}

// Unnormalised fast Walsh-Hadamard transform of nrows contiguous rows of n doubles:
// the strides below kFwhtMaxSmem in shared memory (one block per chunk of that
// length; the chunks tile every row), the larger strides one global pass each.
void fwht_rows(double* rows, long long nrows, int n, cudaStream_t s) {
  if (n < 2 || nrows < 1) return;
  const int chunk = std::min(n, kFwhtMaxSmem);
  const int threads = std::min(kFwhtThreads, std::max(32, chunk / 2));
  fwht_rows_smem_kernel<<<(unsigned)(nrows * (n / chunk)), threads, sizeof(double) * chunk, s>>>(
      rows, chunk);
  const long long pairs = nrows * (n / 2);
  for (int h = chunk; h < n; h <<= 1) fwht_stage_kernel<<<g1d(pairs), 256, 0, s>>>(rows, n, h, pairs);
}

void gemm(bool nt, int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
          int ldc, double alpha, double beta_, bool lower_only, cudaStream_t s, bool a_lower = false,
          bool b_lower = false) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  dim3 grid((n + kGt - 1) / kGt, (m + kGt - 1) / kGt);
  if (nt)
    gemm_f64_kernel<true><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, alpha, beta_,
                                               lower_only ? 1 : 0, a_lower ? 1 : 0, b_lower ? 1 : 0);
  else
    gemm_f64_kernel<false><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, alpha, beta_,
                                                lower_only ? 1 : 0, a_lower ? 1 : 0, b_lower ? 1 : 0);
}

}  // namespace

struct CsState {
  int M = 0, N = 0;
  bool hadamard = false;      // subsampled Hadamard rows in place of the dense matrix
  double xi = 0.0;
  float damping = 0.5f, min_tau = 1e-8f;
  const float* A = nullptr;   // borrowed, M x N FP32
  const float* y = nullptr;   // context copy
  double* G = nullptr;        // M x N: W = L^{-1} A
  double* K = nullptr;        // M x M: K, overwritten by the factorisation
  double* Z = nullptr;        // M x M: L^{-1} (lower)
  double* pool = nullptr;     // M x M: L21 and L21 Z11 blocks of the recursion
  double* c = nullptr;
  double* sqc = nullptr;
  double* m = nullptr;
  double* w = nullptr;
  double* g = nullptr;
  double* t = nullptr;        // M
  double* v = nullptr;        // M
  double* xi_v = nullptr;     // M noise variances (diagonal noise covariance), or NULL
  int* sel = nullptr;         // Hadamard: M Sylvester row indices
  // split-BF16 tensor-core products: packed operands and their row exponents
  uint8_t* pack_a = nullptr;  // left operands: G, Z, the factorisation's blocks
  uint8_t* pack_b = nullptr;  // right operands: G of G G^T, the factorisation's blocks
  uint8_t* pack_at = nullptr; // dense: A^T, packed once
  int* exp_a = nullptr;
  int* exp_b = nullptr;
  int* exp_at = nullptr;
  unsigned* status = nullptr; // the context's status word (set per update)
  Tracer* tr = nullptr;       // the context's tracer (set per update)
  double simt_flops = 0.0;    // FP64 CUDA-core flops of one update (counted on the host)
  double mma_flops = 0.0;     // BF16 tensor flops of one update
};

namespace {

void cs_free(CsState* S) {
  cudaFree(S->G);
  cudaFree(S->K);
  cudaFree(S->Z);
  cudaFree(S->pool);
  cudaFree(S->c);
  cudaFree(S->sqc);
  cudaFree(S->m);
  cudaFree(S->w);
  cudaFree(S->g);
  cudaFree(S->t);
  cudaFree(S->v);
  cudaFree(S->xi_v);
  cudaFree(S->sel);
  cudaFree(S->pack_a);
  cudaFree(S->pack_b);
  cudaFree(S->pack_at);
  cudaFree(S->exp_a);
  cudaFree(S->exp_b);
  cudaFree(S->exp_at);
  delete S;
}

// The tracer brackets the update as CS segments with the tensor-core products
// cut out as CS_MMA segments.
struct Segment {
  CsState* S;
  cudaStream_t s;
  double flops;
  Segment(CsState* S_, cudaStream_t s_, double flops_) : S(S_), s(s_), flops(flops_) {
    S->tr->end(s, 0.0);
    S->tr->begin(EP_TV_K_CS_MMA, s);
  }
  ~Segment() {
    S->tr->end(s, flops);
    S->tr->begin(EP_TV_K_CS, s);
  }
};

// Products of the factorisation at least this large in every dimension run on the
// tensor cores; smaller ones in the FP64 SIMT GEMM.
constexpr int kMmaMin = 64;
// Digit slices of the factorisation's products.  The Schur complement
// K22 - L21 L21^T cancels to the size of xi while its terms carry the capped
// cavity variances, and the split form's error is relative to the rows' largest
// entries.  With the operator products' form (8 slices, FP32 tail from s + t = 7)
// the Hadamard 128^2 case missed parity by 100x; the error was the tail's FP32
// accumulation (10 slices alone changed nothing; a tail from s + t = 8 cut it 70x).
// 10 slices with seven exact diagonals (tail from s + t = 9) reproduce the FP64
// factorisation's parity errors to four digits on every case.
constexpr int kFactorSlices = 10;
constexpr int kFactorMaxK = 8192;  // the 10-slice product's integer accumulators hold k <= 8192

// C = alpha C + beta X Y^T, X (m x k) row-major at ldx, Y(j, kk) = Y[j * ldy + kk]
// or, when y_trans, Y[kk * ldy + j]; x_lower / y_lower: the stored X / Y is lower
// triangular (the SIMT GEMM skips the zero products; the split product stops a
// row tile of a triangular X at its diagonal).  same: Y is X.
void product(CsState* S, const double* X, long long ldx, bool x_lower, const double* Y, long long ldy,
             bool y_trans, bool y_lower, bool same, int m, int n, int k, double* C, long long ldc, double alpha,
             double beta, bool lower_only, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  if (std::min(m, n) < kMmaMin || k < kMmaMin || k > kFactorMaxK) {
    gemm(!y_trans, m, n, k, X, (int)ldx, Y, (int)ldy, C, (int)ldc, alpha, beta, lower_only, s, x_lower,
         y_lower);
    S->simt_flops += (x_lower || y_lower ? 1.0 : 2.0) * m * n * k;  // a triangle halves the products
    return;
  }
  const int sl = kFactorSlices;
  const double f = ozaki_tensor_flops(m, n, k, sl) * (x_lower || lower_only ? 0.5 : 1.0);
  S->mma_flops += f;
  Segment seg(S, s, f);
  ozaki_pack(X, ldx, false, m, k, nullptr, S->exp_a, S->pack_a, OzakiSide::kLeft, true, s, sl);
  if (same)
    ozaki_pack(X, ldx, false, m, k, nullptr, S->exp_a, S->pack_b, OzakiSide::kRight, false, s, sl);
  else
    ozaki_pack(Y, ldy, y_trans, n, k, nullptr, S->exp_b, S->pack_b, OzakiSide::kRight, true, s, sl);
  ozaki_gemm(OzakiOperand{S->pack_a, S->exp_a, sl}, OzakiOperand{S->pack_b, same ? S->exp_a : S->exp_b, sl}, k,
             C, ldc, m, n, alpha, beta, lower_only, x_lower, S->status, s);
}

int split_point(int n) {
  const int half = (n + 1) / 2;
  return (half + kNb - 1) / kNb * kNb;
}

// Cholesky factorisation and triangular inverse together, by halves: for
// K = [K11 .; K21 K22] (lower triangle read),
//   L11 Z11 from K11;  L21 = K21 Z11^T;  K22 <- K22 - L21 L21^T;  L22 Z22 from K22;
//   Z21 = -Z22 (L21 Z11),
// with Z = L^{-1} written into Z (ldz; the block above the diagonal must be zero
// already).  Blocks of at most 64 rows: shared-memory Cholesky and inverse.
// The recursion exposes large FP64 products (the top level's are n/2 square)
// where a column-by-column factorisation has only 64-row panels.
// pool: scratch for the L21 and L21 Z11 blocks of every level.
void chol_inv(CsState* S, double* K, long long ld, double* Z, long long ldz, int n, double* pool,
              cudaStream_t s) {
  if (n <= kNb) {
    potrf_block_kernel<<<1, 256, 0, s>>>(K, (int)ld, 0, n, S->status);
    trinv_block_kernel<<<1, kNb, 0, s>>>(K, ld, Z, ldz, n);
    S->simt_flops += 2.0 * n * n * n / 3.0;
    return;
  }
  const int n1 = split_point(n), n2 = n - n1;
  double* K21 = K + (long long)n1 * ld;
  double* K22 = K21 + n1;
  double* Z21 = Z + (long long)n1 * ldz;
  double* Z22 = Z21 + n1;
  chol_inv(S, K, ld, Z, ldz, n1, pool, s);
  double* L21 = pool;                       // n2 x n1
  double* T = pool + (long long)n2 * n1;    // n2 x n1
  double* rest = T + (long long)n2 * n1;
  product(S, K21, ld, false, Z, ldz, false, true, false, n2, n1, n1, L21, n1, 0.0, 1.0, false, s);
  product(S, L21, n1, false, L21, n1, false, false, true, n2, n2, n1, K22, ld, 1.0, -1.0, true, s);
  chol_inv(S, K22, ld, Z22, ldz, n2, rest, s);
  product(S, L21, n1, false, Z, ldz, true, true, false, n2, n1, n1, T, n1, 0.0, 1.0, false, s);
  product(S, Z22, ldz, true, T, n1, true, false, false, n2, n1, n2, Z21, ldz, 0.0, -1.0, false, s);
}

unsigned bit_reverse(unsigned k, int bits) {
  unsigned out = 0;
  for (int i = 0; i < bits; ++i)
    if (k >> i & 1u) out |= 1u << (bits - 1 - i);
  return out;
}

int log2_exact(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return (1 << b) == v ? b : -1;
}

// Buffers of both operators.
bool alloc_common(CsState* S) {
  const int M = S->M, N = S->N;
  const long long MN = (long long)M * N, MM = (long long)M * M;
  // left operands: G (M x N, dense operator), Z (M x M) and the factorisation's blocks;
  // right operands: G (dense) and the factorisation's blocks
  const size_t fac = ozaki_pack_bytes(M, M, kFactorSlices);
  const size_t pa = std::max(S->hadamard ? 0 : ozaki_pack_bytes(M, N), fac);
  return cudaMalloc(&S->G, sizeof(double) * MN) == cudaSuccess &&
         cudaMalloc(&S->K, sizeof(double) * MM) == cudaSuccess &&
         cudaMalloc(&S->Z, sizeof(double) * MM) == cudaSuccess &&
         cudaMalloc(&S->pool, sizeof(double) * MM) == cudaSuccess &&
         cudaMalloc(&S->c, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&S->sqc, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&S->m, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&S->w, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&S->g, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&S->t, sizeof(double) * M) == cudaSuccess &&
         cudaMalloc(&S->v, sizeof(double) * M) == cudaSuccess &&
         cudaMalloc(&S->pack_a, pa) == cudaSuccess && cudaMalloc(&S->pack_b, pa) == cudaSuccess &&
         cudaMalloc(&S->exp_a, sizeof(int) * M) == cudaSuccess &&
         cudaMalloc(&S->exp_b, sizeof(int) * M) == cudaSuccess;
}

// Hadamard operator: Sylvester row of every Paley-ordered pattern, and
// mu0 = A^T y = W (S^T y) / sqrt(M).
ep_tv_status hadamard_create(const LikelihoodConfig& cfg, CsState* S, cudaStream_t s, float* mu0) {
  const int hb = log2_exact(cfg.height), wb = log2_exact(cfg.width);
  const int M = S->M, N = S->N;
  if (hb < 0 || wb < 0 || !cfg.op->patterns || M > N) return EP_TV_ERR_ARG;
  std::vector<int> sel(M);  // the patterns are distinct and in [0, N) (checked at init)
  for (int i = 0; i < M; ++i) {
    const int p = cfg.op->patterns[i];
    const unsigned kr = (unsigned)(p / cfg.width), kc = (unsigned)(p % cfg.width);
    sel[i] = (int)((bit_reverse(kr, hb) << wb) | bit_reverse(kc, wb));
  }
  if (!alloc_common(S) || cudaMalloc(&S->sel, sizeof(int) * M) != cudaSuccess) {
    cudaGetLastError();
    return EP_TV_ERR_NOMEM;
  }
  if (cudaFuncSetAttribute(fwht_rows_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(double) * kFwhtMaxSmem) != cudaSuccess ||
      cudaMemcpyAsync(S->sel, sel.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(S->g, 0, sizeof(double) * N, s) != cudaSuccess)
    return EP_TV_ERR_CUDA;
  // the host vector must outlive the copy
  if (cudaStreamSynchronize(s) != cudaSuccess) return EP_TV_ERR_CUDA;
  hadamard_place_kernel<<<(M + 255) / 256, 256, 0, s>>>(S->y, S->sel, M, S->g);
  fwht_rows(S->g, 1, N, s);
  to_f32_scaled_kernel<<<(N + 255) / 256, 256, 0, s>>>(S->g, mu0, N, 1.0 / std::sqrt((double)M));
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

}  // namespace

ep_tv_status cs_create(const LikelihoodConfig& cfg, cudaStream_t s, CsState** out, float* mu0) {
  *out = nullptr;
  if (ozaki_init() != EP_TV_OK) return EP_TV_ERR_CUDA;
  CsState* S = new (std::nothrow) CsState();
  if (!S) return EP_TV_ERR_NOMEM;
  S->M = cfg.m;
  S->N = (int)cfg.n;
  S->xi = cfg.p->xi;
  S->damping = (float)cfg.p->damping;
  S->min_tau = (float)(1.0 / cfg.p->var_cap);
  S->A = cfg.op->dense;
  S->y = cfg.y;
  if (cfg.op->op == EP_TV_OP_HADAMARD) {
    S->hadamard = true;
    const ep_tv_status st = hadamard_create(cfg, S, s, mu0);
    if (st != EP_TV_OK) {
      cs_free(S);
      return st;
    }
    *out = S;
    return EP_TV_OK;
  }
  if (!alloc_common(S) || cudaMalloc(&S->pack_at, ozaki_pack_bytes(S->N, S->M)) != cudaSuccess ||
      cudaMalloc(&S->exp_at, sizeof(int) * S->N) != cudaSuccess) {
    cudaGetLastError();
    cs_free(S);
    return EP_TV_ERR_NOMEM;
  }
  // A^T (N rows of M) packed once for W = Z A
  ozaki_pack(S->A, S->N, true, S->N, S->M, nullptr, S->exp_at, S->pack_at, OzakiSide::kRight, true, s);
  // Algorithm 1 initialises the mean of site 0 at y; y has M < N entries here, and
  // the back-projection A^T y takes its place
  aty_kernel<<<(S->N + 255) / 256, 256, 0, s>>>(S->A, S->y, S->M, S->N, mu0);
  if (cudaGetLastError() != cudaSuccess) {
    cs_free(S);
    return EP_TV_ERR_CUDA;
  }
  *out = S;
  return EP_TV_OK;
}

void cs_destroy(CsState* S) {
  if (S) cs_free(S);
}

ep_tv_status cs_set_noise(CsState* S, const float* xi_m, cudaStream_t s) {
  if (!S->xi_v && cudaMalloc(&S->xi_v, sizeof(double) * S->M) != cudaSuccess) {
    cudaGetLastError();
    return EP_TV_ERR_NOMEM;
  }
  f32_to_f64_kernel<<<(S->M + 255) / 256, 256, 0, s>>>(xi_m, S->xi_v, S->M);
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

ep_tv_status cs_update(CsState* S, float* tau0, float* nu0, const float* tp, const float* np,
                       unsigned* status, unsigned long long* counters, Tracer* tr, cudaStream_t s) {
  const int M = S->M, N = S->N;
  const long long MN = (long long)M * N, MM = (long long)M * M;
  S->status = status;
  S->tr = tr;
  S->simt_flops = 0.0;
  S->mma_flops = 0.0;
  tr->begin(EP_TV_K_CS, s);
  cs_cavity_kernel<<<g1d(N), 256, 0, s>>>(tp, np, N, S->c, S->sqc, S->m);
  if (S->hadamard) {
    // K = diag(xi) + (W c)[s_m ^ s_m'] / M
    if (cudaMemcpyAsync(S->g, S->c, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return EP_TV_ERR_CUDA;
    fwht_rows(S->g, 1, N, s);
    hadamard_k_kernel<<<g1d(MM), 256, 0, s>>>(S->K, M, S->sel, S->g, S->xi, S->xi_v);
  } else {
    // K = diag(xi) + (A C^{1/2})(A C^{1/2})^T, lower triangle, on the tensor cores
    init_k_kernel<<<g1d(MM), 256, 0, s>>>(S->K, M, S->xi, S->xi_v);
    const double f = ozaki_tensor_flops(M, M, N) / 2.0;
    S->mma_flops += f;
    Segment seg(S, s, f);
    ozaki_pack(S->A, N, false, M, N, S->sqc, S->exp_a, S->pack_a, OzakiSide::kLeft, true, s);
    ozaki_pack(S->A, N, false, M, N, S->sqc, S->exp_a, S->pack_b, OzakiSide::kRight, false, s);
    ozaki_gemm(OzakiOperand{S->pack_a, S->exp_a}, OzakiOperand{S->pack_b, S->exp_a}, N, S->K, M, M, M, 1.0,
               1.0, true, false, status, s);
  }
  // K = L L^T and Z = L^{-1}
  if (cudaMemsetAsync(S->Z, 0, sizeof(double) * MM, s) != cudaSuccess) return EP_TV_ERR_CUDA;
  chol_inv(S, S->K, M, S->Z, M, M, S->pool, s);
  if (S->hadamard) {
    // W = (L^{-1} S) W_N / sqrt(M): the lower inverse scattered to the selected
    // columns, then a fast transform of every row
    if (cudaMemsetAsync(S->G, 0, sizeof(double) * MN, s) != cudaSuccess) return EP_TV_ERR_CUDA;
    hadamard_scatter_kernel<<<g1d(MM), 256, 0, s>>>(S->Z, M, S->sel, S->G, N);
    fwht_rows(S->G, M, N, s);
  } else {
    // W = Z A on the tensor cores (Z lower triangular)
    const double f = ozaki_tensor_flops(M, N, M) / 2.0;
    S->mma_flops += f;
    Segment seg(S, s, f);
    ozaki_pack(S->Z, M, false, M, M, nullptr, S->exp_a, S->pack_a, OzakiSide::kLeft, true, s);
    ozaki_gemm(OzakiOperand{S->pack_a, S->exp_a}, OzakiOperand{S->pack_at, S->exp_at}, M, S->G, N, M, N, 0.0,
               1.0, false, true, status, s);
  }
  colsq_kernel<<<(N + 255) / 256, 256, 0, s>>>(S->G, M, N, S->w);
  // mean: t = y - A m, v = L^{-1} t, g = W^T v, E = m + c g
  if (S->hadamard) {
    if (cudaMemcpyAsync(S->g, S->m, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return EP_TV_ERR_CUDA;
    fwht_rows(S->g, 1, N, s);
    hadamard_resid_kernel<<<(M + 255) / 256, 256, 0, s>>>(S->y, S->g, S->sel, M, S->t);
  } else {
    resid_vec_kernel<<<(M + 7) / 8, 256, 0, s>>>(S->A, S->y, S->m, M, N, S->t);
  }
  trmv_lower_kernel<<<(M + 7) / 8, 256, 0, s>>>(S->Z, M, S->t, S->v);
  wtv_kernel<<<(N + 255) / 256, 256, 0, s>>>(S->G, S->v, M, N, S->g);
  cs_site0_kernel<<<g1d(N), 256, 0, s>>>(S->w, S->g, S->c, S->m, N, tau0, nu0, S->min_tau, S->damping,
                                         status, counters);
  tr->end(s, (double)N);
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

double cs_flops(const CsState* S) {
  // FP64 flops on the CUDA cores: the small products and blocks of the
  // factorisation (counted during the last update), column sums and the mean
  const double M = S->M, N = S->N;
  return S->simt_flops + 2.0 * M * N + 4.0 * M * N + M * M;
}

double cs_mma_flops(const CsState* S) { return S->mma_flops; }

}  // namespace eptv
