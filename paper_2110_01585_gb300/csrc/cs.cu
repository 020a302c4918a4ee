// Likelihood site q_{x,0} for a dense sensing matrix A (compressive sensing).
//
// Eq. tilted_P_1 with H = A (M x N, M < N): A^T A is low rank, and the paper takes
// the Woodbury identity (Sec. III-C).  With C = diag(c), c the cavity variances of
// site 0 (1 / sum_k tau_k) and m the cavity means,
//   K = xi I_M + A C A^T = L L^T,   W = L^{-1} A,   w_i = sum_m W_mi^2 = a_i^T K^{-1} a_i,
//   Var_i = c_i - c_i^2 w_i,        E = m + C A^T K^{-1} (y - A m) = m + c * W^T L^{-1}(y - A m).
// The site update of Eq. update_q0_x then needs 1/Var_i - 1/c_i = w_i / (1 - c_i w_i).
//
// Precision: all of it runs in FP64.  c spans 1e-2 .. 1e8 (prior sites at their
// variance cap), which drives cond(K) to 1e7 .. 1e8 within a few sweeps and c_i w_i
// to within 1e-4 of 1; an FP32 or BF16 factorisation loses every digit of
// 1 - c_i w_i there.  GB300's FP64 rate is low, so this path is ALU-bound.
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
// Kernels: an FP64 tiled GEMM (C -= A B^T or C -= A B, 64 x 64 tiles, 4 x 4 per
// thread), used for K, the trailing updates of a blocked right-looking Cholesky
// and the block updates of the triangular solve; a 64 x 64 Cholesky of one
// diagonal block in shared memory; panel and block triangular solves; column
// sums; matrix-vector products.
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

namespace eptv {

namespace {

constexpr int kNb = 64;      // Cholesky / triangular-solve block size
constexpr int kGt = 64;      // GEMM tile
constexpr int kGk = 16;      // GEMM k step

// C[i, j] = alpha * C[i, j] + beta_ * sum_k A[i, k] * B(k, j) for a tile of
// (m x n); B(k, j) = B[j * ldb + k] (transposed, "NT") or B[k * ldb + j] ("NN").
// lower_only: skip tiles strictly above the diagonal (C symmetric).
template <bool kNT>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int m, int n, int k, const double* A, int lda,
                                                       const double* B, int ldb, double* C, int ldc,
                                                       double alpha, double beta_, int lower_only) {
  const int bi = blockIdx.y * kGt, bj = blockIdx.x * kGt;
  if (lower_only && bj > bi + kGt - 1) return;
  __shared__ double As[kGk][kGt + 1];
  __shared__ double Bs[kGk][kGt + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 each
  double acc[4][4] = {};
  for (int k0 = 0; k0 < k; k0 += kGk) {
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
      *cp = alpha * *cp + beta_ * acc[u][v];
    }
  }
}

// G = A diag(sqrt(c)) in FP64 (A is FP32, M x N row-major).
__global__ void scale_cols_kernel(const float* A, const double* sqc, double* G, int M, int N) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % N);
    G[e] = (double)A[e] * sqc[i];
  }
}

// A as FP64 (kept for the triangular solve)
__global__ void to_f64_kernel(const float* A, double* out, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)A[e];
}

// K = 0, then the diagonal gets the noise covariance: xi, or xi_v[i] for a
// diagonal (non-i.i.d.) noise covariance (the GEMM adds G G^T with beta = 1).
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

// Panel: rows r >= k0 + b of column block k0..k0+b solve X L_kk^T = K_panel, i.e.
// L[r, k0 + j] = (K[r, k0 + j] - sum_{l<j} L[r, k0 + l] L[k0 + j, k0 + l]) / L[k0 + j, k0 + j].
// One thread per row.
__global__ void trsm_panel_kernel(double* K, int ldk, int k0, int b, int M) {
  __shared__ double Lkk[kNb][kNb + 1];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    Lkk[i][j] = K[(long long)(k0 + i) * ldk + k0 + j];
  }
  __syncthreads();
  const int r = k0 + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  double x[kNb];
  double* row = K + (long long)r * ldk + k0;
  for (int j = 0; j < b; ++j) {
    double v = row[j];
    for (int l = 0; l < j; ++l) v -= x[l] * Lkk[j][l];
    x[j] = v / Lkk[j][j];
  }
  for (int j = 0; j < b; ++j) row[j] = x[j];
}

// Block forward solve: X[rows k0..k0+b, :] = L_kk^{-1} X[rows, :], one thread per column.
__global__ void trsm_block_cols_kernel(const double* L, int ldl, int k0, int b, double* X, int ldx,
                                       int ncols) {
  __shared__ double Lkk[kNb][kNb + 1];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    Lkk[i][j] = L[(long long)(k0 + i) * ldl + k0 + j];
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  double x[kNb];
  for (int i = 0; i < b; ++i) {
    double v = X[(long long)(k0 + i) * ldx + col];
    for (int l = 0; l < i; ++l) v -= Lkk[i][l] * x[l];
    x[i] = v / Lkk[i][i];
    X[(long long)(k0 + i) * ldx + col] = x[i];
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

// X = I (M x M)
__global__ void identity_kernel(double* X, int M) {
  const long long total = (long long)M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e - (long long)i * M);
    X[e] = i == j ? 1.0 : 0.0;
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
          int ldc, double alpha, double beta_, bool lower_only, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  dim3 grid((n + kGt - 1) / kGt, (m + kGt - 1) / kGt);
  if (nt)
    gemm_f64_kernel<true><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, alpha, beta_,
                                               lower_only ? 1 : 0);
  else
    gemm_f64_kernel<false><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, alpha, beta_,
                                                lower_only ? 1 : 0);
}

}  // namespace

struct CsState {
  int M = 0, N = 0;
  bool hadamard = false;      // subsampled Hadamard rows in place of the dense matrix
  double xi = 0.0;
  float damping = 0.5f, min_tau = 1e-8f;
  const float* A = nullptr;   // borrowed, M x N FP32
  const float* y = nullptr;   // context copy
  double* A64 = nullptr;      // M x N
  double* G = nullptr;        // M x N, then W
  double* K = nullptr;        // M x M, then L
  double* c = nullptr;
  double* sqc = nullptr;
  double* m = nullptr;
  double* w = nullptr;
  double* g = nullptr;
  double* t = nullptr;        // M
  double* xi_v = nullptr;     // M noise variances (diagonal noise covariance), or NULL
  int* sel = nullptr;         // Hadamard: M Sylvester row indices
  double* Z = nullptr;        // Hadamard: M x M, L^{-1}
};

namespace {

void cs_free(CsState* S) {
  cudaFree(S->A64);
  cudaFree(S->G);
  cudaFree(S->K);
  cudaFree(S->c);
  cudaFree(S->sqc);
  cudaFree(S->m);
  cudaFree(S->w);
  cudaFree(S->g);
  cudaFree(S->t);
  cudaFree(S->xi_v);
  cudaFree(S->sel);
  cudaFree(S->Z);
  delete S;
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

// Hadamard operator: Sylvester row of every Paley-ordered pattern, the buffers,
// and mu0 = A^T y = W (S^T y) / sqrt(M).
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
  const long long MN = (long long)M * N;
  bool ok = cudaMalloc(&S->G, sizeof(double) * MN) == cudaSuccess &&
            cudaMalloc(&S->K, sizeof(double) * (long long)M * M) == cudaSuccess &&
            cudaMalloc(&S->Z, sizeof(double) * (long long)M * M) == cudaSuccess &&
            cudaMalloc(&S->sel, sizeof(int) * M) == cudaSuccess &&
            cudaMalloc(&S->c, sizeof(double) * N) == cudaSuccess &&
            cudaMalloc(&S->sqc, sizeof(double) * N) == cudaSuccess &&
            cudaMalloc(&S->m, sizeof(double) * N) == cudaSuccess &&
            cudaMalloc(&S->w, sizeof(double) * N) == cudaSuccess &&
            cudaMalloc(&S->g, sizeof(double) * N) == cudaSuccess &&
            cudaMalloc(&S->t, sizeof(double) * M) == cudaSuccess;
  if (!ok) {
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

// X = L^{-1} X in place for the M x ncols block X (ld ldx), L the lower factor in K:
// blocked forward substitution, the block updates as GEMMs.
void forward_solve(const double* L, int M, double* X, int ldx, int ncols, cudaStream_t s) {
  for (int k0 = 0; k0 < M; k0 += kNb) {
    const int b = std::min(kNb, M - k0);
    if (k0 > 0)  // X[k0:k0+b, :] -= L[k0:k0+b, 0:k0] X[0:k0, :]
      gemm(false, b, ncols, k0, L + (long long)k0 * M, M, X, ldx, X + (long long)k0 * ldx, ldx, 1.0,
           -1.0, false, s);
    trsm_block_cols_kernel<<<(ncols + 127) / 128, 128, 0, s>>>(L, M, k0, b, X, ldx, ncols);
  }
}

// Z = L^{-1}: forward substitution on the identity; L^{-1} is lower triangular, so
// block row k0 only involves columns 0 .. k0 + b.
void lower_inverse(const double* L, int M, double* Z, cudaStream_t s) {
  identity_kernel<<<g1d((long long)M * M), 256, 0, s>>>(Z, M);
  for (int k0 = 0; k0 < M; k0 += kNb) {
    const int b = std::min(kNb, M - k0);
    if (k0 > 0)
      gemm(false, b, k0, k0, L + (long long)k0 * M, M, Z, M, Z + (long long)k0 * M, M, 1.0, -1.0,
           false, s);
    trsm_block_cols_kernel<<<(k0 + b + 127) / 128, 128, 0, s>>>(L, M, k0, b, Z, M, k0 + b);
  }
}

}  // namespace

ep_tv_status cs_create(const LikelihoodConfig& cfg, cudaStream_t s, CsState** out, float* mu0) {
  *out = nullptr;
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
  const long long MN = (long long)S->M * S->N;
  bool ok = cudaMalloc(&S->A64, sizeof(double) * MN) == cudaSuccess &&
            cudaMalloc(&S->G, sizeof(double) * MN) == cudaSuccess &&
            cudaMalloc(&S->K, sizeof(double) * (long long)S->M * S->M) == cudaSuccess &&
            cudaMalloc(&S->c, sizeof(double) * S->N) == cudaSuccess &&
            cudaMalloc(&S->sqc, sizeof(double) * S->N) == cudaSuccess &&
            cudaMalloc(&S->m, sizeof(double) * S->N) == cudaSuccess &&
            cudaMalloc(&S->w, sizeof(double) * S->N) == cudaSuccess &&
            cudaMalloc(&S->g, sizeof(double) * S->N) == cudaSuccess &&
            cudaMalloc(&S->t, sizeof(double) * S->M) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cs_free(S);
    return EP_TV_ERR_NOMEM;
  }
  to_f64_kernel<<<g1d(MN), 256, 0, s>>>(S->A, S->A64, MN);
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
  const long long MN = (long long)M * N;
  tr->begin(EP_TV_K_CS, s);
  cs_cavity_kernel<<<g1d(N), 256, 0, s>>>(tp, np, N, S->c, S->sqc, S->m);
  if (S->hadamard) {
    // K = diag(xi) + (W c)[s_m ^ s_m'] / M
    if (cudaMemcpyAsync(S->g, S->c, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return EP_TV_ERR_CUDA;
    fwht_rows(S->g, 1, N, s);
    hadamard_k_kernel<<<g1d((long long)M * M), 256, 0, s>>>(S->K, M, S->sel, S->g, S->xi, S->xi_v);
  } else {
    // K = xi I + (A C^{1/2})(A C^{1/2})^T, lower triangle
    scale_cols_kernel<<<g1d(MN), 256, 0, s>>>(S->A, S->sqc, S->G, M, N);
    init_k_kernel<<<g1d((long long)M * M), 256, 0, s>>>(S->K, M, S->xi, S->xi_v);
    gemm(true, M, M, N, S->G, N, S->G, N, S->K, M, 1.0, 1.0, true, s);
  }
  // blocked right-looking Cholesky K = L L^T (lower)
  for (int k0 = 0; k0 < M; k0 += kNb) {
    const int b = std::min(kNb, M - k0);
    potrf_block_kernel<<<1, 256, 0, s>>>(S->K, M, k0, b, status);
    const int rest = M - k0 - b;
    if (rest > 0) {
      trsm_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(S->K, M, k0, b, M);
      // trailing K[k0+b:, k0+b:] -= L_panel L_panel^T (lower tiles)
      const double* P = S->K + (long long)(k0 + b) * M + k0;
      gemm(true, rest, rest, b, P, M, P, M, S->K + (long long)(k0 + b) * M + (k0 + b), M, 1.0, -1.0,
           true, s);
    }
  }
  if (S->hadamard) {
    // W = (L^{-1} S) W_N / sqrt(M): the lower inverse scattered to the selected
    // columns, then a fast transform of every row
    lower_inverse(S->K, M, S->Z, s);
    if (cudaMemsetAsync(S->G, 0, sizeof(double) * MN, s) != cudaSuccess) return EP_TV_ERR_CUDA;
    hadamard_scatter_kernel<<<g1d((long long)M * M), 256, 0, s>>>(S->Z, M, S->sel, S->G, N);
    fwht_rows(S->G, M, N, s);
  } else {
    // W = L^{-1} A (blocked forward substitution on all N columns), into G
    if (cudaMemcpyAsync(S->G, S->A64, sizeof(double) * MN, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return EP_TV_ERR_CUDA;
    forward_solve(S->K, M, S->G, N, N, s);
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
  forward_solve(S->K, M, S->t, 1, 1, s);
  wtv_kernel<<<(N + 255) / 256, 256, 0, s>>>(S->G, S->t, M, N, S->g);
  cs_site0_kernel<<<g1d(N), 256, 0, s>>>(S->w, S->g, S->c, S->m, N, tau0, nu0, S->min_tau, S->damping,
                                         status, counters);
  tr->end(s, (double)N);
  return cudaGetLastError() == cudaSuccess ? EP_TV_OK : EP_TV_ERR_CUDA;
}

double cs_flops(const CsState* S) {
  const double M = S->M, N = S->N;
  if (S->hadamard) {
    // K from one transform, Cholesky, the lower inverse, M row transforms, column sums, mean
    const double lg = std::log2(N);
    return N * lg + M * M * M / 3.0 + M * M * M / 3.0 + M * N * lg + 2.0 * M * N + 4.0 * M * N;
  }
  // K (lower half of G G^T), Cholesky, W = L^{-1} A, column sums and the mean
  return M * M * N + M * M * M / 3.0 + M * M * N + 2.0 * M * N + 4.0 * M * N;
}

}  // namespace eptv
