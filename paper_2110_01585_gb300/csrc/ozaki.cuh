// FP64-accurate matrix products on the BF16 tensor cores (ozaki.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ep_tv.h"

namespace eptv {

// A packed operand: BF16 digit slices in the tensor core's shared-memory order
// plus one power-of-two exponent per row.
struct OzakiOperand {
  const uint8_t* packed;
  const int* exps;
  int slices = 8;  // digit slices per entry: 8 or 10 (both operands of a product alike)
};

// Which operand a packing is for: left (rows of the output, 128-row tiles) or
// right (columns of the output, 64-row tiles).
enum class OzakiSide { kLeft, kRight };

// Bytes of the packed form of a rows x k operand (either side).
size_t ozaki_pack_bytes(int rows, int k, int slices = 8);
// Raises the kernel's dynamic shared-memory limit (once per process and device).
ep_tv_status ozaki_init();
// Packs rows x k operand X(r, k) = X[r * ld + k] (trans: X[k * ld + r]), times
// kscale[k] when kscale is not NULL, into out (ozaki_pack_bytes(rows, k) bytes);
// with exponents, first writes its row exponents into e (rows ints), else
// uses those in e (packing one matrix for both sides).
// slices: 8 (error about 2^-56 of the rows' largest entries) or 10 (2^-70).
void ozaki_pack(const double* X, long long ld, bool trans, int rows, int k, const double* kscale, int* e,
                uint8_t* out, OzakiSide side, bool exponents, cudaStream_t s, int slices = 8);
void ozaki_pack(const float* X, long long ld, bool trans, int rows, int k, const double* kscale, int* e,
                uint8_t* out, OzakiSide side, bool exponents, cudaStream_t s, int slices = 8);
// C = alpha C + beta A B^T for packed A (m x k, left side) and B (n x k, right
// side); C row-major, ldc.
// With 10 slices k must be at most 8192.
// lower_only: only entries with col <= row are written.  a_lower: A is lower
// triangular (row i has no entries beyond k = i), so row tiles stop early.
// A timed-out wait raises ST_TIMEOUT in status.
void ozaki_gemm(const OzakiOperand& A, const OzakiOperand& B, int k, double* C, long long ldc, int m, int n,
                double alpha, double beta, bool lower_only, bool a_lower, unsigned* status, cudaStream_t s);
// C = A B^T for row-major A (m x k), B (n x k), C (m x n), all device memory,
// with its own packing buffers (the exported ep_tv_tc_gemm_f64).
ep_tv_status ozaki_gemm_standalone(const double* A, const double* B, double* C, int m, int n, int k, int slices,
                                   cudaStream_t s);
// BF16 tensor flops of one product: the S (S + 1) / 2 slice products of m x n x k
// (padding not counted).
double ozaki_tensor_flops(int m, int n, int k, int slices = 8);

}  // namespace eptv
