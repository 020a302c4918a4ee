// FP64-accurate matrix products on the BF16 tensor cores (tcgen05), for the
// compressive-sensing likelihood site (Sec. III-C's Woodbury form: the operator
// products K = A C A^T and W = L^{-1} A = Z A, and the large products of the
// Cholesky factorisation and inverse of K).
//
// Splitting (Ozaki's error-free splitting of a product into exact slice
// products).  Every operand row r is scaled by 2^-e_r, e_r the binary exponent
// of its largest entry, so that every scaled entry x lies in (-1, 1).  x is then
// written as eight 7-bit digits by round-to-nearest,
//   x = sum_{s=1..8} d_s 2^{-7 s} + rho,   |d_1| <= 128, |d_s| <= 64 (s > 1), |rho| <= 2^-57,
// each step exact in FP64.  The slice d_s 2^{-7 s} has at most 8 significant bits, so
// it is exact in BF16, and the product of two slices is exact in FP32.  For a
// row i of A and a row j of B (C = A B^T),
//   sum_k A_ik B_jk = 2^{e_i + f_j} sum_{s,t} 2^{-7(s+t)} sum_k d_s(A_ik) d_t(B_jk),
// kept for s + t <= 9 (the dropped products are below 2^-54 of |A_i||B_j|).  The
// products with the same s + t (a "diagonal", s + t = 2..6) share one FP32
// accumulator in tensor memory; over a chunk of 256 values of k each such sum is
// an integer multiple of 2^{-7(s+t)} below 2^23 of it, so the tensor core adds it
// exactly, and after every chunk the five accumulators are converted to integers
// and added into two 64-bit integers per output (diagonals 2-4 and 5-6).  The
// products with s + t = 7..9
// carry 2^-35 or less of the result and go to a sixth FP32 accumulator over the
// whole of k.  (The tensor core's FP32 accumulation is not round-to-nearest at
// every add: measured on a single product, a tail starting at s + t = 6 left an
// error of 2^-50, which this split removes.)  The error is relative to the rows'
// largest entries, as for every split of this kind:
//   |error| <~ 2^-55 (max|A_i| sum|B_j| + max|B_j| sum|A_i|) + 2^-52 k max|A_i| max|B_j|
// plus one final rounding; for operands of one scale that is an FP64 product's.
//
// Kernel: one CTA per 128 x 64 output tile; K in stages of 16 (one MMA K step),
// four shared-memory stages filled by bulk asynchronous copies (cp.async.bulk,
// the TMA engine) from operands packed in the tensor core's shared-memory
// core-matrix order, so that a stage is two contiguous copies (A: 128 rows, B:
// 64 rows, 8 slices each).  Warp-specialised: one thread issues the copies and
// waits only for stages to free up, one thread issues the 36 MMAs of a stage
// (M = 128, N = 64, K = 16, BF16 inputs, FP32 accumulators in tensor memory) and
// waits only for stages to land, and sixteen warps read the accumulators back
// (tcgen05.ld) at every chunk end, handing them back to the MMA thread through
// a second pair of barriers.  A second form, 10 slices with seven exact
// diagonals (Split<10>), serves the Cholesky factorisation's products.  Every
// wait on an mbarrier gives up after two seconds: the kernel then raises
// ST_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and exits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"
#include "ozaki.cuh"

namespace eptv {

namespace {

constexpr int kDigitBits = 7;
constexpr int kTM = 128;             // output tile rows; packing row tile
constexpr int kTN = 64;              // output tile columns
constexpr int kKS = 16;              // K per stage (one MMA K step)
constexpr int kCore = 128;           // one core matrix: 8 rows x 16 bytes
constexpr int kSliceKc = kTM / 8 * kCore;               // 16 row groups: 2048 bytes
constexpr int kSliceKcB = kTN / 8 * kCore;              // 8 row groups: 1024 bytes
constexpr int kTmemCols = 512;  // the accumulators (at most 7 of 64 columns), rounded up

// Shapes that depend on the number of digit slices S (8 for the operator
// products, 10 where the product is to be more accurate than an FP64 GEMM):
// a stage holds the S slices of a 128 x 16 A block and a 64 x 16 B block; as many
// stages as fit in shared memory (four of 48 KB for S = 8, three of 60 KB for 10).
template <int S>
struct Split {
  // exact accumulators (the diagonals s + t = 2 .. kExact + 1) and the chunk of k
  // over which their sums stay exact integers (below 2^22.2 of their unit): for
  // S = 8 five diagonals over 256 values, the FP32 tail from s + t = 7 (2^-35 of
  // the result); for S = 10 seven over 128, the tail from s + t = 9 (2^-49).  The
  // chunk sums go into two 64-bit integers per output, diagonals 2-4 and the rest,
  // which stay below 2^51 for k <= 8192 (S = 10) or 65536 (S = 8)
  static constexpr int kExact = S <= 8 ? 5 : 7;
  static constexpr int kChunkStages = S <= 8 ? 16 : 8;
  static_assert(kTN * (kExact + 1) <= kTmemCols, "tensor memory");
  static constexpr int kAStage = S * 2 * kSliceKc;
  static constexpr int kBStage = S * 2 * kSliceKcB;
  static constexpr int kStageBytes = kAStage + kBStage;
  static constexpr int kStages = S <= 8 ? 4 : 3;
  // the stages, 8 KB of slack past the last stage (so that every descriptor
  // address stays inside the allocation) and the barriers
  static constexpr int kSmemBytes = 1024 + kStages * kStageBytes + 8192 + 256;
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Waits for the phase of the given parity; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

// The same wait for threads with nothing else to do (the reading warps): each
// try asks the hardware to suspend the thread for up to 20 us until the phase
// completes, so that they do not take issue slots from the MMA thread.
__device__ __forceinline__ bool mbar_wait_idle(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzling, K-major core matrices:
// lbo = bytes between core matrices adjacent in K, sbo = adjacent in M (N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = kTN.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- packing

// Operand entry X(r, k) = X[r * ld + k] (X[k * ld + r] when trans), times ks[k]
// when a k scale is given.
template <typename T>
__device__ __forceinline__ double entry(const T* X, long long ld, int trans, const double* ks, int r, int k) {
  const double x = (double)(trans ? X[(long long)k * ld + r] : X[(long long)r * ld + k]);
  return ks ? x * ks[k] : x;
}

// e[r] = binary exponent of max_k |X(r, k)| (0 for a zero row): |X(r, k)| 2^-e[r] < 1.
template <typename T>
__global__ void row_exponent_kernel(const T* X, long long ld, int trans, const double* ks, int R, int K,
                                    int* e) {
  if (!trans) {
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    double m = 0.0;
    for (int k = lane; k < K; k += 32) m = fmax(m, fabs(entry(X, ld, 0, ks, r, k)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      int ex = 0;
      if (m > 0.0) frexp(m, &ex);
      e[r] = ex;
    }
  } else {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double m = 0.0;
    for (int k = 0; k < K; ++k) m = fmax(m, fabs(entry(X, ld, 1, ks, r, k)));
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);
    e[r] = ex;
  }
}

// Digits of 8 consecutive k of one row, written as 8 slices of 16 bytes into the
// packed layout: blocks of (tile rows TR) x (one K stage of 16) holding, for slice s
// and K half kc (8 values of k), TR / 8 core matrices of 8 rows x 16 bytes:
// byte ((s * 2 + kc) * TR / 8 + g) * 128 + w * 16 of the block for row 8 g + w.
// Every block is one contiguous bulk copy.  Rows >= R and k >= K (the padding)
// are written as zeros.
template <typename T, int S>
__global__ void pack_kernel(const T* X, long long ld, int trans, const double* ks, int R, int K, const int* e,
                            uint8_t* out, int tile_rows, int r_pad, int n_oct) {
  const long long total = (long long)r_pad * n_oct;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int r, o;
  if (trans) {  // consecutive threads: consecutive rows (columns of X) -> coalesced reads
    r = (int)(idx % r_pad);
    o = (int)(idx / r_pad);
  } else {
    o = (int)(idx % n_oct);
    r = (int)(idx / n_oct);
  }
  const int k0 = o * 8;
  double v[8];
  const bool row_ok = r < R;
  const int ex = row_ok ? e[r] : 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = k0 + i;
    double x = 0.0;
    if (row_ok && k < K) x = entry(X, ld, trans, ks, r, k);
    v[i] = ldexp(x, -ex);
  }
  const int nkt = n_oct / 2;
  const int groups = tile_rows / 8;
  const int rt = r / tile_rows, rr = r % tile_rows, g = rr / 8, w = rr % 8;
  const int kt = o / 2, kc = o % 2;
  const long long block_bytes = (long long)S * 2 * groups * kCore;
  uint8_t* base = out + ((long long)rt * nkt + kt) * block_bytes + ((long long)kc * groups + g) * kCore + w * 16;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float w_s = exp2f(-(float)(kDigitBits * (s + 1)));
    uint32_t packed[4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const double x0 = v[i] * 128.0, x1 = v[i + 1] * 128.0;
      const double d0 = rint(x0), d1 = rint(x1);
      v[i] = x0 - d0;
      v[i + 1] = x1 - d1;
      const unsigned short b0 = __bfloat16_as_ushort(__float2bfloat16_rn((float)d0 * w_s));
      const unsigned short b1 = __bfloat16_as_ushort(__float2bfloat16_rn((float)d1 * w_s));
      packed[i / 2] = (uint32_t)b0 | ((uint32_t)b1 << 16);
    }
    *reinterpret_cast<uint4*>(base + (long long)s * 2 * groups * kCore) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// ---- the product

struct GemmArgs {
  const uint8_t* pa;   // packed A (rows of the output), 128-row tiles
  const uint8_t* pb;   // packed B (columns of the output), 64-row tiles
  const int* ea;
  const int* eb;
  int nkt;             // K stages of both packings
  double* C;
  long long ldc;
  int m, n;
  double alpha, beta;
  int lower_only;      // write only col <= row; skip tiles above the diagonal
  int a_lower;         // A lower triangular: row tile i reads k < 128 (i + 1)
  unsigned* status;
};

// Roles: warps 0-15 read the accumulators (warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31, i.e. output rows, and output columns 16 (w / 4) .. + 15);
// warp 16 lane 0 issues the MMAs; warp 17 lane 0 issues the bulk copies.
// Barriers: full[b] (a stage's copies landed), empty[b] (the MMAs reading stage b
// finished), acc_full (a chunk's MMAs finished), acc_empty (the reading warps are
// done with the chunk's accumulators).
constexpr int kEpiWarps = 16;
constexpr int kEpiCols = kTN / 4;  // output columns per reading warp
constexpr int kThreads = (kEpiWarps + 2) * 32;

template <int S>
__global__ void __launch_bounds__(kThreads, 1) ozaki_gemm_kernel(GemmArgs a) {
  using Sh = Split<S>;
  constexpr int kStages = Sh::kStages, kStageBytes = Sh::kStageBytes;
  constexpr int kExact = Sh::kExact, kChunkStages = Sh::kChunkStages;
  constexpr int kAStage = Sh::kAStage, kBStage = Sh::kBStage;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + 8192);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* produced_out = reinterpret_cast<int*>(tmem_slot + 2);
  int* committed_out = reinterpret_cast<int*>(tmem_slot + 3);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
  if (a.lower_only && col0 > row0 + kTM - 1) return;
  int nst = a.nkt;
  if (a.a_lower) nst = min(nst, (row0 + kTM + kKS - 1) / kKS);
  const int n_chunks = (nst + kChunkStages - 1) / kChunkStages;

  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages);
  const uint32_t acc_full = smem_u32(bars + 2 * kStages), acc_empty = acc_full + 8;
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    *abort_flag = 0;
    *produced_out = 0;
    *committed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == kEpiWarps + 1) {
    // producer: one A block (128 x 16, 32 KB) and one B block (64 x 16, 16 KB) per stage
    if (lane == 0) {
      const uint8_t* pa = a.pa + (long long)blockIdx.y * a.nkt * kAStage;
      const uint8_t* pb = a.pb + (long long)blockIdx.x * a.nkt * kBStage;
      int st = 0;
      for (; st < nst && !*abort_flag; ++st) {
        const int b = st % kStages;
        if (st >= kStages && !mbar_wait(empty0 + 8 * b, ((st / kStages) - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t bar = full0 + 8 * b, dst = sbase + b * kStageBytes;
        expect_tx(bar, kStageBytes);
        bulk_load(dst, pa + (long long)st * kAStage, kAStage, bar);
        bulk_load(dst + kAStage, pb + (long long)st * kBStage, kBStage, bar);
      }
      *produced_out = st;
    }
  } else if (warp == kEpiWarps) {
    // MMA issuer
    if (lane == 0) {
      int st = 0;
      bool tail_started = false;  // the tail accumulator runs over the whole of k
      for (int c = 0; c < n_chunks && !*abort_flag; ++c) {
        if (c > 0 && !mbar_wait(acc_empty, (c - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        uint32_t started = 0;  // bit q: accumulator q has been written in this chunk
        const int c1 = min(nst, (c + 1) * kChunkStages);
        for (; st < c1; ++st) {
          const int b = st % kStages;
          if (!mbar_wait(full0 + 8 * b, (st / kStages) & 1)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t ab = sbase + b * kStageBytes, bb = ab + kAStage;
          // the S (S + 1) / 2 slice pairs, unrolled: every offset and accumulator
          // index is a compile-time constant and the flags stay in registers
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const uint64_t ad = smem_desc(ab + s * 2 * kSliceKc, kSliceKc, kCore);
#pragma unroll
            for (int t = 0; t < S - s; ++t) {
              const int q = s + t < kExact ? s + t : kExact;
              const uint64_t bd = smem_desc(bb + t * 2 * kSliceKcB, kSliceKcB, kCore);
              uint32_t accumulate;
              if (q < kExact) {
                accumulate = (started >> q) & 1u;
                started |= 1u << q;
              } else {
                accumulate = tail_started ? 1u : 0u;
                tail_started = true;
              }
              mma_bf16(tmem + q * kTN, ad, bd, accumulate);
            }
          }
          mma_commit(empty0 + 8 * b);
          *committed_out = st + 1;
        }
        if (*abort_flag) break;
        mma_commit(acc_full);  // arrives once every MMA of the chunk has finished
      }
    }
  } else {
    // readers: fold every chunk's exact sums into two 64-bit integers per output,
    // acc_hi for the diagonals s + t = 2..4 (unit 2^-28) and acc_lo for the others
    // (unit 2^-7 (kExact + 1)); write C at the end
    const int quarter = warp % 4, c_part = warp / 4;
    long long acc_hi[kEpiCols], acc_lo[kEpiCols];
#pragma unroll
    for (int j = 0; j < kEpiCols; ++j) acc_hi[j] = acc_lo[j] = 0;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + c_part * kEpiCols;
    for (int c = 0; c < n_chunks; ++c) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_idle(acc_full, c & 1));
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < kExact; ++q) {
        const float to_int = exp2f((float)(kDigitBits * (q + 2)));
        const int shift = q < 3 ? kDigitBits * (2 - q) : kDigitBits * (kExact - 1 - q);
#pragma unroll
        for (int cb = 0; cb < kEpiCols / 16; ++cb) {
          uint32_t r[16];
          tmem_ld16(lane_addr + q * kTN + cb * 16, r);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[i]) * to_int) << shift;
            if (q < 3)
              acc_hi[cb * 16 + i] += v;
            else
              acc_lo[cb * 16 + i] += v;
          }
        }
      }
      if (c == n_chunks - 1) {
        // the tail accumulator, then
        // C = alpha C + beta 2^{e_i + f_j} (acc_hi 2^-28 + acc_lo 2^-7 (kExact + 1) + tail)
        const int row = row0 + quarter * 32 + lane;
        const int ei = row < a.m ? a.ea[row] : 0;
#pragma unroll
        for (int cb = 0; cb < kEpiCols / 16; ++cb) {
          uint32_t r[16];
          tmem_ld16(lane_addr + kExact * kTN + cb * 16, r);
          if (row < a.m) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = col0 + c_part * kEpiCols + cb * 16 + i;
              if (col >= a.n || (a.lower_only && col > row)) continue;
              const int ex = ei + a.eb[col];
              const double v = ldexp((double)acc_hi[cb * 16 + i], ex - kDigitBits * 4) +
                               ldexp((double)acc_lo[cb * 16 + i], ex - kDigitBits * (kExact + 1)) +
                               ldexp((double)__uint_as_float(r[i]), ex);
              double* cp = a.C + (long long)row * a.ldc + col;
              *cp = a.alpha == 0.0 ? a.beta * v : a.alpha * *cp + a.beta * v;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty) : "memory");
    }
  }

  __syncthreads();
  if (*abort_flag && tid == 0) {
    atomicOr(a.status, ST_TIMEOUT);
    // copies and MMAs in flight must land before the CTA's shared and tensor memory go
    const int produced = *produced_out, committed = *committed_out;
    for (int st = max(0, produced - kStages); st < produced; ++st)
      mbar_wait(full0 + 8 * (st % kStages), (st / kStages) & 1);
    if (committed > 0) mbar_wait(empty0 + 8 * ((committed - 1) % kStages), ((committed - 1) / kStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

inline unsigned blocks_for(long long n, int threads) {
  return (unsigned)std::max<long long>(1, (n + threads - 1) / threads);
}

}  // namespace

size_t ozaki_pack_bytes(int rows, int k, int slices) {
  const long long r_pad = (long long)(rows + kTM - 1) / kTM * kTM;  // covers both tile heights
  const long long k_pad = (long long)(k + kKS - 1) / kKS * kKS;
  return (size_t)(r_pad * k_pad * slices * 2);
}

ep_tv_status ozaki_init() {
  const bool ok = cudaFuncSetAttribute(ozaki_gemm_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Split<8>::kSmemBytes) == cudaSuccess &&
                  cudaFuncSetAttribute(ozaki_gemm_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Split<10>::kSmemBytes) == cudaSuccess;
  return ok ? EP_TV_OK : EP_TV_ERR_CUDA;
}

namespace {

template <typename T>
void pack_any(const T* X, long long ld, bool trans, int rows, int k, const double* kscale, int* e, uint8_t* out,
              OzakiSide side, bool exponents, int slices, cudaStream_t s) {
  if (rows <= 0 || k <= 0) return;
  if (exponents) {
    if (trans)
      row_exponent_kernel<T><<<blocks_for(rows, 256), 256, 0, s>>>(X, ld, 1, kscale, rows, k, e);
    else
      row_exponent_kernel<T><<<blocks_for(rows, 8), 256, 0, s>>>(X, ld, 0, kscale, rows, k, e);
  }
  const int tile_rows = side == OzakiSide::kLeft ? kTM : kTN;
  const int r_pad = (rows + tile_rows - 1) / tile_rows * tile_rows;
  const int n_oct = (k + kKS - 1) / kKS * 2;
  const unsigned nb = blocks_for((long long)r_pad * n_oct, 256);
  if (slices == 10)
    pack_kernel<T, 10><<<nb, 256, 0, s>>>(X, ld, trans ? 1 : 0, kscale, rows, k, e, out, tile_rows, r_pad, n_oct);
  else
    pack_kernel<T, 8><<<nb, 256, 0, s>>>(X, ld, trans ? 1 : 0, kscale, rows, k, e, out, tile_rows, r_pad, n_oct);
}

}  // namespace

void ozaki_pack(const double* X, long long ld, bool trans, int rows, int k, const double* kscale, int* e,
                uint8_t* out, OzakiSide side, bool exponents, cudaStream_t s, int slices) {
  pack_any(X, ld, trans, rows, k, kscale, e, out, side, exponents, slices, s);
}

void ozaki_pack(const float* X, long long ld, bool trans, int rows, int k, const double* kscale, int* e,
                uint8_t* out, OzakiSide side, bool exponents, cudaStream_t s, int slices) {
  pack_any(X, ld, trans, rows, k, kscale, e, out, side, exponents, slices, s);
}

void ozaki_gemm(const OzakiOperand& A, const OzakiOperand& B, int k, double* C, long long ldc, int m, int n,
                double alpha, double beta, bool lower_only, bool a_lower, unsigned* status, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  GemmArgs g;
  g.pa = A.packed;
  g.pb = B.packed;
  g.ea = A.exps;
  g.eb = B.exps;
  g.nkt = (k + kKS - 1) / kKS;
  g.C = C;
  g.ldc = ldc;
  g.m = m;
  g.n = n;
  g.alpha = alpha;
  g.beta = beta;
  g.lower_only = lower_only ? 1 : 0;
  g.a_lower = a_lower ? 1 : 0;
  g.status = status;
  dim3 grid((n + kTN - 1) / kTN, (m + kTM - 1) / kTM);
  if (A.slices == 10)
    ozaki_gemm_kernel<10><<<grid, kThreads, Split<10>::kSmemBytes, s>>>(g);
  else
    ozaki_gemm_kernel<8><<<grid, kThreads, Split<8>::kSmemBytes, s>>>(g);
}

ep_tv_status ozaki_gemm_standalone(const double* A, const double* B, double* C, int m, int n, int k, int slices,
                                   cudaStream_t s) {
  if (ozaki_init() != EP_TV_OK) return EP_TV_ERR_CUDA;
  uint8_t *pa = nullptr, *pb = nullptr;
  int *ea = nullptr, *eb = nullptr;
  unsigned* status = nullptr;
  ep_tv_status st = EP_TV_OK;
  if (cudaMalloc(&pa, ozaki_pack_bytes(m, k, slices)) != cudaSuccess ||
      cudaMalloc(&pb, ozaki_pack_bytes(n, k, slices)) != cudaSuccess || cudaMalloc(&ea, sizeof(int) * m) != cudaSuccess ||
      cudaMalloc(&eb, sizeof(int) * n) != cudaSuccess || cudaMalloc(&status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    st = EP_TV_ERR_NOMEM;
  }
  unsigned h_status = 0;
  if (st == EP_TV_OK) {
    cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    ozaki_pack(A, k, false, m, k, nullptr, ea, pa, OzakiSide::kLeft, true, s, slices);
    ozaki_pack(B, k, false, n, k, nullptr, eb, pb, OzakiSide::kRight, true, s, slices);
    ozaki_gemm(OzakiOperand{pa, ea, slices}, OzakiOperand{pb, eb, slices}, k, C, n, m, n, 0.0, 1.0, false, false,
               status, s);
    if (cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = EP_TV_ERR_CUDA;
    else if (h_status & ST_TIMEOUT)
      st = EP_TV_ERR_TIMEOUT;
  }
  cudaFree(pa);
  cudaFree(pb);
  cudaFree(ea);
  cudaFree(eb);
  cudaFree(status);
  return st;
}

double ozaki_tensor_flops(int m, int n, int k, int slices) {
  // the S (S + 1) / 2 slice products of the split form, each a BF16 product of m x n x k
  return slices * (slices + 1) / 2.0 * 2.0 * (double)m * (double)n * (double)k;
}

}  // namespace eptv

extern "C" ep_tv_status ep_tv_tc_gemm_f64(const double* A, const double* B, double* C, int32_t m, int32_t n,
                                          int32_t k, int32_t slices, void* cuda_stream) {
  if (!A || !B || !C || m < 1 || n < 1 || k < 1) return EP_TV_ERR_ARG;
  if (slices != 8 && !(slices == 10 && k <= 8192)) return EP_TV_ERR_ARG;
  return eptv::ozaki_gemm_standalone(A, B, C, m, n, k, slices, static_cast<cudaStream_t>(cuda_stream));
}
