// Fused prior-site pass: the four V_k updates of one EP sweep in one kernel.
//
// Sec. III-C: for each V_k in turn, every edge (i, j) of V_k forms the cavity of
// site k at both pixels, the moments of the Laplace-tilted edge marginal
// (Eq. marginal_tilted_un), the projection onto (x_i, x_j), and the new site k
// (Eq. update_qk_x) with the variance cap and damping.  The edges of one V_k are
// disjoint, so they update in parallel; V_{k+1} sees the result of V_k.
//
// Partition (Fig. 1, Eq. prior1; read as a torus with even H and W):
//   V1 horizontal (r,2a)-(r,2a+1)   V2 horizontal (r,2a+1)-(r,2a+2 mod W)
//   V3 vertical   (2b,c)-(2b+1,c)   V4 vertical   (2b+1,c)-(2b+2 mod H,c)
// The free boundary drops the wrap-around edges.
//
// The prior-site planes are read from one buffer and written to another: a
// tile's halo belongs to neighbouring tiles, which may already have written
// their results when it is staged.
//
// Temporal blocking: a CTA owns a TH x TW tile and stages a (TH+4) x (TW+4)
// region (2-pixel halo) of all ten site planes in shared memory.  Each of the
// two horizontal updates can spoil at most one halo column per side, each of
// the vertical ones one halo row, so after any order of V1..V4 the tile itself
// holds exactly the values a one-update-per-launch schedule would produce.  The
// sweep therefore reads every site plane once and writes the four prior-site
// planes once: 36 B read + 32 B written per pixel for denoising, where site 0 is
// (1/xi, y/xi) and only y is read.
//
// Arithmetic: FP32 with the cancellation-free forms of tilted.cuh; the new
// precision uses tau_i = rho / (c_j + q c_i), which equals 1/Var_i - 1/c_i of
// Eq. update_qk_x (q = Sbar / s^2, rho = 1 - q) without subtracting.  Edges with
// lam * s < 1e-3 (where rho is a small difference of O(1) numbers) are redone in
// FP64 when fp64_tail is set.
#include "internal.cuh"
#include "tilted.cuh"

namespace eptv {

namespace {

constexpr int kTH = 16;
constexpr int kTW = 64;
constexpr int kThreads = 256;
constexpr int kRH = kTH + 4;
constexpr int kRW = kTW + 4;
constexpr int kRN = kRH * kRW;
constexpr int kPlanes = 10;  // tau0..tau4, nu0..nu4
constexpr size_t kSmemBytes = size_t(kPlanes) * kRN * sizeof(float);

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One tile (bx, by) of one image; `part` indexes its a_u partial sum.
template <bool kSite0FromY>
__device__ __forceinline__ void prior_tile(const SweepArgs& a, int bx, int by, int part,
                                           float* smem) {
  float* sT = smem;             // [5][kRN]
  float* sV = smem + 5 * kRN;   // [5][kRN]
  const int H = a.height, W = a.width;
  const long long N = a.n;
  const int r0 = by * kTH;
  const int c0 = bx * kTW;
  const int tid = threadIdx.x;

  // ---- stage the region (positions outside a free-boundary image stay unused)
  for (int idx = tid; idx < kRN; idx += kThreads) {
    const int rr = idx / kRW, cc = idx - rr * kRW;
    int gr = r0 - 2 + rr, gc = c0 - 2 + cc;
    bool present = true;
    if (a.periodic) {
      gr = wrap(gr, H);
      gc = wrap(gc, W);
    } else {
      present = gr >= 0 && gr < H && gc >= 0 && gc < W;
    }
    if (present) {
      const long long p = (long long)gr * W + gc;
      if (kSite0FromY) {
        sT[idx] = a.inv_xi;
        sV[idx] = a.y[p] * a.inv_xi;
      } else {
        sT[idx] = a.tau0[p];
        sV[idx] = a.nu0[p];
      }
#pragma unroll
      for (int s = 1; s < 5; ++s) {
        sT[s * kRN + idx] = a.tin[(s - 1) * N + p];
        sV[s * kRN + idx] = a.nin[(s - 1) * N + p];
      }
    } else {
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        sT[s * kRN + idx] = 1.0f;
        sV[s * kRN + idx] = 0.0f;
      }
    }
  }
  __syncthreads();

  const float lam = (float)(*a.beta);
  const double lam_d = *a.beta;
  const float damp = a.damping, keep = 1.0f - a.damping;
  float eab_acc = 0.0f;
  unsigned n_fp64 = 0, n_capped = 0;
  bool bad = false;

  for (int t = 0; t < 4; ++t) {
    const int k = (a.order >> (4 * t)) & 0xF;
    const bool horiz = k <= 2;
    const int parity = (k == 1 || k == 3) ? 0 : 1;
    // edges (i, i + step) whose first endpoint has the given parity along the axis
    const int along = horiz ? kRW : kRH;
    const int across = horiz ? kRH : kRW;
    const int per_line = (along - parity) / 2;
    const int total = per_line * across;
    for (int e = tid; e < total; e += kThreads) {
      int line, pos;
      if (horiz) {
        line = e / per_line;
        pos = parity + 2 * (e - line * per_line);
      } else {
        // consecutive threads take consecutive columns (conflict-free smem)
        line = e % across;
        pos = parity + 2 * (e / across);
      }
      const int rr = horiz ? line : pos;
      const int cc = horiz ? pos : line;
      const int i = rr * kRW + cc;
      const int j = horiz ? i + 1 : i + kRW;
      // global coordinates of both endpoints (before wrapping)
      const int gri = r0 - 2 + rr, gci = c0 - 2 + cc;
      const int grj = horiz ? gri : gri + 1, gcj = horiz ? gci + 1 : gci;
      if (!a.periodic) {
        if (gri < 0 || gci < 0 || grj >= H || gcj >= W) continue;
      }
      // cavity of site k: sum of the other four sites
      float ti = 0.f, ni = 0.f, tj = 0.f, nj = 0.f;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        if (s == k) continue;
        ti += sT[s * kRN + i];
        ni += sV[s * kRN + i];
        tj += sT[s * kRN + j];
        nj += sV[s * kRN + j];
      }
      const float ci = __frcp_rn(ti), cj = __frcp_rn(tj);
      const float mi = ni * ci, mj = nj * cj;
      const float mu = mi - mj;
      const float s2 = ci + cj;
      // a_u and the counters take each edge once, from the tile owning its first pixel
      const bool owned = rr >= 2 && rr < 2 + kTH && cc >= 2 && cc < 2 + kTW && gri < H && gci < W;
      float d, q, rho, eab;
      const bool tail = a.fp64_tail && lam > 0.0f && (lam * sqrtf(s2) < 1e-3f);
      if (tail) {
        const double ci_d = 1.0 / (double)ti, cj_d = 1.0 / (double)tj;
        const double mu_d = (double)ni * ci_d - (double)nj * cj_d;
        TiltedOut<double> od = laplace_tilted<double>(mu_d, ci_d + cj_d, lam_d);
        d = (float)od.d;
        q = (float)od.q;
        rho = (float)od.rho;
        eab = (float)od.eab;
        n_fp64 += owned;
      } else {
        TiltedOut<float> o = laplace_tilted<float>(mu, s2, lam);
        d = o.d;
        q = o.q;
        rho = o.rho;
        eab = o.eab;
      }
      // Eq. update_qk_x: tau = 1/Var - 1/c, Var from the projection; cap, then mean
      float tni = rho * __frcp_rn(cj + q * ci);
      float tnj = rho * __frcp_rn(ci + q * cj);
      if (!(tni >= a.min_tau)) { tni = a.min_tau; n_capped += owned; }
      if (!(tnj >= a.min_tau)) { tnj = a.min_tau; n_capped += owned; }
      const float Ei = mi + ci * d;
      const float Ej = mj - cj * d;
      const float nni = tni * Ei + d;   // tau E + (E - m) / c
      const float nnj = tnj * Ej - d;
      float* Tk = sT + k * kRN;
      float* Vk = sV + k * kRN;
      const float ti_new = damp * tni + keep * Tk[i];
      const float tj_new = damp * tnj + keep * Tk[j];
      const float vi_new = damp * nni + keep * Vk[i];
      const float vj_new = damp * nnj + keep * Vk[j];
      Tk[i] = ti_new;
      Tk[j] = tj_new;
      Vk[i] = vi_new;
      Vk[j] = vj_new;
      bad |= !(isfinite(ti_new) && isfinite(tj_new) && isfinite(vi_new) && isfinite(vj_new));
      if (owned) eab_acc += eab;
    }
    __syncthreads();
  }

  // ---- write the tile's four prior-site planes
  for (int idx = tid; idx < kTH * kTW; idx += kThreads) {
    const int tr = idx / kTW, tc = idx - tr * kTW;
    const int gr = r0 + tr, gc = c0 + tc;
    if (gr >= H || gc >= W) continue;
    const long long p = (long long)gr * W + gc;
    const int sidx = (tr + 2) * kRW + tc + 2;
#pragma unroll
    for (int s = 1; s < 5; ++s) {
      a.tout[(s - 1) * N + p] = sT[s * kRN + sidx];
      a.nout[(s - 1) * N + p] = sV[s * kRN + sidx];
    }
  }

  // ---- block partial of a_u in FP64, fixed order
  double v = (double)eab_acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __shared__ double red[kThreads / 32];
  __shared__ unsigned red_cnt[2];
  if (tid == 0) { red_cnt[0] = 0; red_cnt[1] = 0; }
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  if (n_fp64) atomicAdd(&red_cnt[0], n_fp64);
  if (n_capped) atomicAdd(&red_cnt[1], n_capped);
  if (bad) atomicOr(a.status, ST_NONFINITE);
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    a.abar_partial[part] = s;
    if (red_cnt[0]) atomicAdd(&a.counters[DC_FP64], (unsigned long long)red_cnt[0]);
    if (red_cnt[1]) atomicAdd(&a.counters[DC_CAPPED], (unsigned long long)red_cnt[1]);
  }
}

template <bool kSite0FromY>
__global__ void __launch_bounds__(kThreads) prior_sweep_kernel(SweepArgs a) {
  extern __shared__ float smem[];
  prior_tile<kSite0FromY>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, smem);
}

// Many images in one launch: block b belongs to the image whose block range holds
// it (binary search over the first blocks); its tiles are numbered row-major.
__global__ void __launch_bounds__(kThreads) prior_sweep_batch_kernel(const BatchItem* items,
                                                                     int n_items) {
  extern __shared__ float smem[];
  const int b = blockIdx.x;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].block_begin <= b) lo = mid; else hi = mid - 1;
  }
  const BatchItem& it = items[lo];
  const int local = b - it.block_begin;
  const int by = local / it.tiles_x, bx = local - by * it.tiles_x;
  if (it.site0_from_y)
    prior_tile<true>(it.a, bx, by, local, smem);
  else
    prior_tile<false>(it.a, bx, by, local, smem);
}

__global__ void abar_reduce_kernel(const double* partial, int n, double* dscal, double n_pixels,
                                   int do_em) {
  __shared__ double buf[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dscal[DS_ABAR] = buf[0];
    if (do_em) dscal[DS_BETA] = n_pixels / buf[0];
  }
}

}  // namespace

double prior_sweep_bytes_per_pixel(bool site0_from_y) {
  // reads: y (or tau0, nu0) and tau1..4, nu1..4; writes: tau1..4, nu1..4
  return site0_from_y ? (9 + 8) * 4.0 : (10 + 8) * 4.0;
}

int prior_sweep_blocks(int height, int width) {
  return ((width + kTW - 1) / kTW) * ((height + kTH - 1) / kTH);
}

int prior_sweep_tiles_x(int width) { return (width + kTW - 1) / kTW; }

void launch_prior_sweep_batch(const BatchItem* items, int n_items, int total_blocks,
                              cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(prior_sweep_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmemBytes);
    attr = true;
  }
  prior_sweep_batch_kernel<<<total_blocks, kThreads, kSmemBytes, s>>>(items, n_items);
}

void launch_prior_sweep(const SweepArgs& a, bool site0_from_y, cudaStream_t s) {
  dim3 grid((a.width + kTW - 1) / kTW, (a.height + kTH - 1) / kTH);
  if (site0_from_y) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(prior_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSmemBytes);
      attr = true;
    }
    prior_sweep_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(a);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(prior_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSmemBytes);
      attr = true;
    }
    prior_sweep_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(a);
  }
}

void launch_abar_reduce(const double* partial, int n_partial, double* dscal, double n_pixels,
                        int do_em, cudaStream_t s) {
  abar_reduce_kernel<<<1, 1024, 0, s>>>(partial, n_partial, dscal, n_pixels, do_em);
}

}  // namespace eptv
