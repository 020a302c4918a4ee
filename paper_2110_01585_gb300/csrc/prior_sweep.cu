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
// Streaming schedule.  A warp owns a strip of 60 columns and walks down it one
// row pair (2b, 2b+1) at a time; lane l holds columns 2l-2 and 2l-1 of the
// strip (lanes 0 and 31 are the 2-column halo), all five sites of those four
// pixels in registers.  V1 is then inside a lane, V2 pairs a lane's right column
// with the next lane's left column (warp shuffles), V3 is inside a row pair and
// V4 joins the last row of one pair with the first row of the next.  For any
// order of V1..V4, a row pair can take every update ordered before V4 as soon as
// it is loaded; V4 then joins it to the previous pair, which takes the updates
// ordered after V4 and is final.  A sweep reads each site plane once and writes
// each prior-site plane once, plus one halo pair per chunk of rows and the
// 2-column strip halo.  Shared memory is private to each warp (two cp.async
// staging slots for the next row pair, the parked carried row and a copy of the
// loop's arguments: 12.9 KB per warp); there is no block barrier.
//
// Work units are 16 row pairs of one strip.  A persistent grid of warps takes
// contiguous ranges of units (images of a batch laid end to end), so one launch
// serves any number of images.  The E|u| sum of each unit is reduced in FP64 in
// a fixed order and stored in its own slot, which makes the result independent
// of how units are spread over warps.
//
// Arithmetic: FP32 with the cancellation-free forms below; the new precision
// uses tau_i = rho / (c_j + q c_i), which equals 1/Var_i - 1/c_i of Eq. update_qk_x
// (q = Sbar / s^2, rho = 1 - q) without subtracting.  Edges with lam * s < 1e-3
// (where rho is a small difference of O(1) numbers) are redone in FP64 when
// fp64_tail is set.
#include <mutex>

#include "internal.cuh"
#include "mills_poly.cuh"
#include "tilted.cuh"

namespace eptv {

namespace {

constexpr int kStripCols = 60;     // owned columns per warp (lanes 1..30, two each)
constexpr int kStepsPerUnit = 16;  // row-pair steps per work unit
constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
constexpr int kMinBlocks = 3;      // blocks per SM the register budget is sized for

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// ------------------------------------------------------------ tilted moments
//
// Sec. III-C, Eq. marginal_tilted_un: for an edge with cavity means m_i, m_j and
// variances c_i, c_j, the tilted law of u = x_i - x_j is N(u; mu, s^2) exp(-lam|u|),
// mu = m_i - m_j, s^2 = c_i + c_j: two Gaussians truncated at zero.  In standard
// units z = mu / s, l = lam s, a+ = l - z, a- = l + z; for a standard normal
// truncated to [a, inf) let h(a) be the inverse Mills ratio, g = h - a its mean
// offset and v = 1 - h g its variance.  The half weights are w+ = h- / (h+ + h-),
// w- = h+ / (h+ + h-) (the erfcx factors of each half are sqrt(2/pi) / h), and
//   d   = (ubar - mu) / s^2 = [w+ (h+ - l) - w- (h- - l)] / s
//   q   = Sbar / s^2        = w+ v+ + w- v- + w+ w- (g+ + g-)^2
//   rho = 1 - q             = w+ h+ g+ + w- h- g- - w+ w- (g+ + g-)^2
//   eab = E|u|              = s (w+ g+ + w- g-)
// g and v for a >= 0 come from the degree-12 polynomial fits of mills_poly.cuh
// (g within 5e-8, v within 1e-6 relative), so no erfcx is evaluated; for a = -b < 0 the reflection
// Q(-b) = 1 - Q(b) of the upper tail Q gives h(a) = phi(b) h(b) / (h(b) - phi(b)).
// tilted2 below evaluates these in an equivalent sorted form.

struct Moments {
  float d, q, rho, eab;
};

// The same moments in FP64 from the cavity natural parameters (rare; kept out of
// line so that the streaming loop stays small).
__device__ __noinline__ Moments tilted_fp64(float ti, float ni, float tj, float nj, double lam) {
  const double ci = 1.0 / (double)ti, cj = 1.0 / (double)tj;
  const double mu = (double)ni * ci - (double)nj * cj;
  const TiltedOut<double> od = laplace_tilted<double>(mu, ci + cj, lam);
  Moments o;
  o.d = (float)od.d;
  o.q = (float)od.q;
  o.rho = (float)od.rho;
  o.eab = (float)od.eab;
  return o;
}

// ------------------------------------------------------------------ state

struct Px {
  float t[5];  // site precisions, t[0] = likelihood site
  float n[5];  // site precision-times-means
};

struct Row {
  Px x[2];  // the lane's two columns
  bool ok;  // the row exists (always, on the torus)
};

struct Ctx {
  float mlog, v1, v2;   // mixture priors: log((1 - omega) / omega), component variances
  float lam, min_tau, damp, keep;
  double lam_d;
  float tail_s2;  // lam s < 1e-3, i.e. s^2 < 1e-6 / lam^2, takes the FP64 moments (-1: never)
  float eab;  // E|u| of the counted edges of this lane since the last flush
  unsigned n_fp64, n_capped;
  float2 fin;  // sum of the stored site values: non-finite iff one of them is
};

// Geometry of one lane: which of its pixels exist and which it owns.
struct Lane {
  int lane;
  bool col_ok[2];  // column exists (always, on the torus)
  bool right_ok;   // the next lane's left column exists
  bool own_col;    // the lane owns its columns (lanes 1..30, inside the image)
};

template <int K>
__device__ __forceinline__ void cavity(const Px& x, float& ct, float& cn) {
  constexpr int first = K == 0 ? 1 : 0;
  ct = x.t[first];
  cn = x.n[first];
#pragma unroll
  for (int s = first + 1; s < 5; ++s) {
    if (s == K) continue;
    ct += x.t[s];
    cn += x.n[s];
  }
}

// One edge of the current update: cavities of site k at both endpoints in, the
// new (capped, undamped) site k at both endpoints out.
struct Edge {
  float ti, ni, tj, nj;
  bool valid, count;
  float tni, nni, tnj, nnj;
};

// ------------------------------------------- two edges at once, packed FP32
//
// The two edges of an update step run through the same arithmetic, so it is
// written on float2 pairs (edge 0, edge 1) with the packed FP32 FMA/ADD/MUL of
// sm_100-family GPUs: one instruction per operation for both edges.  Constant
// pairs come from the constant bank.

static __constant__ float2 kPairs[5] = {{kMillsK, kMillsK},
                                        {-1.0f, -1.0f},
                                        {1.0f, 1.0f},
                                        {0.398942280f, 0.398942280f},   // 1 / sqrt(2 pi)
                                        {-0.721347520f, -0.721347520f}};  // -log2(e) / 2

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, kPairs[1], a); }
__device__ __forceinline__ float2 rcp2(float2 a) {
  return make_float2(rcp_approx(a.x), rcp_approx(a.y));
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct Mills2 {
  float2 h, g, v;
};

// h, g, v of the polynomial fits at b >= 0 (mills_fast without its reflection).
__device__ __forceinline__ Mills2 mills_fit2(float2 b) {
  const float2 r = rcp2(add2(kPairs[0], b));
  const float2 u = mul2(sub2(kPairs[0], b), r);
  const float2 kr = mul2(kPairs[0], r);
  float2 G = make_float2(kMillsG[kMillsDegree], kMillsG[kMillsDegree]);
  float2 V = make_float2(kMillsV[kMillsDegree], kMillsV[kMillsDegree]);
#pragma unroll
  for (int i = kMillsDegree - 1; i >= 0; --i) {
    G = fma2(G, u, make_float2(kMillsG[i], kMillsG[i]));
    V = fma2(V, u, make_float2(kMillsV[i], kMillsV[i]));
  }
  Mills2 m;
  m.g = mul2(G, kr);
  m.v = mul2(mul2(V, kr), kr);
  m.h = add2(m.g, b);
  return m;
}

struct Moments2 {
  float2 d, q, rho, eab;
};

// tilted_fast for two edges, with the two halves taken in sorted order: for
// az = |z| the truncation points are hi = l + az >= l >= 0 and lo = l - az, and
// only lo can be negative (then its h, g, v come from the reflection).  With
// w_lo = h_hi / (h_lo + h_hi), w_hi = h_lo / (h_lo + h_hi) the moments become
//   d   = -sign(z) lam (h_hi - h_lo) / (h_hi + h_lo)
//   q   = w_lo v_lo + w_hi v_hi + w_lo w_hi (g_lo + g_hi)^2
//   rho = 2 l (g_lo + g_hi) h_lo h_hi / (h_lo + h_hi)^2
//   eab = s (w_lo g_lo + w_hi g_hi)
// (the rho form uses h - g = a on each half and lo + hi = 2 l: a product of
// positive terms, free of cancellation).
__device__ __forceinline__ Moments2 tilted2(float2 mu, float2 s2, float2 lam) {
  const float2 rs = make_float2(rsqrtf(s2.x), rsqrtf(s2.y));
  const float2 s = mul2(s2, rs);
  const float2 z = mul2(mu, rs);
  const float2 az = make_float2(fabsf(z.x), fabsf(z.y));
  const float2 l = mul2(lam, s);
  const float2 hi = add2(l, az), lo = sub2(l, az);
  const float2 b = make_float2(fabsf(lo.x), fabsf(lo.y));
  const Mills2 H = mills_fit2(hi);
  Mills2 L = mills_fit2(b);
  // reflection at lo = -b < 0: h(lo) = phi(b) h(b) / (h(b) - phi(b)), h(b) - phi(b) >= 0.4
  const float2 e = mul2(mul2(b, b), kPairs[4]);
  const float2 phi = mul2(kPairs[3], make_float2(ex2_approx(e.x), ex2_approx(e.y)));
  const float2 hn = mul2(mul2(phi, L.h), rcp2(sub2(L.h, phi)));
  const float2 gn = add2(hn, b);
  const float2 vn = sub2(kPairs[2], mul2(hn, gn));
  if (lo.x < 0.0f) { L.h.x = hn.x; L.g.x = gn.x; L.v.x = vn.x; }
  if (lo.y < 0.0f) { L.h.y = hn.y; L.g.y = gn.y; L.v.y = vn.y; }
  const float2 inv = rcp2(add2(H.h, L.h));  // not both h vanish
  const float2 wl = mul2(H.h, inv), wh = mul2(L.h, inv);
  Moments2 o;
  const float2 dm = mul2(mul2(sub2(H.h, L.h), inv), lam);
  o.d = make_float2(copysignf(dm.x, -z.x), copysignf(dm.y, -z.y));
  const float2 gs = add2(L.g, H.g);
  o.q = add2(fma2(wl, L.v, mul2(wh, H.v)), mul2(mul2(wl, wh), mul2(gs, gs)));
  o.rho = mul2(mul2(gs, mul2(wl, L.h)), mul2(add2(l, l), inv));
  o.eab = mul2(s, fma2(wl, L.g, mul2(wh, H.g)));
  return o;
}

// Tilted moments of the two-Gaussian edge factors of Sec. II-B (Eq. MoG2_TV_prior,
// and Eq. BG_TV as v2 = 0):
//   P(u) ~ N(u; mu, s2) [omega N(u; 0, v1) + (1 - omega) N(u; 0, v2)]
//        = W1 N(u; m1, c1) + W2 N(u; m2, c2),  m_k = mu v_k / e_k,  c_k = v_k s2 / e_k,
// e_k = v_k + s2, W1 : W2 = omega N(mu; 0, e1) : (1 - omega) N(mu; 0, e2), i.e.
// W2 = 1 / (1 + exp(-t)) with t = log((1 - omega) / omega) + log(e1 / e2) / 2
// - mu^2 (v1 - v2) / (2 e1 e2).  In the units of the edge update:
//   d   = (ubar - mu) / s2 = -mu (W1 / e1 + W2 / e2)
//   q   = Sbar / s2 = W1 v1 / e1 + W2 v2 / e2 + W1 W2 (m1 - m2)^2 / s2
//   rho = 1 - q = s2 (W1 / e1 + W2 / e2 - W1 W2 mu^2 (v1 - v2)^2 / (e1 e2)^2)
// using m1 - m2 = mu s2 (v1 - v2) / (e1 e2).  rho < 0 (more spread than the
// cavity) happens for these priors, which are not log-concave; the edge update
// then caps the new site.  No EM statistic (eab = 0): EM is for l1-TV only.
__device__ __forceinline__ void mixture_moments(float mu, float s2, float mlog, float v1, float v2,
                                                float& d, float& q, float& rho) {
  const float e1 = v1 + s2, e2 = v2 + s2;
  const float r1 = 1.0f / e1, r2 = 1.0f / e2;
  const float dv = v1 - v2;
  const float t = mlog + 0.5f * logf(e1 * r2) - 0.5f * mu * mu * dv * r1 * r2;
  const float w2 = 1.0f / (1.0f + expf(-t)), w1 = 1.0f / (1.0f + expf(t));
  const float a = w1 * r1 + w2 * r2;
  const float sep = w1 * w2 * mu * mu * dv * dv * (r1 * r2) * (r1 * r2);
  d = -mu * a;
  q = w1 * v1 * r1 + w2 * v2 * r2 + s2 * sep;
  rho = s2 * (a - sep);
}

// The two independent edges of one update step; the FP64 moments replace the
// packed ones for the edges that need them.  Eq. update_qk_x from the tilted moments:
// tau = rho / (c_j + q c_i), the variance cap, then nu = tau E + (E - m) / c.
// kEdge (a separate instantiation each, so that the default code keeps its own
// register allocation): kEdgeL1, l1-TV with the EM statistic E_{P_k}|u| of
// Option 3 (Eq. 3rd_alternative_a0); kEdgeL1Q, l1-TV with E|u| under the
// matched Gaussian Q(u_n) = N(ubar, Sbar) of Option 2 (Eq. au); kEdgeMix, the
// mixture priors (no EM statistic).
enum : int { kEdgeL1 = 0, kEdgeL1Q = 1, kEdgeMix = 2 };

// E|u| for u ~ N(m, v): sqrt(v) sqrt(2/pi) exp(-m^2 / (2 v)) + m erf(m / sqrt(2 v)).
__device__ __forceinline__ float folded_mean(float m, float v) {
  const float r = rsqrtf(v);
  return v * r * 0.797884561f * expf(-0.5f * m * m / v) + m * erff(0.707106781f * m * r);
}

template <int kEdge>
__device__ __forceinline__ void edges2(Ctx& c, Edge& e0, Edge& e1) {
  constexpr bool kMix = kEdge == kEdgeMix;
  const float2 ti = make_float2(e0.ti, e1.ti), tj = make_float2(e0.tj, e1.tj);
  const float2 ci = rcp2(ti), cj = rcp2(tj);
  const float2 mi = mul2(make_float2(e0.ni, e1.ni), ci);
  const float2 mj = mul2(make_float2(e0.nj, e1.nj), cj);
  const float2 s2 = add2(ci, cj);
  const float2 mu = sub2(mi, mj);
  Moments2 o;
  if (kMix) {
    // closed forms in FP32
    mixture_moments(mu.x, s2.x, c.mlog, c.v1, c.v2, o.d.x, o.q.x, o.rho.x);
    mixture_moments(mu.y, s2.y, c.mlog, c.v1, c.v2, o.d.y, o.q.y, o.rho.y);
    o.eab = make_float2(0.0f, 0.0f);
  } else {
    const bool t0 = s2.x < c.tail_s2;  // an invalid edge here costs time only
    const bool t1 = s2.y < c.tail_s2;
    o = tilted2(mu, s2, make_float2(c.lam, c.lam));
    if (t0 || t1) {
      // one call site for both edges keeps the rare path small
#pragma unroll 1
      for (int k = 0; k < 2; ++k) {
        if (!(k ? t1 : t0)) continue;
        const Moments a = tilted_fp64(k ? e1.ti : e0.ti, k ? e1.ni : e0.ni, k ? e1.tj : e0.tj,
                                      k ? e1.nj : e0.nj, c.lam_d);
        if (k) { o.d.y = a.d; o.q.y = a.q; o.rho.y = a.rho; o.eab.y = a.eab; }
        else   { o.d.x = a.d; o.q.x = a.q; o.rho.x = a.rho; o.eab.x = a.eab; }
      }
      c.n_fp64 += (t0 && e0.valid && e0.count) + (t1 && e1.valid && e1.count);
    }
    if (kEdge == kEdgeL1Q) {
      // Option 2: E|u| under N(ubar, Sbar), ubar = mu + s^2 d, Sbar = q s^2
      o.eab.x = folded_mean(fmaf(s2.x, o.d.x, mu.x), o.q.x * s2.x);
      o.eab.y = folded_mean(fmaf(s2.y, o.d.y, mu.y), o.q.y * s2.y);
    }
  }
  float2 tni = mul2(o.rho, rcp2(fma2(o.q, ci, cj)));
  float2 tnj = mul2(o.rho, rcp2(fma2(o.q, cj, ci)));
  const bool k0 = e0.valid && e0.count, k1 = e1.valid && e1.count;
  if (!(tni.x >= c.min_tau && tnj.x >= c.min_tau && tni.y >= c.min_tau && tnj.y >= c.min_tau)) {
    // rare: some new precision is below the cap (or not a number)
    if (!(tni.x >= c.min_tau)) { tni.x = c.min_tau; c.n_capped += k0; }
    if (!(tnj.x >= c.min_tau)) { tnj.x = c.min_tau; c.n_capped += k0; }
    if (!(tni.y >= c.min_tau)) { tni.y = c.min_tau; c.n_capped += k1; }
    if (!(tnj.y >= c.min_tau)) { tnj.y = c.min_tau; c.n_capped += k1; }
  }
  const float2 nd = mul2(o.d, kPairs[1]);
  const float2 nni = fma2(tni, fma2(ci, o.d, mi), o.d);  // tau E + (E - m) / c
  const float2 nnj = fma2(tnj, fma2(cj, nd, mj), nd);
  e0.tni = tni.x; e1.tni = tni.y;
  e0.tnj = tnj.x; e1.tnj = tnj.y;
  e0.nni = nni.x; e1.nni = nni.y;
  e0.nnj = nnj.x; e1.nnj = nnj.y;
  if (k0) c.eab += o.eab.x;
  if (k1) c.eab += o.eab.y;
}

template <int K>
__device__ __forceinline__ void damp_into(const Ctx& c, Px& x, bool valid, float tn, float nn) {
  if (valid) {
    x.t[K] = c.damp * tn + c.keep * x.t[K];
    x.n[K] = c.damp * nn + c.keep * x.n[K];
  }
}

// Gather and scatter of the update steps.  A step updates site K on two
// independent edges; the gather forms the cavities of site K at their endpoints,
// edges2 computes the new sites, the scatter damps them into place.
//   h1: V1, the edge (2a, 2a+1) inside the lane, on rows a and b
//   h2: V2, the edge (2a+1, 2a+2) from a lane's right column to the next lane's
//       left column, on rows a and b; the lane on the left computes it
//   v:  V3 or V4 between vertically adjacent rows, both columns of the lane
__device__ __forceinline__ void gather_h1(const Lane& L, const Row& a, const Row& b, bool cnt_a,
                                          bool cnt_b, Edge& e0, Edge& e1) {
  cavity<1>(a.x[0], e0.ti, e0.ni);
  cavity<1>(a.x[1], e0.tj, e0.nj);
  cavity<1>(b.x[0], e1.ti, e1.ni);
  cavity<1>(b.x[1], e1.tj, e1.nj);
  const bool cols = L.col_ok[0] && L.col_ok[1];
  e0.valid = a.ok && cols;
  e1.valid = b.ok && cols;
  e0.count = cnt_a && L.own_col;
  e1.count = cnt_b && L.own_col;
}

__device__ __forceinline__ void scatter_h1(const Ctx& c, Row& a, Row& b, const Edge& e0,
                                           const Edge& e1) {
  damp_into<1>(c, a.x[0], e0.valid, e0.tni, e0.nni);
  damp_into<1>(c, a.x[1], e0.valid, e0.tnj, e0.nnj);
  damp_into<1>(c, b.x[0], e1.valid, e1.tni, e1.nni);
  damp_into<1>(c, b.x[1], e1.valid, e1.tnj, e1.nnj);
}

__device__ __forceinline__ void gather_h2(const Lane& L, const Row& a, const Row& b, bool cnt_a,
                                          bool cnt_b, Edge& e0, Edge& e1) {
  float tla, nla, tlb, nlb;
  cavity<2>(a.x[0], tla, nla);
  cavity<2>(a.x[1], e0.ti, e0.ni);
  cavity<2>(b.x[0], tlb, nlb);
  cavity<2>(b.x[1], e1.ti, e1.ni);
  e0.tj = __shfl_down_sync(0xffffffffu, tla, 1);
  e0.nj = __shfl_down_sync(0xffffffffu, nla, 1);
  e1.tj = __shfl_down_sync(0xffffffffu, tlb, 1);
  e1.nj = __shfl_down_sync(0xffffffffu, nlb, 1);
  const bool cols = L.col_ok[1] && L.right_ok && L.lane < 31;
  e0.valid = a.ok && cols;
  e1.valid = b.ok && cols;
  e0.count = cnt_a && L.own_col;
  e1.count = cnt_b && L.own_col;
}

__device__ __forceinline__ void scatter_h2(const Ctx& c, const Lane& L, Row& a, Row& b,
                                           const Edge& e0, const Edge& e1) {
  const float rta = __shfl_up_sync(0xffffffffu, e0.tnj, 1);
  const float rna = __shfl_up_sync(0xffffffffu, e0.nnj, 1);
  const float rtb = __shfl_up_sync(0xffffffffu, e1.tnj, 1);
  const float rnb = __shfl_up_sync(0xffffffffu, e1.nnj, 1);
  const unsigned va = __shfl_up_sync(0xffffffffu, e0.valid ? 1u : 0u, 1);
  const unsigned vb = __shfl_up_sync(0xffffffffu, e1.valid ? 1u : 0u, 1);
  damp_into<2>(c, a.x[1], e0.valid, e0.tni, e0.nni);
  damp_into<2>(c, b.x[1], e1.valid, e1.tni, e1.nni);
  damp_into<2>(c, a.x[0], va && L.lane > 0, rta, rna);
  damp_into<2>(c, b.x[0], vb && L.lane > 0, rtb, rnb);
}

template <int K>
__device__ __forceinline__ void gather_v(const Lane& L, const Row& top, const Row& bot, bool cnt,
                                         Edge& e0, Edge& e1) {
  cavity<K>(top.x[0], e0.ti, e0.ni);
  cavity<K>(bot.x[0], e0.tj, e0.nj);
  cavity<K>(top.x[1], e1.ti, e1.ni);
  cavity<K>(bot.x[1], e1.tj, e1.nj);
  const bool rows = top.ok && bot.ok;
  e0.valid = rows && L.col_ok[0];
  e1.valid = rows && L.col_ok[1];
  e0.count = cnt && L.own_col;
  e1.count = cnt && L.own_col;
}

template <int K>
__device__ __forceinline__ void scatter_v(const Ctx& c, Row& top, Row& bot, const Edge& e0,
                                          const Edge& e1) {
  damp_into<K>(c, top.x[0], e0.valid, e0.tni, e0.nni);
  damp_into<K>(c, bot.x[0], e0.valid, e0.tnj, e0.nnj);
  damp_into<K>(c, top.x[1], e1.valid, e1.tni, e1.nni);
  damp_into<K>(c, bot.x[1], e1.valid, e1.tnj, e1.nnj);
}

// Row staging.  Each lane copies its own two pixels of every site plane of the
// next row pair into shared memory with cp.async while it computes on the
// current pair; a warp owns kSlots pair slots of [plane][row][lane] float2.
constexpr int kSlots = 2;
constexpr int kMaxPlanes = 10;
constexpr int kSlotFloats2 = kMaxPlanes * 2 * 32;
constexpr int kCarryFloats2 = 10 * 32;  // the carried row between steps: [t0..t4, n0..n4][lane]
constexpr size_t kSmemPerWarp = size_t(kSlots) * kSlotFloats2 * sizeof(float2);
constexpr size_t kCarryBytes = size_t(kCarryFloats2) * sizeof(float2);
constexpr size_t kIoBytes = 128;  // per-warp copy of the loop's argument fields
constexpr size_t kWarpSmem = kSmemPerWarp + kCarryBytes + kIoBytes;
constexpr size_t kSmemBytes = kWarpSmem * kWarpsPerBlock;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// The fields of SweepArgs the streaming loop touches.  Each warp keeps a copy in
// shared memory and reads it at every use: cheap loads that cost no registers.
struct __align__(16) Io {
  const float* s0;   // y (site 0 from y) or tau0
  const float* s1;   // nu0
  const float* tin;
  const float* nin;
  float* tout;
  float* nout;
  int n;             // plane stride (pixels; images are below 2^31 pixels)
  int height, width;
  bool periodic, vec2;  // periodic: the rows wrap (columns: SweepArgs::periodic)
  float inv_xi;
};

static_assert(sizeof(Io) <= kIoBytes, "argument copy exceeds its shared-memory slot");

__device__ __forceinline__ Io make_io(const SweepArgs& a, bool site0_from_y) {
  Io io;
  io.s0 = site0_from_y ? a.y : a.tau0;
  io.s1 = a.nu0;
  io.tin = a.tin;
  io.nin = a.nin;
  io.tout = a.tout;
  io.nout = a.nout;
  io.n = (int)a.n;
  io.height = a.height;
  io.width = a.width;
  io.periodic = a.periodic_rows != 0;
  io.vec2 = a.vec2 != 0;
  io.inv_xi = a.inv_xi;
  return io;
}

// Image row of the (unwrapped) row index r and whether it exists.
__device__ __forceinline__ int image_row(const Io& io, int r, bool& ok) {
  if (io.periodic) {
    if (r < 0) r += io.height;
    if (r >= io.height) r -= io.height;
    if (r < 0 || r >= io.height) r = wrap(r, io.height);  // tiny heights
    ok = true;
    return r;
  }
  ok = r >= 0 && r < io.height;
  return r;
}

// One 8- or 4-byte cp.async to a shared address plus an immediate offset; a zero
// source size writes zeros and reads nothing.
template <int kBytes, int kOff>
__device__ __forceinline__ void cp_async_imm(unsigned dst, const float* src, int src_size) {
  if (kBytes == 8)
    asm volatile("cp.async.ca.shared.global [%0+%1], [%2], 8, %3;\n" ::"r"(dst), "n"(kOff), "l"(src),
                 "r"(src_size));
  else
    asm volatile("cp.async.ca.shared.global [%0+%1], [%2], 4, %3;\n" ::"r"(dst), "n"(kOff), "l"(src),
                 "r"(src_size));
}

// Copies of one pixel column (kBytes = 8: both pixels of the lane) of every
// staged plane: site 0 (y, or tau0 and nu0), then tau1..4, nu1..4, one plane
// every 64 float2 of the slot.
template <bool kSite0FromY, int kBytes>
__device__ __forceinline__ void issue_planes(const float* s0, const float* s1, const float* tin,
                                             const float* nin, int n, int p, unsigned dst, int size) {
  constexpr int k0 = kSite0FromY ? 1 : 2;
  cp_async_imm<kBytes, 0>(dst, s0 + p, size);
  if (!kSite0FromY) cp_async_imm<kBytes, 512>(dst, s1 + p, size);
  const float* t = tin + p;
  const float* m = nin + p;
  cp_async_imm<kBytes, (k0 + 0) * 512>(dst, t, size);
  cp_async_imm<kBytes, (k0 + 1) * 512>(dst, t + n, size);
  cp_async_imm<kBytes, (k0 + 2) * 512>(dst, t + 2 * n, size);
  cp_async_imm<kBytes, (k0 + 3) * 512>(dst, t + 3 * n, size);
  cp_async_imm<kBytes, (k0 + 4) * 512>(dst, m, size);
  cp_async_imm<kBytes, (k0 + 5) * 512>(dst, m + n, size);
  cp_async_imm<kBytes, (k0 + 6) * 512>(dst, m + 2 * n, size);
  cp_async_imm<kBytes, (k0 + 7) * 512>(dst, m + 3 * n, size);
}

// Issues the copies of image row gr (already wrapped; ok = it exists) into row
// slot r of pair slot `slot`.
template <bool kSite0FromY>
__device__ __forceinline__ void issue_row(const Io& io_ref, const Lane& L, const int (&gcol)[2],
                                          int gr, bool ok, float2* stage, int slot, int r) {
  const float* s0 = io_ref.s0;
  const float* s1 = io_ref.s1;
  const float* tin = io_ref.tin;
  const float* nin = io_ref.nin;
  const int n = io_ref.n;
  const int base = ok ? gr * io_ref.width : 0;
  const unsigned dst =
      (unsigned)__cvta_generic_to_shared(stage + slot * kSlotFloats2 + r * 32 + L.lane);
  if (io_ref.vec2) {
    const bool fill = ok && L.col_ok[0];
    issue_planes<kSite0FromY, 8>(s0, s1, tin, nin, n, fill ? base + gcol[0] : 0, dst, fill ? 8 : 0);
  } else {
    const bool f0 = ok && L.col_ok[0], f1 = ok && L.col_ok[1];
    issue_planes<kSite0FromY, 4>(s0, s1, tin, nin, n, f0 ? base + gcol[0] : 0, dst, f0 ? 4 : 0);
    issue_planes<kSite0FromY, 4>(s0, s1, tin, nin, n, f1 ? base + gcol[1] : 0, dst + 4, f1 ? 4 : 0);
  }
}

// Reads a staged row into registers (missing pixels read as zeros and are never
// the endpoint of a valid edge).
template <bool kSite0FromY>
__device__ __forceinline__ void read_row(const Io& io, const Lane& L, const float2* stage, int slot,
                                         int r, bool ok, Row& R) {
  const float2* src = stage + slot * kSlotFloats2 + r * 32 + L.lane;
  R.ok = ok;
  int q = 0;
  if (kSite0FromY) {
    const float2 y = src[0];
    R.x[0].t[0] = io.inv_xi;
    R.x[1].t[0] = io.inv_xi;
    R.x[0].n[0] = y.x * io.inv_xi;
    R.x[1].n[0] = y.y * io.inv_xi;
    q = 1;
  } else {
    const float2 t = src[0], n = src[64];
    R.x[0].t[0] = t.x;
    R.x[1].t[0] = t.y;
    R.x[0].n[0] = n.x;
    R.x[1].n[0] = n.y;
    q = 2;
  }
#pragma unroll
  for (int s = 1; s < 5; ++s) {
    const float2 t = src[(q + s - 1) * 64];
    const float2 n = src[(q + 4 + s - 1) * 64];
    R.x[0].t[s] = t.x;
    R.x[1].t[s] = t.y;
    R.x[0].n[s] = n.x;
    R.x[1].n[s] = n.y;
  }
}

// Stores a final row; gr is the unwrapped row index (rows outside [0, H) are
// torus copies or do not exist and are not stored).
__device__ __forceinline__ void store_row(const Io& io_ref, Ctx& c, const Lane& L,
                                          const int (&gcol)[2], int gr, const Row& R) {
  const int H = io_ref.height;
  if (!L.own_col || gr < 0 || gr >= H) return;
  const int n = io_ref.n;
  const int base = gr * io_ref.width;
  float* t = io_ref.tout;
  float* m = io_ref.nout;
  if (io_ref.vec2) {
    t += base + gcol[0];
    m += base + gcol[0];
#pragma unroll
    for (int s = 1; s < 5; ++s) {
      const float2 tv = make_float2(R.x[0].t[s], R.x[1].t[s]);
      const float2 nv = make_float2(R.x[0].n[s], R.x[1].n[s]);
      *reinterpret_cast<float2*>(t) = tv;
      *reinterpret_cast<float2*>(m) = nv;
      t += n;
      m += n;
      c.fin = add2(c.fin, add2(tv, nv));
    }
  } else {
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!L.col_ok[k]) continue;
      float* tk = t + base + gcol[k];
      float* mk = m + base + gcol[k];
#pragma unroll
      for (int s = 1; s < 5; ++s) {
        *tk = R.x[k].t[s];
        *mk = R.x[k].n[s];
        tk += n;
        mk += n;
        sum += R.x[k].t[s] + R.x[k].n[s];
      }
    }
    c.fin.x += sum;
  }
}

// Warp sum of the lanes' E|u| in FP64 (fixed tree), stored in the unit's slot.
__device__ __forceinline__ void flush_unit(double* abar_partial, float lane_sum, long long unit) {
  double v = (double)lane_sum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) abar_partial[unit] = v;
}

// One update step of a known kind: 1, 2 (V1, V2 on the pair r0, r1), 3 or 4 (the
// in-pair vertical update kI on r0, r1), 0 (kX joining carry and r0), 5 and 6
// (V1, V2 after kX on carry and r0).
template <int kKind, int kX, int kI, int kEdge>
__device__ __forceinline__ void do_step(Ctx& c, const Lane& L, Row& carry, Row& r0, Row& r1, bool cc,
                                        bool c0, bool c1) {
  Edge e0, e1;
  if (kKind == 1) gather_h1(L, r0, r1, c0, c1, e0, e1);
  else if (kKind == 2) gather_h2(L, r0, r1, c0, c1, e0, e1);
  else if (kKind == 0) gather_v<kX>(L, carry, r0, cc, e0, e1);
  else if (kKind == 5) gather_h1(L, carry, r0, cc, c0, e0, e1);
  else if (kKind == 6) gather_h2(L, carry, r0, cc, c0, e0, e1);
  else gather_v<kI>(L, r0, r1, c0, e0, e1);
  edges2<kEdge>(c, e0, e1);
  if (kKind == 1) scatter_h1(c, r0, r1, e0, e1);
  else if (kKind == 2) scatter_h2(c, L, r0, r1, e0, e1);
  else if (kKind == 0) scatter_v<kX>(c, carry, r0, e0, e1);
  else if (kKind == 5) scatter_h1(c, carry, r0, e0, e1);
  else if (kKind == 6) scatter_h2(c, L, carry, r0, e0, e1);
  else scatter_v<kI>(c, r0, r1, e0, e1);
}

// The carried row waits in shared memory while the next pair takes its updates
// before kX (registers are the occupancy limit); [plane][lane] float2 layout.
__device__ __forceinline__ void save_row(float2* dst, const Row& R) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    dst[s * 32] = make_float2(R.x[0].t[s], R.x[1].t[s]);
    dst[(5 + s) * 32] = make_float2(R.x[0].n[s], R.x[1].n[s]);
  }
}

__device__ __forceinline__ void load_saved_row(const float2* src, bool ok, Row& R) {
  R.ok = ok;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const float2 t = src[s * 32], n = src[(5 + s) * 32];
    R.x[0].t[s] = t.x;
    R.x[1].t[s] = t.y;
    R.x[0].n[s] = n.x;
    R.x[1].n[s] = n.y;
  }
}

// Steps per strip: step b finalises rows 2b - o - 1 and 2b - o (o = 0 when V4 is
// the later vertical update of the order, 1 when V3 is); one spare step covers
// both offsets and odd heights.
__host__ __device__ __forceinline__ int steps_of(int height) { return (height + 1) / 2 + 1; }
__host__ __device__ __forceinline__ int units_per_strip(int height) {
  return (steps_of(height) + kStepsPerUnit - 1) / kStepsPerUnit;
}
__host__ __device__ __forceinline__ int strips_of(int width) {
  return (width + kStripCols - 1) / kStripCols;
}

// Position of the update k in the order word.
__device__ __forceinline__ int order_pos(int order, int k) {
  int t = 0;
  while (t < 3 && ((order >> (4 * t)) & 0xF) != k) ++t;
  return t;
}

// Steps [b_lo, b_hi) of one strip.  kX is the later of V3 and V4 in the update
// order: it joins consecutive row pairs, the other (kI) lies inside a pair.
// Step b loads the pair of rows (2b - o, 2b - o + 1), applies the updates ordered
// before kX to it, joins its first row to the carried last row of the previous
// pair by kX, applies the updates ordered after kX (horizontal ones only) to
// those two rows, which are then final, and carries its second row on.
template <bool kSite0FromY, int kX, int kEdge>
__device__ __noinline__ void run_strip(const SweepArgs& a, int strip, int b_lo, int b_hi,
                                       long long unit_base, float2* stage) {
  constexpr int kI = 7 - kX;
  constexpr int kOff = kX == 4 ? 0 : 1;
  const int W = a.width, H = a.height;
  Lane L;
  L.lane = threadIdx.x & 31;
  const int gc0 = strip * kStripCols - 2 + 2 * L.lane;  // unwrapped column of the left pixel
  int gcol[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int g = gc0 + k;
    if (a.periodic) {
      gcol[k] = wrap(g, W);
      L.col_ok[k] = true;
    } else {
      gcol[k] = g;
      L.col_ok[k] = g >= 0 && g < W;
    }
  }
  L.right_ok = a.periodic || (gc0 + 2 >= 0 && gc0 + 2 < W);
  L.own_col = L.lane >= 1 && L.lane <= 30 && gc0 < W;

  Ctx c;
  c.mlog = a.mix_logit;
  c.v1 = a.mix_v1;
  c.v2 = a.mix_v2;
  c.lam = (float)(*a.beta);
  c.lam_d = *a.beta;
  c.tail_s2 = (a.fp64_tail && c.lam > 0.0f) ? 1e-6f / (c.lam * c.lam) : -1.0f;
  c.min_tau = a.min_tau;
  c.damp = a.damping;
  c.keep = 1.0f - a.damping;
  c.eab = 0.0f;
  c.n_fp64 = 0;
  c.n_capped = 0;
  c.fin = make_float2(0.0f, 0.0f);
  const int order = a.order;
  const int posX = order_pos(order, kX);
  float2* const carry_smem = stage + kSlots * kSlotFloats2 + L.lane;
  Io* const io_smem = reinterpret_cast<Io*>(stage + kSlots * kSlotFloats2 + kCarryFloats2);
  if (L.lane == 0) *io_smem = make_io(a, kSite0FromY);
  __syncwarp();
  const Io& io = *io_smem;
  double* const abar_partial = a.abar_partial;

  // Step b_lo - 1 only applies the updates before kX to its pair, whose second
  // row is carried into step b_lo.  Pair b lives in staging slot b & 1.
  Row r0, r1;
  bool nok0, nok1, carry_ok = false;
  {
    const int rw = 2 * (b_lo - 1) - kOff;
    const int g0 = image_row(io, rw, nok0), g1 = image_row(io, rw + 1, nok1);
    issue_row<kSite0FromY>(io, L, gcol, g0, nok0, stage, (b_lo - 1) & 1, 0);
    issue_row<kSite0FromY>(io, L, gcol, g1, nok1, stage, (b_lo - 1) & 1, 1);
    cp_async_commit();
  }
  for (int b = b_lo - 1; b < b_hi; ++b) {
    const bool warm = b < b_lo;
    const int row0 = 2 * b - kOff;
    const bool ok0 = nok0, ok1 = nok1;
    if (b + 1 < b_hi) {
      // slot (b + 1) & 1 held pair b - 1, already read
      const int g0 = image_row(io, row0 + 2, nok0), g1 = image_row(io, row0 + 3, nok1);
      issue_row<kSite0FromY>(io, L, gcol, g0, nok0, stage, (b + 1) & 1, 0);
      issue_row<kSite0FromY>(io, L, gcol, g1, nok1, stage, (b + 1) & 1, 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    read_row<kSite0FromY>(io, L, stage, b & 1, 0, ok0, r0);
    read_row<kSite0FromY>(io, L, stage, b & 1, 1, ok1, r1);
    // an edge is counted by the step that computes it for its first pixel's row
    // in [count_lo, count_hi) (rows outside are torus copies, do not exist, or
    // belong to another block of a sharded image)
    const int clo = a.count_lo, chi = a.count_hi;
    const bool cc = !warm && row0 - 1 >= clo && row0 - 1 < chi;
    const bool c0 = !warm && row0 >= clo && row0 < chi;
    const bool c1 = !warm && row0 + 1 >= clo && row0 + 1 < chi;
    Row carry;
    if (kX == 4 && order == 0x4321) {
      // the default order V1, V2, V3, V4 as straight-line code
      do_step<1, kX, kI, kEdge>(c, L, carry, r0, r1, cc, c0, c1);
      do_step<2, kX, kI, kEdge>(c, L, carry, r0, r1, cc, c0, c1);
      do_step<kI, kX, kI, kEdge>(c, L, carry, r0, r1, cc, c0, c1);
      if (!warm) {
        load_saved_row(carry_smem, carry_ok, carry);
        save_row(carry_smem, r1);  // r1 is final for this step: frees its registers
        do_step<0, kX, kI, kEdge>(c, L, carry, r0, r1, cc, c0, c1);
      } else {
        save_row(carry_smem, r1);
      }
    } else {
      const int nt = warm ? posX : 4;
      for (int t = 0; t < nt; ++t) {
        const int k = (order >> (4 * t)) & 0xF;
        // 1, 2, kI: updates before kX on this pair; 0: kX; 5, 6: V1, V2 after kX
        const int kind = t < posX ? k : (t == posX ? 0 : 4 + k);
        if (kind == 0) {  // r1 takes no update from kX on
          load_saved_row(carry_smem, carry_ok, carry);
          save_row(carry_smem, r1);
        }
        Edge e0, e1;
        if (kind == 1) gather_h1(L, r0, r1, c0, c1, e0, e1);
        else if (kind == 2) gather_h2(L, r0, r1, c0, c1, e0, e1);
        else if (kind == 0) gather_v<kX>(L, carry, r0, cc, e0, e1);
        else if (kind == 5) gather_h1(L, carry, r0, cc, c0, e0, e1);
        else if (kind == 6) gather_h2(L, carry, r0, cc, c0, e0, e1);
        else gather_v<kI>(L, r0, r1, c0, e0, e1);
        edges2<kEdge>(c, e0, e1);
        if (kind == 1) scatter_h1(c, r0, r1, e0, e1);
        else if (kind == 2) scatter_h2(c, L, r0, r1, e0, e1);
        else if (kind == 0) scatter_v<kX>(c, carry, r0, e0, e1);
        else if (kind == 5) scatter_h1(c, carry, r0, e0, e1);
        else if (kind == 6) scatter_h2(c, L, carry, r0, e0, e1);
        else scatter_v<kI>(c, r0, r1, e0, e1);
      }
      if (warm) save_row(carry_smem, r1);
    }
    if (!warm) {
      store_row(io, c, L, gcol, row0 - 1, carry);
      store_row(io, c, L, gcol, row0, r0);
      if ((b + 1) % kStepsPerUnit == 0 || b + 1 == b_hi) {
        flush_unit(abar_partial, c.eab, unit_base + b / kStepsPerUnit);
        c.eab = 0.0f;
      }
    }
    carry_ok = r1.ok;
  }
  if (!isfinite(c.fin.x + c.fin.y)) atomicOr(a.status, ST_NONFINITE);
  if (c.n_fp64) atomicAdd(&a.counters[DC_FP64], (unsigned long long)c.n_fp64);
  if (c.n_capped) atomicAdd(&a.counters[DC_CAPPED], (unsigned long long)c.n_capped);
}

// The later of V3 and V4 in an order word.
__host__ __device__ __forceinline__ int later_vertical(int order) {
  for (int t = 3; t >= 0; --t) {
    const int k = (order >> (4 * t)) & 0xF;
    if (k == 3 || k == 4) return k;
  }
  return 4;
}

// Units [u_lo, u_hi) of one image (strip-major: unit = strip * units_per_strip + block).
template <bool kSite0FromY, int kX, int kEdge>
__device__ void run_units(const SweepArgs& a, long long u_lo, long long u_hi, float2* stage) {
  const int ups = units_per_strip(a.height);
  const int nsteps = steps_of(a.height);
  long long u = u_lo;
  while (u < u_hi) {
    const int strip = (int)(u / ups);
    const long long strip_end = (long long)(strip + 1) * ups;
    const long long e = u_hi < strip_end ? u_hi : strip_end;
    const int k_lo = (int)(u - (long long)strip * ups), k_hi = (int)(e - (long long)strip * ups);
    run_strip<kSite0FromY, kX, kEdge>(a, strip, k_lo * kStepsPerUnit, min(k_hi * kStepsPerUnit, nsteps),
                               (long long)strip * ups, stage);
    u = e;
  }
}

template <bool kSite0FromY, int kEdge>
__device__ __forceinline__ void run_units_any(const SweepArgs& a, long long u_lo, long long u_hi,
                                              float2* stage) {
  if (later_vertical(a.order) == 4)
    run_units<kSite0FromY, 4, kEdge>(a, u_lo, u_hi, stage);
  else
    run_units<kSite0FromY, 3, kEdge>(a, u_lo, u_hi, stage);
}

// The edge variant of an image's arguments.
__host__ __device__ __forceinline__ int edge_kind(const SweepArgs& a) {
  return a.prior != EP_TV_PRIOR_L1 ? kEdgeMix : (a.em_option == 2 ? kEdgeL1Q : kEdgeL1);
}

// Staging slots of this warp, followed by its argument copy.
__device__ __forceinline__ float2* warp_stage() {
  extern __shared__ float2 stage_all[];
  return stage_all + (threadIdx.x >> 5) * (kWarpSmem / sizeof(float2));
}

__device__ __forceinline__ int global_warp() { return blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); }

// One image: warp w takes strip w % S and the w / S-th of n_seg contiguous
// ranges of that strip's units, so that the warps on neighbouring strips walk
// the same rows at the same time (the strips' halo columns meet in L2).
template <bool kSite0FromY, int kX, int kEdge>
__global__ void __launch_bounds__(kThreads, kMinBlocks) prior_sweep_kernel(SweepArgs a, int n_seg) {
  const int S = strips_of(a.width);
  const int w = global_warp();
  if (w >= S * n_seg) return;
  const int strip = w % S, seg = w / S;
  const long long ups = units_per_strip(a.height);
  const long long lo = ups * seg / n_seg, hi = ups * (seg + 1) / n_seg;
  if (lo < hi) run_units<kSite0FromY, kX, kEdge>(a, strip * ups + lo, strip * ups + hi, warp_stage());
}

// Many images in one launch; units of image i start at items[i].unit_begin and
// warp w of n_warps takes units [U w / n_warps, U (w + 1) / n_warps).
__global__ void __launch_bounds__(kThreads, kMinBlocks) prior_sweep_batch_kernel(const BatchItem* items,
                                                                     int n_items, long long total,
                                                                     int n_warps) {
  const int w = global_warp();
  if (w >= n_warps) return;
  const long long lo = total * w / n_warps, hi = total * (w + 1) / n_warps;
  if (lo >= hi) return;
  int it = 0, top = n_items - 1;
  while (it < top) {  // last image whose first unit is <= lo
    const int mid = (it + top + 1) >> 1;
    if (items[mid].unit_begin <= lo) it = mid; else top = mid - 1;
  }
  long long u = lo;
  while (u < hi && it < n_items) {
    const BatchItem& b = items[it];
    const long long end = b.unit_begin + b.units;
    const long long e = hi < end ? hi : end;
    if (e > u) {
      const int kind = edge_kind(b.a);
      const long long ulo = u - b.unit_begin, uhi = e - b.unit_begin;
      if (b.site0_from_y) {
        if (kind == kEdgeMix) run_units_any<true, kEdgeMix>(b.a, ulo, uhi, warp_stage());
        else if (kind == kEdgeL1Q) run_units_any<true, kEdgeL1Q>(b.a, ulo, uhi, warp_stage());
        else run_units_any<true, kEdgeL1>(b.a, ulo, uhi, warp_stage());
      } else {
        if (kind == kEdgeMix) run_units_any<false, kEdgeMix>(b.a, ulo, uhi, warp_stage());
        else if (kind == kEdgeL1Q) run_units_any<false, kEdgeL1Q>(b.a, ulo, uhi, warp_stage());
        else run_units_any<false, kEdgeL1>(b.a, ulo, uhi, warp_stage());
      }
      u = e;
    }
    ++it;
  }
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

// Warps the whole GPU holds at once for a kernel (cached per device).
template <typename Kern>
int resident_warps(Kern kernel, int slot) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static int cache[kMaxDev][13] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152 * 8;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev][slot]) {
    int per_sm = 0, sms = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, kSmemBytes) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 152 * 8;
    }
    cache[dev][slot] = (per_sm > 0 ? per_sm : 1) * sms * kWarpsPerBlock;
  }
  return cache[dev][slot];
}

void launch_units(long long total, int resident, int& n_warps, int& blocks) {
  long long w = total < resident ? total : resident;
  if (w < 1) w = 1;
  n_warps = (int)w;
  blocks = (n_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
}

template <bool kSite0FromY, int kX, int kEdge>
void launch_single(const SweepArgs& a, cudaStream_t s) {
  // occupancy cache slot of this instantiation: 0..3 and 5..12 (4 is the batch kernel's)
  const int slot = kEdge * 4 + (kSite0FromY ? 0 : 2) + (kX == 4 ? 0 : 1) + (kEdge ? 1 : 0);
  const int S = strips_of(a.width);
  const int ups = units_per_strip(a.height);
  const int resident = resident_warps(prior_sweep_kernel<kSite0FromY, kX, kEdge>, slot);
  int n_seg = resident / S;
  if (n_seg < 1) n_seg = 1;
  if (n_seg > ups) n_seg = ups;
  const int blocks = (S * n_seg + kWarpsPerBlock - 1) / kWarpsPerBlock;
  prior_sweep_kernel<kSite0FromY, kX, kEdge><<<blocks, kThreads, kSmemBytes, s>>>(a, n_seg);
}

template <int kEdge>
void launch_edge(const SweepArgs& a, bool site0_from_y, bool x4, cudaStream_t s) {
  if (site0_from_y) {
    if (x4) launch_single<true, 4, kEdge>(a, s); else launch_single<true, 3, kEdge>(a, s);
  } else {
    if (x4) launch_single<false, 4, kEdge>(a, s); else launch_single<false, 3, kEdge>(a, s);
  }
}

}  // namespace

double prior_sweep_bytes_per_pixel(bool site0_from_y) {
  // reads: y (or tau0, nu0) and tau1..4, nu1..4; writes: tau1..4, nu1..4
  return site0_from_y ? (9 + 8) * 4.0 : (10 + 8) * 4.0;
}

void prior_sweep_prepare(SweepArgs& a) {
  auto al = [](const void* p) { return ((uintptr_t)p & 7) == 0; };
  a.vec2 = (a.width % 2 == 0) && al(a.tau0) && al(a.nu0) && al(a.tin) && al(a.nin) && al(a.tout) &&
           al(a.nout) && al(a.y);
}

int prior_sweep_blocks(int height, int width) {
  return strips_of(width) * units_per_strip(height);
}

void prior_sweep_prewarm() {
  resident_warps(prior_sweep_kernel<true, 4, kEdgeL1>, 0);
  resident_warps(prior_sweep_kernel<true, 3, kEdgeL1>, 1);
  resident_warps(prior_sweep_kernel<false, 4, kEdgeL1>, 2);
  resident_warps(prior_sweep_kernel<false, 3, kEdgeL1>, 3);
  resident_warps(prior_sweep_batch_kernel, 4);
  resident_warps(prior_sweep_kernel<true, 4, kEdgeL1Q>, 5);
  resident_warps(prior_sweep_kernel<true, 3, kEdgeL1Q>, 6);
  resident_warps(prior_sweep_kernel<false, 4, kEdgeL1Q>, 7);
  resident_warps(prior_sweep_kernel<false, 3, kEdgeL1Q>, 8);
  resident_warps(prior_sweep_kernel<true, 4, kEdgeMix>, 9);
  resident_warps(prior_sweep_kernel<true, 3, kEdgeMix>, 10);
  resident_warps(prior_sweep_kernel<false, 4, kEdgeMix>, 11);
  resident_warps(prior_sweep_kernel<false, 3, kEdgeMix>, 12);
}

void launch_prior_sweep_batch(const BatchItem* items, int n_items, long long total_units,
                              cudaStream_t s) {
  int n_warps, blocks;
  launch_units(total_units, resident_warps(prior_sweep_batch_kernel, 4), n_warps, blocks);
  prior_sweep_batch_kernel<<<blocks, kThreads, kSmemBytes, s>>>(items, n_items, total_units, n_warps);
}

void launch_prior_sweep(const SweepArgs& args, bool site0_from_y, cudaStream_t s) {
  SweepArgs a = args;
  prior_sweep_prepare(a);
  const bool x4 = later_vertical(a.order) == 4;
  switch (edge_kind(a)) {
    case kEdgeMix: launch_edge<kEdgeMix>(a, site0_from_y, x4, s); break;
    case kEdgeL1Q: launch_edge<kEdgeL1Q>(a, site0_from_y, x4, s); break;
    default: launch_edge<kEdgeL1>(a, site0_from_y, x4, s); break;
  }
}

void launch_abar_reduce(const double* partial, int n_partial, double* dscal, double n_pixels,
                        int do_em, cudaStream_t s) {
  abar_reduce_kernel<<<1, 1024, 0, s>>>(partial, n_partial, dscal, n_pixels, do_em);
}

}  // namespace eptv
