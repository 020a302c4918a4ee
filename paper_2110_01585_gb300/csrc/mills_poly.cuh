// Generated by gen_mills_poly.py; do not edit.
// g(b) = G(u) K / (b + K), v(b) = V(u) (K / (b + K))^2, u = (K - b) / (K + b), b >= 0;
// coefficients of u^0 .. u^14.
#pragma once

namespace eptv {

constexpr float kMillsK = 2.0f;

__device__ __forceinline__ float mills_G(float u) {
  float p = 1.779735618e-04f;
  p = fmaf(p, u, 6.985943445e-05f);
  p = fmaf(p, u, -1.159832800e-03f);
  p = fmaf(p, u, 3.476753057e-04f);
  p = fmaf(p, u, 3.041465779e-03f);
  p = fmaf(p, u, -3.527105914e-03f);
  p = fmaf(p, u, -2.492271357e-03f);
  p = fmaf(p, u, 1.078331225e-02f);
  p = fmaf(p, u, -9.144003327e-03f);
  p = fmaf(p, u, -1.472682652e-02f);
  p = fmaf(p, u, 4.442855075e-02f);
  p = fmaf(p, u, -1.180622736e-02f);
  p = fmaf(p, u, -1.323406673e-01f);
  p = fmaf(p, u, 1.678016007e-01f);
  p = fmaf(p, u, 7.464310650e-01f);
  return p;
}

__device__ __forceinline__ float mills_V(float u) {
  float p = 4.269059762e-04f;
  p = fmaf(p, u, 1.280884476e-03f);
  p = fmaf(p, u, -4.134165730e-03f);
  p = fmaf(p, u, -3.511105471e-03f);
  p = fmaf(p, u, 1.489520605e-02f);
  p = fmaf(p, u, -3.988641760e-03f);
  p = fmaf(p, u, -2.474652902e-02f);
  p = fmaf(p, u, 3.401531326e-02f);
  p = fmaf(p, u, 4.992823019e-03f);
  p = fmaf(p, u, -7.183591634e-02f);
  p = fmaf(p, u, 7.436602430e-02f);
  p = fmaf(p, u, 6.526947198e-02f);
  p = fmaf(p, u, -2.162265483e-01f);
  p = fmaf(p, u, 3.546015767e-02f);
  p = fmaf(p, u, 4.571163883e-01f);
  return p;
}

}  // namespace eptv
