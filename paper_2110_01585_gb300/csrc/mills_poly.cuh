// Generated by gen_mills_poly.py; do not edit.
// g(b) = G(u) K / (b + K), v(b) = V(u) (K / (b + K))^2, u = (K - b) / (K + b), b >= 0;
// coefficients of u^0 .. u^12 (literals, so that the packed FMAs take them as
// immediates instead of constant-bank loads).
#pragma once

namespace eptv {

constexpr float kMillsK = 2.0f;
constexpr int kMillsDegree = 12;

__device__ constexpr float kMillsG[13] = {
    7.464310867e-01f,
    1.678013790e-01f,
    -1.323427964e-01f,
    -1.180001915e-02f,
    4.446261600e-02f,
    -1.477649222e-02f,
    -9.348394839e-03f,
    1.095359462e-02f,
    -1.908295607e-03f,
    -3.810909866e-03f,
    2.184968013e-03f,
    5.747184676e-04f,
    -5.369253335e-04f,
};

__device__ constexpr float kMillsV[13] = {
    4.571164404e-01f,
    3.545609236e-02f,
    -2.162316553e-01f,
    6.538330058e-02f,
    7.444773677e-02f,
    -7.274654515e-02f,
    4.502548187e-03f,
    3.713746917e-02f,
    -2.334574379e-02f,
    -9.192234943e-03f,
    1.284072104e-02f,
    6.517690757e-04f,
    -2.639994813e-03f,
};

}  // namespace eptv
