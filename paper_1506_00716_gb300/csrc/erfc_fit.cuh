// erfc_fit.cuh -- generated by fit_erfc.py; do not edit.
// erfc(x) = exp(-x^2) R(u), t = 1/(1 + EF_P x), u = EF_UA t + EF_UB, x in [0, EF_XMAX].
// energy fit: degree 12, max relative error 4.41e-11 (4.41e-11 with the head + tail coefficients below)
#pragma once
namespace nbgb {
constexpr float EF_P = 0.4f;
constexpr float EF_XMAX = 6.0f;
constexpr float EF_UA = 2.8333333f;
constexpr float EF_UB = -1.8333334f;
constexpr int EF_NE = 13;
__device__ constexpr float EF_EN_HI[EF_NE] = {0.3454021f, 0.39277083f, 0.19105737f, 0.06116964f, 0.0103621f, -0.00032189983f, -0.00045583156f, -6.419039e-06f, 2.3997538e-05f, -4.913019e-07f, -1.4358875e-06f, 1.203554e-07f, 6.9129975e-08f};
__device__ constexpr float EF_EN_LO[EF_NE] = {-4.4934265e-09f, -5.7412146e-09f, -6.573779e-09f, -5.609882e-10f, -8.8758646e-11f, 4.9718953e-13f, -1.41651925e-11f, 1.4295954e-13f, 2.5595736e-13f, -1.0181217e-14f, -3.9859138e-14f, -2.4092192e-15f, 2.3144078e-15f};
// 2^f on [-0.5, 0.5]: degree 10, max relative error 1.11e-15
constexpr int EX2_N = 11;
__device__ constexpr float EX2_HI[EX2_N] = {1.0f, 0.6931472f, 0.2402265f, 0.05550411f, 0.009618129f, 0.0013333558f, 0.0001540353f, 1.5252659e-05f, 1.3215574e-06f, 1.0208292e-07f, 7.055614e-09f};
__device__ constexpr float EX2_LO[EX2_N] = {0.0f, -1.9046495e-09f, -2.2780267e-10f, -1.0459841e-09f, 4.5809978e-10f, 3.543682e-11f, 3.9846867e-12f, 3.0896604e-13f, 3.3200286e-14f, -2.528519e-15f, 1.7870517e-18f};
}  // namespace nbgb
