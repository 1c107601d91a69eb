// Element product of fe_element.cuh for two load cases at once in paired FP32
// arithmetic: each float2 holds one value of case r (x) and of case r' (y), and
// every case-dependent operation is one f32x2 instruction (sm_100 and later:
// __ffma2_rn, __fmul2_rn, __fadd2_rn), so the arithmetic of two element-case
// products issues as many instructions as one. Geometry (gradients, Lame
// constants, V/20) is per element and shared by both lanes.
//
// The corner displacement gradients are regrouped so that no operand needs a
// negation. With v_mm = 3 u_m and v_mj = 4 u_mj - u_j,
//     H_m = sum_j v_mj (x) g_j = 4 (u_m (x) g_m + sum_{j != m} u_mj (x) g_j) - Hc,
//     Hc  = sum_j u_j (x) g_j   (the gradient of the linear part, common to all m),
// which is the same matrix (exact arithmetic) in 36 + 4 x 36 multiply-adds
// instead of 4 x 48.
#pragma once

#include "fe_element.cuh"

namespace fe {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// s_m = lam tr(H_m) I + mu (H_m + H_m^T) from Hn = -Hc and the scaled gradients g4 = 4 g
template <int M>
__device__ __forceinline__ void corner_stress_x2(const float g4[4][3], float lam, float mu, const float2 Hn[3][3],
                                                 const float2 u[10][3], float2 s[6]) {
  float2 H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) H[a][b] = fma2(u[M][a], bc2(g4[M][b]), Hn[a][b]);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j == M) continue;
    const int e = (M == 0) ? (j == 1 ? 4 : j == 2 ? 6 : 7)
                : (M == 1) ? (j == 0 ? 4 : j == 2 ? 5 : 8)
                : (M == 2) ? (j == 0 ? 6 : j == 1 ? 5 : 9)
                           : (j == 0 ? 7 : j == 1 ? 8 : 9);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) H[a][b] = fma2(u[e][a], bc2(g4[j][b]), H[a][b]);
  }
  const float2 lt = mul2(bc2(lam), add2(add2(H[0][0], H[1][1]), H[2][2]));
  const float2 two_mu = bc2(2.f * mu);
  s[0] = fma2(two_mu, H[0][0], lt);
  s[1] = fma2(two_mu, H[1][1], lt);
  s[2] = fma2(two_mu, H[2][2], lt);
  s[3] = mul2(bc2(mu), add2(H[1][2], H[2][1]));
  s[4] = mul2(bc2(mu), add2(H[0][2], H[2][0]));
  s[5] = mul2(bc2(mu), add2(H[0][1], H[1][0]));
}

// w = A g for a symmetric 3x3 A stored (xx, yy, zz, yz, xz, xy), g per element
__device__ __forceinline__ void sym_mv_x2(const float2 A[6], const float g[3], float2 w[3]) {
  w[0] = fma2(A[4], bc2(g[2]), fma2(A[5], bc2(g[1]), mul2(A[0], bc2(g[0]))));
  w[1] = fma2(A[3], bc2(g[2]), fma2(A[1], bc2(g[1]), mul2(A[5], bc2(g[0]))));
  w[2] = fma2(A[2], bc2(g[2]), fma2(A[3], bc2(g[1]), mul2(A[4], bc2(g[0]))));
}

// y_kl = T_k G4_l + T_l G4_k
template <int K, int L>
__device__ __forceinline__ void edge_out_x2(const float2 t[4][6], const float G4[4][3], float2 y[10][3]) {
  constexpr int e = edge_node(K, L);
  const float2* a = t[K];
  const float2* b = t[L];
  const float* g = G4[L];
  const float* h = G4[K];
  float2 w[3], v[3];
  sym_mv_x2(a, g, w);
  // continue each chain with the second term (T_l G4_k)
  v[0] = fma2(b[4], bc2(h[2]), fma2(b[5], bc2(h[1]), fma2(b[0], bc2(h[0]), w[0])));
  v[1] = fma2(b[3], bc2(h[2]), fma2(b[1], bc2(h[1]), fma2(b[5], bc2(h[0]), w[1])));
  v[2] = fma2(b[2], bc2(h[2]), fma2(b[3], bc2(h[1]), fma2(b[4], bc2(h[0]), w[2])));
  y[e][0] = v[0];
  y[e][1] = v[1];
  y[e][2] = v[2];
}

// y = K_e u for two cases (lanes x and y of every float2)
__device__ __forceinline__ void elem_apply_x2(const ElemGeo<float>& G, const float2 u[10][3], float2 y[10][3]) {
  float g4[4][3], ng[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g4[k][i] = 4.f * G.g[k][i];
      ng[k][i] = -G.g[k][i];
    }
  // Hn = -Hc = sum_j u_j (x) (-g_j)
  float2 Hn[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 h = mul2(u[0][a], bc2(ng[0][b]));
      h = fma2(u[1][a], bc2(ng[1][b]), h);
      h = fma2(u[2][a], bc2(ng[2][b]), h);
      Hn[a][b] = fma2(u[3][a], bc2(ng[3][b]), h);
    }
  float2 s[4][6];
  corner_stress_x2<0>(g4, G.lam, G.mu, Hn, u, s[0]);
  corner_stress_x2<1>(g4, G.lam, G.mu, Hn, u, s[1]);
  corner_stress_x2<2>(g4, G.lam, G.mu, Hn, u, s[2]);
  corner_stress_x2<3>(g4, G.lam, G.mu, Hn, u, s[3]);
  float2 S[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = add2(add2(s[0][q], s[1][q]), add2(s[2][q], s[3][q]));
  float G4[4][3];
  const float c4 = 4.f * G.c;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) G4[k][i] = c4 * G.g[k][i];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) A[q] = fma2(bc2(-0.25f), S[q], s[k][q]);
    sym_mv_x2(A, G4[k], y[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) s[k][q] = add2(s[k][q], S[q]);
  edge_out_x2<0, 1>(s, G4, y);
  edge_out_x2<1, 2>(s, G4, y);
  edge_out_x2<0, 2>(s, G4, y);
  edge_out_x2<0, 3>(s, G4, y);
  edge_out_x2<1, 3>(s, G4, y);
  edge_out_x2<2, 3>(s, G4, y);
}

}  // namespace fe
