// Element arithmetic of the EBE product for straight-sided 10-node tetrahedra.
//
// The element matrix K_e of Eq. 3 is never formed. For an affine element the
// gradients g_k = grad L_k of the volume coordinates are constant, and the
// displacement gradient of the quadratic field is linear in L:
//     grad u = sum_m L_m H_m,   H_m = sum_j v_mj (x) g_j,
//     v_mm = 3 u_m,   v_mj = 4 u_mj - u_j  (j != m, u_mj = edge node of m-j).
// The stress is then sigma = sum_m L_m s_m with s_m = lam tr(H_m) I + mu (H_m + H_m^T),
// and integrating grad N_a . sigma exactly with int L_m L_n dV = V (1 + delta_mn)/20
// gives, with S = sum_m s_m and c = V/20,
//     corner k:      y_k  = c (4 s_k - S) g_k
//     edge node kl:  y_kl = 4c ((S + s_k) g_l + (S + s_l) g_k).
// This equals K_e u for the textbook B^T D B element (exact quadrature), with
// about 460 arithmetic instructions per case (most of them multiply-adds)
// instead of 900 multiply-adds for an explicit 30x30 product.
#pragma once

#include <stdint.h>

namespace fe {

// local node of the edge joining corners a and b (VTK TET10 order)
__host__ __device__ constexpr int edge_node(int a, int b) {
  return (a > b) ? edge_node(b, a)
         : (a == 0 && b == 1) ? 4
         : (a == 1 && b == 2) ? 5
         : (a == 0 && b == 2) ? 6
         : (a == 0 && b == 3) ? 7
         : (a == 1 && b == 3) ? 8
         : 9;  // (2,3)
}

template <typename T>
struct ElemGeo {
  T g[4][3];  // gradients of the volume coordinates
  T lam, mu;  // Lame constants
  T c;        // element volume / 20
};

// Geometry and Lame constants of one element from its corner coordinates.
// Returns 6V (positive for a valid element).
template <typename T>
__device__ __forceinline__ T elem_geometry(const T x0[3], const T x1[3], const T x2[3], const T x3[3],
                                           T E, T nu, ElemGeo<T>& G) {
  T d1[3], d2[3], d3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d1[i] = x1[i] - x0[i];
    d2[i] = x2[i] - x0[i];
    d3[i] = x3[i] - x0[i];
  }
  // rows of the inverse Jacobian: (d2 x d3, d3 x d1, d1 x d2) / det
  T c23[3] = {d2[1] * d3[2] - d2[2] * d3[1], d2[2] * d3[0] - d2[0] * d3[2], d2[0] * d3[1] - d2[1] * d3[0]};
  T c31[3] = {d3[1] * d1[2] - d3[2] * d1[1], d3[2] * d1[0] - d3[0] * d1[2], d3[0] * d1[1] - d3[1] * d1[0]};
  T c12[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
  T det = d1[0] * c23[0] + d1[1] * c23[1] + d1[2] * c23[2];
  T inv = T(1) / det;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G.g[1][i] = c23[i] * inv;
    G.g[2][i] = c31[i] * inv;
    G.g[3][i] = c12[i] * inv;
    G.g[0][i] = -(G.g[1][i] + G.g[2][i] + G.g[3][i]);
  }
  G.c = det * T(1.0 / 120.0);
  T onu = T(1) + nu;
  G.mu = E / (T(2) * onu);
  G.lam = (E * nu) / (onu * (T(1) - T(2) * nu));
  return det;
}

// w = s g for a symmetric 3x3 s stored (xx, yy, zz, yz, xz, xy)
template <typename T>
__device__ __forceinline__ void sym_mv(const T s[6], const T g[3], T w[3]) {
  w[0] = s[0] * g[0] + s[5] * g[1] + s[4] * g[2];
  w[1] = s[5] * g[0] + s[1] * g[1] + s[3] * g[2];
  w[2] = s[4] * g[0] + s[3] * g[1] + s[2] * g[2];
}

// s_m = lam tr(H_m) I + mu (H_m + H_m^T), H_m = sum_j v_mj (x) g_j
template <int M, typename T>
__device__ __forceinline__ void corner_stress(const ElemGeo<T>& G, const T u[10][3], T s[6]) {
  T H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) H[a][b] = T(3) * u[M][a] * G.g[M][b];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j == M) continue;
    // edge node between corners M and j: constant once the loop is unrolled
    const int e = (M == 0) ? (j == 1 ? 4 : j == 2 ? 6 : 7)
                : (M == 1) ? (j == 0 ? 4 : j == 2 ? 5 : 8)
                : (M == 2) ? (j == 0 ? 6 : j == 1 ? 5 : 9)
                           : (j == 0 ? 7 : j == 1 ? 8 : 9);
    T v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = T(4) * u[e][a] - u[j][a];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) H[a][b] += v[a] * G.g[j][b];
  }
  const T lt = G.lam * (H[0][0] + H[1][1] + H[2][2]);
  const T two_mu = T(2) * G.mu;
  s[0] = lt + two_mu * H[0][0];
  s[1] = lt + two_mu * H[1][1];
  s[2] = lt + two_mu * H[2][2];
  s[3] = G.mu * (H[1][2] + H[2][1]);
  s[4] = G.mu * (H[0][2] + H[2][0]);
  s[5] = G.mu * (H[0][1] + H[1][0]);
}

// y_kl = T_k G4_l + T_l G4_k (one chain of multiply-adds)
template <int K, int L, typename T>
__device__ __forceinline__ void edge_out(const T t[4][6], const T G4[4][3], T y[10][3]) {
  constexpr int e = edge_node(K, L);
  const T* a = t[K];
  const T* b = t[L];
  const T* g = G4[L];
  const T* h = G4[K];
  y[e][0] = a[0] * g[0] + a[5] * g[1] + a[4] * g[2] + b[0] * h[0] + b[5] * h[1] + b[4] * h[2];
  y[e][1] = a[5] * g[0] + a[1] * g[1] + a[3] * g[2] + b[5] * h[0] + b[1] * h[1] + b[3] * h[2];
  y[e][2] = a[4] * g[0] + a[3] * g[1] + a[2] * g[2] + b[4] * h[0] + b[3] * h[1] + b[2] * h[2];
}

// y = K_e u for one case; u and y are [10][3] in element-local order.
// With G4_k = 4c g_k the outputs read
//   corner k:     y_k  = (s_k - S/4) G4_k
//   edge node kl: y_kl = T_k G4_l + T_l G4_k,  T_k = S + s_k
// (the factors c and 4c of the derivation folded into the gradients).
template <typename T>
__device__ __forceinline__ void elem_apply(const ElemGeo<T>& G, const T u[10][3], T y[10][3]) {
  T s[4][6];
  corner_stress<0>(G, u, s[0]);
  corner_stress<1>(G, u, s[1]);
  corner_stress<2>(G, u, s[2]);
  corner_stress<3>(G, u, s[3]);
  T S[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = (s[0][q] + s[1][q]) + (s[2][q] + s[3][q]);
  T G4[4][3];
  const T c4 = T(4) * G.c;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) G4[k][i] = c4 * G.g[k][i];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) A[q] = s[k][q] - T(0.25) * S[q];
    sym_mv(A, G4[k], y[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) s[k][q] += S[q];
  edge_out<0, 1>(s, G4, y);
  edge_out<1, 2>(s, G4, y);
  edge_out<0, 2>(s, G4, y);
  edge_out<0, 3>(s, G4, y);
  edge_out<1, 3>(s, G4, y);
  edge_out<2, 3>(s, G4, y);
}

// lambda^T K_e u for one case (adjoint element sensitivity), same arithmetic.
template <typename T>
__device__ __forceinline__ T elem_bilinear(const ElemGeo<T>& G, const T lam[10][3], const T u[10][3]) {
  T y[10][3];
  elem_apply(G, u, y);
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc += lam[a][c] * y[a][c];
  return acc;
}

}  // namespace fe
