// Element product in float-float arithmetic (the FP64-accurate products of the
// outer loop, computed on the FP32 pipe), the formulas of elem_apply with the
// sums of products accumulated in compensated form.
//
// A sum of products sum_i a_i b_i of float-float numbers is accumulated as in
// the compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005): the product of the high parts is
// split exactly (TwoProd, one multiply and one FMA), the running sum of those
// products is kept exact (TwoSum), and all rounding errors are gathered in one
// float together with the cross terms hi*lo and lo*hi of each product; the
// final sum and error are renormalised once. The result is as accurate as
// evaluating in float-float throughout, with about 11 FP32 operations per term
// instead of 18 for a float-float multiply and add. Multiplications by 4, 2 and
// 1/4 scale both parts exactly.
#pragma once

#include "fe_df.cuh"
#include "fe_element.cuh"

namespace fe {

// running compensated sum: value s + c (c holds the rounding errors, not normalised)
struct dfsum {
  float s, c;
};

__device__ __forceinline__ void acc_first(dfsum& A, const df& a, const df& b) {
  const float p = a.hi * b.hi;
  A.s = p;
  A.c = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
}

__device__ __forceinline__ void acc_add(dfsum& A, const df& a, const df& b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  const float s = A.s + p;
  const float bb = s - A.s;
  const float err = (A.s - (s - bb)) + (p - bb);
  A.s = s;
  A.c += err + fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
}

__device__ __forceinline__ df acc_value(const dfsum& A) { return df_two_sum(A.s, A.c); }

// a * k for k a power of two (exact)
__device__ __forceinline__ df dscale(const df& a, float k) { return df(a.hi * k, a.lo * k); }

// 3 a: exact product of the high part plus the scaled low part
__device__ __forceinline__ df dtimes3(const df& a) {
  const float p = 3.f * a.hi;
  return df_fast_two_sum(p, fmaf(3.f, a.lo, fmaf(3.f, a.hi, -p)));
}

// s_m = lam tr(H_m) I + mu (H_m + H_m^T), H_m = sum_j v_mj (x) g_j
template <int M>
__device__ __forceinline__ void corner_stress_df(const ElemGeo<df>& G, const df u[10][3], df s[6]) {
  df v[4][3];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j == M) {
#pragma unroll
      for (int a = 0; a < 3; ++a) v[j][a] = dtimes3(u[M][a]);
    } else {
      // edge node between corners M and j, written out so that it folds to a constant
      const int e = (M == 0) ? (j == 1 ? 4 : j == 2 ? 6 : 7)
                  : (M == 1) ? (j == 0 ? 4 : j == 2 ? 5 : 8)
                  : (M == 2) ? (j == 0 ? 6 : j == 1 ? 5 : 9)
                             : (j == 0 ? 7 : j == 1 ? 8 : 9);
#pragma unroll
      for (int a = 0; a < 3; ++a) v[j][a] = dscale(u[e][a], 4.f) - u[j][a];
    }
  }
  df H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dfsum A;
      acc_first(A, v[0][a], G.g[0][b]);
      acc_add(A, v[1][a], G.g[1][b]);
      acc_add(A, v[2][a], G.g[2][b]);
      acc_add(A, v[3][a], G.g[3][b]);
      H[a][b] = acc_value(A);
    }
  const df lt = G.lam * ((H[0][0] + H[1][1]) + H[2][2]);
  const df two_mu = dscale(G.mu, 2.f);
  s[0] = lt + two_mu * H[0][0];
  s[1] = lt + two_mu * H[1][1];
  s[2] = lt + two_mu * H[2][2];
  s[3] = G.mu * (H[1][2] + H[2][1]);
  s[4] = G.mu * (H[0][2] + H[2][0]);
  s[5] = G.mu * (H[0][1] + H[1][0]);
}

// w = A g for a symmetric 3x3 A stored (xx, yy, zz, yz, xz, xy)
__device__ __forceinline__ void sym_mv_df(const df A[6], const df g[3], df w[3]) {
  dfsum S;
  acc_first(S, A[0], g[0]);
  acc_add(S, A[5], g[1]);
  acc_add(S, A[4], g[2]);
  w[0] = acc_value(S);
  acc_first(S, A[5], g[0]);
  acc_add(S, A[1], g[1]);
  acc_add(S, A[3], g[2]);
  w[1] = acc_value(S);
  acc_first(S, A[4], g[0]);
  acc_add(S, A[3], g[1]);
  acc_add(S, A[2], g[2]);
  w[2] = acc_value(S);
}

// y_kl = T_k G4_l + T_l G4_k
template <int K, int L>
__device__ __forceinline__ void edge_out_df(const df t[4][6], const df G4[4][3], df y[10][3]) {
  constexpr int e = edge_node(K, L);
  const df* a = t[K];
  const df* b = t[L];
  const df* g = G4[L];
  const df* h = G4[K];
  dfsum S;
  acc_first(S, a[0], g[0]);
  acc_add(S, a[5], g[1]);
  acc_add(S, a[4], g[2]);
  acc_add(S, b[0], h[0]);
  acc_add(S, b[5], h[1]);
  acc_add(S, b[4], h[2]);
  y[e][0] = acc_value(S);
  acc_first(S, a[5], g[0]);
  acc_add(S, a[1], g[1]);
  acc_add(S, a[3], g[2]);
  acc_add(S, b[5], h[0]);
  acc_add(S, b[1], h[1]);
  acc_add(S, b[3], h[2]);
  y[e][1] = acc_value(S);
  acc_first(S, a[4], g[0]);
  acc_add(S, a[3], g[1]);
  acc_add(S, a[2], g[2]);
  acc_add(S, b[4], h[0]);
  acc_add(S, b[3], h[1]);
  acc_add(S, b[2], h[2]);
  y[e][2] = acc_value(S);
}

// y = K_e u for one case (float-float); chosen over the generic template by
// overload resolution wherever the element data is float-float
__device__ __forceinline__ void elem_apply(const ElemGeo<df>& G, const df u[10][3], df y[10][3]) {
  df s[4][6];
  corner_stress_df<0>(G, u, s[0]);
  corner_stress_df<1>(G, u, s[1]);
  corner_stress_df<2>(G, u, s[2]);
  corner_stress_df<3>(G, u, s[3]);
  df S[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = (s[0][q] + s[1][q]) + (s[2][q] + s[3][q]);
  df G4[4][3];
  const df c4 = dscale(G.c, 4.f);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) G4[k][i] = c4 * G.g[k][i];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    df A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) A[q] = s[k][q] - dscale(S[q], 0.25f);
    sym_mv_df(A, G4[k], y[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) s[k][q] += S[q];
  edge_out_df<0, 1>(s, G4, y);
  edge_out_df<1, 2>(s, G4, y);
  edge_out_df<0, 2>(s, G4, y);
  edge_out_df<0, 3>(s, G4, y);
  edge_out_df<1, 3>(s, G4, y);
  edge_out_df<2, 3>(s, G4, y);
}

// ---------------------------------------------------------------------------
// The same product with little register state, for kernels that run two blocks
// per SM: the node values (node a, component c) are read from shared memory at
// xa[off[a] + c] where they are used, the element's 16 float-float values
// (g[4][3], lam, mu, V/20) from gs, and the 30 outputs are stored to
// o[a * VR + c] as they are formed. Same operations in the same order as
// elem_apply above.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void corner_stress_df_lean(const df* gs, const df* xa, const int off[10], df s[6]) {
  dfsum A[3][3];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    df v[3];
    if (j == M) {
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = dtimes3(xa[off[M] + a]);
    } else {
      const int e = (M == 0) ? (j == 1 ? 4 : j == 2 ? 6 : 7)
                  : (M == 1) ? (j == 0 ? 4 : j == 2 ? 5 : 8)
                  : (M == 2) ? (j == 0 ? 6 : j == 1 ? 5 : 9)
                             : (j == 0 ? 7 : j == 1 ? 8 : 9);
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = dscale(xa[off[e] + a], 4.f) - xa[off[j] + a];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const df g = gs[3 * j + b];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (j == 0)
          acc_first(A[a][b], v[a], g);
        else
          acc_add(A[a][b], v[a], g);
      }
    }
  }
  df H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) H[a][b] = acc_value(A[a][b]);
  const df lam = gs[12], mu = gs[13];
  const df lt = lam * ((H[0][0] + H[1][1]) + H[2][2]);
  const df two_mu = dscale(mu, 2.f);
  s[0] = lt + two_mu * H[0][0];
  s[1] = lt + two_mu * H[1][1];
  s[2] = lt + two_mu * H[2][2];
  s[3] = mu * (H[1][2] + H[2][1]);
  s[4] = mu * (H[0][2] + H[2][0]);
  s[5] = mu * (H[0][1] + H[1][0]);
}

// y_kl = T_k G4_l + T_l G4_k, stored to o[e VR + c]
template <int K, int L, int VR>
__device__ __forceinline__ void edge_out_df_lean(const df t[4][6], const df G4[4][3], df* o) {
  constexpr int e = edge_node(K, L);
  const df* a = t[K];
  const df* b = t[L];
  const df* g = G4[L];
  const df* h = G4[K];
  dfsum S;
  acc_first(S, a[0], g[0]);
  acc_add(S, a[5], g[1]);
  acc_add(S, a[4], g[2]);
  acc_add(S, b[0], h[0]);
  acc_add(S, b[5], h[1]);
  acc_add(S, b[4], h[2]);
  o[e * VR] = acc_value(S);
  acc_first(S, a[5], g[0]);
  acc_add(S, a[1], g[1]);
  acc_add(S, a[3], g[2]);
  acc_add(S, b[5], h[0]);
  acc_add(S, b[1], h[1]);
  acc_add(S, b[3], h[2]);
  o[e * VR + 1] = acc_value(S);
  acc_first(S, a[4], g[0]);
  acc_add(S, a[3], g[1]);
  acc_add(S, a[2], g[2]);
  acc_add(S, b[4], h[0]);
  acc_add(S, b[3], h[1]);
  acc_add(S, b[2], h[2]);
  o[e * VR + 2] = acc_value(S);
}

template <int VR>
__device__ __forceinline__ void elem_apply_df_lean(const df* gs, const df* xa, const int off[10], df* o) {
  df s[4][6];
  corner_stress_df_lean<0>(gs, xa, off, s[0]);
  corner_stress_df_lean<1>(gs, xa, off, s[1]);
  corner_stress_df_lean<2>(gs, xa, off, s[2]);
  corner_stress_df_lean<3>(gs, xa, off, s[3]);
  df S[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = (s[0][q] + s[1][q]) + (s[2][q] + s[3][q]);
  df G4[4][3];
  const df c4 = dscale(gs[14], 4.f);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) G4[k][i] = c4 * gs[3 * k + i];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    df A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) A[q] = s[k][q] - dscale(S[q], 0.25f);
    df w[3];
    sym_mv_df(A, G4[k], w);
#pragma unroll
    for (int c = 0; c < 3; ++c) o[k * VR + c] = w[c];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) s[k][q] += S[q];
  edge_out_df_lean<0, 1, VR>(s, G4, o);
  edge_out_df_lean<1, 2, VR>(s, G4, o);
  edge_out_df_lean<0, 2, VR>(s, G4, o);
  edge_out_df_lean<0, 3, VR>(s, G4, o);
  edge_out_df_lean<1, 3, VR>(s, G4, o);
  edge_out_df_lean<2, 3, VR>(s, G4, o);
}

}  // namespace fe
