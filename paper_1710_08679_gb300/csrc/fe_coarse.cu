// First-order (TET4) coarse level of the inner solve (Sec. 2: "the same mesh but
// without edge nodes"; inner loop level 1 of Algorithm 1(a): its block Jacobi,
// the restriction of the residual and guess, and the prolongation of the result).
//
//  * the coarse mesh is the corner nodes of the TET10 mesh, with the same elements
//    and materials; the element stiffness of a linear tetrahedron is
//    K_e = V B^T D B with constant B, applied as y_k = V s g_k, s = lam tr(H) I +
//    mu (H + H^T), H = sum_k u_k (x) g_k (g_k: gradients of the volume coordinates);
//  * P1 maps coarse to fine values: a vertex keeps its value, an edge node takes
//    the mean of its two ends (linear interpolation); P1^T is its transpose;
//  * Dirichlet DOFs are kept at zero by both transfers, and the coarse operator is
//    K1_bc = P K1 P + (I - P) with the coarse free mask.
//  * two ways to apply K1_bc: element by element (fe_ebe4_apply), or assembled
//    once per material state into a 3x3 block CSR matrix and applied by a
//    multi-vector block SpMV (what the solver uses when the matrix fits). A TET4
//    element has too little arithmetic to hide its 12 scattered node updates, so
//    on GB300 the matrix-free product is bound by atomics and load latency, while
//    the block SpMV reads about 36 bytes per block once for all R cases.
#include <algorithm>
#include <vector>

#include "fe_element.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) zero4_kernel(int64_t n, T* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = T(0);
}

// W consecutive cases of one node: 3W contiguous values. For float with W = 4
// they are 48 bytes at a 48-byte multiple from a 16-byte aligned base (R is a
// multiple of 4), moved as three 16-byte vectors.
template <typename T, int W>
struct CaseGroup {
  static __device__ __forceinline__ void load(const T* __restrict__ p, T v[3 * W]) {
#pragma unroll
    for (int i = 0; i < 3 * W; ++i) v[i] = __ldg(p + i);
  }
  static __device__ __forceinline__ void store(T* p, const T v[3 * W]) {
#pragma unroll
    for (int i = 0; i < 3 * W; ++i) p[i] = v[i];
  }
  static __device__ __forceinline__ void add(T* p, const T v[3 * W]) {
#pragma unroll
    for (int i = 0; i < 3 * W; ++i) atomicAdd(p + i, v[i]);
  }
};

template <>
struct CaseGroup<float, 4> {
  static __device__ __forceinline__ void load(const float* __restrict__ p, float v[12]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 t = __ldg(q + k);
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  }
  static __device__ __forceinline__ void store(float* p, const float v[12]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
  static __device__ __forceinline__ void add(float* p, const float v[12]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(q + k, make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
  }
};

// Per-element TET4 data of the FP32 products, computed once per material state:
// grad L_0..3 (12 floats), lam V, mu V, 2 pad, from the FP32 corner coordinates.
__global__ void __launch_bounds__(kThreads) coarse_geo_kernel(MeshView<float> M, float4* __restrict__ geo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M.n_elem) return;
  float xc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[k][i] = M.xyz[3 * (int64_t)M.conn[10 * e + k] + i];
  ElemGeo<float> G;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], M.mat[2 * e], M.mat[2 * e + 1], G);
  const float V = 20.f * G.c;
  geo[4 * e + 0] = make_float4(G.g[0][0], G.g[0][1], G.g[0][2], G.g[1][0]);
  geo[4 * e + 1] = make_float4(G.g[1][1], G.g[1][2], G.g[2][0], G.g[2][1]);
  geo[4 * e + 2] = make_float4(G.g[2][2], G.g[3][0], G.g[3][1], G.g[3][2]);
  geo[4 * e + 3] = make_float4(G.lam * V, G.mu * V, 0.f, 0.f);
}

// TET4 element data for one thread: gradients and the volume-weighted Lame
// constants, either read from the per-element buffer (FP32) or computed from the
// corner coordinates (FP64, used for parity checks).
template <typename T>
struct Tet4Geo {
  T g[4][3];
  T lv, mv;  // lam V, mu V
};

__device__ __forceinline__ void tet4_geo(const float4* __restrict__ geo, const MeshView<float>&, int64_t e,
                                         Tet4Geo<float>& G) {
  const float4 a = __ldg(geo + 4 * e), b = __ldg(geo + 4 * e + 1), c = __ldg(geo + 4 * e + 2),
               d = __ldg(geo + 4 * e + 3);
  G.g[0][0] = a.x; G.g[0][1] = a.y; G.g[0][2] = a.z;
  G.g[1][0] = a.w; G.g[1][1] = b.x; G.g[1][2] = b.y;
  G.g[2][0] = b.z; G.g[2][1] = b.w; G.g[2][2] = c.x;
  G.g[3][0] = c.y; G.g[3][1] = c.z; G.g[3][2] = c.w;
  G.lv = d.x;
  G.mv = d.y;
}

__device__ __forceinline__ void tet4_geo(const float4*, const MeshView<double>& M, int64_t e, Tet4Geo<double>& G) {
  const int2 c01 = __ldg(reinterpret_cast<const int2*>(M.conn + 10 * e));
  const int2 c23 = __ldg(reinterpret_cast<const int2*>(M.conn + 10 * e) + 1);
  const int cf[4] = {c01.x, c01.y, c23.x, c23.y};
  double xc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[k][i] = __ldg(M.xyz + 3 * (int64_t)cf[k] + i);
  ElemGeo<double> E;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], __ldg(M.mat + 2 * e), __ldg(M.mat + 2 * e + 1), E);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) G.g[k][i] = E.g[k][i];
  G.lv = E.lam * 20.0 * E.c;
  G.mv = E.mu * 20.0 * E.c;
}

// thread = (element, group of W cases), vector entries in the coarse numbering:
// H = sum_k u_k (x) g_k, s = lam V tr(H) I + mu V (H + H^T), y_k = s g_k.
// Fixed DOFs: the element that owns the corner adds x (y starts at zero), the
// others add zero, so y = x there.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) ebe4_kernel(MeshView<T> M, const float4* __restrict__ geo, int R,
                                                        const int32_t* __restrict__ conn4,
                                                        const uint8_t* __restrict__ nmask4,
                                                        const uint8_t* __restrict__ own4, const T* __restrict__ x,
                                                        T* __restrict__ y, const int* __restrict__ skip) {
  using CG = CaseGroup<T, W>;
  if (skip && *skip) return;
  const int G = R / W;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= M.n_elem * G) return;
  const int64_t e = gid / G;
  const int r0 = (int)(gid - e * G) * W;
  const int4 c4 = __ldg(reinterpret_cast<const int4*>(conn4) + e);
  const int ow = __ldg(own4 + e);
  Tet4Geo<T> G4;
  tet4_geo(geo, M, e, G4);
  const int nd[4] = {c4.x, c4.y, c4.z, c4.w};
  int mk[4];
  T H[W][3][3];
#pragma unroll
  for (int w = 0; w < W; ++w)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) H[w][a][b] = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    mk[k] = __ldg(nmask4 + nd[k]);
    T u[3 * W];
    CG::load(x + ((int64_t)nd[k] * R + r0) * 3, u);
#pragma unroll
    for (int i = 0; i < 3 * W; ++i)
      if (!((mk[k] >> (i % 3)) & 1)) u[i] = T(0);
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) H[w][a][b] += u[3 * w + a] * G4.g[k][b];
  }
  T sg[W][6];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const T lt = G4.lv * (H[w][0][0] + H[w][1][1] + H[w][2][2]);
    sg[w][0] = lt + T(2) * G4.mv * H[w][0][0];
    sg[w][1] = lt + T(2) * G4.mv * H[w][1][1];
    sg[w][2] = lt + T(2) * G4.mv * H[w][2][2];
    sg[w][3] = G4.mv * (H[w][1][2] + H[w][2][1]);
    sg[w][4] = G4.mv * (H[w][0][2] + H[w][2][0]);
    sg[w][5] = G4.mv * (H[w][0][1] + H[w][1][0]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T out[3 * W];
#pragma unroll
    for (int w = 0; w < W; ++w) sym_mv(sg[w], G4.g[k], out + 3 * w);
    T* ya = y + ((int64_t)nd[k] * R + r0) * 3;
    if (mk[k] != 7) {
      const T* xa = x + ((int64_t)nd[k] * R + r0) * 3;
#pragma unroll
      for (int i = 0; i < 3 * W; ++i)
        if (!((mk[k] >> (i % 3)) & 1)) out[i] = ((ow >> k) & 1) ? __ldg(xa + i) : T(0);
    }
    CG::add(ya, out);
  }
}

// r4 = P (P1^T r10), gathered per coarse node: its own vertex value plus half of
// each edge node it ends (the adjacency is built once on the host), so no
// atomics and no zeroing pass.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) restrict_kernel(int64_t N4, int R, const int32_t* __restrict__ vertex,
                                                            const int32_t* __restrict__ adj_ptr,
                                                            const int32_t* __restrict__ adj,
                                                            const uint8_t* __restrict__ nmask4,
                                                            const T* __restrict__ r10, T* __restrict__ r4,
                                                            const int* __restrict__ skip) {
  using CG = CaseGroup<T, W>;
  if (skip && *skip) return;
  const int G = R / W;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N4 * G) return;
  const int64_t a = gid / G;
  const int r0 = (int)(gid - a * G) * W;
  T acc[3 * W], v[3 * W];
  CG::load(r10 + ((int64_t)__ldg(vertex + a) * R + r0) * 3, acc);
  const int j1 = __ldg(adj_ptr + a + 1);
  for (int j = __ldg(adj_ptr + a); j < j1; ++j) {
    CG::load(r10 + ((int64_t)__ldg(adj + j) * R + r0) * 3, v);
#pragma unroll
    for (int i = 0; i < 3 * W; ++i) acc[i] += T(0.5) * v[i];
  }
  const int mk = __ldg(nmask4 + a);
#pragma unroll
  for (int i = 0; i < 3 * W; ++i)
    if (!((mk >> (i % 3)) & 1)) acc[i] = T(0);
  CG::store(r4 + gid * 3 * W, acc);
}

// u10 = P u4: vertex values copied, edge nodes the mean of their ends, then the
// fine Dirichlet DOFs zeroed
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) prolong_kernel(int64_t N10, int R, const int32_t* __restrict__ ends,
                                                           const uint8_t* __restrict__ nmask,
                                                           const T* __restrict__ u4, T* __restrict__ u10,
                                                           const int* __restrict__ skip) {
  using CG = CaseGroup<T, W>;
  if (skip && *skip) return;
  const int G = R / W;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N10 * G) return;
  const int64_t n = gid / G;
  const int r0 = (int)(gid - n * G) * W;
  const int2 ab = __ldg(reinterpret_cast<const int2*>(ends) + n);
  const int mk = __ldg(nmask + n);
  T va[3 * W];
  CG::load(u4 + ((int64_t)ab.x * R + r0) * 3, va);
  if (ab.x != ab.y) {
    T vb[3 * W];
    CG::load(u4 + ((int64_t)ab.y * R + r0) * 3, vb);
#pragma unroll
    for (int i = 0; i < 3 * W; ++i) va[i] = T(0.5) * (va[i] + vb[i]);
  }
#pragma unroll
  for (int i = 0; i < 3 * W; ++i)
    if (!((mk >> (i % 3)) & 1)) va[i] = T(0);
  CG::store(u10 + gid * 3 * W, va);
}

// K1 assembly: per element the 16 blocks K_ab = V [lam g_a g_b^T + mu g_b g_a^T +
// mu (g_a . g_b) I] added (FP64 atomics) at their block positions in row a.
__global__ void assemble4_kernel(MeshView<double> M, const int32_t* __restrict__ conn4,
                                 const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                                 double* __restrict__ vals, int* __restrict__ missing) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M.n_elem) return;
  double xc[4][3];
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 3; ++i) xc[k][i] = M.xyz[3 * (int64_t)M.conn[10 * e + k] + i];
  ElemGeo<double> G;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], M.mat[2 * e], M.mat[2 * e + 1], G);
  const double V = 20.0 * G.c, lv = G.lam * V, mv = G.mu * V;
  for (int a = 0; a < 4; ++a) {
    const int ra = conn4[4 * e + a];
    for (int b = 0; b < 4; ++b) {
      const int cb = conn4[4 * e + b];
      int pos = -1;
      for (int q = rowptr[ra]; q < rowptr[ra + 1]; ++q)
        if (cols[q] == cb) {
          pos = q;
          break;
        }
      if (pos < 0) {
        atomicExch(missing, 1);
        continue;
      }
      const double* ga = G.g[a];
      const double* gb = G.g[b];
      const double gg = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
      double* B = vals + 9 * (int64_t)pos;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          atomicAdd(B + 3 * i + j, lv * ga[i] * gb[j] + mv * gb[i] * ga[j] + (i == j ? mv * gg : 0.0));
    }
  }
}

// FP64 blocks -> FP32 blocks of K1_bc: entries coupling a fixed DOF are dropped
// and fixed DOFs get a unit diagonal
__global__ void mask4_blocks_kernel(int64_t N4, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                                    const uint8_t* __restrict__ nmask4, const double* __restrict__ v64,
                                    float* __restrict__ v32) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= N4) return;
  const int ma = nmask4[a];
  for (int q = rowptr[a]; q < rowptr[a + 1]; ++q) {
    const int b = cols[q];
    const int mb = nmask4[b];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const bool keep = ((ma >> i) & 1) && ((mb >> j) & 1);
        const float unit = (b == a && i == j && !((ma >> i) & 1)) ? 1.f : 0.f;
        v32[9 * (int64_t)q + 3 * i + j] = keep ? (float)v64[9 * (int64_t)q + 3 * i + j] : unit;
      }
  }
}

// y4 = K1_bc x4 for R cases, thread = (row, case): the row's blocks are read by
// the R threads of the row together (the same addresses), x by all R cases at
// once (3R contiguous values per column node)
__global__ void __launch_bounds__(kThreads) spmv4_kernel(int64_t N4, int R, const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ cols,
                                                         const float* __restrict__ vals, const float* __restrict__ x,
                                                         float* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N4 * R) return;
  const int64_t a = gid / R;
  const int r = (int)(gid - a * R);
  float y0 = 0.f, y1 = 0.f, y2 = 0.f;
  const int q1 = __ldg(rowptr + a + 1);
  for (int q = __ldg(rowptr + a); q < q1; ++q) {
    const int64_t b = __ldg(cols + q);
    const float* B = vals + 9 * (int64_t)q;
    const float* xb = x + (b * R + r) * 3;
    const float x0 = __ldg(xb), x1 = __ldg(xb + 1), x2 = __ldg(xb + 2);
    y0 += __ldg(B + 0) * x0 + __ldg(B + 1) * x1 + __ldg(B + 2) * x2;
    y1 += __ldg(B + 3) * x0 + __ldg(B + 4) * x1 + __ldg(B + 5) * x2;
    y2 += __ldg(B + 6) * x0 + __ldg(B + 7) * x1 + __ldg(B + 8) * x2;
  }
  float* ya = y + gid * 3;
  ya[0] = y0;
  ya[1] = y1;
  ya[2] = y2;
}

// the same product with 4 cases per thread (R a multiple of 4): each block is
// loaded once for 4 cases and the 12 x values of a column node come as three
// 16-byte loads (48-byte aligned: (b R + r0) is a multiple of 4)
__global__ void __launch_bounds__(kThreads) spmv4_group_kernel(int64_t N4, int R, const int32_t* __restrict__ rowptr,
                                                               const int32_t* __restrict__ cols,
                                                               const float* __restrict__ vals,
                                                               const float* __restrict__ x, float* __restrict__ y,
                                                               const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int G = R / 4;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N4 * G) return;
  const int64_t a = gid / G;
  const int r0 = (int)(gid - a * G) * 4;
  float acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = 0.f;
  const int q1 = __ldg(rowptr + a + 1);
  for (int q = __ldg(rowptr + a); q < q1; ++q) {
    const int64_t b = __ldg(cols + q);
    const float* B = vals + 9 * (int64_t)q;
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = __ldg(B + k);
    const float4* xb = reinterpret_cast<const float4*>(x + (b * R + r0) * 3);
    const float4 v0 = __ldg(xb), v1 = __ldg(xb + 1), v2 = __ldg(xb + 2);
    const float v[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        acc[3 * w + i] += m[3 * i] * v[3 * w] + m[3 * i + 1] * v[3 * w + 1] + m[3 * i + 2] * v[3 * w + 2];
  }
  float4* o = reinterpret_cast<float4*>(y + (a * R + r0) * 3);
  o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  o[2] = make_float4(acc[8], acc[9], acc[10], acc[11]);
}

// the same product from the sliced copy of the matrix: a warp's threads cover whole
// 8-row slices, so each of the 9 value loads and the column load of a block reads
// one sector for 8 rows (from the plain [nnzb][9] layout each read 8 sectors: ncu
// showed the L1 88 % busy and 13 sectors per load request)
__global__ void __launch_bounds__(kThreads) spmv4_sliced_kernel(int64_t N4, int R, const int32_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ sl_off,
                                                                const int32_t* __restrict__ sl_cols,
                                                                const float* __restrict__ sl_vals,
                                                                const float* __restrict__ x, float* __restrict__ y,
                                                                const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int G = R / 4;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N4 * G) return;
  const int64_t a = gid / G;
  const int r0 = (int)(gid - a * G) * 4;
  const int rr = (int)(a & 7);
  const int len = __ldg(rowptr + a + 1) - __ldg(rowptr + a);
  const int64_t base = __ldg(sl_off + (a >> 3));
  float acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = 0.f;
  for (int t = 0; t < len; ++t) {
    const int64_t slot = base + t;
    const int64_t b = __ldg(sl_cols + slot * 8 + rr);
    const float* B = sl_vals + slot * 72 + rr;
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = __ldg(B + 8 * k);
    const float4* xb = reinterpret_cast<const float4*>(x + (b * R + r0) * 3);
    const float4 v0 = __ldg(xb), v1 = __ldg(xb + 1), v2 = __ldg(xb + 2);
    const float v[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        acc[3 * w + i] += m[3 * i] * v[3 * w] + m[3 * i + 1] * v[3 * w + 1] + m[3 * i + 2] * v[3 * w + 2];
  }
  float4* o = reinterpret_cast<float4*>(y + (a * R + r0) * 3);
  o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  o[2] = make_float4(acc[8], acc[9], acc[10], acc[11]);
}

// copies the assembled blocks into the sliced layout
__global__ void slice_values_kernel(int64_t nnzb, const int32_t* __restrict__ pos, const float* __restrict__ vals,
                                    float* __restrict__ sl_vals) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  const int p = pos[q];
  float* dst = sl_vals + (int64_t)(p >> 3) * 72 + (p & 7);
#pragma unroll
  for (int k = 0; k < 9; ++k) dst[8 * k] = vals[9 * q + k];
}

// diagonal 3x3 blocks of K1: V [(lam + mu) g_a g_a^T + mu |g_a|^2 I] per corner
__global__ void jacobi4_diag_kernel(MeshView<double> M, const int32_t* __restrict__ conn4, double* __restrict__ Dg) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M.n_elem) return;
  double xc[4][3];
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 3; ++i) xc[k][i] = M.xyz[3 * (int64_t)M.conn[10 * e + k] + i];
  ElemGeo<double> G;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], M.mat[2 * e], M.mat[2 * e + 1], G);
  const double V = 20.0 * G.c;
  for (int a = 0; a < 4; ++a) {
    const double* g = G.g[a];
    const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double* D = Dg + 9 * (int64_t)conn4[4 * e + a];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) atomicAdd(D + 3 * i + j, V * ((G.lam + G.mu) * g[i] * g[j] + (i == j ? G.mu * gg : 0.0)));
  }
}

__global__ void jacobi4_invert_kernel(int64_t N, const uint8_t* __restrict__ nmask, const double* __restrict__ Dg,
                                      double* __restrict__ B64, float* __restrict__ B32, int* __restrict__ bad) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int mk = nmask[n];
  double A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const bool fi = (mk >> i) & 1, fj = (mk >> j) & 1;
      A[i][j] = (fi && fj) ? Dg[9 * n + 3 * i + j] : (i == j ? 1.0 : 0.0);
    }
  const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  if (!(det > 0.0) || !isfinite(det)) {
    atomicExch(bad, 1);
    for (int k = 0; k < 9; ++k) {
      B64[9 * n + k] = (k % 4 == 0) ? 1.0 : 0.0;
      B32[9 * n + k] = (k % 4 == 0) ? 1.f : 0.f;
    }
    return;
  }
  const double id = 1.0 / det;
  const double I[9] = {c00 * id,
                       (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id,
                       (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id,
                       c01 * id,
                       (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id,
                       (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id,
                       c02 * id,
                       (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id,
                       (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id};
  for (int k = 0; k < 9; ++k) {
    B64[9 * n + k] = I[k];
    B32[9 * n + k] = (float)I[k];
  }
}

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

}  // namespace

void build_coarse(fe_mesh* m, cudaStream_t s) {
  Coarse& c = m->coarse;
  if (c.ready) return;
  const int64_t N = m->n_nodes, E = m->n_elem;
  std::vector<int32_t> newid((size_t)N, -1);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 4; ++a) newid[(size_t)m->conn_host[(size_t)(10 * e + a)]] = 0;
  std::vector<int32_t> vertex;
  for (int64_t n = 0; n < N; ++n)
    if (newid[(size_t)n] == 0) {
      newid[(size_t)n] = (int32_t)vertex.size();
      vertex.push_back((int32_t)n);
    }
  const int64_t N4 = (int64_t)vertex.size();
  std::vector<int32_t> conn4((size_t)E * 4), ends((size_t)N * 2, -1);
  std::vector<uint8_t> own4((size_t)E, 0), mk4((size_t)N4), seen((size_t)N4, 0);
  static const int EA[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* ce = &m->conn_host[(size_t)(10 * e)];
    for (int a = 0; a < 4; ++a) {
      const int32_t v = newid[(size_t)ce[a]];
      conn4[(size_t)(4 * e + a)] = v;
      ends[(size_t)(2 * ce[a])] = v;
      ends[(size_t)(2 * ce[a] + 1)] = v;
      if (!seen[(size_t)v]) {
        seen[(size_t)v] = 1;
        own4[(size_t)e] |= (uint8_t)(1u << a);
      }
    }
    for (int q = 0; q < 6; ++q) {
      FE_REQUIRE(newid[(size_t)ce[4 + q]] < 0, "node %d is an edge node of element %lld and a corner of another",
                 ce[4 + q], (long long)m->perm_host[(size_t)e]);
      ends[(size_t)(2 * ce[4 + q])] = newid[(size_t)ce[EA[q][0]]];
      ends[(size_t)(2 * ce[4 + q] + 1)] = newid[(size_t)ce[EA[q][1]]];
    }
  }
  for (int64_t n = 0; n < N; ++n)
    FE_REQUIRE(ends[(size_t)(2 * n)] >= 0, "node %lld belongs to no element (no coarse interpolation)",
               (long long)n);
  for (int64_t v = 0; v < N4; ++v) mk4[(size_t)v] = m->nmask_host[(size_t)vertex[(size_t)v]];
  c.nmask4_host.assign(mk4.begin(), mk4.end());
  // coarse node -> the edge nodes it ends (counting sort over the fine nodes)
  std::vector<int32_t> adj_ptr((size_t)N4 + 1, 0), adj;
  for (int64_t n = 0; n < N; ++n)
    if (ends[(size_t)(2 * n)] != ends[(size_t)(2 * n + 1)]) {
      ++adj_ptr[(size_t)ends[(size_t)(2 * n)] + 1];
      ++adj_ptr[(size_t)ends[(size_t)(2 * n + 1)] + 1];
    }
  for (int64_t v = 0; v < N4; ++v) adj_ptr[(size_t)v + 1] += adj_ptr[(size_t)v];
  adj.resize((size_t)adj_ptr[(size_t)N4]);
  {
    std::vector<int32_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
    for (int64_t n = 0; n < N; ++n)
      if (ends[(size_t)(2 * n)] != ends[(size_t)(2 * n + 1)]) {
        adj[(size_t)fill[(size_t)ends[(size_t)(2 * n)]]++] = (int32_t)n;
        adj[(size_t)fill[(size_t)ends[(size_t)(2 * n + 1)]]++] = (int32_t)n;
      }
  }
  c.n_nodes = N4;
  c.conn4.alloc(conn4.size() * 4);
  c.ends.alloc(ends.size() * 4);
  c.nmask4.alloc(mk4.size());
  c.own4.alloc(own4.size());
  c.vertex.alloc(vertex.size() * 4);
  c.adj_ptr.alloc(adj_ptr.size() * 4);
  c.adj.alloc(std::max<size_t>(adj.size(), 1) * 4);
  FE_CUDA(cudaMemcpyAsync(c.conn4.ptr, conn4.data(), conn4.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.ends.ptr, ends.data(), ends.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.nmask4.ptr, mk4.data(), mk4.size(), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.own4.ptr, own4.data(), own4.size(), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.vertex.ptr, vertex.data(), vertex.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.adj_ptr.ptr, adj_ptr.data(), adj_ptr.size() * 4, cudaMemcpyHostToDevice, s));
  if (!adj.empty()) FE_CUDA(cudaMemcpyAsync(c.adj.ptr, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaStreamSynchronize(s));
  c.ready = true;
  c.jacobi_ready = false;
}

void build_coarse_jacobi(fe_mesh* m, cudaStream_t s) {
  build_coarse(m, s);
  Coarse& c = m->coarse;
  if (c.jacobi_ready) return;
  const int64_t N4 = c.n_nodes;
  DevBuf D, bad;
  D.alloc((size_t)N4 * 9 * sizeof(double));
  bad.alloc(sizeof(int));
  if (!c.binv64.ptr) c.binv64.alloc((size_t)N4 * 9 * sizeof(double));
  if (!c.binv32.ptr) c.binv32.alloc((size_t)N4 * 9 * sizeof(float));
  FE_CUDA(cudaMemsetAsync(D.ptr, 0, D.bytes, s));
  FE_CUDA(cudaMemsetAsync(bad.ptr, 0, sizeof(int), s));
  jacobi4_diag_kernel<<<blocks_for(m->n_elem), kThreads, 0, s>>>(m->view<double>(), c.conn4.as<int32_t>(),
                                                                   D.as<double>());
  FE_CHECK_LAUNCH();
  jacobi4_invert_kernel<<<blocks_for(N4), kThreads, 0, s>>>(N4, c.nmask4.as<uint8_t>(), D.as<double>(),
                                                            c.binv64.as<double>(), c.binv32.as<float>(), bad.as<int>());
  FE_CHECK_LAUNCH();
  int hbad = 0;
  FE_CUDA(cudaMemcpyAsync(&hbad, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  FE_REQUIRE(hbad == 0, "coarse block Jacobi: a free node has a singular diagonal block");
  c.jacobi_ready = true;
}

// W = 4 cases per thread where the FP32 case groups are 16-byte vectors (R a
// multiple of 4), else one case per thread.
void build_coarse_geometry(fe_mesh* m, cudaStream_t s) {
  build_coarse(m, s);
  Coarse& c = m->coarse;
  if (c.geo_ready) return;
  if (!c.geo32.ptr) c.geo32.alloc((size_t)m->n_elem * 16 * sizeof(float));
  coarse_geo_kernel<<<blocks_for(m->n_elem), kThreads, 0, s>>>(m->view<float>(), c.geo32.as<float4>());
  FE_CHECK_LAUNCH();
  c.geo_ready = true;
}

bool build_coarse_matrix(fe_mesh* m, cudaStream_t s, bool level2) {
  build_coarse(m, s);
  Coarse& c = m->coarse;
  if (c.csr_ready && (!level2 || c.l2_ready)) return true;
  const int64_t N4 = c.n_nodes, E = m->n_elem;
  if (!c.csr_pattern) {
    // block pattern: each element couples its 4 corners pairwise
    std::vector<int32_t> conn4((size_t)E * 4);
    FE_CUDA(cudaMemcpyAsync(conn4.data(), c.conn4.ptr, conn4.size() * 4, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> cnt((size_t)N4 + 1, 0);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 4; ++a) cnt[(size_t)conn4[(size_t)(4 * e + a)] + 1] += 4;
    for (int64_t v = 0; v < N4; ++v) cnt[(size_t)v + 1] += cnt[(size_t)v];
    std::vector<int32_t> cand((size_t)cnt[(size_t)N4]);
    {
      std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
      for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a) {
          const int32_t ra = conn4[(size_t)(4 * e + a)];
          for (int b = 0; b < 4; ++b) cand[(size_t)fill[(size_t)ra]++] = conn4[(size_t)(4 * e + b)];
        }
    }
    std::vector<int32_t> rowptr((size_t)N4 + 1, 0), cols;
    cols.reserve((size_t)N4 * 16);
    for (int64_t v = 0; v < N4; ++v) {
      auto b0 = cand.begin() + cnt[(size_t)v], b1 = cand.begin() + cnt[(size_t)v + 1];
      std::sort(b0, b1);
      auto e1 = std::unique(b0, b1);
      cols.insert(cols.end(), b0, e1);
      FE_REQUIRE(cols.size() < (size_t)INT32_MAX, "coarse matrix too large for 32-bit block indices");
      rowptr[(size_t)v + 1] = (int32_t)cols.size();
    }
    c.nnzb = (int64_t)cols.size();
    c.rowptr.alloc(rowptr.size() * 4);
    c.cols.alloc(cols.size() * 4);
    FE_CUDA(cudaMemcpyAsync(c.rowptr.ptr, rowptr.data(), rowptr.size() * 4, cudaMemcpyHostToDevice, s));
    FE_CUDA(cudaMemcpyAsync(c.cols.ptr, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, s));
    // sliced layout: slice k holds rows 8k..8k+7 and as many slots as its longest row
    {
      const int64_t ns = (N4 + 7) / 8;
      std::vector<int32_t> off((size_t)ns + 1, 0);
      for (int64_t k = 0; k < ns; ++k) {
        int L = 0;
        for (int64_t v = 8 * k; v < std::min<int64_t>(N4, 8 * k + 8); ++v)
          L = std::max(L, rowptr[(size_t)v + 1] - rowptr[(size_t)v]);
        FE_REQUIRE((int64_t)off[(size_t)k] + L < (int64_t)INT32_MAX / 72, "coarse matrix too large to slice");
        off[(size_t)k + 1] = off[(size_t)k] + L;
      }
      c.n_slots = off[(size_t)ns];
      std::vector<int32_t> scol((size_t)c.n_slots * 8), pos(cols.size());
      for (int64_t k = 0; k < ns; ++k)
        for (int rr = 0; rr < 8; ++rr)
          for (int32_t t = 0; t < off[(size_t)k + 1] - off[(size_t)k]; ++t)
            scol[((size_t)off[(size_t)k] + t) * 8 + rr] = (int32_t)std::min<int64_t>(N4 - 1, 8 * k + rr);
      for (int64_t v = 0; v < N4; ++v) {
        const int64_t k = v / 8, rr = v % 8;
        for (int32_t q = rowptr[(size_t)v]; q < rowptr[(size_t)v + 1]; ++q) {
          const int64_t slot = off[(size_t)k] + (q - rowptr[(size_t)v]);
          scol[(size_t)(slot * 8 + rr)] = cols[(size_t)q];
          pos[(size_t)q] = (int32_t)(slot * 8 + rr);
        }
      }
      c.sl_off.alloc(off.size() * 4);
      c.sl_cols.alloc(scol.size() * 4);
      c.sl_pos.alloc(pos.size() * 4);
      FE_CUDA(cudaMemcpyAsync(c.sl_off.ptr, off.data(), off.size() * 4, cudaMemcpyHostToDevice, s));
      FE_CUDA(cudaMemcpyAsync(c.sl_cols.ptr, scol.data(), scol.size() * 4, cudaMemcpyHostToDevice, s));
      FE_CUDA(cudaMemcpyAsync(c.sl_pos.ptr, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice, s));
      FE_CUDA(cudaStreamSynchronize(s));
    }
    c.rowptr_host = std::move(rowptr);
    c.cols_host = std::move(cols);
    c.csr_pattern = true;
  }
  // the FP32 matrix stays, the FP64 accumulator is temporary: use the assembled
  // form only where both fit in a quarter of the free memory
  size_t free_b = 0, total_b = 0;
  FE_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t need = (size_t)c.nnzb * 9 * (c.vals32.ptr ? sizeof(double) : sizeof(float) + sizeof(double));
  if (!c.sl_vals.ptr) need += (size_t)c.n_slots * 72 * sizeof(float);
  if (level2 && !c.l2_ready) need += level2_bytes(m);
  if (need > free_b / 4) return false;
  DevBuf v64, missing;
  v64.alloc((size_t)c.nnzb * 9 * sizeof(double));
  missing.alloc(sizeof(int));
  if (!c.vals32.ptr) c.vals32.alloc((size_t)c.nnzb * 9 * sizeof(float));
  FE_CUDA(cudaMemsetAsync(v64.ptr, 0, v64.bytes, s));
  FE_CUDA(cudaMemsetAsync(missing.ptr, 0, sizeof(int), s));
  assemble4_kernel<<<blocks_for(E), kThreads, 0, s>>>(m->view<double>(), c.conn4.as<int32_t>(), c.rowptr.as<int32_t>(),
                                                       c.cols.as<int32_t>(), v64.as<double>(), missing.as<int>());
  FE_CHECK_LAUNCH();
  mask4_blocks_kernel<<<blocks_for(N4), kThreads, 0, s>>>(N4, c.rowptr.as<int32_t>(), c.cols.as<int32_t>(),
                                                          c.nmask4.as<uint8_t>(), v64.as<double>(), c.vals32.as<float>());
  FE_CHECK_LAUNCH();
  int hmiss = 0;
  FE_CUDA(cudaMemcpyAsync(&hmiss, missing.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  FE_REQUIRE(hmiss == 0, "coarse matrix assembly: block outside the pattern");
  if (!c.sl_vals.ptr) {
    c.sl_vals.alloc((size_t)c.n_slots * 72 * sizeof(float));
    FE_CUDA(cudaMemsetAsync(c.sl_vals.ptr, 0, c.sl_vals.bytes, s));  // padding slots stay zero
  }
  slice_values_kernel<<<blocks_for(c.nnzb), kThreads, 0, s>>>(c.nnzb, c.sl_pos.as<int32_t>(), c.vals32.as<float>(),
                                                               c.sl_vals.as<float>());
  FE_CHECK_LAUNCH();
  c.csr_ready = true;
  if (level2 && !c.l2_ready) build_level2(m, v64.as<double>(), s);
  return true;
}

void bcsr_spmv(int64_t n, int R, const int32_t* rowptr, const int32_t* cols, const float* vals, const float* x,
               float* y, cudaStream_t s, const int* skip) {
  if (R % 4 == 0) {
    spmv4_group_kernel<<<blocks_for(n * (R / 4)), kThreads, 0, s>>>(n, R, rowptr, cols, vals, x, y, skip);
  } else {
    spmv4_kernel<<<blocks_for(n * R), kThreads, 0, s>>>(n, R, rowptr, cols, vals, x, y, skip);
  }
  FE_CHECK_LAUNCH();
}

void coarse_spmv(const fe_mesh* m, int R, const float* x4, float* y4, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.csr_ready, "coarse matrix not assembled");
  if (R % 4 == 0 && c.sl_vals.ptr) {
    spmv4_sliced_kernel<<<blocks_for(c.n_nodes * (R / 4)), kThreads, 0, s>>>(
        c.n_nodes, R, c.rowptr.as<int32_t>(), c.sl_off.as<int32_t>(), c.sl_cols.as<int32_t>(), c.sl_vals.as<float>(),
        x4, y4, skip);
    FE_CHECK_LAUNCH();
    return;
  }
  bcsr_spmv(c.n_nodes, R, c.rowptr.as<int32_t>(), c.cols.as<int32_t>(), c.vals32.as<float>(), x4, y4, s, skip);
}

template <typename T>
static int case_group(int R) {
  return (sizeof(T) == 4 && R % 4 == 0) ? 4 : 1;
}

template <typename T>
void ebe4_apply(const fe_mesh* m, int R, const T* x4, T* y4, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.ready, "coarse level not built");
  FE_REQUIRE(sizeof(T) == 8 || c.geo_ready, "coarse element data not built");
  const int64_t n4 = c.n_nodes * (int64_t)R * 3;
  zero4_kernel<T><<<std::min<unsigned>(blocks_for(n4), 152 * 16), kThreads, 0, s>>>(n4, y4, skip);
  FE_CHECK_LAUNCH();
  const int W = case_group<T>(R);
  const unsigned grid = blocks_for(m->n_elem * (R / W));
  if constexpr (sizeof(T) == 4) {
    if (W == 4) {
      ebe4_kernel<T, 4><<<grid, kThreads, 0, s>>>(m->view<T>(), c.geo32.as<float4>(), R, c.conn4.as<int32_t>(),
                                                  c.nmask4.as<uint8_t>(), c.own4.as<uint8_t>(), x4, y4, skip);
      FE_CHECK_LAUNCH();
      return;
    }
  }
  ebe4_kernel<T, 1><<<grid, kThreads, 0, s>>>(m->view<T>(), c.geo32.as<float4>(), R, c.conn4.as<int32_t>(),
                                                c.nmask4.as<uint8_t>(), c.own4.as<uint8_t>(), x4, y4, skip);
  FE_CHECK_LAUNCH();
}

template <typename T>
void coarse_restrict(const fe_mesh* m, int R, const T* r10, T* r4, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.ready, "coarse level not built");
  const int W = case_group<T>(R);
  const unsigned grid = blocks_for(c.n_nodes * (R / W));
  if constexpr (sizeof(T) == 4) {
    if (W == 4) {
      restrict_kernel<T, 4><<<grid, kThreads, 0, s>>>(c.n_nodes, R, c.vertex.as<int32_t>(), c.adj_ptr.as<int32_t>(),
                                                      c.adj.as<int32_t>(), c.nmask4.as<uint8_t>(), r10, r4, skip);
      FE_CHECK_LAUNCH();
      return;
    }
  }
  restrict_kernel<T, 1><<<grid, kThreads, 0, s>>>(c.n_nodes, R, c.vertex.as<int32_t>(), c.adj_ptr.as<int32_t>(),
                                                    c.adj.as<int32_t>(), c.nmask4.as<uint8_t>(), r10, r4, skip);
  FE_CHECK_LAUNCH();
}

template <typename T>
void coarse_prolong(const fe_mesh* m, int R, const T* u4, T* u10, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.ready, "coarse level not built");
  const int W = case_group<T>(R);
  const unsigned grid = blocks_for(m->n_nodes * (R / W));
  if constexpr (sizeof(T) == 4) {
    if (W == 4) {
      prolong_kernel<T, 4><<<grid, kThreads, 0, s>>>(m->n_nodes, R, c.ends.as<int32_t>(), m->nmask.as<uint8_t>(), u4,
                                                     u10, skip);
      FE_CHECK_LAUNCH();
      return;
    }
  }
  prolong_kernel<T, 1><<<grid, kThreads, 0, s>>>(m->n_nodes, R, c.ends.as<int32_t>(), m->nmask.as<uint8_t>(), u4,
                                                   u10, skip);
  FE_CHECK_LAUNCH();
}

template void ebe4_apply<float>(const fe_mesh*, int, const float*, float*, cudaStream_t, const int*);
template void ebe4_apply<double>(const fe_mesh*, int, const double*, double*, cudaStream_t, const int*);
template void coarse_restrict<float>(const fe_mesh*, int, const float*, float*, cudaStream_t, const int*);
template void coarse_restrict<double>(const fe_mesh*, int, const double*, double*, cudaStream_t, const int*);
template void coarse_prolong<float>(const fe_mesh*, int, const float*, float*, cudaStream_t, const int*);
template void coarse_prolong<double>(const fe_mesh*, int, const double*, double*, cudaStream_t, const int*);

}  // namespace fe

// ---------------------------------------------------------------------------
// C ABI of the coarse level
// ---------------------------------------------------------------------------
extern "C" fe_status fe_coarse_info(const fe_mesh* mesh, int64_t* n_nodes4, int32_t* vertex_host, void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe_mesh* m = const_cast<fe_mesh*>(mesh);
    fe::DeviceGuard dg(m->device);
    fe::build_coarse(m, (cudaStream_t)stream);
    if (n_nodes4) *n_nodes4 = m->coarse.n_nodes;
    if (vertex_host)
      FE_CUDA(cudaMemcpy(vertex_host, m->coarse.vertex.ptr, m->coarse.vertex.bytes, cudaMemcpyDeviceToHost));
  });
}

namespace {
// shared checks of the three vector entry points
fe_mesh* coarse_args(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* in, void* out) {
  FE_REQUIRE(mesh != nullptr && in != nullptr && out != nullptr, "NULL argument");
  FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
  FE_REQUIRE(dtype == FE_F32 || dtype == FE_F64, "dtype must be FE_F32 or FE_F64");
  FE_REQUIRE(in != out, "input and output must not alias");
  FE_REQUIRE(((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0, "vectors must be 16-byte aligned");
  return const_cast<fe_mesh*>(mesh);
}
}  // namespace

extern "C" fe_status fe_ebe4_apply(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* x4, void* y4,
                                   void* stream) {
  return fe::guarded([&] {
    fe_mesh* m = coarse_args(mesh, R, dtype, x4, y4);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::build_coarse_geometry(m, s);
    if (dtype == FE_F64)
      fe::ebe4_apply<double>(m, R, (const double*)x4, (double*)y4, s);
    else
      fe::ebe4_apply<float>(m, R, (const float*)x4, (float*)y4, s);
  });
}

extern "C" fe_status fe_coarse_restrict(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* r10, void* r4,
                                        void* stream) {
  return fe::guarded([&] {
    fe_mesh* m = coarse_args(mesh, R, dtype, r10, r4);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::build_coarse(m, s);
    if (dtype == FE_F64)
      fe::coarse_restrict<double>(m, R, (const double*)r10, (double*)r4, s);
    else
      fe::coarse_restrict<float>(m, R, (const float*)r10, (float*)r4, s);
  });
}

extern "C" fe_status fe_coarse_prolong(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* u4, void* u10,
                                       void* stream) {
  return fe::guarded([&] {
    fe_mesh* m = coarse_args(mesh, R, dtype, u4, u10);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::build_coarse(m, s);
    if (dtype == FE_F64)
      fe::coarse_prolong<double>(m, R, (const double*)u4, (double*)u10, s);
    else
      fe::coarse_prolong<float>(m, R, (const float*)u4, (float*)u10, s);
  });
}

extern "C" fe_status fe_coarse_block_jacobi(const fe_mesh* mesh, double* binv4_dev, void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(mesh != nullptr && binv4_dev != nullptr, "NULL argument");
    fe_mesh* m = const_cast<fe_mesh*>(mesh);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::build_coarse_jacobi(m, s);
    FE_CUDA(cudaMemcpyAsync(binv4_dev, m->coarse.binv64.ptr, m->coarse.binv64.bytes, cudaMemcpyDeviceToDevice, s));
  });
}

extern "C" fe_status fe_coarse_apply(const fe_mesh* mesh, int32_t R, const float* x4, float* y4, void* stream) {
  return fe::guarded([&] {
    fe_mesh* m = coarse_args(mesh, R, FE_F32, x4, y4);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    FE_REQUIRE(fe::build_coarse_matrix(m, s), "not enough free device memory for the assembled coarse matrix");
    fe::coarse_spmv(m, R, x4, y4, s);
  });
}
