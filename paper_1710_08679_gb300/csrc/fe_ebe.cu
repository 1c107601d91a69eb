// EBE product y = K_bc x for R cases (Eq. 3, multiple vectors of Sec. 3.1).
//
// Several kernels compute the same thing; fe_ebe_tune times them per (R, precision):
//  * EBE_DIRECT: one thread per (element, case). The thread recomputes the
//    element geometry, gathers its 30 inputs straight from global memory (the R
//    threads of one element read the node's 3R contiguous values together) and
//    scatters 30 results with atomic adds, as the paper's GPU port does
//    (Sec. 3.2.2: atomics keep node data local in L2 instead of colouring).
//  * EBE_TILED: elements are grouped into tiles whose nodes are staged in shared
//    memory. One CTA gathers the tile's input values once (coalesced, each node
//    contributing 3R contiguous values), computes every (element, case) product
//    of the tile from shared memory, accumulates them in shared memory and adds
//    each tile node's total to global memory once. This replaces ~10 global
//    atomics per element and case with ~(tile nodes / tile elements) of them.
//  * EBE_GATHER: tiles as above, but each element-case product goes to its own
//    shared-memory slot and each tile node sums its slots (no atomics inside the
//    tile); for 16-byte node rows the persistent pipelined form (prep pass for the
//    geometry, cp.async prefetch of the next tiles) is used.
//  * EBE_GATHER_DF: the pipelined gather kernel in float-float arithmetic (FP64
//    products on the FP32 pipe).
//  * EBE_GATHER_X2: the pipelined gather kernel with two cases per thread in
//    paired FP32 instructions.
//  * EBE_COLOUR: elements coloured so that no two of a colour share a node; one
//    launch per colour, plain read-modify-write instead of atomics.
//  * EBE_WS (fe_ebe_ws.cu): warp-specialised FP32 kernel, compute warps in paired
//    arithmetic and staging warps (loads, geometry, node sums) on greedy tiles.
// All write y = (I - P) x on constrained DOFs (copied from x by the node's owner)
// and only ever add into free DOFs after a zero pass, which yields
// P K P x + (I - P) x.
#include <algorithm>
#include <cstdio>

#include "fe_df.cuh"
#include "fe_element.cuh"
#include "fe_element_df.cuh"
#include "fe_element_x2.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kThreads = 256;

// y = 0 with 16-byte stores (write-only pass before the atomic accumulation)
template <typename T>
__global__ void __launch_bounds__(kThreads) zero_kernel(int64_t n, T* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t n4 = n * (int64_t)sizeof(T) / 16;
  float4* y4 = reinterpret_cast<float4*>(y);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) y4[i] = z;
  // tail (n * sizeof(T) not a multiple of 16)
  for (int64_t i = n4 * 16 / (int64_t)sizeof(T) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = T(0);
}

template <typename T>
__device__ __forceinline__ void load_conn(const int32_t* __restrict__ conn, int64_t e, int nd[10]) {
  const int2* c2 = reinterpret_cast<const int2*>(conn + 10 * e);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int2 v = __ldg(c2 + q);
    nd[2 * q] = v.x;
    nd[2 * q + 1] = v.y;
  }
}

template <typename T>
__device__ __forceinline__ void load_geometry(const MeshView<T>& M, int64_t e, const int nd[10], ElemGeo<T>& G) {
  T xc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[k][i] = __ldg(M.xyz + 3 * (int64_t)nd[k] + i);
  elem_geometry(xc[0], xc[1], xc[2], xc[3], __ldg(M.mat + 2 * e), __ldg(M.mat + 2 * e + 1), G);
}

// ---------------------------------------------------------------------------
// direct kernel: thread = (element, case)
// ---------------------------------------------------------------------------
// FP32: at most 128 registers so that two 256-thread blocks fit per SM
template <typename T>
struct MinBlocks {
  static constexpr int value = sizeof(T) == 4 ? 2 : 1;
};

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) ebe_direct_kernel(MeshView<T> M, int R, const uint16_t* __restrict__ own,
                                                              const T* __restrict__ x, T* __restrict__ y,
                                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= M.n_elem * R) return;
  const int64_t e = gid / R;
  const int r = (int)(gid - e * R);
  int nd[10];
  load_conn<T>(M.conn, e, nd);
  ElemGeo<T> G;
  load_geometry(M, e, nd, G);
  T u[10][3];
  int mk[10];
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    mk[a] = __ldg(M.nmask + nd[a]);
    const T* xa = x + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[a][c] = ((mk[a] >> c) & 1) ? __ldg(xa + c) : T(0);
  }
  T yl[10][3];
  elem_apply(G, u, yl);
  const int ow = __ldg(own + e);
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    T* ya = y + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if ((mk[a] >> c) & 1)
        atomicAdd(ya + c, yl[a][c]);
      else if ((ow >> a) & 1)   // constrained DOF: (I - P) x, written once by the node's owner element
        ya[c] = __ldg(x + ((int64_t)nd[a] * R + r) * 3 + c);
    }
  }
}

// ---------------------------------------------------------------------------
// colour kernel: thread = (element of one colour, case). No two elements of a
// colour share a node, and the colours run one launch after another on one
// stream, so each free value of y is read, increased and written by one thread
// at a time: no atomics, and the summation order is fixed (deterministic y).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) ebe_colour_kernel(
    MeshView<T> M, int R, const int32_t* __restrict__ elems, int64_t n, const uint16_t* __restrict__ own,
    const T* __restrict__ x, T* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= n * R) return;
  const int64_t i = gid / R;
  const int r = (int)(gid - i * R);
  const int64_t e = __ldg(elems + i);
  int nd[10];
  load_conn<T>(M.conn, e, nd);
  ElemGeo<T> G;
  load_geometry(M, e, nd, G);
  T u[10][3];
  int mk[10];
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    mk[a] = __ldg(M.nmask + nd[a]);
    const T* xa = x + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[a][c] = ((mk[a] >> c) & 1) ? __ldg(xa + c) : T(0);
  }
  T yl[10][3];
  elem_apply(G, u, yl);
  const int ow = __ldg(own + e);
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    T* ya = y + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if ((mk[a] >> c) & 1)
        ya[c] += yl[a][c];
      else if ((ow >> a) & 1)   // constrained DOF: (I - P) x, written once by the node's owner element
        ya[c] = __ldg(x + ((int64_t)nd[a] * R + r) * 3 + c);
    }
  }
}

// ---------------------------------------------------------------------------
// tiled kernel: CTA = tile of elements. Shared memory holds the tile's node
// inputs and accumulated outputs as [local node][R][3], the element geometry
// (computed once per element, shared by its R case threads) and the local
// connectivity.
// ---------------------------------------------------------------------------
constexpr int kGeo = 16;   // per element: g[4][3], lam, mu, c (15 used)

template <typename T>
__global__ void __launch_bounds__(kThreads) ebe_tiled_kernel(MeshView<T> M, int R, int tile_elems,
                                                             const int32_t* __restrict__ node_ptr,
                                                             const int32_t* __restrict__ node_ids,
                                                             const uint8_t* __restrict__ node_own,
                                                             const uint16_t* __restrict__ lconn,
                                                             const T* __restrict__ x, T* __restrict__ y,
                                                             const int* __restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const int64_t tile = blockIdx.x;
  const int nb = __ldg(node_ptr + tile);
  const int nn = __ldg(node_ptr + tile + 1) - nb;
  const int64_t e0 = tile * (int64_t)tile_elems;
  const int64_t rem = M.n_elem - e0;
  const int ne = rem < (int64_t)tile_elems ? (int)rem : tile_elems;
  const int vr = 3 * R;                                           // values per node
  T* xs = reinterpret_cast<T*>(smem_raw);                         // [nn][3R] masked inputs
  T* ys = xs + (size_t)nn * vr;                                   // [nn][3R] accumulated outputs
  T* geo = ys + (size_t)nn * vr;                                  // [ne][kGeo]
  uint16_t* lc = reinterpret_cast<uint16_t*>(geo + (size_t)tile_elems * kGeo);  // [ne][10]
  int* ids = reinterpret_cast<int*>(lc + (size_t)tile_elems * 10 + (tile_elems & 1) * 2);  // [nn]
  unsigned char* mks = reinterpret_cast<unsigned char*>(ids + nn);                        // [nn]
  unsigned char* own = mks + nn;                                                           // [nn]

  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int g = __ldg(node_ids + nb + i);
    ids[i] = g;
    mks[i] = __ldg(M.nmask + g);
    own[i] = __ldg(node_own + nb + i);
  }
  for (int i = threadIdx.x; i < ne * 10; i += blockDim.x) lc[i] = __ldg(lconn + 10 * e0 + i);
  // element geometry, once per element
  for (int le = threadIdx.x; le < ne; le += blockDim.x) {
    int nd[10];
    load_conn<T>(M.conn, e0 + le, nd);
    ElemGeo<T> G;
    load_geometry(M, e0 + le, nd, G);
    T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) gp[3 * k + i] = G.g[k][i];
    gp[12] = G.lam;
    gp[13] = G.mu;
    gp[14] = G.c;
  }
  __syncthreads();
  // gather inputs: consecutive threads read consecutive values of one node's 3R run
  const int total = nn * vr;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int ln = k / vr;
    const int w = k - ln * vr;
    const int c = w % 3;
    const T v = __ldg(x + (int64_t)ids[ln] * vr + w);
    xs[k] = ((mks[ln] >> c) & 1) ? v : T(0);
    ys[k] = T(0);
  }
  __syncthreads();

  const int items = ne * R;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int le = it / R;
    const int r = it - le * R;
    ElemGeo<T> G;
    const T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) G.g[k][i] = gp[3 * k + i];
    G.lam = gp[12];
    G.mu = gp[13];
    G.c = gp[14];
    int ln[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) ln[a] = lc[10 * le + a];
    T u[10][3];
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) u[a][c] = xs[ln[a] * vr + 3 * r + c];
    T yl[10][3];
    elem_apply(G, u, yl);
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(ys + ln[a] * vr + 3 * r + c, yl[a][c]);
  }
  __syncthreads();
  // one global add per tile node value (free DOFs); constrained DOFs: y = x,
  // stored once by the node's owner tile
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int lnn = k / vr;
    const int w = k - lnn * vr;
    const int c = w % 3;
    const int64_t gi = (int64_t)ids[lnn] * vr + w;
    if ((mks[lnn] >> c) & 1)
      atomicAdd(y + gi, ys[k]);
    else if (own[lnn])
      y[gi] = __ldg(x + gi);
  }
}

// ---------------------------------------------------------------------------
// gather kernel: CTA = tile of elements, no atomics inside the tile.
//   phase 1  node ids, masks, slot lists, element geometry -> shared; the tile's
//            node inputs -> xs [nn][3R] (16-byte loads)
//   phase 2  thread = (element, case): u from xs, y_e = K_e u_e, the 30 results
//            written to the element's own slot ob[le][a][3R] (plain stores;
//            the element stride S = 30R + (3R mod 32) keeps the lanes of
//            neighbouring elements on different banks)
//   phase 3  thread = (tile node, 16 bytes of its 3R values): sum of the slots
//            of the node's incident elements (16-byte loads), one 16-byte global
//            atomic add (free DOFs) or the owner's store of x (constrained DOFs)
// ---------------------------------------------------------------------------
template <typename T, int R>
struct GatherCfg {
  static constexpr int VR = 3 * R;                      // values per node
  static constexpr int V = 16 / (int)sizeof(T);         // values per 16-byte vector
  static constexpr bool VEC = (VR % V) == 0;
  static constexpr int S = 30 * R + ((3 * R) % 32);     // element slot stride
};

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

__device__ __forceinline__ float vget(const float4& v, int t) {
  return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}
__device__ __forceinline__ double vget(const double2& v, int t) { return t == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4& v, int t, float x) {
  if (t == 0) v.x = x; else if (t == 1) v.y = x; else if (t == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int t, double x) {
  if (t == 0) v.x = x; else v.y = x;
}
// four FP32 additions as two paired ones (same results)
__device__ __forceinline__ void vadd(float4& a, const float4& b) {
  const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
  a = make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ void vadd(double2& a, const double2& b) {
  a.x += b.x; a.y += b.y;
}
__device__ __forceinline__ void vzero(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vzero(double2& a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ void vred(float4* p, const float4& v) { atomicAdd(p, v); }
__device__ __forceinline__ void vred(double2* p, const double2& v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int R>
__host__ __device__ size_t gather_smem_bytes(int nn, int te) {
  using C = GatherCfg<T, R>;
  return align16((size_t)nn * C::VR * sizeof(T)) + align16((size_t)te * C::S * sizeof(T)) +
         align16((size_t)te * kGeo * sizeof(T)) + align16((size_t)nn * sizeof(int)) +
         align16((size_t)te * 10 * sizeof(uint16_t)) * 2 + align16((size_t)(nn + 1) * sizeof(uint16_t)) +
         align16((size_t)nn) * 2;
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) ebe_gather_kernel(MeshView<T> M, int tile_elems,
                                                              const int32_t* __restrict__ node_ptr,
                                                              const int32_t* __restrict__ node_ids,
                                                              const uint8_t* __restrict__ node_own,
                                                              const uint16_t* __restrict__ lconn,
                                                              const uint16_t* __restrict__ inc,
                                                              const uint16_t* __restrict__ inc_start,
                                                              const T* __restrict__ x, T* __restrict__ y,
                                                              const int* __restrict__ skip) {
  using C = GatherCfg<T, R>;
  using VT = typename Vec16<T>::type;
  constexpr int VR = C::VR, V = C::V, S = C::S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const int64_t tile = blockIdx.x;
  const int nb = __ldg(node_ptr + tile);
  const int nn = __ldg(node_ptr + tile + 1) - nb;
  const int64_t e0 = tile * (int64_t)tile_elems;
  const int64_t rem = M.n_elem - e0;
  const int ne = rem < (int64_t)tile_elems ? (int)rem : tile_elems;

  unsigned char* sp = smem_raw;
  T* xs = reinterpret_cast<T*>(sp);
  sp += align16((size_t)nn * VR * sizeof(T));
  T* ob = reinterpret_cast<T*>(sp);
  sp += align16((size_t)tile_elems * S * sizeof(T));
  T* geo = reinterpret_cast<T*>(sp);
  sp += align16((size_t)tile_elems * kGeo * sizeof(T));
  int* ids = reinterpret_cast<int*>(sp);
  sp += align16((size_t)nn * sizeof(int));
  uint16_t* lc = reinterpret_cast<uint16_t*>(sp);
  sp += align16((size_t)tile_elems * 10 * sizeof(uint16_t));
  uint16_t* ic = reinterpret_cast<uint16_t*>(sp);
  sp += align16((size_t)tile_elems * 10 * sizeof(uint16_t));
  uint16_t* is = reinterpret_cast<uint16_t*>(sp);
  sp += align16((size_t)(nn + 1) * sizeof(uint16_t));
  unsigned char* mks = sp;
  sp += align16((size_t)nn);
  unsigned char* own = sp;

  // ---- phase 1
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int g = __ldg(node_ids + nb + i);
    ids[i] = g;
    mks[i] = __ldg(M.nmask + g);
    own[i] = __ldg(node_own + nb + i);
    is[i] = __ldg(inc_start + nb + i);
  }
  if (threadIdx.x == 0) is[nn] = (uint16_t)(ne * 10);
  for (int i = threadIdx.x; i < ne * 10; i += blockDim.x) {
    lc[i] = __ldg(lconn + 10 * e0 + i);
    ic[i] = __ldg(inc + 10 * e0 + i);
  }
  for (int le = threadIdx.x; le < ne; le += blockDim.x) {
    int nd[10];
    load_conn<T>(M.conn, e0 + le, nd);
    ElemGeo<T> G;
    load_geometry(M, e0 + le, nd, G);
    T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) gp[3 * k + i] = G.g[k][i];
    gp[12] = G.lam;
    gp[13] = G.mu;
    gp[14] = G.c;
  }
  __syncthreads();
  if constexpr (C::VEC) {
    constexpr int CPN = VR / V;   // 16-byte chunks per node
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      VT v = __ldg(reinterpret_cast<const VT*>(x + (int64_t)ids[ln] * VR) + q);
      const int mk = mks[ln];
      if (mk != 7) {
#pragma unroll
        for (int t = 0; t < V; ++t)
          if (!((mk >> ((q * V + t) % 3)) & 1)) vset(v, t, T(0));
      }
      reinterpret_cast<VT*>(xs + ln * VR)[q] = v;
    }
  } else {
    for (int k = threadIdx.x; k < nn * VR; k += blockDim.x) {
      const int ln = k / VR;
      const int w = k - ln * VR;
      const T v = __ldg(x + (int64_t)ids[ln] * VR + w);
      xs[k] = ((mks[ln] >> (w % 3)) & 1) ? v : T(0);
    }
  }
  __syncthreads();

  // ---- phase 2
  for (int it = threadIdx.x; it < ne * R; it += blockDim.x) {
    const int le = it / R;
    const int r = it - le * R;
    ElemGeo<T> G;
    const T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) G.g[k][i] = gp[3 * k + i];
    G.lam = gp[12];
    G.mu = gp[13];
    G.c = gp[14];
    T u[10][3];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const T* xa = xs + lc[10 * le + a] * VR + 3 * r;
#pragma unroll
      for (int c = 0; c < 3; ++c) u[a][c] = xa[c];
    }
    T yl[10][3];
    elem_apply(G, u, yl);
    T* o = ob + le * S + 3 * r;
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) o[a * VR + c] = yl[a][c];
  }
  __syncthreads();

  // ---- phase 3
  if constexpr (C::VEC) {
    constexpr int CPN = VR / V;
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      VT acc;
      vzero(acc);
      const int j1 = is[ln + 1];
      for (int j = is[ln]; j < j1; ++j) {
        const int code = ic[j];
        const int le = code / 10;
        const int a = code - 10 * le;
        vadd(acc, reinterpret_cast<const VT*>(ob + le * S + a * VR)[q]);
      }
      const int64_t gi = (int64_t)ids[ln] * VR + q * V;
      const int mk = mks[ln];
      if (mk == 7) {
        vred(reinterpret_cast<VT*>(y + gi), acc);
      } else {
#pragma unroll
        for (int t = 0; t < V; ++t) {
          if ((mk >> ((q * V + t) % 3)) & 1)
            atomicAdd(y + gi + t, vget(acc, t));
          else if (own[ln])
            y[gi + t] = __ldg(x + gi + t);
        }
      }
    }
  } else {
    for (int k = threadIdx.x; k < nn * VR; k += blockDim.x) {
      const int ln = k / VR;
      const int w = k - ln * VR;
      T acc = T(0);
      const int j1 = is[ln + 1];
      for (int j = is[ln]; j < j1; ++j) {
        const int code = ic[j];
        const int le = code / 10;
        const int a = code - 10 * le;
        acc += ob[le * S + a * VR + w];
      }
      const int64_t gi = (int64_t)ids[ln] * VR + w;
      if ((mks[ln] >> (w % 3)) & 1)
        atomicAdd(y + gi, acc);
      else if (own[ln])
        y[gi] = __ldg(x + gi);
    }
  }
}

// ---------------------------------------------------------------------------
// pipelined gather kernel (persistent CTAs).
// A prep pass computes every element's geometry once per product (from the node
// coordinates and (E, nu), as the product requires) into geo[E][16] and zeroes y.
// Each CTA then walks its tiles t = blockIdx.x, + gridDim.x, ... with cp.async
// prefetch: while tile i is computed, the inputs of tile i+1 (gathered by node
// id) and the packet of tile i+2 are in flight. Phases 2 and 3 are those of the
// gather kernel. cp.async groups are waited with cp.async.wait_group (hardware
// wait, no spinning).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(kThreads) prep_kernel(MeshView<T> M, T* __restrict__ geo, int64_t nv,
                                                        T* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using VT = typename Vec16<T>::type;
  constexpr int V = 16 / (int)sizeof(T);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t e = gid; e < M.n_elem; e += stride) {
    int nd[10];
    load_conn<T>(M.conn, e, nd);
    ElemGeo<T> G;
    load_geometry(M, e, nd, G);
    T v[kGeo];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) v[3 * k + i] = G.g[k][i];
    v[12] = G.lam;
    v[13] = G.mu;
    v[14] = G.c;
    v[15] = T(0);
    VT* dst = reinterpret_cast<VT*>(geo + e * kGeo);
#pragma unroll
    for (int q = 0; q < kGeo / V; ++q) {
      VT w;
#pragma unroll
      for (int t = 0; t < V; ++t) vset(w, t, v[q * V + t]);
      dst[q] = w;
    }
  }
  const int64_t n16 = nv * (int64_t)sizeof(T) / 16;
  VT z;
  vzero(z);
  for (int64_t i = gid; i < n16; i += stride) reinterpret_cast<VT*>(y)[i] = z;
  for (int64_t i = n16 * V + gid; i < nv; i += stride) y[i] = T(0);
}

// Element slot stride of the pipelined kernel. One case per thread: the gather
// kernel's. Two cases per thread: R/2 threads per element, so 64/R elements share a
// warp; a stride of R/2 banks (mod 32) between neighbouring elements puts the
// lanes of all of them on different banks (for R = 4 the multiple of 16 bytes
// nearest to that, 2-way). Always a multiple of 16 bytes.
template <typename T, int R, int CPT>
struct PipeCfg {
  static constexpr int RC = R / CPT;  // threads per element
  static constexpr int S = CPT == 1 ? GatherCfg<T, R>::S
                                    : 30 * R + ((((RC + 3) & ~3) - 30 * R) % 32 + 32) % 32;
  static_assert(S % (16 / (int)sizeof(T)) == 0, "slot stride must keep 16-byte rows aligned");
};

template <typename T, int R, int CPT = 1>
__host__ __device__ size_t pipe_smem_bytes(int nnmax, int te, int pk) {
  using C = GatherCfg<T, R>;
  return (size_t)3 * pk + (size_t)3 * te * kGeo * sizeof(T) + (size_t)2 * nnmax * C::VR * sizeof(T) +
         (size_t)te * PipeCfg<T, R, CPT>::S * sizeof(T) + (size_t)((te * 10 + 3) & ~3) * sizeof(int) +
         (size_t)te * 12 * sizeof(int);
}

// Threads per CTA of the pipelined kernel. FP32, one case per thread: up to 768
// (one thread per element-case item of a tile, 80 registers per thread; measured
// 1 % faster than 1024 threads at 64 registers on the crust block). FP32, two
// cases per thread (paired arithmetic): up to 384, which leaves 168 registers for
// the two cases' values. FP64: 256.
template <typename T, int CPT>
struct PipeThreads {
  static constexpr int value = sizeof(T) == 4 ? (CPT == 2 ? 384 : 768) : kThreads;
};

template <typename T, int R, int CPT = 1>
__global__ void __launch_bounds__(PipeThreads<T, CPT>::value) ebe_pipe_kernel(int64_t n_tiles, int64_t n_elem, int te, int nnmax,
                                                            const unsigned char* __restrict__ packets, int pk,
                                                            const T* __restrict__ geo, const T* __restrict__ x,
                                                            T* __restrict__ y, const int* __restrict__ skip) {
  using C = GatherCfg<T, R>;
  using VT = typename Vec16<T>::type;
  constexpr int VR = C::VR, V = C::V, S = PipeCfg<T, R, CPT>::S, CPN = VR / V;
  static_assert(C::VEC, "pipelined kernel needs 16-byte node rows");
  static_assert(CPT == 1 || (CPT == 2 && sizeof(T) == 4 && R % 2 == 0), "two cases per thread: FP32, even R");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const PacketLayout L(nnmax, te);
  unsigned char* meta = smem_raw;                                   // [3][pk]
  T* geo_s = reinterpret_cast<T*>(meta + 3 * (size_t)pk);           // [3][te][16]
  T* xs = geo_s + 3 * (size_t)te * kGeo;                            // [2][nnmax][VR]
  T* ob = xs + 2 * (size_t)nnmax * VR;                              // [te][S]
  int* io = reinterpret_cast<int*>(ob + (size_t)te * S);            // [te*10] slot offsets in ob, by node
  int* no = io + ((te * 10 + 3) & ~3);                             // [te][12] node row offsets in xs (16-byte aligned)
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  if (t >= n_tiles) return;

  auto issue_meta = [&](int64_t tile, int stage) {
    const unsigned char* src = packets + tile * (int64_t)pk;
    unsigned char* dst = meta + (size_t)stage * pk;
    for (int k = threadIdx.x; k < pk / 16; k += blockDim.x) cp_async16(dst + 16 * k, src + 16 * k);
    const int64_t rem = n_elem - tile * (int64_t)te;
    const int ne = rem < (int64_t)te ? (int)rem : te;
    const T* gsrc = geo + tile * (int64_t)te * kGeo;
    T* gdst = geo_s + (size_t)stage * te * kGeo;
    const int nchunk = ne * kGeo / V;
    for (int k = threadIdx.x; k < nchunk; k += blockDim.x) cp_async16(gdst + k * V, gsrc + k * V);
  };
  auto issue_x = [&](int stage_meta, int stage_x) {
    const unsigned char* mb = meta + (size_t)stage_meta * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    T* dst = xs + (size_t)stage_x * nnmax * VR;
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      cp_async16(dst + ln * VR + q * V, x + (int64_t)ids[ln] * VR + q * V);
    }
  };

  issue_meta(t, 0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  issue_x(0, 0);
  if (t + G < n_tiles) issue_meta(t + G, 1);
  cp_async_commit();

  for (int i = 0; t < n_tiles; ++i, t += G) {
    const int ms = i % 3, xb = i & 1;
    cp_async_wait_all();
    __syncthreads();
    const unsigned char* mb = meta + (size_t)ms * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int ne = reinterpret_cast<const int*>(mb)[1];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    const unsigned char* mks = mb + L.mask;
    const unsigned char* own = mb + L.own;
    const uint16_t* is = reinterpret_cast<const uint16_t*>(mb + L.inc_start);
    const uint16_t* lc = reinterpret_cast<const uint16_t*>(mb + L.lconn);
    const uint16_t* ic = reinterpret_cast<const uint16_t*>(mb + L.inc);
    const T* gs = geo_s + (size_t)ms * te * kGeo;
    T* xcur = xs + (size_t)xb * nnmax * VR;
    // constrained components of the inputs are zero (P x)
    for (int ln = threadIdx.x; ln < nn; ln += blockDim.x) {
      const int mk = mks[ln];
      if (mk != 7)
        for (int w = 0; w < VR; ++w)
          if (!((mk >> (w % 3)) & 1)) xcur[ln * VR + w] = T(0);
    }
    // offsets: slot of each (element, node) incidence in ob, row of each element node in xs
    for (int j = threadIdx.x; j < ne * 10; j += blockDim.x) {
      const int code = ic[j];
      const int le = code / 10;
      io[j] = le * S + (code - 10 * le) * VR;
      const int e = j / 10;
      no[e * 12 + (j - 10 * e)] = lc[j] * VR;
    }
    // prefetch: inputs of the next tile, packet and geometry of the one after
    if (t + G < n_tiles) issue_x((i + 1) % 3, (i + 1) & 1);
    if (t + 2 * G < n_tiles) issue_meta(t + 2 * G, (i + 2) % 3);
    cp_async_commit();
    __syncthreads();

    // phase 2: element products into their slots; a thread takes CPT cases of one
    // element (cases r and r + R/2 when CPT = 2)
    constexpr int RC = PipeCfg<T, R, CPT>::RC;
    for (int it = threadIdx.x; it < ne * RC; it += blockDim.x) {
      const int le = it / RC;
      const int r = it - le * RC;
      ElemGeo<T> Gm;
      T gv[kGeo];
#pragma unroll
      for (int q = 0; q < kGeo / V; ++q) {
        const VT w = reinterpret_cast<const VT*>(gs + le * kGeo)[q];
#pragma unroll
        for (int t2 = 0; t2 < V; ++t2) gv[q * V + t2] = vget(w, t2);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) Gm.g[k][d] = gv[3 * k + d];
      Gm.lam = gv[12];
      Gm.mu = gv[13];
      Gm.c = gv[14];
      int off[12];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int4 w = reinterpret_cast<const int4*>(no + le * 12)[q];
        off[4 * q] = w.x;
        off[4 * q + 1] = w.y;
        off[4 * q + 2] = w.z;
        off[4 * q + 3] = w.w;
      }
      T* o = ob + le * S + 3 * r;
      if constexpr (CPT == 2) {
        float2 u[10][3];
#pragma unroll
        for (int a = 0; a < 10; ++a) {
          const T* xa = xcur + off[a] + 3 * r;
#pragma unroll
          for (int c = 0; c < 3; ++c) u[a][c] = make_float2(xa[c], xa[c + 3 * RC]);
        }
        float2 yl[10][3];
        elem_apply_x2(Gm, u, yl);
#pragma unroll
        for (int a = 0; a < 10; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            o[a * VR + c] = yl[a][c].x;
            o[a * VR + c + 3 * RC] = yl[a][c].y;
          }
      } else {
        T u[10][3];
#pragma unroll
        for (int a = 0; a < 10; ++a) {
          const T* xa = xcur + off[a] + 3 * r;
#pragma unroll
          for (int c = 0; c < 3; ++c) u[a][c] = xa[c];
        }
        T yl[10][3];
        elem_apply(Gm, u, yl);
#pragma unroll
        for (int a = 0; a < 10; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) o[a * VR + c] = yl[a][c];
      }
    }
    __syncthreads();

    // phase 3: node sums, one 16-byte atomic per 16 bytes of free values. With two
    // cases per thread (half as many threads) a thread takes two chunks of one node
    // (q0 and q0 + CPN/2): they share the node's slot offsets and loop, and their
    // loads are independent (measured: 0.859 -> 0.794 ms at R = 16, tile 24). With
    // one case per thread the single-chunk form is faster (0.810 vs 0.847 ms at tile
    // 48: two chunks per thread leave a short second round that the CTA waits for).
    constexpr int QP = (CPT == 2 && CPN % 2 == 0) ? 2 : 1;
    constexpr int CQ = CPN / QP;
    constexpr int U = QP >= 4 ? 1 : 4 / QP;  // incidences per iteration (up to 4 loads in flight)
    static_assert(U >= 1, "the incidence loop must advance");
    for (int k = threadIdx.x; k < nn * CQ; k += blockDim.x) {
      const int ln = k / CQ;
      const int q0 = k - ln * CQ;
      VT acc[2][QP];
#pragma unroll
      for (int p = 0; p < QP; ++p) {
        vzero(acc[0][p]);
        vzero(acc[1][p]);
      }
      const int j1 = is[ln + 1];
      const T* obq = ob + q0 * V;
      int j = is[ln];
      for (; j + U - 1 < j1; j += U) {
        int o[U];
#pragma unroll
        for (int u = 0; u < U; ++u) o[u] = io[j + u];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int p = 0; p < QP; ++p)
            vadd(acc[u & 1][p], *reinterpret_cast<const VT*>(obq + p * CQ * V + o[u]));
      }
      for (; j < j1; ++j) {
        const int o0 = io[j];
#pragma unroll
        for (int p = 0; p < QP; ++p) vadd(acc[0][p], *reinterpret_cast<const VT*>(obq + p * CQ * V + o0));
      }
      const int mk = mks[ln];
      const int64_t gbase = (int64_t)ids[ln] * VR;
#pragma unroll
      for (int p = 0; p < QP; ++p) {
        vadd(acc[0][p], acc[1][p]);
        const int q = q0 + p * CQ;
        const int64_t gi = gbase + q * V;
        if (mk == 7) {
          vred(reinterpret_cast<VT*>(y + gi), acc[0][p]);
        } else {
#pragma unroll
          for (int tt = 0; tt < V; ++tt) {
            if ((mk >> ((q * V + tt) % 3)) & 1)
              atomicAdd(y + gi + tt, vget(acc[0][p], tt));
            else if (own[ln])
              y[gi + tt] = __ldg(x + gi + tt);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64-accurate pipelined gather kernel in float-float arithmetic.
// Same tiles, packets and phases as ebe_pipe_kernel<double>, but the element
// products and the node sums run on the FP32 pipe in float-float (fe_df.cuh):
// the prep pass computes the geometry in FP64 and splits it into float-float,
// phase 1 splits the gathered FP64 inputs in place (integer operations), and
// phase 3 converts each node sum back to FP64 before its atomic add.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) prep_df_kernel(MeshView<double> M, df* __restrict__ geo, int64_t nv,
                                                           double* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t e = gid; e < M.n_elem; e += stride) {
    int nd[10];
    load_conn<double>(M.conn, e, nd);
    ElemGeo<double> G;
    load_geometry(M, e, nd, G);
    double v[kGeo];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) v[3 * k + i] = G.g[k][i];
    v[12] = G.lam;
    v[13] = G.mu;
    v[14] = G.c;
    v[15] = 0.0;
    float4* dst = reinterpret_cast<float4*>(geo + e * kGeo);
#pragma unroll
    for (int q = 0; q < kGeo / 2; ++q) {
      const df a = df_split(v[2 * q]), b = df_split(v[2 * q + 1]);
      dst[q] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  }
  const int64_t n16 = nv / 2;
  for (int64_t i = gid; i < n16; i += stride) reinterpret_cast<double2*>(y)[i] = make_double2(0.0, 0.0);
  for (int64_t i = n16 * 2 + gid; i < nv; i += stride) y[i] = 0.0;
}

template <int R>
__host__ __device__ size_t pipe_df_smem_bytes(int nnmax, int te, int pk) {
  // same carve-up as the FP64 kernel: float-float values are 8 bytes like doubles
  return pipe_smem_bytes<double, R>(nnmax, te, pk);
}

template <int R>
__global__ void __launch_bounds__(kThreads) ebe_pipe_df_kernel(int64_t n_tiles, int64_t n_elem, int te, int nnmax,
                                                               const unsigned char* __restrict__ packets, int pk,
                                                               const df* __restrict__ geo, const double* __restrict__ x,
                                                               double* __restrict__ y, const int* __restrict__ skip) {
  using C = GatherCfg<double, R>;
  constexpr int VR = C::VR, S = C::S, CPN = VR / 2;   // 16-byte chunks of two values
  static_assert(C::VEC, "float-float kernel needs 16-byte node rows");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const PacketLayout L(nnmax, te);
  unsigned char* meta = smem_raw;                                   // [3][pk]
  df* geo_s = reinterpret_cast<df*>(meta + 3 * (size_t)pk);         // [3][te][16]
  double* xs = reinterpret_cast<double*>(geo_s + 3 * (size_t)te * kGeo);  // [2][nnmax][VR], split in place
  df* ob = reinterpret_cast<df*>(xs + 2 * (size_t)nnmax * VR);      // [te][S]
  int* io = reinterpret_cast<int*>(ob + (size_t)te * S);            // [te*10]
  int* no = io + ((te * 10 + 3) & ~3);                              // [te][12]
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  if (t >= n_tiles) return;

  auto issue_meta = [&](int64_t tile, int stage) {
    const unsigned char* src = packets + tile * (int64_t)pk;
    unsigned char* dst = meta + (size_t)stage * pk;
    for (int k = threadIdx.x; k < pk / 16; k += blockDim.x) cp_async16(dst + 16 * k, src + 16 * k);
    const int64_t rem = n_elem - tile * (int64_t)te;
    const int ne = rem < (int64_t)te ? (int)rem : te;
    const df* gsrc = geo + tile * (int64_t)te * kGeo;
    df* gdst = geo_s + (size_t)stage * te * kGeo;
    for (int k = threadIdx.x; k < ne * kGeo / 2; k += blockDim.x) cp_async16(gdst + 2 * k, gsrc + 2 * k);
  };
  auto issue_x = [&](int stage_meta, int stage_x) {
    const unsigned char* mb = meta + (size_t)stage_meta * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    double* dst = xs + (size_t)stage_x * nnmax * VR;
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      cp_async16(dst + ln * VR + 2 * q, x + (int64_t)ids[ln] * VR + 2 * q);
    }
  };

  issue_meta(t, 0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  issue_x(0, 0);
  if (t + G < n_tiles) issue_meta(t + G, 1);
  cp_async_commit();

  for (int i = 0; t < n_tiles; ++i, t += G) {
    const int ms = i % 3, xb = i & 1;
    cp_async_wait_all();
    __syncthreads();
    const unsigned char* mb = meta + (size_t)ms * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int ne = reinterpret_cast<const int*>(mb)[1];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    const unsigned char* mks = mb + L.mask;
    const unsigned char* own = mb + L.own;
    const uint16_t* is = reinterpret_cast<const uint16_t*>(mb + L.inc_start);
    const uint16_t* lc = reinterpret_cast<const uint16_t*>(mb + L.lconn);
    const uint16_t* ic = reinterpret_cast<const uint16_t*>(mb + L.inc);
    const df* gs = geo_s + (size_t)ms * te * kGeo;
    double* xd = xs + (size_t)xb * nnmax * VR;
    df* xcur = reinterpret_cast<df*>(xd);
    // split the inputs in place (P x: constrained components become zero)
    for (int k = threadIdx.x; k < nn * VR; k += blockDim.x) {
      const int ln = k / VR;
      const int w = k - ln * VR;
      const double v = xd[k];
      xcur[k] = ((mks[ln] >> (w % 3)) & 1) ? df_split(v) : df(0.f, 0.f);
    }
    for (int j = threadIdx.x; j < ne * 10; j += blockDim.x) {
      const int code = ic[j];
      const int le = code / 10;
      io[j] = le * S + (code - 10 * le) * VR;
      const int e = j / 10;
      no[e * 12 + (j - 10 * e)] = lc[j] * VR;
    }
    if (t + G < n_tiles) issue_x((i + 1) % 3, (i + 1) & 1);
    if (t + 2 * G < n_tiles) issue_meta(t + 2 * G, (i + 2) % 3);
    cp_async_commit();
    __syncthreads();

    for (int it = threadIdx.x; it < ne * R; it += blockDim.x) {
      const int le = it / R;
      const int r = it - le * R;
      ElemGeo<df> Gm;
      df gv[kGeo];
#pragma unroll
      for (int q = 0; q < kGeo / 2; ++q) {
        const float4 w = reinterpret_cast<const float4*>(gs + le * kGeo)[q];
        gv[2 * q] = df(w.x, w.y);
        gv[2 * q + 1] = df(w.z, w.w);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) Gm.g[k][d] = gv[3 * k + d];
      Gm.lam = gv[12];
      Gm.mu = gv[13];
      Gm.c = gv[14];
      int off[12];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int4 w = reinterpret_cast<const int4*>(no + le * 12)[q];
        off[4 * q] = w.x;
        off[4 * q + 1] = w.y;
        off[4 * q + 2] = w.z;
        off[4 * q + 3] = w.w;
      }
      df u[10][3];
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        const df* xa = xcur + off[a] + 3 * r;
#pragma unroll
        for (int c = 0; c < 3; ++c) u[a][c] = xa[c];
      }
      df yl[10][3];
      elem_apply(Gm, u, yl);
      df* o = ob + le * S + 3 * r;
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[a * VR + c] = yl[a][c];
    }
    __syncthreads();

    // node sums in float-float, converted to FP64 for the global atomic add
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      df a0, a1;
      const int j1 = is[ln + 1];
      const df* obq = ob + 2 * q;
      for (int j = is[ln]; j < j1; ++j) {
        const float4 w = *reinterpret_cast<const float4*>(obq + io[j]);
        a0 += df(w.x, w.y);
        a1 += df(w.z, w.w);
      }
      const int64_t gi = (int64_t)ids[ln] * VR + 2 * q;
      const int mk = mks[ln];
      const df acc[2] = {a0, a1};
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        if ((mk >> ((2 * q + tt) % 3)) & 1)
          atomicAdd(y + gi + tt, df_to_double(acc[tt]));
        else if (own[ln])
          y[gi + tt] = __ldg(x + gi + tt);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Float-float kernel for two blocks per SM (FE_EBE_DF_LEAN). The tiles, packets,
// split, slots and node sums of ebe_pipe_df_kernel, with
//  * elem_apply_df_lean: node values and geometry read from shared memory where
//    they are used and outputs stored as they are formed, so the product fits in
//    128 registers per thread;
//  * one input stage: the next tile's rows are copied while this tile's node
//    sums run (they read only the slots), which halves that buffer.
// Two 256-thread blocks per SM then overlap each other's phases (split, element
// products, node sums) where the one-block kernel waits on its own latencies.
// ---------------------------------------------------------------------------
template <int R>
__host__ __device__ size_t pipe_df_lean_smem_bytes(int nnmax, int te, int pk) {
  using C = GatherCfg<double, R>;
  return (size_t)3 * pk + (size_t)3 * te * kGeo * sizeof(df) + (size_t)nnmax * C::VR * sizeof(double) +
         (size_t)te * C::S * sizeof(df) + (size_t)((te * 10 + 3) & ~3) * sizeof(int) + (size_t)te * 12 * sizeof(int);
}

template <int R>
__global__ void __launch_bounds__(kThreads, 2) ebe_pipe_df_lean_kernel(int64_t n_tiles, int64_t n_elem, int te,
                                                                       int nnmax,
                                                                       const unsigned char* __restrict__ packets,
                                                                       int pk, const df* __restrict__ geo,
                                                                       const double* __restrict__ x,
                                                                       double* __restrict__ y,
                                                                       const int* __restrict__ skip) {
  using C = GatherCfg<double, R>;
  constexpr int VR = C::VR, S = C::S, CPN = VR / 2;   // 16-byte chunks of two values
  static_assert(C::VEC, "float-float kernel needs 16-byte node rows");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const PacketLayout L(nnmax, te);
  unsigned char* meta = smem_raw;                                   // [3][pk]
  df* geo_s = reinterpret_cast<df*>(meta + 3 * (size_t)pk);         // [3][te][16]
  double* xd = reinterpret_cast<double*>(geo_s + 3 * (size_t)te * kGeo);  // [nnmax][VR], split in place
  df* ob = reinterpret_cast<df*>(xd + (size_t)nnmax * VR);          // [te][S]
  int* io = reinterpret_cast<int*>(ob + (size_t)te * S);            // [te*10]
  int* no = io + ((te * 10 + 3) & ~3);                              // [te][12]
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  if (t >= n_tiles) return;

  auto issue_meta = [&](int64_t tile, int stage) {
    const unsigned char* src = packets + tile * (int64_t)pk;
    unsigned char* dst = meta + (size_t)stage * pk;
    for (int k = threadIdx.x; k < pk / 16; k += blockDim.x) cp_async16(dst + 16 * k, src + 16 * k);
    const int64_t rem = n_elem - tile * (int64_t)te;
    const int ne = rem < (int64_t)te ? (int)rem : te;
    const df* gsrc = geo + tile * (int64_t)te * kGeo;
    df* gdst = geo_s + (size_t)stage * te * kGeo;
    for (int k = threadIdx.x; k < ne * kGeo / 2; k += blockDim.x) cp_async16(gdst + 2 * k, gsrc + 2 * k);
  };
  auto issue_x = [&](int stage_meta) {
    const unsigned char* mb = meta + (size_t)stage_meta * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      cp_async16(xd + ln * VR + 2 * q, x + (int64_t)ids[ln] * VR + 2 * q);
    }
  };

  issue_meta(t, 0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  issue_x(0);
  if (t + G < n_tiles) issue_meta(t + G, 1);
  cp_async_commit();

  for (int i = 0; t < n_tiles; ++i, t += G) {
    const int ms = i % 3;
    cp_async_wait_all();      // this tile's rows and the next tile's packet
    __syncthreads();
    const unsigned char* mb = meta + (size_t)ms * pk;
    const int nn = reinterpret_cast<const int*>(mb)[0];
    const int ne = reinterpret_cast<const int*>(mb)[1];
    const int* ids = reinterpret_cast<const int*>(mb + L.ids);
    const unsigned char* mks = mb + L.mask;
    const unsigned char* own = mb + L.own;
    const uint16_t* is = reinterpret_cast<const uint16_t*>(mb + L.inc_start);
    const uint16_t* lc = reinterpret_cast<const uint16_t*>(mb + L.lconn);
    const uint16_t* ic = reinterpret_cast<const uint16_t*>(mb + L.inc);
    const df* gs = geo_s + (size_t)ms * te * kGeo;
    df* xcur = reinterpret_cast<df*>(xd);
    // split the inputs in place (P x: constrained components become zero)
    for (int k = threadIdx.x; k < nn * VR; k += blockDim.x) {
      const int ln = k / VR;
      const int w = k - ln * VR;
      const double v = xd[k];
      xcur[k] = ((mks[ln] >> (w % 3)) & 1) ? df_split(v) : df(0.f, 0.f);
    }
    for (int j = threadIdx.x; j < ne * 10; j += blockDim.x) {
      const int code = ic[j];
      const int le = code / 10;
      io[j] = le * S + (code - 10 * le) * VR;
      const int e = j / 10;
      no[e * 12 + (j - 10 * e)] = lc[j] * VR;
    }
    if (t + 2 * G < n_tiles) issue_meta(t + 2 * G, (i + 2) % 3);
    cp_async_commit();
    __syncthreads();

    for (int it = threadIdx.x; it < ne * R; it += blockDim.x) {
      const int le = it / R;
      const int r = it - le * R;
      int off[12];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int4 w = reinterpret_cast<const int4*>(no + le * 12)[q];
        off[4 * q] = w.x;
        off[4 * q + 1] = w.y;
        off[4 * q + 2] = w.z;
        off[4 * q + 3] = w.w;
      }
      elem_apply_df_lean<VR>(gs + le * kGeo, xcur + 3 * r, off, ob + le * S + 3 * r);
    }
    __syncthreads();
    // the next tile's rows into the one input buffer while the node sums run
    if (t + G < n_tiles) issue_x((i + 1) % 3);
    cp_async_commit();

    // node sums in float-float, converted to FP64 for the global atomic add
    for (int k = threadIdx.x; k < nn * CPN; k += blockDim.x) {
      const int ln = k / CPN;
      const int q = k - ln * CPN;
      df a0, a1;
      const int j1 = is[ln + 1];
      const df* obq = ob + 2 * q;
      for (int j = is[ln]; j < j1; ++j) {
        const float4 w = *reinterpret_cast<const float4*>(obq + io[j]);
        a0 += df(w.x, w.y);
        a1 += df(w.z, w.w);
      }
      const int64_t gi = (int64_t)ids[ln] * VR + 2 * q;
      const int mk = mks[ln];
      const df acc[2] = {a0, a1};
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        if ((mk >> ((2 * q + tt) % 3)) & 1)
          atomicAdd(y + gi + tt, df_to_double(acc[tt]));
        else if (own[ln])
          y[gi + tt] = __ldg(x + gi + tt);
      }
    }
  }
}

template <typename T>
size_t tiled_smem_bytes(int max_nodes, int tile_elems, int R) {
  size_t b = (size_t)max_nodes * 3 * R * sizeof(T) * 2 + (size_t)tile_elems * kGeo * sizeof(T) +
             (size_t)tile_elems * 10 * sizeof(uint16_t) + 4 + (size_t)max_nodes * (sizeof(int) + 2);
  return (b + 15) & ~size_t(15);
}

}  // namespace

template <typename T>
static void launch_direct(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip) {
  const MeshView<T> M = m->view<T>();
  const int64_t total = M.n_elem * R;
  const int64_t blocks = (total + kThreads - 1) / kThreads;
  ebe_direct_kernel<T><<<(unsigned)blocks, kThreads, 0, s>>>(M, R, m->own_elem.as<uint16_t>(), x, y, skip);
  FE_CHECK_LAUNCH();
}

template <typename T>
static void launch_colour(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip) {
  const Colouring& c = m->colouring;
  FE_REQUIRE(c.ready, "element colouring was not built");
  const MeshView<T> M = m->view<T>();
  for (int k = 0; k < c.n_colours; ++k) {
    const int64_t n = c.ptr[(size_t)k + 1] - c.ptr[(size_t)k];
    if (n == 0) continue;
    const int64_t blocks = (n * R + kThreads - 1) / kThreads;
    ebe_colour_kernel<T><<<(unsigned)blocks, kThreads, 0, s>>>(M, R, c.elems.as<int32_t>() + c.ptr[(size_t)k], n,
                                                              m->own_elem.as<uint16_t>(), x, y, skip);
    FE_CHECK_LAUNCH();
  }
}

static int max_smem_optin(int device) {
  int v = 0;
  FE_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  return v;
}

bool gather_supported(int R) { return R == 1 || R == 2 || R == 3 || R == 4 || R == 8 || R == 16 || R == 32; }

template <typename T>
static size_t gather_bytes(int R, int nn, int te) {
  switch (R) {
    case 1: return gather_smem_bytes<T, 1>(nn, te);
    case 2: return gather_smem_bytes<T, 2>(nn, te);
    case 3: return gather_smem_bytes<T, 3>(nn, te);
    case 4: return gather_smem_bytes<T, 4>(nn, te);
    case 8: return gather_smem_bytes<T, 8>(nn, te);
    case 16: return gather_smem_bytes<T, 16>(nn, te);
    case 32: return gather_smem_bytes<T, 32>(nn, te);
    default: return (size_t)1 << 40;
  }
}

bool tiled_fits(const fe_mesh* m, int tile_elems, int R, int is_f32, int kind) {
  auto it = m->tilings.find(tile_elems);
  // before the tiling exists, bound its node count by 10 nodes per element
  const int nodes = it != m->tilings.end() ? it->second->max_nodes : 10 * tile_elems;
  size_t smem;
  if (kind == FE_EBE_GATHER)
    smem = is_f32 ? gather_bytes<float>(R, nodes, tile_elems) : gather_bytes<double>(R, nodes, tile_elems);
  else
    smem = is_f32 ? tiled_smem_bytes<float>(nodes, tile_elems, R) : tiled_smem_bytes<double>(nodes, tile_elems, R);
  return smem <= (size_t)max_smem_optin(m->device);
}

template <typename T, int R>
static void launch_gather_r(const fe_mesh* m, const Tiling& t, const T* x, T* y, cudaStream_t s, const int* skip) {
  const size_t smem = gather_smem_bytes<T, R>(t.max_nodes, t.tile_elems);
  FE_REQUIRE(smem <= (size_t)max_smem_optin(m->device), "gather tile of %d elements needs %zu B shared memory",
             t.tile_elems, smem);
  FE_CUDA(cudaFuncSetAttribute(ebe_gather_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ebe_gather_kernel<T, R><<<(unsigned)t.n_tiles, kThreads, smem, s>>>(
      m->view<T>(), t.tile_elems, t.node_ptr.as<int32_t>(), t.node_ids.as<int32_t>(), t.node_own.as<uint8_t>(),
      t.lconn.as<uint16_t>(), t.inc.as<uint16_t>(), t.inc_start.as<uint16_t>(), x, y, skip);
  FE_CHECK_LAUNCH();
}

template <typename T, int R, int CPT = 1>
static bool launch_pipe_r(const fe_mesh* m, const Tiling& t, const T* x, T* y, cudaStream_t s, const int* skip) {
  if constexpr (!GatherCfg<T, R>::VEC || (CPT == 2 && (sizeof(T) != 4 || R % 2 != 0))) {
    return false;
  } else {
    const DevBuf& gb = sizeof(T) == 4 ? m->geo32 : m->geo64;
    if (!gb.ptr || t.packet_bytes == 0) return false;
    const size_t smem = pipe_smem_bytes<T, R, CPT>(t.max_nodes, t.tile_elems, t.packet_bytes);
    if (smem > (size_t)max_smem_optin(m->device)) return false;
    FE_CUDA(cudaFuncSetAttribute(ebe_pipe_kernel<T, R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    // one thread per element item (CPT cases) of a full tile (FP32), in whole warps
    int threads = kThreads;
    if (sizeof(T) == 4) {
      constexpr int tmax = PipeThreads<T, CPT>::value;
      threads = ((t.tile_elems * (R / CPT) + 31) / 32) * 32;
      threads = threads < 128 ? 128 : (threads > tmax ? tmax : threads);
    }
    int per_sm = 0, sms = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ebe_pipe_kernel<T, R, CPT>, threads, smem));
    FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    if (per_sm < 1) return false;
    const int64_t nv = m->n_nodes * (int64_t)R * 3;
    prep_kernel<T><<<(unsigned)(sms * 8), kThreads, 0, s>>>(m->view<T>(), gb.as<T>(), nv, y, skip);
    FE_CHECK_LAUNCH();
    const int64_t grid = std::min<int64_t>(t.n_tiles, (int64_t)per_sm * sms);
    ebe_pipe_kernel<T, R, CPT><<<(unsigned)grid, threads, smem, s>>>(
        t.n_tiles, m->n_elem, t.tile_elems, t.max_nodes, t.packets.as<unsigned char>(), t.packet_bytes, gb.as<T>(),
        x, y, skip);
    FE_CHECK_LAUNCH();
    return true;
  }
}

template <int R>
static bool launch_pipe_df_r(const fe_mesh* m, const Tiling& t, const double* x, double* y, cudaStream_t s,
                             const int* skip) {
  if (!m->geodf.ptr || t.packet_bytes == 0) return false;
  const size_t smem = pipe_df_smem_bytes<R>(t.max_nodes, t.tile_elems, t.packet_bytes);
  if (smem > (size_t)max_smem_optin(m->device)) return false;
  FE_CUDA(cudaFuncSetAttribute(ebe_pipe_df_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ebe_pipe_df_kernel<R>, kThreads, smem));
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  if (per_sm < 1) return false;
  const int64_t nv = m->n_nodes * (int64_t)R * 3;
  prep_df_kernel<<<(unsigned)(sms * 8), kThreads, 0, s>>>(m->view<double>(), m->geodf.as<df>(), nv, y, skip);
  FE_CHECK_LAUNCH();
  const int64_t grid = std::min<int64_t>(t.n_tiles, (int64_t)per_sm * sms);
  ebe_pipe_df_kernel<R><<<(unsigned)grid, kThreads, smem, s>>>(t.n_tiles, m->n_elem, t.tile_elems, t.max_nodes,
                                                               t.packets.as<unsigned char>(), t.packet_bytes,
                                                               m->geodf.as<df>(), x, y, skip);
  FE_CHECK_LAUNCH();
  return true;
}

static bool launch_pipe_df(const fe_mesh* m, const Tiling& t, int R, const double* x, double* y, cudaStream_t s,
                           const int* skip) {
  switch (R) {
    case 2: return launch_pipe_df_r<2>(m, t, x, y, s, skip);
    case 4: return launch_pipe_df_r<4>(m, t, x, y, s, skip);
    case 8: return launch_pipe_df_r<8>(m, t, x, y, s, skip);
    case 16: return launch_pipe_df_r<16>(m, t, x, y, s, skip);
    case 32: return launch_pipe_df_r<32>(m, t, x, y, s, skip);
    default: return false;
  }
}

template <int R>
static bool launch_pipe_df_lean_r(const fe_mesh* m, const Tiling& t, const double* x, double* y, cudaStream_t s,
                                  const int* skip) {
  if (!m->geodf.ptr || t.packet_bytes == 0) return false;
  const size_t smem = pipe_df_lean_smem_bytes<R>(t.max_nodes, t.tile_elems, t.packet_bytes);
  if (smem > (size_t)max_smem_optin(m->device)) return false;
  FE_CUDA(cudaFuncSetAttribute(ebe_pipe_df_lean_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ebe_pipe_df_lean_kernel<R>, kThreads, smem));
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  if (per_sm < 1) return false;
  const int64_t nv = m->n_nodes * (int64_t)R * 3;
  prep_df_kernel<<<(unsigned)(sms * 8), kThreads, 0, s>>>(m->view<double>(), m->geodf.as<df>(), nv, y, skip);
  FE_CHECK_LAUNCH();
  const int64_t grid = std::min<int64_t>(t.n_tiles, (int64_t)per_sm * sms);
  ebe_pipe_df_lean_kernel<R><<<(unsigned)grid, kThreads, smem, s>>>(
      t.n_tiles, m->n_elem, t.tile_elems, t.max_nodes, t.packets.as<unsigned char>(), t.packet_bytes,
      m->geodf.as<df>(), x, y, skip);
  FE_CHECK_LAUNCH();
  return true;
}

static bool launch_pipe_df_lean(const fe_mesh* m, const Tiling& t, int R, const double* x, double* y,
                                cudaStream_t s, const int* skip) {
  switch (R) {
    case 2: return launch_pipe_df_lean_r<2>(m, t, x, y, s, skip);
    case 4: return launch_pipe_df_lean_r<4>(m, t, x, y, s, skip);
    case 8: return launch_pipe_df_lean_r<8>(m, t, x, y, s, skip);
    case 16: return launch_pipe_df_lean_r<16>(m, t, x, y, s, skip);
    case 32: return launch_pipe_df_lean_r<32>(m, t, x, y, s, skip);
    default: return false;
  }
}

// FP32 pipelined kernel with two cases per thread (paired arithmetic), R in {4, 8, 16, 32}
static bool launch_pipe_x2(const fe_mesh* m, const Tiling& t, int R, const float* x, float* y, cudaStream_t s,
                           const int* skip) {
  switch (R) {
    case 4: return launch_pipe_r<float, 4, 2>(m, t, x, y, s, skip);
    case 8: return launch_pipe_r<float, 8, 2>(m, t, x, y, s, skip);
    case 16: return launch_pipe_r<float, 16, 2>(m, t, x, y, s, skip);
    case 32: return launch_pipe_r<float, 32, 2>(m, t, x, y, s, skip);
    default: return false;
  }
}

template <typename T>
static bool launch_pipe(const fe_mesh* m, const Tiling& t, int R, const T* x, T* y, cudaStream_t s,
                        const int* skip) {
  switch (R) {
    case 4: return launch_pipe_r<T, 4>(m, t, x, y, s, skip);
    case 8: return launch_pipe_r<T, 8>(m, t, x, y, s, skip);
    case 16: return launch_pipe_r<T, 16>(m, t, x, y, s, skip);
    case 32: return launch_pipe_r<T, 32>(m, t, x, y, s, skip);
    case 2: return launch_pipe_r<T, 2>(m, t, x, y, s, skip);
    default: return false;
  }
}

template <typename T>
static void launch_gather(const fe_mesh* m, const Tiling& t, int R, const T* x, T* y, cudaStream_t s,
                          const int* skip) {
  switch (R) {
    case 1: return launch_gather_r<T, 1>(m, t, x, y, s, skip);
    case 2: return launch_gather_r<T, 2>(m, t, x, y, s, skip);
    case 3: return launch_gather_r<T, 3>(m, t, x, y, s, skip);
    case 4: return launch_gather_r<T, 4>(m, t, x, y, s, skip);
    case 8: return launch_gather_r<T, 8>(m, t, x, y, s, skip);
    case 16: return launch_gather_r<T, 16>(m, t, x, y, s, skip);
    case 32: return launch_gather_r<T, 32>(m, t, x, y, s, skip);
    default: FE_REQUIRE(false, "gather kernel not compiled for R = %d", R);
  }
}

template <typename T>
static void launch_tiled(const fe_mesh* m, const Tiling& t, int R, const T* x, T* y, cudaStream_t s,
                         const int* skip) {
  const size_t smem = tiled_smem_bytes<T>(t.max_nodes, t.tile_elems, R);
  FE_REQUIRE(smem <= (size_t)max_smem_optin(m->device), "tile of %d elements needs %zu B shared memory",
             t.tile_elems, smem);
  FE_CUDA(cudaFuncSetAttribute(ebe_tiled_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const MeshView<T> M = m->view<T>();
  ebe_tiled_kernel<T><<<(unsigned)t.n_tiles, kThreads, smem, s>>>(
      M, R, t.tile_elems, t.node_ptr.as<int32_t>(), t.node_ids.as<int32_t>(), t.node_own.as<uint8_t>(),
      t.lconn.as<uint16_t>(), x, y, skip);
  FE_CHECK_LAUNCH();
}

int ebe_get_variant(const fe_mesh* m, int R, int is_f32) {
  const int v = m->variant[is_f32 ? 1 : 0][R];
  return v < 0 ? 0 : v;
}

void ebe_set_variant(fe_mesh* m, int R, int is_f32, int variant) { m->variant[is_f32 ? 1 : 0][R] = variant; }

template <typename T>
static void zero_pass(const fe_mesh* m, int R, T* y, cudaStream_t s, const int* skip) {
  const int64_t nv = m->n_nodes * (int64_t)R * 3;
  int sms = 0;
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  const int64_t zb = (nv * (int64_t)sizeof(T) / 16 + kThreads - 1) / kThreads;
  zero_kernel<T><<<(unsigned)(zb < (int64_t)sms * 16 ? (zb > 0 ? zb : 1) : (int64_t)sms * 16), kThreads, 0, s>>>(
      nv, y, skip);
  FE_CHECK_LAUNCH();
}

template <typename T>
void ebe_apply(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip) {
  const int v = ebe_get_variant(m, R, sizeof(T) == 4);
  const int kind = v / 65536, tile = v % 65536;
  if (kind == FE_EBE_COLOUR) {
    zero_pass<T>(m, R, y, s, skip);
    launch_colour<T>(m, R, x, y, s, skip);
    return;
  }
  if (kind == FE_EBE_WS || kind == FE_EBE_WS2) {
    if constexpr (sizeof(T) == 4) {
      auto it = m->ws_tilings.find(tile * 256 + R);
      FE_REQUIRE(it != m->ws_tilings.end(), "warp-specialised tiling of %d elements for R = %d was not built", tile,
                 R);
      zero_pass<T>(m, R, y, s, skip);
      launch_ws(m, *it->second, x, y, s, skip, kind == FE_EBE_WS2 ? 256 : 512);
    } else {
      FE_REQUIRE(false, "the warp-specialised kernel computes FP32 products only");
    }
    return;
  }
  if (kind != FE_EBE_DIRECT) {
    auto it = m->tilings.find(tile);
    FE_REQUIRE(it != m->tilings.end(), "tiling of %d elements was not built", tile);
    if (kind == FE_EBE_GATHER_DF || kind == FE_EBE_DF_LEAN) {
      if constexpr (sizeof(T) == 8) {
        const bool ok = kind == FE_EBE_GATHER_DF ? launch_pipe_df(m, *it->second, R, x, y, s, skip)
                                                 : launch_pipe_df_lean(m, *it->second, R, x, y, s, skip);
        FE_REQUIRE(ok, "float-float kernel unavailable for R = %d with tiles of %d elements", R, tile);
      } else {
        FE_REQUIRE(false, "the float-float kernel computes FP64 products only");
      }
    } else if (kind == FE_EBE_GATHER_X2) {
      if constexpr (sizeof(T) == 4) {
        FE_REQUIRE(launch_pipe_x2(m, *it->second, R, x, y, s, skip),
                   "paired-arithmetic kernel unavailable for R = %d with tiles of %d elements", R, tile);
      } else {
        FE_REQUIRE(false, "the paired-arithmetic kernel computes FP32 products only");
      }
    } else if (kind == FE_EBE_GATHER) {
      if (launch_pipe<T>(m, *it->second, R, x, y, s, skip)) return;
      zero_pass<T>(m, R, y, s, skip);
      launch_gather<T>(m, *it->second, R, x, y, s, skip);
    } else {
      zero_pass<T>(m, R, y, s, skip);
      launch_tiled<T>(m, *it->second, R, x, y, s, skip);
    }
    return;
  }
  zero_pass<T>(m, R, y, s, skip);
  launch_direct<T>(m, R, x, y, s, skip);
}

void ensure_geometry_buffer(fe_mesh* m, int is_f32) {
  DevBuf& b = is_f32 ? m->geo32 : m->geo64;
  if (!b.ptr) b.alloc((size_t)m->n_elem * kGeo * (is_f32 ? sizeof(float) : sizeof(double)));
  if (!is_f32 && !m->geodf.ptr) m->geodf.alloc((size_t)m->n_elem * kGeo * sizeof(df));
}

bool df_supported(int R) { return R == 2 || R == 4 || R == 8 || R == 16 || R == 32; }

bool x2_supported(int R) { return R == 4 || R == 8 || R == 16 || R == 32; }

bool x2_fits(const fe_mesh* m, int tile_elems, int R) {
  auto it = m->tilings.find(tile_elems);
  if (it == m->tilings.end()) return false;
  const Tiling& t = *it->second;
  if (t.packet_bytes == 0) return false;
  size_t smem;
  switch (R) {
    case 4: smem = pipe_smem_bytes<float, 4, 2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 8: smem = pipe_smem_bytes<float, 8, 2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 16: smem = pipe_smem_bytes<float, 16, 2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 32: smem = pipe_smem_bytes<float, 32, 2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    default: return false;
  }
  return smem <= (size_t)max_smem_optin(m->device);
}

bool df_fits(const fe_mesh* m, int tile_elems, int R) {
  auto it = m->tilings.find(tile_elems);
  if (it == m->tilings.end()) return false;
  const Tiling& t = *it->second;
  size_t smem;
  switch (R) {
    case 2: smem = pipe_df_smem_bytes<2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 4: smem = pipe_df_smem_bytes<4>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 8: smem = pipe_df_smem_bytes<8>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 16: smem = pipe_df_smem_bytes<16>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 32: smem = pipe_df_smem_bytes<32>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    default: return false;
  }
  return smem <= (size_t)max_smem_optin(m->device);
}

bool df_lean_fits(const fe_mesh* m, int tile_elems, int R) {
  auto it = m->tilings.find(tile_elems);
  if (it == m->tilings.end()) return false;
  const Tiling& t = *it->second;
  size_t smem;
  switch (R) {
    case 2: smem = pipe_df_lean_smem_bytes<2>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 4: smem = pipe_df_lean_smem_bytes<4>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 8: smem = pipe_df_lean_smem_bytes<8>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 16: smem = pipe_df_lean_smem_bytes<16>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    case 32: smem = pipe_df_lean_smem_bytes<32>(t.max_nodes, t.tile_elems, t.packet_bytes); break;
    default: return false;
  }
  return smem <= (size_t)max_smem_optin(m->device);
}

template void ebe_apply<float>(const fe_mesh*, int, const float*, float*, cudaStream_t, const int*);
template void ebe_apply<double>(const fe_mesh*, int, const double*, double*, cudaStream_t, const int*);

// Times each candidate kernel for (R, precision) on this mesh (scratch vectors
// of ones, 2 warm-up and 5 timed products each, CUDA events on `s`) and keeps
// the fastest. Candidates, where the tile's shared-memory footprint fits: direct;
// gather with 12..256 elements per tile; tiled with 24..96; for FP64 the
// float-float gather with 4..24; for FP32 the paired-arithmetic gather with 16..96
// and the warp-specialised kernel with 256 to 512 element-case items per tile;
// and the colour-by-colour kernel.
template <typename T>
static void tune(fe_mesh* m, int R, cudaStream_t s, int* best_variant, float* best_ms) {
  const size_t n = (size_t)m->n_nodes * R * 3;
  DevBuf xb, yb;
  xb.alloc(n * sizeof(T));
  yb.alloc(n * sizeof(T));
  FE_CUDA(cudaMemsetAsync(xb.ptr, 0, n * sizeof(T), s));
  cudaEvent_t e0, e1;
  FE_CUDA(cudaEventCreate(&e0));
  FE_CUDA(cudaEventCreate(&e1));
  std::vector<int> cands = {0};
  for (int te : {12, 16, 24, 32, 48, 64, 96, 128, 192, 256})
    if (gather_supported(R) && tiled_fits(m, te, R, sizeof(T) == 4, FE_EBE_GATHER))
      cands.push_back(FE_EBE_GATHER * 65536 + te);
  for (int te : {24, 48, 96})
    if (tiled_fits(m, te, R, sizeof(T) == 4, FE_EBE_TILED)) cands.push_back(FE_EBE_TILED * 65536 + te);
  if (sizeof(T) == 8 && df_supported(R))
    for (int te : {4, 8, 12, 16, 24})
      if (tiled_fits(m, te, R, 0, FE_EBE_GATHER)) {
        cands.push_back(FE_EBE_GATHER_DF * 65536 + te);
        cands.push_back(FE_EBE_DF_LEAN * 65536 + te);
      }
  if (sizeof(T) == 4 && x2_supported(R))
    for (int te : {16, 24, 32, 48, 64, 96})
      if (tiled_fits(m, te, R, 1, FE_EBE_GATHER)) cands.push_back(FE_EBE_GATHER_X2 * 65536 + te);
  if (sizeof(T) == 4 && ws_supported(R))
    for (int items : {256, 320, 384, 448, 512})   // element-case items per tile: 4 to 8 compute warps
      if (items % R == 0) cands.push_back(FE_EBE_WS * 65536 + items / R);
  if (sizeof(T) == 4 && ws_supported(R))
    for (int items : {64, 128, 192, 256})         // two blocks per SM: 1 to 4 compute warps each
      if (items % R == 0) cands.push_back(FE_EBE_WS2 * 65536 + items / R);
  cands.push_back(FE_EBE_COLOUR * 65536);  // the colour count is filled in once the colouring exists
  *best_variant = 0;
  *best_ms = 1e30f;
  const int old = m->variant[sizeof(T) == 4][R];
  ensure_geometry_buffer(m, sizeof(T) == 4);
  for (int v : cands) {
    if (v / 65536 == FE_EBE_COLOUR) {
      build_colouring(m, s);
      v = FE_EBE_COLOUR * 65536 + m->colouring.n_colours;
    } else if (v > 0) {
      if (v / 65536 != FE_EBE_WS && v / 65536 != FE_EBE_WS2) get_tiling(m, v % 65536, s);
      if (v / 65536 == FE_EBE_WS || v / 65536 == FE_EBE_WS2) {
        if (!ws_fits(m, v % 65536, R, v / 65536 == FE_EBE_WS2 ? 256 : 512)) continue;
      } else if (v / 65536 == FE_EBE_GATHER_DF) {
        if (!df_fits(m, v % 65536, R)) continue;
      } else if (v / 65536 == FE_EBE_DF_LEAN) {
        if (!df_lean_fits(m, v % 65536, R)) continue;
      } else if (v / 65536 == FE_EBE_GATHER_X2) {
        if (!x2_fits(m, v % 65536, R)) continue;
      } else if (!tiled_fits(m, v % 65536, R, sizeof(T) == 4, v / 65536)) {
        continue;
      }
    }
    ebe_set_variant(m, R, sizeof(T) == 4, v);
    for (int i = 0; i < 2; ++i) ebe_apply<T>(m, R, xb.as<T>(), yb.as<T>(), s);
    FE_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < 5; ++i) ebe_apply<T>(m, R, xb.as<T>(), yb.as<T>(), s);
    FE_CUDA(cudaEventRecord(e1, s));
    FE_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 5.f;
    if (ms < *best_ms) {
      *best_ms = ms;
      *best_variant = v;
    }
  }
  m->variant[sizeof(T) == 4][R] = old;
  ebe_set_variant(m, R, sizeof(T) == 4, *best_variant);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace fe

// Picks the fastest EBE kernel for (R, dtype) on this mesh by timing (see tune()).
// Synchronous. *variant = 0 (direct) or the tile size of the tiled kernel;
// *us = its time per product in microseconds.
extern "C" fe_status fe_ebe_tune(fe_mesh* m, int32_t R, fe_dtype dtype, void* stream, int32_t* variant, int32_t* us) {
  try {
    fe::clear_error();
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range", R);
    fe::DeviceGuard dg(m->device);
    int v = 0;
    float ms = 0.f;
    if (dtype == FE_F32)
      fe::tune<float>(m, R, (cudaStream_t)stream, &v, &ms);
    else
      fe::tune<double>(m, R, (cudaStream_t)stream, &v, &ms);
    if (variant) *variant = v;
    if (us) *us = (int32_t)(ms * 1000.f);
    return FE_OK;
  } catch (const fe::Failure& f) {
    return f.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}
