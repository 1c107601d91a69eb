// Warp-specialised EBE product y = K_bc x in FP32 for R in {4, 8, 16, 32} cases
// (Eq. 3, with the multiple vectors of Sec. 3.1).
//
// One CTA per SM (FE_EBE_WS, 512 threads; FE_EBE_WS2: two 256-thread CTAs) walks its
// tiles t = blockIdx.x, + gridDim.x, ... Its warps keep one role for the whole kernel:
//  * compute warps: thread (element le, pair p) computes cases 2p and 2p + 1 of
//    element le in paired FP32 instructions (elem_apply_ws), reading the element's
//    node inputs (component-major rows) and geometry from shared memory and writing
//    its 30 outputs per case to the element's own slot (no atomics inside the tile);
//  * staging warps, in three roles that each run their own loop over the tiles:
//      geometry (warp 0): gradients of the volume coordinates and Lame constants of
//        every element of a tile from the packet's coordinates and materials (the
//        element matrix is recomputed on every product, never stored);
//      loaders (the next two or three warps): each tile node's row of x read from
//        global memory into registers (48 contiguous bytes per thread and load),
//        transposed to component-major order with constrained components zeroed
//        (P x) and stored into the stage;
//      node sums (the other warps): every tile node's slots summed and added into y
//        with one 16-byte atomic add per 4 values (owner tiles write (I - P) x on
//        constrained components). A node with more than kVnMax incidences in the tile
//        is summed in pieces ("virtual nodes") of at most kVnMax incidences, each added
//        into y on its own, so that lanes run short loops of similar length. The
//        summing threads also issue the packet loads: one bulk copy (cp.async.bulk,
//        completing on an mbarrier) per tile of its packet (node ids, coordinates,
//        materials, offsets), npk tiles ahead.
// Two buffer sets ("stages") alternate between consecutive tiles; the roles meet only
// on mbarriers (waiting on one is not an arrival, so warps drift apart and overlap one
// warp's loads with another's arithmetic):
//   READY[s]  every staging thread arrives when stage s holds the inputs and
//             geometry of tile i and the node sums of tile i - 2 (same slots) are
//             done; the compute warps wait for it before tile i;
//   DONE[s]   every compute thread arrives after its products of tile i; the staging
//             warps wait for it before refilling stage s and summing tile i;
//   PKF[k]    packet slot k holds its tile's packet (transaction bytes).
// Before waiting for DONE, each staging role does the part of its work that needs
// only packets: the loaders issue the global loads of tile i + 2's rows, the summing
// threads read their first task's slot offsets, node id and mask, so that after DONE
// only shared-memory stores, slot reads and atomics remain on the path to READY.
// Each mbarrier wait is bounded (about one second of SM clock): a wait that gives
// up records it in the mesh's device status word (fe_mesh_device_status), after
// which the thread waits no more; before it exits, a thread that gave up waits (again
// bounded) for the packet copies it may have left in flight. y must be zero before
// the launch (the caller's zero pass).
//
// Tiles come from a greedy partition (get_ws_tiling): starting from the first
// unassigned element in the mesh's locality order, a tile repeatedly takes the
// unassigned element that shares the most nodes with it (ties: nearest to the
// tile's centroid), up to te elements and a node budget. Compact tiles have fewer
// nodes per element, hence fewer node sums, input rows and global atomics per
// element-case product.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kWsThreads = 512;   // 16 warps, one CTA per SM (128 registers per thread); FE_EBE_WS2:
                                  // half that, two CTAs per SM
constexpr int kGeoWs = 40;        // floats of element data per element in shared memory
constexpr int kPkMin = 4;         // packet slots in shared memory: at least (tiles i .. i + 3 are read)
constexpr int kPkMax = 6;         // and at most
constexpr int kBarSum = 1;        // named barrier of the node-sum warps (0 is __syncthreads)
constexpr int kVnMax = 4;         // incidences per virtual node (node-sum task)
// mbarriers at the start of shared memory (byte offsets)
constexpr int kReady = 0;         // READY[2]
constexpr int kDone = 16;         // DONE[2]
constexpr int kPkf = 32;          // PKF[kPkMax]
constexpr int kMbarBytes = 128;

template <int R>
struct WsCfg {
  static constexpr int RC = R / 2;                  // compute threads per element
  static constexpr int XR = 3 * R;                  // floats per node row
  static constexpr int S = 30 * R + (3 * R) % 32;   // slot stride per element: S = R (mod 32)
  static constexpr int G4 = R / 4;                  // node-sum lanes per node row (4 cases each)
  static_assert(R % 4 == 0 && S % 4 == 0, "rows must stay 16-byte aligned");
};

__host__ __device__ constexpr int ws_slot_stride(int R) { return 30 * R + (3 * R) % 32; }
__host__ __device__ constexpr int a16i(int b) { return (b + 15) & ~15; }

// Node budget of a tile of te elements (the greedy tiler stops a tile that would
// exceed it): bounds the shared memory of the row buffers.
int ws_node_cap(int te) { return std::max(24, (11 * te) / 4 + 24); }

}  // namespace

// Byte layout of one packet (host and device agree on it); sections 16-byte aligned:
//   int32 {nn, ne, nv, 0} | float4 crd[nnmax] (node coordinates, FP32) | float4
//   mat[te] (E, nu, 0, 0 per element) | int32 ids[nnmax] (global node ids) | int32
//   elem[te] (internal element ids) | uint8 mask[nnmax] (free-DOF bits) | uint8
//   own[nnmax] (1 in the node's first tile) | uint32 vn[nvmax] (virtual nodes: local
//   node in bits 0-11, first piece of its node in bit 12, incidence count in bits
//   13-16, first incidence in bits 17-31; longest first) | uint16 inc_off[10 te] (slot
//   offset le S + a 3R of each element-node incidence, grouped by node) | uint16
//   eoff[te][16] (0..9: row offset ln 3R of the element's nodes, 10..13: local ids of
//   its corners, 14..15: 0)
struct WsLayout {
  int crd, mat, ids, elem, mask, own, vn, inc_off, eoff, bytes;
  __host__ __device__ WsLayout(int nnmax, int nvmax, int te) {
    crd = 16;
    mat = crd + 16 * nnmax;
    ids = mat + 16 * te;
    elem = ids + a16i(4 * nnmax);
    mask = elem + a16i(4 * te);
    own = mask + a16i(nnmax);
    vn = own + a16i(nnmax);
    inc_off = vn + a16i(4 * nvmax);
    eoff = inc_off + a16i(20 * te);
    bytes = eoff + 32 * te;
  }
};

// Shared-memory carve-up (bytes): mbarriers | packets [npk][pk] | xs [2][nnmax][3R]
// (component-major node rows) | geo [2][te][40] | ob [2][te][S] (slots). Every
// section is 16-byte aligned.
struct WsSmem {
  int pk = 0, xs = 0, geo = 0, ob = 0, bytes = 0;
  WsSmem() = default;
  __host__ __device__ WsSmem(int te, int R, int nnmax, int pkb, int npk) {
    pk = kMbarBytes;
    xs = pk + npk * pkb;
    geo = xs + 2 * nnmax * 12 * R;
    ob = geo + 2 * te * kGeoWs * 4;
    bytes = ob + 2 * te * ws_slot_stride(R) * 4;
  }
};

struct WsArgs {
  int64_t n_tiles;
  int te, nnmax, nvmax, pk, npk, cw, nlw;   // elements per tile, max nodes and virtual nodes, packet
                                            // bytes, packet slots, compute warps, loader warps
  const unsigned char* packets;
  const float* x;                  // [N][R][3]
  float* y;                        // [N][R][3], zero on entry
  const int* skip;
  int* status;                     // set to 1 when a bounded wait gives up
  long long timeout;               // SM clock cycles an mbarrier wait may take
  WsSmem sm;
};

namespace {

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// arrival that also expects `bytes` of bulk-copy transactions in the current phase
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `bar` with parity `parity`, at most `timeout` cycles. A wait
// that gives up records it in *status and clears ok, after which this thread waits
// no more (the kernel then finishes; its results are flagged invalid).
__device__ __forceinline__ void mbar_wait(int* status, long long timeout, uint32_t bar, uint32_t parity, bool& ok) {
  if (!ok || mbar_try(bar, parity)) return;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > timeout) {
      ok = false;
      atomicExch(status, 1);
      return;
    }
  }
}
// bounded wait used only after a wait gave up: drains a bulk copy that may be in flight
__device__ __forceinline__ void mbar_drain(long long timeout, uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity) && clock64() - t0 <= timeout) {
  }
}
// global -> this CTA's shared memory, completion counted on `bar` (addresses 16-byte
// aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// orders this thread's earlier shared-memory accesses before later bulk copies into them
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ float2 b2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// w = A g, A symmetric 3x3 stored (xx, yy, zz, yz, xz, xy), continuing the chains of w0
__device__ __forceinline__ void symmv_acc(const float2 A[6], float g0, float g1, float g2, float2 w[3]) {
  w[0] = f2fma(A[4], b2(g2), f2fma(A[5], b2(g1), f2fma(A[0], b2(g0), w[0])));
  w[1] = f2fma(A[3], b2(g2), f2fma(A[1], b2(g1), f2fma(A[5], b2(g0), w[1])));
  w[2] = f2fma(A[2], b2(g2), f2fma(A[3], b2(g1), f2fma(A[4], b2(g0), w[2])));
}
__device__ __forceinline__ void symmv(const float2 A[6], float g0, float g1, float g2, float2 w[3]) {
  w[0] = f2fma(A[4], b2(g2), f2fma(A[5], b2(g1), f2mul(A[0], b2(g0))));
  w[1] = f2fma(A[3], b2(g2), f2fma(A[1], b2(g1), f2mul(A[5], b2(g0))));
  w[2] = f2fma(A[2], b2(g2), f2fma(A[3], b2(g1), f2mul(A[4], b2(g0))));
}

// Element product for two cases (lanes x and y of every float2) from the element
// data gv[40]: g (gradients of the volume coordinates, [k][i]), -g, 4g,
// lam' = lam V/5, 2 mu', mu' = mu V/5. With v_mm = 3 u_m, v_mj = 4 u_mj - u_j,
//   H_m = sum_j v_mj (x) g_j = 4 (u_m (x) g_m + sum_{j != m} u_mj (x) g_j) - sum_j u_j (x) g_j,
//   s_m = lam' tr(H_m) I + mu' (H_m + H_m^T),  S = sum_m s_m,
//   corner k:     y_k  = (s_k - S/4) g_k,
//   edge node kl: y_kl = (S + s_k) g_l + (S + s_l) g_k,
// the exact-integration product K_e u_e of the straight-sided 10-node tetrahedron
// (the factor V/5 of the integrals folded into lam' and mu').
__device__ __forceinline__ void elem_apply_ws(const float gv[kGeoWs], const float2 u[10][3], float2 y[10][3]) {
  // Hn = -sum_j u_j (x) g_j over the corners
  float2 Hn[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 h = f2mul(u[0][a], b2(gv[12 + b]));
      h = f2fma(u[1][a], b2(gv[15 + b]), h);
      h = f2fma(u[2][a], b2(gv[18 + b]), h);
      Hn[a][b] = f2fma(u[3][a], b2(gv[21 + b]), h);
    }
  float2 s[4][6];
  const float lam = gv[36], mu2 = gv[37], mu = gv[38];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float2 H[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) H[a][b] = f2fma(u[m][a], b2(gv[24 + 3 * m + b]), Hn[a][b]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j == m) continue;
      // edge node between corners m and j (VTK order), constant after unrolling
      const int e = (m == 0) ? (j == 1 ? 4 : j == 2 ? 6 : 7)
                  : (m == 1) ? (j == 0 ? 4 : j == 2 ? 5 : 8)
                  : (m == 2) ? (j == 0 ? 6 : j == 1 ? 5 : 9)
                             : (j == 0 ? 7 : j == 1 ? 8 : 9);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) H[a][b] = f2fma(u[e][a], b2(gv[24 + 3 * j + b]), H[a][b]);
    }
    const float2 lt = f2mul(b2(lam), f2add(f2add(H[0][0], H[1][1]), H[2][2]));
    s[m][0] = f2fma(b2(mu2), H[0][0], lt);
    s[m][1] = f2fma(b2(mu2), H[1][1], lt);
    s[m][2] = f2fma(b2(mu2), H[2][2], lt);
    s[m][3] = f2mul(b2(mu), f2add(H[1][2], H[2][1]));
    s[m][4] = f2mul(b2(mu), f2add(H[0][2], H[2][0]));
    s[m][5] = f2mul(b2(mu), f2add(H[0][1], H[1][0]));
  }
  float2 S[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = f2add(f2add(s[0][q], s[1][q]), f2add(s[2][q], s[3][q]));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) A[q] = f2fma(b2(-0.25f), S[q], s[k][q]);
    symmv(A, gv[3 * k], gv[3 * k + 1], gv[3 * k + 2], y[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) s[k][q] = f2add(s[k][q], S[q]);
  // edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3) -> nodes 4..9
  constexpr int EK[6] = {0, 1, 0, 0, 1, 2};
  constexpr int EL[6] = {1, 2, 2, 3, 3, 3};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int k = EK[q], l = EL[q];
    symmv(s[k], gv[3 * l], gv[3 * l + 1], gv[3 * l + 2], y[4 + q]);
    symmv_acc(s[l], gv[3 * k], gv[3 * k + 1], gv[3 * k + 2], y[4 + q]);
  }
}

// ---------------------------------------------------------------------------
// compute warps
// ---------------------------------------------------------------------------
__device__ __forceinline__ const unsigned char* pk_at(const WsArgs& A, const unsigned char* sm, int i) {
  return sm + A.sm.pk + (i % A.npk) * A.pk;
}

template <int R>
__device__ __forceinline__ void ws_compute(const WsArgs& A, unsigned char* sm, const WsLayout& L, int n_it,
                                           bool& ok) {
  using C = WsCfg<R>;
  const uint32_t mb = smem_u32(sm);
  const int le = threadIdx.x / C::RC, p = threadIdx.x - le * C::RC;
  const float* xs = reinterpret_cast<const float*>(sm + A.sm.xs);
  const float* geo = reinterpret_cast<const float*>(sm + A.sm.geo);
  float* ob = reinterpret_cast<float*>(sm + A.sm.ob);
  for (int i = 0; i < n_it; ++i) {
    const int st = i & 1;
    mbar_wait(A.status, A.timeout, mb + kReady + 8 * st, (uint32_t)((i >> 1) & 1), ok);
    const unsigned char* pk = pk_at(A, sm, i);
    const int ne = reinterpret_cast<const int*>(pk)[1];
    bool work = le < ne;
    if (work) {
      const uint16_t* eo = reinterpret_cast<const uint16_t*>(pk + L.eoff) + le * 16;
      const uint4 w0 = *reinterpret_cast<const uint4*>(eo);
      const unsigned w1 = *reinterpret_cast<const unsigned*>(eo + 8);
      const int off[10] = {(int)(w0.x & 0xffff), (int)(w0.x >> 16), (int)(w0.y & 0xffff), (int)(w0.y >> 16),
                           (int)(w0.z & 0xffff), (int)(w0.z >> 16), (int)(w0.w & 0xffff), (int)(w0.w >> 16),
                           (int)(w1 & 0xffff),   (int)(w1 >> 16)};
      const float* xb = xs + (size_t)st * A.nnmax * C::XR + 2 * p;
      float2 u[10][3];
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) u[a][k] = *reinterpret_cast<const float2*>(xb + off[a] + k * R);
      float gv[kGeoWs];
      const float4* gq = reinterpret_cast<const float4*>(geo + ((size_t)st * A.te + le) * kGeoWs);
#pragma unroll
      for (int q = 0; q < kGeoWs / 4; ++q) {
        const float4 w = gq[q];
        gv[4 * q] = w.x;
        gv[4 * q + 1] = w.y;
        gv[4 * q + 2] = w.z;
        gv[4 * q + 3] = w.w;
      }
      float2 yv[10][3];
      elem_apply_ws(gv, u, yv);
      float* o = ob + ((size_t)st * A.te + le) * C::S + 2 * p;
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) *reinterpret_cast<float2*>(o + a * C::XR + k * R) = yv[a][k];
    }
    mbar_arrive(mb + kDone + 8 * st);
  }
}

// ---------------------------------------------------------------------------
// staging warps
// ---------------------------------------------------------------------------
// node row of one 4-case group, [case][comp] -> component-major [comp][case], P x
template <int R>
__device__ __forceinline__ void put_row(float* xs_st, int ln, int g, int mk, const float4 v[3]) {
  float4 w[3];
  w[0] = make_float4(v[0].x, v[0].w, v[1].z, v[2].y);
  w[1] = make_float4(v[0].y, v[1].x, v[1].w, v[2].z);
  w[2] = make_float4(v[0].z, v[1].y, v[2].x, v[2].w);
  if (mk != 7) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (!((mk >> k) & 1)) w[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float* d = xs_st + ln * WsCfg<R>::XR + 4 * g;
#pragma unroll
  for (int k = 0; k < 3; ++k) *reinterpret_cast<float4*>(d + k * R) = w[k];
}

// Node rows of a tile from x into a stage, split in two so that the global loads can
// be in flight while the stage is still in use: rows_fetch loads the tasks k0, k0 + nl,
// ... (kLdBatch of them) of loader thread k0 into registers, rows_put transposes and
// stores them. Task (local node, group of 4 cases) = 48 contiguous bytes of x;
// consecutive lanes take consecutive groups.
constexpr int kLdBatch = 5;
template <int R>
__device__ __forceinline__ void rows_fetch(const WsArgs& A, const unsigned char* pk, const WsLayout& L, int k0, int nl,
                                           float4 (&v)[kLdBatch][3]) {
  using C = WsCfg<R>;
  const int ntask = reinterpret_cast<const int*>(pk)[0] * C::G4;
  const int* ids = reinterpret_cast<const int*>(pk + L.ids);
#pragma unroll
  for (int b = 0; b < kLdBatch; ++b) {
    const int k = k0 + b * nl;
    if (k < ntask) {
      const int ln = k / C::G4, g = k - ln * C::G4;
      const float4* src = reinterpret_cast<const float4*>(A.x + (int64_t)ids[ln] * C::XR) + 3 * g;
#pragma unroll
      for (int q = 0; q < 3; ++q) v[b][q] = __ldcg(src + q);
    }
  }
}
template <int R>
__device__ __forceinline__ void rows_put(const WsArgs& A, unsigned char* sm, const unsigned char* pk, const WsLayout& L,
                                         int st, int k0, int nl, const float4 (&v)[kLdBatch][3]) {
  using C = WsCfg<R>;
  const int ntask = reinterpret_cast<const int*>(pk)[0] * C::G4;
  const unsigned char* mks = pk + L.mask;
  float* xs_st = reinterpret_cast<float*>(sm + A.sm.xs) + (size_t)st * A.nnmax * C::XR;
#pragma unroll
  for (int b = 0; b < kLdBatch; ++b) {
    const int k = k0 + b * nl;
    if (k < ntask) {
      const int ln = k / C::G4, g = k - ln * C::G4;
      put_row<R>(xs_st, ln, g, mks[ln], v[b]);
    }
  }
}

// Element data of element le of a tile (its packet's coordinates and materials):
// gradients g of the volume coordinates, -g, 4g, lam V/5, 2 mu V/5, mu V/5, 0.
__device__ __forceinline__ void geo_compute(const unsigned char* pk, const WsLayout& L, int le, float (&v)[kGeoWs]) {
  const float4* crd = reinterpret_cast<const float4*>(pk + L.crd);
  const float4* mat = reinterpret_cast<const float4*>(pk + L.mat);
  const uint16_t* eo = reinterpret_cast<const uint16_t*>(pk + L.eoff) + le * 16;
  const unsigned c01 = *reinterpret_cast<const unsigned*>(eo + 10);   // local ids of corners 0, 1
  const unsigned c23 = *reinterpret_cast<const unsigned*>(eo + 12);   // corners 2, 3
  const float4 x0 = crd[c01 & 0xffff], x1 = crd[c01 >> 16], x2 = crd[c23 & 0xffff], x3 = crd[c23 >> 16];
  const float d1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
  const float d2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
  const float d3[3] = {x3.x - x0.x, x3.y - x0.y, x3.z - x0.z};
  const float e23[3] = {d2[1] * d3[2] - d2[2] * d3[1], d2[2] * d3[0] - d2[0] * d3[2], d2[0] * d3[1] - d2[1] * d3[0]};
  const float e31[3] = {d3[1] * d1[2] - d3[2] * d1[1], d3[2] * d1[0] - d3[0] * d1[2], d3[0] * d1[1] - d3[1] * d1[0]};
  const float e12[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
  const float det = d1[0] * e23[0] + d1[1] * e23[1] + d1[2] * e23[2];
  const float inv = 1.f / det;
  float g[4][3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    g[1][q] = e23[q] * inv;
    g[2][q] = e31[q] * inv;
    g[3][q] = e12[q] * inv;
    g[0][q] = -(g[1][q] + g[2][q] + g[3][q]);
  }
  const float4 em = mat[le];
  const float onu = 1.f + em.y;
  const float mu = em.x / (2.f * onu);
  const float lam = (em.x * em.y) / (onu * (1.f - 2.f * em.y));
  const float f = det * (1.f / 30.f);   // 4 V / 20 with V = det / 6
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      v[3 * k + q] = g[k][q];
      v[12 + 3 * k + q] = -g[k][q];
      v[24 + 3 * k + q] = 4.f * g[k][q];
    }
  v[36] = lam * f;
  v[37] = 2.f * mu * f;
  v[38] = mu * f;
  v[39] = 0.f;
}
__device__ __forceinline__ void geo_store(const WsArgs& A, unsigned char* sm, int st, int le, const float (&v)[kGeoWs]) {
  float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(sm + A.sm.geo) + ((size_t)st * A.te + le) * kGeoWs);
#pragma unroll
  for (int q = 0; q < kGeoWs / 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void add4(float4& a, const float4 b) {
  const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
  a = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// One node-sum task (virtual node v, group g of 4 cases): what it needs from the
// packet, read before the tile's slots are ready.
struct SumTask {
  int n;          // incidences (0: no task)
  int g, mk;
  bool ow;        // constrained components are written by this task ((I - P) x)
  int64_t gi;     // offset of the group's 12 values in x and y
  int o[kVnMax];  // slot offsets of the incidences
};

template <int R>
__device__ __forceinline__ void sum_fetch(const unsigned char* pk, const WsLayout& L, int k, SumTask& t) {
  using C = WsCfg<R>;
  const int nv = reinterpret_cast<const int*>(pk)[2];
  t.n = 0;
  if (k >= nv * C::G4) return;
  const int v = k / C::G4;
  t.g = k - v * C::G4;
  const unsigned w = reinterpret_cast<const unsigned*>(pk + L.vn)[v];
  const int ln = (int)(w & 0xfff);
  const int j = (int)(w >> 17);
  t.n = (int)((w >> 13) & 0xf);
  t.mk = pk[L.mask + ln];
  t.ow = ((w >> 12) & 1) && pk[L.own + ln] != 0;
  t.gi = (int64_t)reinterpret_cast<const int*>(pk + L.ids)[ln] * C::XR + 12 * t.g;
  const uint16_t* io = reinterpret_cast<const uint16_t*>(pk + L.inc_off);
#pragma unroll
  for (int u = 0; u < kVnMax; ++u) t.o[u] = u < t.n ? io[j + u] : 0;
}

// the task's sums over its incidences' slots (stage st) added into y, four incidences
// with their loads in flight at a time
template <int R>
__device__ __forceinline__ void sum_run(const WsArgs& A, const unsigned char* sm, int st, const SumTask& t) {
  using C = WsCfg<R>;
  if (t.n == 0) return;
  const float* b = reinterpret_cast<const float*>(sm + A.sm.ob) + (size_t)st * A.te * C::S + 4 * t.g;
  float4 a[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int nn_ = t.n;
#pragma unroll
  for (int h = 0; h < kVnMax; h += 4) {
    if (h < nn_) {
      float4 x4[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (h + u < nn_)
#pragma unroll
          for (int q = 0; q < 3; ++q) x4[u][q] = *reinterpret_cast<const float4*>(b + t.o[h + u] + q * R);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (h + u < nn_)
#pragma unroll
          for (int q = 0; q < 3; ++q) add4(a[q], x4[u][q]);
    }
  }
  // component-major sums -> the node's [case][comp] values of the group
  const float f[12] = {a[0].x, a[1].x, a[2].x, a[0].y, a[1].y, a[2].y, a[0].z, a[1].z, a[2].z, a[0].w, a[1].w, a[2].w};
  float* yg = A.y + t.gi;
  if (t.mk == 7) {
    atomicAdd(reinterpret_cast<float4*>(yg), make_float4(f[0], f[1], f[2], f[3]));
    atomicAdd(reinterpret_cast<float4*>(yg) + 1, make_float4(f[4], f[5], f[6], f[7]));
    atomicAdd(reinterpret_cast<float4*>(yg) + 2, make_float4(f[8], f[9], f[10], f[11]));
  } else {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if ((t.mk >> (q % 3)) & 1)
        atomicAdd(yg + q, f[q]);
      else if (t.ow)
        yg[q] = __ldg(A.x + t.gi + q);   // constrained DOF: (I - P) x, written once by the node's first tile
    }
  }
}

// Staging roles. Each runs its own loop over the CTA's tiles i = 0 .. n - 1; before
// waiting for tile i's products (DONE), it does the work that needs only packets.
struct Stg {
  uint32_t mb;
  int64_t t0, G;
  int n;
  __device__ uint32_t pkf(const WsArgs& A, int i) const { return mb + kPkf + 8 * (i % A.npk); }
  __device__ uint32_t pkpar(const WsArgs& A, int i) const { return (uint32_t)((i / A.npk) & 1); }
  __device__ uint32_t done(int i) const { return mb + kDone + 8 * (i & 1); }
  __device__ uint32_t ready(int i) const { return mb + kReady + 8 * (i & 1); }
};

// one thread: the packet of tile i into its slot, completion counted on PKF
__device__ __forceinline__ void issue_packet(const WsArgs& A, unsigned char* sm, const Stg& c, int i) {
  unsigned char* dst = sm + A.sm.pk + (i % A.npk) * A.pk;
  fence_proxy_async();
  mbar_arrive_tx(c.pkf(A, i), (uint32_t)A.pk);
  bulk_g2s(dst, A.packets + (c.t0 + (int64_t)i * c.G) * A.pk, (uint32_t)A.pk, c.pkf(A, i));
}

// loaders: node rows of tile i + 2 into stage i & 1 (tiles 0 and 1 before the loop)
template <int R>
__device__ __forceinline__ void role_load(const WsArgs& A, unsigned char* sm, const WsLayout& L, const Stg& c, int lt,
                                          int NL, bool& ok) {
  using C = WsCfg<R>;
  for (int j = -2; j < c.n - 2; ++j) {
    const int t = j + 2;   // tile whose rows this iteration stages
    float4 rv[kLdBatch][3];
    mbar_wait(A.status, A.timeout, c.pkf(A, t), c.pkpar(A, t), ok);
    const unsigned char* pk = pk_at(A, sm, t);
    rows_fetch<R>(A, pk, L, lt, NL, rv);
    if (j >= 0) mbar_wait(A.status, A.timeout, c.done(j), (uint32_t)((j >> 1) & 1), ok);   // stage free
    rows_put<R>(A, sm, pk, L, t & 1, lt, NL, rv);
    const int ntask = reinterpret_cast<const int*>(pk)[0] * C::G4;
    for (int k0 = lt + kLdBatch * NL; k0 < ntask; k0 += kLdBatch * NL) {
      rows_fetch<R>(A, pk, L, k0, NL, rv);
      rows_put<R>(A, sm, pk, L, t & 1, k0, NL, rv);
    }
    mbar_arrive(c.ready(t));
  }
  for (int i = c.n - 2; i < c.n; ++i)   // the last two tiles: nothing to stage, DONE still waited
    if (i >= 0) mbar_wait(A.status, A.timeout, c.done(i), (uint32_t)((i >> 1) & 1), ok);
}

// geometry warp: element data of tile i + 2 into stage i & 1
__device__ __forceinline__ void role_geo(const WsArgs& A, unsigned char* sm, const WsLayout& L, const Stg& c, int lane,
                                         bool& ok) {
  for (int j = -2; j < c.n - 2; ++j) {
    const int t = j + 2;
    float gv[kGeoWs];
    mbar_wait(A.status, A.timeout, c.pkf(A, t), c.pkpar(A, t), ok);
    const unsigned char* pk = pk_at(A, sm, t);
    const int ne = reinterpret_cast<const int*>(pk)[1];
    if (lane < ne) geo_compute(pk, L, lane, gv);
    if (j >= 0) mbar_wait(A.status, A.timeout, c.done(j), (uint32_t)((j >> 1) & 1), ok);
    if (lane < ne) geo_store(A, sm, t & 1, lane, gv);
    for (int le = lane + 32; le < ne; le += 32) {
      geo_compute(pk, L, le, gv);
      geo_store(A, sm, t & 1, le, gv);
    }
    mbar_arrive(c.ready(t));
  }
  for (int i = c.n - 2; i < c.n; ++i)
    if (i >= 0) mbar_wait(A.status, A.timeout, c.done(i), (uint32_t)((i >> 1) & 1), ok);
}

// summing threads: node sums of tile i (stage i & 1) into y, then the packet of tile
// i + npk into tile i's packet slot
template <int R>
__device__ __forceinline__ void role_sum(const WsArgs& A, unsigned char* sm, const WsLayout& L, const Stg& c, int sumt,
                                         int NS, int& last_pk, bool& ok) {
  using C = WsCfg<R>;
  for (int j = 0; j < 2 && j < c.n; ++j) mbar_arrive(c.ready(j));   // stages 0 and 1 hold no earlier sums
  for (int i = 0; i < c.n; ++i) {
    SumTask tk;
    mbar_wait(A.status, A.timeout, c.pkf(A, i), c.pkpar(A, i), ok);   // tile i's packet landed
    const unsigned char* pk = pk_at(A, sm, i);
    sum_fetch<R>(pk, L, sumt, tk);
    mbar_wait(A.status, A.timeout, c.done(i), (uint32_t)((i >> 1) & 1), ok);   // tile i computed
    sum_run<R>(A, sm, i & 1, tk);
    const int ntask = reinterpret_cast<const int*>(pk)[2] * C::G4;
    for (int k = sumt + NS; k < ntask; k += NS) {
      sum_fetch<R>(pk, L, k, tk);
      sum_run<R>(A, sm, i & 1, tk);
    }
    if (i + 2 < c.n) mbar_arrive(c.ready(i + 2));
    if (i + A.npk < c.n) {
      bar_sync(kBarSum, NS);              // every summing thread is done with tile i's packet
      if (sumt == 0) {
        issue_packet(A, sm, c, i + A.npk);
        last_pk = i + A.npk;
      }
    }
  }
}

template <int R, int NT>
__device__ __forceinline__ void ws_staging(const WsArgs& A, unsigned char* sm, const WsLayout& L, int n, int64_t t0,
                                           int64_t G, bool& ok) {
  const int mt = threadIdx.x - A.cw * 32;   // staging thread 0 .. NM - 1
  const int NM = NT - A.cw * 32;
  const int wid = mt >> 5;
  const Stg c{smem_u32(sm), t0, G, n};
  int last_pk = -1;   // the latest packet this thread issued
  if (mt == 0)        // packets of the first npk tiles
    for (int k = 0; k < A.npk && k < n; ++k) {
      issue_packet(A, sm, c, k);
      last_pk = k;
    }
  if (wid == 0)
    role_geo(A, sm, L, c, mt, ok);
  else if (wid <= A.nlw)
    role_load<R>(A, sm, L, c, mt - 32, 32 * A.nlw, ok);
  else
    role_sum<R>(A, sm, L, c, mt - 32 * (1 + A.nlw), NM - 32 * (1 + A.nlw), last_pk, ok);
  if (!ok)   // a wait gave up: let the packet copies this thread issued land before the CTA exits
    for (int k = std::max(0, last_pk - A.npk + 1); k <= last_pk; ++k)
      mbar_drain(A.timeout, c.pkf(A, k), c.pkpar(A, k));
}

template <int R, int NT>
__global__ void __launch_bounds__(NT, kWsThreads / NT) ebe_ws_kernel(const WsArgs A) {
  extern __shared__ __align__(128) unsigned char sm[];
  if (A.skip && *A.skip) return;
  const int64_t G = gridDim.x, t0 = blockIdx.x;
  if (t0 >= A.n_tiles) return;
  const int n_it = (int)((A.n_tiles - t0 + G - 1) / G);
  const WsLayout L(A.nnmax, A.nvmax, A.te);
  if (threadIdx.x == 0) {
    const uint32_t mb = smem_u32(sm);
    mbar_init(mb + kReady, NT - 32 * A.cw);        // READY[0], READY[1]: every staging thread
    mbar_init(mb + kReady + 8, NT - 32 * A.cw);
    mbar_init(mb + kDone, 32 * A.cw);              // DONE[0], DONE[1]: every compute thread
    mbar_init(mb + kDone + 8, 32 * A.cw);
    for (int k = 0; k < A.npk; ++k)                // PKF[k]: one arrival with the expected bytes
      mbar_init(mb + kPkf + 8 * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  if ((int)(threadIdx.x >> 5) < A.cw)
    ws_compute<R>(A, sm, L, n_it, ok);
  else
    ws_staging<R, NT>(A, sm, L, n_it, t0, G, ok);
}

// Materials of every element slot of every packet from matv (after a material
// change, and once when the packets are built).
__global__ void ws_refresh_mat_kernel(unsigned char* packets, int64_t n_tiles, int pk, int te, int mat_off,
                                      int elem_off, const float4* matv) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_tiles * te) return;
  const int64_t t = k / te;
  const int le = (int)(k - t * te);
  unsigned char* p = packets + t * (int64_t)pk;
  const int ne = reinterpret_cast<const int*>(p)[1];
  float4* mat = reinterpret_cast<float4*>(p + mat_off);
  const int* el = reinterpret_cast<const int*>(p + elem_off);
  mat[le] = le < ne ? matv[el[le]] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// host: greedy tiles and packets
// ---------------------------------------------------------------------------
// Partition of the elements into tiles of at most te elements and nncap nodes (see the
// file header).
void greedy_tiles(const fe_mesh* m, int te, int nncap, std::vector<int32_t>& elems, std::vector<int64_t>& tptr) {
  const int64_t E = m->n_elem, N = m->n_nodes;
  const int32_t* cn = m->conn_host.data();
  std::vector<int64_t> np((size_t)N + 1, 0);
  for (int64_t i = 0; i < 10 * E; ++i) np[(size_t)cn[i] + 1]++;
  for (int64_t n = 0; n < N; ++n) np[(size_t)n + 1] += np[(size_t)n];
  std::vector<int32_t> n2e((size_t)(10 * E));
  {
    std::vector<int64_t> pos(np.begin(), np.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 10; ++a) n2e[(size_t)pos[(size_t)cn[10 * e + a]]++] = (int32_t)e;
  }
  std::vector<float> cen((size_t)(3 * E));
  for (int64_t e = 0; e < E; ++e)
    for (int i = 0; i < 3; ++i) {
      double c = 0.0;
      for (int a = 0; a < 4; ++a) c += m->xyz_host[(size_t)(3 * (int64_t)cn[10 * e + a] + i)];
      cen[(size_t)(3 * e + i)] = (float)(0.25 * c);
    }
  std::vector<uint8_t> assigned((size_t)E, 0), score((size_t)E, 0), mark((size_t)N, 0);
  std::vector<int32_t> marked, touched;
  std::vector<int32_t> bucket[11];
  elems.clear();
  elems.reserve((size_t)E);
  tptr.assign(1, 0);
  int64_t nxt = 0;
  for (int64_t seed = 0; seed < E; ++seed) {
    if (assigned[(size_t)seed]) continue;
    double cs[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
    auto add = [&](int32_t e) {
      assigned[(size_t)e] = 1;
      elems.push_back(e);
      for (int i = 0; i < 3; ++i) cs[i] += cen[(size_t)(3 * (int64_t)e + i)];
      ++cnt;
      for (int a = 0; a < 10; ++a) {
        const int32_t n = cn[10 * (int64_t)e + a];
        if (mark[(size_t)n]) continue;
        mark[(size_t)n] = 1;
        marked.push_back(n);
        for (int64_t k = np[(size_t)n]; k < np[(size_t)n + 1]; ++k) {
          const int32_t e2 = n2e[(size_t)k];
          if (assigned[(size_t)e2]) continue;
          if (score[(size_t)e2] == 0) touched.push_back(e2);
          const int sc = ++score[(size_t)e2];
          bucket[sc].push_back(e2);
        }
      }
    };
    add((int32_t)seed);
    while (cnt < te) {
      int32_t best = -1;
      for (int sc = 10; sc >= 1 && best < 0; --sc) {
        std::vector<int32_t>& B = bucket[sc];
        const double cx = cs[0] / cnt, cy = cs[1] / cnt, cz = cs[2] / cnt;
        double bd = INFINITY;
        size_t w = 0;
        for (size_t q = 0; q < B.size(); ++q) {
          const int32_t e2 = B[q];
          if (assigned[(size_t)e2] || score[(size_t)e2] != sc) continue;
          B[w++] = e2;
          const double dx = cen[(size_t)(3 * (int64_t)e2)] - cx, dy = cen[(size_t)(3 * (int64_t)e2 + 1)] - cy,
                       dz = cen[(size_t)(3 * (int64_t)e2 + 2)] - cz;
          const double d = dx * dx + dy * dy + dz * dz;
          if (d < bd) {
            bd = d;
            best = e2;
          }
        }
        B.resize(w);
      }
      if (best < 0) {
        while (nxt < E && assigned[(size_t)nxt]) ++nxt;
        if (nxt >= E) break;
        best = (int32_t)nxt;
      }
      if ((int)marked.size() + 10 - (int)score[(size_t)best] > nncap) break;   // node budget of a tile
      add(best);
    }
    tptr.push_back((int64_t)elems.size());
    for (int32_t n : marked) mark[(size_t)n] = 0;
    marked.clear();
    for (int32_t e2 : touched) score[(size_t)e2] = 0;
    touched.clear();
    for (auto& B : bucket) B.clear();
  }
}

}  // namespace

namespace {
// One warp initialises an mbarrier that expects one arrival, which never comes, and
// waits on it with the kernel's bounded wait (mbar_wait), limited to `cycles`: the
// wait gives up, records it in *status and the kernel returns.
__global__ void mbar_wait_selftest_kernel(int* status, long long cycles) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  __syncthreads();
  bool ok = true;
  mbar_wait(status, cycles, b, 0, ok);
}
}  // namespace

void ws_wait_selftest(const fe_mesh* m, long long cycles, cudaStream_t s) {
  mbar_wait_selftest_kernel<<<1, 32, 0, s>>>(m->dev_status.as<int>(), cycles);
  FE_CHECK_LAUNCH();
}

bool ws_supported(int R) { return R == 4 || R == 8 || R == 16 || R == 32; }

// Loader warps of a block with sw staging warps (one geometry warp, the rest sum nodes).
static int ws_loader_warps(int sw) { return sw >= 8 ? 3 : 2; }

static int ws_compute_warps(int te, int R) {
  const int t = te * (R / 2);
  return (t % 32 == 0) ? t / 32 : -1;
}

static void refresh_tiling_materials(const fe_mesh* m, const WsTiling& t, cudaStream_t s) {
  const WsLayout L(t.nnmax, t.nvmax, t.te);
  const int64_t n = t.n_tiles * t.te;
  if (n == 0) return;
  ws_refresh_mat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t.packets.as<unsigned char>(), t.n_tiles,
                                                                    t.pk_bytes, t.te, L.mat, L.elem,
                                                                    m->matv.as<float4>());
  FE_CHECK_LAUNCH();
}

void ws_refresh_materials(fe_mesh* m, cudaStream_t s) {
  for (auto& kv : m->ws_tilings) refresh_tiling_materials(m, *kv.second, s);
}

const WsTiling* get_ws_tiling(fe_mesh* m, int te, int R, cudaStream_t s) {
  FE_REQUIRE(ws_supported(R), "the warp-specialised kernel is built for R in {4, 8, 16, 32}, not %d", R);
  const int cw = ws_compute_warps(te, R);
  FE_REQUIRE(cw >= 1 && cw <= 12, "tile of %d elements at R = %d: te * R / 2 must be a multiple of 32 with "
             "at most 12 compute warps", te, R);
  const int key = te * 256 + R;
  auto found = m->ws_tilings.find(key);
  if (found != m->ws_tilings.end()) return found->second.get();
  std::vector<int32_t> elems;
  std::vector<int64_t> tptr;
  greedy_tiles(m, te, ws_node_cap(te), elems, tptr);
  const int64_t nt = (int64_t)tptr.size() - 1;
  const int XR = 3 * R, S = ws_slot_stride(R);
  FE_REQUIRE((int64_t)te * S + 10 * XR < 65536, "tile of %d elements too large for 16-bit slot offsets", te);
  // Tile-local nodes sorted by descending incidence count, then node id. The node
  // sums run over virtual nodes: a node's incidences (grouped by node) split into
  // ceil(count / kVnMax) near-equal consecutive pieces, longest pieces first, so that
  // the lanes of a warp run loops of similar length.
  std::vector<std::vector<int32_t>> tnodes((size_t)nt);
  std::vector<std::vector<int>> tdeg((size_t)nt);
  int nnmax = 0, nvmax = 0;
  int64_t node_sum = 0;
  {
    std::vector<int32_t> buf;
    for (int64_t t = 0; t < nt; ++t) {
      buf.clear();
      for (int64_t q = tptr[(size_t)t]; q < tptr[(size_t)t + 1]; ++q)
        for (int a = 0; a < 10; ++a) buf.push_back(m->conn_host[(size_t)(10 * (int64_t)elems[(size_t)q] + a)]);
      std::sort(buf.begin(), buf.end());
      std::vector<std::pair<int, int32_t>> cnt;  // (-count, id)
      for (size_t q = 0; q < buf.size();) {
        size_t r = q;
        while (r < buf.size() && buf[r] == buf[q]) ++r;
        cnt.push_back({-(int)(r - q), buf[q]});
        q = r;
      }
      std::sort(cnt.begin(), cnt.end());
      std::vector<int32_t>& tn = tnodes[(size_t)t];
      std::vector<int>& td = tdeg[(size_t)t];
      int nv = 0;
      for (auto& pr : cnt) {
        tn.push_back(pr.second);
        td.push_back(-pr.first);
        nv += (-pr.first + kVnMax - 1) / kVnMax;
      }
      nnmax = std::max(nnmax, (int)tn.size());
      nvmax = std::max(nvmax, nv);
      node_sum += (int64_t)tn.size();
    }
  }
  FE_REQUIRE((int64_t)nnmax * XR < 65536 && nnmax < 4096,
             "tile of %d elements has too many nodes (%d) for 16-bit row offsets", te, nnmax);
  const WsLayout L(nnmax, nvmax, te);
  std::vector<unsigned char> pk((size_t)nt * L.bytes, 0);
  std::vector<uint8_t> seen((size_t)m->n_nodes, 0);
  std::vector<int32_t> lid((size_t)m->n_nodes, -1);
  std::vector<std::pair<int, unsigned>> vns;
  for (int64_t t = 0; t < nt; ++t) {
    unsigned char* b = pk.data() + (size_t)t * L.bytes;
    const std::vector<int32_t>& tn = tnodes[(size_t)t];
    const int nn = (int)tn.size();
    const int ne = (int)(tptr[(size_t)t + 1] - tptr[(size_t)t]);
    std::memcpy(b + L.ids, tn.data(), (size_t)nn * 4);
    std::memcpy(b + L.elem, &elems[(size_t)tptr[(size_t)t]], (size_t)ne * 4);
    float* crd = reinterpret_cast<float*>(b + L.crd);
    for (int i = 0; i < nn; ++i) {
      const int32_t g = tn[(size_t)i];
      lid[(size_t)g] = i;
      for (int c = 0; c < 3; ++c) crd[4 * i + c] = (float)m->xyz_host[(size_t)(3 * (int64_t)g + c)];
      b[L.mask + i] = m->nmask_host[(size_t)g];
      b[L.own + i] = seen[(size_t)g] ? 0 : 1;
      seen[(size_t)g] = 1;
    }
    // incidences grouped by node (counting sort over local ids)
    std::vector<int> cnt((size_t)nn + 1, 0);
    for (int i = 0; i < nn; ++i) cnt[(size_t)i + 1] = cnt[(size_t)i] + tdeg[(size_t)t][(size_t)i];
    // virtual nodes: (-length, record), record = ln | first << 12 | length << 13 | start << 17
    vns.clear();
    for (int i = 0; i < nn; ++i) {
      const int d = tdeg[(size_t)t][(size_t)i];
      const int pieces = (d + kVnMax - 1) / kVnMax;
      int start = cnt[(size_t)i];
      for (int q = 0; q < pieces; ++q) {
        const int len = d / pieces + (q < d % pieces ? 1 : 0);
        vns.push_back({-len, (unsigned)i | (q == 0 ? 1u << 12 : 0u) | ((unsigned)len << 13) | ((unsigned)start << 17)});
        start += len;
      }
    }
    std::stable_sort(vns.begin(), vns.end(),
                     [](const std::pair<int, unsigned>& x, const std::pair<int, unsigned>& y) { return x.first < y.first; });
    const int nv = (int)vns.size();
    unsigned* vr = reinterpret_cast<unsigned*>(b + L.vn);
    for (int v = 0; v < nv; ++v) vr[v] = vns[(size_t)v].second;
    const int32_t hdr[4] = {nn, ne, nv, 0};
    std::memcpy(b, hdr, 16);
    uint16_t* io = reinterpret_cast<uint16_t*>(b + L.inc_off);
    uint16_t* eo = reinterpret_cast<uint16_t*>(b + L.eoff);
    for (int le = 0; le < ne; ++le) {
      const int32_t* nd = &m->conn_host[(size_t)(10 * (int64_t)elems[(size_t)(tptr[(size_t)t] + le)])];
      for (int a = 0; a < 10; ++a) {
        const int ln = lid[(size_t)nd[a]];
        io[cnt[(size_t)ln]++] = (uint16_t)(le * S + a * XR);
        eo[le * 16 + a] = (uint16_t)(ln * XR);
        if (a < 4) eo[le * 16 + 10 + a] = (uint16_t)ln;
      }
    }
    for (int i = 0; i < nn; ++i) lid[(size_t)tn[(size_t)i]] = -1;
  }
  std::unique_ptr<WsTiling> tp(new WsTiling());
  tp->te = te;
  tp->R = R;
  tp->nnmax = nnmax;
  tp->nvmax = nvmax;
  tp->pk_bytes = L.bytes;
  tp->n_tiles = nt;
  tp->nodes_per_elem = (double)node_sum / (double)m->n_elem;
  tp->packets.alloc(pk.size());
  FE_CUDA(cudaMemcpyAsync(tp->packets.ptr, pk.data(), pk.size(), cudaMemcpyHostToDevice, s));
  refresh_tiling_materials(m, *tp, s);
  FE_CUDA(cudaStreamSynchronize(s));
  const WsTiling* out = tp.get();
  m->ws_tilings[key] = std::move(tp);
  return out;
}

// Shared memory a block of nth threads may use: the opt-in maximum for one block
// per SM, half of the SM's shared memory (less the per-block reservation) for two.
static int ws_smem_budget(int device, int nth) {
  int optin = 0, per_sm = 0, reserved = 0;
  FE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  if (nth == kWsThreads) return optin;
  FE_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  FE_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
  return std::min(optin, per_sm / 2 - reserved);
}

// Packet slots that fit beside the tile's other buffers (at most kPkMax; fewer than
// kPkMin means the tiling does not fit).
static int ws_packet_slots(const WsTiling& t, int R, int budget) {
  const WsSmem base(t.te, R, t.nnmax, t.pk_bytes, 0);
  if (base.bytes >= budget) return 0;
  return std::min(kPkMax, (budget - base.bytes) / t.pk_bytes);
}

// The tiling fits when its buffers fit in shared memory with at least kPkMin packet
// slots and the block keeps at least 4 staging warps (geometry, two loaders, node sums).
bool ws_fits(fe_mesh* m, int te, int R, int nth) {
  if (!ws_supported(R) || (nth != kWsThreads && nth != kWsThreads / 2)) return false;
  const int cw = ws_compute_warps(te, R);
  if (cw < 1 || cw > nth / 32 - 4) return false;
  const WsTiling* t = get_ws_tiling(m, te, R, nullptr);
  return ws_packet_slots(*t, R, ws_smem_budget(m->device, nth)) >= kPkMin;
}

template <int R, int NT>
static void launch_ws_r(const fe_mesh* m, const WsTiling& t, const float* x, float* y, cudaStream_t s,
                        const int* skip) {
  WsArgs A;
  A.n_tiles = t.n_tiles;
  A.te = t.te;
  A.nnmax = t.nnmax;
  A.nvmax = t.nvmax;
  A.pk = t.pk_bytes;
  A.npk = ws_packet_slots(t, R, ws_smem_budget(m->device, NT));
  A.cw = ws_compute_warps(t.te, R);
  A.nlw = ws_loader_warps(NT / 32 - A.cw);
  A.packets = t.packets.as<unsigned char>();
  A.x = x;
  A.y = y;
  A.skip = skip;
  A.status = m->dev_status.as<int>();
  A.timeout = 1LL << 31;   // about one second at 2 GHz
  A.sm = WsSmem(t.te, R, t.nnmax, t.pk_bytes, A.npk);
  FE_REQUIRE(A.cw >= 1 && A.cw <= NT / 32 - 4, "invalid tile size %d for R = %d with %d threads", t.te, R, NT);
  FE_REQUIRE(A.npk >= kPkMin && A.npk <= kPkMax, "warp-specialised tile needs %d B of shared memory",
             WsSmem(t.te, R, t.nnmax, t.pk_bytes, kPkMin).bytes);
  FE_CUDA(cudaFuncSetAttribute(ebe_ws_kernel<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, A.sm.bytes));
  int sms = 0, per_sm = 0;
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ebe_ws_kernel<R, NT>, NT, A.sm.bytes));
  FE_REQUIRE(per_sm >= 1, "warp-specialised kernel does not fit on an SM");
  const int64_t grid = std::min<int64_t>(t.n_tiles, (int64_t)sms * std::min(per_sm, kWsThreads / NT));
  ebe_ws_kernel<R, NT><<<(unsigned)grid, NT, A.sm.bytes, s>>>(A);
  FE_CHECK_LAUNCH();
}

template <int NT>
static void launch_ws_nt(const fe_mesh* m, const WsTiling& t, const float* x, float* y, cudaStream_t s,
                         const int* skip) {
  switch (t.R) {
    case 4: return launch_ws_r<4, NT>(m, t, x, y, s, skip);
    case 8: return launch_ws_r<8, NT>(m, t, x, y, s, skip);
    case 16: return launch_ws_r<16, NT>(m, t, x, y, s, skip);
    case 32: return launch_ws_r<32, NT>(m, t, x, y, s, skip);
    default: FE_REQUIRE(false, "the warp-specialised kernel is built for R in {4, 8, 16, 32}, not %d", t.R);
  }
}

void launch_ws(const fe_mesh* m, const WsTiling& t, const float* x, float* y, cudaStream_t s, const int* skip,
               int nth) {
  if (nth == kWsThreads / 2)
    launch_ws_nt<kWsThreads / 2>(m, t, x, y, s, skip);
  else
    launch_ws_nt<kWsThreads>(m, t, x, y, s, skip);
}

}  // namespace fe

