// Internal declarations of libfe (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fe.h"

namespace fe {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Failure {
  fe_status status;
};

#define FE_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t err__ = (call);                                                           \
    if (err__ != cudaSuccess) {                                                           \
      ::fe::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(err__), __FILE__, \
                      __LINE__);                                                          \
      throw ::fe::Failure{FE_ECUDA};                                                      \
    }                                                                                     \
  } while (0)

#define FE_CHECK_LAUNCH() FE_CUDA(cudaGetLastError())

#define FE_REQUIRE(cond, ...)          \
  do {                                 \
    if (!(cond)) {                     \
      ::fe::set_error(__VA_ARGS__);    \
      throw ::fe::Failure{FE_EINVAL};  \
    }                                  \
  } while (0)

// Runs f, converting library failures and C++ exceptions into a status.
template <typename F>
inline fe_status guarded(F&& f) {
  try {
    clear_error();
    f();
    return FE_OK;
  } catch (const Failure& x) {
    return x.status;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return FE_ENOMEM;
  } catch (...) {
    set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}

// Sets the mesh's device current for the scope and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void alloc(size_t n);
  void release();
  template <typename T>
  T* as() const { return static_cast<T*>(ptr); }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// Pointers a kernel needs to evaluate element products in precision T.
template <typename T>
struct MeshView {
  int64_t n_nodes;
  int64_t n_elem;
  const int32_t* conn;   // [E][10]
  const T* xyz;          // [N][3]
  const T* mat;          // [E][2]  (E, nu)
  const uint8_t* nmask;  // [N]     bit c set <=> DOF c of the node is free
};

// Tiles of elements for the shared-memory accumulation kernel.
struct Tiling {
  int tile_elems = 0;     // elements per tile (last tile may be shorter)
  int max_nodes = 0;      // largest node count of a tile
  int64_t n_tiles = 0;
  DevBuf node_ptr;        // int32 [n_tiles+1] offsets into node_ids
  DevBuf node_ids;        // int32 [sum of tile node counts] global node ids per tile
  DevBuf node_own;        // uint8, parallel to node_ids: 1 if this is the node's first tile
  DevBuf lconn;           // uint16 [E][10] tile-local node index per element corner
  DevBuf inc;             // uint16 [E][10] per tile: element-node slots (le*10 + a) sorted by local node
  DevBuf inc_start;       // uint16, parallel to node_ids: first slot of the node in `inc` (tile-relative)
  // per-tile packets for the pipelined gather kernel: every array of one tile in
  // one contiguous block of `packet_bytes` (see PacketLayout)
  int packet_bytes = 0;
  DevBuf packets;
};

// Element colouring: no two elements of one colour share a node, so the products
// of one colour can be added into y without atomics (one launch per colour).
struct Colouring {
  bool ready = false;
  int n_colours = 0;
  std::vector<int64_t> ptr;  // [n_colours + 1] offsets into elems
  DevBuf elems;              // int32 [E] internal element ids grouped by colour, ascending within a colour
};

// Byte layout of a tile packet (host and device agree on it):
//   int32 {nn, ne, 0, 0} | int32 ids[nnmax] | uint8 mask[nnmax] | uint8 own[nnmax] |
//   uint16 inc_start[nnmax + 1] | uint16 lconn[te * 10] | uint16 inc[te * 10]
// each section padded to 16 bytes.
struct PacketLayout {
  int ids, mask, own, inc_start, lconn, inc, bytes;
  __host__ __device__ static int a16(int b) { return (b + 15) & ~15; }
  __host__ __device__ PacketLayout(int nnmax, int te) {
    ids = 16;
    mask = ids + a16(4 * nnmax);
    own = mask + a16(nnmax);
    inc_start = own + a16(nnmax);
    lconn = inc_start + a16(2 * (nnmax + 1));
    inc = lconn + a16(20 * te);
    bytes = inc + a16(20 * te);
  }
};

// First-order (TET4) coarse level: the same mesh without edge nodes (Sec. 2).
struct Coarse {
  bool ready = false;
  int64_t n_nodes = 0;      // N4: corner nodes of the TET10 mesh
  DevBuf conn4;             // int32 [E][4] coarse node ids (internal element order)
  DevBuf ends;              // int32 [N][2] coarse ends of each TET10 node (equal for a vertex)
  DevBuf nmask4;            // uint8 [N4] free-DOF bits
  DevBuf own4;              // uint8 [E] bit a set if element e is the first holding its corner a
  DevBuf vertex;            // int32 [N4] TET10 id of each coarse node
  DevBuf adj_ptr, adj;      // int32 [N4 + 1], [2 * edge nodes]: edge nodes ending at each coarse node
  bool jacobi_ready = false;
  DevBuf binv64, binv32;    // [N4][9] inverse diagonal blocks of K1_bc
  bool geo_ready = false;
  DevBuf geo32;             // float [E][16]: grad L_0..3, lam V, mu V, pad (FP32 TET4 products)
  // assembled K1_bc in 3x3 block CSR (built on first use, per material state)
  bool csr_pattern = false, csr_ready = false;
  int64_t nnzb = 0;
  DevBuf rowptr, cols;      // int32 [N4 + 1], [nnzb] (columns sorted per row)
  DevBuf vals32;            // float [nnzb][9]
  // sliced copy of K1_bc for the product: rows in slices of 8, slot t of a slice
  // holds block t of each of its rows, values interleaved by row ([slot][9][8]) so
  // that one load instruction of a warp reads a value of 8 rows from one sector
  int64_t n_slots = 0;
  DevBuf sl_off;            // int32 [slices + 1] first slot of each slice
  DevBuf sl_cols;           // int32 [n_slots][8] block column (padding: the row itself)
  DevBuf sl_pos;            // int32 [nnzb] slot * 8 + row in slice of each block
  DevBuf sl_vals;           // float [n_slots][9][8]
  std::vector<int32_t> rowptr_host, cols_host, nmask4_host;  // host copies for the level-2 set-up
  // level 2: aggregation of the coarse nodes and its Galerkin matrix A2
  bool l2_pattern = false, l2_ready = false;
  int64_t n_agg = 0, nnzb2 = 0;
  DevBuf agg;               // int32 [N4] aggregate of each coarse node
  DevBuf mptr, members;     // int32 [NA + 1], [N4]: member nodes of each aggregate
  DevBuf nmask2;            // uint8 [NA] free-DOF bits of the aggregates
  DevBuf pos2;              // int32 [nnzb] position in A2 of each K1 block
  DevBuf rowptr2, cols2;    // int32 [NA + 1], [nnzb2] (columns sorted per row)
  DevBuf vals2_32;          // float [nnzb2][9]
  DevBuf binv2_64, binv2_32;  // [NA][9] inverse diagonal blocks of A2
};

// Products with host-resident vectors (fe_ebe_apply_host): two device buffer
// sets used alternately and three streams, so that the copy-in of one call, the
// product of the previous one and the copy-out of the one before overlap.
struct HostPipe {
  int R = 0;
  int dtype = -1;
  DevBuf x[2], y[2];
  cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
  cudaEvent_t h2d[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, d2h[2] = {nullptr, nullptr};
  int next = 0;
  HostPipe() = default;
  HostPipe(const HostPipe&) = delete;
  HostPipe& operator=(const HostPipe&) = delete;
  ~HostPipe();
};

// Tiles of the warp-specialised EBE kernel (fe_ebe_ws.cu), built per (tile size, R):
// elements grouped by greedy growth (each tile adds the element sharing most nodes
// with it), one packet per tile with the tile's node ids and coordinates, element
// ids and materials, slot offsets and row offsets for R cases (see WsLayout in
// fe_ebe_ws.cu); the materials are rewritten when the mesh's materials change.
struct WsTiling {
  int te = 0;             // elements per tile (the last tiles may hold fewer)
  int R = 0;              // cases the offsets are laid out for
  int nnmax = 0;          // largest node count of a tile
  int nvmax = 0;          // largest virtual-node count of a tile (node-sum tasks per 4 cases)
  int pk_bytes = 0;       // bytes per packet (multiple of 16)
  int64_t n_tiles = 0;
  double nodes_per_elem = 0.0;  // sum of tile node counts / elements
  DevBuf packets;
};

struct SolverWork;  // defined in fe_solver.cu

}  // namespace fe

struct fe_mesh {
  int device = 0;
  int64_t n_nodes = 0;
  int64_t n_elem = 0;
  fe::DevBuf conn;      // int32 [E][10]
  fe::DevBuf xyz64;     // double [N][3]
  fe::DevBuf xyz32;     // float [N][3]
  fe::DevBuf mat64;     // double [E][2]
  fe::DevBuf mat32;     // float [E][2]
  fe::DevBuf nmask;     // uint8 [N]
  std::vector<double> young_host;
  std::vector<double> poisson_host;
  // 3x3 block Jacobi (built lazily, invalidated when materials change)
  bool jacobi_ready = false;
  fe::DevBuf binv64;    // double [N][9]
  fe::DevBuf binv32;    // float [N][9]
  // element tilings for the shared-memory EBE kernel, by elements per tile (built lazily)
  std::map<int, std::unique_ptr<fe::Tiling>> tilings;
  // tilings of the warp-specialised kernel, by tile size * 256 + R (built lazily)
  std::map<int, std::unique_ptr<fe::WsTiling>> ws_tilings;
  fe::DevBuf matv;      // float4 [E]: (E, nu, 0, 0) in FP32 (copied into the warp-specialised packets)
  fe::DevBuf dev_status;  // int32: set by a kernel whose bounded wait gave up (fe_mesh_device_status)
  std::vector<double> xyz_host;  // [N][3] coordinates as given
  // EBE kernel per precision (0 = FP64, 1 = FP32) and R: -1 = default, else
  // kind * 65536 + elements per tile (kind: fe_ebe_variant)
  int32_t variant[2][65];
  // internal element order -> caller's element id (elements are stored in a
  // locality-preserving order)
  std::vector<int64_t> perm_host;
  fe::DevBuf perm;      // int64 [E]
  fe::DevBuf own_elem;  // uint16 [E]: bit a set if element e is the first element holding its node a
  // per-product element geometry (g[4][3], lam, mu, V/20, pad) written by the
  // pipelined kernel's prep pass, FP64 and FP32 (allocated when that kernel is chosen)
  fe::DevBuf geo64, geo32;
  fe::DevBuf geodf;     // float-float geometry [E][16] for the float-float FP64 kernel
  std::vector<int32_t> conn_host;  // [E][10] in internal order
  std::vector<uint8_t> nmask_host; // [N] free-DOF bits
  // element colouring for the colour-by-colour EBE kernel (built on first use)
  fe::Colouring colouring;
  // TET4 coarse level (built on first use)
  fe::Coarse coarse;
  // solver workspace (allocated lazily per R)
  fe::SolverWork* work = nullptr;
  // buffers and streams of products with host vectors (allocated on first use)
  std::unique_ptr<fe::HostPipe> host_pipe;

  template <typename T>
  fe::MeshView<T> view() const;
};

namespace fe {

// EBE product dispatch (fe_ebe.cu). x, y: device [N][R][3] of T.
// If `skip` is non-NULL, every launched kernel returns at once when *skip != 0
// (used for inner-loop steps after the stop test fired inside a CUDA graph).
template <typename T>
void ebe_apply(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip = nullptr);

// kernel choice, encoded kind * 65536 + tile (kind: fe_ebe_variant)
int ebe_get_variant(const fe_mesh* m, int R, int is_f32);
void ebe_set_variant(fe_mesh* m, int R, int is_f32, int variant);
bool gather_supported(int R);
void ensure_geometry_buffer(fe_mesh* m, int is_f32);
bool df_supported(int R);
bool df_fits(const fe_mesh* m, int tile_elems, int R);
bool df_lean_fits(const fe_mesh* m, int tile_elems, int R);
bool x2_supported(int R);
bool x2_fits(const fe_mesh* m, int tile_elems, int R);
const Tiling* get_tiling(fe_mesh* m, int tile_elems, cudaStream_t s);
void build_colouring(fe_mesh* m, cudaStream_t s);
// largest tile (elements) whose shared-memory footprint fits for (R, precision)
bool tiled_fits(const fe_mesh* m, int tile_elems, int R, int is_f32, int kind);

// Warp-specialised FP32 kernel (fe_ebe_ws.cu), R in {4, 8, 16, 32}
bool ws_supported(int R);
const WsTiling* get_ws_tiling(fe_mesh* m, int tile_elems, int R, cudaStream_t s);
// nth: threads per block, 512 (FE_EBE_WS, one block per SM) or 256 (FE_EBE_WS2, two)
bool ws_fits(fe_mesh* m, int tile_elems, int R, int nth);
// Rewrites the materials held in the packets of every warp-specialised tiling (after
// the mesh's materials changed).
void ws_refresh_materials(fe_mesh* m, cudaStream_t s);
void launch_ws(const fe_mesh* m, const WsTiling& t, const float* x, float* y, cudaStream_t s, const int* skip,
               int nth);

// Self-tests of the bounded device-side waits (fe_wait_selftest): a wait that nothing
// ends, limited to `cycles`; each records its timeout in the mesh's status word.
void ws_wait_selftest(const fe_mesh* m, long long cycles, cudaStream_t s);    // fe_ebe_ws.cu, mbarrier
void grid_wait_selftest(const fe_mesh* m, long long cycles, cudaStream_t s);  // fe_solver.cu, grid barrier

// Block Jacobi (fe_solver.cu)
void build_block_jacobi(fe_mesh* m, cudaStream_t s);

// Adjoint (fe_adjoint.cu)
void adjoint_grad(const fe_mesh* m, int R, const double* u, const double* lam, double* g, cudaStream_t s);

void free_solver_work(fe_mesh* m);

// Coarse level (fe_coarse.cu)
void build_coarse(fe_mesh* m, cudaStream_t s);
void build_coarse_jacobi(fe_mesh* m, cudaStream_t s);
void build_coarse_geometry(fe_mesh* m, cudaStream_t s);
// false: not enough device memory. With level2, also builds the aggregation level.
bool build_coarse_matrix(fe_mesh* m, cudaStream_t s, bool level2 = false);
void coarse_spmv(const fe_mesh* m, int R, const float* x4, float* y4, cudaStream_t s, const int* skip = nullptr);
// y = A x for a 3x3 block CSR matrix, R cases of [n][R][3] FP32 vectors
void bcsr_spmv(int64_t n, int R, const int32_t* rowptr, const int32_t* cols, const float* vals, const float* x,
               float* y, cudaStream_t s, const int* skip);

// Level 2 (fe_level2.cu)
void build_level2(fe_mesh* m, const double* k1_64, cudaStream_t s);  // K1 blocks in FP64, unmasked
size_t level2_bytes(const fe_mesh* m);                                 // device bytes level 2 will need
void level2_restrict(const fe_mesh* m, int R, const float* r4, float* r2, cudaStream_t s, const int* skip = nullptr);
void level2_prolong(const fe_mesh* m, int R, const float* u2, float* u4, cudaStream_t s, const int* skip = nullptr);
template <typename T>
void ebe4_apply(const fe_mesh* m, int R, const T* x4, T* y4, cudaStream_t s, const int* skip = nullptr);
template <typename T>
void coarse_restrict(const fe_mesh* m, int R, const T* r10, T* r4, cudaStream_t s, const int* skip = nullptr);
template <typename T>
void coarse_prolong(const fe_mesh* m, int R, const T* u4, T* u10, cudaStream_t s, const int* skip = nullptr);

}  // namespace fe
