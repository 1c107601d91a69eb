// C ABI of libfe: mesh creation and validation, EBE product entry point, errors.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

static thread_local std::string g_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
}

void clear_error() { g_error.clear(); }

DeviceGuard::DeviceGuard(int dev) {
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != dev) FE_CUDA(cudaSetDevice(dev));
}

DeviceGuard::~DeviceGuard() {
  int cur = -1;
  if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

void DevBuf::alloc(size_t n) {
  release();
  if (n == 0) return;
  cudaError_t e = cudaMalloc(&ptr, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    set_error("cudaMalloc of %zu bytes failed: %s", n, cudaGetErrorString(e));
    throw Failure{FE_ENOMEM};
  }
  bytes = n;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------------------
// element order and tiles
// ---------------------------------------------------------------------------

static uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

// Morton (Z-curve) order of element centroids: neighbouring elements get
// neighbouring indices, so element tiles are compact and node data is reused
// from L2 while it is hot.
static std::vector<int64_t> morton_order(int64_t N, const double* xyz, int64_t E, const int32_t* conn) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t n = 0; n < N; ++n)
    for (int i = 0; i < 3; ++i) {
      lo[i] = std::min(lo[i], xyz[3 * n + i]);
      hi[i] = std::max(hi[i], xyz[3 * n + i]);
    }
  double scale = 0.0;
  for (int i = 0; i < 3; ++i) scale = std::max(scale, hi[i] - lo[i]);
  scale = scale > 0 ? (double)((1 << 21) - 1) / scale : 0.0;
  std::vector<uint64_t> key((size_t)E);
  for (int64_t e = 0; e < E; ++e) {
    uint64_t k = 0;
    for (int i = 0; i < 3; ++i) {
      double c = 0.0;
      for (int a = 0; a < 4; ++a) c += xyz[3 * (int64_t)conn[10 * e + a] + i];
      c = 0.25 * c;
      uint64_t q = (uint64_t)std::llround((c - lo[i]) * scale);
      k |= spread3(q) << i;
    }
    key[(size_t)e] = k;
  }
  std::vector<int64_t> order((size_t)E);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[(size_t)a] < key[(size_t)b]; });
  return order;
}

const Tiling* get_tiling(fe_mesh* m, int tile_elems, cudaStream_t s) {
  FE_REQUIRE(tile_elems >= 1 && tile_elems <= 4096, "tile size %d out of range", tile_elems);
  auto found = m->tilings.find(tile_elems);
  if (found != m->tilings.end()) return found->second.get();
  std::unique_ptr<Tiling> tp(new Tiling());
  Tiling& t = *tp;
  const int64_t E = m->n_elem;
  const int64_t nt = (E + tile_elems - 1) / tile_elems;
  std::vector<int32_t> ptr((size_t)nt + 1, 0);
  std::vector<int32_t> ids;
  std::vector<uint16_t> lconn((size_t)E * 10);
  std::vector<uint16_t> inc((size_t)E * 10);
  std::vector<uint16_t> inc_start;
  inc_start.reserve((size_t)E * 3);
  ids.reserve((size_t)E * 3);
  std::vector<int32_t> buf;
  std::vector<uint8_t> own;
  own.reserve((size_t)E * 3);
  std::vector<uint8_t> seen((size_t)m->n_nodes, 0);
  int max_nodes = 0;
  for (int64_t ti = 0; ti < nt; ++ti) {
    const int64_t e0 = ti * tile_elems, e1 = std::min(E, e0 + tile_elems);
    buf.assign(m->conn_host.begin() + 10 * e0, m->conn_host.begin() + 10 * e1);
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    FE_REQUIRE(buf.size() <= 65535 && (e1 - e0) * 10 <= 65535, "tile too large");
    max_nodes = std::max(max_nodes, (int)buf.size());
    // tile-local node order: most incident elements first, so that the lanes of a
    // warp that sum node contributions run loops of similar length
    {
      const int nb = (int)buf.size();
      std::vector<int> cnt((size_t)nb, 0), slot((size_t)(e1 - e0) * 10);
      for (int64_t e = e0; e < e1; ++e)
        for (int a = 0; a < 10; ++a) {
          const int32_t g = m->conn_host[(size_t)(10 * e + a)];
          const int k = (int)(std::lower_bound(buf.begin(), buf.end(), g) - buf.begin());
          slot[(size_t)((e - e0) * 10 + a)] = k;
          cnt[(size_t)k]++;
        }
      std::vector<int> order((size_t)nb), newpos((size_t)nb);
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[(size_t)a] > cnt[(size_t)b]; });
      std::vector<int32_t> sorted((size_t)nb);
      for (int i = 0; i < nb; ++i) {
        newpos[(size_t)order[(size_t)i]] = i;
        sorted[(size_t)i] = buf[(size_t)order[(size_t)i]];
      }
      buf.swap(sorted);
      for (int64_t e = e0; e < e1; ++e)
        for (int a = 0; a < 10; ++a)
          lconn[(size_t)(10 * e + a)] = (uint16_t)newpos[(size_t)slot[(size_t)((e - e0) * 10 + a)]];
    }
    FE_REQUIRE(ids.size() + buf.size() < (size_t)INT32_MAX, "tiling too large");
    ids.insert(ids.end(), buf.begin(), buf.end());
    for (int32_t g : buf) {
      own.push_back(seen[(size_t)g] ? 0 : 1);
      seen[(size_t)g] = 1;
    }
    // element-node slots of the tile grouped by local node (counting sort)
    const int nn = (int)buf.size();
    std::vector<int> cnt((size_t)nn + 1, 0);
    for (int64_t e = e0; e < e1; ++e)
      for (int a = 0; a < 10; ++a) cnt[(size_t)lconn[(size_t)(10 * e + a)] + 1]++;
    for (int i = 0; i < nn; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
    for (int i = 0; i < nn; ++i) inc_start.push_back((uint16_t)cnt[(size_t)i]);
    for (int64_t e = e0; e < e1; ++e)
      for (int a = 0; a < 10; ++a) {
        const int ln = lconn[(size_t)(10 * e + a)];
        inc[(size_t)(10 * e0 + cnt[(size_t)ln]++)] = (uint16_t)((e - e0) * 10 + a);
      }
    ptr[(size_t)ti + 1] = (int32_t)ids.size();
  }
  t.node_ptr.alloc(ptr.size() * sizeof(int32_t));
  t.node_ids.alloc(ids.size() * sizeof(int32_t));
  t.lconn.alloc(lconn.size() * sizeof(uint16_t));
  t.node_own.alloc(own.size());
  t.inc.alloc(inc.size() * sizeof(uint16_t));
  t.inc_start.alloc(inc_start.size() * sizeof(uint16_t));
  FE_CUDA(cudaMemcpyAsync(t.inc.ptr, inc.data(), inc.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(t.inc_start.ptr, inc_start.data(), inc_start.size() * sizeof(uint16_t),
                          cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(t.node_own.ptr, own.data(), own.size(), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(t.node_ptr.ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(t.node_ids.ptr, ids.data(), ids.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(t.lconn.ptr, lconn.data(), lconn.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaStreamSynchronize(s));
  // packets: one contiguous block per tile
  {
    const PacketLayout L(max_nodes, tile_elems);
    std::vector<unsigned char> pk((size_t)nt * L.bytes, 0);
    for (int64_t ti = 0; ti < nt; ++ti) {
      unsigned char* b = pk.data() + (size_t)ti * L.bytes;
      const int64_t e0 = ti * tile_elems, e1 = std::min(E, e0 + tile_elems);
      const int p0 = ptr[(size_t)ti], nn = ptr[(size_t)ti + 1] - p0, ne = (int)(e1 - e0);
      int32_t hdr[4] = {nn, ne, 0, 0};
      std::memcpy(b, hdr, 16);
      std::memcpy(b + L.ids, &ids[(size_t)p0], (size_t)nn * 4);
      for (int i = 0; i < nn; ++i) {
        const int32_t g = ids[(size_t)p0 + i];
        const uint8_t mk = (uint8_t)(m->nmask_host[(size_t)g]);
        b[L.mask + i] = mk;
        b[L.own + i] = own[(size_t)p0 + i];
      }
      std::memcpy(b + L.inc_start, &inc_start[(size_t)p0], (size_t)nn * 2);
      const uint16_t endv = (uint16_t)(ne * 10);
      std::memcpy(b + L.inc_start + 2 * nn, &endv, 2);
      std::memcpy(b + L.lconn, &lconn[(size_t)e0 * 10], (size_t)ne * 20);
      std::memcpy(b + L.inc, &inc[(size_t)e0 * 10], (size_t)ne * 20);
    }
    t.packets.alloc(pk.size());
    FE_CUDA(cudaMemcpyAsync(t.packets.ptr, pk.data(), pk.size(), cudaMemcpyHostToDevice, s));
    FE_CUDA(cudaStreamSynchronize(s));
    t.packet_bytes = L.bytes;
  }
  t.tile_elems = tile_elems;
  t.max_nodes = max_nodes;
  t.n_tiles = nt;
  const Tiling* out = tp.get();
  m->tilings[tile_elems] = std::move(tp);
  return out;
}

// ---------------------------------------------------------------------------
// element colouring (greedy, first fit, elements in internal order): each element
// takes the lowest colour that none of the elements sharing one of its nodes has
// taken, read from a per-node bit set of used colours (up to 256 colours)
// ---------------------------------------------------------------------------
void build_colouring(fe_mesh* m, cudaStream_t s) {
  Colouring& c = m->colouring;
  if (c.ready) return;
  constexpr int W = 4;  // 64-bit words of colour bits per node
  const int64_t E = m->n_elem;
  std::vector<uint64_t> used((size_t)m->n_nodes * W, 0);
  std::vector<int32_t> colour((size_t)E);
  int n_colours = 0;
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* nd = &m->conn_host[(size_t)(10 * e)];
    int col = -1;
    for (int w = 0; w < W && col < 0; ++w) {
      uint64_t taken = 0;
      for (int a = 0; a < 10; ++a) taken |= used[(size_t)nd[a] * W + w];
      if (~taken) {
        uint64_t free_bits = ~taken;
        int b = 0;
        while (!(free_bits & 1)) {
          free_bits >>= 1;
          ++b;
        }
        col = 64 * w + b;
      }
    }
    FE_REQUIRE(col >= 0, "element colouring needs more than %d colours", 64 * W);
    for (int a = 0; a < 10; ++a) used[(size_t)nd[a] * W + col / 64] |= uint64_t(1) << (col % 64);
    colour[(size_t)e] = col;
    n_colours = std::max(n_colours, col + 1);
  }
  // group by colour (counting sort keeps internal order within a colour)
  c.ptr.assign((size_t)n_colours + 1, 0);
  for (int64_t e = 0; e < E; ++e) c.ptr[(size_t)colour[(size_t)e] + 1]++;
  for (int k = 0; k < n_colours; ++k) c.ptr[(size_t)k + 1] += c.ptr[(size_t)k];
  std::vector<int64_t> pos(c.ptr.begin(), c.ptr.end() - 1);
  std::vector<int32_t> elems((size_t)E);
  for (int64_t e = 0; e < E; ++e) elems[(size_t)pos[(size_t)colour[(size_t)e]]++] = (int32_t)e;
  c.elems.alloc(elems.size() * sizeof(int32_t));
  FE_CUDA(cudaMemcpyAsync(c.elems.ptr, elems.data(), elems.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaStreamSynchronize(s));
  c.n_colours = n_colours;
  c.ready = true;
}

// ---------------------------------------------------------------------------
// materials upload (internal element order)
// ---------------------------------------------------------------------------
static void upload_materials(fe_mesh* m, cudaStream_t s) {
  const int64_t E = m->n_elem;
  std::vector<double> m64((size_t)E * 2);
  std::vector<float> m32((size_t)E * 2);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t src = m->perm_host[(size_t)e];
    m64[2 * e] = m->young_host[(size_t)src];
    m64[2 * e + 1] = m->poisson_host[(size_t)src];
    m32[2 * e] = (float)m64[2 * e];
    m32[2 * e + 1] = (float)m64[2 * e + 1];
  }
  std::vector<float> mv((size_t)E * 4, 0.f);
  for (int64_t e = 0; e < E; ++e) {
    mv[(size_t)(4 * e)] = m32[(size_t)(2 * e)];
    mv[(size_t)(4 * e + 1)] = m32[(size_t)(2 * e + 1)];
  }
  FE_CUDA(cudaMemcpyAsync(m->mat64.ptr, m64.data(), m64.size() * 8, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(m->mat32.ptr, m32.data(), m32.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(m->matv.ptr, mv.data(), mv.size() * 4, cudaMemcpyHostToDevice, s));
  fe::ws_refresh_materials(m, s);
  FE_CUDA(cudaStreamSynchronize(s));
  m->jacobi_ready = false;
  m->coarse.jacobi_ready = false;
  m->coarse.geo_ready = false;
  m->coarse.csr_ready = false;
  m->coarse.l2_ready = false;
}

}  // namespace fe

template <>
fe::MeshView<double> fe_mesh::view<double>() const {
  return {n_nodes, n_elem, conn.as<int32_t>(), xyz64.as<double>(), mat64.as<double>(), nmask.as<uint8_t>()};
}
template <>
fe::MeshView<float> fe_mesh::view<float>() const {
  return {n_nodes, n_elem, conn.as<int32_t>(), xyz32.as<float>(), mat32.as<float>(), nmask.as<uint8_t>()};
}

using namespace fe;

extern "C" {

const char* fe_last_error(void) { return g_error.c_str(); }

const char* fe_version(void) { return "libfe 0.1 (sm_103a)"; }

void fe_solve_opts_default(fe_solve_opts* o) {
  if (!o) return;
  o->solver = FE_SOLVER_FCG_MIXED;
  o->tol = 1e-8;
  o->max_outer = 20000;
  o->n_inner = 30;
  o->eps_inner = 0.1;
  o->use_graph = 1;
  o->literal_beta = 0;
  o->check_every = 1;
  o->verbose = 0;
  o->n_inner1 = 300;
  o->eps_inner1 = 0.05;
  o->coarse_op = 0;
  o->n_inner2 = 3000;
  o->eps_inner2 = 0.025;
  o->cg_coef = nullptr;
  o->cg_coef_len = 0;
  o->inner_kernel = 1;
}

fe_status fe_mesh_create(int64_t n_nodes, const double* coords, int64_t n_elem, const int32_t* conn,
                         const double* young, const double* poisson, const uint8_t* free_mask, int32_t device,
                         void* stream, fe_mesh** out) {
  if (out) *out = nullptr;
  fe_mesh* m = nullptr;
  fe_status st = guarded([&] {
    FE_REQUIRE(out != nullptr, "out is NULL");
    FE_REQUIRE(coords && conn && young && poisson && free_mask, "NULL input array");
    FE_REQUIRE(n_nodes > 0 && n_nodes < (int64_t)INT32_MAX, "n_nodes = %lld out of range", (long long)n_nodes);
    FE_REQUIRE(n_elem > 0 && n_elem < ((int64_t)1 << 40), "n_elem = %lld out of range", (long long)n_elem);
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
      FE_REQUIRE(std::isfinite(coords[i]), "coordinate of node %lld is not finite", (long long)(i / 3));
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
      FE_REQUIRE(free_mask[i] <= 1, "free_mask of node %lld is not 0/1", (long long)(i / 3));
    for (int64_t e = 0; e < n_elem; ++e) {
      const int32_t* ce = conn + 10 * e;
      for (int a = 0; a < 10; ++a) {
        FE_REQUIRE(ce[a] >= 0 && ce[a] < n_nodes, "element %lld: node id %d out of range", (long long)e, ce[a]);
        for (int b = 0; b < a; ++b)
          FE_REQUIRE(ce[a] != ce[b], "element %lld: node %d repeated", (long long)e, ce[a]);
      }
      FE_REQUIRE(std::isfinite(young[e]) && young[e] > 0.0, "element %lld: Young's modulus must be > 0",
                 (long long)e);
      FE_REQUIRE(std::isfinite(poisson[e]) && poisson[e] > -1.0 && poisson[e] < 0.5,
                 "element %lld: Poisson ratio must lie in (-1, 0.5)", (long long)e);
      const double* x0 = coords + 3 * (int64_t)ce[0];
      double d[3][3];
      double hmax = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) {
          d[k][i] = coords[3 * (int64_t)ce[k + 1] + i] - x0[i];
          hmax = std::max(hmax, std::fabs(d[k][i]));
        }
      const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                         d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                         d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
      FE_REQUIRE(det > 1e-12 * hmax * hmax * hmax, "element %lld: non-positive volume (inverted or flat)",
                 (long long)e);
      static const int EA[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
      for (int q = 0; q < 6; ++q)
        for (int i = 0; i < 3; ++i) {
          const double mid = 0.5 * (coords[3 * (int64_t)ce[EA[q][0]] + i] + coords[3 * (int64_t)ce[EA[q][1]] + i]);
          FE_REQUIRE(std::fabs(coords[3 * (int64_t)ce[4 + q] + i] - mid) <= 1e-6 * hmax,
                     "element %lld: edge node %d is not at its edge midpoint (elements must be straight-sided)",
                     (long long)e, 4 + q);
        }
    }
    int ndev = 0;
    FE_CUDA(cudaGetDeviceCount(&ndev));
    FE_REQUIRE(device >= 0 && device < ndev, "device %d not present (%d devices)", device, ndev);
    DeviceGuard dg(device);
    cudaStream_t s = (cudaStream_t)stream;
    m = new fe_mesh();
    m->device = device;
    m->n_nodes = n_nodes;
    m->n_elem = n_elem;
    std::memset(m->variant, -1, sizeof(m->variant));
    m->perm_host = morton_order(n_nodes, coords, n_elem, conn);
    m->conn_host.resize((size_t)n_elem * 10);
    for (int64_t e = 0; e < n_elem; ++e)
      std::memcpy(&m->conn_host[(size_t)e * 10], conn + 10 * m->perm_host[(size_t)e], 10 * sizeof(int32_t));
    m->young_host.assign(young, young + n_elem);
    m->xyz_host.assign(coords, coords + 3 * n_nodes);
    m->poisson_host.assign(poisson, poisson + n_elem);
    std::vector<float> xyz32((size_t)n_nodes * 3);
    for (int64_t i = 0; i < 3 * n_nodes; ++i) xyz32[(size_t)i] = (float)coords[i];
    std::vector<uint8_t> nm((size_t)n_nodes);
    for (int64_t n = 0; n < n_nodes; ++n)
      nm[(size_t)n] = (uint8_t)(free_mask[3 * n] | (free_mask[3 * n + 1] << 1) | (free_mask[3 * n + 2] << 2));
    m->conn.alloc((size_t)n_elem * 10 * sizeof(int32_t));
    m->xyz64.alloc((size_t)n_nodes * 3 * sizeof(double));
    m->xyz32.alloc((size_t)n_nodes * 3 * sizeof(float));
    m->mat64.alloc((size_t)n_elem * 2 * sizeof(double));
    m->mat32.alloc((size_t)n_elem * 2 * sizeof(float));
    m->matv.alloc((size_t)n_elem * 4 * sizeof(float));
    m->dev_status.alloc(sizeof(int32_t));
    FE_CUDA(cudaMemsetAsync(m->dev_status.ptr, 0, sizeof(int32_t), s));
    m->nmask.alloc((size_t)n_nodes);
    m->perm.alloc((size_t)n_elem * sizeof(int64_t));
    m->own_elem.alloc((size_t)n_elem * sizeof(uint16_t));
    {
      std::vector<uint16_t> ow((size_t)n_elem, 0);
      std::vector<uint8_t> seen((size_t)n_nodes, 0);
      for (int64_t e = 0; e < n_elem; ++e)
        for (int a = 0; a < 10; ++a) {
          const int32_t g = m->conn_host[(size_t)(10 * e + a)];
          if (!seen[(size_t)g]) {
            seen[(size_t)g] = 1;
            ow[(size_t)e] |= (uint16_t)(1u << a);
          }
        }
      FE_CUDA(cudaMemcpyAsync(m->own_elem.ptr, ow.data(), ow.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
      FE_CUDA(cudaStreamSynchronize(s));
    }
    FE_CUDA(cudaMemcpyAsync(m->conn.ptr, m->conn_host.data(), m->conn.bytes, cudaMemcpyHostToDevice, s));
    FE_CUDA(cudaMemcpyAsync(m->xyz64.ptr, coords, m->xyz64.bytes, cudaMemcpyHostToDevice, s));
    FE_CUDA(cudaMemcpyAsync(m->xyz32.ptr, xyz32.data(), m->xyz32.bytes, cudaMemcpyHostToDevice, s));
    FE_CUDA(cudaMemcpyAsync(m->nmask.ptr, nm.data(), m->nmask.bytes, cudaMemcpyHostToDevice, s));
    m->nmask_host = nm;
    FE_CUDA(cudaMemcpyAsync(m->perm.ptr, m->perm_host.data(), m->perm.bytes, cudaMemcpyHostToDevice, s));
    upload_materials(m, s);
    *out = m;
  });
  if (st != FE_OK) {
    delete m;
    if (out) *out = nullptr;
  }
  return st;
}

void fe_mesh_destroy(fe_mesh* m) {
  if (!m) return;
  try {
    DeviceGuard dg(m->device);
    cudaDeviceSynchronize();
    free_solver_work(m);
    delete m;
  } catch (...) {
  }
}

fe_status fe_mesh_device_status(const fe_mesh* m, void* stream) {
  int32_t v = 0;
  const fe_status st = guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    FE_CUDA(cudaMemcpyAsync(&v, m->dev_status.ptr, sizeof(v), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemsetAsync(m->dev_status.ptr, 0, sizeof(v), s));
    FE_CUDA(cudaStreamSynchronize(s));
  });
  if (st != FE_OK) return st;
  if (v != 0) {
    set_error("a bounded device-side wait gave up; the results of the kernels since the last check are invalid");
    return FE_ETIMEOUT;
  }
  return FE_OK;
}

fe_status fe_wait_selftest(const fe_mesh* m, int32_t which, int64_t cycles, void* stream) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(which == 0 || which == 1, "which must be 0 (mbarrier wait) or 1 (grid barrier), got %d", which);
    FE_REQUIRE(cycles >= 1 && cycles <= (int64_t)1 << 32, "cycles must be in [1, 2^32], got %lld",
               (long long)cycles);
    DeviceGuard dg(m->device);
    if (which == 0)
      ws_wait_selftest(m, (long long)cycles, (cudaStream_t)stream);
    else
      grid_wait_selftest(m, (long long)cycles, (cudaStream_t)stream);
  });
}

fe_status fe_mesh_info(const fe_mesh* m, int64_t* n_nodes, int64_t* n_elem) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_elem) *n_elem = m->n_elem;
  });
}

fe_status fe_ebe_apply(const fe_mesh* m, int32_t R, fe_dtype dtype, const void* x, void* y, void* stream) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    FE_REQUIRE(dtype == FE_F64 || dtype == FE_F32, "unknown dtype %d", (int)dtype);
    FE_REQUIRE(x != nullptr && y != nullptr, "NULL vector");
    FE_REQUIRE(x != y, "x and y must not alias");
    FE_REQUIRE(((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0, "vectors must be 16-byte aligned");
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == FE_F64)
      ebe_apply<double>(m, R, static_cast<const double*>(x), static_cast<double*>(y), s);
    else
      ebe_apply<float>(m, R, static_cast<const float*>(x), static_cast<float*>(y), s);
  });
}

fe_status fe_ebe_set_variant(fe_mesh* m, int32_t R, fe_dtype dtype, int32_t variant, int32_t tile_elems,
                             void* stream) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range", R);
    FE_REQUIRE(variant == FE_EBE_DIRECT || variant == FE_EBE_TILED || variant == FE_EBE_GATHER ||
                   variant == FE_EBE_GATHER_DF || variant == FE_EBE_GATHER_X2 || variant == FE_EBE_COLOUR ||
                   variant == FE_EBE_WS || variant == FE_EBE_DF_LEAN || variant == FE_EBE_WS2,
               "unknown variant %d", variant);
    FE_REQUIRE((variant != FE_EBE_WS && variant != FE_EBE_WS2) || (dtype == FE_F32 && ws_supported(R)),
               "the warp-specialised kernel computes FP32 products for R in {4, 8, 16, 32}");
    FE_REQUIRE((variant != FE_EBE_GATHER_DF && variant != FE_EBE_DF_LEAN) || (dtype == FE_F64 && df_supported(R)),
               "the float-float kernel computes FP64 products for R in {2, 4, 8, 16, 32}");
    FE_REQUIRE(variant != FE_EBE_GATHER_X2 || (dtype == FE_F32 && x2_supported(R)),
               "the paired-arithmetic kernel computes FP32 products for R in {4, 8, 16, 32}");
    DeviceGuard dg(m->device);
    if (variant == FE_EBE_DIRECT) {
      ebe_set_variant(m, R, dtype == FE_F32, 0);
      return;
    }
    if (variant == FE_EBE_COLOUR) {
      build_colouring(m, (cudaStream_t)stream);
      ebe_set_variant(m, R, dtype == FE_F32, FE_EBE_COLOUR * 65536 + m->colouring.n_colours);
      return;
    }
    if (variant == FE_EBE_WS || variant == FE_EBE_WS2) {
      FE_REQUIRE(tile_elems >= 1 && tile_elems <= 4096, "tile size %d out of range", tile_elems);
      FE_REQUIRE(ws_fits(m, tile_elems, R, variant == FE_EBE_WS2 ? 256 : 512),
                 "warp-specialised tiles of %d elements do not fit for R = %d", tile_elems, R);
      ebe_set_variant(m, R, 1, variant * 65536 + tile_elems);
      return;
    }
    FE_REQUIRE(variant != FE_EBE_GATHER || gather_supported(R),
               "the gather kernel is compiled for R in {1, 2, 3, 4, 8, 16, 32}, not %d", R);
    get_tiling(m, tile_elems, (cudaStream_t)stream);
    if (variant != FE_EBE_TILED) ensure_geometry_buffer(m, dtype == FE_F32);
    if (variant == FE_EBE_GATHER_DF)
      FE_REQUIRE(df_fits(m, tile_elems, R), "tile of %d elements does not fit in shared memory for R = %d",
                 tile_elems, R);
    else if (variant == FE_EBE_DF_LEAN)
      FE_REQUIRE(df_lean_fits(m, tile_elems, R), "tile of %d elements does not fit in shared memory for R = %d",
                 tile_elems, R);
    else if (variant == FE_EBE_GATHER_X2)
      FE_REQUIRE(x2_fits(m, tile_elems, R), "tile of %d elements does not fit in shared memory for R = %d",
                 tile_elems, R);
    else
      FE_REQUIRE(tiled_fits(m, tile_elems, R, dtype == FE_F32, variant),
                 "tile of %d elements does not fit in shared memory for R = %d", tile_elems, R);
    ebe_set_variant(m, R, dtype == FE_F32, variant * 65536 + tile_elems);
  });
}

fe_status fe_ebe_get_variant(const fe_mesh* m, int32_t R, fe_dtype dtype, int32_t* variant, int32_t* tile_elems) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range", R);
    const int v = ebe_get_variant(m, R, dtype == FE_F32);
    if (variant) *variant = v / 65536;
    if (tile_elems) *tile_elems = v % 65536;
  });
}

fe_status fe_mesh_set_log_young(fe_mesh* m, const double* logE_dev, void* stream) {
  return guarded([&] {
    FE_REQUIRE(m != nullptr && logE_dev != nullptr, "NULL argument");
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> le((size_t)m->n_elem);
    FE_CUDA(cudaMemcpyAsync(le.data(), logE_dev, le.size() * 8, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    for (int64_t e = 0; e < m->n_elem; ++e) {
      const double v = std::exp(le[(size_t)e]);
      FE_REQUIRE(std::isfinite(v) && v > 0.0, "exp(logE) of element %lld is not a positive finite number",
                 (long long)e);
      m->young_host[(size_t)e] = v;
    }
    upload_materials(m, s);
  });
}

}  // extern "C"
