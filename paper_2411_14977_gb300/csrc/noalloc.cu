// pmg_apply_noalloc: the actual-geometry operator apply (the same kernels as pmg_apply)
// for callers that cannot allocate device memory -- code running inside a host framework
// that owns all device allocations (a fixed memory pool, an embedded or real-time host
// that forbids allocation after start-up, a caller holding a CUDA stream capture open).
// Everything that pmg_apply keeps in a handle (geometry factors, sigma table, slab-edge
// exchange buffers) lives here in one file-scope device array instead.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "host_basis.h"
#include "pmg.h"
#include "pmg_kernels.h"

namespace pmg {
int init_constants_for_device(int dev);
void set_last_error(const char* msg);
}  // namespace pmg

using namespace pmg;

namespace {

// The static scratch: 4 MiB, held by every GPU that loads the library until exit.
constexpr size_t kScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device (host code may not use the symbol
// itself as a pointer: it is a host-side stand-in).
std::mutex g_mu;
void* g_scratch_ptr[64] = {};
double g_nodes[MAXP + 1][MAXP + 1];  // LGL nodes per order, filled by the first set-up
bool g_nodes_ready = false;

// Once per device, with that device current: constant tables, LGL node table (once per
// process) and the device address of the static scratch.
pmg_status setup_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) {
    set_last_error("device index out of range");
    return PMG_ERR_INVALID;
  }
  if (!g_nodes_ready) {
    for (int p = 1; p <= MAXP; ++p) {
      std::vector<double> r, w;
      lgl(p, r, w);
      for (int i = 0; i <= p; ++i) g_nodes[p][i] = r[i];
    }
    g_nodes_ready = true;
  }
  if (!g_scratch_ptr[dev]) {
    if (init_constants_for_device(dev) != 0) return PMG_ERR_CUDA;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned NULL");
      return PMG_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return PMG_OK;
}

struct Nodes {
  double r[MAXP + 1];
};

__global__ void k_sigma_rows(int NZ, int P, int Nz, Nodes nodes, double* sigma) {
  int iz = blockIdx.x * blockDim.x + threadIdx.x;
  if (iz >= NZ) return;
  int ez = min(iz / P, Nz - 1), j = iz - ez * P;
  sigma[iz] = (ez + (nodes.r[j] + 1.0) / 2.0) / Nz;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The call reads nothing back, so a depth d = eta + h that is not positive and finite
// (flagged by the geometry kernel in *status) is reported in the output: every entry of y
// becomes NaN.
__global__ void k_poison_on_bad_geometry(const int* status, double* y, size_t n) {
  if (*status == 0) return;
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = nan;
}

}  // namespace

extern "C" pmg_status pmg_apply_noalloc(const pmg_mesh_desc* mesh, const double* eta_dev, const double* x_dev,
                                        double* y_dev, void* stream) {
  if (!mesh || !eta_dev || !x_dev || !y_dev) {
    set_last_error("mesh, eta, x and y must be non-NULL");
    return PMG_ERR_INVALID;
  }
  const pmg_mesh_desc& m = *mesh;
  // the mesh rules of pmg_create (orders, cell bounds, a power-of-two periodic cells_x),
  // checked before any size is formed from the descriptor
  int nlev = 0;
  if (pmg_level_sequence(mesh, nullptr, &nlev, nullptr, nullptr) != PMG_OK) return PMG_ERR_INVALID;
  if (m.order_z != 0 && m.order_z != m.order) {
    set_last_error("pmg_apply_noalloc needs equal orders along x and sigma (order_z 0 or order)");
    return PMG_ERR_INVALID;
  }
  const size_t cx = (size_t)m.cells_x, P = (size_t)m.order;
  const size_t NZ = (size_t)m.cells_z * P + 1, NX = cx * P + (m.periodic_x ? 0 : 1);
  // scratch layout: [geometry status][column factors][sigma][edge counters][edge buffers]
  const size_t nedges = cx + 1;
  const size_t off_geo = 256;
  const size_t off_sig = off_geo + align256(cx * (P + 1) * 4 * sizeof(double));
  const size_t off_cnt = off_sig + align256(NZ * sizeof(double));
  const size_t off_buf = off_cnt + align256(nedges * sizeof(unsigned));
  const size_t end = off_buf + align256(nedges * NZ * sizeof(double));
  if (end > kScratchBytes) {
    set_last_error("mesh too large for pmg_apply_noalloc: its static scratch holds 4 MiB = 4194304 bytes, and the "
                   "mesh needs 256 + a(32 cells_x (order + 1)) + a(8 NZ) + a(4 (cells_x + 1)) + "
                   "a(8 (cells_x + 1) NZ) bytes, NZ = cells_z order + 1, a(n) = n rounded up to a multiple of 256 "
                   "(use pmg_apply with a handle)");
    return PMG_ERR_INVALID;
  }
  Shape F{};
  F.P = m.order;
  F.PZ = m.order;
  F.Nx = m.cells_x;
  F.Nz = m.cells_z;
  F.periodic = m.periodic_x;
  F.NX = (int)NX;
  F.NZ = (int)NZ;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_last_error("cudaGetDevice failed");
    return PMG_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  pmg_status s = setup_device(dev, &base);
  if (s != PMG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess) set_last_error(cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  // the exchange counters and buffers must start at zero (the kernel leaves them zero,
  // but an earlier call that failed part-way might not have)
  if (!ck(cudaMemsetAsync(base, 0, 256, st)) || !ck(cudaMemsetAsync(base + off_cnt, 0, end - off_cnt, st)))
    return PMG_ERR_CUDA;
  double dx = (m.x1 - m.x0) / m.cells_x, dsig = 1.0 / m.cells_z;
  double* geo = reinterpret_cast<double*>(base + off_geo);
  double* sig = reinterpret_cast<double*>(base + off_sig);
  if (!ck(geometry<double>(F, eta_dev, m.h, nullptr, dx, dsig, 0, geo, reinterpret_cast<int*>(base), st))) return PMG_ERR_CUDA;
  Nodes nodes{};
  for (int i = 0; i <= m.order; ++i) nodes.r[i] = g_nodes[m.order][i];
  k_sigma_rows<<<(F.NZ + 127) / 128, 128, 0, st>>>(F.NZ, m.order, m.cells_z, nodes, sig);
  if (!ck(cudaGetLastError())) return PMG_ERR_CUDA;
  CurvedArgs a{};
  a.s = F;
  a.mode = 0;
  a.x = x_dev;
  a.y = y_dev;
  a.geo = geo;
  a.sigma = sig;
  a.scale = 1.0;
  a.mask_input = 1;
  a.sc.edgebuf = base + off_buf;
  a.sc.edgecnt = reinterpret_cast<unsigned*>(base + off_cnt);
  if (!ck(curved_op<double>(a, st))) return PMG_ERR_CUDA;
  k_poison_on_bad_geometry<<<152, 256, 0, st>>>(reinterpret_cast<const int*>(base), y_dev, NX * NZ);
  if (!ck(cudaGetLastError())) return PMG_ERR_CUDA;
  return PMG_OK;
}
