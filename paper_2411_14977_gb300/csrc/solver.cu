// Host orchestration and C ABI of the p-multigrid-preconditioned Krylov pressure solve.
//
// Setup (pmg_create): level orders by the coarsening rule (Sec. 5.1), the flat level
// operators (Sec. 5.4: time-constant preconditioner on the linearised geometry), Schwarz
// fast-diagonalisation factors per element class (Sec. 5.3), transfer matrices
// I = Phi V^-1 (Sec. 5.2) and the coarse factor; all uploaded once.
// Solve (pmg_solve): FP64 PCG / flexible CG / defect correction on the actual-geometry
// operator with one V-cycle as preconditioner (Sec. 5, Sec. 5.4), or FP64 iterative
// refinement around an FP32 flexible-CG solve whose V-cycle runs in FP32 (coarse solve FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <set>
#include <string>
#include <vector>

#include "host_basis.h"
#include "pmg.h"
#include "pmg_kernels.h"
#include "k_levels_batch.h"

using namespace pmg;

namespace {

thread_local std::string g_err;

pmg_status fail(pmg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? PMG_ERR_OOM : PMG_ERR_CUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    }                                                                                      \
  } while (0)

#define CKS(call)                                                                          \
  do {                                                                                     \
    pmg_status s_ = (call);                                                                \
    if (s_ != PMG_OK) return s_;                                                           \
  } while (0)

struct DeviceGuard {
  int old = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&old);
    if (old != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (old >= 0 && cur != old) cudaSetDevice(old);
  }
};

std::mutex g_const_mu;
std::set<int> g_const_devices;

void fdm_class(int P, int O, int dir, int cls, double* V, double* lam, int& k);

pmg_status ensure_constants(int dev) {
  std::lock_guard<std::mutex> lk(g_const_mu);
  if (g_const_devices.count(dev)) return PMG_OK;
  static ConstTables t;
  std::memset(&t, 0, sizeof(t));
  for (int P = 1; P <= MAXP; ++P) {
    std::vector<double> x, w;
    lgl(P, x, w);
    std::vector<double> D = diff_matrix(P);
    int n = P + 1;
    for (int i = 0; i < n; ++i) {
      t.w[P][i] = w[i];
      t.wf[P][i] = (float)w[i];
      t.wd[P][i] = df64_from_double(w[i]);
      for (int m = 0; m < n; ++m) {
        t.D[P][i][m] = D[i * n + m];
        t.Df[P][i][m] = (float)D[i * n + m];
        t.Dd[P][i][m] = df64_from_double(D[i * n + m]);
        double k = 0.0;
        for (int q = 0; q < n; ++q) k += D[q * n + i] * w[q] * D[q * n + m];
        t.K[P][i][m] = k;
        t.Kf[P][i][m] = (float)k;
      }
    }
  }
  CK(init_consts_apply(&t));
  CK(init_consts_apply_tc(&t));
  CK(init_consts_levels(&t));
  CK(init_consts_stepper(&t));
  CK(init_consts_apply_bathy(&t));
  CK(init_consts_apply_aniso(&t));
  CK(init_consts_levels_aniso(&t));
  CK(init_consts_dense(&t));
  CK(init_consts_vtail(&t));
  {
    std::vector<float> tab(fdm32_table_size(), 0.f);
    for (int P = 2; P <= MAXP; ++P)
      for (int O = 0; O <= MAXO; ++O) {
        if (O > (P - 1) / 2) continue;
        int NB = P + 1 + 2 * O, off = fdm32_offset(P, O), k;
        std::vector<double> V(NB * NB), lam(NB);
        for (int dir = 0; dir < 2; ++dir)
          for (int cls = 0; cls < 4; ++cls) {
            fdm_class(P, O, dir, cls, V.data(), lam.data(), k);
            for (int i = 0; i < NB * NB; ++i) tab[off + (dir * 4 + cls) * NB * NB + i] = (float)V[i];
          }
      }
    CK(init_consts_fdm32(tab.data(), tab.size(), &t.Kf[0][0][0], sizeof(t.Kf) / sizeof(float)));
    CK(init_consts_fdm32z(tab.data(), tab.size(), &t.Kf[0][0][0], sizeof(t.Kf) / sizeof(float)));
    CK(init_consts_fdm32b(tab.data(), tab.size(), &t.Kf[0][0][0], sizeof(t.Kf) / sizeof(float)));
    CK(init_consts_vtail32(tab.data(), tab.size(), &t.Kf[0][0][0], sizeof(t.Kf) / sizeof(float)));
  }
  g_const_devices.insert(dev);
  return PMG_OK;
}

// Assembled 1D LGL stiffness entry K[a][b] of order p over ncell cells (periodic or not),
// and assembled weights.
struct Line1D {
  int p, ncell, periodic, n;  // n nodes
  std::vector<double> K1, w;  // element stiffness (p+1)^2, weights
  Line1D(int p_, int nc, int per) : p(p_), ncell(nc), periodic(per) {
    n = nc * p + (per ? 0 : 1);
    std::vector<double> x;
    lgl(p, x, w);
    std::vector<double> D = diff_matrix(p);
    K1.assign((p + 1) * (p + 1), 0.0);
    for (int i = 0; i <= p; ++i)
      for (int m = 0; m <= p; ++m) {
        double s = 0.0;
        for (int q = 0; q <= p; ++q) s += D[q * (p + 1) + i] * w[q] * D[q * (p + 1) + m];
        K1[i * (p + 1) + m] = s;
      }
  }
  int wrap(int a) const { return periodic ? ((a % n) + n) % n : a; }
  // elements (cells) containing node a, with local index
  void owners(int a, int* e, int* loc, int& cnt) const {
    cnt = 0;
    a = wrap(a);
    int c = a / p, l = a - c * p;
    if (!periodic && c == ncell) { c = ncell - 1; l = p; }
    e[cnt] = c; loc[cnt] = l; ++cnt;
    if (l == 0) {
      int cl = c - 1;
      if (periodic) cl = (cl + ncell) % ncell;
      if (cl >= 0) { e[cnt] = cl; loc[cnt] = p; ++cnt; }
    }
  }
  double K(int a, int b) const {
    int ea[2], la[2], eb[2], lb[2], na, nb;
    owners(a, ea, la, na);
    owners(b, eb, lb, nb);
    double s = 0.0;
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j)
        if (ea[i] == eb[j]) s += K1[la[i] * (p + 1) + lb[j]];
    return s;
  }
  double M(int a) const {
    int e[2], l[2], c;
    owners(a, e, l, c);
    double s = 0.0;
    for (int i = 0; i < c; ++i) s += w[l[i]];
    return s;
  }
};

// Schwarz fast-diagonalisation factors of one element class, from a canonical 1D line:
// the subdomain of an element is its P+1 node lines plus O overlap lines of each
// neighbour (clipped at walls; in z the surface line is Dirichlet and excluded).  The
// factors depend only on (P, O, direction, class): class 0 interior, 1 first element
// (wall / bottom), 2 last element (wall / surface), 3 both.  V (NB x NB, row = local
// node, column = mode, rows of absent nodes zero) satisfies V^T M V = I, V^T K V = diag.
void fdm_class(int P, int O, int dir, int cls, double* V, double* lam, int& k) {
  int NB = P + 1 + 2 * O;
  int ncell = cls == 0 ? 3 : (cls == 3 ? 1 : 2);
  int e = (cls == 0 || cls == 2) ? 1 : 0;
  Line1D line(P, ncell, 0);
  int last = line.n - 1 - (dir == 1 ? 1 : 0);
  std::vector<int> loc, glob;
  for (int a = 0; a < NB; ++a) {
    int g = e * P - O + a;
    if (g < 0 || g > last) continue;
    loc.push_back(a);
    glob.push_back(g);
  }
  k = (int)glob.size();
  std::vector<double> K(k * k), M(k), Vk, lk;
  for (int i = 0; i < k; ++i) {
    M[i] = line.M(glob[i]);
    for (int j = 0; j < k; ++j) K[i * k + j] = line.K(glob[i], glob[j]);
  }
  gen_eig_diag(k, K, M, Vk, lk);
  for (int i = 0; i < NB * NB; ++i) V[i] = 0.0;
  for (int i = 0; i < NB; ++i) lam[i] = 0.0;
  for (int i = 0; i < k; ++i)
    for (int a = 0; a < k; ++a) V[loc[i] * NB + a] = Vk[i * k + a];
  for (int a = 0; a < k; ++a) lam[a] = lk[a];
}

template <typename T>
T* upload(const std::vector<double>& v, std::vector<void*>& allocs, cudaError_t& err) {
  T* d = nullptr;
  err = cudaMalloc(&d, std::max<size_t>(1, v.size()) * sizeof(T));
  if (err != cudaSuccess) return nullptr;
  allocs.push_back(d);
  std::vector<T> h(v.begin(), v.end());
  err = cudaMemcpy(d, h.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return d;
}

}  // namespace

struct LevelDev {
  int order = 0, overlap = 0;
  int order_z = 0, overlap_z = 0;  // along sigma (equal to order / overlap unless semi-coarsened)
  bool aniso = false;              // different orders along x and sigma
  double* Jz = nullptr;            // transfer from level l+1 along sigma (J when the orders agree)
  Shape s{};
  void* mX[2]{};
  void* mZ[2]{};
  void* Vx[2]{};
  void* Vz[2]{};
  void* invden[2]{};
  void* wx[2]{};
  void* wz[2]{};
  double* J = nullptr;  // transfer from level l+1 (coarse) to this level
  int thr_flat32 = 256, thr_fdm32 = 256, thr_xfer = 256;  // CTA sizes (autotuner)
  // thr_fdm32 >= 1000: the z-split sweep with thr_fdm32 / 1000 element rows and
  // thr_fdm32 % 1000 threads per CTA
  bool fuse_res = false;  // FP32 sweeps form their own residual (autotuner, when faster)
  bool fuse_restrict = false;  // the restriction forms the level residual (autotuner, when faster)
  void* b[2]{};
  void* x[2]{};
  void* t[2]{};
  // varying still-water depth (pmg_set_bathymetry): the level keeps each node column's
  // depth and drops the bottom-slope terms; tables per element column
  bool var = false;
  void* Kx[2]{};       // [Nx][p+1][p+1] element x-stiffness (dsig/dx) D^T diag(w d) D
  void* mXd[2]{};      // [NX] (dx/dsig) sum over the column's elements of w / d
  void* Vxc[2]{};      // [Nx][NB][NB] Schwarz x-eigenvectors of each element column
  void* invdenc[2]{};  // [Nx][4][NB][NB] 1 / (lambda_x + lambda_z)
  // dense Schwarz (PMG_ASM_DENSE): subdomain inverses of the level operator and scratch
  bool dense = false;
  void* dinv[2]{};           // [Nx*Nz][NB*NB] FP64 / FP32
  void* dU[2]{};             // [Nx*Nz][NB]
  double* dgeo = nullptr;    // [Nx][P+1][4] column factors of the level operator
  double* dsig = nullptr;    // [NZ] sigma rows of the level
  // PMG_ACTUAL: the level re-discretised on the current surface
  bool actual = false;
  double* Eeta = nullptr;    // [(p+1) x (P+1)] the fine surface polynomial at this level's nodes
  double* aeta = nullptr;    // [NX] surface at this level's node columns
  void* ageo[2]{};           // [Nx][p+1][4] column factors of the level operator
  float* asig32 = nullptr;   // [NZ] sigma rows (FP32)
};

struct pmg_handle {
  pmg_mesh_desc mesh{};
  pmg_opts opts{};
  int device = 0;
  int thr_curved32 = 256, thr_curved64 = 256;  // CTA sizes of the actual-geometry operators (autotuner)
  int tc = 0;  // FP32 operator in the inner solve: 0 CUDA cores, 3 BF16 tensor cores (hi/lo split)
  bool df64_outer = false;  // outer operator in double-float arithmetic (FP64 in and out)
  double dx = 0, dsig = 0, cx = 0, cz = 0;
  size_t N = 0, Nfree = 0;
  std::vector<int> orders, orders_z;  // level orders along x and along sigma
  bool aniso = false;                 // the finest orders differ (Sec. 5.1 semi-coarsening)
  std::vector<LevelDev> lv;
  std::vector<void*> allocs;
  std::vector<double> xcols, sigrows;
  // fine geometry
  double* eta = nullptr;
  void* geo[2]{};
  double* geo_div = nullptr;
  void* sigma[2]{};
  int* status = nullptr;      // [0] inputs of the current solve, [1] geometry, [2] a bounded device wait gave up
  long long wait_cycles = kWaitCyclesDefault;  // bound of the device-side waits
  CoarseArgs coarse{};
  // FP64 Krylov vectors
  double *x = nullptr, *r = nullptr, *p = nullptr, *w = nullptr, *z = nullptr, *rold = nullptr;
  // FP32 inner vectors
  float *r32 = nullptr, *c32 = nullptr, *p32 = nullptr, *w32 = nullptr, *z32 = nullptr, *rold32 = nullptr;
  double* scal = nullptr;
  double* scal_host = nullptr;
  int* status_host = nullptr;
  double* io = nullptr;  // pmg_solve_host: out, b, p_D, x0
  double* filt = nullptr;  // (P+1)^2 nodal spectral filter, set by pmg_set_filter
  double* geo5 = nullptr;  // mixed-stage column factors [Nx][P+1][5] (pmg_set_geometry_mixed)
  double* eta_prev = nullptr;
  bool mixed_stage = false;  // the outer operator is the mixed-stage one
  // varying still-water depth h(x) (pmg_set_bathymetry)
  bool bathy = false;
  double* hcol = nullptr;    // [NX] depth per node column
  void* geo6[2]{};           // [Nx][P+1][6] column factors of the operator over it
  double* mb = nullptr;      // [NX] bottom edge weights sum_e w_i (dx/2) sqrt(1 + h_x^2)
  // flexible GMRES(m): Arnoldi basis V [(m+1) N], preconditioned directions Z [m N], device
  // coefficients (two Gram-Schmidt passes and the new norm), block partials, ticket, y
  double *gm_V = nullptr, *gm_Z = nullptr, *gm_h = nullptr, *gm_part = nullptr, *gm_y = nullptr;
  unsigned* gm_cnt = nullptr;
  Scratch sc{};
  // profiling: per-class launch counts; optional CUDA-event pairs around launches
  bool timing = false;
  int64_t launches[PMG_K_COUNT] = {};
  double bytes[PMG_K_COUNT] = {};              // algorithmic bytes moved by the launches
  double flops[PMG_K_COUNT] = {};              // algorithmic floating-point operations
  std::vector<cudaEvent_t> ev_pool;            // pairs: [2k] start, [2k+1] stop
  std::vector<std::pair<int, int>> ev_used;    // (class, pair index)
  // device-side Krylov loops: graphs with a while-node, built on first use
  cudaStream_t cap = nullptr;                  // capture stream
  int* d_iter = nullptr;                       // [2] iteration counters (FP64 loop, FP32 inner loop)
  int* iter_host = nullptr;                    // pinned copy
  struct Loop {
    cudaGraphExec_t exec = nullptr;
    int64_t init_launches[PMG_K_COUNT] = {};   // kernels of the first iteration
    int64_t body_launches[PMG_K_COUNT] = {};   // kernels of every further iteration
    double init_bytes[PMG_K_COUNT] = {}, body_bytes[PMG_K_COUNT] = {};
    double init_flops[PMG_K_COUNT] = {}, body_flops[PMG_K_COUNT] = {};
  } loop64, loop32, loop_gm, loop_pdc;
  bool loop_gm_mix = false, loop_pdc_mix = false;  // operator kind the loop captured (mixed-stage or not)
  double* gm_state = nullptr;  // device GMRES cycle: H [(m+1) m], cs [m], sn [m], g [m+1]
  int* gm_ctr = nullptr;       // device GMRES cycle: j, iteration cap
  double* b_copy = nullptr;    // right-hand side captured by the PDC loop
  // fused coarse V-cycle (k_vtail.cu): the FP32 V-cycle from level vt_l0 down to the coarse
  // solve and back up in one cooperative launch
  int vt_l0 = -1;              // first fused level (-1: the levels do not qualify)
  bool vt_on = false;          // the FP32 V-cycle uses the fused launch
  void* vt_tab = nullptr;      // device step table (in allocs)
  unsigned* vt_bar = nullptr;  // [2] grid barrier words (arrivals, abort)
  size_t vt_smem = 0;
  int vt_threads = 128, vt_per_sm = 2, vt_sms = 0;
  float vt_us[2] = {0.f, 0.f};  // pmg_autotune: FP32 V-cycle microseconds without / with it
  std::vector<VtStep>* rec = nullptr;  // while set, level steps are recorded here, not launched
  bool rec_ok = true;          // every recorded step is of a form the fused kernel runs
  double rec_bytes = 0, rec_flops = 0;  // algorithmic cost of the recorded steps
  double vt_bytes = 0, vt_flops = 0;    // ... of the fused launch

  template <typename T> T* alloc(size_t n, cudaError_t& e) {
    T* d = nullptr;
    e = cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) allocs.push_back(d);
    return d;
  }
  ~pmg_handle() {
    for (Loop* l : {&loop64, &loop32, &loop_gm, &loop_pdc})
      if (l->exec) cudaGraphExecDestroy(l->exec);
    if (cap) cudaStreamDestroy(cap);
    if (iter_host) cudaFreeHost(iter_host);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (void* a : allocs) cudaFree(a);
    if (scal_host) cudaFreeHost(scal_host);
    if (status_host) cudaFreeHost(status_host);
  }
};

namespace {

template <typename T> constexpr int PI = std::is_same<T, double>::value ? 0 : 1;

// Every kernel launch goes through here: counts it under its class and, when timing is
// on, brackets it with a pair of CUDA events on the launching stream.
// Algorithmic cost of a launch, for the roofline: bytes that must cross DRAM at least
// once and floating-point operations (an FMA counts 2).
struct Cost {
  double bytes = 0, flops = 0;
};

template <class F>
pmg_status launch(pmg_handle* h, int cls, int nkernels, cudaStream_t st, Cost c, F&& f) {
  h->launches[cls] += nkernels;
  h->bytes[cls] += c.bytes;
  h->flops[cls] += c.flops;
  int pair = -1;
  if (h->timing) {
    pair = (int)h->ev_used.size();
    if ((size_t)(2 * pair + 2) > h->ev_pool.size()) {
      for (int k = 0; k < 512; ++k) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->ev_pool.push_back(e);
      }
    }
    CK(cudaEventRecord(h->ev_pool[2 * pair], st));
  }
  CK(f());
  if (pair >= 0) {
    CK(cudaEventRecord(h->ev_pool[2 * pair + 1], st));
    h->ev_used.push_back({cls, pair});
  }
  return PMG_OK;
}
template <class F>
pmg_status launch(pmg_handle* h, int cls, int nkernels, cudaStream_t st, F&& f) {
  return launch(h, cls, nkernels, st, Cost{}, f);
}

// ---- setup helpers -----------------------------------------------------------------
// Dense Schwarz tables of level l (PMG_ASM_DENSE): the level operator's column factors
// (flat: depth dl per node column of the level, or the constant depth; no slope terms),
// its sigma rows, and the subdomain inverses built on the device.
pmg_status build_level_dense(pmg_handle* h, int l, const std::vector<double>* dl) {
  LevelDev& L = h->lv[l];
  const pmg_mesh_desc& m = h->mesh;
  const int p = L.order, pz = L.order_z, n = p + 1;
  std::vector<double> xg, w, zg, wzv;
  lgl(p, xg, w);
  lgl(pz, zg, wzv);
  std::vector<double> geo((size_t)m.cells_x * n * 4, 0.0), sig(L.s.NZ);
  Line1D lx(p, m.cells_x, m.periodic_x);
  for (int ex = 0; ex < m.cells_x; ++ex)
    for (int i = 0; i < n; ++i) {
      const double d = dl ? (*dl)[lx.wrap(ex * p + i)] : m.h;
      double* g = &geo[((size_t)ex * n + i) * 4];
      g[0] = w[i] * d * h->dsig / h->dx;
      g[2] = w[i] * (h->dx / h->dsig) / d;
    }
  for (int iz = 0; iz < L.s.NZ; ++iz) {
    int ez = std::min(iz / pz, m.cells_z - 1), j = iz - ez * pz;
    sig[iz] = (ez + (zg[j] + 1.0) / 2.0) * h->dsig;
  }
  cudaError_t e = cudaSuccess;
  const size_t E = (size_t)m.cells_x * m.cells_z, nb2 = dense_block_elems(L.s, L.overlap, L.overlap_z);
  const size_t nb = (size_t)(p + 1 + 2 * L.overlap) * (pz + 1 + 2 * L.overlap_z);
  if (!L.dinv[0]) {
    L.dinv[0] = h->alloc<double>(E * nb2, e); CK(e);
    L.dinv[1] = h->alloc<float>(E * nb2, e); CK(e);
    L.dU[0] = h->alloc<double>(E * nb, e); CK(e);
    L.dU[1] = h->alloc<float>(E * nb, e); CK(e);
    L.dgeo = h->alloc<double>(geo.size(), e); CK(e);
    L.dsig = h->alloc<double>(sig.size(), e); CK(e);
  }
  CK(cudaMemcpy(L.dgeo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.dsig, sig.data(), sig.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(dense_setup(L.s, L.overlap, L.overlap_z, L.dgeo, L.dsig, (double*)L.dinv[0], (float*)L.dinv[1], nullptr));
  CK(cudaDeviceSynchronize());
  L.dense = true;
  L.fuse_res = false;
  L.fuse_restrict = false;
  return PMG_OK;
}

pmg_status build_level(pmg_handle* h, int l) {
  LevelDev& L = h->lv[l];
  const pmg_mesh_desc& m = h->mesh;
  int p = h->orders[l], pz = h->orders_z[l];
  L.order = p;
  L.order_z = pz;
  L.aniso = pz != p;
  L.fuse_res = h->opts.fuse_residual == 1 && !L.aniso;
  if (h->opts.sweep_kernel == 1) L.thr_fdm32 = 8128;  // z-split forced: 8 element rows, 128 threads
  if (sweep_code_ok(h->opts.sweep_kernel)) L.thr_fdm32 = h->opts.sweep_kernel;
  if (h->opts.flat_kernel == 1) L.thr_flat32 = -128;
  if (h->opts.flat_kernel == 2) L.thr_flat32 = 11608;  // tiled: 16 element columns x 8 rows
  if (h->opts.flat_kernel == 3) L.thr_flat32 = 1256;   // bulk-staged slab CTAs of 256 threads
  if (flat_tile_code_ok(h->opts.flat_kernel) || flat_bulk_code_ok(h->opts.flat_kernel))
    L.thr_flat32 = h->opts.flat_kernel;
  L.fuse_restrict = h->opts.fuse_residual == 1 && !L.aniso;
  L.s.P = p;
  L.s.PZ = pz;
  L.s.Nx = m.cells_x;
  L.s.Nz = m.cells_z;
  L.s.periodic = m.periodic_x;
  L.s.NX = m.cells_x * p + (m.periodic_x ? 0 : 1);
  L.s.NZ = m.cells_z * pz + 1;
  size_t NL = (size_t)L.s.NX * L.s.NZ;
  Line1D lx(p, m.cells_x, m.periodic_x), lz(pz, m.cells_z, 0);
  std::vector<double> mX(L.s.NX), mZ(L.s.NZ);
  for (int a = 0; a < L.s.NX; ++a) mX[a] = lx.M(a);
  for (int a = 0; a < L.s.NZ; ++a) mZ[a] = lz.M(a);
  cudaError_t e;
  L.mX[0] = upload<double>(mX, h->allocs, e); CK(e);
  L.mX[1] = upload<float>(mX, h->allocs, e); CK(e);
  L.mZ[0] = upload<double>(mZ, h->allocs, e); CK(e);
  L.mZ[1] = upload<float>(mZ, h->allocs, e); CK(e);
  for (int k = 0; k < 2; ++k) {
    size_t sz = k == 0 ? sizeof(double) : sizeof(float);
    for (void** v : {&L.b[k], &L.x[k], &L.t[k]}) {
      CK(cudaMalloc(v, NL * sz));
      h->allocs.push_back(*v);
      CK(cudaMemset(*v, 0, NL * sz));
    }
  }
  bool coarsest = l == (int)h->orders.size() - 1;
  if (coarsest) return PMG_OK;

  // ---- Schwarz factors (fast diagonalisation per element class), per direction with its
  // own order and overlap
  int O = (p >= 3) ? h->opts.overlap : 0;  // overlap lines of two neighbours must not meet
  int OZ = (pz >= 3) ? h->opts.overlap : 0;
  L.overlap = O;
  L.overlap_z = OZ;
  int NB = p + 1 + 2 * O, NBZ = pz + 1 + 2 * OZ;
  std::vector<double> Vx(4 * NB * NB, 0.0), Vz(4 * NBZ * NBZ, 0.0);
  std::vector<double> lamx(4 * NB, 0.0), lamz(4 * NBZ, 0.0);
  int kx[4] = {0, 0, 0, 0}, kz[4] = {0, 0, 0, 0};  // eigenpairs per class (modes >= k are padding)
  std::vector<double> wx(L.s.NX, 0.0), wz(L.s.NZ, 0.0);
  auto xsub = [&](int ex, std::vector<int>& loc, std::vector<int>& glob) {
    loc.clear(); glob.clear();
    for (int a = 0; a < NB; ++a) {
      int g = ex * p - O + a;
      if (!m.periodic_x && (g < 0 || g >= L.s.NX)) continue;
      loc.push_back(a);
      glob.push_back(lx.wrap(g));
    }
  };
  auto zsub = [&](int ez, std::vector<int>& loc, std::vector<int>& glob) {
    loc.clear(); glob.clear();
    for (int b = 0; b < NBZ; ++b) {
      int g = ez * pz - OZ + b;
      if (g < 0 || g >= L.s.NZ - 1) continue;  // Dirichlet row excluded
      loc.push_back(b);
      glob.push_back(g);
    }
  };
  std::vector<int> loc, glob;
  for (int cls = 0; cls < 4; ++cls) {
    fdm_class(p, O, 0, cls, &Vx[cls * NB * NB], &lamx[cls * NB], kx[cls]);
    fdm_class(pz, OZ, 1, cls, &Vz[cls * NBZ * NBZ], &lamz[cls * NBZ], kz[cls]);
  }
  std::vector<double> invden(16 * NB * NBZ, 0.0);
  for (int xc = 0; xc < 4; ++xc)
    for (int zc = 0; zc < 4; ++zc)
      for (int a = 0; a < NB; ++a)
        for (int b = 0; b < NBZ; ++b) {
          double la = lamx[xc * NB + a], lb = lamz[zc * NBZ + b];
          if (a < kx[xc] && b < kz[zc]) {
            double d = h->cx * la + h->cz * lb;
            invden[((xc * 4 + zc) * NB + a) * NBZ + b] = d > 0.0 ? 1.0 / d : 0.0;
          }
        }
  for (int ex = 0; ex < m.cells_x; ++ex) { xsub(ex, loc, glob); for (int g : glob) wx[g] += 1.0; }
  for (int ez = 0; ez < m.cells_z; ++ez) { zsub(ez, loc, glob); for (int g : glob) wz[g] += 1.0; }
  for (auto& v : wx) v = v > 0 ? 1.0 / v : 0.0;
  for (auto& v : wz) v = v > 0 ? 1.0 / v : 0.0;
  L.Vx[0] = upload<double>(Vx, h->allocs, e); CK(e);
  L.Vx[1] = upload<float>(Vx, h->allocs, e); CK(e);
  L.Vz[0] = upload<double>(Vz, h->allocs, e); CK(e);
  L.Vz[1] = upload<float>(Vz, h->allocs, e); CK(e);
  L.invden[0] = upload<double>(invden, h->allocs, e); CK(e);
  L.invden[1] = upload<float>(invden, h->allocs, e); CK(e);
  L.wx[0] = upload<double>(wx, h->allocs, e); CK(e);
  L.wx[1] = upload<float>(wx, h->allocs, e); CK(e);
  L.wz[0] = upload<double>(wz, h->allocs, e); CK(e);
  L.wz[1] = upload<float>(wz, h->allocs, e); CK(e);
  // transfers per direction: the coarse interpolant at the fine nodes, the identity along a
  // direction that this level step does not coarsen
  auto transfer_or_identity = [](int pc, int pf) {
    if (pc != pf) return transfer_matrix(pc, pf);
    std::vector<double> I((size_t)(pf + 1) * (pf + 1), 0.0);
    for (int i = 0; i <= pf; ++i) I[(size_t)i * (pf + 1) + i] = 1.0;
    return I;
  };
  const int pcx = h->orders[l + 1], pcz = h->orders_z[l + 1];
  L.J = upload<double>(transfer_or_identity(pcx, p), h->allocs, e); CK(e);
  if (pcz == pcx && pz == p) {
    L.Jz = L.J;
  } else {
    L.Jz = upload<double>(transfer_or_identity(pcz, pz), h->allocs, e); CK(e);
  }
  if (h->opts.smoother == PMG_ASM_DENSE) CKS(build_level_dense(h, l, nullptr));
  if (h->opts.precond_geom == PMG_ACTUAL) {
    // the surface and column factors are filled by pmg_set_geometry
    const int P = h->orders[0];
    std::vector<double> E;
    if (p == P) {
      E.assign((size_t)(P + 1) * (P + 1), 0.0);
      for (int i = 0; i <= P; ++i) E[(size_t)i * (P + 1) + i] = 1.0;
    } else {
      E = transfer_matrix(P, p);
    }
    L.Eeta = upload<double>(E, h->allocs, e); CK(e);
    L.aeta = h->alloc<double>(L.s.NX, e); CK(e);
    L.ageo[0] = h->alloc<double>((size_t)m.cells_x * (p + 1) * 4, e); CK(e);
    L.ageo[1] = h->alloc<float>((size_t)m.cells_x * (p + 1) * 4, e); CK(e);
    std::vector<double> sg(L.s.NZ), zg, wzv;
    lgl(pz, zg, wzv);
    for (int iz = 0; iz < L.s.NZ; ++iz) {
      int ez = std::min(iz / pz, m.cells_z - 1), j = iz - ez * pz;
      sg[iz] = (ez + (zg[j] + 1.0) / 2.0) * h->dsig;
    }
    L.asig32 = upload<float>(sg, h->allocs, e); CK(e);
    L.actual = true;
  }
  return PMG_OK;
}

// ---- varying still-water depth: level tables ----------------------------------------
// Element x-stiffness (dsig/dx) D^T diag(w d) D of every element column for the nodal depth
// dl of an order-p level, row-major [Nx][p+1][p+1].
std::vector<double> element_kx(int p, const Line1D& lx, const std::vector<double>& dl, double ax) {
  int n = p + 1, Nx = lx.ncell;
  std::vector<double> xg, w;
  lgl(p, xg, w);
  std::vector<double> D = diff_matrix(p);
  std::vector<double> Kx((size_t)Nx * n * n);
  for (int ex = 0; ex < Nx; ++ex)
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += D[q * n + i] * w[q] * dl[lx.wrap(ex * p + q)] * D[q * n + k];
        Kx[((size_t)ex * n + i) * n + k] = ax * s;
      }
  return Kx;
}

// Assembled entry (a, b) of the 1D x-stiffness from per-element matrices.
double kx_assembled(const Line1D& lx, const std::vector<double>& Kx, int a, int b) {
  int n = lx.p + 1;
  int ea[2], la[2], eb[2], lb[2], na, nb;
  lx.owners(a, ea, la, na);
  lx.owners(b, eb, lb, nb);
  double s = 0.0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      if (ea[i] == eb[j]) s += Kx[((size_t)ea[i] * n + la[i]) * n + lb[j]];
  return s;
}

template <typename T>
pmg_status upload_into(void*& dst, const std::vector<double>& v, pmg_handle* h) {
  cudaError_t e = cudaSuccess;
  if (!dst) {
    dst = upload<T>(v, h->allocs, e);
    CK(e);
    return PMG_OK;
  }
  std::vector<T> t(v.begin(), v.end());
  CK(cudaMemcpy(dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PMG_OK;
}

// Level l over the nodal depth dl (NX_l values): the slope-free level operator
// A = K_X[d] (x) M_Z + M_X[1/d] (x) K_Z and its Schwarz factors per element column.  The
// x-direction generalized eigenproblem of each subdomain is solved here; the z factors are
// the depth-free class factors of the constant-depth level.
pmg_status build_level_var(pmg_handle* h, int l, const std::vector<double>& dl) {
  LevelDev& L = h->lv[l];
  const pmg_mesh_desc& m = h->mesh;
  const int p = L.order, n = p + 1, Nx = m.cells_x, NX = L.s.NX;
  const double ax = h->dsig / h->dx, az = h->dx / h->dsig;
  Line1D lx(p, Nx, m.periodic_x);
  std::vector<double> Kx = element_kx(p, lx, dl, ax), mXd(NX, 0.0);
  for (int a = 0; a < NX; ++a) mXd[a] = az * lx.M(a) / dl[a];
  for (int k = 0; k < 2; ++k) {
    CKS(k == 0 ? upload_into<double>(L.Kx[0], Kx, h) : upload_into<float>(L.Kx[1], Kx, h));
    CKS(k == 0 ? upload_into<double>(L.mXd[0], mXd, h) : upload_into<float>(L.mXd[1], mXd, h));
  }
  L.var = true;
  L.fuse_res = false;
  L.fuse_restrict = false;
  if (l == (int)h->orders.size() - 1) return PMG_OK;
  const int O = L.overlap, NB = n + 2 * O;
  std::vector<double> Vz(NB * NB), lamz(4 * NB, 0.0);
  int kz[4];
  for (int cls = 0; cls < 4; ++cls) fdm_class(p, O, 1, cls, Vz.data(), &lamz[cls * NB], kz[cls]);
  std::vector<double> Vx((size_t)Nx * NB * NB, 0.0), invden((size_t)Nx * 4 * NB * NB, 0.0);
  std::vector<int> loc, glob;
  for (int ex = 0; ex < Nx; ++ex) {
    loc.clear();
    glob.clear();
    for (int a = 0; a < NB; ++a) {
      int g = ex * p - O + a;
      if (!m.periodic_x && (g < 0 || g >= NX)) continue;
      loc.push_back(a);
      glob.push_back(lx.wrap(g));
    }
    const int k = (int)glob.size();
    std::vector<double> K(k * k), M(k), Vk, lk;
    for (int i = 0; i < k; ++i) {
      M[i] = mXd[glob[i]];
      for (int j = 0; j < k; ++j) K[i * k + j] = kx_assembled(lx, Kx, glob[i], glob[j]);
    }
    gen_eig_diag(k, K, M, Vk, lk);
    for (int i = 0; i < k; ++i)
      for (int a = 0; a < k; ++a) Vx[((size_t)ex * NB + loc[i]) * NB + a] = Vk[i * k + a];
    for (int zc = 0; zc < 4; ++zc)
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < kz[zc]; ++b) {
          double d = lk[a] + lamz[zc * NB + b];
          invden[(((size_t)ex * 4 + zc) * NB + a) * NB + b] = d > 0.0 ? 1.0 / d : 0.0;
        }
  }
  CKS(upload_into<double>(L.Vxc[0], Vx, h));
  CKS(upload_into<float>(L.Vxc[1], Vx, h));
  CKS(upload_into<double>(L.invdenc[0], invden, h));
  CKS(upload_into<float>(L.invdenc[1], invden, h));
  return PMG_OK;
}

// Coarse (order 1) tables: sigma eigenmodes V (Nz x Nz) and, per mode, the PCR
// elimination factors of the x-tridiagonal system (K_X + mu_k M_X).  d1 == NULL: constant
// depth (cx K_X, cz M_X); otherwise the slope-free operator over the nodal depth d1.
void coarse_tables(pmg_handle* h, const std::vector<double>* d1, std::vector<double>& V, std::vector<double>& coef,
                   std::vector<double>& inv, int& nsteps) {
  const pmg_mesh_desc& m = h->mesh;
  int Nz = m.cells_z, NX1 = m.cells_x + (m.periodic_x ? 0 : 1);
  Line1D lx(1, m.cells_x, m.periodic_x), lz(1, m.cells_z, 0);
  std::vector<double> K(Nz * Nz), M(Nz), mu;
  for (int i = 0; i < Nz; ++i) {
    M[i] = lz.M(i);
    for (int j = 0; j < Nz; ++j) K[i * Nz + j] = lz.K(i, j);
  }
  gen_eig_diag(Nz, K, M, V, mu);
  int n = NX1;
  nsteps = 0;
  while ((1 << nsteps) < n) ++nsteps;
  std::vector<double> Kx1;
  if (d1) Kx1 = element_kx(1, lx, *d1, h->dsig / h->dx);
  auto kx = [&](int i, int j) { return d1 ? kx_assembled(lx, Kx1, i, j) : h->cx * lx.K(i, j); };
  auto mx = [&](int i) { return d1 ? (h->dx / h->dsig) * lx.M(i) / (*d1)[i] : h->cz * lx.M(i); };
  coef.assign((size_t)Nz * nsteps * n * 2, 0.0);
  inv.assign((size_t)Nz * n, 0.0);
  for (int k = 0; k < Nz; ++k) {
    std::vector<double> a(n), b(n), c(n), a2(n), b2(n), c2(n);
    for (int i = 0; i < n; ++i) {
      b[i] = kx(i, i) + mu[k] * mx(i);
      a[i] = (m.periodic_x || i > 0) ? kx(i, lx.wrap(i - 1)) : 0.0;
      c[i] = (m.periodic_x || i < n - 1) ? kx(i, lx.wrap(i + 1)) : 0.0;
    }
    int s = 1;
    for (int step = 0; step < nsteps; ++step, s <<= 1) {
      for (int i = 0; i < n; ++i) {
        int im = i - s, ip = i + s;
        bool vm = true, vp = true;
        if (m.periodic_x) { im = ((im % n) + n) % n; ip %= n; }
        else { vm = im >= 0; vp = ip < n; }
        double k1 = vm ? a[i] / b[im] : 0.0, k2 = vp ? c[i] / b[ip] : 0.0;
        a2[i] = vm ? -k1 * a[im] : 0.0;
        c2[i] = vp ? -k2 * c[ip] : 0.0;
        b2[i] = b[i] - (vm ? k1 * c[im] : 0.0) - (vp ? k2 * a[ip] : 0.0);
        coef[(((size_t)k * nsteps + step) * n + i) * 2 + 0] = k1;
        coef[(((size_t)k * nsteps + step) * n + i) * 2 + 1] = k2;
      }
      a.swap(a2); b.swap(b2); c.swap(c2);
    }
    for (int i = 0; i < n; ++i) inv[(size_t)k * n + i] = 1.0 / (m.periodic_x ? a[i] + b[i] + c[i] : b[i]);
  }
}

pmg_status build_coarse(pmg_handle* h) {
  const pmg_mesh_desc& m = h->mesh;
  int Nz = m.cells_z, NX1 = m.cells_x + (m.periodic_x ? 0 : 1);
  int n = NX1, nsteps = 0;
  std::vector<double> V, coef, inv;
  coarse_tables(h, nullptr, V, coef, inv, nsteps);
  cudaError_t e;
  h->coarse.NX1 = NX1;
  h->coarse.NZ1 = Nz + 1;
  h->coarse.periodic = m.periodic_x;
  h->coarse.nsteps = nsteps;
  h->coarse.V = upload<double>(V, h->allocs, e); CK(e);
  h->coarse.coef = upload<double>(coef, h->allocs, e); CK(e);
  h->coarse.inv = upload<double>(inv, h->allocs, e); CK(e);
  h->coarse.work = h->alloc<double>((size_t)Nz * n, e); CK(e);
  h->coarse.pcr_buf = nullptr;
  if (2 * (size_t)n * sizeof(double) > 200 * 1024) {
    h->coarse.pcr_buf = h->alloc<double>((size_t)Nz * 2 * n, e); CK(e);
  }
  return PMG_OK;
}

// ---- level operations --------------------------------------------------------------
template <typename T>
pmg_status level_residual(pmg_handle* h, int l, const void* b, const void* x, void* y, int residual,
                          cudaStream_t st) {
  LevelDev& L = h->lv[l];
  if (L.actual && h->rec) {
    h->rec_ok = false;
    return PMG_OK;
  }
  if (L.actual) {  // the actual-geometry operator at the level's order and surface
    CurvedArgs c{};
    c.s = L.s;
    c.mode = residual ? 1 : 0;
    c.x = x;
    c.b = b;
    c.y = y;
    c.geo = L.ageo[PI<T>];
    c.sigma = PI<T> ? (const void*)L.asig32 : (const void*)L.dsig;
    c.scale = 1.0;
    c.mask_input = residual ? 0 : 1;
    c.result = h->scal + SLOT_AUX + 5;
    c.sc = h->sc;
    c.threads = 256;
    double NL = (double)L.s.NX * L.s.NZ, E = (double)L.s.Nx * L.s.Nz, n = L.s.P + 1;
    Cost cc{(residual ? 3.0 : 2.0) * NL * sizeof(T), E * (8.0 * n * n * n + 12.0 * n * n)};
    return launch(h, PI<T> ? PMG_K_LEVEL32 : PMG_K_LEVEL64, 1, st, cc, [&] { return curved_op<T>(c, st); });
  }
  FlatArgs a{L.s, x, b, y, L.var ? 1.0 : h->cx, L.var ? 1.0 : h->cz, L.var ? L.mXd[PI<T>] : L.mX[PI<T>],
             L.mZ[PI<T>], residual, PI<T> ? L.thr_flat32 : 256};
  if (L.var) a.Kx = L.Kx[PI<T>];
  a.wait_cycles = h->wait_cycles;
  a.timeout_flag = h->status + 2;
  if (h->rec) {
    if (L.var || !residual) h->rec_ok = false;
    const double NR = (double)L.s.NX * L.s.NZ;
    h->rec_bytes += 3.0 * NR * sizeof(T);
    h->rec_flops += NR * (4.0 * (L.s.P + 2) + 4.0);
    VtStep v{};
    v.kind = VT_RESID;
    v.flat = a;
    h->rec->push_back(v);
    return PMG_OK;
  }
  double NL = (double)L.s.NX * L.s.NZ;
  Cost c{(residual ? 3.0 : 2.0) * NL * sizeof(T), NL * (4.0 * (L.s.P + 2) + 4.0)};
  return launch(h, PI<T> ? PMG_K_LEVEL32 : PMG_K_LEVEL64, 1, st, c, [&] { return flat_op<T>(a, st); });
}

// One Schwarz sweep xout = x + B_l r.  r given, or (FP32 with fused_b) r = fused_b - A_l x
// formed inside the sweep; xout (default: x, in place) must differ from x when fused.
template <typename T>
pmg_status level_fdm(pmg_handle* h, int l, const void* r, void* x, int post, cudaStream_t st,
                     const void* fused_b = nullptr, void* xout = nullptr, bool xzero = false) {
  LevelDev& L = h->lv[l];
  FdmArgs a{L.s, L.overlap, r, x, post, h->opts.omega, L.Vx[PI<T>], L.Vz[PI<T>], L.invden[PI<T>],
            L.wx[PI<T>], L.wz[PI<T>], h->sc, PI<T> ? L.thr_fdm32 : 256};
  a.overlap_z = L.overlap_z;
  double NL = (double)L.s.NX * L.s.NZ, E = (double)L.s.Nx * L.s.Nz;
  double NB = L.s.P + 1 + 2 * L.overlap;
  Cost c{3.0 * NL * sizeof(T), E * 2.0 * (2.0 * L.s.P * NB * NB + 2.0 * NB * NB * NB)};
  if (PI<T>) {
    a.xout = xout;
    a.xzero = xzero ? 1 : 0;
  }
  if (h->rec) {
    if (L.dense || L.var || L.aniso || fused_b || (xout && xout != x)) h->rec_ok = false;
    h->rec_bytes += c.bytes;
    h->rec_flops += c.flops;
    VtStep v{};
    v.kind = VT_SWEEP;
    v.fdm = a;
    h->rec->push_back(v);
    return PMG_OK;
  }
  if (L.dense) {
    if (fused_b || (xout && xout != x)) return fail(PMG_ERR_INVALID, "fused sweep with the dense smoother");
    return launch(h, PI<T> ? PMG_K_SMOOTH32 : PMG_K_SMOOTH64, 2, st, c, [&] {
      return dense_sweep<T>(L.s, L.overlap, L.overlap_z, (const T*)L.dinv[PI<T>], (const T*)r, (T*)x,
                            (const T*)L.wx[PI<T>], (const T*)L.wz[PI<T>], post, h->opts.omega, (T*)L.dU[PI<T>], st);
    });
  }
  if (L.var || L.aniso) {
    // per element column x-classes (varying depth) or different orders: the generic sweep
    // (tables from global memory), in place
    if (fused_b || (xout && xout != x)) return fail(PMG_ERR_INVALID, "fused sweep on this level");
    if (L.var) {
      a.Vx = L.Vxc[PI<T>];
      a.invden = L.invdenc[PI<T>];
      a.xpercol = 1;
    }
    a.threads = 256;
    return launch(h, PI<T> ? PMG_K_SMOOTH32 : PMG_K_SMOOTH64, 1, st, c, [&] { return fdm_smooth<T>(a, st); });
  }
  if (fused_b) {
    a.b = fused_b;
    a.cx = h->cx;
    a.cz = h->cz;
    a.mX = L.mX[1];
    a.mZ = L.mZ[1];
    c.flops += NL * (4.0 * (L.s.P + 2) + 4.0);
  }
  if (PI<T> && L.thr_fdm32 >= 1000) {
    // the z-split sweep (no fused residual; 16-byte aligned vectors), else slab CTAs
    FdmArgs z = a;
    z.zc = L.thr_fdm32 / 1000;
    z.threads = L.thr_fdm32 % 1000;
    z.wait_cycles = h->wait_cycles;
    z.timeout_flag = h->status + 2;
    if (fdm32z_usable(z)) a = z;
    else a.threads = 256;
  }
  return launch(h, PI<T> ? PMG_K_SMOOTH32 : PMG_K_SMOOTH64, 1, st, c,
                [&] { return PI<T> ? fdm_smooth32(a, st) : fdm_smooth<T>(a, st); });
}

// nu sweeps on A_l x = b (x updated); x_zero: x is known to be zero on entry.
// FP32: every sweep after a zero start forms its residual inside the sweep kernel and the
// iterate alternates between x and the level scratch t (t's surface row stays zero),
// arranged so that the last sweep writes x.
template <typename T>
pmg_status level_smooth(pmg_handle* h, int l, const void* b, void* x, int post, bool x_zero,
                        cudaStream_t st) {
  LevelDev& L = h->lv[l];
  const int nu = h->opts.nu;
  if (PI<T> && L.s.P >= 2 && L.fuse_res && !h->rec) {
    void* tb = L.t[1];
    void* src = (nu % 2 == 0) ? x : tb;  // buffer read by the first sweep
    if (src != x && !x_zero) {
      size_t NL = (size_t)L.s.NX * L.s.NZ;
      CK(cudaMemcpyAsync(tb, x, NL * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    for (int it = 0; it < nu; ++it) {
      void* dst = (src == x) ? tb : x;
      if (it == 0 && x_zero) CKS(level_fdm<T>(h, l, b, src, post, st, nullptr, dst, true));
      else CKS(level_fdm<T>(h, l, nullptr, src, post, st, b, dst, false));
      src = dst;
    }
    return PMG_OK;
  }
  for (int it = 0; it < nu; ++it) {
    if (it == 0 && x_zero) {
      CKS(level_fdm<T>(h, l, b, x, post, st, nullptr, nullptr, PI<T> && !L.var && !L.aniso && !L.dense));
    } else {
      CKS(level_residual<T>(h, l, b, x, L.t[PI<T>], 1, st));
      CKS(level_fdm<T>(h, l, L.t[PI<T>], x, post, st));
    }
  }
  return PMG_OK;
}

// Transfer between levels l and l+1.  Restriction with xf: restricts b - A_l xf (the
// level residual formed inside the restriction kernel; `in` = b).
template <typename T>
pmg_status transfer_op(pmg_handle* h, int l, const void* in, void* out, int restrict_, cudaStream_t st,
                       const void* xf = nullptr) {
  LevelDev& L = h->lv[l];
  TransferArgs a{L.s, h->lv[l + 1].s, in, out, L.J, L.thr_xfer};
  a.Jz = L.Jz;
  double Nf = (double)L.s.NX * L.s.NZ, Nc = (double)h->lv[l + 1].s.NX * h->lv[l + 1].s.NZ;
  double pf = L.s.P, pc = h->lv[l + 1].s.P;
  Cost c{(restrict_ ? Nf + Nc : 2.0 * Nf + Nc) * sizeof(T), 2.0 * (Nf * (pc + 1) + Nc * (pf + 1))};
  if (restrict_ && xf) {
    a.xf = xf;
    a.cx = h->cx;
    a.cz = h->cz;
    a.mX = L.mX[PI<T>];
    a.mZ = L.mZ[PI<T>];
    c.bytes += Nf * sizeof(T);
    c.flops += Nf * (4.0 * (pf + 2) + 4.0);
  }
  if (h->rec) {
    h->rec_bytes += c.bytes;
    h->rec_flops += c.flops;
    VtStep v{};
    v.kind = restrict_ ? VT_RESTRICT : VT_PROLONG;
    v.xfer = a;
    h->rec->push_back(v);
    return PMG_OK;
  }
  return launch(h, PMG_K_TRANSFER, 1, st, c, [&] { return transfer<T>(a, restrict_, st); });
}

template <typename T>
Cost coarse_cost(pmg_handle* h) {
  const CoarseArgs& c = h->coarse;
  double n1 = (double)c.NX1 * c.NZ1, nz = c.NZ1 - 1;
  double tables = nz * nz * 8.0 + nz * c.nsteps * c.NX1 * 16.0 + nz * c.NX1 * 8.0;
  return Cost{n1 * 2.0 * sizeof(T) + tables + 2.0 * nz * c.NX1 * 8.0 * 2.0,
              2.0 * (2.0 * c.NX1 * nz * nz + 2.0 * nz * c.NX1 * c.nsteps)};
}

// The fused coarse V-cycle: levels vt_l0 .. coarsest on lv[vt_l0].b[1] -> lv[vt_l0].x[1].
pmg_status vtail_run(pmg_handle* h, cudaStream_t st) {
  const int grid = h->vt_per_sm * h->vt_sms;
  return launch(h, PMG_K_VCYCLE, 1, st, Cost{h->vt_bytes, h->vt_flops}, [&] {
    return vtail_launch(h->vt_tab, grid, h->vt_threads, h->vt_smem, h->wait_cycles, st);
  });
}

template <typename T>
pmg_status vcycle(pmg_handle* h, int l, const void* b, void* x, cudaStream_t st);

// Records the FP32 V-cycle from the first level whose order (and every coarser one's) the
// fused kernel is built for, and uploads the fused kernel's step table.  Levels that do
// not qualify (varying depth, different orders, dense blocks, re-discretised levels)
// leave vt_l0 = -1 and the launch-per-step V-cycle in place.  Only the FP32 V-cycle fuses.
pmg_status vtail_setup(pmg_handle* h) {
  h->vt_l0 = -1;
  h->vt_on = false;
  if (h->vt_tab) {
    h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), h->vt_tab));
    CK(cudaFree(h->vt_tab));
    h->vt_tab = nullptr;
  }
  const int nl = (int)h->lv.size();
  if (nl < 2 || h->opts.fuse_coarse == 0) return PMG_OK;
  int l0 = nl - 1;
  while (l0 - 1 >= 1 && h->lv[l0 - 1].order <= kVtMaxP && h->lv[l0 - 1].order_z == h->lv[l0 - 1].order) --l0;
  std::vector<VtStep> steps;
  h->rec = &steps;
  h->rec_ok = true;
  h->rec_bytes = h->rec_flops = 0;
  pmg_status s = vcycle<float>(h, l0, h->lv[l0].b[1], h->lv[l0].x[1], nullptr);
  h->rec = nullptr;
  if (s != PMG_OK) return s;
  if (!h->rec_ok) return PMG_OK;
  cudaError_t e;
  if (!h->vt_bar) {
    h->vt_bar = h->alloc<unsigned>(4, e);
    CK(e);
  }
  CK(cudaMemset(h->vt_bar, 0, 4 * sizeof(unsigned)));
  void* tab = nullptr;
  size_t sm = 0;
  e = vtail_table(steps.data(), (int)steps.size(), h->coarse, h->lv[nl - 1].b[1], h->lv[nl - 1].x[1], h->vt_bar,
                  h->status + 2, &tab, &sm);
  if (e == cudaErrorInvalidValue) return PMG_OK;  // a step of another form
  CK(e);
  h->allocs.push_back(tab);
  h->vt_tab = tab;
  h->vt_smem = sm;
  h->vt_l0 = l0;
  h->vt_bytes = h->rec_bytes;
  h->vt_flops = h->rec_flops;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&h->vt_sms, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  int per_sm = 0;
  if (coop) CK(vtail_occupancy(h->vt_threads, h->vt_smem, &per_sm));
  if (per_sm < 1) {  // no cooperative launch of this kernel here
    h->vt_sms = 0;
    h->vt_l0 = -1;
    return PMG_OK;
  }
  h->vt_per_sm = std::min(per_sm, h->vt_per_sm);
  h->vt_on = h->opts.fuse_coarse == 1;
  return PMG_OK;
}

template <typename T>
pmg_status vcycle(pmg_handle* h, int l, const void* b, void* x, cudaStream_t st) {
  int nl = (int)h->lv.size();
  LevelDev& L = h->lv[l];
  size_t NL = (size_t)L.s.NX * L.s.NZ;
  if (PI<T> && !h->rec && h->vt_on && l == h->vt_l0) return vtail_run(h, st);
  if (l == nl - 1) {
    if (h->rec) {
      const Cost cc = coarse_cost<T>(h);
      h->rec_bytes += cc.bytes;
      h->rec_flops += cc.flops;
      VtStep v{};
      v.kind = VT_COARSE;
      h->rec->push_back(v);
      return PMG_OK;
    }
    return launch(h, PMG_K_COARSE, 3, st, coarse_cost<T>(h), [&] { return coarse_solve<T>(h->coarse, b, x, st); });
  }
  // x = 0 before the first sweep.  The FP32 sweep of constant-memory tables reads a zero
  // iterate as zero without loading it and writes every node below the surface row, so on
  // the handle's own level buffers (surface row zeroed at setup, never written) the clear
  // is implicit; elsewhere (the caller's level-0 output, the generic sweep) it is a memset.
  const bool implicit_zero = PI<T> && l > 0 && !L.var && !L.aniso && !L.dense;
  if (!implicit_zero && h->rec) h->rec_ok = false;
  else if (!implicit_zero) CK(cudaMemsetAsync(x, 0, NL * sizeof(T), st));
  CKS(level_smooth<T>(h, l, b, x, 0, true, st));
  LevelDev& C = h->lv[l + 1];
  if (L.fuse_restrict) {
    CKS(transfer_op<T>(h, l, b, C.b[PI<T>], 1, st, x));  // restricts b - A_l x
  } else {
    CKS(level_residual<T>(h, l, b, x, L.t[PI<T>], 1, st));
    CKS(transfer_op<T>(h, l, L.t[PI<T>], C.b[PI<T>], 1, st));
  }
  CKS(vcycle<T>(h, l + 1, C.b[PI<T>], C.x[PI<T>], st));
  CKS(transfer_op<T>(h, l, C.x[PI<T>], x, 0, st));
  CKS(level_smooth<T>(h, l, b, x, 1, false, st));
  return PMG_OK;
}

// tc: tensor-core variant of the FP32 operator (-1: the handle's, 0 CUDA cores, 1/3 BF16)
template <typename T>
pmg_status curved(pmg_handle* h, int mode, const void* x, const void* b, void* y, int mask, double* result,
                  cudaStream_t st, int tc = -1) {
  CurvedArgs a{};
  a.s = h->lv[0].s;
  a.mode = mode;
  a.x = x;
  a.b = b;
  a.y = y;
  a.geo = h->geo[PI<T>];
  a.sigma = h->sigma[PI<T>];
  a.scale = 1.0;
  a.mask_input = mask;
  a.result = result;
  a.sc = h->sc;
  a.threads = PI<T> ? h->thr_curved32 : h->thr_curved64;
  if (PI<T> && (mode == 0 || mode == 2)) a.tc = tc >= 0 ? tc : h->tc;
  if (!PI<T> && h->mixed_stage && (mode == 0 || mode == 1)) {
    a.mix = 1;
    a.geo5 = h->geo5;
  }
  if (h->bathy) {
    a.bathy = 1;
    a.geo6 = h->geo6[PI<T>];
    a.tc = 0;
  }
  const Shape& F = a.s;
  double N = (double)F.NX * F.NZ, E = (double)F.Nx * F.Nz, n = F.P + 1;
  Cost c{(mode == 1 ? 3.0 : 2.0) * N * sizeof(T), E * (8.0 * n * n * n + 12.0 * n * n)};
  if (!PI<T> && h->df64_outer && mode != 3)
    return launch(h, PMG_K_CURVED64, 1, st, c, [&] { return curved_op<df64>(a, st); });
  return launch(h, PI<T> ? PMG_K_CURVED32 : PMG_K_CURVED64, 1, st, c, [&] { return curved_op<T>(a, st); });
}

pmg_status read_scalars(pmg_handle* h, cudaStream_t st) {
  CK(cudaMemcpyAsync(h->scal_host, h->scal, SLOT_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->status_host, h->status, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->iter_host, h->d_iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PMG_OK;
}

// ---- solvers -----------------------------------------------------------------------
// r = b - A x with the surface row of x holding p_D (lifted residual), ||r||^2 -> slot
pmg_status outer_residual(pmg_handle* h, const double* b, int slot, cudaStream_t st) {
  return curved<double>(h, 1, h->x, b, h->r, 0, h->scal + slot, st);
}

// ||b~||^2: residual of the zero free guess (x0 == NULL: equals the first residual)
pmg_status lifted_norm(pmg_handle* h, const double* b, const double* pD, const double* x0, cudaStream_t st) {
  size_t N = h->N;
  int NZ = h->lv[0].s.NZ;
  if (!x0) {
    CKS(outer_residual(h, b, SLOT_BB, st));
    CK(cudaMemcpyAsync(h->scal + SLOT_RR64, h->scal + SLOT_BB, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PMG_OK;
  }
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 0.0}, [&] { return init_x(N, NZ, h->p, nullptr, pD, h->status, st); }));
  CKS(curved<double>(h, 1, h->p, b, h->w, 0, h->scal + SLOT_BB, st));
  CKS(outer_residual(h, b, SLOT_RR64, st));
  return PMG_OK;
}


// Build a graph "init; while (cond) body" where init and body are captured launch
// sequences that end with the loop-condition kernel.  Launch counts seen during capture
// are moved from the live counters into the loop's per-replay tallies.
template <class Init, class Body>
pmg_status build_loop(pmg_handle* h, pmg_handle::Loop& L, Init&& init, Body&& body) {
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  bool timing = h->timing;
  h->timing = false;
  struct Restore { pmg_handle* h; bool t; ~Restore() { h->timing = t; } } restore{h, timing};
  int64_t snap[PMG_K_COUNT];
  double snapb[PMG_K_COUNT], snapf[PMG_K_COUNT];
  std::memcpy(snap, h->launches, sizeof(snap));
  std::memcpy(snapb, h->bytes, sizeof(snapb));
  std::memcpy(snapf, h->flops, sizeof(snapf));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  struct GraphDel { cudaGraph_t g; ~GraphDel() { if (g) cudaGraphDestroy(g); } } del{g};
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
  cudaGraph_t out = nullptr;
  CK(cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pmg_status s = init(h->cap, hc);
  cudaError_t e = cudaStreamEndCapture(h->cap, &out);
  if (s != PMG_OK) return s;
  CK(e);
  for (int k = 0; k < PMG_K_COUNT; ++k) {
    L.init_launches[k] = h->launches[k] - snap[k]; h->launches[k] = snap[k];
    L.init_bytes[k] = h->bytes[k] - snapb[k]; h->bytes[k] = snapb[k];
    L.init_flops[k] = h->flops[k] - snapf[k]; h->flops[k] = snapf[k];
  }
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn), leaves;
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (cudaGraphNode_t nd : nodes) {
    size_t k = 0;
    CK(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &k));
    if (k == 0) leaves.push_back(nd);
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  CK(cudaGraphAddNode(&cn, g, leaves.data(), nullptr, leaves.size(), &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(h->cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  s = body(h->cap, hc);
  e = cudaStreamEndCapture(h->cap, &out);
  if (s != PMG_OK) return s;
  CK(e);
  for (int k = 0; k < PMG_K_COUNT; ++k) {
    L.body_launches[k] = h->launches[k] - snap[k]; h->launches[k] = snap[k];
    L.body_bytes[k] = h->bytes[k] - snapb[k]; h->bytes[k] = snapb[k];
    L.body_flops[k] = h->flops[k] - snapf[k]; h->flops[k] = snapf[k];
  }
  CK(cudaGraphInstantiate(&L.exec, g, 0));
  return PMG_OK;
}

// Run a built loop; returns the iterations it made (after a stream sync).
pmg_status run_loop(pmg_handle* h, pmg_handle::Loop& L, int which, cudaStream_t st, int* iters) {
  CK(cudaGraphLaunch(L.exec, st));
  CKS(read_scalars(h, st));
  int it = h->iter_host[which];
  int extra = std::max(0, it - 1);
  for (int k = 0; k < PMG_K_COUNT; ++k) {
    h->launches[k] += L.init_launches[k] + (int64_t)extra * L.body_launches[k];
    h->bytes[k] += L.init_bytes[k] + extra * L.body_bytes[k];
    h->flops[k] += L.init_flops[k] + extra * L.body_flops[k];
  }
  *iters = it;
  return PMG_OK;
}


// FP64 PCG / flexible CG iteration sequence (first: p = z instead of the beta update).
// A mixed-precision V-cycle is not exactly linear, so it always runs as flexible CG.
// z = B r, then <r, z> (and <r_old, z> when flexible) and p = z + beta p (p = z when
// `first`).  Mixed precision: the FP32 V-cycle reads the FP32 copy of r that the previous
// update wrote (made here when `first`), and its FP32 output feeds the inner products and
// the direction update directly (exact widening), so no cast kernels run in the loop.
pmg_status precondition_dir(pmg_handle* h, bool first, int flexible, cudaStream_t st) {
  const size_t N = h->N;
  double* s = h->scal + GROUP_OUTER;
  const double* ro = (flexible && !first) ? h->rold : nullptr;
  if (h->opts.precision == PMG_FP64) {
    CKS(vcycle<double>(h, 0, h->r, h->z, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 8, 4.0 * N}, [&] { return rz<double>(N, h->r, h->z, ro, s, h->sc, st); }));
    return launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 8, 2.0 * N}, [&] { return p_update<double>(N, h->p, h->z, s, flexible, first ? 1 : 0, st); });
  }
  if (first) CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 0.0}, [&] { return cast_f32(N, h->r, h->r32, st); }));
  CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 8 - 4.0 * N, 4.0 * N}, [&] { return rz<double, float>(N, h->r, h->z32, ro, s, h->sc, st); }));
  return launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 8 - 4.0 * N, 2.0 * N}, [&] { return p_update<double, float>(N, h->p, h->z32, s, flexible, first ? 1 : 0, st); });
}

pmg_status cg64_step(pmg_handle* h, bool first, cudaStream_t st, cudaGraphConditionalHandle hc) {
  size_t N = h->N;
  double* s = h->scal + GROUP_OUTER;
  int flexible = h->opts.outer == PMG_FCG || h->opts.precision != PMG_FP64;
  if (first) CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), st));
  const bool mixed = h->opts.precision != PMG_FP64;
  CKS(precondition_dir(h, first, flexible, st));
  CKS(curved<double>(h, 2, h->p, nullptr, h->w, 1, s + SLOT_PAP, st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{7.0 * N * 8 + (mixed ? 4.0 * N : 0.0), 6.0 * N}, [&] {
    return cg_update<double>(N, h->x, h->r, h->p, h->w, flexible ? h->rold : nullptr, s, h->sc, st,
                             mixed ? h->r32 : nullptr);
  }));
  const double tol2 = h->opts.tol * h->opts.tol;
  return launch(h, PMG_K_VECTOR, 1, st, [&] { return loop_cond(hc, s, h->scal + SLOT_BB, tol2, h->d_iter, h->opts.max_iter, st); });
}

// FP32 inner flexible-CG iteration sequence on A c = r32 (c = 0 at the start).
pmg_status cg32_step(pmg_handle* h, bool first, cudaStream_t st, cudaGraphConditionalHandle hc) {
  size_t N = h->N;
  double* s = h->scal + GROUP_INNER;
  if (first) {
    CK(cudaMemsetAsync(h->d_iter + 1, 0, sizeof(int), st));
    CK(cudaMemsetAsync(h->c32, 0, N * sizeof(float), st));
  }
  CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
  const float* ro = first ? nullptr : h->rold32;
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 4.0 * N}, [&] { return rz<float>(N, h->r32, h->z32, ro, s, h->sc, st); }));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 2.0 * N}, [&] { return p_update<float>(N, h->p32, h->z32, s, 1, first ? 1 : 0, st); }));
  CKS(curved<float>(h, 2, h->p32, nullptr, h->w32, 1, s + SLOT_PAP, st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{7.0 * N * 4, 6.0 * N}, [&] { return cg_update<float>(N, h->c32, h->r32, h->p32, h->w32, h->rold32, s, h->sc, st); }));
  const double itol2 = h->opts.inner_tol * h->opts.inner_tol;
  return launch(h, PMG_K_VECTOR, 1, st, [&] { return loop_cond(hc, s, nullptr, itol2, h->d_iter + 1, h->opts.inner_max, st); });
}

pmg_status solve_krylov64_graph(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  const double tol2 = h->opts.tol * h->opts.tol;
  double bb = h->scal_host[SLOT_BB];
  if (h->scal_host[SLOT_RR64] <= tol2 * bb) {
    if (info) info->iterations = 0;
    return PMG_OK;
  }
  if (!h->loop64.exec)
    CKS(build_loop(h, h->loop64, [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return cg64_step(h, true, cs, hc); },
                   [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return cg64_step(h, false, cs, hc); }));
  int total = 0;
  while (total < h->opts.max_iter) {
    int it = 0;
    CKS(run_loop(h, h->loop64, 0, st, &it));
    total += it;
    double rr = h->scal_host[GROUP_OUTER + SLOT_RR];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    // confirm with the true residual; restart from it on drift
    CKS(outer_residual(h, b, SLOT_RR64, st));
    CKS(read_scalars(h, st));
    if (h->scal_host[SLOT_RR64] <= tol2 * bb) break;
  }
  if (info) info->iterations = total;
  return PMG_OK;
}

pmg_status solve_refine_graph(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  size_t N = h->N;
  const double tol2 = h->opts.tol * h->opts.tol;
  double bb = h->scal_host[SLOT_BB];
  if (!h->loop32.exec)
    CKS(build_loop(h, h->loop32, [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return cg32_step(h, true, cs, hc); },
                   [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return cg32_step(h, false, cs, hc); }));
  int outer = 0, inner_total = 0;
  while (outer < h->opts.max_iter) {
    double rr = h->scal_host[SLOT_RR64];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 * bb) break;
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 1.0 * N}, [&] { return to_f32_scaled(N, h->r, h->r32, h->scal, SLOT_RR64, st); }));
    int it = 0;
    CKS(run_loop(h, h->loop32, 1, st, &it));
    inner_total += it;
    if (!std::isfinite(h->scal_host[GROUP_INNER + SLOT_RR])) return fail(PMG_ERR_NONFINITE, "non-finite inner residual");
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{20.0 * N, 2.0 * N}, [&] { return add_f32_scaled(N, h->x, h->c32, h->scal, SLOT_RR64, st); }));
    ++outer;
    CKS(outer_residual(h, b, SLOT_RR64, st));
    CKS(read_scalars(h, st));
  }
  if (info) {
    info->iterations = outer;
    info->inner_iterations = inner_total;
  }
  return PMG_OK;
}

pmg_status solve_krylov64(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  // PCG (or flexible CG) on A_FF with the FP64 V-cycle; x, r = b~ - A x already set.
  size_t N = h->N;
  double* s = h->scal + GROUP_OUTER;
  const double tol2 = h->opts.tol * h->opts.tol;
  int flexible = h->opts.outer == PMG_FCG || h->opts.precision != PMG_FP64;
  double bb = h->scal_host[SLOT_BB];
  int it = 0;
  bool restart = true;
  if (h->scal_host[SLOT_RR64] <= tol2 * bb) {  // the initial guess already meets the tolerance
    if (info) info->iterations = 0;
    return PMG_OK;
  }
  while (it < h->opts.max_iter) {
    const bool mixed = h->opts.precision != PMG_FP64;
    if (restart) {
      CKS(precondition_dir(h, true, flexible, st));
      restart = false;
    }
    CKS(curved<double>(h, 2, h->p, nullptr, h->w, 1, s + SLOT_PAP, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{7.0 * N * 8 + (mixed ? 4.0 * N : 0.0), 6.0 * N}, [&] {
      return cg_update<double>(N, h->x, h->r, h->p, h->w, flexible ? h->rold : nullptr, s, h->sc, st,
                               mixed ? h->r32 : nullptr);
    }));
    ++it;
    CKS(read_scalars(h, st));
    double rr = h->scal_host[GROUP_OUTER + SLOT_RR];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 * bb) {
      // confirm with the true residual; restart on drift
      CKS(outer_residual(h, b, SLOT_RR64, st));
      CKS(read_scalars(h, st));
      if (h->scal_host[SLOT_RR64] <= tol2 * bb) break;
      restart = true;
      continue;
    }
    CKS(precondition_dir(h, false, flexible, st));
  }
  if (info) info->iterations = it;
  return PMG_OK;
}

// z = B v with the handle's V-cycle (FP32 V-cycle on the rounded vector when mixed)
pmg_status precondition_vec(pmg_handle* h, const double* v, double* z, cudaStream_t st) {
  size_t N = h->N;
  if (h->opts.precision == PMG_FP64) return vcycle<double>(h, 0, v, z, st);
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 0.0}, [&] { return cast_f32(N, v, h->r32, st); }));
  CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
  return launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 0.0}, [&] { return cast_f64(N, h->z32, z, st); });
}

// Flexible GMRES(m) with right preconditioning by the V-cycle (Sec. 5.4's GMRES-MG on the
// same-stage operator): Arnoldi by classical Gram-Schmidt applied twice (device multi-dot
// and multi-axpy kernels), the Hessenberg least-squares problem by Givens rotations on the
// host (one synchronisation per iteration), x += Z y at the end of a cycle, the true FP64
// residual at every restart.
pmg_status solve_gmres(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  const size_t N = h->N;
  const int m = h->opts.gmres_restart;
  const double tol2 = h->opts.tol * h->opts.tol * h->scal_host[SLOT_BB];
  double* V = h->gm_V;
  double* Z = h->gm_Z;
  double* hd = h->gm_h;  // [0, m]: first pass, [m+1, 2m+1]: second pass, [2m+2]: ||w||^2
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), col(2 * (m + 1) + 1);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  CKS(outer_residual(h, b, SLOT_RR64, st));
  CKS(read_scalars(h, st));
  int its = 0;
  while (true) {
    const double rr = h->scal_host[SLOT_RR64];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 || its >= h->opts.max_iter) break;
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{16.0 * N, 1.0 * N}, [&] { return gmres_scale(N, h->r, h->scal + SLOT_RR64, V, st); }));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = std::sqrt(rr);
    int k = 0;
    for (int j = 0; j < m && its < h->opts.max_iter; ++j) {
      double* vj = V + (size_t)j * N;
      CKS(precondition_vec(h, vj, Z + (size_t)j * N, st));
      CKS(curved<double>(h, 0, Z + (size_t)j * N, nullptr, h->w, 1, nullptr, st));
      const int nv = j + 1;
      for (int pass = 0; pass < 2; ++pass) {
        double* c = hd + pass * (m + 1);
        CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (nv + 1), 2.0 * N * nv},
                   [&] { return gmres_mdot(N, h->w, V, nv, c, h->gm_part, h->gm_cnt, st); }));
        CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (nv + 2), 2.0 * N * nv},
                   [&] { return gmres_maxpy(N, h->w, V, nv, c, -1.0, st); }));
      }
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N, 2.0 * N},
                 [&] { return dot<double, double>(N, h->w, h->w, hd + 2 * (m + 1), 0, h->sc, st); }));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{16.0 * N, 1.0 * N},
                 [&] { return gmres_scale(N, h->w, hd + 2 * (m + 1), V + (size_t)(j + 1) * N, st); }));
      CK(cudaMemcpyAsync(col.data(), hd, col.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i <= j; ++i) Hij(i, j) = col[i] + col[(m + 1) + i];
      const double hn = std::sqrt(std::max(col[2 * (m + 1)], 0.0));
      if (!std::isfinite(hn)) return fail(PMG_ERR_NONFINITE, "non-finite Arnoldi vector");
      for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
        double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), hn);
      if (!(den > 0.0)) return fail(PMG_ERR_NONFINITE, "GMRES breakdown");
      cs[j] = Hij(j, j) / den;
      sn[j] = hn / den;
      Hij(j, j) = den;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      if (g[j + 1] * g[j + 1] <= tol2 || !(hn > 0.0)) break;  // converged or lucky breakdown
    }
    for (int i = k - 1; i >= 0; --i) {  // back substitution H y = g
      double v = g[i];
      for (int l = i + 1; l < k; ++l) v -= Hij(i, l) * y[l];
      y[i] = v / Hij(i, i);
    }
    CK(cudaMemcpyAsync(h->gm_y, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (k + 2), 2.0 * N * k},
               [&] { return gmres_maxpy(N, h->x, Z, k, h->gm_y, 1.0, st); }));
    CKS(outer_residual(h, b, SLOT_RR64, st));
    CKS(read_scalars(h, st));
  }
  if (info) info->iterations = its;
  return PMG_OK;
}

// One device-side Arnoldi step of flexible GMRES (the body of the cycle's while-node): the
// V-cycle on V_j (read through the device index j into fixed buffers), Z_j, w = A Z_j, two
// classical Gram-Schmidt passes and the new basis vector, then the Givens update of the
// Hessenberg column and the loop condition (k_gm_givens).
pmg_status gmres_step(pmg_handle* h, cudaStream_t st, cudaGraphConditionalHandle hc) {
  const size_t N = h->N;
  const int m = h->opts.gmres_restart;
  const bool fp64 = h->opts.precision == PMG_FP64;
  double* V = h->gm_V;
  double* Z = h->gm_Z;
  double* hd = h->gm_h;
  int* jd = h->gm_ctr;
  double* H = h->gm_state;
  double *cs = H + (size_t)(m + 1) * m, *sn = cs + m, *g = sn + m;
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{16.0 * N, 0.0},
             [&] { return gmres_gather(N, V, jd, fp64 ? h->p : nullptr, fp64 ? nullptr : h->r32, st); }));
  if (fp64) CKS(vcycle<double>(h, 0, h->p, h->z, st));
  else CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{(fp64 ? 16.0 : 20.0) * N, 0.0},
             [&] { return gmres_scatter(N, fp64 ? h->z : nullptr, fp64 ? nullptr : h->z32, Z, jd, fp64 ? nullptr : h->z, st); }));
  CKS(curved<double>(h, 0, h->z, nullptr, h->w, 1, nullptr, st));
  for (int pass = 0; pass < 2; ++pass) {
    double* c = hd + pass * (m + 1);
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (m / 2 + 1), 2.0 * N * (m / 2)},
               [&] { return gmres_mdot(N, h->w, V, 0, c, h->gm_part, h->gm_cnt, st, jd); }));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (m / 2 + 2), 2.0 * N * (m / 2)},
               [&] { return gmres_maxpy(N, h->w, V, 0, c, -1.0, st, jd, 1); }));
  }
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N, 2.0 * N},
             [&] { return dot<double, double>(N, h->w, h->w, hd + 2 * (m + 1), 0, h->sc, st); }));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{16.0 * N, 1.0 * N},
             [&] { return gmres_scale(N, h->w, hd + 2 * (m + 1), V, st, jd); }));
  const double tol2 = h->opts.tol * h->opts.tol;
  return launch(h, PMG_K_VECTOR, 1, st, [&] {
    return gmres_givens(hc, hd, hd + (m + 1), hd + 2 * (m + 1), H, cs, sn, g, m, jd, jd + 1, h->d_iter, tol2,
                        h->scal + SLOT_BB, h->scal + SLOT_GM_RES, st);
  });
}

// Flexible GMRES(m) with the cycle on the device: one graph launch (a while-node over
// gmres_step) per restart cycle, then y = H^-1 g and x += Z y on the device and the true
// FP64 residual; the host reads the scalars once per cycle.  The loop is rebuilt only when
// the operator kind (mixed-stage or not) changes.
pmg_status solve_gmres_graph(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  const size_t N = h->N;
  const int m = h->opts.gmres_restart;
  const double tol2 = h->opts.tol * h->opts.tol * h->scal_host[SLOT_BB];
  double* H = h->gm_state;
  double* g = H + (size_t)(m + 1) * m + 2 * m;
  CKS(outer_residual(h, b, SLOT_RR64, st));
  CKS(read_scalars(h, st));
  if (h->loop_gm.exec && h->loop_gm_mix != h->mixed_stage) {
    cudaGraphExecDestroy(h->loop_gm.exec);
    h->loop_gm.exec = nullptr;
  }
  if (!h->loop_gm.exec) {
    CKS(build_loop(h, h->loop_gm, [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return gmres_step(h, cs, hc); },
                   [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return gmres_step(h, cs, hc); }));
    h->loop_gm_mix = h->mixed_stage;
  }
  int total = 0;
  while (true) {
    const double rr = h->scal_host[SLOT_RR64];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 || total >= h->opts.max_iter) break;
    const int cap = std::min(m, h->opts.max_iter - total);
    CKS(launch(h, PMG_K_VECTOR, 1, st, [&] { return gmres_init(h->scal + SLOT_RR64, g, m, h->gm_ctr, h->gm_ctr + 1, cap, h->d_iter, st); }));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{16.0 * N, 1.0 * N}, [&] { return gmres_scale(N, h->r, h->scal + SLOT_RR64, h->gm_V, st); }));
    int it = 0;
    CKS(run_loop(h, h->loop_gm, 0, st, &it));
    total += it;
    if (h->scal_host[SLOT_GM_BREAK] != 0.0) return fail(PMG_ERR_NONFINITE, "GMRES breakdown");
    CKS(launch(h, PMG_K_VECTOR, 1, st, [&] { return gmres_backsub(H, g, h->gm_y, m, h->gm_ctr, st); }));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N * (it + 2), 2.0 * N * it},
               [&] { return gmres_maxpy(N, h->x, h->gm_Z, 0, h->gm_y, 1.0, st, h->gm_ctr, 0); }));
    CKS(outer_residual(h, b, SLOT_RR64, st));
    CKS(read_scalars(h, st));
  }
  if (info) info->iterations = total;
  return PMG_OK;
}

// PDC with the loop on the device: x <- x + B r and the true residual r = b~ - A x per
// iteration inside one while-node (the right-hand side is copied into the handle so the
// captured residual kernel does not depend on the caller's buffer).
pmg_status pdc_step(pmg_handle* h, bool first, cudaStream_t st, cudaGraphConditionalHandle hc) {
  const size_t N = h->N;
  if (first) CK(cudaMemsetAsync(h->d_iter, 0, sizeof(int), st));
  if (h->opts.precision == PMG_FP64) {
    CKS(vcycle<double>(h, 0, h->r, h->z, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 1.0 * N}, [&] { return add<double>(N, h->x, h->z, st); }));
  } else {
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 1.0 * N}, [&] { return to_f32_scaled(N, h->r, h->r32, h->scal, SLOT_RR64, st); }));
    CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{20.0 * N, 2.0 * N}, [&] { return add_f32_scaled(N, h->x, h->z32, h->scal, SLOT_RR64, st); }));
  }
  CKS(outer_residual(h, h->b_copy, SLOT_RR64, st));
  const double tol2 = h->opts.tol * h->opts.tol;
  return launch(h, PMG_K_VECTOR, 1, st, [&] {
    return loop_cond(hc, h->scal + SLOT_RR64, h->scal + SLOT_BB, tol2, h->d_iter, h->opts.max_iter, st);
  });
}

pmg_status solve_pdc_graph(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  const size_t N = h->N;
  const double tol2 = h->opts.tol * h->opts.tol;
  if (!h->b_copy) {
    cudaError_t e = cudaSuccess;
    h->b_copy = h->alloc<double>(N, e);
    CK(e);
  }
  CK(cudaMemcpyAsync(h->b_copy, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CKS(read_scalars(h, st));
  const double rr = h->scal_host[SLOT_RR64];
  if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
  if (rr <= tol2 * h->scal_host[SLOT_BB]) {
    if (info) info->iterations = 0;
    return PMG_OK;
  }
  if (h->loop_pdc.exec && h->loop_pdc_mix != h->mixed_stage) {
    cudaGraphExecDestroy(h->loop_pdc.exec);
    h->loop_pdc.exec = nullptr;
  }
  if (!h->loop_pdc.exec) {
    CKS(build_loop(h, h->loop_pdc, [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return pdc_step(h, true, cs, hc); },
                   [&](cudaStream_t cs, cudaGraphConditionalHandle hc) { return pdc_step(h, false, cs, hc); }));
    h->loop_pdc_mix = h->mixed_stage;
  }
  int it = 0;
  CKS(run_loop(h, h->loop_pdc, 0, st, &it));
  if (!std::isfinite(h->scal_host[SLOT_RR64])) return fail(PMG_ERR_NONFINITE, "non-finite residual");
  if (info) info->iterations = it;
  return PMG_OK;
}

pmg_status solve_pdc(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  // x <- x + B (b~ - A x) (Sec. 5.4); B = V-cycle in the handle's precision
  size_t N = h->N;
  const double tol2 = h->opts.tol * h->opts.tol;
  double bb = h->scal_host[SLOT_BB];
  int it = 0;
  while (it < h->opts.max_iter) {
    CKS(read_scalars(h, st));
    double rr = h->scal_host[SLOT_RR64];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 * bb) break;
    if (h->opts.precision == PMG_FP64) {
      CKS(vcycle<double>(h, 0, h->r, h->z, st));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 1.0 * N}, [&] { return add<double>(N, h->x, h->z, st); }));
    } else {
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 1.0 * N}, [&] { return to_f32_scaled(N, h->r, h->r32, h->scal, SLOT_RR64, st); }));
      CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{20.0 * N, 2.0 * N}, [&] { return add_f32_scaled(N, h->x, h->z32, h->scal, SLOT_RR64, st); }));
    }
    ++it;
    CKS(outer_residual(h, b, SLOT_RR64, st));
  }
  if (info) info->iterations = it;
  return PMG_OK;
}

pmg_status solve_refine(pmg_handle* h, const double* b, pmg_solve_info* info, cudaStream_t st) {
  // FP64 iterative refinement: r = b~ - A x (FP64); inner FP32 flexible CG on A c = r/||r||
  // with the FP32 V-cycle; x += ||r|| c.
  size_t N = h->N;
  const double tol2 = h->opts.tol * h->opts.tol;
  double bb = h->scal_host[SLOT_BB];
  double* s = h->scal + GROUP_INNER;
  double itol2 = h->opts.inner_tol * h->opts.inner_tol;
  int outer = 0, inner_total = 0;
  while (outer < h->opts.max_iter) {
    CKS(read_scalars(h, st));
    double rr = h->scal_host[SLOT_RR64];
    if (!std::isfinite(rr)) return fail(PMG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol2 * bb) break;
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{12.0 * N, 1.0 * N}, [&] { return to_f32_scaled(N, h->r, h->r32, h->scal, SLOT_RR64, st); }));
    CK(cudaMemsetAsync(h->c32, 0, N * sizeof(float), st));
    CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 4.0 * N}, [&] { return rz<float>(N, h->r32, h->z32, nullptr, s, h->sc, st); }));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 2.0 * N}, [&] { return p_update<float>(N, h->p32, h->z32, s, 0, 1, st); }));
    for (int j = 0; j < h->opts.inner_max; ++j) {
      CKS(curved<float>(h, 2, h->p32, nullptr, h->w32, 1, s + SLOT_PAP, st));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{7.0 * N * 4, 6.0 * N}, [&] { return cg_update<float>(N, h->c32, h->r32, h->p32, h->w32, h->rold32, s, h->sc, st); }));
      ++inner_total;
      CKS(read_scalars(h, st));
      double irr = h->scal_host[GROUP_INNER + SLOT_RR];
      if (!std::isfinite(irr)) return fail(PMG_ERR_NONFINITE, "non-finite inner residual");
      if (irr <= itol2) break;
      CKS(vcycle<float>(h, 0, h->r32, h->z32, st));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 4.0 * N}, [&] { return rz<float>(N, h->r32, h->z32, h->rold32, s, h->sc, st); }));
      CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{3.0 * N * 4, 2.0 * N}, [&] { return p_update<float>(N, h->p32, h->z32, s, 1, 0, st); }));
    }
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{20.0 * N, 2.0 * N}, [&] { return add_f32_scaled(N, h->x, h->c32, h->scal, SLOT_RR64, st); }));
    ++outer;
    CKS(outer_residual(h, b, SLOT_RR64, st));
  }
  if (info) {
    info->iterations = outer;
    info->inner_iterations = inner_total;
  }
  return PMG_OK;
}

pmg_status check_handle(const pmg_handle* h) {
  if (!h) return fail(PMG_ERR_INVALID, "null handle");
  return PMG_OK;
}

}  // namespace

namespace pmg {
// Per-order constant tables on device `dev` (used by entry points that have no handle).
int init_constants_for_device(int dev) { return ensure_constants(dev) == PMG_OK ? 0 : 1; }
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace pmg


// =====================================================================================
// Autotuner: CTA size per kernel and shape
// =====================================================================================
namespace {

enum { TK_FLAT32 = 0, TK_FDM32 = 1, TK_XFER = 2, TK_CURVED32 = 3, TK_CURVED64 = 4, TK_FLAT32V = 5,
       TK_CURVED32B = 6, TK_CURVED64B = 7, TK_VTAIL = 8, TK_COUNT = 9 };
const char* kTuneNames[] = {"flat32", "fdm32", "transfer", "curved32", "curved64", "flat32_depth", "curved32_depth",
                            "curved64_depth", "fused_vcycle"};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;  // (kernel, order, rows, columns) -> threads
bool g_tune_loaded = false;

// Optional persistent cache: JSON lines {"kernel": ..., "P": .., "NZ": .., "Nx": .., "threads": ..}
// in the file named by PMG_TUNE_CACHE.
void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("PMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char name[64];
    int P, NZ, Nx, thr;
    if (std::sscanf(line, "{\"kernel\": \"%63[^\"]\", \"P\": %d, \"NZ\": %d, \"Nx\": %d, \"threads\": %d}", name, &P,
                    &NZ, &Nx, &thr) == 5)
      for (int k = 0; k < TK_COUNT; ++k)
        if (!std::strcmp(name, kTuneNames[k])) g_tune[std::make_tuple(k, P, NZ, Nx)] = thr;
  }
  std::fclose(f);
}
void tune_cache_store(int k, int P, int NZ, int Nx, int thr) {
  const char* path = std::getenv("PMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "{\"kernel\": \"%s\", \"P\": %d, \"NZ\": %d, \"Nx\": %d, \"threads\": %d}\n", kTuneNames[k], P, NZ, Nx,
               thr);
  std::fclose(f);
}

// Device time per launch of `reps` graph-captured launches issued by run(threads).
template <class Run>
pmg_status time_launches(pmg_handle* h, Run&& run, int threads, int reps, float* us) {
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  bool timing = h->timing;
  h->timing = false;
  int64_t snap[PMG_K_COUNT];
  double sb[PMG_K_COUNT], sf[PMG_K_COUNT];
  std::memcpy(snap, h->launches, sizeof(snap));
  std::memcpy(sb, h->bytes, sizeof(sb));
  std::memcpy(sf, h->flops, sizeof(sf));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  pmg_status s = PMG_OK;
  for (int r = 0; r < reps && s == PMG_OK; ++r) s = run(threads, h->cap);
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  std::memcpy(h->launches, snap, sizeof(snap));
  std::memcpy(h->bytes, sb, sizeof(sb));
  std::memcpy(h->flops, sf, sizeof(sf));
  h->timing = timing;
  if (s != PMG_OK) { if (g) cudaGraphDestroy(g); return s; }
  CK(e);
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms = 0.f;
  cudaError_t err = cudaGraphLaunch(ge, h->cap);
  if (err == cudaSuccess) err = cudaEventRecord(e0, h->cap);
  if (err == cudaSuccess) err = cudaGraphLaunch(ge, h->cap);
  if (err == cudaSuccess) err = cudaEventRecord(e1, h->cap);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  CK(err);
  *us = 1000.f * ms / reps;
  return PMG_OK;
}

template <class Run>
pmg_status tune_one(pmg_handle* h, int kernel, int P, int NZ, Run&& run, int* out,
                    const std::vector<int>& cands = {64, 128, 192, 256, 320, 384, 512}) {
  auto key = std::make_tuple(kernel, P, NZ, h->mesh.cells_x);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { *out = it->second; return PMG_OK; }
  }
  int best = 256;
  float best_us = 1e30f;
  for (int thr : cands) {
    float us;
    CKS(time_launches(h, run, thr, 10, &us));
    if (us < best_us * 0.97f) { best_us = us; best = thr; }
  }
  *out = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  tune_cache_store(kernel, P, NZ, h->mesh.cells_x, best);
  return PMG_OK;
}

}  // namespace

// =====================================================================================
// Batches of independent problems
// =====================================================================================
struct pmg_batch {
  std::vector<pmg_handle*> h;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  // ---- the batched path: one CUDA graph whose launches each cover every problem
  struct Sub {     // one launch: the problems of one order in a stage
    int kind;      // 0 sweep, 1 level residual, 2 restriction, 3 prolongation, 4 coarse solve,
                   // 5 outer operator with <p, A p>, 6 outer residual
    int P, O;      // order and overlap of its kernel instantiation (transfers: fine and coarse order)
    int threads;   // CTA size
    void* table;   // device table
    int nctas[3];
    size_t smem;
  };
  struct Stage {   // the launches of one stage run as parallel branches of the graph
    std::vector<Sub> subs;
  };
  struct Group {   // the problems of one order: one chain of launches through an iteration
    std::vector<Sub> vdown, vup;  // V-cycle stages (one launch each), finest first / coarsest first
    Sub coarse{}, dot{}, res0{}, res{};
    void* vec = nullptr;          // vector-kernel table of the group
    int vec_ctas[VB_COUNT] = {};
  };
  bool graph_built = false, tables_built = false;
  int path = 0;                 // pmg_batch_set_path: 0 graph, 1 host-driven loop, 2 per-problem loops
  bool eager = false;           // path 1: the iteration loop driven by the host
  int* any_dev = nullptr;       // "some problem is still active", written by the confirm kernel
  int* any_host = nullptr;      // pinned copy (host-driven loop)
  std::vector<void*> dev;       // device allocations of the batched path (tables, state, copies)
  std::vector<Group> groups;
  void* vec = nullptr;          // vector-kernel table of every problem (state machine, copies)
  int vec_ctas[VB_COUNT] = {};
  BatchState state{};
  int* state_ints = nullptr;    // [5][n]
  double* state_dbl = nullptr;  // [2][n]
  BatchIO* io = nullptr;        // [n] device
  BatchIO* io_host = nullptr;   // [n] pinned
  int* st_host = nullptr;       // pinned copies of status, total
  double* dbl_host = nullptr;   // pinned copies of bb, rr64
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> aux;     // branches of a stage
  std::vector<cudaEvent_t> aux_ev;   // fork event, then one join event per branch
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_iter = 0, launches_init = 0;
  ~pmg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    for (cudaStream_t a : aux) cudaStreamDestroy(a);
    for (cudaEvent_t e : aux_ev) cudaEventDestroy(e);
    for (void* d : dev) cudaFree(d);
    if (io_host) cudaFreeHost(io_host);
    if (st_host) cudaFreeHost(st_host);
    if (dbl_host) cudaFreeHost(dbl_host);
    if (any_host) cudaFreeHost(any_host);
    for (cudaStream_t s : st) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : done) if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (pmg_handle* x : h) pmg_destroy(x);
  }
};

// Validates a mesh and options as pmg_create does and plans the level orders (Sec. 5.1:
// the coarsening rule, semi-coarsening for two orders, or the caller's list).
static pmg_status plan_levels(const pmg_mesh_desc& m, const pmg_opts& o, std::vector<int>& orders,
                              std::vector<int>& orders_z) {
  if (m.order < 1 || m.order > MAXP) return fail(PMG_ERR_INVALID, "order must be in 1..10");
  if (m.cells_x < 1 || m.cells_z < 1) return fail(PMG_ERR_INVALID, "cells must be >= 1");
  if (m.cells_x > 65535 || m.cells_z > 64) return fail(PMG_ERR_INVALID, "too many cells (cells_z <= 64)");
  if (!(m.x1 > m.x0) || !(m.h > 0.0)) return fail(PMG_ERR_INVALID, "need x1 > x0 and h > 0");
  if (m.periodic_x && (m.cells_x < 3 || (m.cells_x & (m.cells_x - 1))))
    return fail(PMG_ERR_INVALID, "periodic_x needs cells_x >= 3 and a power of two");
  if (o.precision < 0 || o.precision > PMG_MIXED_BF16) return fail(PMG_ERR_INVALID, "unsupported precision");
  if (o.precision == PMG_MIXED_BF16 && o.outer != PMG_IR)
    return fail(PMG_ERR_INVALID, "the BF16 operator runs in the inner solve of iterative refinement (outer = PMG_IR)");
  if (o.outer < PMG_PCG || o.outer > PMG_GMRES) return fail(PMG_ERR_INVALID, "bad outer method");
  if (o.outer == PMG_GMRES && (o.gmres_restart < 1 || o.gmres_restart > 60))
    return fail(PMG_ERR_INVALID, "gmres_restart must be in 1..60");
  if (o.outer == PMG_IR && o.precision == PMG_FP64)
    return fail(PMG_ERR_INVALID, "iterative refinement needs a mixed precision");
  if ((o.smoother != PMG_ASM_FDM && o.smoother != PMG_ASM_DENSE) ||
      (o.precond_geom != PMG_FLAT_LINEARISED && o.precond_geom != PMG_ACTUAL))
    return fail(PMG_ERR_INVALID, "unsupported smoother or preconditioner geometry");
  if (o.precond_geom == PMG_ACTUAL && o.smoother != PMG_ASM_DENSE)
    return fail(PMG_ERR_INVALID, "levels on the actual geometry are not separable: they need PMG_ASM_DENSE");
  if (o.precond_geom == PMG_ACTUAL && m.order_z != 0 && m.order_z != m.order)
    return fail(PMG_ERR_INVALID, "levels on the actual geometry need equal orders along x and sigma");
  if (o.overlap < 0 || o.overlap > MAXO || o.nu < 1 || !(o.omega > 0) || !(o.tol > 0) || o.max_iter < 1 ||
      o.inner_max < 1 || !(o.inner_tol > 0) || o.fuse_residual < -1 || o.fuse_residual > 1 || o.df64_outer < -1 ||
      o.df64_outer > 1 || o.flat_kernel < -1 ||
      (o.flat_kernel > 3 && !flat_tile_code_ok(o.flat_kernel) && !flat_bulk_code_ok(o.flat_kernel)) ||
      o.sweep_kernel < -1 || (o.sweep_kernel > 1 && !sweep_code_ok(o.sweep_kernel)) || o.fuse_coarse < -1 ||
      o.fuse_coarse > 1)
    return fail(PMG_ERR_INVALID, "bad solver options");
  const int order_z = m.order_z == 0 ? m.order : m.order_z;
  if (order_z < 1 || order_z > MAXP) return fail(PMG_ERR_INVALID, "order_z must be 0 or in 1..10");
  orders.clear();
  orders_z.clear();
  if (order_z != m.order) {
    // semi-coarsening (Sec. 5.1): the higher order is reduced until both match
    if (o.nlevels > 0) return fail(PMG_ERR_INVALID, "custom level orders need equal orders along x and sigma");
    if (o.precision == PMG_MIXED_BF16) return fail(PMG_ERR_INVALID, "the BF16 operator needs equal orders");
    if (!aniso_pair_supported(m.order, order_z, true))
      return fail(PMG_ERR_INVALID, "order pair not built (order_z = 8 with order 2..10 are)");
    for (auto pr : semi_coarsening_sequence(m.order, order_z)) {
      orders.push_back(pr.first);
      orders_z.push_back(pr.second);
      if (pr.first != pr.second && !aniso_pair_supported(pr.first, pr.second, false))
        return fail(PMG_ERR_INVALID, "level order pair not built");
    }
  } else if (o.nlevels > 0) {
    if (o.nlevels > 8) return fail(PMG_ERR_INVALID, "at most 8 levels");
    for (int i = 0; i < o.nlevels; ++i) orders.push_back(o.level_orders[i]);
    if (orders[0] != m.order || orders.back() != 1) return fail(PMG_ERR_INVALID, "levels must run from order to 1");
    for (size_t i = 1; i < orders.size(); ++i)
      if (orders[i] >= orders[i - 1]) return fail(PMG_ERR_INVALID, "level orders must decrease");
  } else {
    orders = coarsening_sequence(m.order);
  }
  if (orders_z.empty()) orders_z = orders;
  if (o.smoother == PMG_ASM_DENSE)
    for (size_t l = 0; l + 1 < orders.size(); ++l) {
      const int ox = orders[l] >= 3 ? o.overlap : 0, oz = orders_z[l] >= 3 ? o.overlap : 0;
      const size_t nb = (size_t)(orders[l] + 1 + 2 * ox) * (orders_z[l] + 1 + 2 * oz);
      if (nb * nb * sizeof(double) > 227 * 1024)
        return fail(PMG_ERR_INVALID, "dense Schwarz blocks too large for one CTA (order 10 with overlap 1)");
    }
  if (orders.size() < 2) return fail(PMG_ERR_INVALID, "order must be >= 2 (the coarsest level is order 1)");
  return PMG_OK;
}

// =====================================================================================
// Batched path of pmg_batch_solve: every stage of the mixed-precision flexible CG is one
// launch over the work items of all problems (their element columns or nodes), and the
// whole solve -- start, iterations, convergence checks, restarts -- is one CUDA graph with
// a device-side while node.  Levels are aligned by their distance from the order-1 level,
// so problems with fewer levels simply have no items in the top stages.
// =====================================================================================
namespace {

// The batched path covers the mixed FP32 V-cycle (fast-diagonalisation Schwarz, flat
// levels, constant depth, equal orders) under the FP64 flexible CG with the double-float
// outer operator; other options run through the concurrent per-problem path.
bool batch_eligible(const pmg_batch* B) {
  if (B->h.size() > (size_t)kMaxBatch) return false;
  for (const pmg_handle* h : B->h) {
    if (h->opts.precision != PMG_MIXED_FP32 || (h->opts.outer != PMG_PCG && h->opts.outer != PMG_FCG) ||
        !h->df64_outer || h->mixed_stage || h->bathy || h->aniso || h->tc)
      return false;
    for (const LevelDev& L : h->lv)
      if (L.var || L.aniso || L.dense || L.actual) return false;
  }
  return true;
}

template <typename T>
T* batch_alloc(pmg_batch* B, size_t n, cudaError_t& e) {
  T* d = nullptr;
  e = cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) B->dev.push_back(d);
  return d;
}

pmg_status batch_build_tables(pmg_batch* B) {
  const int n = (int)B->h.size();
  cudaError_t e;
  B->state_ints = batch_alloc<int>(B, 5 * (size_t)n, e);
  CK(e);
  B->state_dbl = batch_alloc<double>(B, 2 * (size_t)n, e);
  CK(e);
  B->io = batch_alloc<BatchIO>(B, n, e);
  CK(e);
  B->any_dev = batch_alloc<int>(B, 1, e);
  CK(e);
  CK(cudaMallocHost(&B->any_host, sizeof(int)));
  CK(cudaMemset(B->state_ints, 0, 5 * (size_t)n * sizeof(int)));
  B->state = BatchState{B->state_ints, B->state_ints + n, B->state_ints + 2 * n, B->state_ints + 3 * n,
                        B->state_ints + 4 * n, B->state_dbl, B->state_dbl + n};
  CK(cudaMallocHost(&B->io_host, n * sizeof(BatchIO)));
  CK(cudaMallocHost(&B->st_host, 2 * (size_t)n * sizeof(int)));
  CK(cudaMallocHost(&B->dbl_host, 2 * (size_t)n * sizeof(double)));
  // per-problem vector kernel arguments and outer-operator arguments
  std::vector<VecProb> vp(n);
  std::vector<CurvedArgs> dot(n), res0(n), res(n);
  // chains: the problems of one fine order (the same level orders) and one column-depth
  // class (cells_z in 1-8, 9-16, ...: a chain's slab CTAs take one thread per node row of
  // its deepest column, so shallow tanks do not run in CTAs sized for deep ones); splitting
  // an order into chains of 4 problems (more, smaller branches) measured the same
  // throughput at config 4
  constexpr int kChain = kMaxBatch;
  std::map<std::pair<int, int>, std::vector<int>> of_order;
  for (int i = 0; i < n; ++i) of_order[{B->h[i]->lv[0].order, (B->h[i]->mesh.cells_z + 7) / 8}].push_back(i);
  std::map<std::pair<int, int>, std::vector<int>> by_fine;
  for (auto& kv : of_order)
    for (size_t k = 0; k < kv.second.size(); ++k)
      by_fine[{kv.first.first, 1000 * kv.first.second + (int)(k / kChain)}].push_back(kv.second[k]);
  for (int i = 0; i < n; ++i) {
    pmg_handle* h = B->h[i];
    double* bcopy = batch_alloc<double>(B, h->N, e);
    CK(e);
    CK(cudaMemset(h->z32, 0, h->N * sizeof(float)));  // its surface row stays zero
    VecProb& q = vp[i];
    q.n = h->N;
    q.NZ = h->lv[0].s.NZ;
    q.x = h->x;
    q.r = h->r;
    q.p = h->p;
    q.w = h->w;
    q.rold = h->rold;
    q.r32 = h->r32;
    q.z32 = h->z32;
    q.s = h->scal;
    q.sc = h->sc;
    q.status = h->status;
    q.bcopy = bcopy;
    q.max_iter = h->opts.max_iter;
    q.tol2 = h->opts.tol * h->opts.tol;
    CurvedArgs a{};
    a.s = h->lv[0].s;
    a.geo = h->geo[0];
    a.sigma = h->sigma[0];
    a.scale = 1.0;
    a.sc = h->sc;
    a.mode = MODE_DOT;
    a.x = h->p;
    a.y = h->w;
    a.mask_input = 1;
    a.result = h->scal + GROUP_OUTER + SLOT_PAP;
    dot[i] = a;
    a.mode = MODE_RESIDUAL;
    a.x = h->x;
    a.b = bcopy;
    a.y = h->r;
    a.mask_input = 0;
    a.result = h->scal + SLOT_BB;
    res0[i] = a;
    a.result = h->scal + SLOT_RR64;
    res[i] = a;
  }
  CK(vec_batch_table(vp.data(), n, B->state, B->io, &B->vec, B->vec_ctas, nullptr));
  B->dev.push_back(B->vec);
  for (auto& kv : by_fine) {
    const std::vector<int>& pi = kv.second;
    const int m = (int)pi.size();
    pmg_batch::Group G;
    auto keep = [&](pmg_batch::Sub& u) { B->dev.push_back(u.table); };
    {
      std::vector<VecProb> gv;
      std::vector<CurvedArgs> d1, r0, r1;
      for (int i : pi) {
        gv.push_back(vp[i]);
        d1.push_back(dot[i]);
        r0.push_back(res0[i]);
        r1.push_back(res[i]);
      }
      CK(vec_batch_table(gv.data(), m, B->state, B->io, &G.vec, G.vec_ctas, pi.data()));
      B->dev.push_back(G.vec);
      pmg_batch::Sub u{};
      u.P = kv.first.first;
      u.threads = 256;
      u.kind = 5;
      CK(curved_batch_table(MODE_DOT, d1.data(), pi.data(), m, B->state.active, &u.table, u.nctas, &u.smem));
      keep(u);
      G.dot = u;
      u.kind = 6;
      CK(curved_batch_table(MODE_RESIDUAL, r0.data(), pi.data(), m, nullptr, &u.table, u.nctas, &u.smem));
      keep(u);
      G.res0 = u;
      CK(curved_batch_table(MODE_RESIDUAL, r1.data(), pi.data(), m, B->state.confirm, &u.table, u.nctas, &u.smem));
      keep(u);
      G.res = u;
    }
    const int D = (int)B->h[pi[0]]->lv.size() - 1;
    std::vector<std::vector<pmg_batch::Sub>> ups;
    for (int l = 0; l < D; ++l) {
      std::vector<FdmArgs> sw0, sw1, swp;
      std::vector<FlatArgs> rs;
      std::vector<TransferArgs> rt, pl;
      int O = 0, P = 0, nzmax = 1;
      for (int i : pi) {
        pmg_handle* h = B->h[i];
        LevelDev& L = h->lv[l];
        LevelDev& C = h->lv[l + 1];
        void* bl = l == 0 ? (void*)h->r32 : L.b[1];
        void* xl = l == 0 ? (void*)h->z32 : L.x[1];
        O = L.overlap;
        P = L.order;
        nzmax = std::max(nzmax, L.s.NZ);
        FdmArgs f{L.s, L.overlap, bl, xl, 0, h->opts.omega, L.Vx[1], L.Vz[1], L.invden[1], L.wx[1], L.wz[1], h->sc,
                  256};
        f.xzero = 1;
        sw0.push_back(f);
        f.r = L.t[1];
        f.xzero = 0;
        sw1.push_back(f);
        f.post = 1;
        swp.push_back(f);
        rs.push_back(FlatArgs{L.s, xl, bl, L.t[1], h->cx, h->cz, L.mX[1], L.mZ[1], 1, 256});
        TransferArgs ta{L.s, C.s, L.t[1], C.b[1], L.J, 256};
        ta.Jz = L.Jz;
        rt.push_back(ta);
        TransferArgs tp{L.s, C.s, C.x[1], xl, L.J, 256};
        tp.Jz = L.Jz;
        pl.push_back(tp);
      }
      pmg_batch::Sub s0{}, r{}, s1{}, sp{}, rst{}, prl{};
      s0.P = r.P = s1.P = sp.P = rst.P = prl.P = P;
      // slab CTAs: about one thread per node row of the deepest column; node-parallel: 256
      const int slab_thr = std::min(256, std::max(64, (nzmax + 31) / 32 * 32));
      s0.threads = s1.threads = sp.threads = rst.threads = prl.threads = slab_thr;
      r.threads = 256;
      s0.O = s1.O = sp.O = O;
      rst.O = prl.O = B->h[pi[0]]->lv[l + 1].order;  // transfers: the coarse order of the pair
      s0.kind = s1.kind = sp.kind = 0;
      r.kind = 1;
      rst.kind = 2;
      prl.kind = 3;
      CK(fdm32_batch_table(sw0.data(), pi.data(), m, B->state.active, &s0.table, s0.nctas, &s0.smem));
      keep(s0);
      CK(fdm32_batch_table(sw1.data(), pi.data(), m, B->state.active, &s1.table, s1.nctas, &s1.smem));
      keep(s1);
      CK(fdm32_batch_table(swp.data(), pi.data(), m, B->state.active, &sp.table, sp.nctas, &sp.smem));
      keep(sp);
      CK(flat_batch_table(rs.data(), pi.data(), m, B->state.active, 256, &r.table, r.nctas));
      keep(r);
      CK(transfer_batch_table(rt.data(), pi.data(), m, B->state.active, 1, &rst.table, rst.nctas, &rst.smem));
      keep(rst);
      CK(transfer_batch_table(pl.data(), pi.data(), m, B->state.active, 0, &prl.table, prl.nctas, &prl.smem));
      keep(prl);
      // down: sweep from x = 0, residual, sweep, residual, restriction
      for (const pmg_batch::Sub* u : {&s0, &r, &s1, &r, &rst}) G.vdown.push_back(*u);
      // up: prolongation, then twice (residual, adjoint sweep)
      ups.push_back({prl, r, sp, r, sp});
    }
    for (int k = (int)ups.size() - 1; k >= 0; --k) G.vup.insert(G.vup.end(), ups[k].begin(), ups[k].end());
    {
      std::vector<CoarseArgs> ca;
      std::vector<const float*> cb;
      std::vector<float*> cx;
      for (int i : pi) {
        pmg_handle* h = B->h[i];
        LevelDev& C = h->lv.back();
        ca.push_back(h->coarse);
        cb.push_back((const float*)C.b[1]);
        cx.push_back((float*)C.x[1]);
      }
      pmg_batch::Sub u{};
      u.kind = 4;
      u.threads = 256;
      CK(coarse_batch_table(ca.data(), cb.data(), cx.data(), pi.data(), m, B->state.active, &u.table, u.nctas,
                            &u.smem));
      keep(u);
      G.coarse = u;
    }
    B->groups.push_back(G);
  }
  const size_t ng = B->groups.size();
  for (size_t k = 0; k + 1 < ng; ++k) {
    cudaStream_t a;
    CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    B->aux.push_back(a);
  }
  for (size_t k = 0; k < ng; ++k) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    B->aux_ev.push_back(ev);
  }
  return PMG_OK;
}

pmg_status batch_sub(const pmg_batch::Sub& u, cudaStream_t cs) {
  switch (u.kind) {
    case 0: CK(fdm32_batch_launch(u.table, u.P, u.O, u.nctas[0], u.threads, u.smem, cs)); break;
    case 1: CK(flat_batch_launch(u.table, u.P, u.nctas[0], u.threads, cs)); break;
    case 2: CK(transfer_batch_launch_pair(u.table, 1, u.P, u.O, u.nctas[0], u.threads, u.smem, cs)); break;
    case 3: CK(transfer_batch_launch_pair(u.table, 0, u.P, u.O, u.nctas[0], u.threads, u.smem, cs)); break;
    case 4: CK(coarse_batch_launch(u.table, u.nctas, u.smem, cs)); break;
    case 5: CK(curved_batch_launch(MODE_DOT, u.table, u.P, u.nctas[0], u.threads, u.smem, cs)); break;
    default: CK(curved_batch_launch(MODE_RESIDUAL, u.table, u.P, u.nctas[0], u.threads, u.smem, cs)); break;
  }
  return PMG_OK;
}

// Runs f(group, stream) for every group as parallel branches: fork from cs, join into cs.
template <class F>
pmg_status batch_branches(pmg_batch* B, cudaStream_t cs, F&& f) {
  const size_t ng = B->groups.size();
  if (ng == 1) return f(B->groups[0], cs);
  CK(cudaEventRecord(B->aux_ev[0], cs));
  for (size_t j = 1; j < ng; ++j) {
    CK(cudaStreamWaitEvent(B->aux[j - 1], B->aux_ev[0], 0));
    CKS(f(B->groups[j], B->aux[j - 1]));
    CK(cudaEventRecord(B->aux_ev[j], B->aux[j - 1]));
  }
  CKS(f(B->groups[0], cs));
  for (size_t j = 1; j < ng; ++j) CK(cudaStreamWaitEvent(cs, B->aux_ev[j], 0));
  return PMG_OK;
}

// One iteration of the batched flexible CG: each group of one order runs its chain -- the
// V-cycle, the inner products, the direction update, the outer operator, the CG update --
// as a branch of its own; then, over every problem, the convergence test, the true residual
// of the problems that met it and the restart / finish decision.
pmg_status batch_iteration(pmg_batch* B, cudaStream_t cs, cudaGraphConditionalHandle hc, int in_graph) {
  const int n = (int)B->h.size();
  int64_t k = 0;
  CKS(batch_branches(B, cs, [&](pmg_batch::Group& G, cudaStream_t st) -> pmg_status {
    CK(vec_batch_launch(VB_CAST_FIRST, G.vec, G.vec_ctas, st));
    for (const auto& u : G.vdown) CKS(batch_sub(u, st));
    CKS(batch_sub(G.coarse, st));
    for (const auto& u : G.vup) CKS(batch_sub(u, st));
    CK(vec_batch_launch(VB_RZ, G.vec, G.vec_ctas, st));
    CK(vec_batch_launch(VB_P_UPDATE, G.vec, G.vec_ctas, st));
    CKS(batch_sub(G.dot, st));
    CK(vec_batch_launch(VB_CG_UPDATE, G.vec, G.vec_ctas, st));
    k += 6 + 3 + (int64_t)(G.vdown.size() + G.vup.size());
    return PMG_OK;
  }));
  CK(batch_cond(B->vec, n, cs));
  CKS(batch_branches(B, cs, [&](pmg_batch::Group& G, cudaStream_t st) { ++k; return batch_sub(G.res, st); }));
  CK(batch_confirm(B->vec, n, hc, in_graph, B->any_dev, cs));
  B->launches_per_iter = k + 2;
  return PMG_OK;
}

// The start of a batch solve: inputs, the lifted residual of x = (0, p_D), the initial state.
pmg_status batch_start(pmg_batch* B, cudaStream_t cs) {
  CK(vec_batch_launch(VB_INIT, B->vec, B->vec_ctas, cs));
  CKS(batch_branches(B, cs, [&](pmg_batch::Group& G, cudaStream_t st) { return batch_sub(G.res0, st); }));
  CK(batch_state_init(B->vec, (int)B->h.size(), cs));
  return PMG_OK;
}

pmg_status batch_build_graph(pmg_batch* B) {
  if (!B->tables_built) {
    CKS(batch_build_tables(B));
    B->tables_built = true;
  }
  CK(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  struct GraphDel { cudaGraph_t g; ~GraphDel() { if (g) cudaGraphDestroy(g); } } del{g};
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
  cudaGraph_t out = nullptr;
  // start: inputs, the lifted residual of x = (0, p_D), the initial state
  CK(cudaStreamBeginCaptureToGraph(B->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pmg_status s = batch_start(B, B->cap);
  cudaError_t e = cudaStreamEndCapture(B->cap, &out);
  if (s != PMG_OK) return s;
  CK(e);
  B->launches_init = 2 + (int64_t)B->groups.size();
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn), leaves;
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (cudaGraphNode_t nd : nodes) {
    size_t kk = 0;
    CK(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &kk));
    if (kk == 0) leaves.push_back(nd);
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  CK(cudaGraphAddNode(&cn, g, leaves.data(), nullptr, leaves.size(), &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(B->cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  s = batch_iteration(B, B->cap, hc, 1);
  e = cudaStreamEndCapture(B->cap, &out);
  if (s != PMG_OK) return s;
  CK(e);
  CK(cudaGraphInstantiate(&B->exec, g, 0));
  B->graph_built = true;
  return PMG_OK;
}

pmg_status batch_solve_graph(pmg_batch* B, const double* const* bv, const double* const* pdv, double* const* pout,
                             pmg_solve_info* infos, cudaStream_t cs) {
  const int n = (int)B->h.size();
  auto t0 = std::chrono::steady_clock::now();
  DeviceGuard dg(B->h[0]->device);
  if (!B->eager && !B->graph_built) CKS(batch_build_graph(B));
  if (B->eager && !B->tables_built) {
    CKS(batch_build_tables(B));
    B->tables_built = true;
  }
  for (int i = 0; i < n; ++i) B->io_host[i] = BatchIO{bv[i], pdv[i], pout[i]};
  CK(cudaMemcpyAsync(B->io, B->io_host, n * sizeof(BatchIO), cudaMemcpyHostToDevice, cs));
  if (!B->eager) {
    CK(cudaGraphLaunch(B->exec, cs));
  } else {
    // the same launches, the loop driven by the host (one synchronisation per iteration)
    CKS(batch_start(B, cs));
    int cap = 0;
    for (pmg_handle* h : B->h) cap = std::max(cap, 2 * h->opts.max_iter + 2);
    for (int it = 0; it < cap; ++it) {
      CKS(batch_iteration(B, cs, cudaGraphConditionalHandle{}, 0));
      CK(cudaMemcpyAsync(B->any_host, B->any_dev, sizeof(int), cudaMemcpyDeviceToHost, cs));
      CK(cudaStreamSynchronize(cs));
      if (!*B->any_host) break;
    }
  }
  CK(vec_batch_launch(VB_COPY_OUT, B->vec, B->vec_ctas, cs));
  CK(cudaMemcpyAsync(B->st_host, B->state.total, n * sizeof(int), cudaMemcpyDeviceToHost, cs));
  CK(cudaMemcpyAsync(B->st_host + n, B->state.status, n * sizeof(int), cudaMemcpyDeviceToHost, cs));
  CK(cudaMemcpyAsync(B->dbl_host, B->state_dbl, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, cs));
  CK(cudaStreamSynchronize(cs));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  pmg_status result = PMG_OK;
  for (int i = 0; i < n; ++i) {
    pmg_solve_info info{};
    const double bb = B->dbl_host[i], rr = B->dbl_host[n + i];
    info.iterations = B->st_host[i];
    info.rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    info.seconds = secs;
    info.status = B->st_host[n + i];
    if (info.status == PMG_OK && !(info.rel_residual <= B->h[i]->opts.tol))
      info.status = std::isfinite(info.rel_residual) ? PMG_ERR_NOT_CONVERGED : PMG_ERR_NONFINITE;
    if (info.status != PMG_OK && result == PMG_OK) {
      result = (pmg_status)info.status;
      fail(result, "a batch problem failed (see its info)");
    }
    if (infos) infos[i] = info;
  }
  return result;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

void pmg_default_opts(pmg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = PMG_FP64;
  o->outer = PMG_PCG;
  o->smoother = PMG_ASM_FDM;
  o->precond_geom = PMG_FLAT_LINEARISED;
  o->overlap = 1;
  o->nu = 2;
  o->omega = 0.8;
  o->tol = 1e-10;
  o->max_iter = 500;
  o->inner_max = 40;
  o->inner_tol = 1e-5;
  o->nlevels = 0;
  o->fuse_residual = 0;
  o->flat_kernel = -1;
  o->df64_outer = -1;
  o->gmres_restart = 30;
  o->sweep_kernel = -1;
  o->fuse_coarse = -1;
}

const char* pmg_last_error(void) { return g_err.c_str(); }

pmg_status pmg_level_sequence(const pmg_mesh_desc* mesh, const pmg_opts* opts, int* nlevels, int* orders,
                              int* orders_z) {
  if (!mesh || !nlevels) return fail(PMG_ERR_INVALID, "mesh or nlevels is NULL");
  pmg_opts o;
  if (opts) o = *opts; else pmg_default_opts(&o);
  std::vector<int> ox, oz;
  CKS(plan_levels(*mesh, o, ox, oz));
  *nlevels = (int)ox.size();
  for (size_t l = 0; l < ox.size(); ++l) {
    if (orders) orders[l] = ox[l];
    if (orders_z) orders_z[l] = oz[l];
  }
  return PMG_OK;
}

pmg_status pmg_basis_tables(int p, int pc, double* nodes, double* weights, double* D, double* J) {
  if (p < 1 || p > MAXP) return fail(PMG_ERR_INVALID, "order must be in 1..10");
  if (pc < 0 || pc > p) return fail(PMG_ERR_INVALID, "pc must be in 0..p");
  std::vector<double> x, w;
  lgl(p, x, w);
  if (nodes) std::copy(x.begin(), x.end(), nodes);
  if (weights) std::copy(w.begin(), w.end(), weights);
  if (D) {
    const std::vector<double> d = diff_matrix(p);
    std::copy(d.begin(), d.end(), D);
  }
  if (J && pc >= 1) {
    const std::vector<double> j = transfer_matrix(pc, p);
    std::copy(j.begin(), j.end(), J);
  }
  return PMG_OK;
}

pmg_status pmg_schwarz_class(int p, int o, int dir, int cls, double* V, double* lam, int* k) {
  if (p < 1 || p > MAXP || o < 0 || o > MAXO || dir < 0 || dir > 1 || cls < 0 || cls > 3)
    return fail(PMG_ERR_INVALID, "need 1 <= p <= 10, 0 <= o <= 1, dir 0 or 1 and cls 0..3");
  if (!V || !lam || !k) return fail(PMG_ERR_INVALID, "V, lam and k must not be NULL");
  fdm_class(p, o, dir, cls, V, lam, *k);
  return PMG_OK;
}

pmg_status pmg_create(const pmg_mesh_desc* mesh, const pmg_opts* opts, pmg_handle** out) {
  if (!out) return fail(PMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!mesh) return fail(PMG_ERR_INVALID, "mesh is NULL");
  pmg_opts o;
  if (opts) o = *opts; else pmg_default_opts(&o);
  const pmg_mesh_desc& m = *mesh;
  std::vector<int> orders, orders_z;
  CKS(plan_levels(m, o, orders, orders_z));
  const int order_z = orders_z[0];

  auto* h = new (std::nothrow) pmg_handle();
  if (!h) return fail(PMG_ERR_OOM, "host allocation failed");
  auto bail = [&](pmg_status s) { delete h; return s; };
  cudaGetDevice(&h->device);
  DeviceGuard dg(h->device);
  if (ensure_constants(h->device) != PMG_OK) return bail(PMG_ERR_CUDA);
  h->mesh = m;
  h->mesh.order_z = order_z;
  h->opts = o;
  h->tc = o.precision == PMG_MIXED_BF16 ? 3 : 0;
  h->df64_outer = o.df64_outer == 1 || (o.df64_outer < 0 && o.precision != PMG_FP64);
  h->orders = orders;
  h->orders_z = orders_z;
  h->aniso = order_z != m.order;
  h->dx = (m.x1 - m.x0) / m.cells_x;
  h->dsig = 1.0 / m.cells_z;
  h->cx = m.h * h->dsig / h->dx;
  h->cz = h->dx / (m.h * h->dsig);
  h->lv.resize(orders.size());
  for (size_t l = 0; l < orders.size(); ++l) {
    pmg_status s = build_level(h, (int)l);
    if (s != PMG_OK) return bail(s);
  }
  {
    pmg_status s = build_coarse(h);
    if (s != PMG_OK) return bail(s);
  }
  const Shape& F = h->lv[0].s;
  h->N = (size_t)F.NX * F.NZ;
  h->Nfree = (size_t)F.NX * (F.NZ - 1);
  // node coordinates
  std::vector<double> x, w;
  lgl(m.order, x, w);
  h->xcols.resize(F.NX);
  for (int ix = 0; ix < F.NX; ++ix) {
    int ex = ix / m.order, i = ix % m.order;
    h->xcols[ix] = m.x0 + (ex + (x[i] + 1.0) / 2.0) * h->dx;
  }
  std::vector<double> xz, wz;
  lgl(order_z, xz, wz);
  h->sigrows.resize(F.NZ);
  for (int iz = 0; iz < F.NZ; ++iz) {
    int ez = std::min(iz / order_z, m.cells_z - 1), j = iz - ez * order_z;
    h->sigrows[iz] = (ez + (xz[j] + 1.0) / 2.0) * h->dsig;
  }
  cudaError_t e;
#define ALLOC(ptr, T, n)                                   \
  do {                                                     \
    ptr = h->alloc<T>((n), e);                             \
    if (e != cudaSuccess) {                                \
      fail(PMG_ERR_OOM, "device allocation failed");       \
      return bail(PMG_ERR_OOM);                            \
    }                                                      \
  } while (0)
  ALLOC(h->eta, double, F.NX);
  ALLOC(h->geo[0], double, (size_t)m.cells_x * (m.order + 1) * 4);
  ALLOC(h->geo[1], float, (size_t)m.cells_x * (m.order + 1) * 4);
  ALLOC(h->geo_div, double, (size_t)m.cells_x * (m.order + 1) * 4);
  h->sigma[0] = upload<double>(h->sigrows, h->allocs, e);
  if (e != cudaSuccess) return bail(fail(PMG_ERR_OOM, "upload failed"));
  h->sigma[1] = upload<float>(h->sigrows, h->allocs, e);
  if (e != cudaSuccess) return bail(fail(PMG_ERR_OOM, "upload failed"));
  ALLOC(h->status, int, 3);
  ALLOC(h->x, double, h->N);
  ALLOC(h->r, double, h->N);
  ALLOC(h->p, double, h->N);
  ALLOC(h->w, double, h->N);
  ALLOC(h->z, double, h->N);
  ALLOC(h->rold, double, h->N);
  ALLOC(h->r32, float, h->N);
  ALLOC(h->c32, float, h->N);
  ALLOC(h->p32, float, h->N);
  ALLOC(h->w32, float, h->N);
  ALLOC(h->z32, float, h->N);
  ALLOC(h->rold32, float, h->N);
  ALLOC(h->scal, double, SLOT_COUNT);
  ALLOC(h->d_iter, int, 2);
  size_t nedges = (size_t)m.cells_x + 1;
  size_t ebuf = nedges * (2 * MAXO + 1) * (size_t)F.NZ;
  h->sc.edgebuf = h->alloc<double>(ebuf, e);
  if (e != cudaSuccess) return bail(fail(PMG_ERR_OOM, "device allocation failed"));
  h->sc.xbuf = h->alloc<double>(ebuf, e);
  if (e != cudaSuccess) return bail(fail(PMG_ERR_OOM, "device allocation failed"));
  if (arm_exchange(h->sc.xbuf, ebuf) != cudaSuccess) return bail(fail(PMG_ERR_CUDA, "exchange init failed"));
  ALLOC(h->sc.edgecnt, unsigned, nedges);
  ALLOC(h->sc.partials, double, std::max<size_t>(1024, 2 * (size_t)m.cells_x + 8));
  ALLOC(h->sc.edgepart, double, nedges);
  ALLOC(h->sc.redcnt, unsigned, 1);
  if (o.outer == PMG_GMRES) {
    const size_t mm = (size_t)o.gmres_restart;
    ALLOC(h->gm_V, double, (mm + 1) * h->N);
    ALLOC(h->gm_Z, double, mm * h->N);
    ALLOC(h->gm_h, double, 2 * (mm + 1) + 1);
    ALLOC(h->gm_part, double, (mm + 1) * 304);
    ALLOC(h->gm_y, double, mm);
    ALLOC(h->gm_cnt, unsigned, 1);
    ALLOC(h->gm_state, double, (mm + 1) * mm + 3 * mm + 1);
    ALLOC(h->gm_ctr, int, 2);
    if (cudaMemset(h->gm_cnt, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->gm_V, 0, (mm + 1) * h->N * sizeof(double)) != cudaSuccess ||
        cudaMemset(h->gm_Z, 0, mm * h->N * sizeof(double)) != cudaSuccess)
      return bail(fail(PMG_ERR_CUDA, "memset failed"));
  }
#undef ALLOC
  if (cudaMemset(h->sc.edgebuf, 0, ebuf * sizeof(double)) != cudaSuccess ||
      cudaMemset(h->sc.edgecnt, 0, nedges * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->sc.redcnt, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->status, 0, 3 * sizeof(int)) != cudaSuccess ||
      cudaMemset(h->scal, 0, SLOT_COUNT * sizeof(double)) != cudaSuccess ||
      cudaMemset(h->eta, 0, F.NX * sizeof(double)) != cudaSuccess)
    return bail(fail(PMG_ERR_CUDA, "memset failed"));
  if (cudaMallocHost(&h->scal_host, SLOT_COUNT * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&h->status_host, 3 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&h->iter_host, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(h->d_iter, 0, 2 * sizeof(int)) != cudaSuccess)
    return bail(fail(PMG_ERR_OOM, "pinned allocation failed"));
  pmg_status s = pmg_set_geometry(h, h->eta, nullptr);
  if (s != PMG_OK) return bail(s);
  s = vtail_setup(h);
  if (s != PMG_OK) return bail(s);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(PMG_ERR_CUDA, "setup failed"));
  *out = h;
  return PMG_OK;
}

pmg_status pmg_destroy(pmg_handle* h) {
  if (!h) return PMG_OK;
  DeviceGuard dg(h->device);
  cudaDeviceSynchronize();
  delete h;
  return PMG_OK;
}

pmg_status pmg_num_nodes(const pmg_handle* h, int64_t* n, int64_t* n_free, int* nx, int* nz, int* nlevels) {
  CKS(check_handle(h));
  if (n) *n = (int64_t)h->N;
  if (n_free) *n_free = (int64_t)h->Nfree;
  if (nx) *nx = h->lv[0].s.NX;
  if (nz) *nz = h->lv[0].s.NZ;
  if (nlevels) *nlevels = (int)h->lv.size();
  return PMG_OK;
}

pmg_status pmg_level_info(const pmg_handle* h, int level, int* order, int* nx, int* nz) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size()) return fail(PMG_ERR_INVALID, "bad level");
  if (order) *order = h->lv[level].order;
  if (nx) *nx = h->lv[level].s.NX;
  if (nz) *nz = h->lv[level].s.NZ;
  return PMG_OK;
}

pmg_status pmg_level_kernels(const pmg_handle* h, int level, int* flat32, int* fdm32, int* xfer) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size()) return fail(PMG_ERR_INVALID, "bad level");
  if (flat32) *flat32 = h->lv[level].thr_flat32;
  if (fdm32) *fdm32 = h->lv[level].thr_fdm32;
  if (xfer) *xfer = h->lv[level].thr_xfer;
  return PMG_OK;
}

pmg_status pmg_fused_vcycle_info(const pmg_handle* h, int* first_level, int* on, int* threads, int* ctas_per_sm,
                                 float* us) {
  CKS(check_handle(h));
  if (first_level) *first_level = h->vt_l0;
  if (on) *on = h->vt_on ? 1 : 0;
  if (threads) *threads = h->vt_threads;
  if (ctas_per_sm) *ctas_per_sm = h->vt_per_sm;
  if (us) {
    us[0] = h->vt_us[0];
    us[1] = h->vt_us[1];
  }
  return PMG_OK;
}

pmg_status pmg_set_fused_vcycle(pmg_handle* h, int on) {
  CKS(check_handle(h));
  if (on != 0 && on != 1) return fail(PMG_ERR_INVALID, "on must be 0 or 1");
  if (on && h->vt_l0 < 0) return fail(PMG_ERR_INVALID, "the levels do not qualify for the fused V-cycle");
  if (h->vt_on != (on == 1)) {
    h->vt_on = on == 1;
    // captured loops hold the other form of the V-cycle: rebuild on next use
    for (pmg_handle::Loop* lp : {&h->loop64, &h->loop32, &h->loop_gm, &h->loop_pdc})
      if (lp->exec) { cudaGraphExecDestroy(lp->exec); lp->exec = nullptr; }
  }
  return PMG_OK;
}

pmg_status pmg_node_coords(const pmg_handle* h, double* xc, double* sr) {
  CKS(check_handle(h));
  if (xc) std::memcpy(xc, h->xcols.data(), h->xcols.size() * sizeof(double));
  if (sr) std::memcpy(sr, h->sigrows.data(), h->sigrows.size() * sizeof(double));
  return PMG_OK;
}

pmg_status pmg_set_geometry(pmg_handle* h, const double* eta_dev, void* stream) {
  CKS(check_handle(h));
  if (!eta_dev) return fail(PMG_ERR_INVALID, "eta is NULL");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Shape& F = h->lv[0].s;
  if (eta_dev != h->eta) CK(cudaMemcpyAsync(h->eta, eta_dev, F.NX * sizeof(double), cudaMemcpyDeviceToDevice, st));
  int* gst = h->status + 1;
  CK(cudaMemsetAsync(gst, 0, sizeof(int), st));
  const double* hc = h->bathy ? h->hcol : nullptr;
  if (h->bathy) {
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry_bathy<double>(F, h->eta, hc, h->dx, h->dsig, (double*)h->geo6[0], gst, st); }));
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry_bathy<float>(F, h->eta, hc, h->dx, h->dsig, (float*)h->geo6[1], gst, st); }));
  } else {
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry<double>(F, h->eta, h->mesh.h, nullptr, h->dx, h->dsig, 0, (double*)h->geo[0], gst, st); }));
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry<float>(F, h->eta, h->mesh.h, nullptr, h->dx, h->dsig, 0, (float*)h->geo[1], gst, st); }));
  }
  CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry<double>(F, h->eta, h->mesh.h, hc, h->dx, h->dsig, 1, h->geo_div, gst, st); }));
  for (LevelDev& L : h->lv) {
    if (!L.actual) continue;
    // the level on the current surface: eta at its nodes, column factors, dense inverses
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return eta_level(F, L.s, L.Eeta, h->eta, L.aeta, st); }));
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry<double>(L.s, L.aeta, h->mesh.h, nullptr, h->dx, h->dsig, 0, (double*)L.ageo[0], gst, st); }));
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] { return geometry<float>(L.s, L.aeta, h->mesh.h, nullptr, h->dx, h->dsig, 0, (float*)L.ageo[1], gst, st); }));
    CKS(launch(h, PMG_K_SETUP, 1, st, [&] {
      return dense_setup(L.s, L.overlap, L.overlap_z, (const double*)L.ageo[0], L.dsig, (double*)L.dinv[0],
                         (float*)L.dinv[1], st);
    }));
  }
  h->mixed_stage = false;
  return PMG_OK;
}

pmg_status pmg_set_bathymetry(pmg_handle* h, const double* h_dev, void* stream) {
  CKS(check_handle(h));
  if (!h_dev) return fail(PMG_ERR_INVALID, "depth is NULL");
  if (h->aniso) return fail(PMG_ERR_INVALID, "a varying depth needs equal orders along x and sigma");
  if (h->opts.precond_geom == PMG_ACTUAL)
    return fail(PMG_ERR_INVALID, "levels on the actual geometry take a constant depth only");
  if (h->tc) return fail(PMG_ERR_INVALID, "the BF16 tensor-core operator takes a constant depth only");
  if (h->mesh.periodic_x && h->mesh.cells_x < 2) return fail(PMG_ERR_INVALID, "periodic mesh needs 2 or more cells");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const pmg_mesh_desc& m = h->mesh;
  const Shape& F = h->lv[0].s;
  const int P = m.order, n = P + 1;
  std::vector<double> hc(F.NX);
  CK(cudaMemcpyAsync(hc.data(), h_dev, F.NX * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (double v : hc)
    if (!(v > 0.0) || !std::isfinite(v)) return fail(PMG_ERR_INVALID, "still-water depth must be positive and finite");
  Line1D lf(P, m.cells_x, m.periodic_x);
  // level depths: the fine interpolant of each cell evaluated at the level's nodes
  std::vector<std::vector<double>> dl(h->lv.size());
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const int p = h->lv[l].order;
    if (p == P) { dl[l] = hc; continue; }
    std::vector<double> E = transfer_matrix(P, p);  // (p+1) x (P+1): order-P data at order-p nodes
    Line1D ll(p, m.cells_x, m.periodic_x);
    dl[l].assign(h->lv[l].s.NX, 0.0);
    for (int ex = 0; ex < m.cells_x; ++ex)
      for (int i = 0; i <= p; ++i) {
        double v = 0.0;
        for (int k = 0; k < n; ++k) v += E[i * n + k] * hc[lf.wrap(ex * P + k)];
        dl[l][ll.wrap(ex * p + i)] = v;
      }
    for (double v : dl[l])
      if (!(v > 0.0)) return fail(PMG_ERR_INVALID, "the depth interpolated to a coarse level is not positive");
  }
  for (size_t l = 0; l < h->lv.size(); ++l) {
    CKS(build_level_var(h, (int)l, dl[l]));
    if (h->opts.smoother == PMG_ASM_DENSE && l + 1 < h->lv.size()) CKS(build_level_dense(h, (int)l, &dl[l]));
  }
  {
    std::vector<double> V, coef, inv;
    int nsteps = 0;
    coarse_tables(h, &dl.back(), V, coef, inv, nsteps);
    CK(cudaMemcpy((void*)h->coarse.V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)h->coarse.coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)h->coarse.inv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  // bottom edge weights: arc length of the mapped bottom z = -h(x) per node column
  std::vector<double> xg, w, D = diff_matrix(P), mb(F.NX, 0.0);
  lgl(P, xg, w);
  for (int ex = 0; ex < m.cells_x; ++ex)
    for (int i = 0; i < n; ++i) {
      double hx = 0.0;
      for (int k = 0; k < n; ++k) hx += D[i * n + k] * hc[lf.wrap(ex * P + k)];
      hx *= 2.0 / h->dx;
      mb[lf.wrap(ex * P + i)] += w[i] * (h->dx * 0.5) * std::sqrt(1.0 + hx * hx);
    }
  cudaError_t e = cudaSuccess;
  if (!h->hcol) {
    h->hcol = h->alloc<double>(F.NX, e); CK(e);
    h->mb = h->alloc<double>(F.NX, e); CK(e);
    h->geo6[0] = h->alloc<double>((size_t)m.cells_x * n * 6, e); CK(e);
    h->geo6[1] = h->alloc<float>((size_t)m.cells_x * n * 6, e); CK(e);
  }
  CK(cudaMemcpy(h->hcol, hc.data(), F.NX * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->mb, mb.data(), F.NX * sizeof(double), cudaMemcpyHostToDevice));
  h->bathy = true;
  // graphs captured before hold the constant-depth kernels: rebuild on next use
  for (pmg_handle::Loop* lp : {&h->loop64, &h->loop32, &h->loop_gm, &h->loop_pdc})
    if (lp->exec) { cudaGraphExecDestroy(lp->exec); lp->exec = nullptr; }
  CKS(vtail_setup(h));  // the levels now vary: back to one launch per step
  return pmg_set_geometry(h, h->eta, stream);
}

pmg_status pmg_set_geometry_mixed(pmg_handle* h, const double* eta_dev, const double* eta_prev_dev, void* stream) {
  CKS(check_handle(h));
  if (h->bathy) return fail(PMG_ERR_INVALID, "the mixed-stage operator takes a constant depth only");
  if (h->aniso) return fail(PMG_ERR_INVALID, "the mixed-stage operator needs equal orders along x and sigma");
  CKS(pmg_set_geometry(h, eta_dev, stream));
  if (!eta_prev_dev) return fail(PMG_ERR_INVALID, "eta_prev is NULL");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Shape& F = h->lv[0].s;
  cudaError_t e = cudaSuccess;
  if (!h->geo5) {
    h->geo5 = h->alloc<double>((size_t)h->mesh.cells_x * (h->mesh.order + 1) * 5, e);
    CK(e);
    h->eta_prev = h->alloc<double>(F.NX, e);
    CK(e);
  }
  CK(cudaMemcpyAsync(h->eta_prev, eta_prev_dev, F.NX * sizeof(double), cudaMemcpyDeviceToDevice, st));
  int* gst = h->status + 1;
  CKS(launch(h, PMG_K_SETUP, 1, st, [&] {
    return geometry_mixed(F, h->eta, h->eta_prev, h->mesh.h, h->dx, h->dsig, h->geo5, gst, st);
  }));
  h->mixed_stage = true;
  return PMG_OK;
}

pmg_status pmg_assemble_rhs(pmg_handle* h, const double* f, const double* gb, const double* gl,
                            const double* gr, double* b, void* stream) {
  CKS(check_handle(h));
  if (!f || !b) return fail(PMG_ERR_INVALID, "f and b must be non-NULL");
  DeviceGuard dg(h->device);
  LevelDev& L = h->lv[0];
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, [&] {
    return rhs_source(L.s, h->eta, h->mesh.h, h->bathy ? h->hcol : nullptr, h->dx, h->dsig, (const double*)L.mX[0],
                      (const double*)L.mZ[0], h->bathy ? h->mb : nullptr, f, gb,
                      h->mesh.periodic_x ? nullptr : gl, h->mesh.periodic_x ? nullptr : gr, b, st);
  });
}

pmg_status pmg_assemble_rhs_div(pmg_handle* h, const double* u, const double* w, double scale, double* b,
                                void* stream) {
  CKS(check_handle(h));
  if (!u || !w || !b) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  CurvedArgs a{};
  a.s = h->lv[0].s;
  a.mode = 3;
  a.x = u;
  a.x2 = w;
  a.y = b;
  a.geo = h->geo_div;
  a.sigma = h->sigma[0];
  a.scale = scale;
  a.sc = h->sc;
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, [&] { return curved_op<double>(a, st); });
}

pmg_status pmg_apply(pmg_handle* h, const double* x, double* y, void* stream) {
  CKS(check_handle(h));
  if (!x || !y) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  return curved<double>(h, 0, x, nullptr, y, 1, nullptr, (cudaStream_t)stream);
}

pmg_status pmg_apply_f32(pmg_handle* h, const float* x, float* y, void* stream) {
  CKS(check_handle(h));
  if (!x || !y) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  return curved<float>(h, 0, x, nullptr, y, 1, nullptr, (cudaStream_t)stream, 0);
}

pmg_status pmg_apply_bf16(pmg_handle* h, const float* x, float* y, int split, void* stream) {
  CKS(check_handle(h));
  if (!x || !y || split < 0 || split > 1) return fail(PMG_ERR_INVALID, "NULL vector or bad split flag");
  DeviceGuard dg(h->device);
  return curved<float>(h, 0, x, nullptr, y, 1, nullptr, (cudaStream_t)stream, split ? 3 : 1);
}

pmg_status pmg_level_apply(pmg_handle* h, int level, const void* x, void* y, int f32, void* stream) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size() || !x || !y) return fail(PMG_ERR_INVALID, "bad level or vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? level_residual<float>(h, level, nullptr, x, y, 0, st) : level_residual<double>(h, level, nullptr, x, y, 0, st);
}

pmg_status pmg_level_sweep(pmg_handle* h, int level, const void* r, void* x, int post, int f32, void* stream) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size() - 1 || !r || !x) return fail(PMG_ERR_INVALID, "bad level or vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? level_fdm<float>(h, level, r, x, post, st) : level_fdm<double>(h, level, r, x, post, st);
}

pmg_status pmg_level_smooth(pmg_handle* h, int level, const void* b, void* x, int post, int f32, void* stream) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size() - 1 || !b || !x) return fail(PMG_ERR_INVALID, "bad level or vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? level_smooth<float>(h, level, b, x, post, false, st) : level_smooth<double>(h, level, b, x, post, false, st);
}

pmg_status pmg_restrict(pmg_handle* h, int level, const void* rf, void* rc, int f32, void* stream) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size() - 1 || !rf || !rc) return fail(PMG_ERR_INVALID, "bad level or vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? transfer_op<float>(h, level, rf, rc, 1, st) : transfer_op<double>(h, level, rf, rc, 1, st);
}

pmg_status pmg_prolong(pmg_handle* h, int level, const void* xc, void* xf, int f32, void* stream) {
  CKS(check_handle(h));
  if (level < 0 || level >= (int)h->lv.size() - 1 || !xc || !xf) return fail(PMG_ERR_INVALID, "bad level or vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? transfer_op<float>(h, level, xc, xf, 0, st) : transfer_op<double>(h, level, xc, xf, 0, st);
}

pmg_status pmg_coarse_solve(pmg_handle* h, const double* b, double* x, void* stream) {
  CKS(check_handle(h));
  if (!b || !x) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_COARSE, 3, st, [&] { return coarse_solve<double>(h->coarse, b, x, st); });
}

pmg_status pmg_vcycle(pmg_handle* h, const void* r, void* z, int f32, void* stream) {
  CKS(check_handle(h));
  if (!r || !z) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return f32 ? vcycle<float>(h, 0, r, z, st) : vcycle<double>(h, 0, r, z, st);
}

pmg_status pmg_solve(pmg_handle* h, const double* b, const double* pD, const double* x0, double* p_out,
                     pmg_solve_info* info, void* stream) {
  CKS(check_handle(h));
  if (!b || !pD || !p_out) return fail(PMG_ERR_INVALID, "b, p_dirichlet and p_out must be non-NULL");
  DeviceGuard dg(h->device);
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  pmg_solve_info loc{};
  size_t N = h->N;
  if (h->mixed_stage && h->opts.outer != PMG_PDC && h->opts.outer != PMG_GMRES)
    return fail(PMG_ERR_INVALID, "the mixed-stage operator is nonsymmetric: use outer PMG_PDC or PMG_GMRES");
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N, 0.0}, [&] { return check_finite(N, b, h->status, st); }));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 0.0}, [&] { return init_x(N, h->lv[0].s.NZ, h->x, x0, pD, h->status, st); }));
  CKS(lifted_norm(h, b, pD, x0, st));
  CKS(read_scalars(h, st));
  pmg_status result = PMG_OK;
  double bb = h->scal_host[SLOT_BB];
  if (h->status_host[1]) {
    result = fail(PMG_ERR_INVALID, "geometry has a non-positive or non-finite water depth");
  } else if (h->status_host[0]) {
    result = fail(PMG_ERR_NONFINITE, "non-finite input (b, p_D or x0)");
  } else if (!std::isfinite(bb)) {
    result = fail(PMG_ERR_NONFINITE, "non-finite right-hand side");
  } else if (bb > 0.0) {
    pmg_status s;
    if (h->opts.outer == PMG_PDC) s = h->timing ? solve_pdc(h, b, &loc, st) : solve_pdc_graph(h, b, &loc, st);
    else if (h->opts.outer == PMG_GMRES) s = h->timing ? solve_gmres(h, b, &loc, st) : solve_gmres_graph(h, b, &loc, st);
    else if (h->opts.outer == PMG_IR)
      s = h->timing ? solve_refine(h, b, &loc, st) : solve_refine_graph(h, b, &loc, st);
    else
      s = h->timing ? solve_krylov64(h, b, &loc, st) : solve_krylov64_graph(h, b, &loc, st);
    if (s != PMG_OK) result = s;
    // final true residual
    CKS(outer_residual(h, b, SLOT_RR64, st));
    CKS(read_scalars(h, st));
    double rel = std::sqrt(h->scal_host[SLOT_RR64] / bb);
    loc.rel_residual = rel;
    if (result == PMG_OK && !(rel <= h->opts.tol)) {
      result = std::isfinite(rel) ? PMG_ERR_NOT_CONVERGED : PMG_ERR_NONFINITE;
      fail(result, "solve did not reach the tolerance");
    }
  }
  if (h->status_host[2]) {  // a bounded device wait gave up during this solve (or before it)
    result = fail(PMG_ERR_TIMEOUT, "a bounded device-side wait gave up (pmg_set_wait_limit)");
    CK(cudaMemsetAsync(h->status + 2, 0, sizeof(int), st));
    if (h->vt_bar) CK(cudaMemsetAsync(h->vt_bar, 0, 4 * sizeof(unsigned), st));  // an aborted grid barrier
  }
  CK(cudaMemcpyAsync(p_out, h->x, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  loc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  loc.status = result;
  if (info) *info = loc;
  return result;
}

pmg_status pmg_residual_norm(pmg_handle* h, const double* b, const double* pD, const double* x, double* norm,
                             void* stream) {
  CKS(check_handle(h));
  if (!b || !pD || !x || !norm) return fail(PMG_ERR_INVALID, "b, p_dirichlet, x and norm must be non-NULL");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  size_t N = h->N;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 0.0}, [&] { return init_x(N, h->lv[0].s.NZ, h->p, x, pD, h->status, st); }));
  CKS(curved<double>(h, 1, h->p, b, h->w, 0, h->scal + SLOT_AUX, st));
  CKS(read_scalars(h, st));
  if (h->status_host[1]) return fail(PMG_ERR_INVALID, "geometry has a non-positive or non-finite water depth");
  *norm = std::sqrt(h->scal_host[SLOT_AUX]);
  if (h->status_host[0] || !std::isfinite(*norm)) return fail(PMG_ERR_NONFINITE, "non-finite input or residual");
  return PMG_OK;
}

pmg_status pmg_profile_reset(pmg_handle* h, int timing) {
  CKS(check_handle(h));
  DeviceGuard dg(h->device);
  CK(cudaDeviceSynchronize());
  for (auto& v : h->launches) v = 0;
  for (auto& v : h->bytes) v = 0;
  for (auto& v : h->flops) v = 0;
  h->ev_used.clear();
  h->timing = timing != 0;
  return PMG_OK;
}

pmg_status pmg_profile_read(pmg_handle* h, int64_t* launches, double* ms, double* bytes, double* flops) {
  CKS(check_handle(h));
  DeviceGuard dg(h->device);
  CK(cudaDeviceSynchronize());
  double acc[PMG_K_COUNT] = {};
  for (auto& u : h->ev_used) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->ev_pool[2 * u.second], h->ev_pool[2 * u.second + 1]));
    acc[u.first] += t;
  }
  for (int k = 0; k < PMG_K_COUNT; ++k) {
    if (launches) launches[k] = h->launches[k];
    if (ms) ms[k] = acc[k];
    if (bytes) bytes[k] = h->bytes[k];
    if (flops) flops[k] = h->flops[k];
  }
  return PMG_OK;
}

pmg_status pmg_gradient(pmg_handle* h, const double* f, double* fx, double* fz, void* stream) {
  CKS(check_handle(h));
  if (!f || !fx || !fz) return fail(PMG_ERR_INVALID, "NULL vector");
  if (h->aniso) return fail(PMG_ERR_INVALID, "gradient recovery needs equal orders along x and sigma");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Shape& F = h->lv[0].s;
  return launch(h, PMG_K_SETUP, 1, st, Cost{24.0 * h->N, 0.0}, [&] {
    return gradient(F, f, fx, fz, h->eta, (const double*)h->sigma[0], h->mesh.h, h->dx, h->dsig, st,
                    h->bathy ? h->hcol : nullptr);
  });
}

pmg_status pmg_set_filter(pmg_handle* h, int cutoff, double alpha, double beta) {
  CKS(check_handle(h));
  if (h->aniso) return fail(PMG_ERR_INVALID, "the stepper kernels need equal orders along x and sigma");
  const int P = h->mesh.order, n = P + 1;
  if (cutoff < 0 || cutoff > P || !std::isfinite(alpha) || alpha > 0.0 || !(beta > 0.0) || !std::isfinite(beta))
    return fail(PMG_ERR_INVALID, "filter needs 0 <= cutoff <= P, finite alpha <= 0, beta > 0");
  DeviceGuard dg(h->device);
  // F = V diag(S) V^-1, V[i][k] = P~_k(r_i) (orthonormal Legendre at the LGL nodes)
  std::vector<double> r, wq;
  lgl(P, r, wq);
  std::vector<double> V(n * n), Vi, d(n), tmp(n);
  for (int i = 0; i < n; ++i) {
    legendre_orthonormal(P, r[i], tmp.data(), d.data());
    for (int k = 0; k < n; ++k) V[i * n + k] = tmp[k];
  }
  Vi = V;
  if (!invert(n, Vi)) return fail(PMG_ERR_INVALID, "singular Vandermonde matrix");
  std::vector<double> F(n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    double S = k <= cutoff ? 1.0 : std::exp(alpha * std::pow((double)(k - cutoff) / (P + 1 - cutoff), beta));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) F[i * n + j] += V[i * n + k] * S * Vi[k * n + j];
  }
  cudaError_t e = cudaSuccess;
  if (!h->filt) {
    h->filt = h->alloc<double>(n * n, e);
    CK(e);
  }
  CK(cudaMemcpy(h->filt, F.data(), n * n * sizeof(double), cudaMemcpyHostToDevice));
  return PMG_OK;
}

pmg_status pmg_filter(pmg_handle* h, const double* f, double* out, int surface, void* stream) {
  CKS(check_handle(h));
  if (h->aniso) return fail(PMG_ERR_INVALID, "the stepper kernels need equal orders along x and sigma");
  if (!f || !out || f == out) return fail(PMG_ERR_INVALID, "filter needs distinct non-NULL input and output");
  if (!h->filt) return fail(PMG_ERR_INVALID, "no filter set (pmg_set_filter)");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  double nv = surface ? (double)h->lv[0].s.NX : (double)h->N;
  return launch(h, PMG_K_SETUP, 1, st, Cost{16.0 * nv, 0.0},
                [&] { return spectral_filter(h->lv[0].s, f, out, h->filt, surface, st); });
}

pmg_status pmg_surface_slope(pmg_handle* h, double* etax, void* stream) {
  CKS(check_handle(h));
  if (!etax) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, [&] { return surface_slope(h->lv[0].s, h->eta, h->dx, etax, st); });
}

pmg_status pmg_forcing(pmg_handle* h, const double* u, const double* w, const double* ux, const double* uz,
                       const double* wx, const double* wz, const double* etax, double g, double* Fu, double* Fw,
                       void* stream) {
  CKS(check_handle(h));
  if (h->aniso) return fail(PMG_ERR_INVALID, "the stepper kernels need equal orders along x and sigma");
  if (!u || !w || !ux || !uz || !wx || !wz || !etax || !Fu || !Fw) return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, Cost{64.0 * h->N, 8.0 * h->N}, [&] {
    return forcing(h->N, h->lv[0].s.NZ, u, w, ux, uz, wx, wz, etax, g, Fu, Fw, st);
  });
}

pmg_status pmg_stage_rates(pmg_handle* h, const double* u, const double* w, const double* uz, const double* wz,
                           const double* Fu, const double* Fw, const double* px, const double* pz, const double* etax,
                           double rho, double* du, double* dw, double* deta, void* stream) {
  CKS(check_handle(h));
  if (h->aniso) return fail(PMG_ERR_INVALID, "the stepper kernels need equal orders along x and sigma");
  if (!u || !w || !uz || !wz || !Fu || !Fw || !px || !pz || !etax || !du || !dw || !deta)
    return fail(PMG_ERR_INVALID, "NULL vector");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, Cost{88.0 * h->N, 12.0 * h->N}, [&] {
    return rates(h->N, h->lv[0].s.NZ, (const double*)h->sigma[0], u, w, uz, wz, Fu, Fw, px, pz, etax, rho, du, dw,
                 deta, st);
  });
}

pmg_status pmg_axpy(pmg_handle* h, int64_t n, double a, const double* x, const double* y, double* out,
                    void* stream) {
  CKS(check_handle(h));
  if (!x || !y || !out || n < 0) return fail(PMG_ERR_INVALID, "bad axpy arguments");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  return launch(h, PMG_K_SETUP, 1, st, Cost{24.0 * n, 2.0 * n}, [&] { return axpy((size_t)n, a, x, y, out, st); });
}

pmg_status pmg_set_wait_limit(pmg_handle* h, int64_t cycles) {
  CKS(check_handle(h));
  h->wait_cycles = cycles < 0 ? kWaitCyclesDefault : (long long)cycles;
  // captured loops hold the old bound in their kernel parameters: rebuild on next use
  for (pmg_handle::Loop* lp : {&h->loop64, &h->loop32, &h->loop_gm, &h->loop_pdc})
    if (lp->exec) { cudaGraphExecDestroy(lp->exec); lp->exec = nullptr; }
  return PMG_OK;
}

pmg_status pmg_autotune(pmg_handle* h) {
  CKS(check_handle(h));
  DeviceGuard dg(h->device);
  int nl = (int)h->lv.size();
  for (int l = 0; l < nl; ++l) {
    LevelDev& L = h->lv[l];
    void* x = L.x[1];
    void* b = L.b[1];
    void* t = L.t[1];
    // slab CTAs (positive sizes), node-parallel CTAs (negative) or tiled CTAs (codes
    // 10000 + 100 element columns + element rows; constant depth, equal orders up to 8)
    if (!L.actual) {
      const std::vector<int> slab{64, 128, 192, 256, 320, 384, 512}, np{-64, -128, -256},
          tile{10804, 10808, 11604, 11608, 13204, 13208}, bulk{1128, 1192, 1256, 1384, 1512};
      const bool tile_ok = !L.var && !L.aniso && L.order <= 8;
      const bool bulk_ok = !L.var && !L.aniso;
      const int fk = h->opts.flat_kernel;
      std::vector<int> cands = fk == 1 ? np : fk == 0 ? slab : (fk == 2 && tile_ok) ? tile : (fk == 3 && bulk_ok) ? bulk : slab;
      if (fk >= 10000) cands = tile_ok ? std::vector<int>{fk} : slab;
      if (flat_bulk_code_ok(fk)) cands = bulk_ok ? std::vector<int>{fk} : slab;
      if (fk == -1) {
        cands.insert(cands.end(), np.begin(), np.end());
        if (tile_ok) cands.insert(cands.end(), tile.begin(), tile.end());
        if (bulk_ok) cands.insert(cands.end(), bulk.begin(), bulk.end());
      }
      // a forced kernel family tunes (and caches) apart from the free choice
      const int key = L.order + 100 * (L.aniso ? L.order_z : 0) +
                      (fk >= 1000 ? 100 * fk : fk >= 0 ? 10000 * (fk + 1) : 0);
      CKS(tune_one(h, L.var ? TK_FLAT32V : TK_FLAT32, key, L.s.NZ,
                   [&](int thr, cudaStream_t cs) {
        L.thr_flat32 = thr;
        return level_residual<float>(h, l, b, x, t, 1, cs);
      }, &L.thr_flat32, cands));
    }
    if (l == nl - 1) continue;
    if (L.var || L.aniso || L.dense) {
      // varying depth, different orders or dense blocks: no k_fdm32 sweep, split residuals;
      // only the transfers tune
      LevelDev& C = h->lv[l + 1];
      CKS(tune_one(h, TK_XFER, L.order * 16 + C.order + 1000 * (L.aniso ? L.order_z : 0), L.s.NZ,
                   [&](int thr, cudaStream_t cs) {
        L.thr_xfer = thr;
        return transfer_op<float>(h, l, t, C.b[1], 1, cs);
      }, &L.thr_xfer));
      continue;
    }
    {
      // slab CTAs of 64..512 threads, or z-split CTAs (codes 1000 zc + threads) of zc
      // element rows; a forced family tunes (and caches) apart from the free choice
      // (up to order 6 the slab sweep is built for at most 256 threads)
      // (sizes one warp above 64, 128 and 192 let one thread take one node row of the
      // 65-, 129- and 193-row columns of 32-cell tanks)
      const std::vector<int> slab = L.order <= 6 ? std::vector<int>{64, 96, 128, 160, 192, 224, 256}
                                                 : std::vector<int>{64, 128, 192, 256, 320, 384, 512};
      std::vector<int> zsplit;
      for (int zc : {2, 4, 8, 16})
        if (zc <= 2 * L.s.Nz)
          for (int thr : {64, 96, 128, 192, 256}) zsplit.push_back(1000 * zc + thr);
      const int sk = h->opts.sweep_kernel;
      std::vector<int> cands = sk == 0 ? slab : sk >= 1000 ? std::vector<int>{sk} : zsplit;
      if (sk == -1) cands.insert(cands.end(), slab.begin(), slab.end());
      const int skey = sk >= 1000 ? 3 + sk : sk + 1;
      CKS(tune_one(h, TK_FDM32, L.order * 16 + L.overlap + 1000 * skey, L.s.NZ, [&](int thr, cudaStream_t cs) {
        L.thr_fdm32 = thr;
        return level_fdm<float>(h, l, t, x, 0, cs);
      }, &L.thr_fdm32, cands));
    }
    {
      // residual launch + sweep, or one sweep that forms its residual (x -> t ping-pong);
      // the fused form must win by 10% (the two are within timing noise at config 2)
      float us_split = 0.f, us_fused = 0.f;
      CKS(time_launches(h, [&](int thr, cudaStream_t cs) {
        CKS(level_residual<float>(h, l, b, x, t, 1, cs));
        return level_fdm<float>(h, l, t, x, 0, cs);
      }, L.thr_fdm32, 10, &us_split));
      CKS(time_launches(h, [&](int thr, cudaStream_t cs) {
        return level_fdm<float>(h, l, nullptr, x, 0, cs, b, t, false);
      }, L.thr_fdm32, 10, &us_fused));
      if (h->opts.fuse_residual < 0) L.fuse_res = L.order >= 2 && us_fused < 0.9f * us_split;
    }
    LevelDev& C = h->lv[l + 1];
    CKS(tune_one(h, TK_XFER, L.order * 16 + C.order, L.s.NZ, [&](int thr, cudaStream_t cs) {
      L.thr_xfer = thr;
      return transfer_op<float>(h, l, t, C.b[1], 1, cs);
    }, &L.thr_xfer));
    {
      // residual launch + restriction, or a restriction that forms the residual itself
      float us_split = 0.f, us_fused = 0.f;
      CKS(time_launches(h, [&](int thr, cudaStream_t cs) {
        CKS(level_residual<float>(h, l, b, x, t, 1, cs));
        return transfer_op<float>(h, l, t, C.b[1], 1, cs);
      }, L.thr_xfer, 10, &us_split));
      CKS(time_launches(h, [&](int thr, cudaStream_t cs) {
        return transfer_op<float>(h, l, b, C.b[1], 1, cs, x);
      }, L.thr_xfer, 10, &us_fused));
      if (h->opts.fuse_residual < 0) L.fuse_restrict = us_fused < 0.9f * us_split;
    }
  }
  // the FP32 build differs with the tensor-core mode and the FP64-vector build with
  // double-float arithmetic: each variant tunes under its own key
  const int curved_key = h->mesh.order + 100 * (h->aniso ? h->mesh.order_z : 0);
  // besides the usual sizes: the operator's work-item counts per CTA rounded up to whole
  // warps (the node rows of the x-contractions, the (column, element) pairs of the
  // sigma-contractions, which also divide the metric phase's element nodes), so that no
  // phase leaves a partial round of threads idle
  std::vector<int> curved_cands = {64, 128, 192, 256, 320, 384, 512};
  {
    const int NZ0 = h->lv[0].s.NZ, L0 = h->mesh.cells_z * (h->mesh.order + 1);
    for (int c : {(NZ0 + 31) / 32 * 32, (L0 + 31) / 32 * 32})
      if (c >= 64 && c <= 512 && std::find(curved_cands.begin(), curved_cands.end(), c) == curved_cands.end())
        curved_cands.push_back(c);
    std::sort(curved_cands.begin(), curved_cands.end());
  }
  CKS(tune_one(h, h->bathy ? TK_CURVED32B : TK_CURVED32, curved_key + 10000 * h->tc, h->lv[0].s.NZ,
               [&](int thr, cudaStream_t cs) {
    h->thr_curved32 = thr;
    return curved<float>(h, 0, h->r32, nullptr, h->w32, 1, nullptr, cs);
  }, &h->thr_curved32, curved_cands));
  CKS(tune_one(h, h->bathy ? TK_CURVED64B : TK_CURVED64, curved_key + 10000 * (h->df64_outer ? 1 : 0), h->lv[0].s.NZ,
               [&](int thr, cudaStream_t cs) {
    h->thr_curved64 = thr;
    return curved<double>(h, 0, h->p, nullptr, h->w, 1, nullptr, cs);
  }, &h->thr_curved64, curved_cands));
  // fused coarse V-cycle: the step table again (the tuned residual forms change the
  // recorded steps), then its CTA size and CTAs per SM by timing the whole FP32 V-cycle;
  // with fuse_coarse = -1 it is switched on only where that V-cycle is faster than with
  // one launch per step (on a GB300 at config 2 it is not: a grid barrier of the resident
  // CTAs costs more than the kernel boundary it replaces)
  CKS(vtail_setup(h));
  // the decision of the free choice (fuse_coarse = -1) is remembered like a CTA size:
  // 100000 on + 1000 CTAs per SM + threads
  // keyed by the fine order and the orders of the fused levels (a custom level sequence
  // fuses other levels on the same mesh)
  int vorders = h->mesh.order;
  for (int l = std::max(h->vt_l0, 1); l < (int)h->lv.size(); ++l) vorders = vorders * 11 + h->lv[l].order;
  const auto vkey = std::make_tuple((int)TK_VTAIL, vorders, h->lv[0].s.NZ, h->mesh.cells_x);
  int vcached = -1;
  if (h->vt_l0 >= 0 && h->vt_sms > 0 && h->opts.fuse_coarse == -1) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(vkey);
    if (it != g_tune.end()) vcached = it->second;
  }
  if (vcached >= 0) {
    h->vt_on = vcached >= 100000;
    h->vt_per_sm = (vcached % 100000) / 1000;
    h->vt_threads = vcached % 1000;
  } else if (h->vt_l0 >= 0 && h->vt_sms > 0) {
    auto run = [&](int, cudaStream_t cs) { return vcycle<float>(h, 0, h->r32, h->z32, cs); };
    h->vt_on = false;
    float us_off = 0.f;
    CKS(time_launches(h, run, 0, 10, &us_off));
    float best = 1e30f;
    int bt = h->vt_threads, bp = h->vt_per_sm;
    for (int thr : {128, 256}) {
      int occ = 0;
      CK(vtail_occupancy(thr, h->vt_smem, &occ));
      for (int per = 1; per <= std::min(occ, 4); ++per) {
        h->vt_on = true;
        h->vt_threads = thr;
        h->vt_per_sm = per;
        float us = 0.f;
        CKS(time_launches(h, run, 0, 10, &us));
        if (us < best) { best = us; bt = thr; bp = per; }
      }
    }
    // the launch-per-step V-cycle again: the first timing may run on cold clocks and caches
    h->vt_on = false;
    float us_off2 = 0.f;
    CKS(time_launches(h, run, 0, 10, &us_off2));
    us_off = std::min(us_off, us_off2);
    h->vt_threads = bt;
    h->vt_per_sm = bp;
    h->vt_on = h->opts.fuse_coarse == 1 || best < 0.97f * us_off;
    h->vt_us[0] = us_off;
    h->vt_us[1] = best;
    if (h->opts.fuse_coarse == -1) {
      const int code = (h->vt_on ? 100000 : 0) + 1000 * h->vt_per_sm + h->vt_threads;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[vkey] = code;
      tune_cache_store(TK_VTAIL, std::get<1>(vkey), std::get<2>(vkey), std::get<3>(vkey), code);
    }
  }
  // graphs built before tuning keep the old sizes: rebuild on next use
  for (pmg_handle::Loop* lp : {&h->loop64, &h->loop32, &h->loop_gm, &h->loop_pdc})
    if (lp->exec) { cudaGraphExecDestroy(lp->exec); lp->exec = nullptr; }
  CK(cudaDeviceSynchronize());
  return PMG_OK;
}

pmg_status pmg_batch_create(int n, const pmg_mesh_desc* meshes, const pmg_opts* opts, pmg_batch** out) {
  if (!out) return fail(PMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || !meshes) return fail(PMG_ERR_INVALID, "need n >= 1 meshes");
  auto* b = new (std::nothrow) pmg_batch();
  if (!b) return fail(PMG_ERR_OOM, "host allocation failed");
  for (int i = 0; i < n; ++i) {
    pmg_handle* h = nullptr;
    pmg_status s = pmg_create(&meshes[i], opts, &h);
    if (s != PMG_OK) { delete b; return s; }
    b->h.push_back(h);
    s = pmg_autotune(h);
    if (s != PMG_OK) { delete b; return s; }
    // the problems' own loops may run side by side on their streams (pmg_batch_set_path
    // 2): cooperative grids sized to fill the GPU would contend, so they step level by level
    h->vt_on = false;
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      delete b;
      return fail(PMG_ERR_CUDA, "stream creation failed");
    }
    b->st.push_back(st);
    b->done.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return fail(PMG_ERR_CUDA, "event creation failed");
  }
  *out = b;
  return PMG_OK;
}

pmg_status pmg_batch_destroy(pmg_batch* b) {
  if (b) {
    cudaDeviceSynchronize();
    delete b;
  }
  return PMG_OK;
}

pmg_status pmg_batch_set_path(pmg_batch* b, int path) {
  if (!b || path < 0 || path > 2) return fail(PMG_ERR_INVALID, "batch is NULL or path not 0, 1 or 2");
  b->path = path;
  b->eager = path == 1;
  return PMG_OK;
}

pmg_status pmg_batch_info(const pmg_batch* b, int* batched, int* launches) {
  if (!b) return fail(PMG_ERR_INVALID, "batch is NULL");
  if (batched) *batched = (b->path != 2 && batch_eligible(b)) ? 1 : 0;
  if (launches) *launches = b->graph_built ? (int)b->launches_per_iter : 0;
  return PMG_OK;
}

pmg_status pmg_batch_handle(pmg_batch* b, int i, pmg_handle** h) {
  if (!b || !h || i < 0 || i >= (int)b->h.size()) return fail(PMG_ERR_INVALID, "bad batch index");
  *h = b->h[i];
  return PMG_OK;
}

pmg_status pmg_batch_solve(pmg_batch* B, const double* const* bv, const double* const* pdv, double* const* pout,
                           pmg_solve_info* infos, void* stream) {
  if (!B || !bv || !pdv || !pout) return fail(PMG_ERR_INVALID, "NULL argument");
  int n = (int)B->h.size();
  for (int i = 0; i < n; ++i)
    if (!bv[i] || !pdv[i] || !pout[i]) return fail(PMG_ERR_INVALID, "NULL vector in batch");
  if (B->path != 2 && batch_eligible(B)) return batch_solve_graph(B, bv, pdv, pout, infos, (cudaStream_t)stream);
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t cs = (cudaStream_t)stream;
  CK(cudaEventRecord(B->fork, cs));
  std::vector<pmg_solve_info> loc(n);
  std::vector<int> active(n, 0), total(n, 0);
  // phase 1: inputs, lifted residual and its norm on every problem's stream
  for (int i = 0; i < n; ++i) {
    pmg_handle* h = B->h[i];
    cudaStream_t st = B->st[i];
    size_t N = h->N;
    CK(cudaStreamWaitEvent(st, B->fork, 0));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{8.0 * N, 0.0}, [&] { return check_finite(N, bv[i], h->status, st); }));
    CKS(launch(h, PMG_K_VECTOR, 1, st, Cost{24.0 * N, 0.0}, [&] { return init_x(N, h->lv[0].s.NZ, h->x, nullptr, pdv[i], h->status, st); }));
    CKS(lifted_norm(h, bv[i], pdv[i], nullptr, st));
    CK(cudaMemcpyAsync(h->scal_host, h->scal, SLOT_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->status_host, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(B->st[i]));
  // phase 2: every problem's device-side Krylov loop, concurrently; restarts on drift
  for (int round = 0; round < 4; ++round) {
    int launched = 0;
    for (int i = 0; i < n; ++i) {
      pmg_handle* h = B->h[i];
      double bb = h->scal_host[SLOT_BB], tol2 = h->opts.tol * h->opts.tol;
      if (round == 0) {
        if (h->status_host[0] || h->status_host[1] || !std::isfinite(bb)) {
          loc[i].status = h->status_host[1] ? PMG_ERR_INVALID : PMG_ERR_NONFINITE;
          continue;
        }
        active[i] = bb > 0.0 && h->scal_host[SLOT_RR64] > tol2 * bb;
      } else {
        active[i] = active[i] && h->scal_host[SLOT_RR64] > tol2 * bb && total[i] < h->opts.max_iter &&
                    std::isfinite(h->scal_host[SLOT_RR64]);
      }
      if (!active[i]) continue;
      if (!h->loop64.exec)
        CKS(build_loop(h, h->loop64, [&](cudaStream_t c2, cudaGraphConditionalHandle hc) { return cg64_step(h, true, c2, hc); },
                       [&](cudaStream_t c2, cudaGraphConditionalHandle hc) { return cg64_step(h, false, c2, hc); }));
      CK(cudaGraphLaunch(h->loop64.exec, B->st[i]));
      CK(cudaMemcpyAsync(h->iter_host, h->d_iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, B->st[i]));
      CKS(outer_residual(h, bv[i], SLOT_RR64, B->st[i]));
      CK(cudaMemcpyAsync(h->scal_host, h->scal, SLOT_COUNT * sizeof(double), cudaMemcpyDeviceToHost, B->st[i]));
      ++launched;
    }
    if (!launched) break;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      CK(cudaStreamSynchronize(B->st[i]));
      pmg_handle* h = B->h[i];
      int it = h->iter_host[0];
      total[i] += it;
      int extra = std::max(0, it - 1);
      for (int k = 0; k < PMG_K_COUNT; ++k) {
        h->launches[k] += h->loop64.init_launches[k] + (int64_t)extra * h->loop64.body_launches[k];
        h->bytes[k] += h->loop64.init_bytes[k] + extra * h->loop64.body_bytes[k];
        h->flops[k] += h->loop64.init_flops[k] + extra * h->loop64.body_flops[k];
      }
    }
  }
  // phase 3: results
  pmg_status result = PMG_OK;
  for (int i = 0; i < n; ++i) {
    pmg_handle* h = B->h[i];
    double bb = h->scal_host[SLOT_BB];
    loc[i].iterations = total[i];
    if (loc[i].status == PMG_OK) {
      double rel = bb > 0.0 ? std::sqrt(h->scal_host[SLOT_RR64] / bb) : 0.0;
      loc[i].rel_residual = rel;
      if (!(rel <= h->opts.tol)) loc[i].status = std::isfinite(rel) ? PMG_ERR_NOT_CONVERGED : PMG_ERR_NONFINITE;
    }
    if (loc[i].status != PMG_OK && result == PMG_OK) {
      result = (pmg_status)loc[i].status;
      fail(result, "a batch problem failed (see its info)");
    }
    CK(cudaMemcpyAsync(pout[i], h->x, h->N * sizeof(double), cudaMemcpyDeviceToDevice, B->st[i]));
    CK(cudaEventRecord(B->done[i], B->st[i]));
    CK(cudaStreamWaitEvent(cs, B->done[i], 0));
  }
  CK(cudaStreamSynchronize(cs));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < n; ++i) {
    loc[i].seconds = secs;
    if (infos) infos[i] = loc[i];
  }
  return result;
}

pmg_status pmg_solve_host(pmg_handle* h, const double* b, const double* pD, const double* x0, double* p_out,
                          pmg_solve_info* info, void* stream) {
  CKS(check_handle(h));
  if (!b || !pD || !p_out) return fail(PMG_ERR_INVALID, "b, p_dirichlet and p_out must be non-NULL");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  size_t N = h->N;
  if (!h->io) {
    cudaError_t e;
    h->io = h->alloc<double>(4 * N, e);
    if (e != cudaSuccess) { h->io = nullptr; return fail(PMG_ERR_OOM, "device allocation failed"); }
  }
  double *dout = h->io, *db = h->io + N, *dpd = h->io + 2 * N, *dx0 = h->io + 3 * N;
  CK(cudaMemcpyAsync(db, b, N * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dpd, pD, N * sizeof(double), cudaMemcpyHostToDevice, st));
  if (x0) CK(cudaMemcpyAsync(dx0, x0, N * sizeof(double), cudaMemcpyHostToDevice, st));
  pmg_status s = pmg_solve(h, db, dpd, x0 ? dx0 : nullptr, dout, info, stream);
  CK(cudaMemcpyAsync(p_out, dout, N * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

}  // extern "C"
