// Launchers of the device kernels (host-callable, no device code here).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "pmg_common.cuh"

namespace pmg {

struct ConvDims {
  int S, C, O, X, K;  // samples, input channels, output channels, positions, taps
};
struct NnScales {
  double eta, deta, p, dp;  // surface, surface change, pressure, pressure change
};

// Device scalar slots.  A Krylov solve uses one group of five consecutive slots
// (offsets below) starting at its base: GROUP_OUTER or GROUP_INNER.
enum Slot {
  SLOT_RR = 0,      // ||r||^2 of the current (recursive) residual
  SLOT_PAP = 1,     // <p, A p>
  SLOT_RZ = 2,      // <r, z>
  SLOT_RZOLD = 3,   // previous <r, z>
  SLOT_ZRO = 4,     // <z, r_old> (flexible CG)
  GROUP_OUTER = 0,
  GROUP_INNER = 8,
  SLOT_BB = 16,     // ||b~||^2 (lifted right-hand side)
  SLOT_RR64 = 17,   // ||b~ - A x||^2 of the FP64 outer residual
  SLOT_AUX = 18,    // residual norms requested outside a solve
  SLOT_GM_RES = 21,   // device-side GMRES: |g_(j+1)|^2, the residual estimate of the cycle
  SLOT_GM_BREAK = 22, // device-side GMRES: 1 after a breakdown (zero or non-finite pivot)
  SLOT_COUNT = 24
};

// Per-TU constant-table initialisers.
cudaError_t init_consts_apply(const ConstTables* host);
cudaError_t init_consts_apply_tc(const ConstTables* host);
cudaError_t init_consts_levels(const ConstTables* host);
cudaError_t init_consts_fdm32(const float* table, size_t n, const float* K, size_t nk);
cudaError_t init_consts_fdm32z(const float* table, size_t n, const float* K, size_t nk);
cudaError_t init_consts_fdm32b(const float* table, size_t n, const float* K, size_t nk);
cudaError_t init_consts_stepper(const ConstTables* host);
cudaError_t init_consts_apply_bathy(const ConstTables* host);
cudaError_t init_consts_apply_aniso(const ConstTables* host);
cudaError_t init_consts_levels_aniso(const ConstTables* host);
cudaError_t init_consts_dense(const ConstTables* host);
cudaError_t init_consts_vtail(const ConstTables* host);
cudaError_t init_consts_vtail32(const float* table, size_t n, const float* K, size_t nk);

// Layout of the FP32 Schwarz eigenvector table (constant memory of the FP32 smoother):
// for every (P, O) with 2 <= P <= MAXP and O <= (P-1)/2, eight NB x NB blocks
// (x classes 0..3, then z classes 0..3), NB = P + 1 + 2 O.
__host__ __device__ constexpr int fdm32_offset(int P, int O) {
  int off = 0;
  for (int p = 2; p <= MAXP; ++p)
    for (int o = 0; o <= MAXO; ++o) {
      if (o > (p - 1) / 2) continue;
      if (p == P && o == O) return off;
      off += 8 * (p + 1 + 2 * o) * (p + 1 + 2 * o);
    }
  return off;
}
__host__ __device__ constexpr int fdm32_table_size() { return fdm32_offset(MAXP + 1, 0); }

// Modes of the actual-geometry operator kernel (CurvedArgs.mode).
enum { MODE_APPLY = 0, MODE_RESIDUAL = 1, MODE_DOT = 2, MODE_DIV = 3 };

struct CurvedArgs {
  Shape s;
  int mode;            // 0 apply (masked), 1 residual b - A x, 2 y = A x with <x, y>, 3 divergence load
  const void* x;
  const void* x2;
  const void* b;
  void* y;
  const void* geo;     // column factors (type of the operator)
  const void* sigma;   // [NZ] (type of the operator)
  double scale;
  int mask_input;
  double* result;
  Scratch sc;
  int threads = 256;   // CTA size (autotuned; 64..512)
  int tc = 0;          // FP32 only: 0 CUDA cores, 1 BF16 tensor cores, 3 BF16 hi/lo split
  int mix = 0;         // FP64 / double-float apply and residual: the mixed-stage operator
  const void* geo5 = nullptr;  // its column factors [Nx][P+1][5] (FP64)
  int bathy = 0;       // varying still-water depth: the six-factor operator (CUDA cores)
  const void* geo6 = nullptr;  // its column factors [Nx][P+1][6] (type of the operator)
};
template <typename T> cudaError_t curved_op(const CurvedArgs& a, cudaStream_t st);
cudaError_t curved_op_tc(const CurvedArgs& a, cudaStream_t st);
template <typename T> cudaError_t curved_op_bathy(const CurvedArgs& a, cudaStream_t st);
// Column factors of the actual-geometry operator.  hcol: still-water depth per node column
// (NULL: the constant h).  div = 0 writes [A, B, C, E] (constant depth only), div = 1 the
// divergence-load factors [w d dsig/2, w d_x, w dx/2, w h_x]; geometry_bathy writes the six
// factors [A, B, C, d_x, w h_x, h_x] of the operator over a varying depth.
template <typename T>
cudaError_t geometry(const Shape& s, const double* eta, double h, const double* hcol, double dx, double dsig,
                     int div, T* geo, int* status, cudaStream_t st);
template <typename T>
cudaError_t geometry_bathy(const Shape& s, const double* eta, const double* hcol, double dx, double dsig,
                           T* geo, int* status, cudaStream_t st);
cudaError_t geometry_mixed(const Shape& s, const double* eta, const double* etap, double h, double dx, double dsig,
                           double* geo, int* status, cudaStream_t st);
// hcol: depth per node column (NULL: h); mb: bottom edge weights per node column, the sum
// over the column's elements of w_i (dx/2) sqrt(1 + h_x^2) (NULL: mX dx/2, a flat bottom)
cudaError_t rhs_source(const Shape& s, const double* eta, double h, const double* hcol, double dx, double dsig,
                       const double* mX, const double* mZ, const double* mb, const double* f, const double* gb,
                       const double* gl, const double* gr, double* b, cudaStream_t st);

struct FlatArgs {
  Shape s;
  const void* x;
  const void* b;
  void* y;
  double cx, cz;
  const void* mX;
  const void* mZ;
  int residual;
  int threads = 256;   // > 0: slab CTA size; < 0: node-parallel kernel with -threads per CTA;
                       // a tiled-shape code (flat_tile_code_ok): the tiled kernel
  // varying depth: per element column x-stiffness [Nx][P+1][P+1] with cx folded in (then
  // cx = cz = 1 and mX holds the depth-weighted x weights)
  const void* Kx = nullptr;
  // bulk-staged kernel (flat_bulk_code_ok): bound of its mbarrier wait and the flag it
  // raises when the wait gives up
  long long wait_cycles = 0;
  int* timeout_flag = nullptr;
};
template <typename T> cudaError_t flat_op(const FlatArgs& a, cudaStream_t st);
// Launch code of the bulk-staged FP32 level operator: 1000 + threads per CTA (64..512,
// whole warps); one CTA per element column, the x slab (and b) staged by TMA bulk copies.
inline bool flat_bulk_code_ok(int code) {
  return code >= 1064 && code <= 1512 && code % 32 == 1000 % 32;
}

// Tiled-variant CTA shapes, coded in the launch parameter as 10000 + 100 EXT + ZT
// (EXT element columns of 8, 16 or 32; ZT element rows of 4 or 8; at most 256 threads).
inline bool flat_tile_code_ok(int code) {
  if (code < 10000) return false;
  int ext = (code / 100) % 100, zt = code % 100;
  return (ext == 8 || ext == 16 || ext == 32) && (zt == 4 || zt == 8) && code / 10000 == 1 &&
         (ext * zt) % 32 == 0 && ext * zt <= 256;
}


struct FdmArgs {
  Shape s;
  int overlap;
  const void* r;
  void* x;
  int post;
  double omega;
  const void* Vx;
  const void* Vz;
  const void* invden;
  const void* wx;
  const void* wz;
  Scratch sc;
  int threads = 256;
  // FP32 sweep only: with b set, the sweep forms r = b - A x itself (r is ignored) and
  // xout must differ from x; xzero: the iterate in is zero and is not read
  void* xout = nullptr;
  int xzero = 0;
  const void* b = nullptr;
  double cx = 0.0, cz = 0.0;
  const void* mX = nullptr;
  const void* mZ = nullptr;
  int xpercol = 0;  // generic sweep: Vx / invden hold one x-class per element column
  int overlap_z = -1;  // overlap along sigma (-1: overlap)
  // FP32 sweep split along z (k_fdm32z): zc > 0 element rows per CTA, TMA-staged slabs
  // (r and x 16-byte aligned, no fused residual; xout may differ from x); its bounded
  // wait raises *timeout_flag
  int zc = 0;
  long long wait_cycles = 1ll << 31;
  int* timeout_flag = nullptr;
};

// Shared-memory layout of the z-split FP32 sweep (k_fdm32z.cu), in floats unless noted:
// residual rows [NB][RP] (reused for the update U [NB][UP]), iterate rows [NB][XP],
// x-transformed rows [NB][TP], z-transformed blocks [zc + 2][NB][NB], z eigenvectors and
// inverse eigenvalue sums [8][NB][NB], row and column weights, then 2 NB + 1 ints and the
// mbarrier.  RP and XP are multiples of 4 floats so that every staged column starts on a
// 16-byte boundary, and leave room for the widening of a copy to 16-byte boundaries.
struct Fdm32zLayout {
  int TRmax, RP, XP, TP, UP, T3n;
  size_t bar_off, bytes;
};
__host__ __device__ inline Fdm32zLayout fdm32z_layout(int P, int O, int zc) {
  Fdm32zLayout L;
  const int NB = P + 1 + 2 * O;
  L.TRmax = (zc + 2) * P + 2 * O + 1;
  L.RP = (L.TRmax + 6 + 3) & ~3;
  L.XP = (zc * P + 6 + 3) & ~3;
  L.TP = L.TRmax | 1;
  L.UP = zc * P;
  L.T3n = (zc + 2) * NB * NB;
  const size_t floats = (size_t)NB * (L.RP + L.XP + L.TP) + L.T3n + 8 * NB * NB + L.TRmax + NB;
  const size_t off = (floats + 2 * NB + 1) * 4;
  L.bar_off = (off + 15) & ~(size_t)15;
  L.bytes = L.bar_off + 16;
  return L;
}
bool fdm32z_usable(const FdmArgs& a);
cudaError_t fdm_smooth32z(const FdmArgs& a, cudaStream_t st);  // the z-split sweep (k_fdm32z.cu)
// A forced z-split sweep shape, coded 1000 zc + threads (1 <= zc <= 64 element rows per
// CTA, 32..256 threads in whole warps).
inline bool sweep_code_ok(int code) {
  const int zc = code / 1000, thr = code % 1000;
  return zc >= 1 && zc <= 64 && thr >= 32 && thr <= 256 && thr % 32 == 0;
}
template <typename T> cudaError_t fdm_smooth(const FdmArgs& a, cudaStream_t st);
// Dense additive Schwarz (k_dense.cu): block inverses of the level operator described by
// the per-column factors geo [Nx][P+1][4] (A, B, C, E as the operator kernels) and sigma
// rows, FP64 and FP32 [Nx*Nz][NB*NB]; a sweep x += omega (W) sum R^T A_e^-1 R (W) r with
// the per-subdomain scratch U [Nx*Nz][NB].
size_t dense_block_elems(const Shape& s, int ox, int oz);
// the fine surface polynomial of each cell at a level's nodes: out = E eta per cell
cudaError_t eta_level(const Shape& fine, const Shape& lev, const double* E, const double* eta, double* out,
                      cudaStream_t st);
cudaError_t dense_setup(const Shape& s, int ox, int oz, const double* geo, const double* sigma, double* inv64,
                        float* inv32, cudaStream_t st);
template <typename T>
cudaError_t dense_sweep(const Shape& s, int ox, int oz, const T* inv, const T* r, T* x, const T* wx, const T* wz,
                        int post, double omega, T* U, cudaStream_t st);
// Level operator, generic sweep and actual-geometry operator for different orders along x
// and sigma (s.pz() != s.P): the pairs of the paper's scaling study (k_levels_aniso.cu,
// k_apply_aniso.cu); other pairs return cudaErrorInvalidValue.
template <typename T> cudaError_t flat_op_aniso(const FlatArgs& a, cudaStream_t st);
template <typename T> cudaError_t fdm_smooth_aniso(const FdmArgs& a, cudaStream_t st);
template <typename T> cudaError_t curved_op_aniso(const CurvedArgs& a, cudaStream_t st);
bool aniso_pair_supported(int P, int PZ, bool fine);
// (P, PZ) pairs with kernels: the finest levels of the scaling study (order_z = 8) and the
// levels that its semi-coarsening visits
#define PMG_ANISO_FINE(X) X(2, 8) X(3, 8) X(4, 8) X(5, 8) X(6, 8) X(7, 8) X(9, 8) X(10, 8)
#define PMG_ANISO_COARSE(X) X(2, 5) X(3, 5) X(4, 5) X(2, 3)
// FP32 sweep with the eigenvectors in constant memory (k_fdm32.cu; the z-split form in
// k_fdm32z.cu, the batched form in k_fdm32_batch.cu)
cudaError_t fdm_smooth32(const FdmArgs& a, cudaStream_t st);

struct TransferArgs {
  Shape f, c;
  const void* in;
  void* out;
  const double* J;     // transfer along x, [(Pf+1)][(Pc+1)]
  int threads = 256;
  // restriction only: with xf set, `in` is the fine right-hand side and the kernel
  // restricts r = in - A_f xf (flat level operator cx, cz, assembled weights mX, mZ)
  const void* xf = nullptr;
  double cx = 0.0, cz = 0.0;
  const void* mX = nullptr;
  const void* mZ = nullptr;
  const double* Jz = nullptr;  // transfer along sigma when the orders differ (NULL: J)
};
template <typename T> cudaError_t transfer(const TransferArgs& a, int restrict_, cudaStream_t st);

struct CoarseArgs {
  int NX1, NZ1, periodic, nsteps;
  const double* V;     // [Nz][Nz]
  const double* coef;  // [Nz][nsteps][NX1][2]
  const double* inv;   // [Nz][NX1]
  double* work;        // [Nz][NX1]
  double* pcr_buf;     // [Nz][2][NX1] when 2 NX1 doubles exceed the shared-memory budget
};
template <typename T> cudaError_t coarse_solve(const CoarseArgs& a, const void* b, void* x, cudaStream_t st);

// Fused coarse V-cycle (k_vtail.cu): the FP32 V-cycle from one level down to the order-1
// coarse solve and back up in one cooperative launch.  The steps are recorded from the
// launch-per-step V-cycle: sweeps (slab form, split residual), level residuals (flat,
// constant depth), restrictions and prolongations, and the coarse solve.
enum { VT_SWEEP = 0, VT_RESID = 1, VT_RESTRICT = 2, VT_PROLONG = 3, VT_COARSE = 7 };
constexpr int kVtMaxP = 4;          // highest level order the fused kernel is built for
constexpr int kVtMaxOps = 160;      // steps of one fused V-cycle (grid barriers between them)
constexpr int kVtMaxSteps = 64;     // sweeps, residuals and transfers, each
constexpr int kVtMaxThreads = 256;  // CTA size bound of the fused kernel
constexpr size_t kVtPcrSmem = 48 * 1024;  // larger cyclic reductions ping-pong in global memory
struct VtStep {
  int kind;
  FdmArgs fdm;       // VT_SWEEP
  FlatArgs flat;     // VT_RESID
  TransferArgs xfer; // VT_RESTRICT, VT_PROLONG
};
// Builds the device table of a fused V-cycle (owned by the caller, one cudaFree): the
// steps in order, the coarse solve's arguments with its FP32 right-hand side cb and
// solution cx, the grid barrier words bar[2] (zero) and the timeout flag.
// cudaErrorInvalidValue when a step is not of the supported forms.  *smem: dynamic shared
// memory per CTA.
cudaError_t vtail_table(const VtStep* steps, int n, const CoarseArgs& co, const void* cb, void* cx, unsigned* bar,
                        int* timeout_flag, void** table, size_t* smem);
// CTAs of the fused kernel resident per SM at this CTA size and shared memory
cudaError_t vtail_occupancy(int threads, size_t smem, int* per_sm);
// Cooperative launch of `grid` CTAs (at most the resident count times the SMs); every
// grid barrier waits at most wait_cycles SM clock cycles.
cudaError_t vtail_launch(const void* table, int grid, int threads, size_t smem, long long wait_cycles, cudaStream_t st);

template <typename TA, typename TB>
cudaError_t dot(size_t n, const TA* x, const TB* y, double* out, int shift, const Scratch& sc, cudaStream_t st);
template <typename T>
cudaError_t cg_update(size_t n, T* x, T* r, const T* p, const T* w, T* r_old, double* s, const Scratch& sc,
                      cudaStream_t st, float* r32 = nullptr);  // r32: also write (float)r
template <typename T, typename TZ = T>
cudaError_t rz(size_t n, const T* r, const TZ* z, const T* r_old, double* s, const Scratch& sc, cudaStream_t st);
template <typename T, typename TZ = T>
cudaError_t p_update(size_t n, T* p, const TZ* z, const double* s, int flexible, int first, cudaStream_t st);
cudaError_t to_f32_scaled(size_t n, const double* x, float* y, const double* s, int slot, cudaStream_t st);
cudaError_t add_f32_scaled(size_t n, double* x, const float* c, const double* s, int slot, cudaStream_t st);
template <typename T> cudaError_t add(size_t n, T* x, const T* y, cudaStream_t st);
cudaError_t cast_f32(size_t n, const double* x, float* y, cudaStream_t st);
// GMRES: h[k] = <w, V_k> (k < nv, deterministic; part: >= nv * 304 doubles, cnt zeroed),
// w += sign sum_k c[k] V_k (nv <= 64), v = w / sqrt(*nrm2)
// Arnoldi kernels; jdev / nvdev (device ints): the count comes from the device-side
// Arnoldi index (nv = j + 1 for the dot and scale, nv = *nvdev + nvadd for the axpy)
cudaError_t gmres_mdot(size_t n, const double* w, const double* V, int nv, double* h, double* part, unsigned* cnt,
                       cudaStream_t st, const int* jdev = nullptr);
cudaError_t gmres_maxpy(size_t n, double* w, const double* V, int nv, const double* c, double sign, cudaStream_t st,
                        const int* nvdev = nullptr, int nvadd = 0);
cudaError_t gmres_scale(size_t n, const double* w, const double* nrm2, double* v, cudaStream_t st,
                        const int* jdev = nullptr);
cudaError_t gmres_gather(size_t n, const double* V, const int* jdev, double* v64, float* v32, cudaStream_t st);
cudaError_t gmres_scatter(size_t n, const double* z64, const float* z32, double* Z, const int* jdev, double* zw,
                          cudaStream_t st);
cudaError_t gmres_init(const double* rr, double* g, int m, int* jdev, int* capdev, int cap, int* iter,
                       cudaStream_t st);
cudaError_t gmres_givens(cudaGraphConditionalHandle hnd, const double* c1, const double* c2, const double* hn2,
                         double* H, double* cs, double* sn, double* g, int m, int* jdev, const int* capdev,
                         int* iter, double tol2, const double* bb, double* out, cudaStream_t st);
cudaError_t gmres_backsub(const double* H, const double* g, double* y, int m, const int* jdev, cudaStream_t st);
// time-stepper kernels (k_stepper.cu)
cudaError_t gradient(const Shape& s, const double* f, double* fx, double* fz, const double* eta, const double* sigma,
                     double h, double dx, double dsig, cudaStream_t st,
                     const double* hcol = nullptr);
cudaError_t surface_slope(const Shape& s, const double* eta, double dx, double* etax, cudaStream_t st);
cudaError_t spectral_filter(const Shape& s, const double* f, double* out, const double* F, int surface,
                            cudaStream_t st);
cudaError_t forcing(size_t N, int NZ, const double* u, const double* w, const double* ux, const double* uz,
                    const double* wx, const double* wz, const double* etax, double g, double* Fu, double* Fw,
                    cudaStream_t st);
cudaError_t rates(size_t N, int NZ, const double* sigma, const double* u, const double* w, const double* uz,
                  const double* wz, const double* Fu, const double* Fw, const double* px, const double* pz,
                  const double* etax, double rho, double* du, double* dw, double* deta, cudaStream_t st);
cudaError_t axpy(size_t n, double a, const double* x, const double* y, double* out, cudaStream_t st);
cudaError_t cast_f64(size_t n, const float* x, double* y, cudaStream_t st);
cudaError_t init_x(size_t n, int NZ, double* x, const double* x0, const double* pD, int* status, cudaStream_t st);
cudaError_t check_finite(size_t n, const double* v, int* status, cudaStream_t st);
// Arm the fence-free exchange slots (pmg_common.cuh swap_exchange) with the empty marker.
cudaError_t arm_exchange(void* buf, size_t n8);  // synchronous, at set-up
cudaError_t arm_exchange_f64(void* buf, size_t n8, cudaStream_t st);
cudaError_t loop_cond(cudaGraphConditionalHandle hnd, const double* s, const double* bb, double thresh2, int* iter,
                      int max_iter, cudaStream_t st);

// ---- batched launches over the problems of a batch (one launch per stage) ------------
// Each *_batch_table writes a device table (cudaMalloc'ed, owned and freed by the caller)
// whose range i is problem prob[i] with the arguments a[i]; `active` (device, one int per
// problem of the batch, or NULL for all) decides per launch which ranges work (the others
// return at once); *nctas is the grid of the launch, *smem its dynamic shared memory.  The
// sweep, level-operator and outer-operator tables hold one order (and overlap) each: their
// kernels are instantiated per order, and the launch names it.
cudaError_t fdm32_batch_table(const FdmArgs* a, const int* prob, int n, const int* active, void** table, int* nctas,
                              size_t* smem);
cudaError_t fdm32_batch_launch(const void* table, int P, int O, int nctas, int threads, size_t smem, cudaStream_t st);
cudaError_t flat_batch_table(const FlatArgs* a, const int* prob, int n, const int* active, int threads, void** table,
                             int* nctas);
cudaError_t flat_batch_launch(const void* table, int P, int nctas, int threads, cudaStream_t st);
cudaError_t transfer_batch_table(const TransferArgs* a, const int* prob, int n, const int* active, int restrict_,
                                 void** table, int* nctas, size_t* smem);
cudaError_t transfer_batch_launch(const void* table, int restrict_, int nctas, int threads, size_t smem,
                                  cudaStream_t st);
// coarse solve of every problem (b, x: the FP32 coarse-level vectors); three launches
cudaError_t coarse_batch_table(const CoarseArgs* a, const float* const* b, float* const* x, const int* prob, int n,
                               const int* active, void** table, int nctas[3], size_t* smem);
cudaError_t coarse_batch_launch(const void* table, const int nctas[3], size_t smem, cudaStream_t st);
// double-float outer operator of every problem: mode 2 (y = A x with <x, y> into *result)
// or 1 (y = b - A x with ||y||^2 into *result)
cudaError_t curved_batch_table(int mode, const CurvedArgs* a, const int* prob, int n, const int* active, void** table,
                               int* nctas, size_t* smem);
cudaError_t curved_batch_launch(int mode, const void* table, int P, int nctas, int threads, size_t smem,
                                cudaStream_t st);

// Krylov vectors and loop state of one problem of a batched flexible-CG solve (FP64 outer
// vectors, FP32 V-cycle input r32 and output z32, the handle's scalar slots and scratch).
struct VecProb {
  size_t n;
  int NZ;
  double *x, *r, *p, *w, *rold;
  float* r32;
  const float* z32;
  double* s;       // the handle's scalar slots (group GROUP_OUTER, SLOT_BB, SLOT_RR64)
  Scratch sc;
  int* status;     // the handle's status words: [0] inputs, [1] geometry
  double* bcopy;   // the problem's load vector for this solve (copied from the caller's)
  int max_iter;
  double tol2;
};
// Per-problem solve state (device, one int each): active (still iterating), first (the
// next iteration starts the CG recurrence afresh: p = z), confirm (the recursive residual
// met the tolerance or the cap: check the true residual), total (outer iterations),
// status (pmg_status of the problem).
struct BatchState {
  int *active, *first, *confirm, *total, *status;
  double *bb, *rr64;  // ||b~||^2 and the last true ||b~ - A x||^2 per problem
};
// Per-call device pointers of problem i: load vector, Dirichlet data, output pressure.
struct BatchIO {
  const double* b;
  const double* pD;
  double* out;
};
enum { VB_INIT = 0, VB_CAST_FIRST, VB_RZ, VB_P_UPDATE, VB_CG_UPDATE, VB_COPY_OUT, VB_COUNT };
// prob: problem index (into the state and io arrays) of each entry of a (NULL: 0..n-1); the
// state kernels below take the table of every problem (prob NULL).
cudaError_t vec_batch_table(const VecProb* a, int n, BatchState st, const BatchIO* io, void** table,
                            int nctas[VB_COUNT], const int* prob);
cudaError_t vec_batch_launch(int which, const void* table, const int nctas[VB_COUNT], cudaStream_t st);
// One thread per problem: after the lifted residual of x = (0, p_D) set BB, the initial
// state (inactive when the inputs failed, b~ = 0 or the start meets the tolerance).
cudaError_t batch_state_init(const void* table, int n, cudaStream_t st);
// After the CG update: count the iteration, end the recurrence's first step, flag
// problems whose recursive residual met the tolerance or the cap (or went non-finite).
cudaError_t batch_cond(const void* table, int n, cudaStream_t st);
// After the true residual of the flagged problems: finish them (tolerance met, or the cap
// reached: PMG_ERR_NOT_CONVERGED) or restart the recurrence from the true residual; then
// the while-node keeps looping while any problem is active (in_graph; *any receives the
// same flag either way: a host-driven loop reads it).
cudaError_t batch_confirm(const void* table, int n, cudaGraphConditionalHandle hnd, int in_graph, int* any,
                          cudaStream_t st);

// learned warm start (k_nn.cu)
cudaError_t nn_conv_forward(const ConvDims& d, const float* X, const float* W, const float* b, float* Y,
                            cudaStream_t st);
cudaError_t nn_conv_backward_input(const ConvDims& d, const float* dY, const float* W, float* dX, cudaStream_t st);
cudaError_t nn_conv_backward_weight(const ConvDims& d, const float* X, const float* dY, float* dW, cudaStream_t st);
cudaError_t nn_bias_grad(const ConvDims& d, const float* dY, float* db, cudaStream_t st);
cudaError_t nn_tanh(size_t n, float* y, cudaStream_t st);
cudaError_t nn_tanh_back(size_t n, const float* y, float* dy, cudaStream_t st);
cudaError_t nn_loss(int S, int NZ, int X, const float* y, const float* t, float* dy, double lam, double* loss,
                    cudaStream_t st);
cudaError_t nn_adam(size_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                    int t, cudaStream_t st);
cudaError_t nn_pack(int X, int NZ, int Q, const double* eta, const double* eta_prev, const double* etax,
                    const double* p, NnScales sc, float* in, cudaStream_t st);
cudaError_t nn_unpack(int X, int NZ, const double* p, const float* out, double s_dp, double* x0, cudaStream_t st);
cudaError_t nn_target(int X, int NZ, const double* p, const double* pprev, double s_dp, float* tgt, cudaStream_t st);

}  // namespace pmg
