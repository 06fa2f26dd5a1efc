// Actual-geometry operator of the sigma-mapped SEM (Sec. 2.2, Sec. 4.2-4.3) and its
// load vectors.
//
// Per element (ex, ez) with local nodes (i, j) (i along x, j along sigma):
//   U_r = D U,  U_s = U D^T                               (reference derivatives)
//   W_r = G_rr U_r + G_rs U_s,  W_s = G_rs U_r + G_ss U_s  (metric, LGL collocation)
//   Y   = D^T W_r + W_s D                                 (test-function derivatives)
// with, from x = x*, z = sigma d(x) - h, d = eta + h (Sec. 2.2 metric formulas):
//   G_rr = w_i w_j d (dsig/dx),  G_rs = -w_i w_j sigma d_x,
//   G_ss = w_i w_j (dx/dsig) (1 + sigma^2 d_x^2) / d,
// d, d_x per element-local node column (d_x = (2/dx) D d) and sigma per node row.  The
// column factors A = w_i d dsig/dx, B = w_i d_x, C = w_i (dx/dsig)/d, E = d_x^2 are built
// once per geometry (k_geometry), so no metric field is streamed.
//
// Assembly (Sec. 4.2, global = sum of local): a CTA takes one element column; W_r of the
// two elements that share a node row are summed before the x-contraction, the sigma
// contraction of each node row is done by the thread that owns the row, and the two
// element-edge node columns are summed across CTAs by the edge exchange.
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_apply)

#include "k_curved.cuh"

namespace pmg {

// Per (element column, local column i): total depth d = eta + h and the slopes d_x, h_x of
// the element's interpolants (x-derivative (2/dx) D of the nodal values); hcol == NULL:
// constant depth h, h_x = 0.
template <int P>
__device__ __forceinline__ bool column_depth(const Shape& s, const double* eta, double h, const double* hcol,
                                             double dx, int ex, int i, double& d, double& dd, double& hx) {
  constexpr int n = P + 1;
  dd = 0.0;
  hx = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) {
    int c = wrap_col(s, ex * P + m);
    dd += cT.D[P][i][m] * eta[c];
    if (hcol) hx += cT.D[P][i][m] * hcol[c];
  }
  hx *= 2.0 / dx;
  dd = dd * (2.0 / dx) + hx;  // d_x = eta_x + h_x
  int c = wrap_col(s, ex * P + i);
  d = eta[c] + (hcol ? hcol[c] : h);
  return d > 0.0 && isfinite(dd) && isfinite(hx);
}

template <int P, typename T>
__global__ void k_geometry(Shape s, const double* eta, double h, const double* hcol, double dx, double dsig, int div,
                           T* geo, int* status) {
  // one thread per (element column, local column i)
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n = P + 1;
  if (t >= s.Nx * n) return;
  int ex = t / n, i = t % n;
  double d, dd, hx;
  if (!column_depth<P>(s, eta, h, hcol, dx, ex, i, d, dd, hx)) atomicExch(status, 1);
  double w = cT.w[P][i];
  T* g = geo + (size_t)t * 4;
  if (!div) {
    g[0] = (T)(w * d * dsig / dx);
    g[1] = (T)(w * dd);
    g[2] = (T)(w * (dx / dsig) / d);
    g[3] = (T)(dd * dd);
  } else {
    g[0] = (T)(w * d * dsig / 2.0);
    g[1] = (T)(w * dd);
    g[2] = (T)(w * dx / 2.0);
    g[3] = (T)(w * hx);
  }
}

// Over a varying still-water depth the sigma map z = sigma d(x) - h(x) gives the metric
//   G_rr = w_i w_j d dsig/dx,  G_rs = w_i w_j (h_x - sigma d_x),
//   G_ss = w_i w_j (dx/dsig) (1 + (h_x - sigma d_x)^2) / d        (Sec. 2.2)
// stored as six column factors [w d dsig/dx, w d_x, w (dx/dsig)/d, d_x, w h_x, h_x].
template <int P, typename T>
__global__ void k_geometry_bathy(Shape s, const double* eta, const double* hcol, double dx, double dsig, T* geo,
                                 int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n = P + 1;
  if (t >= s.Nx * n) return;
  int ex = t / n, i = t % n;
  double d, dd, hx;
  if (!column_depth<P>(s, eta, 0.0, hcol, dx, ex, i, d, dd, hx)) atomicExch(status, 1);
  double w = cT.w[P][i];
  T* g = geo + (size_t)t * 6;
  g[0] = (T)(w * d * dsig / dx);
  g[1] = (T)(w * dd);
  g[2] = (T)(w * (dx / dsig) / d);
  g[3] = (T)dd;
  g[4] = (T)(w * hx);
  g[5] = (T)hx;
}

// Column factors of the mixed-stage operator (stage k surface eta, stage k-1 surface etap):
// A = w d dsig/dx, B1 = w d_x' d/d', B2 = w d_x, C = w (dx/dsig)/d', E = d_x d_x'.
template <int P>
__global__ void k_geometry_mixed(Shape s, const double* eta, const double* etap, double h, double dx, double dsig,
                                 double* geo, int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n = P + 1;
  if (t >= s.Nx * n) return;
  int ex = t / n, i = t % n;
  double dd = 0.0, ddp = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) {
    int c = wrap_col(s, ex * P + m);
    dd += cT.D[P][i][m] * eta[c];
    ddp += cT.D[P][i][m] * etap[c];
  }
  dd *= 2.0 / dx;
  ddp *= 2.0 / dx;
  int c = wrap_col(s, ex * P + i);
  double d = eta[c] + h, dp = etap[c] + h;
  if (!(d > 0.0) || !(dp > 0.0) || !isfinite(dd) || !isfinite(ddp)) atomicExch(status, 1);
  double w = cT.w[P][i];
  double* g = geo + (size_t)t * 5;
  g[0] = w * d * dsig / dx;
  g[1] = w * ddp * d / dp;
  g[2] = w * dd;
  g[3] = w * (dx / dsig) / dp;
  g[4] = dd * ddp;
}

cudaError_t geometry_mixed(const Shape& s, const double* eta, const double* etap, double h, double dx, double dsig,
                           double* geo, int* status, cudaStream_t st) {
  int n = s.P + 1, tot = s.Nx * n, bs = 128, nb = (tot + bs - 1) / bs;
  switch (s.P) {
#define PMG_CASE(PP) case PP: k_geometry_mixed<PP><<<nb, bs, 0, st>>>(s, eta, etap, h, dx, dsig, geo, status); break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// b = -w_i w_j J f + edge terms; J = (dx/2)(dsig/2) d summed over the elements of a node
// equals d (dx dsig / 4) mX mZ with mX, mZ the assembled LGL weights.  The bottom edge
// term uses the arc length of the mapped bottom (mb), the walls d dsig / 2.
__global__ void k_rhs_source(Shape s, const double* eta, double h, const double* hcol, double dx, double dsig,
                             const double* mX, const double* mZ, const double* mb, const double* f,
                             const double* gb, const double* gl, const double* gr, double* b) {
  size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t N = (size_t)s.NX * s.NZ;
  if (g >= N) return;
  int ix = (int)(g / s.NZ), iz = (int)(g % s.NZ);
  if (iz == s.NZ - 1) { b[g] = 0.0; return; }
  double d = eta[ix] + (hcol ? hcol[ix] : h);
  double v = -f[g] * d * (dx * dsig * 0.25) * mX[ix] * mZ[iz];
  if (iz == 0 && gb) v += (mb ? mb[ix] : mX[ix] * (dx * 0.5)) * gb[ix];
  if (!s.periodic) {
    if (ix == 0 && gl) v += mZ[iz] * (dsig * 0.5) * d * gl[iz];
    if (ix == s.NX - 1 && gr) v += mZ[iz] * (dsig * 0.5) * d * gr[iz];
  }
  b[g] = v;
}

template <typename T>
cudaError_t curved_op(const CurvedArgs& a, cudaStream_t st) {
  if (a.s.pz() != a.s.P) return curved_op_aniso<T>(a, st);
  using IO = typename IOT<T>::type;
  CurvedParams<T> p;
  p.s = a.s;
  p.x = (const IO*)a.x;
  p.x2 = (const IO*)a.x2;
  p.b = (const IO*)a.b;
  p.y = (IO*)a.y;
  p.geo = (const IO*)a.geo;
  p.sigma = (const IO*)a.sigma;
  p.scale = from_io<T>((IO)a.scale);
  p.mask_input = a.mask_input;
  p.result = a.result;
  p.sc = a.sc;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  if (a.tc) {
    if (!std::is_same<T, float>::value || (a.mode != MODE_APPLY && a.mode != MODE_DOT) || a.bathy)
      return cudaErrorInvalidValue;
    return curved_op_tc(a, st);
  }
  if (a.bathy) {
    if (a.mix || a.mode == MODE_DIV) return cudaErrorInvalidValue;
    return curved_op_bathy<T>(a, st);
  }
  if (a.mix) {
    if constexpr (std::is_same<T, float>::value) {
      return cudaErrorInvalidValue;
    } else {
      p.geo = (const IO*)a.geo5;
      if (a.mode == MODE_APPLY) return launch_curved<T, MODE_APPLY, 0, true>(p, thr, st);
      if (a.mode == MODE_RESIDUAL) return launch_curved<T, MODE_RESIDUAL, 0, true>(p, thr, st);
      return cudaErrorInvalidValue;
    }
  }
  switch (a.mode) {
    case MODE_APPLY: return launch_curved<T, MODE_APPLY, 0>(p, thr, st);
    case MODE_RESIDUAL: return launch_curved<T, MODE_RESIDUAL, 0>(p, thr, st);
    case MODE_DOT: return launch_curved<T, MODE_DOT, 0>(p, thr, st);
    case MODE_DIV:
      if constexpr (!std::is_same<T, df64>::value) return launch_curved<T, MODE_DIV, 0>(p, thr, st);
      break;
  }
  return cudaErrorInvalidValue;
}
template cudaError_t curved_op<double>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op<float>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op<df64>(const CurvedArgs&, cudaStream_t);

template <typename T>
cudaError_t geometry(const Shape& s, const double* eta, double h, const double* hcol, double dx, double dsig,
                     int div, T* geo, int* status, cudaStream_t st) {
  if (hcol && !div) return cudaErrorInvalidValue;  // the operator over a varying depth takes six factors
  int n = s.P + 1, tot = s.Nx * n, bs = 128, nb = (tot + bs - 1) / bs;
  switch (s.P) {
#define PMG_CASE(PP) case PP: k_geometry<PP, T><<<nb, bs, 0, st>>>(s, eta, h, hcol, dx, dsig, div, geo, status); break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t geometry<double>(const Shape&, const double*, double, const double*, double, double, int, double*,
                                      int*, cudaStream_t);
template cudaError_t geometry<float>(const Shape&, const double*, double, const double*, double, double, int, float*,
                                     int*, cudaStream_t);

template <typename T>
cudaError_t geometry_bathy(const Shape& s, const double* eta, const double* hcol, double dx, double dsig,
                           T* geo, int* status, cudaStream_t st) {
  if (!hcol) return cudaErrorInvalidValue;
  int n = s.P + 1, tot = s.Nx * n, bs = 128, nb = (tot + bs - 1) / bs;
  switch (s.P) {
#define PMG_CASE(PP) case PP: k_geometry_bathy<PP, T><<<nb, bs, 0, st>>>(s, eta, hcol, dx, dsig, geo, status); break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t geometry_bathy<double>(const Shape&, const double*, const double*, double, double, double*, int*,
                                            cudaStream_t);
template cudaError_t geometry_bathy<float>(const Shape&, const double*, const double*, double, double, float*, int*,
                                           cudaStream_t);

cudaError_t rhs_source(const Shape& s, const double* eta, double h, const double* hcol, double dx, double dsig,
                       const double* mX, const double* mZ, const double* mb, const double* f, const double* gb,
                       const double* gl, const double* gr, double* b, cudaStream_t st) {
  size_t N = (size_t)s.NX * s.NZ;
  int bs = 256;
  k_rhs_source<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(s, eta, h, hcol, dx, dsig, mX, mZ, mb, f, gb, gl, gr, b);
  return cudaGetLastError();
}

// ---- batched double-float outer operator (mode 2: y = A x with <x, y>; mode 1: residual)
template <int MODE>
static cudaError_t curved_batch_table_m(const CurvedArgs* a, const int* prob, int n, const int* active, void** table,
                                        int* nctas, size_t* smem) {
  using Tab = CurvedBatch<df64, MODE>;
  Tab* h = new (std::nothrow) Tab();
  if (!h) return cudaErrorMemoryAllocation;
  h->m.nrange = n;
  h->m.active = active;
  h->m.start[0] = 0;
  size_t sm = 0;
  for (int i = 0; i < n; ++i) {
    if (a[i].s.pz() != a[i].s.P || a[i].mix || a[i].bathy || a[i].tc || a[i].s.P < 2 || a[i].s.P > MAXP ||
        a[i].s.P != a[0].s.P) {
      delete h;
      return cudaErrorInvalidValue;
    }
    CurvedParams<df64>& p = h->prm[i];
    p.s = a[i].s;
    p.x = (const double*)a[i].x;
    p.x2 = nullptr;
    p.b = (const double*)a[i].b;
    p.y = (double*)a[i].y;
    p.geo = (const double*)a[i].geo;
    p.sigma = (const double*)a[i].sigma;
    p.scale = df64(1.f);
    p.mask_input = a[i].mask_input;
    p.result = a[i].result;
    p.sc = a[i].sc;
    h->m.prob[i] = prob[i];
    h->m.start[i + 1] = h->m.start[i] + a[i].s.Nx;
    sm = std::max(sm, curved_smem<df64>(a[i].s.P, a[i].s.NZ, a[i].s.Nz, MODE == MODE_RESIDUAL));
  }
  *nctas = h->m.start[n];
  *smem = sm;
  BatchMap* maps[1] = {&h->m};
  cudaError_t e = batch_upload(h, maps, 1, table);
  delete h;
  return e;
}

cudaError_t curved_batch_table(int mode, const CurvedArgs* a, const int* prob, int n, const int* active, void** table,
                               int* nctas, size_t* smem) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  if (mode == MODE_DOT) return curved_batch_table_m<MODE_DOT>(a, prob, n, active, table, nctas, smem);
  if (mode == MODE_RESIDUAL) return curved_batch_table_m<MODE_RESIDUAL>(a, prob, n, active, table, nctas, smem);
  return cudaErrorInvalidValue;
}

template <int MODE, int P>
static cudaError_t launch_curved_batch(const void* table, int nctas, int threads, size_t smem, cudaStream_t st) {
  auto k = k_curved_batch<df64, MODE, P>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  int grid = 0;
  e = batch_grid(k, threads, smem, nctas, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(static_cast<const CurvedBatch<df64, MODE>*>(table));
  return cudaGetLastError();
}
template <int MODE>
static cudaError_t curved_batch_launch_m(const void* table, int P, int nctas, int threads, size_t smem,
                                         cudaStream_t st) {
  switch (P) {
#define PMG_CASE(PP) case PP: return launch_curved_batch<MODE, PP>(table, nctas, threads, smem, st);
    PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5) PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
  }
  return cudaErrorInvalidValue;
}
cudaError_t curved_batch_launch(int mode, const void* table, int P, int nctas, int threads, size_t smem,
                                cudaStream_t st) {
  if (mode == MODE_DOT) return curved_batch_launch_m<MODE_DOT>(table, P, nctas, threads, smem, st);
  if (mode == MODE_RESIDUAL) return curved_batch_launch_m<MODE_RESIDUAL>(table, P, nctas, threads, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace pmg
