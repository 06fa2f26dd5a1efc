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
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_apply)

namespace pmg {

enum { MODE_APPLY = 0, MODE_RESIDUAL = 1, MODE_DOT = 2, MODE_DIV = 3 };

template <typename T>
struct CurvedParams {
  Shape s;
  const T* x;       // input (MODE_DIV: u)
  const T* x2;      // MODE_DIV: w
  const T* b;       // MODE_RESIDUAL: load vector
  T* y;             // output
  const T* geo;     // [Nx][P+1][4]: A, B, C, E
  const T* sigma;   // [NZ]
  T scale;          // MODE_DIV: scale
  int mask_input;   // 1: surface-row input read as zero
  double* result;   // MODE_RESIDUAL: ||r||^2, MODE_DOT: <x, y>
  Scratch sc;
};

template <int P, typename T, int MODE>
__global__ void __launch_bounds__(512) k_curved(CurvedParams<T> p) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int L = Nz * n;
  const int ex = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);   // [n][NZp]   input slab, later Y
  T* Ur = X + n * NZp;                      // [n][NZp]   U_r per node row
  T* Ws = Ur + n * NZp;                     // [Nz][n][n] (ez, j, i): U_s then W_s
  T* Wr = Ws + L * n;                       // [Nz][n][n] (ez, j, i): W_r
  T* G = Wr + L * n;                        // [n][4]
  T* SG = G + 4 * n;                        // [NZ] sigma
  T* BB = SG + NZ;                          // [n][NZp] b (MODE_RESIDUAL) or x (MODE_DOT) of the slab
  size_t red_off = (((size_t)(3 * n * NZp + 2 * L * n + 4 * n + NZ) * sizeof(T)) + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem_raw + red_off);  // 34 doubles
  int* s_flag = reinterpret_cast<int*>(red + 34);
  T* Y = X;

  const int col0 = ex * P;
  // ---- load the slab, the column factors and sigma
  for_slab(n, NZ, [&](int i, int iz) {
    size_t g = (size_t)wrap_col(s, col0 + i) * NZ + iz;
    bool ok = !(MODE != MODE_DIV && p.mask_input && iz == NZ - 1);
    cp_async_elem(&X[i * NZp + iz], p.x + g, ok);
    if (MODE == MODE_DIV) cp_async_elem(&Ur[i * NZp + iz], p.x2 + g, true);
    if (MODE == MODE_RESIDUAL) cp_async_elem(&BB[i * NZp + iz], p.b + g, true);
    if (MODE == MODE_DOT) cp_async_elem(&BB[i * NZp + iz], p.x + g, ok);  // X is reused for Y
  });
  cp_async_wait_all();
  for (int t = threadIdx.x; t < 4 * n; t += blockDim.x) G[t] = p.geo[(size_t)ex * 4 * n + t];
  for (int t = threadIdx.x; t < NZ; t += blockDim.x) SG[t] = p.sigma[t];
  __syncthreads();

  if (MODE != MODE_DIV) {
    // ---- phase 1: U_r along x, one node row per thread
    for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
      T xv[n];
#pragma unroll
      for (int m = 0; m < n; ++m) xv[m] = X[m * NZp + iz];
#pragma unroll
      for (int i = 0; i < n; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < n; ++m) acc += CT<T>::D(cT, P, i, m) * xv[m];
        Ur[i * NZp + iz] = acc;
      }
    }
    // ---- phase 2: U_s along sigma, one (column i, element ez) per thread
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      int i = t % n, ez = t / n;
      T xv[n];
#pragma unroll
      for (int m = 0; m < n; ++m) xv[m] = X[i * NZp + ez * P + m];
#pragma unroll
      for (int j = 0; j < n; ++j) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < n; ++m) acc += CT<T>::D(cT, P, j, m) * xv[m];
        Ws[(ez * n + j) * n + i] = acc;
      }
    }
    __syncthreads();
    // ---- phase 3: pointwise metric
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
      int i = t % n, r = t / n, j = r % n, ez = r / n;
      int iz = ez * P + j;
      T wj = CT<T>::w(cT, P, j);
      T sg = SG[iz];
      T ur = Ur[i * NZp + iz];
      T us = Ws[t];
      T grr = wj * G[i * 4 + 0];
      T grs = -wj * sg * G[i * 4 + 1];
      T gss = wj * G[i * 4 + 2] * (T(1) + sg * sg * G[i * 4 + 3]);
      Wr[t] = grr * ur + grs * us;
      Ws[t] = grs * ur + gss * us;
    }
  } else {
    // ---- divergence load vector: W_r = w_i w_j (d dsig/2) u, W_s = w_i w_j (dx/2)(w - sigma d_x u)
    // Column factors in this mode: A = w_i d dsig/2, B = w_i d_x, C = w_i dx/2.
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
      int i = t % n, r = t / n, j = r % n, ez = r / n;
      int iz = ez * P + j;
      T wj = CT<T>::w(cT, P, j);
      T u = X[i * NZp + iz], w = Ur[i * NZp + iz];
      Wr[t] = p.scale * wj * G[i * 4 + 0] * u;
      Ws[t] = p.scale * wj * (G[i * 4 + 2] * w - SG[iz] * G[i * 4 + 1] * (G[i * 4 + 2] / CT<T>::w(cT, P, i)) * u);
    }
  }
  __syncthreads();
  // ---- phase 4a: x-contraction Y[i][iz] = sum_k D[k][i] sum_{ez owning iz} W_r
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    int ez = min(iz / P, Nz - 1), j = iz - ez * P;
    T wv[n];
#pragma unroll
    for (int k = 0; k < n; ++k) wv[k] = Wr[(ez * n + j) * n + k];
    if (j == 0 && ez > 0) {
#pragma unroll
      for (int k = 0; k < n; ++k) wv[k] += Wr[((ez - 1) * n + P) * n + k];
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < n; ++k) acc += CT<T>::D(cT, P, k, i) * wv[k];
      Y[i * NZp + iz] = acc;
    }
  }
  __syncthreads();
  // ---- phase 4b: sigma-contraction of the rows [ez P, ez P + P) owned by (i, ez)
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    int i = t % n, ez = t / n;
    T wv[n];
#pragma unroll
    for (int k = 0; k < n; ++k) wv[k] = Ws[(ez * n + k) * n + i];
    T below = T(0);
    if (ez > 0) {
#pragma unroll
      for (int k = 0; k < n; ++k) below += CT<T>::D(cT, P, k, P) * Ws[((ez - 1) * n + k) * n + i];
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T acc = (j == 0) ? below : T(0);
#pragma unroll
      for (int k = 0; k < n; ++k) acc += CT<T>::D(cT, P, k, j) * wv[k];
      Y[i * NZp + ez * P + j] += acc;
    }
    if (ez == Nz - 1) {  // surface row: used by MODE_DIV only (masked otherwise)
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < n; ++k) acc += CT<T>::D(cT, P, k, P) * wv[k];
      Y[i * NZp + NZ - 1] += acc;
    }
  }
  __syncthreads();

  // ---- epilogue
  auto finish = [&](int ix, int i, int iz, T val, Acc<T>& ac) {  // i: local column of ix
    size_t g = (size_t)ix * NZ + iz;
    bool top = iz == NZ - 1;
    if (MODE == MODE_APPLY) {
      p.y[g] = top ? p.x[g] : val;
    } else if (MODE == MODE_RESIDUAL) {
      T r = top ? T(0) : BB[i * NZp + iz] - val;
      p.y[g] = r;
      ac.fma(r, r);
    } else if (MODE == MODE_DOT) {
      T v = top ? T(0) : val;
      p.y[g] = v;
      ac.fma(BB[i * NZp + iz], v);
    } else {
      p.y[g] = top ? T(0) : val;
    }
  };
  Acc<T> acc;
  for_slab(P - 1, NZ, [&](int c, int iz) { finish(col0 + 1 + c, c + 1, iz, Y[(c + 1) * NZp + iz], acc); });
  const int nedges = s.periodic ? s.Nx : s.Nx + 1;
  T* eb = reinterpret_cast<T*>(p.sc.edgebuf);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    int i = side == 0 ? 0 : P;
    int e = side == 0 ? ex : (s.periodic ? (ex + 1) % s.Nx : ex + 1);
    bool single = !s.periodic && (e == 0 || e == s.Nx);
    int ix = e * P;
    Acc<T> eacc;
    if (single) {
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) finish(ix, i, iz, Y[i * NZp + iz], eacc);
    } else {
      T* buf = eb + (size_t)e * NZ;
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) atomic_add_t(buf + iz, Y[i * NZp + iz]);
      if (!edge_arrive(p.sc.edgecnt + e, 2, s_flag)) continue;
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) finish(ix, i, iz, take_t(buf + iz), eacc);
    }
    if (MODE == MODE_RESIDUAL || MODE == MODE_DOT) {
      double v = block_sum(eacc.value(), red);
      if (threadIdx.x == 0) p.sc.edgepart[e] = v;
    }
  }
  if (MODE == MODE_RESIDUAL || MODE == MODE_DOT) {
    double v = block_sum(acc.value(), red);
    grid_reduce(p.sc, v, nedges, p.result, red, s_flag);
  }
}

template <int P, typename T>
__global__ void k_geometry(Shape s, const double* eta, double h, double dx, double dsig, int div,
                           T* geo, int* status) {
  // one thread per (element column, local column i)
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n = P + 1;
  if (t >= s.Nx * n) return;
  int ex = t / n, i = t % n;
  double dd = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) dd += cT.D[P][i][m] * eta[wrap_col(s, ex * P + m)];
  dd *= 2.0 / dx;
  double d = eta[wrap_col(s, ex * P + i)] + h;
  if (!(d > 0.0) || !isfinite(dd)) atomicExch(status, 1);
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
    g[3] = (T)0;
  }
}

// b = -w_i w_j J f + edge terms; J = (dx/2)(dsig/2) d summed over the elements of a node
// equals d (dx dsig / 4) mX mZ with mX, mZ the assembled LGL weights.
__global__ void k_rhs_source(Shape s, const double* eta, double h, double dx, double dsig,
                             const double* mX, const double* mZ, const double* f, const double* gb,
                             const double* gl, const double* gr, double* b) {
  size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t N = (size_t)s.NX * s.NZ;
  if (g >= N) return;
  int ix = (int)(g / s.NZ), iz = (int)(g % s.NZ);
  if (iz == s.NZ - 1) { b[g] = 0.0; return; }
  double d = eta[ix] + h;
  double v = -f[g] * d * (dx * dsig * 0.25) * mX[ix] * mZ[iz];
  if (iz == 0 && gb) v += mX[ix] * (dx * 0.5) * gb[ix];
  if (!s.periodic) {
    if (ix == 0 && gl) v += mZ[iz] * (dsig * 0.5) * d * gl[iz];
    if (ix == s.NX - 1 && gr) v += mZ[iz] * (dsig * 0.5) * d * gr[iz];
  }
  b[g] = v;
}

template <typename T>
static size_t curved_smem(int P, int NZ, int Nz) {
  int n = P + 1, NZp = slab_pitch(NZ), L = Nz * n;
  size_t e = (size_t)3 * n * NZp + (size_t)2 * L * n + 4 * n + NZ;
  return ((e * sizeof(T) + 15) & ~(size_t)15) + 34 * sizeof(double) + 16;
}

template <int P, typename T, int MODE>
static cudaError_t launch_curved_p(const CurvedParams<T>& prm, int threads, cudaStream_t st) {
  size_t sm = curved_smem<T>(P, prm.s.NZ, prm.s.Nz);
  auto k = k_curved<P, T, MODE>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_curved(const CurvedParams<T>& prm, int threads, cudaStream_t st) {
  switch (prm.s.P) {
#define PMG_CASE(PP) case PP: return launch_curved_p<PP, T, MODE>(prm, threads, st);
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t curved_op(const CurvedArgs& a, cudaStream_t st) {
  CurvedParams<T> p;
  p.s = a.s;
  p.x = (const T*)a.x;
  p.x2 = (const T*)a.x2;
  p.b = (const T*)a.b;
  p.y = (T*)a.y;
  p.geo = (const T*)a.geo;
  p.sigma = (const T*)a.sigma;
  p.scale = (T)a.scale;
  p.mask_input = a.mask_input;
  p.result = a.result;
  p.sc = a.sc;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  switch (a.mode) {
    case MODE_APPLY: return launch_curved<T, MODE_APPLY>(p, thr, st);
    case MODE_RESIDUAL: return launch_curved<T, MODE_RESIDUAL>(p, thr, st);
    case MODE_DOT: return launch_curved<T, MODE_DOT>(p, thr, st);
    case MODE_DIV: return launch_curved<T, MODE_DIV>(p, thr, st);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t curved_op<double>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op<float>(const CurvedArgs&, cudaStream_t);

template <typename T>
cudaError_t geometry(const Shape& s, const double* eta, double h, double dx, double dsig, int div,
                     T* geo, int* status, cudaStream_t st) {
  int n = s.P + 1, tot = s.Nx * n, bs = 128, nb = (tot + bs - 1) / bs;
  switch (s.P) {
#define PMG_CASE(PP) case PP: k_geometry<PP, T><<<nb, bs, 0, st>>>(s, eta, h, dx, dsig, div, geo, status); break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t geometry<double>(const Shape&, const double*, double, double, double, int, double*, int*, cudaStream_t);
template cudaError_t geometry<float>(const Shape&, const double*, double, double, double, int, float*, int*, cudaStream_t);

cudaError_t rhs_source(const Shape& s, const double* eta, double h, double dx, double dsig,
                       const double* mX, const double* mZ, const double* f, const double* gb,
                       const double* gl, const double* gr, double* b, cudaStream_t st) {
  size_t N = (size_t)s.NX * s.NZ;
  int bs = 256;
  k_rhs_source<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(s, eta, h, dx, dsig, mX, mZ, f, gb, gl, gr, b);
  return cudaGetLastError();
}

}  // namespace pmg
