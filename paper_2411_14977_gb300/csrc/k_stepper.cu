// Kernels of the free-surface time stepper around the pressure solve (scaffold of the
// wave-tank workload): nodal physical gradients by lumped L2 projection on the sigma-mesh
// (the paper's gradient recovery, Sec. 4), the surface slope, the explicit forcing of the
// inviscid sigma-transformed momentum equations (Sec. 2.2), the stage rates including
// the kinematic free-surface condition (Eq. freesurf1), and the modal exponential
// cut-off filter (Sec. "Spectral Filtering").  FP64.
//
// Gradient of a nodal field f on element (ex, ez), local node (i, j):
//   f_r = sum_m D[i][m] f[m][j],  f_s = sum_m D[j][m] f[i][m]
//   f_x = (2/dx) f_r + beta f_s,  f_z = gamma f_s,
//   beta = -sigma d_x (2/dsig) / d,  gamma = 2 / (d dsig)
// and the lumped-mass L2 projection averages the element values at shared nodes with
// weights w_i w_j J, which are equal on both sides of an element edge (LGL weights are
// symmetric and J is continuous), i.e. the plain mean over the elements of the node.
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_stepper)

namespace pmg {

struct GradParams {
  Shape s;
  const double* f;
  double* fx;
  double* fz;
  const double* eta;    // [NX]
  const double* sigma;  // [NZ]
  double h, dx, dsig;
  const double* hcol;   // [NX] still-water depth per node column (NULL: the constant h)
};

template <int P>
__global__ void __launch_bounds__(256) k_grad(GradParams p) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  const bool left = s.periodic || ex > 0;
  const bool last = !s.periodic && ex == s.Nx - 1;
  const int own = last ? n : P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* F = reinterpret_cast<double*>(smem_raw);  // [2P+1][NZp]: columns col0 - P ..
  double* E = F + (2 * P + 1) * NZp;                 // [2P+1] eta
  double* DX = E + 2 * P + 1;                        // [2][n] eta_x of the left and own elements
  double* SG = DX + 2 * n;                           // [NZ]
  double* HC = SG + NZ;                              // [2P+1] still-water depth
  double* HX = HC + 2 * P + 1;                       // [2][n] h_x (zero over a constant depth)
  for_slab(2 * P + 1, NZ, [&](int c, int iz) {
    bool ok = c >= P || left;
    cp_async_elem(&F[c * NZp + iz], p.f + (ok ? (size_t)wrap_col(s, col0 - P + c) * NZ + iz : 0), ok);
  });
  if (threadIdx.x < 2 * P + 1) {
    int c = threadIdx.x;
    bool ok = c >= P || left;
    E[c] = ok ? p.eta[wrap_col(s, col0 - P + c)] : 0.0;
    HC[c] = (ok && p.hcol) ? p.hcol[wrap_col(s, col0 - P + c)] : p.h;
  }
  for (int t = threadIdx.x; t < NZ; t += blockDim.x) SG[t] = p.sigma[t];
  cp_async_wait_all();
  __syncthreads();
  if (threadIdx.x < 2 * n) {
    int el = threadIdx.x / n, i = threadIdx.x % n;  // el 0: left element, 1: own element
    double acc = 0.0, hacc = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      acc += cT.D[P][i][m] * E[el * P + m];
      if (p.hcol) hacc += cT.D[P][i][m] * HC[el * P + m];
    }
    DX[el * n + i] = acc * (2.0 / p.dx);
    HX[el * n + i] = hacc * (2.0 / p.dx);
  }
  __syncthreads();
  // one thread per owned node: mean of the element values over the elements of the node
  for_slab(own, NZ, [&](int i, int iz) {
    int ec0 = (i == 0 && left) ? 0 : 1;  // element columns containing the node: left (0) and/or own (1)
    int ez_hi = min(iz / P, Nz - 1);
    int ez0 = (iz == ez_hi * P && ez_hi > 0) ? ez_hi - 1 : ez_hi;
    double sx = 0.0, sz = 0.0;
    int cnt = 0;
    for (int el = ec0; el <= 1; ++el) {
      int li = el == 0 ? P : i;            // local column in that element
      const double* Fc = F + (el * P) * NZp;  // element's first column in the slab
      double d = E[el * P + li] + HC[el * P + li];
      double hx = HX[el * n + li];
      double ddx = DX[el * n + li] + hx;  // d_x = eta_x + h_x
      for (int ez = ez0; ez <= ez_hi; ++ez) {
        int lj = iz - ez * P;
        double fr = 0.0, fs = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          fr += cT.D[P][li][m] * Fc[m * NZp + iz];
          fs += cT.D[P][lj][m] * Fc[li * NZp + ez * P + m];
        }
        double sg = SG[iz];
        // sigma_x = (h_x - sigma d_x) / d (Sec. 2.2)
        double beta = (hx - sg * ddx) * (2.0 / p.dsig) / d, gamma = 2.0 / (d * p.dsig);
        sx += (2.0 / p.dx) * fr + beta * fs;
        sz += gamma * fs;
        ++cnt;
      }
    }
    size_t g = (size_t)(col0 + i) * NZ + iz;
    p.fx[g] = sx / cnt;
    p.fz[g] = sz / cnt;
  });
}

// Spectral filter of a nodal field: per element F (x) F with the (P+1)^2 nodal filter
// matrix F = V diag(S) V^-1 (row-major, device), then the mean over the elements of each
// node (the same averaging as the gradient recovery).  Same slab layout as k_grad.
struct FilterParams {
  Shape s;
  const double* f;
  double* out;
  const double* F;  // [n][n]
};

template <int P>
__global__ void __launch_bounds__(256) k_filter(FilterParams p) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  const bool left = s.periodic || ex > 0;
  const bool last = !s.periodic && ex == s.Nx - 1;
  const int own = last ? n : P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Fs = reinterpret_cast<double*>(smem_raw);  // [2P+1][NZp]
  double* Fm = Fs + (2 * P + 1) * NZp;               // [n][n]
  for_slab(2 * P + 1, NZ, [&](int c, int iz) {
    bool ok = c >= P || left;
    cp_async_elem(&Fs[c * NZp + iz], p.f + (ok ? (size_t)wrap_col(s, col0 - P + c) * NZ + iz : 0), ok);
  });
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Fm[t] = p.F[t];
  cp_async_wait_all();
  __syncthreads();
  for_slab(own, NZ, [&](int i, int iz) {
    int ec0 = (i == 0 && left) ? 0 : 1;
    int ez_hi = min(iz / P, Nz - 1);
    int ez0 = (iz == ez_hi * P && ez_hi > 0) ? ez_hi - 1 : ez_hi;
    double sum = 0.0;
    int cnt = 0;
    for (int el = ec0; el <= 1; ++el) {
      int li = el == 0 ? P : i;
      const double* Fc = Fs + (el * P) * NZp;
      for (int ez = ez0; ez <= ez_hi; ++ez) {
        int lj = iz - ez * P;
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          double g = 0.0;
#pragma unroll
          for (int q = 0; q < n; ++q) g += Fm[lj * n + q] * Fc[m * NZp + ez * P + q];
          acc += Fm[li * n + m] * g;
        }
        sum += acc;
        ++cnt;
      }
    }
    p.out[(size_t)(col0 + i) * NZ + iz] = sum / cnt;
  });
}

// The same filter on the surface elevation (one value per node column).
template <int P>
__global__ void k_filter_surface(Shape s, const double* eta, const double* F, double* out) {
  int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= s.NX) return;
  int ex = ix / P, i = ix - ex * P;
  if (!s.periodic && ex == s.Nx) { ex = s.Nx - 1; i = P; }
  double acc = 0.0;
  int cnt = 0;
  for (int el = 0; el < 2; ++el) {
    int e = ex - el, li = el == 0 ? i : P;
    if (el == 1 && i != 0) break;
    if (e < 0) {
      if (!s.periodic) break;
      e += s.Nx;
    }
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < P + 1; ++m) v += F[li * (P + 1) + m] * eta[wrap_col(s, e * P + m)];
    acc += v;
    ++cnt;
  }
  out[ix] = acc / cnt;
}

// eta_x per node column: mean of the element-local derivatives of the surface polynomial.
template <int P>
__global__ void k_slope(Shape s, const double* eta, double dx, double* etax) {
  int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= s.NX) return;
  int ex = ix / P, i = ix - ex * P;
  if (!s.periodic && ex == s.Nx) { ex = s.Nx - 1; i = P; }
  double acc = 0.0;
  int cnt = 0;
  for (int el = 0; el < 2; ++el) {
    int e = ex - el, li = el == 0 ? i : P;
    if (el == 1 && i != 0) break;
    if (e < 0) {
      if (!s.periodic) break;
      e += s.Nx;
    }
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < P + 1; ++m) v += cT.D[P][li][m] * eta[wrap_col(s, e * P + m)];
    acc += v * (2.0 / dx);
    ++cnt;
  }
  etax[ix] = acc / cnt;
}

// F = -(u . grad) u - g eta_x e_x  (static pressure folded in: p = p_D + rho g (eta - z))
__global__ void k_forcing(size_t N, int NZ, const double* u, const double* w, const double* ux, const double* uz,
                          const double* wx, const double* wz, const double* etax, double g, double* Fu, double* Fw) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    size_t ix = i / NZ;
    Fu[i] = -(u[i] * ux[i] + w[i] * uz[i]) - g * etax[ix];
    Fw[i] = -(u[i] * wx[i] + w[i] * wz[i]);
  }
}

// Stage rates at fixed sigma: eta_t = w~ - u~ eta_x (surface row);
// du/dt = F - grad(p_D)/rho + sigma eta_t d(u)/dz  (mesh velocity z_t = sigma eta_t)
__global__ void k_rates(size_t N, int NZ, const double* sigma, const double* u, const double* w, const double* uz,
                        const double* wz, const double* Fu, const double* Fw, const double* px, const double* pz,
                        const double* etax, double rho, double* du, double* dw, double* deta) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    size_t ix = i / NZ;
    int iz = (int)(i - ix * NZ);
    size_t top = ix * NZ + NZ - 1;
    double et = w[top] - u[top] * etax[ix];
    double sg = sigma[iz];
    du[i] = Fu[i] - px[i] / rho + sg * et * uz[i];
    dw[i] = Fw[i] - pz[i] / rho + sg * et * wz[i];
    if (iz == NZ - 1) deta[ix] = et;
  }
}

// out = y + a x  (RK stage states and accumulation)
__global__ void k_axpy(size_t n, double a, const double* x, const double* y, double* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = y[i] + a * x[i];
}

static unsigned grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 1216 ? (b ? b : 1) : 1216);
}

cudaError_t gradient(const Shape& s, const double* f, double* fx, double* fz, const double* eta, const double* sigma,
                     double h, double dx, double dsig, cudaStream_t st, const double* hcol) {
  GradParams p{s, f, fx, fz, eta, sigma, h, dx, dsig, hcol};
  int NZp = slab_pitch(s.NZ);
  size_t sm = ((size_t)(2 * s.P + 1) * NZp + 2 * (2 * s.P + 1) + 4 * (s.P + 1) + s.NZ) * sizeof(double) + 16;
  switch (s.P) {
#define PMG_CASE(PP)                                                        \
  case PP: {                                                                \
    static std::atomic<unsigned long long> mask{0};                        \
    cudaError_t e = ensure_max_smem(k_grad<PP>, mask);                      \
    if (e != cudaSuccess) return e;                                         \
    k_grad<PP><<<s.Nx, 256, sm, st>>>(p);                                  \
    break;                                                                  \
  }
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t surface_slope(const Shape& s, const double* eta, double dx, double* etax, cudaStream_t st) {
  int nb = (s.NX + 127) / 128;
  switch (s.P) {
#define PMG_CASE(PP) case PP: k_slope<PP><<<nb, 128, 0, st>>>(s, eta, dx, etax); break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t spectral_filter(const Shape& s, const double* f, double* out, const double* F, int surface,
                            cudaStream_t st) {
  if (surface) {
    int nb = (s.NX + 127) / 128;
    switch (s.P) {
#define PMG_CASE(PP) case PP: k_filter_surface<PP><<<nb, 128, 0, st>>>(s, f, F, out); break;
      PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  FilterParams p{s, f, out, F};
  int NZp = slab_pitch(s.NZ);
  size_t sm = ((size_t)(2 * s.P + 1) * NZp + (size_t)(s.P + 1) * (s.P + 1)) * sizeof(double) + 16;
  switch (s.P) {
#define PMG_CASE(PP)                                                        \
  case PP: {                                                                \
    static std::atomic<unsigned long long> mask{0};                        \
    cudaError_t e = ensure_max_smem(k_filter<PP>, mask);                    \
    if (e != cudaSuccess) return e;                                         \
    k_filter<PP><<<s.Nx, 256, sm, st>>>(p);                                \
    break;                                                                  \
  }
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t forcing(size_t N, int NZ, const double* u, const double* w, const double* ux, const double* uz,
                    const double* wx, const double* wz, const double* etax, double g, double* Fu, double* Fw,
                    cudaStream_t st) {
  k_forcing<<<grid_for(N), 256, 0, st>>>(N, NZ, u, w, ux, uz, wx, wz, etax, g, Fu, Fw);
  return cudaGetLastError();
}

cudaError_t rates(size_t N, int NZ, const double* sigma, const double* u, const double* w, const double* uz,
                  const double* wz, const double* Fu, const double* Fw, const double* px, const double* pz,
                  const double* etax, double rho, double* du, double* dw, double* deta, cudaStream_t st) {
  k_rates<<<grid_for(N), 256, 0, st>>>(N, NZ, sigma, u, w, uz, wz, Fu, Fw, px, pz, etax, rho, du, dw, deta);
  return cudaGetLastError();
}

cudaError_t axpy(size_t n, double a, const double* x, const double* y, double* out, cudaStream_t st) {
  k_axpy<<<grid_for(n), 256, 0, st>>>(n, a, x, y, out);
  return cudaGetLastError();
}

}  // namespace pmg
