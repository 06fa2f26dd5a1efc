// Additive Schwarz with dense subdomain inverses (Sec. 5.3; the alternative to fast
// diagonalisation for level operators that are not Kronecker sums).  Subdomain of element
// (ex, ez): its node lines plus `overlap` lines of each neighbour (clipped at walls, the
// Dirichlet surface row left out), NB = NBX * NBZ nodes in the padded local frame.
//
// Setup (once per level operator): the block A_i = R_i A R_i^T of the assembled level
// matrix is summed from the element matrices of the 3 x 3 element neighbourhood, each entry
// in closed form from the per-column metric factors (the same factors as the operator
// kernels: G_rr = w_j A_i, G_rs = -w_j sigma B_i, G_ss = w_j C_i (1 + sigma^2 E_i)):
//   K[(i,j),(k,l)] = d_jl sum_m Dx[m][i] Dx[m][k] G_rr(m,j) + Dx[k][i] G_rs(k,j) Dz[j][l]
//                  + Dz[l][j] G_rs(i,l) Dx[i][k] + d_ik sum_m Dz[m][j] Dz[m][l] G_ss(i,m),
// then inverted in place by Gauss-Jordan elimination (SPD: no pivoting) in shared memory;
// absent nodes of the padded frame carry an identity row.
// Sweep: u_i = A_i^-1 R_i r per subdomain (symmetric A_i^-1: thread a reads column a,
// coalesced), then per node the sum over the covering subdomains in a fixed order
// (deterministic, no atomics) and x += omega W u (pre) or x += omega u with W on r (post).
#include "pmg_common.cuh"
#include "pmg_kernels.h"

#include <algorithm>

PMG_DEFINE_CONST_TABLES(init_consts_dense)

namespace pmg {

struct DenseFrame {
  Shape s;
  int px, pz, ox, oz, NBX, NBZ;
};

__device__ __forceinline__ DenseFrame dense_frame(const Shape& s, int ox, int oz) {
  DenseFrame f;
  f.s = s;
  f.px = s.P;
  f.pz = s.pz();
  f.ox = ox;
  f.oz = oz;
  f.NBX = f.px + 1 + 2 * ox;
  f.NBZ = f.pz + 1 + 2 * oz;
  return f;
}

// unwrapped global column / row of local node (ai, aj) of subdomain (ex, ez); validity
__device__ __forceinline__ bool dense_node(const DenseFrame& f, int ex, int ez, int ai, int aj, int& cu, int& row) {
  cu = ex * f.px - f.ox + ai;
  row = ez * f.pz - f.oz + aj;
  bool okc = f.s.periodic || (cu >= 0 && cu < f.s.NX);
  return okc && row >= 0 && row < f.s.NZ - 1;
}

// Element matrix entry of element column exu (unwrapped; factors of exu mod Nx) and element
// row ez2 between local nodes (i, j) and (k, l).
__device__ double elem_entry(const DenseFrame& f, const double* geo, const double* sigma, int exu, int ez2, int i,
                             int j, int k, int l) {
  const int px = f.px, pz = f.pz;
  int exw = exu;
  if (f.s.periodic) exw = ((exu % f.s.Nx) + f.s.Nx) % f.s.Nx;
  const double* g = geo + (size_t)exw * (px + 1) * 4;  // [i][A, B, C, E]
  auto sg = [&](int qj) { return sigma[ez2 * pz + qj]; };
  double v = 0.0;
  if (j == l) {
    double a = 0.0;
    for (int m = 0; m <= px; ++m) a += cT.D[px][m][i] * cT.D[px][m][k] * g[m * 4 + 0];
    v += cT.w[pz][j] * a;
  }
  // cross terms: G_rs(q) = -w_qj sigma(qj) B(qi)
  v += cT.D[px][k][i] * (-cT.w[pz][j] * sg(j) * g[k * 4 + 1]) * cT.D[pz][j][l];
  v += cT.D[pz][l][j] * (-cT.w[pz][l] * sg(l) * g[i * 4 + 1]) * cT.D[px][i][k];
  if (i == k) {
    double a = 0.0;
    for (int m = 0; m <= pz; ++m) {
      double s = sg(m);
      a += cT.D[pz][m][j] * cT.D[pz][m][l] * cT.w[pz][m] * g[i * 4 + 2] * (1.0 + s * s * g[i * 4 + 3]);
    }
    v += a;
  }
  return v;
}

// One CTA per subdomain: assemble the block, invert it in place, store FP64 and FP32.
__global__ void __launch_bounds__(512) k_dense_setup(Shape s, int ox, int oz, const double* geo, const double* sigma,
                                                     double* inv64, float* inv32) {
  const DenseFrame f = dense_frame(s, ox, oz);
  const int NB = f.NBX * f.NBZ;
  const int e = blockIdx.x, ex = e / s.Nz, ez = e - ex * s.Nz;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // [NB][NB]
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int a = t / NB, b = t - a * NB;
    const int ai = a / f.NBZ, aj = a - ai * f.NBZ, bi = b / f.NBZ, bj = b - bi * f.NBZ;
    int ca, ra, cb, rb;
    const bool va = dense_node(f, ex, ez, ai, aj, ca, ra), vb = dense_node(f, ex, ez, bi, bj, cb, rb);
    double v = 0.0;
    if (va && vb) {
      for (int dx = -1; dx <= 1; ++dx) {
        const int exu = ex + dx;
        if (!s.periodic && (exu < 0 || exu >= s.Nx)) continue;
        const int i = ca - exu * f.px, k = cb - exu * f.px;
        if (i < 0 || i > f.px || k < 0 || k > f.px) continue;
        for (int dz = -1; dz <= 1; ++dz) {
          const int ez2 = ez + dz;
          if (ez2 < 0 || ez2 >= s.Nz) continue;
          const int j = ra - ez2 * f.pz, l = rb - ez2 * f.pz;
          if (j < 0 || j > f.pz || l < 0 || l > f.pz) continue;
          v += elem_entry(f, geo, sigma, exu, ez2, i, j, k, l);
        }
      }
    } else if (a == b) {
      v = 1.0;
    }
    A[t] = v;
  }
  __syncthreads();
  // in-place Gauss-Jordan inverse (symmetric positive definite: no pivoting)
  for (int k = 0; k < NB; ++k) {
    const double piv = 1.0 / A[k * NB + k];
    __syncthreads();
    // column k of the other rows, saved before row k changes
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
      const int i = t / NB, j = t - i * NB;
      if (i == k || j == k) continue;
      A[t] -= A[i * NB + k] * A[k * NB + j] * piv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NB; t += blockDim.x) {
      if (t == k) continue;
      A[k * NB + t] *= piv;
      A[t * NB + k] *= -piv;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[k * NB + k] = piv;
    __syncthreads();
  }
  double* o64 = inv64 + (size_t)e * NB * NB;
  float* o32 = inv32 + (size_t)e * NB * NB;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    o64[t] = A[t];
    o32[t] = (float)A[t];
  }
}

// u_e = A_e^-1 (R_e r), r weighted by W at the node in post-smoothing
template <typename T>
__global__ void __launch_bounds__(256) k_dense_local(Shape s, int ox, int oz, const T* inv, const T* r, const T* wx,
                                                     const T* wz, int post, T* U) {
  const DenseFrame f = dense_frame(s, ox, oz);
  const int NB = f.NBX * f.NBZ;
  const int e = blockIdx.x, ex = e / s.Nz, ez = e - ex * s.Nz;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rs = reinterpret_cast<T*>(smem_raw);  // [NB]
  for (int b = threadIdx.x; b < NB; b += blockDim.x) {
    const int bi = b / f.NBZ, bj = b - bi * f.NBZ;
    int cu, row;
    T v = T(0);
    if (dense_node(f, ex, ez, bi, bj, cu, row)) {
      const int c = wrap_col(s, cu);
      v = r[(size_t)c * s.NZ + row];
      if (post) v *= wx[c] * wz[row];
    }
    rs[b] = v;
  }
  __syncthreads();
  const T* Ai = inv + (size_t)e * NB * NB;
  T* Ue = U + (size_t)e * NB;
  for (int a = threadIdx.x; a < NB; a += blockDim.x) {
    T acc = T(0);
    for (int b = 0; b < NB; ++b) acc += Ai[(size_t)b * NB + a] * rs[b];  // A_e^-1 symmetric
    Ue[a] = acc;
  }
}

// x += omega (W) sum over covering subdomains of u_e at the node, in a fixed order
template <typename T>
__global__ void __launch_bounds__(256) k_dense_gather(Shape s, int ox, int oz, const T* U, const T* wx, const T* wz,
                                                      int post, T omega, T* x) {
  const DenseFrame f = dense_frame(s, ox, oz);
  const int NB = f.NBX * f.NBZ;
  const size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (g >= (size_t)s.NX * s.NZ) return;
  const int ix = (int)(g / s.NZ), iz = (int)(g - (size_t)ix * s.NZ);
  if (iz == s.NZ - 1) return;
  const int ex0 = min(ix / f.px, s.Nx - 1), ez0 = min(iz / f.pz, s.Nz - 1);
  T acc = T(0);
  for (int dx = -1; dx <= 1; ++dx) {
    for (int sh = -1; sh <= 1; ++sh) {  // periodic images of the column
      if (!s.periodic && sh != 0) continue;
      const int exu = ex0 + dx;
      if (!s.periodic && (exu < 0 || exu >= s.Nx)) continue;
      const int ai = ix + sh * s.NX - (exu * f.px - f.ox);
      if (ai < 0 || ai >= f.NBX) continue;
      const int exw = s.periodic ? ((exu % s.Nx) + s.Nx) % s.Nx : exu;
      for (int dz = -1; dz <= 1; ++dz) {
        const int ez = ez0 + dz;
        if (ez < 0 || ez >= s.Nz) continue;
        const int aj = iz - (ez * f.pz - f.oz);
        if (aj < 0 || aj >= f.NBZ) continue;
        acc += U[((size_t)exw * s.Nz + ez) * NB + ai * f.NBZ + aj];
      }
    }
  }
  const T w = post ? T(1) : wx[ix] * wz[iz];
  x[g] += omega * w * acc;
}

// One thread per (element column, level-local column): the element's surface polynomial of
// the fine order at the level's node (E = [(p+1) x (P+1)]).  A node shared by two cells is
// written by both with the same value (E is exact at the cell ends).
__global__ void k_eta_level(Shape f, Shape c, const double* E, const double* eta, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = c.P + 1, nf = f.P + 1;
  if (t >= c.Nx * nc) return;
  const int ex = t / nc, i = t - ex * nc;
  double v = 0.0;
  for (int m = 0; m < nf; ++m) v += E[i * nf + m] * eta[wrap_col(f, ex * f.P + m)];
  out[wrap_col(c, ex * c.P + i)] = v;
}

cudaError_t eta_level(const Shape& fine, const Shape& lev, const double* E, const double* eta, double* out,
                      cudaStream_t st) {
  const int tot = lev.Nx * (lev.P + 1);
  k_eta_level<<<(tot + 127) / 128, 128, 0, st>>>(fine, lev, E, eta, out);
  return cudaGetLastError();
}

size_t dense_block_elems(const Shape& s, int ox, int oz) {
  size_t NB = (size_t)(s.P + 1 + 2 * ox) * (s.pz() + 1 + 2 * oz);
  return NB * NB;
}

cudaError_t dense_setup(const Shape& s, int ox, int oz, const double* geo, const double* sigma, double* inv64,
                        float* inv32, cudaStream_t st) {
  const size_t nb2 = dense_block_elems(s, ox, oz);
  const size_t sm = nb2 * sizeof(double);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> mask{0};
  cudaError_t e = ensure_max_smem(k_dense_setup, mask);
  if (e != cudaSuccess) return e;
  k_dense_setup<<<s.Nx * s.Nz, 512, sm, st>>>(s, ox, oz, geo, sigma, inv64, inv32);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dense_sweep(const Shape& s, int ox, int oz, const T* inv, const T* r, T* x, const T* wx, const T* wz,
                        int post, double omega, T* U, cudaStream_t st) {
  const int NB = (s.P + 1 + 2 * ox) * (s.pz() + 1 + 2 * oz);
  const int thr = std::min(256, (NB + 31) / 32 * 32);  // one thread per block row, whole warps
  k_dense_local<T><<<s.Nx * s.Nz, thr, NB * sizeof(T), st>>>(s, ox, oz, inv, r, wx, wz, post, U);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t N = (size_t)s.NX * s.NZ;
  k_dense_gather<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(s, ox, oz, U, wx, wz, post, (T)omega, x);
  return cudaGetLastError();
}
template cudaError_t dense_sweep<double>(const Shape&, int, int, const double*, const double*, double*, const double*,
                                         const double*, int, double, double*, cudaStream_t);
template cudaError_t dense_sweep<float>(const Shape&, int, int, const float*, const float*, float*, const float*,
                                        const float*, int, double, float*, cudaStream_t);

}  // namespace pmg
