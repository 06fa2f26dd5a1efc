// Multigrid level kernels on the flat, linearised geometry (Sec. 5, Sec. 5.4):
//
//  * level operator: on eta = 0 every element has the same metric, and the assembled
//    level matrix is the Kronecker sum  A = cx K_X (x) M_Z + cz M_X (x) K_Z  of 1D LGL
//    stiffness K = assembled D^T diag(w) D and 1D LGL weights M (cx = h dsig/dx,
//    cz = dx/(h dsig)).  Each output node sums 1D element stencils along its row and
//    its column; the CTA of an element column also evaluates the left element's share of
//    its first column, so no exchange is needed.
//  * additive Schwarz smoother (Sec. 5.3): subdomain = element block plus `overlap` node
//    lines, block = submatrix of the assembled level matrix, which is again a Kronecker
//    sum; its inverse is applied exactly by fast diagonalisation with the per-class
//    generalized eigenvectors (V^T M V = I):  A_i^-1 = (Vx (x) Vz) diag(1/(cx lx + cz lz)) (Vx (x) Vz)^T.
//  * transfers (Sec. 5.2): prolongation = coarse polynomial evaluated at the fine nodes,
//    J (x) J per element; restriction = its transpose, summed over distinct fine nodes.
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_levels)

namespace pmg {

// ------------------------------------------------------------------------------------
// level operator / residual
// ------------------------------------------------------------------------------------
template <typename T>
struct FlatParams {
  Shape s;
  const T* x;
  const T* b;
  T* y;
  T cx, cz;
  const T* mX;  // [NX] assembled weights along x
  const T* mZ;  // [NZ]
  int residual; // 0: y = A x (surface row y = x); 1: y = b - A x (surface row 0)
  const T* Kx;  // VAR: [Nx][n][n] x-stiffness of each element column (cx folded in)
};

// Level operator A = cx K_X (x) M_Z + cz M_X (x) K_Z (the flat level of Sec. 5, a Kronecker
// sum).  VAR: over a varying depth the level keeps each node column's depth d and drops
// the bottom-slope terms, A = K_X[d] (x) M_Z + M_X[1/d] (x) K_Z, with the element x-stiffness
// (dsig/dx) D^T diag(w d) D of each element column in Kx and (dx/dsig) M_X[1/d] in mX
// (cx = cz = 1): still a Kronecker sum, so the same kernels apply.
template <int P, typename T, bool VAR>
__device__ __forceinline__ T kx_coef(const T* KE, int i, int m) {
  if constexpr (VAR) return KE[i * (P + 1) + m];
  else return CT<T>::K(cT, P, i, m);
}

template <int P, typename T, bool VAR>
__global__ void __launch_bounds__(512) k_flat(FlatParams<T> p) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  const bool left = s.periodic || ex > 0;
  const bool last = !s.periodic && ex == s.Nx - 1;
  const int own = last ? n : P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);  // [2P+1][NZp], local column c <-> col0 - P + c
  T* Y = X + (2 * P + 1) * NZp;            // [n][NZp]
  T* MZ = Y + n * NZp;                     // [NZ] cx * assembled weights along z
  T* MX = MZ + NZ;                         // [n]  cz * assembled weights along x (own columns)
  T* B = MX + n;                           // [n][NZp] right-hand side of the own columns
  T* KO = B + n * NZp;                     // VAR: [n][n] own element's x-stiffness
  T* KL = KO + n * n;                      // VAR: [n] last row of the left element's
  const int c_begin = left ? 0 : P;
  if constexpr (VAR) {
    const T* ko = p.Kx + (size_t)ex * n * n;
    const T* kl = p.Kx + (size_t)(left ? (ex == 0 ? s.Nx - 1 : ex - 1) : ex) * n * n + P * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) KO[t] = ko[t];
    if (threadIdx.x < n) KL[threadIdx.x] = kl[threadIdx.x];
  }
  for_slab(2 * P + 1, NZ, [&](int c, int iz) {
    bool ok = c >= c_begin && iz != NZ - 1;
    cp_async_elem(&X[c * NZp + iz], p.x + (ok ? (size_t)wrap_col(s, col0 - P + c) * NZ + iz : 0), ok);
  });
  if (p.residual)
    for_slab(own, NZ, [&](int i, int iz) { cp_async_elem(&B[i * NZp + iz], p.b + (size_t)(col0 + i) * NZ + iz, true); });
  for (int t = threadIdx.x; t < NZ; t += blockDim.x) MZ[t] = p.cx * p.mZ[t];
  if (threadIdx.x < own) MX[threadIdx.x] = p.cz * p.mX[wrap_col(s, col0 + threadIdx.x)];
  cp_async_wait_all();
  __syncthreads();
  // x-direction stencils, one node row per thread
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    T xo[n], xl[n];
#pragma unroll
    for (int m = 0; m < n; ++m) { xo[m] = X[(P + m) * NZp + iz]; xl[m] = X[m * NZp + iz]; }
    T f = MZ[iz];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      if (i == P && !last) break;
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < n; ++m) acc += kx_coef<P, T, VAR>(KO, i, m) * xo[m];
      if (i == 0 && left) {  // the left element's share of the shared first column
#pragma unroll
        for (int m = 0; m < n; ++m) acc += (VAR ? KL[m] : CT<T>::K(cT, P, P, m)) * xl[m];
      }
      Y[i * NZp + iz] = f * acc;
    }
  }
  __syncthreads();
  // z-direction stencils, one (column, element row) per thread, owning rows [ez P, ez P + P)
  for (int t = threadIdx.x; t < own * Nz; t += blockDim.x) {
    int ez = t / own, i = t - ez * own;
    const T* col = X + (P + i) * NZp;
    T xv[n];
#pragma unroll
    for (int m = 0; m < n; ++m) xv[m] = col[ez * P + m];
    T below = T(0);
    if (ez > 0) {
#pragma unroll
      for (int m = 0; m < n; ++m) below += CT<T>::K(cT, P, P, m) * col[(ez - 1) * P + m];
    }
    T f = MX[i];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T acc = (j == 0) ? below : T(0);
#pragma unroll
      for (int m = 0; m < n; ++m) acc += CT<T>::K(cT, P, j, m) * xv[m];
      Y[i * NZp + ez * P + j] += f * acc;
    }
  }
  __syncthreads();
  const size_t base = (size_t)col0 * NZ;
  for_slab(own, NZ, [&](int i, int iz) {
    size_t g = base + (size_t)i * NZ + iz;
    bool top = iz == NZ - 1;
    T v = Y[i * NZp + iz];
    if (p.residual) p.y[g] = top ? T(0) : B[i * NZp + iz] - v;
    else p.y[g] = top ? p.x[g] : v;
  });
}

// The same level operator node-parallel: one thread per node reads its x- and z-stencil
// neighbours straight from global memory (L1/L2 serve the reuse), no shared memory and no
// barriers, so a CTA's critical path is one load wave and ~2(P+1) FMAs.
template <int P, typename T, bool VAR>
__global__ void __launch_bounds__(256) k_flat_np(FlatParams<T> p) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz;
  const size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (g >= (size_t)s.NX * NZ) return;
  const int ix = (int)(g / NZ), iz = (int)(g - (size_t)ix * NZ);
  if (iz == NZ - 1) {
    p.y[g] = p.residual ? T(0) : p.x[g];
    return;
  }
  // x stencil: the element(s) of column ix (the wall side has one)
  const int ex = min(ix / P, s.Nx - 1), i = ix - ex * P;
  const T* ko = VAR ? p.Kx + (size_t)ex * n * n : nullptr;
  T ax = T(0);
#pragma unroll
  for (int m = 0; m < n; ++m) ax += kx_coef<P, T, VAR>(ko, i, m) * p.x[(size_t)wrap_col(s, ex * P + m) * NZ + iz];
  if (i == 0 && (s.periodic || ex > 0)) {
    const T* kl = VAR ? p.Kx + (size_t)(ex == 0 ? s.Nx - 1 : ex - 1) * n * n : nullptr;
#pragma unroll
    for (int m = 0; m < n; ++m) ax += kx_coef<P, T, VAR>(kl, P, m) * p.x[(size_t)wrap_col(s, (ex - 1) * P + m) * NZ + iz];
  }
  // z stencil along the column (the surface row of x is read as zero)
  const T* col = p.x + (size_t)ix * NZ;
  const int ez = min(iz / P, Nz - 1), j = iz - ez * P;
  T az = T(0);
#pragma unroll
  for (int m = 0; m < n; ++m) {
    int r = ez * P + m;
    az += CT<T>::K(cT, P, j, m) * (r == NZ - 1 ? T(0) : col[r]);
  }
  if (j == 0 && ez > 0) {
#pragma unroll
    for (int m = 0; m < n; ++m) az += CT<T>::K(cT, P, P, m) * col[(ez - 1) * P + m];
  }
  T v = p.cx * p.mZ[iz] * ax + p.cz * p.mX[ix] * az;
  p.y[g] = p.residual ? p.b[g] - v : v;
}

template <int P, typename T, bool VAR>
static cudaError_t launch_flat_p(const FlatParams<T>& prm, int threads, cudaStream_t st) {
  if (threads < 0) {  // node-parallel variant, -threads per CTA
    size_t N = (size_t)prm.s.NX * prm.s.NZ;
    int bs = -threads;
    k_flat_np<P, T, VAR><<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(prm);
    return cudaGetLastError();
  }
  int NZp = slab_pitch(prm.s.NZ);
  size_t sm = ((size_t)((2 * P + 1) + 2 * (P + 1)) * NZp + prm.s.NZ + P + 1 + (VAR ? (P + 1) * (P + 2) : 0)) * sizeof(T);
  auto k = k_flat<P, T, VAR>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t flat_op(const FlatArgs& a, cudaStream_t st) {
  FlatParams<T> p;
  p.s = a.s;
  p.x = (const T*)a.x;
  p.b = (const T*)a.b;
  p.y = (T*)a.y;
  p.cx = (T)a.cx;
  p.cz = (T)a.cz;
  p.mX = (const T*)a.mX;
  p.mZ = (const T*)a.mZ;
  p.residual = a.residual;
  p.Kx = (const T*)a.Kx;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : (a.threads <= -32 && a.threads >= -256) ? a.threads : 256;
  switch (a.s.P) {
#define PMG_CASE(PP) case PP: return p.Kx ? launch_flat_p<PP, T, true>(p, thr, st) : launch_flat_p<PP, T, false>(p, thr, st);
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
  }
  return cudaErrorInvalidValue;
}
template cudaError_t flat_op<double>(const FlatArgs&, cudaStream_t);
template cudaError_t flat_op<float>(const FlatArgs&, cudaStream_t);

// ------------------------------------------------------------------------------------
// Schwarz smoother by fast diagonalisation
// ------------------------------------------------------------------------------------
template <typename T>
struct FdmParams {
  Shape s;
  const T* r;       // residual b - A x
  T* x;             // updated in place
  int post;         // 0: x += omega W sum R^T A^-1 R r;  1: x += omega sum R^T A^-1 R W r
  T omega;
  const T* Vx;      // [4][NB][NB]  (a, alpha): class x-eigenvectors in the padded local frame
  const T* Vz;      // [4][NB][NB]  (b, beta)
  const T* invden;  // [4][4][NB][NB] (xcls, zcls, alpha, beta): 1/(cx lx + cz lz), 0 if padded
  const T* wx;      // [NX] inverse 1D cover counts
  const T* wz;      // [NZ]
  Scratch sc;
  int xpercol;      // Vx [Nx][NB][NB] and invden [Nx][4][NB][NB]: one x-class per element column
};

__device__ __forceinline__ int xclass(const Shape& s, int ex) {
  if (s.periodic) return 0;
  return (ex == 0 ? 1 : 0) | (ex == s.Nx - 1 ? 2 : 0);
}
__device__ __forceinline__ int zclass(const Shape& s, int ez) {
  return (ez == 0 ? 1 : 0) | (ez == s.Nz - 1 ? 2 : 0);
}

template <int P, int O, typename T>
__global__ void __launch_bounds__(256) k_fdm(FdmParams<T> p) {
  constexpr int NB = P + 1 + 2 * O;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  const int xc = p.xpercol ? ex : xclass(s, ex);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* R = reinterpret_cast<T*>(smem_raw);  // [NB][NZp]  input, later U
  T* T1 = R + NB * NZp;                    // [NB][NZp]  x-transformed rows
  T* T3 = T1 + NB * NZp;                   // [Nz][NB][NB] (ez, b, alpha)
  T* VX = T3 + Nz * NB * NB;               // [NB][NB]
  T* VZ = VX + NB * NB;                     // [4][NB][NB]
  T* ID = VZ + 4 * NB * NB;                // [4][NB][NB]
  T* XS = ID + 4 * NB * NB;                // [NB][NZp] x on the subdomain columns (prefetched)
  size_t red_off = (((size_t)(3 * NB * NZp + Nz * NB * NB + 9 * NB * NB) * sizeof(T)) + 15) & ~(size_t)15;
  int* s_flag = reinterpret_cast<int*>(smem_raw + red_off);

  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) VX[t] = p.Vx[xc * NB * NB + t];
  for (int t = threadIdx.x; t < 4 * NB * NB; t += blockDim.x) {
    VZ[t] = p.Vz[t];
    ID[t] = p.invden[xc * 4 * NB * NB + t];
  }
  for_slab(NB, NZ, [&](int a, int iz) {
    int gc = col0 - O + a;
    bool ok = col_valid(s, gc) && iz != NZ - 1;
    size_t g = ok ? (size_t)wrap_col(s, gc) * NZ + iz : 0;
    cp_async_elem(&R[a * NZp + iz], p.r + g, ok);
    cp_async_elem(&XS[a * NZp + iz], p.x + g, ok);
  });
  cp_async_wait_all();
  __syncthreads();
  if (p.post)
    for_slab(NB, NZ, [&](int a, int iz) {
      int gc = col0 - O + a;
      if (col_valid(s, gc)) {
        int c = wrap_col(s, gc);
        R[a * NZp + iz] *= p.wx[c] * p.wz[iz];
      }
    });
  __syncthreads();
  // phase 1: T1[alpha][iz] = sum_a Vx[a][alpha] R[a][iz]
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    T rv[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) rv[a] = R[a * NZp + iz];
#pragma unroll
    for (int al = 0; al < NB; ++al) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a < NB; ++a) acc += VX[a * NB + al] * rv[a];
      T1[al * NZp + iz] = acc;
    }
  }
  __syncthreads();
  // phase 2: per (alpha, ez): sigma transform, diagonal solve, inverse sigma transform
  for (int t = threadIdx.x; t < NB * Nz; t += blockDim.x) {
    int al = t % NB, ez = t / NB;
    int zc = zclass(s, ez);
    const T* vz = VZ + zc * NB * NB;
    const T* idn = ID + (zc * NB + al) * NB;
    T tz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      int iz = ez * P - O + b;
      tz[b] = (iz >= 0 && iz < NZ - 1) ? T1[al * NZp + iz] : T(0);
    }
    T t2[NB];
#pragma unroll
    for (int be = 0; be < NB; ++be) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < NB; ++b) acc += vz[b * NB + be] * tz[b];
      t2[be] = acc * idn[be];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      T acc = T(0);
#pragma unroll
      for (int be = 0; be < NB; ++be) acc += vz[b * NB + be] * t2[be];
      T3[(ez * NB + b) * NB + al] = acc;
    }
  }
  __syncthreads();
  // phase 3: per row, sum the covering elements, inverse x transform -> U[a][iz] (in R)
  T* U = R;
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    T sv[NB];
#pragma unroll
    for (int al = 0; al < NB; ++al) sv[al] = T(0);
    int e0 = (iz + O) / P;
#pragma unroll
    for (int d = -2; d <= 0; ++d) {
      int ez = e0 + d;
      if (ez < 0 || ez >= Nz) continue;
      int b = iz - ez * P + O;
      if (b < 0 || b >= NB) continue;
#pragma unroll
      for (int al = 0; al < NB; ++al) sv[al] += T3[(ez * NB + b) * NB + al];
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      T acc = T(0);
#pragma unroll
      for (int al = 0; al < NB; ++al) acc += VX[a * NB + al] * sv[al];
      U[a * NZp + iz] = acc;
    }
  }
  __syncthreads();
  // phase 4: x update; owned interior columns directly, the two zones by exchange
  auto upd = [&](int a, int iz, T u) {  // local column a <-> global col0 - O + a
    if (iz == NZ - 1) return;
    int c = wrap_col(s, col0 - O + a);
    size_t g = (size_t)c * NZ + iz;
    T w = p.post ? T(1) : p.wx[c] * p.wz[iz];
    p.x[g] = XS[a * NZp + iz] + p.omega * w * u;
  };
  for_slab(P - 1 - 2 * O, NZ, [&](int c, int iz) {
    int a = 2 * O + 1 + c;
    upd(a, iz, U[a * NZp + iz]);
  });
  constexpr int ZW = 2 * O + 1;
  T* eb = reinterpret_cast<T*>(p.sc.edgebuf);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    int a0 = side == 0 ? 0 : P;
    int e = side == 0 ? ex : (s.periodic ? (ex + 1) % s.Nx : ex + 1);
    bool single = !s.periodic && (e == 0 || e == s.Nx);
    int gbase = e * P - O;
    if (single) {
      for_slab(ZW, NZ, [&](int c, int iz) {
        if (col_valid(s, gbase + c)) upd(a0 + c, iz, U[(a0 + c) * NZp + iz]);
      });
    } else {
      T* buf = eb + (size_t)e * ZW * NZ;
      for_slab(ZW, NZ, [&](int c, int iz) { atomic_add_t(buf + c * NZ + iz, U[(a0 + c) * NZp + iz]); });
      if (!edge_arrive(p.sc.edgecnt + e, 2, s_flag)) continue;
      for_slab(ZW, NZ, [&](int c, int iz) { upd(a0 + c, iz, take_t(buf + c * NZ + iz)); });
    }
  }
}

template <int P, int O, typename T>
static cudaError_t launch_fdm_p(const FdmParams<T>& prm, int threads, cudaStream_t st) {
  constexpr int NB = P + 1 + 2 * O;
  int NZp = slab_pitch(prm.s.NZ);
  size_t elems = (size_t)3 * NB * NZp + (size_t)prm.s.Nz * NB * NB + 9 * NB * NB;
  size_t sm = ((elems * sizeof(T) + 15) & ~(size_t)15) + 16;
  auto k = k_fdm<P, O, T>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fdm_smooth(const FdmArgs& a, cudaStream_t st) {
  FdmParams<T> p;
  p.s = a.s;
  p.r = (const T*)a.r;
  p.x = (T*)a.x;
  p.post = a.post;
  p.omega = (T)a.omega;
  p.Vx = (const T*)a.Vx;
  p.Vz = (const T*)a.Vz;
  p.invden = (const T*)a.invden;
  p.wx = (const T*)a.wx;
  p.wz = (const T*)a.wz;
  p.sc = a.sc;
  p.xpercol = a.xpercol;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  if (a.overlap == 0) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm_p<PP, 0, T>(p, thr, st);
      PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  } else if (a.overlap == 1) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm_p<PP, 1, T>(p, thr, st);
      PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  }
  return cudaErrorInvalidValue;
}
template cudaError_t fdm_smooth<double>(const FdmArgs&, cudaStream_t);
template cudaError_t fdm_smooth<float>(const FdmArgs&, cudaStream_t);

// ------------------------------------------------------------------------------------
// transfers
// ------------------------------------------------------------------------------------
template <typename T>
struct TransferParams {
  Shape f, c;       // fine and coarse shapes (same cells)
  const T* in;      // prolong: x_c; restrict: r_f, or b_f when xf is set
  T* out;
  const double* J;  // [(Pf+1)][(Pc+1)]
  // restriction of the residual formed in the kernel: r_f = in - A_f xf (flat level operator)
  const T* xf;
  T cx, cz;
  const T* mX;      // [NXf] assembled LGL weights of the fine level
  const T* mZ;      // [NZf]
};

// x_f += P x_c
template <typename T>
__global__ void __launch_bounds__(512) k_prolong(TransferParams<T> p) {
  const Shape f = p.f, c = p.c;
  const int Pf = f.P, Pc = c.P, nf = Pf + 1, nc = Pc + 1;
  const int NZf = f.NZ, NZc = c.NZ, NZcp = slab_pitch(NZc), NZfp = slab_pitch(NZf);
  const int ex = blockIdx.x;
  const bool last = !f.periodic && ex == f.Nx - 1;
  const int own = last ? nf : Pf;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xc = reinterpret_cast<T*>(smem_raw);  // [nc][NZcp]
  T* Tz = Xc + nc * NZcp;                   // [nc][NZfp]
  T* Js = Tz + nc * NZfp;                   // [nf][nc]
  T* Xf = Js + nf * nc;                     // [nf][NZfp] fine values of the own columns
  for_slab(nc, NZc, [&](int k, int iz) { cp_async_elem(&Xc[k * NZcp + iz], p.in + (size_t)wrap_col(c, ex * Pc + k) * NZc + iz, true); });
  for_slab(own, NZf, [&](int i, int iz) { cp_async_elem(&Xf[i * NZfp + iz], p.out + (size_t)(ex * Pf + i) * NZf + iz, true); });
  for (int t = threadIdx.x; t < nf * nc; t += blockDim.x) Js[t] = (T)p.J[t];
  cp_async_wait_all();
  __syncthreads();
  for_slab(nc, NZf, [&](int k, int iz) {
    int ez = min(iz / Pf, f.Nz - 1), j = iz - ez * Pf;
    T acc = T(0);
    for (int l = 0; l < nc; ++l) acc += Js[j * nc + l] * Xc[k * NZcp + ez * Pc + l];
    Tz[k * NZfp + iz] = acc;
  });
  __syncthreads();
  for_slab(own, NZf, [&](int i, int iz) {
    if (iz == NZf - 1) return;
    T acc = T(0);
    for (int k = 0; k < nc; ++k) acc += Js[i * nc + k] * Tz[k * NZfp + iz];
    p.out[(size_t)(ex * Pf + i) * NZf + iz] = Xf[i * NZfp + iz] + acc;
  });
}

// r_c = P^T r_f
template <typename T>
__global__ void __launch_bounds__(512) k_restrict(TransferParams<T> p) {
  const Shape f = p.f, c = p.c;
  const int Pf = f.P, Pc = c.P, nf = Pf + 1, nc = Pc + 1;
  const int NZf = f.NZ, NZc = c.NZ, NZfp = slab_pitch(NZf), NZcp = slab_pitch(NZc);
  const int ex = blockIdx.x;
  const bool left = f.periodic || ex > 0;
  const bool last = !f.periodic && ex == f.Nx - 1;
  const int own = last ? nc : Pc;
  const int ncol = 2 * Pf + 1;  // local fine column q <-> (ex-1) Pf + q
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Rf = reinterpret_cast<T*>(smem_raw);  // [ncol][NZfp]
  T* Sz = Rf + ncol * NZfp;                 // [ncol][NZcp]
  T* Js = Sz + ncol * NZcp;                 // [nf][nc]
  T* Xs = Js + nf * nc;                     // fused: [ncol][NZfp] fine iterate
  T* MZ = Xs + ncol * NZfp;                 // fused: [NZf] cx * assembled z weights
  T* MX = MZ + NZf;                         // fused: [ncol] cz * assembled x weights
  const bool fused = p.xf != nullptr;
  for (int t = threadIdx.x; t < nf * nc; t += blockDim.x) Js[t] = (T)p.J[t];
  for_slab(ncol, NZf, [&](int q, int iz) {
    int gc = (ex - 1) * Pf + q;
    bool ok = (q >= Pf || left) && (q < 2 * Pf || last) && iz != NZf - 1;
    cp_async_elem(&Rf[q * NZfp + iz], p.in + (ok ? (size_t)wrap_col(f, gc) * NZf + iz : 0), ok);
    if (fused) {
      bool okx = (q >= Pf || left) && iz != NZf - 1;  // x of the left and own elements
      cp_async_elem(&Xs[q * NZfp + iz], p.xf + (okx ? (size_t)wrap_col(f, gc) * NZf + iz : 0), okx);
    }
  });
  if (fused) {
    for (int t = threadIdx.x; t < NZf; t += blockDim.x) MZ[t] = p.cx * p.mZ[t];
    for (int q = threadIdx.x; q < ncol; q += blockDim.x) {
      int gc = (ex - 1) * Pf + q;
      MX[q] = (q >= Pf || left) ? p.cz * p.mX[wrap_col(f, gc)] : T(0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (fused) {
    // Rf = b - A_f x on the fine columns the restriction reads: (ex-1)Pf + 1 .. (ex+1)Pf - 1,
    // and (ex+1)Pf on the wall CTA.  Element 0 of the slab is the left one (absent at a
    // wall: its stencil is skipped, not only its data zeroed), element 1 the own one.
    for_slab(ncol, NZf, [&](int q, int iz) {
      if (iz == NZf - 1 || q == 0 || (q == 2 * Pf && !last) || (q < Pf && !left)) return;
      int e = q / Pf, li = q - e * Pf;
      if (e == 2) { e = 1; li = Pf; }
      T kx = T(0);
      for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, li, m) * Xs[(e * Pf + m) * NZfp + iz];
      if (li == 0 && e == 1 && left)
        for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, Pf, m) * Xs[m * NZfp + iz];
      const int ez = min(iz / Pf, f.Nz - 1), lj = iz - ez * Pf;
      const T* col = Xs + q * NZfp;
      T kz = T(0);
      for (int m = 0; m < nf; ++m) kz += CT<T>::K(cT, Pf, lj, m) * col[ez * Pf + m];
      if (lj == 0 && ez > 0)
        for (int m = 0; m < nf; ++m) kz += CT<T>::K(cT, Pf, Pf, m) * col[(ez - 1) * Pf + m];
      Rf[q * NZfp + iz] -= MZ[iz] * kx + MX[q] * kz;
    });
    __syncthreads();
  }
  for_slab(ncol, NZc, [&](int q, int lc) {
    T acc = T(0);
    if (lc != NZc - 1) {
      int ez = min(lc / Pc, c.Nz - 1), l = lc - ez * Pc;
      const T* col = Rf + q * NZfp;
      if (l == 0) {
        acc = col[ez * Pf];
        for (int j = 1; j < Pf; ++j) acc += Js[j * nc + 0] * col[ez * Pf + j];
        if (ez > 0)
          for (int j = 1; j < Pf; ++j) acc += Js[j * nc + Pc] * col[(ez - 1) * Pf + j];
      } else {
        for (int j = 1; j < Pf; ++j) acc += Js[j * nc + l] * col[ez * Pf + j];
      }
    }
    Sz[q * NZcp + lc] = acc;
  });
  __syncthreads();
  for_slab(own, NZc, [&](int k, int lc) {
    T acc = T(0);
    if (lc != NZc - 1) {
      if (k == 0) {
        acc = Sz[Pf * NZcp + lc];
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + 0] * Sz[(Pf + i) * NZcp + lc];
        if (left)
          for (int i = 1; i < Pf; ++i) acc += Js[i * nc + Pc] * Sz[i * NZcp + lc];
      } else if (k == Pc) {
        acc = Sz[2 * Pf * NZcp + lc];
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + Pc] * Sz[(Pf + i) * NZcp + lc];
      } else {
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + k] * Sz[(Pf + i) * NZcp + lc];
      }
    }
    p.out[(size_t)(ex * Pc + k) * NZc + lc] = acc;
  });
}

template <typename T>
cudaError_t transfer(const TransferArgs& a, int restrict_, cudaStream_t st) {
  TransferParams<T> p;
  p.f = a.f;
  p.c = a.c;
  p.in = (const T*)a.in;
  p.out = (T*)a.out;
  p.J = a.J;
  p.xf = (const T*)a.xf;
  p.cx = (T)a.cx;
  p.cz = (T)a.cz;
  p.mX = (const T*)a.mX;
  p.mZ = (const T*)a.mZ;
  int nf = a.f.P + 1, nc = a.c.P + 1;
  int NZfp = slab_pitch(a.f.NZ), NZcp = slab_pitch(a.c.NZ);
  cudaError_t e;
  if (restrict_) {
    size_t sm = ((size_t)(2 * a.f.P + 1) * (NZfp + NZcp) + nf * nc) * sizeof(T) + 16;
    if (a.xf) sm += ((size_t)(2 * a.f.P + 1) * (NZfp + 1) + a.f.NZ) * sizeof(T);
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_restrict<T>, s_mask);
    if (e != cudaSuccess) return e;
    k_restrict<T><<<a.f.Nx, (a.threads >= 32 && a.threads <= 512) ? a.threads : 256, sm, st>>>(p);
  } else {
    size_t sm = ((size_t)nc * (NZcp + NZfp) + nf * nc + (size_t)nf * NZfp) * sizeof(T) + 16;
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_prolong<T>, s_mask);
    if (e != cudaSuccess) return e;
    k_prolong<T><<<a.f.Nx, (a.threads >= 32 && a.threads <= 512) ? a.threads : 256, sm, st>>>(p);
  }
  return cudaGetLastError();
}
template cudaError_t transfer<double>(const TransferArgs&, int, cudaStream_t);
template cudaError_t transfer<float>(const TransferArgs&, int, cudaStream_t);

}  // namespace pmg
