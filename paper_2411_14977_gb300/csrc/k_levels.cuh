// Level-operator and Schwarz-sweep kernel templates (Sec. 5.3), shared by k_levels.cu
// (equal orders) and k_levels_aniso.cu (different orders along x and sigma).  The
// including translation unit defines the constant tables cT first.
#pragma once
#include <type_traits>

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
  long long wait_cycles = 0;    // k_flat_bulk: bound of the mbarrier wait
  int* timeout_flag = nullptr;  // k_flat_bulk: raised when the wait gives up
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

// PZ: order along sigma when it differs from P (the z stencils use PZ + 1 nodes).
template <int P, typename T, bool VAR, int PZ = P>
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
  // z-direction stencils, one (column, element row) per thread, owning rows [ez PZ, ez PZ + PZ)
  constexpr int nz = PZ + 1;
  for (int t = threadIdx.x; t < own * Nz; t += blockDim.x) {
    int ez = t / own, i = t - ez * own;
    const T* col = X + (P + i) * NZp;
    T xv[nz];
#pragma unroll
    for (int m = 0; m < nz; ++m) xv[m] = col[ez * PZ + m];
    T below = T(0);
    if (ez > 0) {
#pragma unroll
      for (int m = 0; m < nz; ++m) below += CT<T>::K(cT, PZ, PZ, m) * col[(ez - 1) * PZ + m];
    }
    T f = MX[i];
#pragma unroll
    for (int j = 0; j < PZ; ++j) {
      T acc = (j == 0) ? below : T(0);
#pragma unroll
      for (int m = 0; m < nz; ++m) acc += CT<T>::K(cT, PZ, j, m) * xv[m];
      Y[i * NZp + ez * PZ + j] += f * acc;
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
template <int P, typename T, bool VAR, int PZ = P>
__device__ __forceinline__ void flat_np_body(const FlatParams<T>& p, const size_t g) {
  constexpr int n = P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz;
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
  const int ez = min(iz / PZ, Nz - 1), j = iz - ez * PZ;
  T az = T(0);
#pragma unroll
  for (int m = 0; m <= PZ; ++m) {
    int r = ez * PZ + m;
    az += CT<T>::K(cT, PZ, j, m) * (r == NZ - 1 ? T(0) : col[r]);
  }
  if (j == 0 && ez > 0) {
#pragma unroll
    for (int m = 0; m <= PZ; ++m) az += CT<T>::K(cT, PZ, PZ, m) * col[(ez - 1) * PZ + m];
  }
  T v = p.cx * p.mZ[iz] * ax + p.cz * p.mX[ix] * az;
  p.y[g] = p.residual ? p.b[g] - v : v;
}
template <int P, typename T, bool VAR, int PZ = P>
__global__ void __launch_bounds__(256) k_flat_np(FlatParams<T> p) {
  flat_np_body<P, T, VAR, PZ>(p, blockIdx.x * (size_t)blockDim.x + threadIdx.x);
}

// The same level operator (FP32, constant depth, equal orders) with the CTA's inputs staged
// by TMA bulk copies: an element column's x stencil slab -- node columns col0 - P ..
// col0 + P, z-fastest, i.e. one contiguous run of (2P + 1) NZ floats (two runs where a
// periodic tank wraps) -- and, for the residual, b on its own columns (one run).  Thread 0
// widens each run to 16-byte boundaries (the start rounded down, the end rounded up but
// clipped at the vector's last 16-byte boundary; the clipped tail is read with plain
// loads), announces the bytes on one mbarrier and issues one cp.async.bulk per run, so a
// CTA has its whole slab in flight after a handful of instructions.  The wait is bounded
// (wait_cycles): a CTA that gives up raises *timeout_flag, waits for its copies to land
// and leaves y unwritten.  Each thread then forms whole output nodes: x stencil along the
// node row and z stencil along the node column, both from shared memory (the surface row
// read as zero), written straight to y (consecutive threads, consecutive rows).
struct FlatBulkRun {
  long long a0, a1, end;  // copied [a0, a1) by TMA, [a1, end) by plain loads
  int dst;                // shared-memory float index of global element a0
};
__device__ __forceinline__ FlatBulkRun flat_bulk_run(long long start, long long end, long long nal, int dst) {
  FlatBulkRun r;
  r.a0 = start & ~3ll;
  r.a1 = min((end + 3) & ~3ll, nal);
  if (r.a1 < r.a0) r.a1 = r.a0;
  r.end = end;
  r.dst = dst;
  return r;
}
template <int P>
__global__ void __launch_bounds__(512) k_flat_bulk(FlatParams<float> p) {
  constexpr int n = P + 1, NC = 2 * P + 1;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz;
  const int ex = blockIdx.x, col0 = ex * P;
  const bool left = s.periodic || ex > 0;
  const bool last = !s.periodic && ex == s.Nx - 1;
  const int own = last ? n : P;
  const int cb = left ? 0 : P;  // first staged local column (c <-> global col0 - P + c)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
  int* XO = reinterpret_cast<int*>(smem_raw + 8);  // [NC] shared float index of column c's row 0
  int* s_misc = XO + NC;                           // [0] ok, [1] b's row-0 index
  float* S = reinterpret_cast<float*>(smem_raw + ((8 + 4 * (NC + 2) + 15) & ~15));
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    const long long N = (long long)s.NX * NZ, nal = N & ~3ll;
    // runs of consecutive global columns among the staged ones (at most two: a periodic
    // tank wraps once), then b's own columns
    FlatBulkRun run[3];
    int nrun = 0, dst = 0;
    int c = cb;
    while (c < NC) {
      const int g0 = wrap_col(s, col0 - P + c);
      int c1 = c + 1;
      while (c1 < NC && wrap_col(s, col0 - P + c1) == g0 + (c1 - c)) ++c1;
      run[nrun] = flat_bulk_run((long long)g0 * NZ, (long long)(g0 + c1 - c) * NZ, nal, dst);
      for (int k = c; k < c1; ++k) XO[k] = dst + (int)((long long)(g0 + k - c) * NZ - run[nrun].a0);
      dst += (int)(((run[nrun].end - run[nrun].a0) + 3) & ~3ll);
      ++nrun;
      c = c1;
    }
    for (int k = 0; k < cb; ++k) XO[k] = -1;
    if (p.residual) {
      run[nrun] = flat_bulk_run((long long)col0 * NZ, (long long)(col0 + own) * NZ, nal, dst);
      s_misc[1] = dst + (int)((long long)col0 * NZ - run[nrun].a0);
      ++nrun;
    }
    unsigned total = 0;
    for (int r = 0; r < nrun; ++r) total += (unsigned)(run[r].a1 - run[r].a0) * 4u;
    mbar_arrive_expect_tx(bar, total);
    const int nx = p.residual ? nrun - 1 : nrun;
    for (int r = 0; r < nrun; ++r) {
      const float* src = r < nx ? p.x : p.b;
      if (run[r].a1 > run[r].a0)
        bulk_load_1d(S + run[r].dst, src + run[r].a0, (unsigned)(run[r].a1 - run[r].a0) * 4u, bar);
      for (long long g = run[r].a1; g < run[r].end; ++g) S[run[r].dst + (int)(g - run[r].a0)] = src[g];
    }
  }
  // coefficients while the copies fly
  int xo[n], xl[n];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < n; ++m) {
    xo[m] = XO[P + m];
    xl[m] = left ? XO[m] : 0;
  }
  if (tid == 0) {
    const bool ok = mbar_wait_bounded(bar, 0, p.wait_cycles);
    if (!ok) {
      atomicExch(p.timeout_flag, 1);
      mbar_wait_bounded(bar, 0, kWaitCyclesDefault);  // the copies in flight land before exit
    }
    s_misc[0] = ok ? 1 : 0;
  }
  __syncthreads();
  if (s_misc[0] == 0) return;
  (void)mbar_try_wait(bar, 0);  // the phase is complete: each thread acquires the copied data
  // the surface row of x is read as zero by the stencils
  for (int c = cb + tid; c < NC; c += blockDim.x) S[XO[c] + NZ - 1] = 0.f;
  const int bo = s_misc[1];
  __syncthreads();
  const float cx = p.cx, cz = p.cz;
  const size_t base = (size_t)col0 * NZ;
  for_slab(own, NZ, [&](int i, int iz) {
    const size_t g = base + (size_t)i * NZ + iz;
    if (iz == NZ - 1) {
      p.y[g] = p.residual ? 0.f : p.x[g];
      return;
    }
    float ax = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) ax = fmaf(CT<float>::K(cT, P, i, m), S[xo[m] + iz], ax);
    if (i == 0 && left) {
#pragma unroll
      for (int m = 0; m < n; ++m) ax = fmaf(CT<float>::K(cT, P, P, m), S[xl[m] + iz], ax);
    }
    const float* col = S + XO[P + i];
    const int ez = min(iz / P, Nz - 1), j = iz - ez * P;
    float az = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) az = fmaf(CT<float>::K(cT, P, j, m), col[ez * P + m], az);
    if (j == 0 && ez > 0) {
#pragma unroll
      for (int m = 0; m < n; ++m) az = fmaf(CT<float>::K(cT, P, P, m), col[(ez - 1) * P + m], az);
    }
    const float v = cx * p.mZ[iz] * ax + cz * p.mX[col0 + i] * az;
    p.y[g] = p.residual ? S[bo + i * NZ + iz] - v : v;
  });
}
// shared memory of k_flat_bulk: mbarrier, column table, the staged runs (each widened by
// at most 3 floats at its start and padded to 16 bytes), b's run
inline size_t flat_bulk_smem(int P, const Shape& s, int residual) {
  const size_t NC = 2 * P + 1;
  const size_t hdr = (8 + 4 * (NC + 2) + 15) & ~(size_t)15;
  const size_t xs = NC * s.NZ + 2 * 8;
  const size_t bs = residual ? (size_t)(P + 1) * s.NZ + 8 : 0;
  return hdr + (xs + bs) * sizeof(float);
}

// The same level operator tiled: one thread per element, a CTA over EXT element columns x
// ZT element rows (thread t: column t % EXT, row t / EXT, so a warp's lanes sit in distinct
// element columns).  The CTA stages its x tile -- the P node columns to the left and the
// PZ node rows below as halo -- in shared memory, node rows contiguous per node column,
// with an even column pitch CP and one pad word per element column: lanes one element
// column apart are then P CP + 1 words apart, an odd stride, so with EXT = 32 a warp reads
// 32 distinct banks (EXT = 8 or 16 puts 4 or 2 element rows in a warp, which may share
// banks).  Each thread forms the outputs of the nodes its element owns (columns ex P ..
// ex P + P - 1, the wall column too for the last element; rows ez PZ .. ez PZ + PZ - 1) in
// registers: x stencils one node row at a time from 2P + 1 staged values (serving P owned
// nodes), z stencils one node column at a time from 2PZ + 1 staged values (serving PZ), so
// a node costs about (2P + 1)/P + (2PZ + 1)/PZ shared-memory loads.  ZT is a template parameter so that CP, and with it every staged
// offset of an element, is a compile-time constant off one base address.  The outputs go
// back through the same buffer and leave as whole column runs (coalesced), the surface
// row taken from x (operator) or set to 0 (residual).
template <int ZT, int PZ>
struct FlatTile {
  static constexpr int nrow = (ZT + 1) * PZ + 1;  // tile row r <-> node row ez0 PZ - PZ + r
  static constexpr int CP = (nrow + 1) & ~1;
};

template <int P, typename T, int ZT, int PZ = P>
__global__ void __launch_bounds__(256) k_flat_tile(FlatParams<T> p, int EXT) {
  constexpr int n = P + 1;
  constexpr int nrow = FlatTile<ZT, PZ>::nrow, CP = FlatTile<ZT, PZ>::CP;
  const Shape s = p.s;
  const int NZ = s.NZ;
  const int ex0 = blockIdx.x * EXT, ez0 = blockIdx.y * ZT;
  const int ncol = (EXT + 1) * P + 1;  // tile column c <-> node column ex0 P - P + c
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);  // (c, r) at c CP + r + c / P
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int gc0 = ex0 * P - P, gr0 = ez0 * PZ - PZ;
  // output block of the tile: node columns ex0 P .. (+ the wall column), rows ez0 PZ ..
  const int exn = min(ex0 + EXT, s.Nx) - ex0, ezn = min(ez0 + ZT, s.Nz) - ez0;
  const int ncy = exn * P + ((!s.periodic && ex0 + exn == s.Nx) ? 1 : 0);
  const int nry = ezn * PZ + ((ez0 + ezn == s.Nz) ? 1 : 0);
  T* Bs = X + ncol * CP + (ncol - 1) / P + 1;  // [ncy][nrow] right-hand side (residual)
  // every copy in flight at once (cp.async; zero-filled off the mesh and on the surface
  // row, which is read as 0), then one wait
  for (int c = warp; c < ncol; c += nwarps) {
    const int gc = gc0 + c;
    const bool cok = col_valid(s, gc);
    const T* src = p.x + (size_t)(cok ? wrap_col(s, gc) : 0) * NZ;
    T* dst = X + c * CP + c / P;
    for (int r = lane; r < nrow; r += 32) {
      const int gr = gr0 + r;
      const bool ok = cok && gr >= 0 && gr < NZ - 1;
      cp_async_elem(&dst[r], src + (ok ? gr : 0), ok);
    }
  }
  if (p.residual) {
    for (int c = warp; c < ncy; c += nwarps) {
      const T* src = p.b + (size_t)(ex0 * P + c) * NZ + (size_t)ez0 * PZ;
      for (int r = lane; r < nry; r += 32) cp_async_elem(&Bs[c * nrow + r], src + r, true);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int exl = (int)threadIdx.x % EXT, ezl = (int)threadIdx.x / EXT;
  const int ex = ex0 + exl, ez = ez0 + ezl;
  const bool active = ex < s.Nx && ez < s.Nz;
  // (exl P + m, (ezl + 1) PZ + q) at Xe[m CP + m / P + q]
  const T* Xe = X + exl * (P * CP + 1) + (ezl + 1) * PZ;
  T acc[n][PZ];
  if (active) {
    const bool left = s.periodic || ex > 0;
#pragma unroll
    for (int j = 0; j < PZ; ++j) {
      T xr[2 * P + 1];
#pragma unroll
      for (int m = 0; m <= 2 * P; ++m) xr[m] = Xe[m * CP + m / P + j];
      const T f = p.cx * p.mZ[ez * PZ + j];
#pragma unroll
      for (int i = 0; i < n; ++i) {
        T a = T(0);
#pragma unroll
        for (int m = 0; m < n; ++m) a += CT<T>::K(cT, P, i, m) * xr[P + m];
        if (i == 0 && left) {  // the left element's share of the shared first column
#pragma unroll
          for (int m = 0; m < n; ++m) a += CT<T>::K(cT, P, P, m) * xr[m];
        }
        acc[i][j] = f * a;
      }
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
      T xc[2 * PZ + 1];
#pragma unroll
      for (int m = 0; m <= 2 * PZ; ++m) xc[m] = Xe[(P + i) * CP + (P + i) / P + m - PZ];
      const T f = p.cz * p.mX[wrap_col(s, ex * P + i)];
#pragma unroll
      for (int j = 0; j < PZ; ++j) {
        T a = T(0);
#pragma unroll
        for (int m = 0; m <= PZ; ++m) a += CT<T>::K(cT, PZ, j, m) * xc[PZ + m];
        if (j == 0 && ez > 0) {  // the lower element's share of the shared first row
#pragma unroll
          for (int m = 0; m <= PZ; ++m) a += CT<T>::K(cT, PZ, PZ, m) * xc[m];
        }
        acc[i][j] += f * a;
      }
    }
  }
  __syncthreads();
  if (active) {
    const bool wall = !s.periodic && ex == s.Nx - 1;
    // output (exl P + i, ezl PZ + j) at the staging position (c, r) = (exl P + i, ezl PZ + j)
    T* Ye = X + exl * (P * CP + 1) + ezl * PZ;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      if (i == P && !wall) break;
#pragma unroll
      for (int j = 0; j < PZ; ++j) Ye[i * CP + i / P + j] = acc[i][j];
    }
  }
  __syncthreads();
  for (int c = warp; c < ncy; c += nwarps) {
    const size_t gb = (size_t)(ex0 * P + c) * NZ + (size_t)ez0 * PZ;
    const T* Yc = X + c * CP + c / P;
    const T* Bc = Bs + c * nrow;
    for (int r = lane; r < nry; r += 32) {
      const size_t g = gb + r;
      if (ez0 * PZ + r == NZ - 1) p.y[g] = p.residual ? T(0) : p.x[g];
      else p.y[g] = p.residual ? Bc[r] - Yc[r] : Yc[r];
    }
  }
}

template <int P, typename T, int ZT, int PZ = P>
static cudaError_t launch_flat_tile_z(const FlatParams<T>& prm, int EXT, cudaStream_t st) {
  const int ncol = (EXT + 1) * P + 1;
  // x tile, then the right-hand side of the output block (EXT P + 1 columns of nrow)
  size_t sm = ((size_t)ncol * FlatTile<ZT, PZ>::CP + (ncol - 1) / P + 1 +
               (size_t)(EXT * P + 1) * FlatTile<ZT, PZ>::nrow) * sizeof(T);
  auto k = k_flat_tile<P, T, ZT, PZ>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((prm.s.Nx + EXT - 1) / EXT), (unsigned)((prm.s.Nz + ZT - 1) / ZT));
  k<<<grid, EXT * ZT, sm, st>>>(prm, EXT);
  return cudaGetLastError();
}

template <int P, typename T, int PZ = P>
static cudaError_t launch_flat_tile(const FlatParams<T>& prm, int code, cudaStream_t st) {
  const int EXT = (code / 100) % 100, ZT = code % 100;
  return ZT == 4 ? launch_flat_tile_z<P, T, 4, PZ>(prm, EXT, st) : launch_flat_tile_z<P, T, 8, PZ>(prm, EXT, st);
}

template <int P, typename T, bool VAR, int PZ = P>
static cudaError_t launch_flat_p(const FlatParams<T>& prm, int threads, cudaStream_t st) {
  if (flat_bulk_code_ok(threads)) {
    if constexpr (!VAR && std::is_same<T, float>::value && PZ == P) {
      const size_t sm = flat_bulk_smem(P, prm.s, prm.residual);
      if (prm.timeout_flag && ((uintptr_t)prm.x & 15u) == 0 && (!prm.residual || ((uintptr_t)prm.b & 15u) == 0) &&
          sm <= 227 * 1024) {
        auto k = k_flat_bulk<P>;
        static std::atomic<unsigned long long> s_mask{0};
        cudaError_t e = ensure_max_smem(k, s_mask);
        if (e != cudaSuccess) return e;
        k<<<prm.s.Nx, threads - 1000, sm, st>>>(prm);
        return cudaGetLastError();
      }
    }
    threads = 256;  // constant-depth FP32 levels of equal orders on aligned vectors only; else slab CTAs
  }
  if (threads >= 10000) {
    if constexpr (!VAR && std::is_same<T, float>::value && P <= 8 && PZ == P)
      if (flat_tile_code_ok(threads)) return launch_flat_tile<P, T, PZ>(prm, threads, st);
    threads = 256;  // constant-depth FP32 levels of equal orders up to 8 only; else slab CTAs
  }
  if (threads < 0) {  // node-parallel variant, -threads per CTA
    size_t N = (size_t)prm.s.NX * prm.s.NZ;
    int bs = -threads;
    k_flat_np<P, T, VAR, PZ><<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(prm);
    return cudaGetLastError();
  }
  int NZp = slab_pitch(prm.s.NZ);
  size_t sm = ((size_t)((2 * P + 1) + 2 * (P + 1)) * NZp + prm.s.NZ + P + 1 + (VAR ? (P + 1) * (P + 2) : 0)) * sizeof(T);
  auto k = k_flat<P, T, VAR, PZ>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

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
  const T* Vz;      // [4][NBZ][NBZ]  (b, beta)
  const T* invden;  // [4][4][NB][NBZ] (xcls, zcls, alpha, beta): 1/(cx lx + cz lz), 0 if padded
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

// PZ, OZ: order and overlap along sigma when they differ from P, O.  Subdomain blocks are
// NBX = P + 1 + 2 O node lines along x by NBZ = PZ + 1 + 2 OZ along sigma.
template <int P, int O, typename T, int PZ = P, int OZ = O>
__global__ void __launch_bounds__(256) k_fdm(FdmParams<T> p) {
  constexpr int NB = P + 1 + 2 * O;     // along x
  constexpr int NBZ = PZ + 1 + 2 * OZ;  // along sigma
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  const int xc = p.xpercol ? ex : xclass(s, ex);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* R = reinterpret_cast<T*>(smem_raw);  // [NB][NZp]  input, later U
  T* T1 = R + NB * NZp;                    // [NB][NZp]  x-transformed rows
  T* T3 = T1 + NB * NZp;                   // [Nz][NBZ][NB] (ez, b, alpha)
  T* VX = T3 + Nz * NBZ * NB;              // [NB][NB]
  T* VZ = VX + NB * NB;                     // [4][NBZ][NBZ]
  T* ID = VZ + 4 * NBZ * NBZ;              // [4][NB][NBZ]
  T* XS = ID + 4 * NB * NBZ;               // [NB][NZp] x on the subdomain columns (prefetched)
  size_t red_off = (((size_t)(3 * NB * NZp + Nz * NBZ * NB + NB * NB + 4 * NBZ * NBZ + 4 * NB * NBZ) * sizeof(T)) +
                    15) & ~(size_t)15;
  int* s_flag = reinterpret_cast<int*>(smem_raw + red_off);

  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) VX[t] = p.Vx[xc * NB * NB + t];
  for (int t = threadIdx.x; t < 4 * NBZ * NBZ; t += blockDim.x) VZ[t] = p.Vz[t];
  for (int t = threadIdx.x; t < 4 * NB * NBZ; t += blockDim.x) ID[t] = p.invden[xc * 4 * NB * NBZ + t];
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
    const T* vz = VZ + zc * NBZ * NBZ;
    const T* idn = ID + (zc * NB + al) * NBZ;
    T tz[NBZ];
#pragma unroll
    for (int b = 0; b < NBZ; ++b) {
      int iz = ez * PZ - OZ + b;
      tz[b] = (iz >= 0 && iz < NZ - 1) ? T1[al * NZp + iz] : T(0);
    }
    T t2[NBZ];
#pragma unroll
    for (int be = 0; be < NBZ; ++be) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < NBZ; ++b) acc += vz[b * NBZ + be] * tz[b];
      t2[be] = acc * idn[be];
    }
#pragma unroll
    for (int b = 0; b < NBZ; ++b) {
      T acc = T(0);
#pragma unroll
      for (int be = 0; be < NBZ; ++be) acc += vz[b * NBZ + be] * t2[be];
      T3[(ez * NBZ + b) * NB + al] = acc;
    }
  }
  __syncthreads();
  // phase 3: per row, sum the covering elements, inverse x transform -> U[a][iz] (in R)
  T* U = R;
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    T sv[NB];
#pragma unroll
    for (int al = 0; al < NB; ++al) sv[al] = T(0);
    int e0 = (iz + OZ) / PZ;
#pragma unroll
    for (int d = -2; d <= 0; ++d) {
      int ez = e0 + d;
      if (ez < 0 || ez >= Nz) continue;
      int b = iz - ez * PZ + OZ;
      if (b < 0 || b >= NBZ) continue;
#pragma unroll
      for (int al = 0; al < NB; ++al) sv[al] += T3[(ez * NBZ + b) * NB + al];
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

template <int P, int O, typename T, int PZ = P, int OZ = O>
static cudaError_t launch_fdm_p(const FdmParams<T>& prm, int threads, cudaStream_t st) {
  constexpr int NB = P + 1 + 2 * O, NBZ = PZ + 1 + 2 * OZ;
  int NZp = slab_pitch(prm.s.NZ);
  size_t elems = (size_t)3 * NB * NZp + (size_t)prm.s.Nz * NBZ * NB + NB * NB + 4 * NBZ * NBZ + 4 * NB * NBZ;
  size_t sm = ((elems * sizeof(T) + 15) & ~(size_t)15) + 16;
  auto k = k_fdm<P, O, T, PZ, OZ>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// transfers (Sec. 5.2): one CTA per fine element column
// ------------------------------------------------------------------------------------
template <typename T>
struct TransferParams {
  Shape f, c;       // fine and coarse shapes (same cells)
  const T* in;      // prolong: x_c; restrict: r_f, or b_f when xf is set
  T* out;
  const double* J;   // along x: [(Pf+1)][(Pc+1)]
  const double* Jz;  // along sigma: [(Pfz+1)][(Pcz+1)] (equal orders: J)
  // restriction of the residual formed in the kernel: r_f = in - A_f xf (flat level operator)
  const T* xf;
  T cx, cz;
  const T* mX;      // [NXf] assembled LGL weights of the fine level
  const T* mZ;      // [NZf]
};

// x_f += P x_c.  PF, PC > 0: the fine and coarse orders (equal along x and sigma) as
// compile-time constants, so that the 1D interpolation loops unroll and the row-in-element
// division is by a constant; 0: the orders of the shapes at run time.
template <typename T, int PF = 0, int PC = 0>
__device__ __forceinline__ void prolong_body(const TransferParams<T>& p, const int ex) {
  const Shape f = p.f, c = p.c;
  const int Pf = PF ? PF : f.P, Pc = PC ? PC : c.P, nf = Pf + 1, nc = Pc + 1;  // along x
  const int Pfz = PF ? PF : f.pz(), Pcz = PC ? PC : c.pz(), nfz = Pfz + 1, ncz = Pcz + 1;  // along sigma
  const int NZf = f.NZ, NZc = c.NZ, NZcp = slab_pitch(NZc), NZfp = slab_pitch(NZf);
  const bool last = !f.periodic && ex == f.Nx - 1;
  const int own = last ? nf : Pf;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xc = reinterpret_cast<T*>(smem_raw);  // [nc][NZcp]
  T* Tz = Xc + nc * NZcp;                   // [nc][NZfp]
  T* Js = Tz + nc * NZfp;                   // [nf][nc]
  T* Jzs = Js + nf * nc;                    // [nfz][ncz]
  T* Xf = Jzs + nfz * ncz;                  // [nf][NZfp] fine values of the own columns
  for_slab(nc, NZc, [&](int k, int iz) { cp_async_elem(&Xc[k * NZcp + iz], p.in + (size_t)wrap_col(c, ex * Pc + k) * NZc + iz, true); });
  for_slab(own, NZf, [&](int i, int iz) { cp_async_elem(&Xf[i * NZfp + iz], p.out + (size_t)(ex * Pf + i) * NZf + iz, true); });
  for (int t = threadIdx.x; t < nf * nc; t += blockDim.x) Js[t] = (T)p.J[t];
  for (int t = threadIdx.x; t < nfz * ncz; t += blockDim.x) Jzs[t] = (T)p.Jz[t];
  cp_async_wait_all();
  __syncthreads();
  for_slab(nc, NZf, [&](int k, int iz) {
    int ez = min(iz / Pfz, f.Nz - 1), j = iz - ez * Pfz;
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < ncz; ++l) acc += Jzs[j * ncz + l] * Xc[k * NZcp + ez * Pcz + l];
    Tz[k * NZfp + iz] = acc;
  });
  __syncthreads();
  for_slab(own, NZf, [&](int i, int iz) {
    if (iz == NZf - 1) return;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < nc; ++k) acc += Js[i * nc + k] * Tz[k * NZfp + iz];
    p.out[(size_t)(ex * Pf + i) * NZf + iz] = Xf[i * NZfp + iz] + acc;
  });
}
// r_c = P^T r_f (PF, PC as for prolong_body)
template <typename T, int PF = 0, int PC = 0>
__device__ __forceinline__ void restrict_body(const TransferParams<T>& p, const int ex) {
  const Shape f = p.f, c = p.c;
  const int Pf = PF ? PF : f.P, Pc = PC ? PC : c.P, nf = Pf + 1, nc = Pc + 1;  // along x
  const int Pfz = PF ? PF : f.pz(), Pcz = PC ? PC : c.pz(), nfz = Pfz + 1, ncz = Pcz + 1;  // along sigma
  const int NZf = f.NZ, NZc = c.NZ, NZfp = slab_pitch(NZf), NZcp = slab_pitch(NZc);
  const bool left = f.periodic || ex > 0;
  const bool last = !f.periodic && ex == f.Nx - 1;
  const int own = last ? nc : Pc;
  const int ncol = 2 * Pf + 1;  // local fine column q <-> (ex-1) Pf + q
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Rf = reinterpret_cast<T*>(smem_raw);  // [ncol][NZfp]
  T* Sz = Rf + ncol * NZfp;                 // [ncol][NZcp]
  T* Js = Sz + ncol * NZcp;                 // [nf][nc]
  T* Jzs = Js + nf * nc;                    // [nfz][ncz]
  T* Xs = Jzs + nfz * ncz;                  // fused: [ncol][NZfp] fine iterate
  T* MZ = Xs + ncol * NZfp;                 // fused: [NZf] cx * assembled z weights
  T* MX = MZ + NZf;                         // fused: [ncol] cz * assembled x weights
  const bool fused = p.xf != nullptr;
  for (int t = threadIdx.x; t < nf * nc; t += blockDim.x) Js[t] = (T)p.J[t];
  for (int t = threadIdx.x; t < nfz * ncz; t += blockDim.x) Jzs[t] = (T)p.Jz[t];
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
#pragma unroll
      for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, li, m) * Xs[(e * Pf + m) * NZfp + iz];
      if (li == 0 && e == 1 && left) {
#pragma unroll
        for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, Pf, m) * Xs[m * NZfp + iz];
      }
      const int ez = min(iz / Pfz, f.Nz - 1), lj = iz - ez * Pfz;
      const T* col = Xs + q * NZfp;
      T kz = T(0);
#pragma unroll
      for (int m = 0; m < nfz; ++m) kz += CT<T>::K(cT, Pfz, lj, m) * col[ez * Pfz + m];
      if (lj == 0 && ez > 0) {
#pragma unroll
        for (int m = 0; m < nfz; ++m) kz += CT<T>::K(cT, Pfz, Pfz, m) * col[(ez - 1) * Pfz + m];
      }
      Rf[q * NZfp + iz] -= MZ[iz] * kx + MX[q] * kz;
    });
    __syncthreads();
  }
  for_slab(ncol, NZc, [&](int q, int lc) {
    T acc = T(0);
    if (lc != NZc - 1) {
      int ez = min(lc / Pcz, c.Nz - 1), l = lc - ez * Pcz;
      const T* col = Rf + q * NZfp;
      if (l == 0) {
        acc = col[ez * Pfz];
  #pragma unroll
        for (int j = 1; j < Pfz; ++j) acc += Jzs[j * ncz + 0] * col[ez * Pfz + j];
        if (ez > 0) {
  #pragma unroll
          for (int j = 1; j < Pfz; ++j) acc += Jzs[j * ncz + Pcz] * col[(ez - 1) * Pfz + j];
        }
      } else {
  #pragma unroll
        for (int j = 1; j < Pfz; ++j) acc += Jzs[j * ncz + l] * col[ez * Pfz + j];
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
  #pragma unroll
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + 0] * Sz[(Pf + i) * NZcp + lc];
        if (left) {
  #pragma unroll
          for (int i = 1; i < Pf; ++i) acc += Js[i * nc + Pc] * Sz[i * NZcp + lc];
        }
      } else if (k == Pc) {
        acc = Sz[2 * Pf * NZcp + lc];
  #pragma unroll
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + Pc] * Sz[(Pf + i) * NZcp + lc];
      } else {
  #pragma unroll
        for (int i = 1; i < Pf; ++i) acc += Js[i * nc + k] * Sz[(Pf + i) * NZcp + lc];
      }
    }
    p.out[(size_t)(ex * Pc + k) * NZc + lc] = acc;
  });
}
template <typename T>
static inline TransferParams<T> transfer_params(const TransferArgs& a) {
  TransferParams<T> p;
  p.f = a.f;
  p.c = a.c;
  p.in = (const T*)a.in;
  p.out = (T*)a.out;
  p.J = a.J;
  p.Jz = a.Jz ? a.Jz : a.J;
  p.xf = (const T*)a.xf;
  p.cx = (T)a.cx;
  p.cz = (T)a.cz;
  p.mX = (const T*)a.mX;
  p.mZ = (const T*)a.mZ;
  return p;
}
static inline size_t transfer_smem(const TransferArgs& a, int restrict_, size_t word) {
  int nf = a.f.P + 1, nc = a.c.P + 1, nfz = a.f.pz() + 1, ncz = a.c.pz() + 1;
  int NZfp = slab_pitch(a.f.NZ), NZcp = slab_pitch(a.c.NZ);
  if (restrict_) {
    size_t sm = ((size_t)(2 * a.f.P + 1) * (NZfp + NZcp) + nf * nc + nfz * ncz) * word + 16;
    if (a.xf) sm += ((size_t)(2 * a.f.P + 1) * (NZfp + 1) + a.f.NZ) * word;
    return sm;
  }
  return ((size_t)nc * (NZcp + NZfp) + nf * nc + nfz * ncz + (size_t)nf * NZfp) * word + 16;
}

}  // namespace pmg
