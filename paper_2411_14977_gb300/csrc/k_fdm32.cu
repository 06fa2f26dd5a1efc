// FP32 additive-Schwarz sweep by fast diagonalisation (Sec. 5.3), the V-cycle smoother of
// the mixed-precision path.  Same algorithm and data flow as the generic k_fdm (see
// k_levels.cu), but the per-class eigenvectors -- which depend only on the order, the
// overlap and the element class, not on the mesh -- sit in constant memory and are
// addressed at compile time, so every multiply-add of the three transforms is one FFMA
// with a constant-bank operand instead of a shared-memory load plus an FFMA.
//   phase 1  T1 = Vx^T R        per node row (x-transform shared by the element column)
//   phase 2  T3 = Vz (D^-1 o (Vz^T T1_window))   per (x-mode, element)
//   phase 3  U  = Vx (sum of the covering elements' T3)   per node row
//   phase 4  x += omega W U (pre) / omega U with W applied to r (post); slab-edge exchange
// With a right-hand side b the sweep also forms its own residual (phase 0): the CTA loads
// x on the 3P+1 columns that the stencils of its subdomain columns touch and evaluates
// r = b - (cx K_X (x) M_Z + cz M_X (x) K_Z) x there, so the level residual needs neither
// a launch of its own nor a round trip through global memory.  Those columns include the
// neighbouring CTAs' interiors, which they update in the same launch, so the fused sweep
// reads the iterate from one buffer and writes it to another (x -> xout).
#include "pmg_common.cuh"
#include "pmg_kernels.h"

namespace pmg {

static __constant__ float cV32[fdm32_table_size()];
static __constant__ float cK32[MAXP + 1][MAXP + 1][MAXP + 1];  // 1D LGL stiffness per order

cudaError_t init_consts_fdm32(const float* table, size_t n, const float* K, size_t nk) {
  if (n != (size_t)fdm32_table_size() || nk != (size_t)(MAXP + 1) * (MAXP + 1) * (MAXP + 1))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyToSymbol(cV32, table, n * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(cK32, K, nk * sizeof(float));
}

struct Fdm32Params {
  Shape s;
  const float* r;
  float* x;     // iterate in
  float* xout;  // iterate out (== x: in place; required distinct when b is set)
  int xzero;    // the iterate in is zero: not read
  int post;
  float omega;
  const float* Vz;      // [4][NB][NB] z eigenvectors (boundary classes read from shared memory)
  const float* invden;  // [4][4][NB][NB]
  const float* wx;
  const float* wz;
  Scratch sc;
  // fused residual (b != nullptr): r = b - A x with the flat level operator
  const float* b;
  float cx, cz;
  const float* mX;  // [NX] assembled LGL weights along x
  const float* mZ;  // [NZ]
};

__device__ __forceinline__ int xclass32(const Shape& s, int ex) {
  if (s.periodic) return 0;
  return (ex == 0 ? 1 : 0) | (ex == s.Nx - 1 ? 2 : 0);
}

template <int P, int O, int XC, bool RES>
__device__ __forceinline__ void fdm32_body(const Fdm32Params& p, unsigned char* smem_raw) {
  constexpr int NB = P + 1 + 2 * O;
  constexpr int OFF = fdm32_offset(P, O);
  constexpr int VX = OFF + XC * NB * NB;  // x eigenvectors of this CTA's class
  constexpr int VZI = OFF + 4 * NB * NB;  // z eigenvectors of interior elements
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int ex = blockIdx.x, col0 = ex * P;
  float* R = reinterpret_cast<float*>(smem_raw);  // [NB][NZp]  input, later U
  float* T1 = R + NB * NZp;                        // [NB][NZp]
  float* T3 = T1 + NB * NZp;                       // [Nz][NB][NB] (ez, b, alpha)
  float* VZ = T3 + Nz * NB * NB;                   // [4][NB][NB]
  float* ID = VZ + 4 * NB * NB;                    // [4][NB][NB] (zc, alpha, beta)
  // x slab: the subdomain columns [NB][NZp], or with RES the stencil columns [3P+1][NZp]
  // (local column c <-> global col0 - P + c; subdomain column a sits at c = a - O + P)
  constexpr int XCOLS = RES ? 3 * P + 1 : NB;
  constexpr int XOFF = RES ? P - O : 0;
  float* XS = ID + 4 * NB * NB;                    // [XCOLS][NZp]
  float* WZ = XS + XCOLS * NZp;                    // [NZ] inverse cover counts along z
  float* WX = WZ + NZ;                             // [NB] inverse cover counts of the subdomain columns
  float* MZC = WX + NB;                            // [NZ] cx * assembled z weights (RES)
  float* MXC = MZC + (RES ? NZ : 0);               // [NB] cz * assembled x weights (RES)
  size_t red_off = (((size_t)((2 + 0) * NB * NZp + XCOLS * NZp + Nz * NB * NB + 8 * NB * NB + NZ + NB +
                              (RES ? NZ + NB : 0)) * sizeof(float)) + 15) & ~(size_t)15;
  int* s_flag = reinterpret_cast<int*>(smem_raw + red_off);

  if (RES) {
    for_slab(XCOLS, NZ, [&](int c, int iz) {
      int gc = col0 - P + c;
      bool ok = col_valid(s, gc) && iz != NZ - 1;
      ok = ok && !p.xzero;
      cp_async_elem(&XS[c * NZp + iz], p.x + (ok ? (size_t)wrap_col(s, gc) * NZ + iz : 0), ok);
    });
    for_slab(NB, NZ, [&](int a, int iz) {
      int gc = col0 - O + a;
      bool ok = col_valid(s, gc) && iz != NZ - 1;
      cp_async_elem(&R[a * NZp + iz], p.b + (ok ? (size_t)wrap_col(s, gc) * NZ + iz : 0), ok);
    });
    for (int t = threadIdx.x; t < NZ; t += blockDim.x) MZC[t] = p.cx * p.mZ[t];
    if (threadIdx.x < NB) {
      int gc = col0 - O + threadIdx.x;
      MXC[threadIdx.x] = col_valid(s, gc) ? p.cz * p.mX[wrap_col(s, gc)] : 0.f;
    }
  } else {
    for_slab(NB, NZ, [&](int a, int iz) {
      int gc = col0 - O + a;
      bool ok = col_valid(s, gc) && iz != NZ - 1;
      size_t g = ok ? (size_t)wrap_col(s, gc) * NZ + iz : 0;
      cp_async_elem(&R[a * NZp + iz], p.r + g, ok);
      cp_async_elem(&XS[a * NZp + iz], p.x + g, ok && !p.xzero);
    });
  }
  for (int t = threadIdx.x; t < 4 * NB * NB; t += blockDim.x) {
    VZ[t] = p.Vz[t];
    ID[t] = p.invden[XC * 4 * NB * NB + t];
  }
  for (int t = threadIdx.x; t < NZ; t += blockDim.x) WZ[t] = p.wz[t];
  if (threadIdx.x < NB) {
    int gc = col0 - O + threadIdx.x;
    WX[threadIdx.x] = col_valid(s, gc) ? p.wx[wrap_col(s, gc)] : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  if (RES) {
    // phase 0: R = b - A x on the subdomain columns (R holds b, zero off the mesh and on
    // the surface row, which stay zero)
    for_slab(NB, NZ, [&](int a, int iz) {
      if (iz == NZ - 1 || MXC[a] == 0.f) return;
      const int c = a + XOFF;
      const int e = c / P, li = c - e * P;  // element of the slab (0 left, 1 own, 2 right)
      // a wall column is also the last (first) column of the missing element beyond it,
      // whose stencil must not be added: zero data alone does not exclude it
      auto exists = [&](int el) { int g = ex - 1 + el; return s.periodic || (g >= 0 && g < s.Nx); };
      float kx = 0.f;
      if (exists(e)) {
#pragma unroll
        for (int m = 0; m <= P; ++m) kx = fmaf(cK32[P][li][m], XS[(e * P + m) * NZp + iz], kx);
      }
      if (li == 0 && e > 0 && exists(e - 1)) {
#pragma unroll
        for (int m = 0; m <= P; ++m) kx = fmaf(cK32[P][P][m], XS[((e - 1) * P + m) * NZp + iz], kx);
      }
      const int ez = min(iz / P, Nz - 1), lj = iz - ez * P;
      const float* col = XS + c * NZp;
      float kz = 0.f;
#pragma unroll
      for (int m = 0; m <= P; ++m) kz = fmaf(cK32[P][lj][m], col[ez * P + m], kz);
      if (lj == 0 && ez > 0) {
#pragma unroll
        for (int m = 0; m <= P; ++m) kz = fmaf(cK32[P][P][m], col[(ez - 1) * P + m], kz);
      }
      R[a * NZp + iz] -= MZC[iz] * kx + MXC[a] * kz;
    });
    __syncthreads();
  }
  if (p.post) {
    for_slab(NB, NZ, [&](int a, int iz) { R[a * NZp + iz] *= WX[a] * WZ[iz]; });
    __syncthreads();
  }
  // phase 1
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    float rv[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) rv[a] = R[a * NZp + iz];
#pragma unroll
    for (int al = 0; al < NB; ++al) {
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < NB; ++a) acc = fmaf(cV32[VX + a * NB + al], rv[a], acc);
      T1[al * NZp + iz] = acc;
    }
  }
  __syncthreads();
  // phase 2
  for (int t = threadIdx.x; t < NB * Nz; t += blockDim.x) {
    int ez = t / NB, al = t - ez * NB;
    int zc = (ez == 0 ? 1 : 0) | (ez == Nz - 1 ? 2 : 0);
    const float* idn = ID + (zc * NB + al) * NB;
    float tz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      int iz = ez * P - O + b;
      tz[b] = (iz >= 0 && iz < NZ - 1) ? T1[al * NZp + iz] : 0.f;
    }
    float t2[NB];
    float* out = T3 + (ez * NB) * NB + al;
    if (zc == 0) {
#pragma unroll
      for (int be = 0; be < NB; ++be) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) acc = fmaf(cV32[VZI + b * NB + be], tz[b], acc);
        t2[be] = acc * idn[be];
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float acc = 0.f;
#pragma unroll
        for (int be = 0; be < NB; ++be) acc = fmaf(cV32[VZI + b * NB + be], t2[be], acc);
        out[b * NB] = acc;
      }
    } else {
      const float* vz = VZ + zc * NB * NB;
#pragma unroll
      for (int be = 0; be < NB; ++be) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) acc = fmaf(vz[b * NB + be], tz[b], acc);
        t2[be] = acc * idn[be];
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float acc = 0.f;
#pragma unroll
        for (int be = 0; be < NB; ++be) acc = fmaf(vz[b * NB + be], t2[be], acc);
        out[b * NB] = acc;
      }
    }
  }
  __syncthreads();
  // phase 3
  float* U = R;
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    float sv[NB];
#pragma unroll
    for (int al = 0; al < NB; ++al) sv[al] = 0.f;
    int e0 = (iz + O) / P;
#pragma unroll
    for (int d = -2; d <= 0; ++d) {
      int ez = e0 + d;
      if (ez < 0 || ez >= Nz) continue;
      int b = iz - ez * P + O;
      if (b < 0 || b >= NB) continue;
      const float* src = T3 + (ez * NB + b) * NB;
#pragma unroll
      for (int al = 0; al < NB; ++al) sv[al] += src[al];
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      float acc = 0.f;
#pragma unroll
      for (int al = 0; al < NB; ++al) acc = fmaf(cV32[VX + a * NB + al], sv[al], acc);
      U[a * NZp + iz] = acc;
    }
  }
  __syncthreads();
  // phase 4
  auto upd = [&](int a, int iz, float u) {
    if (iz == NZ - 1) return;
    int c = wrap_col(s, col0 - O + a);
    float w = p.post ? 1.f : WX[a] * WZ[iz];
    p.xout[(size_t)c * NZ + iz] = XS[(a + XOFF) * NZp + iz] + p.omega * w * u;
  };
  constexpr int ZW = 2 * O + 1;
  unsigned long long* xb = reinterpret_cast<unsigned long long*>(p.sc.xbuf);
  for_slab(P - 1 - 2 * O, NZ, [&](int c, int iz) {
    int a = 2 * O + 1 + c;
    upd(a, iz, U[a * NZp + iz]);
  });
  // Edge zones of both sides, 2 ZW NZ nodes.  A thread swaps up to K partials into their
  // slots back to back -- independent atomics in flight together instead of one L2 round
  // trip per node -- and then finalises those whose partner had already arrived.
  {
    const int e_left = ex, e_right = s.periodic ? (ex + 1) % s.Nx : ex + 1;
    const bool sh_left = s.periodic || ex != 0, sh_right = s.periodic || ex + 1 != s.Nx;
    const int zone = ZW * NZ, total = 2 * zone;
    constexpr int K = 4;
    for (int base = threadIdx.x; base < total; base += K * blockDim.x) {
      unsigned long long old[K];
      unsigned long long* slot[K];
      float u[K];
      int aa[K], zz[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        old[k] = kEmpty64;
        slot[k] = nullptr;
        const int idx = base + k * blockDim.x;
        if (idx >= total) continue;
        const int side = idx >= zone ? 1 : 0;
        const int rem = idx - side * zone;
        const int c = rem / NZ, iz = rem - c * NZ;
        aa[k] = (side ? P : 0) + c;
        zz[k] = iz;
        u[k] = U[aa[k] * NZp + iz];
        const int e = side ? e_right : e_left;
        if (side ? sh_right : sh_left) {
          slot[k] = xb + ((size_t)e * ZW + c) * NZ + iz;
          old[k] = atomicExch(slot[k], (unsigned long long)__float_as_uint(u[k]));
        } else if (col_valid(s, e * P - O + c)) {
          upd(aa[k], iz, u[k]);  // wall: this CTA is the only contributor
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (slot[k] && old[k] != kEmpty64) {  // second to arrive: the sum is complete
          float tot = u[k] + __uint_as_float((unsigned)old[k]);
          atomicExch(slot[k], kEmpty64);
          upd(aa[k], zz[k], tot);
        }
      }
    }
  }
}

template <int P, int O, bool RES>
__global__ void __launch_bounds__(512) k_fdm32(Fdm32Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  switch (xclass32(p.s, blockIdx.x)) {
    case 0: fdm32_body<P, O, 0, RES>(p, smem_raw); break;
    case 1: fdm32_body<P, O, 1, RES>(p, smem_raw); break;
    case 2: fdm32_body<P, O, 2, RES>(p, smem_raw); break;
    default: fdm32_body<P, O, 3, RES>(p, smem_raw); break;
  }
}

template <int P, int O, bool RES>
static cudaError_t launch_fdm32_pr(const Fdm32Params& prm, int threads, cudaStream_t st) {
  constexpr int NB = P + 1 + 2 * O;
  constexpr int XCOLS = RES ? 3 * P + 1 : NB;
  int NZp = slab_pitch(prm.s.NZ);
  size_t elems = (size_t)(2 * NB + XCOLS) * NZp + (size_t)prm.s.Nz * NB * NB + 8 * NB * NB + prm.s.NZ + NB +
                 (RES ? prm.s.NZ + NB : 0);
  size_t sm = ((elems * sizeof(float) + 15) & ~(size_t)15) + 16;
  auto k = k_fdm32<P, O, RES>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

template <int P, int O>
static cudaError_t launch_fdm32_p(const Fdm32Params& prm, int threads, cudaStream_t st) {
  return prm.b ? launch_fdm32_pr<P, O, true>(prm, threads, st) : launch_fdm32_pr<P, O, false>(prm, threads, st);
}

cudaError_t fdm_smooth32(const FdmArgs& a, cudaStream_t st) {
  Fdm32Params p;
  p.s = a.s;
  p.r = (const float*)a.r;
  p.x = (float*)a.x;
  p.xout = a.xout ? (float*)a.xout : (float*)a.x;
  p.xzero = a.xzero;
  if (a.b && p.xout == p.x) return cudaErrorInvalidValue;  // neighbours read x while it is written
  p.post = a.post;
  p.omega = (float)a.omega;
  p.Vz = (const float*)a.Vz;
  p.invden = (const float*)a.invden;
  p.wx = (const float*)a.wx;
  p.wz = (const float*)a.wz;
  p.sc = a.sc;
  p.b = (const float*)a.b;
  p.cx = (float)a.cx;
  p.cz = (float)a.cz;
  p.mX = (const float*)a.mX;
  p.mZ = (const float*)a.mZ;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  if (a.overlap == 0) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm32_p<PP, 0>(p, thr, st);
      PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  } else if (a.overlap == 1) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm32_p<PP, 1>(p, thr, st);
      PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace pmg
