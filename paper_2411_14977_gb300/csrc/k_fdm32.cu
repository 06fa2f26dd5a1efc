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
#include <algorithm>
#include <new>

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

}  // namespace pmg

#include "k_fdm32.cuh"

namespace pmg {

// CTA-size bound of the slab sweep: up to order 6 at most 256 threads and three CTAs per
// SM, which caps its registers at 80 (the two slab edges' exchanges in flight together
// otherwise take 100); higher orders 512.
template <int P> constexpr int kFdm32MaxThreads = P <= 6 ? 256 : 512;
template <int P, int O, bool RES>
__global__ void __launch_bounds__(kFdm32MaxThreads<P>, P <= 6 ? 3 : 1) k_fdm32(Fdm32Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ex = blockIdx.x;
  switch (xclass32(p.s, ex)) {
    case 0: fdm32_body<P, O, 0, RES>(p, smem_raw, ex); break;
    case 1: fdm32_body<P, O, 1, RES>(p, smem_raw, ex); break;
    case 2: fdm32_body<P, O, 2, RES>(p, smem_raw, ex); break;
    default: fdm32_body<P, O, 3, RES>(p, smem_raw, ex); break;
  }
}

template <int P, int O, bool RES>
static cudaError_t launch_fdm32_pr(const Fdm32Params& prm, int threads, cudaStream_t st) {
  if (threads > kFdm32MaxThreads<P>) threads = kFdm32MaxThreads<P>;
  size_t sm = fdm32_smem(P, O, RES, prm.s);
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
  if (a.zc > 0) {
    if (!fdm32z_usable(a)) return cudaErrorInvalidValue;
    return fdm_smooth32z(a, st);
  }
  if (a.b && (!a.xout || a.xout == a.x)) return cudaErrorInvalidValue;  // neighbours read x while it is written
  const Fdm32Params p = fdm32_params(a);
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
