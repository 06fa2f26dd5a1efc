// Coarsest-level solve and Krylov vector kernels.
//
// Coarse level (order 1, flat geometry): A_1 = cx K_X (x) M_Z + cz M_X (x) K_Z on the free
// nodes.  With the generalized eigenvectors of (K_Z, M_Z) on the free rows
// (V^T M_Z V = I, V^T K_Z V = diag(mu)) the system splits into one tridiagonal system
// (cx K_X + cz mu_k M_X) u_k = (V^T r)_k per vertical mode k, solved by parallel cyclic
// reduction in shared memory with multipliers precomputed on the host; u = V u_hat.
// All coarse arithmetic is FP64 whatever the precision of the V-cycle.
//
// Vector kernels: dot products and the CG/FCG updates, with FP64 accumulation and the
// deterministic grid reduction of pmg_common.cuh.  Step scalars (alpha, beta, norms) live
// in device memory; no host round trip is needed inside an iteration.
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"
#include "k_coarse.cuh"

namespace pmg {

template <typename T>
__global__ void k_coarse_fwd(int NX1, int NZ1, const T* b, const double* V, double* rhat) {
  coarse_fwd_body<T>(NX1, NZ1, b, V, rhat, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_coarse_pcr(int n, int nsteps, int periodic, const double* coef, const double* inv,
                             double* rhat, double* gbuf) {
  extern __shared__ double sbuf[];
  coarse_pcr_body(n, nsteps, periodic, coef, inv, rhat, gbuf, blockIdx.x, sbuf);
}

template <typename T>
__global__ void k_coarse_bwd(int NX1, int NZ1, const double* V, const double* uhat, T* x) {
  coarse_bwd_body<T>(NX1, NZ1, V, uhat, x, blockIdx.x * (size_t)blockDim.x + threadIdx.x);
}

template <typename T>
cudaError_t coarse_solve(const CoarseArgs& a, const void* b, void* x, cudaStream_t st) {
  int Nz = a.NZ1 - 1;
  int tot = a.NX1 * Nz, bs = 256;
  k_coarse_fwd<T><<<(tot + bs - 1) / bs, bs, 0, st>>>(a.NX1, a.NZ1, (const T*)b, a.V, a.work);
  int thr = a.NX1 < 1024 ? ((a.NX1 + 31) / 32) * 32 : 1024;
  size_t sm = 2 * (size_t)a.NX1 * sizeof(double);
  double* gbuf = nullptr;
  if (sm > 200 * 1024) {  // does not fit in shared memory: ping-pong through global scratch
    gbuf = a.pcr_buf;
    sm = 0;
  } else if (sm > 48 * 1024) {
    static std::atomic<unsigned long long> s_mask{0};
    cudaError_t e = ensure_max_smem(k_coarse_pcr, s_mask);
    if (e != cudaSuccess) return e;
  }
  k_coarse_pcr<<<Nz, thr, sm, st>>>(a.NX1, a.nsteps, a.periodic, a.coef, a.inv, a.work, gbuf);
  size_t N = (size_t)a.NX1 * a.NZ1;
  k_coarse_bwd<T><<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(a.NX1, a.NZ1, a.V, a.work, (T*)x);
  return cudaGetLastError();
}
template cudaError_t coarse_solve<double>(const CoarseArgs&, const void*, void*, cudaStream_t);
template cudaError_t coarse_solve<float>(const CoarseArgs&, const void*, void*, cudaStream_t);

// ------------------------------------------------------------------------------------
// vector kernels
// ------------------------------------------------------------------------------------
constexpr int VEC_BLOCKS = 304;  // 2 x 152 SMs
constexpr int VEC_THREADS = 512;

// out[0] = <x, y> (FP64 accumulation); shift: out[1] = old out[0] first.
template <typename TA, typename TB>
__global__ void __launch_bounds__(VEC_THREADS) k_dot(size_t n, const TA* x, const TB* y, double* out,
                                                     int shift, Scratch sc) {
  __shared__ double red[34];
  __shared__ int s_flag;
  Acc<TA> a;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a.fma(x[i], (TA)y[i]);
  double acc = block_sum(a.value(), red);
  if (threadIdx.x == 0) {
    sc.partials[blockIdx.x] = acc;
    __threadfence();
    s_flag = (atomicAdd(sc.redcnt, 1u) == gridDim.x - 1);
    if (s_flag) __threadfence();
  }
  __syncthreads();
  if (!s_flag) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)sc.partials)[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    if (shift) out[1] = out[0];
    out[0] = v;
    *sc.redcnt = 0u;
  }
}

// Scalars layout (double): see Slot in pmg_kernels.h.
// x += alpha p, r -= alpha w, (r_old = r), RR = ||r||^2;  alpha = RZ / PAP.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS) k_cg_update(size_t n, T* x, T* r, const T* p, const T* w,
                                                           T* r_old, double* s, Scratch sc, float* r32) {
  __shared__ double red[34];
  __shared__ int s_flag;
  __shared__ T s_alpha;
  if (threadIdx.x == 0) s_alpha = (T)(s[SLOT_RZ] / s[SLOT_PAP]);  // one FP64 division per block
  __syncthreads();
  const T a = s_alpha;
  Acc<T> ac;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T ri = r[i];
    if (r_old) r_old[i] = ri;
    x[i] += a * p[i];
    ri -= a * w[i];
    r[i] = ri;
    if (r32) r32[i] = (float)ri;  // the FP32 copy the next V-cycle reads
    ac.fma(ri, ri);
  }
  double acc = block_sum(ac.value(), red);
  if (threadIdx.x == 0) {
    sc.partials[blockIdx.x] = acc;
    __threadfence();
    s_flag = (atomicAdd(sc.redcnt, 1u) == gridDim.x - 1);
    if (s_flag) __threadfence();
  }
  __syncthreads();
  if (!s_flag) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)sc.partials)[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    s[SLOT_RR] = v;
    *sc.redcnt = 0u;
  }
}

// RZ_new = <r, z> (and for flexible CG ZRO = <z, r_old>), shifting RZ -> RZOLD.
template <typename T, typename TZ>
__global__ void __launch_bounds__(VEC_THREADS) k_rz(size_t n, const T* r, const TZ* z, const T* r_old,
                                                    double* s, Scratch sc) {
  __shared__ double red[34];
  __shared__ int s_flag;
  Acc<T> c1, c2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T zi = (T)z[i];  // an FP32 preconditioned residual widens exactly
    c1.fma(r[i], zi);
    if (r_old) c2.fma(r_old[i], zi);
  }
  double a1 = block_sum(c1.value(), red);
  double a2 = block_sum(c2.value(), red);
  if (threadIdx.x == 0) {
    sc.partials[2 * blockIdx.x] = a1;
    sc.partials[2 * blockIdx.x + 1] = a2;
    __threadfence();
    s_flag = (atomicAdd(sc.redcnt, 1u) == gridDim.x - 1);
    if (s_flag) __threadfence();
  }
  __syncthreads();
  if (!s_flag) return;
  double v1 = 0.0, v2 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    v1 += ((volatile double*)sc.partials)[2 * i];
    v2 += ((volatile double*)sc.partials)[2 * i + 1];
  }
  v1 = block_sum(v1, red);
  v2 = block_sum(v2, red);
  if (threadIdx.x == 0) {
    s[SLOT_RZOLD] = s[SLOT_RZ];
    s[SLOT_RZ] = v1;
    s[SLOT_ZRO] = v2;
    *sc.redcnt = 0u;
  }
}

// p = z + beta p with beta = RZ/RZOLD (CG) or (RZ - ZRO)/RZOLD (flexible CG); first: p = z.
template <typename T, typename TZ>
__global__ void k_p_update(size_t n, T* p, const TZ* z, const double* s, int flexible, int first) {
  __shared__ T s_beta;
  if (threadIdx.x == 0)
    s_beta = first ? T(0) : (T)((flexible ? (s[SLOT_RZ] - s[SLOT_ZRO]) : s[SLOT_RZ]) / s[SLOT_RZOLD]);
  __syncthreads();
  const T b = s_beta;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = first ? (T)z[i] : (T)z[i] + b * p[i];
}

// y = (float)(x * (1/sqrt(s[slot])))  (unit-norm scaling of a residual for the FP32 solve)
__global__ void k_to_f32_scaled(size_t n, const double* x, float* y, const double* s, int slot) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double nr = sqrt(s[slot]);
    s_inv = nr > 0.0 ? 1.0 / nr : 0.0;
  }
  __syncthreads();
  const double inv = s_inv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)(x[i] * inv);
}
// x += sqrt(s[slot]) * (double)c
__global__ void k_add_f32_scaled(size_t n, double* x, const float* c, const double* s, int slot) {
  __shared__ double s_nr;
  if (threadIdx.x == 0) s_nr = sqrt(s[slot]);
  __syncthreads();
  const double nr = s_nr;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += nr * (double)c[i];
}
// y = (float)x and x = (double)y casts (the FP32 preconditioner inside an FP64 Krylov loop)
__global__ void k_cast_f32(size_t n, const double* x, float* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_cast_f64(size_t n, const float* x, double* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
// x += y (same type)
template <typename T>
__global__ void k_add(size_t n, T* x, const T* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += y[i];
}
// x = x0 (or 0) on free nodes, p_D on the surface row; out-of-range values flagged.
__global__ void k_init_x(size_t n, int NZ, double* x, const double* x0, const double* pD, int* status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    bool top = (int)(i % NZ) == NZ - 1;
    double v = top ? pD[i] : (x0 ? x0[i] : 0.0);
    if (!isfinite(v)) atomicExch(status, 1);
    x[i] = v;
  }
}
__global__ void k_check_finite(size_t n, const double* v, int* status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) atomicExch(status, 1);
}

// Device-side loop control of a graph while-node: counts the iteration and keeps the loop
// running while ||r||^2 > thresh2 * (bb ? *bb : 1) and the cap is not reached (a NaN stops it).
__global__ void k_loop_cond(cudaGraphConditionalHandle hnd, const double* s, const double* bb, double thresh2,
                            int* iter, int max_iter) {
  int it = ++(*iter);
  double lim = thresh2 * (bb ? *bb : 1.0);
  unsigned more = (s[SLOT_RR] > lim && it < max_iter) ? 1u : 0u;
  cudaGraphSetConditional(hnd, more);
}

cudaError_t loop_cond(cudaGraphConditionalHandle hnd, const double* s, const double* bb, double thresh2, int* iter,
                      int max_iter, cudaStream_t st) {
  k_loop_cond<<<1, 1, 0, st>>>(hnd, s, bb, thresh2, iter, max_iter);
  return cudaGetLastError();
}

// Fill the 8-byte exchange slots with the empty marker.
__global__ void k_arm_exchange(unsigned long long* buf, size_t n8) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = kEmpty64;
}

static unsigned vec_grid(size_t n) {
  size_t b = (n + VEC_THREADS - 1) / VEC_THREADS;
  return (unsigned)(b < (size_t)VEC_BLOCKS ? (b > 0 ? b : 1) : VEC_BLOCKS);
}

template <typename TA, typename TB>
cudaError_t dot(size_t n, const TA* x, const TB* y, double* out, int shift, const Scratch& sc, cudaStream_t st) {
  k_dot<TA, TB><<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, y, out, shift, sc);
  return cudaGetLastError();
}
template cudaError_t dot<double, double>(size_t, const double*, const double*, double*, int, const Scratch&, cudaStream_t);
template cudaError_t dot<float, float>(size_t, const float*, const float*, double*, int, const Scratch&, cudaStream_t);

template <typename T>
cudaError_t cg_update(size_t n, T* x, T* r, const T* p, const T* w, T* r_old, double* s, const Scratch& sc,
                      cudaStream_t st, float* r32) {
  k_cg_update<T><<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, r, p, w, r_old, s, sc, r32);
  return cudaGetLastError();
}
template cudaError_t cg_update<double>(size_t, double*, double*, const double*, const double*, double*, double*,
                                       const Scratch&, cudaStream_t, float*);
template cudaError_t cg_update<float>(size_t, float*, float*, const float*, const float*, float*, double*,
                                      const Scratch&, cudaStream_t, float*);

template <typename T, typename TZ>
cudaError_t rz(size_t n, const T* r, const TZ* z, const T* r_old, double* s, const Scratch& sc, cudaStream_t st) {
  k_rz<T, TZ><<<vec_grid(n), VEC_THREADS, 0, st>>>(n, r, z, r_old, s, sc);
  return cudaGetLastError();
}
template cudaError_t rz<double, double>(size_t, const double*, const double*, const double*, double*, const Scratch&, cudaStream_t);
template cudaError_t rz<double, float>(size_t, const double*, const float*, const double*, double*, const Scratch&, cudaStream_t);
template cudaError_t rz<float, float>(size_t, const float*, const float*, const float*, double*, const Scratch&, cudaStream_t);

template <typename T, typename TZ>
cudaError_t p_update(size_t n, T* p, const TZ* z, const double* s, int flexible, int first, cudaStream_t st) {
  k_p_update<T, TZ><<<vec_grid(n), VEC_THREADS, 0, st>>>(n, p, z, s, flexible, first);
  return cudaGetLastError();
}
template cudaError_t p_update<double, double>(size_t, double*, const double*, const double*, int, int, cudaStream_t);
template cudaError_t p_update<double, float>(size_t, double*, const float*, const double*, int, int, cudaStream_t);
template cudaError_t p_update<float, float>(size_t, float*, const float*, const double*, int, int, cudaStream_t);

cudaError_t to_f32_scaled(size_t n, const double* x, float* y, const double* s, int slot, cudaStream_t st) {
  k_to_f32_scaled<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, y, s, slot);
  return cudaGetLastError();
}
cudaError_t add_f32_scaled(size_t n, double* x, const float* c, const double* s, int slot, cudaStream_t st) {
  k_add_f32_scaled<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, c, s, slot);
  return cudaGetLastError();
}
cudaError_t cast_f32(size_t n, const double* x, float* y, cudaStream_t st) {
  k_cast_f32<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, y);
  return cudaGetLastError();
}
cudaError_t cast_f64(size_t n, const float* x, double* y, cudaStream_t st) {
  k_cast_f64<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, y);
  return cudaGetLastError();
}
template <typename T>
cudaError_t add(size_t n, T* x, const T* y, cudaStream_t st) {
  k_add<T><<<vec_grid(n), VEC_THREADS, 0, st>>>(n, x, y);
  return cudaGetLastError();
}
template cudaError_t add<double>(size_t, double*, const double*, cudaStream_t);
template cudaError_t add<float>(size_t, float*, const float*, cudaStream_t);

cudaError_t init_x(size_t n, int NZ, double* x, const double* x0, const double* pD, int* status, cudaStream_t st) {
  k_init_x<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, NZ, x, x0, pD, status);
  return cudaGetLastError();
}
cudaError_t arm_exchange(void* buf, size_t n8) {
  k_arm_exchange<<<vec_grid(n8), VEC_THREADS>>>(static_cast<unsigned long long*>(buf), n8);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaDeviceSynchronize();
}
cudaError_t arm_exchange_f64(void* buf, size_t n8, cudaStream_t st) {
  k_arm_exchange<<<vec_grid(n8), VEC_THREADS, 0, st>>>(static_cast<unsigned long long*>(buf), n8);
  return cudaGetLastError();
}

cudaError_t check_finite(size_t n, const double* v, int* status, cudaStream_t st) {
  k_check_finite<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, v, status);
  return cudaGetLastError();
}

// ---- GMRES (Arnoldi) vector kernels -------------------------------------------------
// h[k] = <w, V_k> for k < nv (V_k = V + k n): per-block partials of every k, then the last
// block to finish (ticket) adds them in block order, so the sums are deterministic.
__global__ void __launch_bounds__(VEC_THREADS) k_mdot(size_t n, const double* w, const double* V, int nv,
                                                      double* h, double* part, unsigned* cnt, const int* nvdev) {
  __shared__ double red[34];
  __shared__ int s_flag;
  if (nvdev) nv = *nvdev + 1;  // device-side Arnoldi index j: the vectors V_0 .. V_j
  for (int k = 0; k < nv; ++k) {
    const double* v = V + (size_t)k * n;
    double a = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      a = fma(w[i], v[i], a);
    a = block_sum(a, red);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = a;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_flag = (atomicAdd(cnt, 1u) == gridDim.x - 1);
    if (s_flag) __threadfence();
  }
  __syncthreads();
  if (!s_flag) return;
  for (int k = 0; k < nv; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += ((volatile double*)part)[(size_t)k * gridDim.x + b];
    v = block_sum(v, red);
    if (threadIdx.x == 0) h[k] = v;
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// w += sign sum_k c[k] V_k  (c on the device; nvdev: nv = *nvdev + nvadd)
__global__ void k_maxpy(size_t n, double* w, const double* V, int nv, const double* c, double sign, const int* nvdev,
                        int nvadd) {
  __shared__ double cs[64];
  if (nvdev) nv = *nvdev + nvadd;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = sign * c[k];
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int k = 0; k < nv; ++k) a = fma(cs[k], V[(size_t)k * n + i], a);
    w[i] = a;
  }
}

// v = w / sqrt(*nrm2)   (a zero norm leaves v unused: the caller stops the cycle);
// jdev: v is the basis vector V_(j+1) of v = V
__global__ void k_scale_inv_norm(size_t n, const double* w, const double* nrm2, double* v, const int* jdev) {
  double s = 1.0 / sqrt(*nrm2);
  if (jdev) v += (size_t)(*jdev + 1) * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * s;
}

cudaError_t gmres_mdot(size_t n, const double* w, const double* V, int nv, double* h, double* part, unsigned* cnt,
                       cudaStream_t st, const int* jdev) {
  k_mdot<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(n, w, V, nv, h, part, cnt, jdev);
  return cudaGetLastError();
}
cudaError_t gmres_maxpy(size_t n, double* w, const double* V, int nv, const double* c, double sign, cudaStream_t st,
                        const int* nvdev, int nvadd) {
  if (nv > 64) return cudaErrorInvalidValue;
  k_maxpy<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, w, V, nv, c, sign, nvdev, nvadd);
  return cudaGetLastError();
}
cudaError_t gmres_scale(size_t n, const double* w, const double* nrm2, double* v, cudaStream_t st, const int* jdev) {
  k_scale_inv_norm<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, w, nrm2, v, jdev);
  return cudaGetLastError();
}

// ---- device-side GMRES cycle (graph with a while-node) -----------------------------
// State: j (the Arnoldi index, = the cycle's iteration count), the cap of iterations for
// this cycle, the Hessenberg matrix H [(m+1) x m] after the rotations, their cosines and
// sines, g (the rotated right-hand side, ||r|| e_1 at the start) and y.

// V_j (device j) into the V-cycle input: FP64 (v64) or FP32 (v32)
__global__ void k_gm_gather(size_t n, const double* V, const int* jdev, double* v64, float* v32) {
  const double* vj = V + (size_t)(*jdev) * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (v64) v64[i] = vj[i];
    else v32[i] = (float)vj[i];
  }
}

// Z_j = z (the V-cycle output: FP64 z64, or FP32 z32 widened, also into zw)
__global__ void k_gm_scatter(size_t n, const double* z64, const float* z32, double* Z, const int* jdev, double* zw) {
  double* zj = Z + (size_t)(*jdev) * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double v = z64 ? z64[i] : (double)z32[i];
    zj[i] = v;
    if (zw) zw[i] = v;
  }
}

// Start of a cycle: j = 0, g = ||r|| e_1, cap = this cycle's iteration limit, counter 0.
__global__ void k_gm_init(const double* rr, double* g, int m, int* jdev, int* capdev, int cap, int* iter) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? sqrt(*rr) : 0.0;
  if (threadIdx.x == 0) {
    *jdev = 0;
    *capdev = cap;
    *iter = 0;
  }
}

// Column j of H from the two Gram-Schmidt passes (c1, c2) and ||w||^2 (hn2), the earlier
// rotations on it, a new rotation zeroing H[j+1][j], g rotated.  Continue while the
// residual estimate |g[j+1]|^2 is above tol2 ||b~||^2 (*bb), the cycle has room, and no breakdown
// (a zero or non-finite ||w|| or pivot).  out[0] = |g[j+1]|^2, out[1] = 1 on breakdown.
__global__ void k_gm_givens(cudaGraphConditionalHandle hnd, const double* c1, const double* c2, const double* hn2,
                            double* H, double* cs, double* sn, double* g, int m, int* jdev, const int* capdev,
                            int* iter, double tol2, const double* bb, double* out) {
  const int j = *jdev;
  double* col = H + j;  // H[i][j] = H[i * m + j]
  for (int i = 0; i <= j; ++i) col[(size_t)i * m] = c1[i] + c2[i];
  const double hn = sqrt(fmax(*hn2, 0.0));
  for (int i = 0; i < j; ++i) {
    double a = col[(size_t)i * m], b = col[(size_t)(i + 1) * m];
    col[(size_t)i * m] = cs[i] * a + sn[i] * b;
    col[(size_t)(i + 1) * m] = -sn[i] * a + cs[i] * b;
  }
  const double hjj = col[(size_t)j * m];
  const double den = hypot(hjj, hn);
  const bool ok = den > 0.0 && isfinite(den);
  double c = ok ? hjj / den : 1.0, sv = ok ? hn / den : 0.0;
  cs[j] = c;
  sn[j] = sv;
  col[(size_t)j * m] = ok ? den : hjj;
  g[j + 1] = -sv * g[j];
  g[j] = c * g[j];
  const int it = ++(*iter);
  *jdev = j + 1;
  const double r2 = g[j + 1] * g[j + 1];
  out[0] = r2;
  out[1] = ok ? 0.0 : 1.0;
  const bool more = ok && hn > 0.0 && isfinite(r2) && r2 > tol2 * (*bb) && j + 1 < m && it < *capdev;
  cudaGraphSetConditional(hnd, more ? 1u : 0u);
}

// y = H^-1 g over the k = j leading rows (back substitution)
__global__ void k_gm_backsub(const double* H, const double* g, double* y, int m, const int* jdev) {
  const int k = *jdev;
  for (int i = k - 1; i >= 0; --i) {
    double v = g[i];
    for (int l = i + 1; l < k; ++l) v -= H[(size_t)i * m + l] * y[l];
    y[i] = v / H[(size_t)i * m + i];
  }
}

cudaError_t gmres_gather(size_t n, const double* V, const int* jdev, double* v64, float* v32, cudaStream_t st) {
  k_gm_gather<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, V, jdev, v64, v32);
  return cudaGetLastError();
}
cudaError_t gmres_scatter(size_t n, const double* z64, const float* z32, double* Z, const int* jdev, double* zw,
                          cudaStream_t st) {
  k_gm_scatter<<<vec_grid(n), VEC_THREADS, 0, st>>>(n, z64, z32, Z, jdev, zw);
  return cudaGetLastError();
}
cudaError_t gmres_init(const double* rr, double* g, int m, int* jdev, int* capdev, int cap, int* iter,
                       cudaStream_t st) {
  k_gm_init<<<1, 64, 0, st>>>(rr, g, m, jdev, capdev, cap, iter);
  return cudaGetLastError();
}
cudaError_t gmres_givens(cudaGraphConditionalHandle hnd, const double* c1, const double* c2, const double* hn2,
                         double* H, double* cs, double* sn, double* g, int m, int* jdev, const int* capdev,
                         int* iter, double tol2, const double* bb, double* out, cudaStream_t st) {
  k_gm_givens<<<1, 1, 0, st>>>(hnd, c1, c2, hn2, H, cs, sn, g, m, jdev, capdev, iter, tol2, bb, out);
  return cudaGetLastError();
}
cudaError_t gmres_backsub(const double* H, const double* g, double* y, int m, const int* jdev, cudaStream_t st) {
  k_gm_backsub<<<1, 1, 0, st>>>(H, g, y, m, jdev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// batched launches: the coarse solves and Krylov vector kernels of a batch of problems
// ------------------------------------------------------------------------------------
struct CoarseBatch {
  BatchMap m[3];  // fwd, pcr, bwd
  CoarseArgs a[kMaxBatch];
  const float* b[kMaxBatch];
  float* x[kMaxBatch];
  int gbuf[kMaxBatch];  // 1: the PCR ping-pong runs in the problem's global scratch
};
__global__ void __launch_bounds__(256) k_coarse_fwd_batch(const CoarseBatch* tab) {
  batch_items(tab->m[0], [&](int r, int k) {
    const CoarseArgs& a = tab->a[r];
    coarse_fwd_body<float>(a.NX1, a.NZ1, tab->b[r], a.V, a.work, k * blockDim.x + threadIdx.x);
  });
}
__global__ void __launch_bounds__(1024) k_coarse_pcr_batch(const CoarseBatch* tab) {
  extern __shared__ double sbuf[];
  batch_items(tab->m[1], [&](int r, int k) {
    const CoarseArgs& a = tab->a[r];
    coarse_pcr_body(a.NX1, a.nsteps, a.periodic, a.coef, a.inv, a.work, tab->gbuf[r] ? a.pcr_buf : nullptr, k,
                    sbuf);
    __syncthreads();
  });
}
__global__ void __launch_bounds__(256) k_coarse_bwd_batch(const CoarseBatch* tab) {
  batch_items(tab->m[2], [&](int r, int k) {
    const CoarseArgs& a = tab->a[r];
    coarse_bwd_body<float>(a.NX1, a.NZ1, a.V, a.work, tab->x[r], (size_t)k * blockDim.x + threadIdx.x);
  });
}

cudaError_t coarse_batch_table(const CoarseArgs* a, const float* const* b, float* const* x, const int* prob, int n,
                               const int* active, void** table, int nctas[3], size_t* smem) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  CoarseBatch* h = new (std::nothrow) CoarseBatch();
  if (!h) return cudaErrorMemoryAllocation;
  size_t sm = 0;
  for (int k = 0; k < 3; ++k) {
    h->m[k].nrange = n;
    h->m[k].active = active;
    h->m[k].start[0] = 0;
  }
  for (int i = 0; i < n; ++i) {
    h->a[i] = a[i];
    h->b[i] = b[i];
    h->x[i] = x[i];
    const int Nz = a[i].NZ1 - 1;
    const size_t pcr = 2 * (size_t)a[i].NX1 * sizeof(double);
    h->gbuf[i] = pcr > 200 * 1024 ? 1 : 0;
    if (!h->gbuf[i]) sm = std::max(sm, pcr);
    for (int k = 0; k < 3; ++k) h->m[k].prob[i] = prob[i];
    h->m[0].start[i + 1] = h->m[0].start[i] + (a[i].NX1 * Nz + 255) / 256;
    h->m[1].start[i + 1] = h->m[1].start[i] + Nz;
    h->m[2].start[i + 1] = h->m[2].start[i] + (int)(((size_t)a[i].NX1 * a[i].NZ1 + 255) / 256);
  }
  for (int k = 0; k < 3; ++k) nctas[k] = h->m[k].start[n];
  *smem = sm;
  BatchMap* maps[3] = {&h->m[0], &h->m[1], &h->m[2]};
  cudaError_t e = batch_upload(h, maps, 3, table);
  delete h;
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> s_mask{0};
  return ensure_max_smem(k_coarse_pcr_batch, s_mask);
}
cudaError_t coarse_batch_launch(const void* table, const int nctas[3], size_t smem, cudaStream_t st) {
  const CoarseBatch* t = static_cast<const CoarseBatch*>(table);
  int g0 = 0, g1 = 0, g2 = 0;
  cudaError_t e = batch_grid(k_coarse_fwd_batch, 256, 0, nctas[0], &g0);
  if (e == cudaSuccess) e = batch_grid(k_coarse_pcr_batch, 1024, smem, nctas[1], &g1);
  if (e == cudaSuccess) e = batch_grid(k_coarse_bwd_batch, 256, 0, nctas[2], &g2);
  if (e != cudaSuccess) return e;
  k_coarse_fwd_batch<<<g0, 256, 0, st>>>(t);
  k_coarse_pcr_batch<<<g1, 1024, smem, st>>>(t);
  k_coarse_bwd_batch<<<g2, 256, 0, st>>>(t);
  return cudaGetLastError();
}

struct VecBatch {
  BatchMap m[VB_COUNT];
  VecProb prm[kMaxBatch];
  int nb[kMaxBatch];  // CTAs of each problem in the reduction kernels
  BatchState st;
  const BatchIO* io;
  int n;
};
constexpr int VB_THREADS = 512;

// The work of item bx (one CTA's share) of range r of a vector kernel.
template <int WHICH>
__device__ __forceinline__ void vec_item(const VecBatch* tab, int r, int bx, double* red, int* s_flag) {
  const BatchMap& m = tab->m[WHICH];
  const int prob = m.prob[r];
  const VecProb& q = tab->prm[r];
  const size_t n = q.n;
  if constexpr (WHICH == VB_INIT || WHICH == VB_COPY_OUT) {
    const size_t g = (size_t)bx * VB_THREADS + threadIdx.x;
    if (g >= n) return;
    const BatchIO io = tab->io[prob];
    if constexpr (WHICH == VB_INIT) {
      // the load vector into the problem's copy; x = 0 with p_D on the surface row
      const double bv = io.b[g];
      if (!isfinite(bv)) atomicExch(q.status, 1);
      q.bcopy[g] = bv;
      const bool top = (int)(g % q.NZ) == q.NZ - 1;
      const double v = top ? io.pD[g] : 0.0;
      if (!isfinite(v)) atomicExch(q.status, 1);
      q.x[g] = v;
    } else {
      io.out[g] = q.x[g];
    }
  } else {
    const int nb = tab->nb[r];
    const size_t stride = (size_t)nb * VB_THREADS;
    const size_t i0 = (size_t)bx * VB_THREADS + threadIdx.x;
    double* s = q.s;
    if constexpr (WHICH == VB_CAST_FIRST) {
      for (size_t i = i0; i < n; i += stride) q.r32[i] = (float)q.r[i];
    } else if constexpr (WHICH == VB_RZ) {
      // RZ = <r, z>, ZRO = <r_old, z> (flexible CG; none at the first step), RZ -> RZOLD
      const bool first = tab->st.first[prob] != 0;
      Acc<double> c1, c2;
      for (size_t i = i0; i < n; i += stride) {
        const double zi = (double)q.z32[i];
        c1.fma(q.r[i], zi);
        if (!first) c2.fma(q.rold[i], zi);
      }
      const double a1 = block_sum(c1.value(), red);
      const double a2 = block_sum(c2.value(), red);
      if (!local_reduce_last(q.sc, bx, nb, a1, a2, s_flag)) return;
      double v1 = 0.0, v2 = 0.0;
      for (int k = threadIdx.x; k < nb; k += VB_THREADS) {
        v1 += ((volatile double*)q.sc.partials)[2 * k];
        v2 += ((volatile double*)q.sc.partials)[2 * k + 1];
      }
      v1 = block_sum(v1, red);
      v2 = block_sum(v2, red);
      if (threadIdx.x == 0) {
        s[GROUP_OUTER + SLOT_RZOLD] = s[GROUP_OUTER + SLOT_RZ];
        s[GROUP_OUTER + SLOT_RZ] = v1;
        s[GROUP_OUTER + SLOT_ZRO] = v2;
        *q.sc.redcnt = 0u;
      }
    } else if constexpr (WHICH == VB_P_UPDATE) {
      // p = z (first step) or z + beta p, beta = (RZ - ZRO) / RZOLD (flexible CG)
      const bool first = tab->st.first[prob] != 0;
      const double beta = first ? 0.0
                                : (s[GROUP_OUTER + SLOT_RZ] - s[GROUP_OUTER + SLOT_ZRO]) / s[GROUP_OUTER + SLOT_RZOLD];
      for (size_t i = i0; i < n; i += stride) q.p[i] = first ? (double)q.z32[i] : (double)q.z32[i] + beta * q.p[i];
    } else if constexpr (WHICH == VB_CG_UPDATE) {
      // alpha = RZ / PAP; r_old = r; x += alpha p; r -= alpha w; r32 = (float) r; RR = ||r||^2
      const double a = s[GROUP_OUTER + SLOT_RZ] / s[GROUP_OUTER + SLOT_PAP];
      Acc<double> ac;
      for (size_t i = i0; i < n; i += stride) {
        double ri = q.r[i];
        q.rold[i] = ri;
        q.x[i] += a * q.p[i];
        ri -= a * q.w[i];
        q.r[i] = ri;
        q.r32[i] = (float)ri;
        ac.fma(ri, ri);
      }
      const double a1 = block_sum(ac.value(), red);
      if (!local_reduce_last(q.sc, bx, nb, a1, 0.0, s_flag)) return;
      double v = 0.0;
      for (int k = threadIdx.x; k < nb; k += VB_THREADS) v += ((volatile double*)q.sc.partials)[2 * k];
      v = block_sum(v, red);
      if (threadIdx.x == 0) {
        s[GROUP_OUTER + SLOT_RR] = v;
        *q.sc.redcnt = 0u;
      }
    }
  }
}

template <int WHICH>
__global__ void __launch_bounds__(VB_THREADS) k_vec_batch(const VecBatch* tab) {
  __shared__ double red[34];
  __shared__ int s_flag;
  batch_items(tab->m[WHICH], [&](int r, int bx) {
    vec_item<WHICH>(tab, r, bx, red, &s_flag);
    __syncthreads();
  });
}

cudaError_t vec_batch_table(const VecProb* a, int n, BatchState st, const BatchIO* io, void** table,
                            int nctas[VB_COUNT], const int* prob) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  VecBatch* h = new (std::nothrow) VecBatch();
  if (!h) return cudaErrorMemoryAllocation;
  h->st = st;
  h->io = io;
  h->n = n;
  const int* act[VB_COUNT] = {nullptr, st.first, st.active, st.active, st.active, nullptr};
  for (int k = 0; k < VB_COUNT; ++k) {
    h->m[k].nrange = n;
    h->m[k].active = act[k];
    h->m[k].start[0] = 0;
  }
  for (int i = 0; i < n; ++i) {
    h->prm[i] = a[i];
    const size_t nodes = (a[i].n + VB_THREADS - 1) / VB_THREADS;
    h->nb[i] = (int)std::min<size_t>(std::max<size_t>((a[i].n + 4 * VB_THREADS - 1) / (4 * VB_THREADS), 1), 64);
    for (int k = 0; k < VB_COUNT; ++k) {
      h->m[k].prob[i] = prob ? prob[i] : i;
      const int c = (k == VB_INIT || k == VB_COPY_OUT) ? (int)nodes : h->nb[i];
      h->m[k].start[i + 1] = h->m[k].start[i] + c;
    }
  }
  for (int k = 0; k < VB_COUNT; ++k) nctas[k] = h->m[k].start[n];
  BatchMap* maps[VB_COUNT];
  for (int k = 0; k < VB_COUNT; ++k) maps[k] = &h->m[k];
  cudaError_t e = batch_upload(h, maps, VB_COUNT, table);
  delete h;
  return e;
}
template <int WHICH>
static cudaError_t launch_vec_batch(const VecBatch* t, int items, cudaStream_t st) {
  int grid = 0;
  cudaError_t e = batch_grid(k_vec_batch<WHICH>, VB_THREADS, 0, items, &grid);
  if (e != cudaSuccess) return e;
  k_vec_batch<WHICH><<<grid, VB_THREADS, 0, st>>>(t);
  return cudaGetLastError();
}
cudaError_t vec_batch_launch(int which, const void* table, const int nctas[VB_COUNT], cudaStream_t st) {
  const VecBatch* t = static_cast<const VecBatch*>(table);
  switch (which) {
    case VB_INIT: return launch_vec_batch<VB_INIT>(t, nctas[which], st);
    case VB_CAST_FIRST: return launch_vec_batch<VB_CAST_FIRST>(t, nctas[which], st);
    case VB_RZ: return launch_vec_batch<VB_RZ>(t, nctas[which], st);
    case VB_P_UPDATE: return launch_vec_batch<VB_P_UPDATE>(t, nctas[which], st);
    case VB_CG_UPDATE: return launch_vec_batch<VB_CG_UPDATE>(t, nctas[which], st);
    case VB_COPY_OUT: return launch_vec_batch<VB_COPY_OUT>(t, nctas[which], st);
    default: return cudaErrorInvalidValue;
  }
}

// ---- per-problem state machine of the batched flexible CG (one thread per problem)
__global__ void k_batch_state_init(const VecBatch* tab) {
  const int i = threadIdx.x;
  if (i >= tab->n) return;
  const VecProb& q = tab->prm[i];
  const BatchState& st = tab->st;
  double* s = q.s;
  const double bb = s[SLOT_BB];  // the lifted residual of x = (0, p_D): ||b~||^2
  s[SLOT_RR64] = bb;
  st.bb[i] = bb;
  st.rr64[i] = bb;
  int status = 0;
  if (q.status[1]) status = 1;                    // PMG_ERR_INVALID: bad geometry
  else if (q.status[0] || !isfinite(bb)) status = 5;  // PMG_ERR_NONFINITE
  q.status[0] = 0;
  st.status[i] = status;
  st.active[i] = (status == 0 && bb > 0.0) ? 1 : 0;
  st.first[i] = st.active[i];
  st.confirm[i] = 0;
  st.total[i] = 0;
}
__global__ void k_batch_cond(const VecBatch* tab) {
  const int i = threadIdx.x;
  if (i >= tab->n) return;
  const BatchState& st = tab->st;
  if (!st.active[i]) return;
  const VecProb& q = tab->prm[i];
  const double rr = q.s[GROUP_OUTER + SLOT_RR];
  const int total = ++st.total[i];
  st.first[i] = 0;
  if (!isfinite(rr)) {
    st.status[i] = 5;
    st.active[i] = 0;
  } else if (rr <= q.tol2 * st.bb[i] || total >= q.max_iter) {
    st.confirm[i] = 1;
  }
}
__global__ void k_batch_confirm(const VecBatch* tab, cudaGraphConditionalHandle hnd, int in_graph, int* any_out) {
  __shared__ int any;
  const int i = threadIdx.x;
  if (i == 0) any = 0;
  __syncthreads();
  const BatchState& st = tab->st;
  if (i < tab->n) {
    if (st.confirm[i]) {
      const VecProb& q = tab->prm[i];
      const double rr = q.s[SLOT_RR64];
      st.rr64[i] = rr;
      st.confirm[i] = 0;
      if (!isfinite(rr)) {
        st.status[i] = 5;
        st.active[i] = 0;
      } else if (rr <= q.tol2 * st.bb[i]) {
        st.active[i] = 0;  // converged
      } else if (st.total[i] >= q.max_iter) {
        st.status[i] = 4;  // PMG_ERR_NOT_CONVERGED
        st.active[i] = 0;
      } else {
        st.first[i] = 1;   // drift: restart the recurrence from the true residual
      }
    }
    if (st.active[i]) atomicOr(&any, 1);
  }
  __syncthreads();
  if (i == 0) {
    *any_out = any;
    if (in_graph) cudaGraphSetConditional(hnd, any ? 1u : 0u);
  }
}
cudaError_t batch_state_init(const void* table, int n, cudaStream_t st) {
  k_batch_state_init<<<1, ((n + 31) / 32) * 32, 0, st>>>(static_cast<const VecBatch*>(table));
  return cudaGetLastError();
}
cudaError_t batch_cond(const void* table, int n, cudaStream_t st) {
  k_batch_cond<<<1, ((n + 31) / 32) * 32, 0, st>>>(static_cast<const VecBatch*>(table));
  return cudaGetLastError();
}
cudaError_t batch_confirm(const void* table, int n, cudaGraphConditionalHandle hnd, int in_graph, int* any,
                          cudaStream_t st) {
  k_batch_confirm<<<1, ((n + 31) / 32) * 32, 0, st>>>(static_cast<const VecBatch*>(table), hnd, in_graph, any);
  return cudaGetLastError();
}

}  // namespace pmg
