// Coarsest-level solve (order 1, flat geometry), device bodies shared by the three
// coarse-solve kernels (k_coarse_vec.cu) and the fused coarse V-cycle (k_vtail.cu).
// A_1 = cx K_X (x) M_Z + cz M_X (x) K_Z splits, with the generalized eigenvectors V of
// (K_Z, M_Z) on the free rows, into one periodic or wall tridiagonal system per vertical
// mode k: forward transform rhat = V^T b, a parallel cyclic reduction per mode, backward
// transform x = V uhat.  FP64 arithmetic whatever the precision of b and x.
#pragma once

namespace pmg {

// rhat[k][ix] = sum_iz V[iz][k] b[ix][iz] for t = ix Nz + k
template <typename T>
__device__ __forceinline__ void coarse_fwd_body(int NX1, int NZ1, const T* b, const double* V, double* rhat, int t) {
  int Nz = NZ1 - 1;
  if (t >= NX1 * Nz) return;
  int ix = t / Nz, k = t % Nz;
  const T* col = b + (size_t)ix * NZ1;
  double acc = 0.0;
  for (int iz = 0; iz < Nz; ++iz) acc += V[iz * Nz + k] * (double)col[iz];
  rhat[(size_t)k * NX1 + ix] = acc;
}
// PCR: d'_i = d_i - k1_i d_{i-s} - k2_i d_{i+s} per step; x_i = d_i * inv_i.  The two
// ping-pong vectors live in shared memory, or (long tanks) in the global scratch gbuf.
__device__ __forceinline__ void coarse_pcr_body(int n, int nsteps, int periodic, const double* coef, const double* inv,
                                                double* rhat, double* gbuf, int k, double* sbuf) {
  double* d0 = gbuf ? gbuf + (size_t)k * 2 * n : sbuf;
  double* d1 = d0 + n;
  const double* ck = coef + (size_t)k * nsteps * n * 2;
  double* rk = rhat + (size_t)k * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) d0[i] = rk[i];
  __syncthreads();
  int st = 1;
  for (int step = 0; step < nsteps; ++step, st <<= 1) {
    const double* c = ck + (size_t)step * n * 2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int im = i - st, ip = i + st;
      double v = d0[i];
      if (periodic) {
        im = ((im % n) + n) % n;
        ip = ip % n;
        v -= c[2 * i] * d0[im] + c[2 * i + 1] * d0[ip];
      } else {
        if (im >= 0) v -= c[2 * i] * d0[im];
        if (ip < n) v -= c[2 * i + 1] * d0[ip];
      }
      d1[i] = v;
    }
    __syncthreads();
    double* tmp = d0; d0 = d1; d1 = tmp;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) rk[i] = d0[i] * inv[(size_t)k * n + i];
}
template <typename T>
__device__ __forceinline__ void coarse_bwd_body(int NX1, int NZ1, const double* V, const double* uhat, T* x,
                                                size_t t) {
  int Nz = NZ1 - 1;
  if (t >= (size_t)NX1 * NZ1) return;
  int ix = (int)(t / NZ1), iz = (int)(t % NZ1);
  double acc = 0.0;
  if (iz < Nz)
    for (int k = 0; k < Nz; ++k) acc += V[iz * Nz + k] * uhat[(size_t)k * NX1 + ix];
  x[t] = (T)acc;
}
}  // namespace pmg
