// Device-side common definitions: per-order constant tables, launch parameter blocks,
// block reductions, the slab-edge exchange and the deterministic grid reduction.
//
// Work decomposition shared by every mesh kernel: one CTA per element column ex (all
// cells_z elements of it), i.e. the contiguous slab of node columns [ex P, ex P + P] of a
// z-fastest vector.  A CTA owns the node columns [ex P, ex P + P) (the last CTA of a
// walled tank also owns the wall column).  Node columns shared by two CTAs (element
// edges, widened by the Schwarz overlap) are summed by the edge exchange: both CTAs add
// their partial into a zeroed buffer, the second one to arrive takes the sum and clears
// the buffer.  With exactly two addends into zero the result is independent of arrival
// order, so every kernel is bitwise deterministic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace pmg {

constexpr int MAXP = 10;
constexpr int MAXO = 1;
constexpr int MAXNB = MAXP + 1 + 2 * MAXO;

struct ConstTables {
  double D[MAXP + 1][MAXP + 1][MAXP + 1];  // D[P][i][m] = d h_m/dr at r_i
  double K[MAXP + 1][MAXP + 1][MAXP + 1];  // 1D stiffness D^T diag(w) D
  double w[MAXP + 1][MAXP + 1];            // LGL weights
  float Df[MAXP + 1][MAXP + 1][MAXP + 1];
  float Kf[MAXP + 1][MAXP + 1][MAXP + 1];
  float wf[MAXP + 1][MAXP + 1];
};

template <typename T> struct CT;
template <> struct CT<double> {
  static __device__ __forceinline__ double D(const ConstTables& c, int P, int i, int m) { return c.D[P][i][m]; }
  static __device__ __forceinline__ double K(const ConstTables& c, int P, int i, int m) { return c.K[P][i][m]; }
  static __device__ __forceinline__ double w(const ConstTables& c, int P, int i) { return c.w[P][i]; }
};
template <> struct CT<float> {
  static __device__ __forceinline__ float D(const ConstTables& c, int P, int i, int m) { return c.Df[P][i][m]; }
  static __device__ __forceinline__ float K(const ConstTables& c, int P, int i, int m) { return c.Kf[P][i][m]; }
  static __device__ __forceinline__ float w(const ConstTables& c, int P, int i) { return c.wf[P][i]; }
};

// Scratch shared by all kernels of a handle (kernels on one stream run one at a time).
struct Scratch {
  void* edgebuf;       // [max edges][2*MAXO+1][NZ] doubles, zero between launches
  unsigned* edgecnt;   // [max edges], zero between launches
  double* partials;    // [max CTAs]
  double* edgepart;    // [max edges]
  unsigned* redcnt;    // [1], zero between launches
};

// Mesh shape of one level.
struct Shape {
  int NX, NZ, Nx, Nz, P, periodic;
};

__device__ __forceinline__ int wrap_col(const Shape& s, int c) {
  if (s.periodic) { c %= s.NX; if (c < 0) c += s.NX; return c; }
  return c;
}
__device__ __forceinline__ bool col_valid(const Shape& s, int c) {
  return s.periodic || (c >= 0 && c < s.NX);
}
// Odd row pitch of a shared-memory slab (conflict-free column-parallel access).
__host__ __device__ __forceinline__ int slab_pitch(int NZ) { return NZ | 1; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the block; every thread gets the result.  red: >= 33 doubles of smem.
__device__ __forceinline__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ void atomic_add_t(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_t(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ double take_t(double* p) {
  return __longlong_as_double((long long)atomicExch((unsigned long long*)p, 0ull));
}
__device__ __forceinline__ float take_t(float* p) { return atomicExch(p, 0.0f); }

// Edge exchange, part 1: every thread adds its values (count n, index by callback) into
// buf, then the block learns whether it arrived last among `contributors`.
// Returns true in every thread of the last-arriving block.
__device__ __forceinline__ bool edge_arrive(unsigned* cnt, int contributors, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(cnt, 1u);
    bool last = (int)t == contributors - 1;
    if (last) *cnt = 0u;  // reset for the next launch
    *s_flag = last ? 1 : 0;
  }
  __syncthreads();
  bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Deterministic grid reduction: block b stores partials[b]; the last block sums
// partials[0..nblocks) then edgepart[0..nedges) in index order into *out.
__device__ __forceinline__ void grid_reduce(const Scratch& sc, double block_value, int nedges,
                                            double* out, double* red, int* s_flag) {
  if (threadIdx.x == 0) sc.partials[blockIdx.x] = block_value;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(sc.redcnt, 1u);
    *s_flag = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return;
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)sc.partials)[i];
  for (int i = threadIdx.x; i < nedges; i += blockDim.x) v += ((volatile double*)sc.edgepart)[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    *out = v;
    *sc.redcnt = 0u;
  }
}

// Raise a kernel's dynamic shared-memory limit to the SM maximum once per device
// (the attribute is per function and device); `mask` is the instantiation's own flag set.
template <typename K>
inline cudaError_t ensure_max_smem(K kernel, std::atomic<unsigned long long>& mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned long long bit = 1ull << (dev & 63);
  if (mask.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) mask.fetch_or(bit);
  return e;
}

}  // namespace pmg

// Each translation unit that uses the per-order tables defines its own copy and an
// initialiser (constant memory is per module and per device).
#define PMG_DEFINE_CONST_TABLES(NAME)                                               \
  namespace pmg {                                                                   \
  static __constant__ ConstTables cT;                                               \
  cudaError_t NAME(const ConstTables* host) {                                       \
    return cudaMemcpyToSymbol(cT, host, sizeof(ConstTables));                       \
  }                                                                                 \
  }
