// Batched FP32 Schwarz sweep (Sec. 5.3): the slab sweep body of k_fdm32.cuh over the element
// columns of every problem of a batch table, one launch per stage.  Its own translation
// unit (and copy of the constant tables) keeps the build parallel.
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"

namespace pmg {

static __constant__ float cV32[fdm32_table_size()];
static __constant__ float cK32[MAXP + 1][MAXP + 1][MAXP + 1];  // 1D LGL stiffness per order

cudaError_t init_consts_fdm32b(const float* table, size_t n, const float* K, size_t nk) {
  if (n != (size_t)fdm32_table_size() || nk != (size_t)(MAXP + 1) * (MAXP + 1) * (MAXP + 1))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyToSymbol(cV32, table, n * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(cK32, K, nk * sizeof(float));
}

}  // namespace pmg

#include "k_fdm32.cuh"

namespace pmg {

// Batched: one CTA per element column of every problem in the table (split residual, in
// place), the order and overlap dispatched per CTA.
struct Fdm32Batch {
  BatchMap m;
  Fdm32Params prm[kMaxBatch];
  int overlap[kMaxBatch];
};
template <int P, int O>
__device__ __forceinline__ void fdm32_cta(const Fdm32Params& p, unsigned char* smem_raw, int ex) {
  switch (xclass32(p.s, ex)) {
    case 0: fdm32_body<P, O, 0, false>(p, smem_raw, ex); break;
    case 1: fdm32_body<P, O, 1, false>(p, smem_raw, ex); break;
    case 2: fdm32_body<P, O, 2, false>(p, smem_raw, ex); break;
    default: fdm32_body<P, O, 3, false>(p, smem_raw, ex); break;
  }
}
// one instantiation per (order, overlap): every range of a table shares them
template <int P, int O>
__global__ void __launch_bounds__(256) k_fdm32_batch(const Fdm32Batch* tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  batch_items(tab->m, [&](int r, int ex) {
    fdm32_cta<P, O>(tab->prm[r], smem_raw, ex);
    __syncthreads();
  });
}

// Batched sweep table: range r is problem prob[r]'s level a[r] (split residual, in place),
// one CTA per element column.  The table is written to device memory owned by the caller.
cudaError_t fdm32_batch_table(const FdmArgs* a, const int* prob, int n, const int* active, void** table, int* nctas,
                              size_t* smem) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  Fdm32Batch* h = new (std::nothrow) Fdm32Batch();
  if (!h) return cudaErrorMemoryAllocation;
  h->m.nrange = n;
  h->m.active = active;
  h->m.start[0] = 0;
  size_t sm = 0;
  for (int i = 0; i < n; ++i) {
    if (a[i].b || (a[i].xout && a[i].xout != a[i].x) || a[i].s.P < 2 || a[i].s.P > MAXP ||
        (a[i].overlap == 1 && a[i].s.P < 3) || a[i].s.P != a[0].s.P || a[i].overlap != a[0].overlap) {
      delete h;
      return cudaErrorInvalidValue;
    }
    h->prm[i] = fdm32_params(a[i]);
    h->overlap[i] = a[i].overlap;
    h->m.prob[i] = prob[i];
    h->m.start[i + 1] = h->m.start[i] + a[i].s.Nx;
    sm = std::max(sm, fdm32_smem(a[i].s.P, a[i].overlap, false, a[i].s));
  }
  *nctas = h->m.start[n];
  *smem = sm;
  BatchMap* maps[1] = {&h->m};
  cudaError_t e = batch_upload(h, maps, 1, table);
  delete h;
  return e;
}

template <int P, int O>
static cudaError_t launch_fdm32_batch(const void* table, int nctas, int threads, size_t smem, cudaStream_t st) {
  auto k = k_fdm32_batch<P, O>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  int grid = 0;
  e = batch_grid(k, threads, smem, nctas, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(static_cast<const Fdm32Batch*>(table));
  return cudaGetLastError();
}
cudaError_t fdm32_batch_launch(const void* table, int P, int O, int nctas, int threads, size_t smem, cudaStream_t st) {
  if (O == 1) {
    switch (P) {
#define PMG_CASE(PP) case PP: return launch_fdm32_batch<PP, 1>(table, nctas, threads, smem, st);
      PMG_CASE(3) PMG_CASE(4) PMG_CASE(5) PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  } else if (O == 0) {
    switch (P) {
#define PMG_CASE(PP) case PP: return launch_fdm32_batch<PP, 0>(table, nctas, threads, smem, st);
      PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5) PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace pmg
