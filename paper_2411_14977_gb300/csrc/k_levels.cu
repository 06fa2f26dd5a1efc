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
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_levels)

#include "k_levels.cuh"
#include "k_levels_batch.h"

namespace pmg {

template <typename T>
cudaError_t flat_op(const FlatArgs& a, cudaStream_t st) {
  if (a.s.pz() != a.s.P) return flat_op_aniso<T>(a, st);
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
  p.wait_cycles = a.wait_cycles;
  p.timeout_flag = a.timeout_flag;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : (a.threads <= -32 && a.threads >= -256) ? a.threads
            : (flat_tile_code_ok(a.threads) || flat_bulk_code_ok(a.threads)) ? a.threads : 256;
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

template <typename T>
cudaError_t fdm_smooth(const FdmArgs& a, cudaStream_t st) {
  if (a.s.pz() != a.s.P) return fdm_smooth_aniso<T>(a, st);
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
template <typename T, int PF = 0, int PC = 0>
__global__ void __launch_bounds__(512) k_prolong(TransferParams<T> p) {
  prolong_body<T, PF, PC>(p, blockIdx.x);
}

template <typename T, int PF = 0, int PC = 0>
__global__ void __launch_bounds__(512) k_restrict(TransferParams<T> p) {
  restrict_body<T, PF, PC>(p, blockIdx.x);
}

template <typename T, int PF, int PC>
static cudaError_t launch_transfer(const TransferParams<T>& p, int restrict_, int nx, int thr, size_t sm,
                                   cudaStream_t st) {
  cudaError_t e;
  if (restrict_) {
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_restrict<T, PF, PC>, s_mask);
    if (e != cudaSuccess) return e;
    k_restrict<T, PF, PC><<<nx, thr, sm, st>>>(p);
  } else {
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_prolong<T, PF, PC>, s_mask);
    if (e != cudaSuccess) return e;
    k_prolong<T, PF, PC><<<nx, thr, sm, st>>>(p);
  }
  return cudaGetLastError();
}

// Level pairs of the coarsening rule (P_c = ceil((P_f + 1) / 2), and 2 -> 1) with equal
// orders along x and sigma run with compile-time orders; any other pair (custom level
// orders, semi-coarsened levels) with the orders read at run time.
template <typename T>
cudaError_t transfer(const TransferArgs& a, int restrict_, cudaStream_t st) {
  const TransferParams<T> p = transfer_params<T>(a);
  const size_t sm = transfer_smem(a, restrict_, sizeof(T));
  const int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  const int nx = a.f.Nx;
  if (a.f.pz() == a.f.P && a.c.pz() == a.c.P) {
    switch (a.f.P * 16 + a.c.P) {
#define PMG_PAIR(PF, PC) case PF * 16 + PC: return launch_transfer<T, PF, PC>(p, restrict_, nx, thr, sm, st);
      PMG_PAIR(2, 1) PMG_PAIR(3, 2) PMG_PAIR(4, 3) PMG_PAIR(5, 3) PMG_PAIR(6, 4)
      PMG_PAIR(7, 4) PMG_PAIR(8, 5) PMG_PAIR(9, 5) PMG_PAIR(10, 6)
#undef PMG_PAIR
      default: break;
    }
  }
  return launch_transfer<T, 0, 0>(p, restrict_, nx, thr, sm, st);
}
template cudaError_t transfer<double>(const TransferArgs&, int, cudaStream_t);
template cudaError_t transfer<float>(const TransferArgs&, int, cudaStream_t);

// ---- batched launches (FP32 V-cycle of a batch of independent problems) ---------------
struct FlatBatch {
  BatchMap m;
  FlatParams<float> prm[kMaxBatch];
};
template <int P>
__global__ void __launch_bounds__(256) k_flat_np_batch(const FlatBatch* tab) {
  batch_items(tab->m, [&](int r, int k) {
    flat_np_body<P, float, false>(tab->prm[r], (size_t)k * blockDim.x + threadIdx.x);
  });
}
struct XferBatch {
  BatchMap m;
  TransferParams<float> prm[kMaxBatch];
};
template <int RESTRICT, int PF = 0, int PC = 0>
__global__ void __launch_bounds__(512) k_transfer_batch(const XferBatch* tab) {
  batch_items(tab->m, [&](int r, int ex) {
    if (RESTRICT) restrict_body<float, PF, PC>(tab->prm[r], ex);
    else prolong_body<float, PF, PC>(tab->prm[r], ex);
    __syncthreads();
  });
}

template <class Tab>
static cudaError_t upload_table(Tab* h, void** table) {
  BatchMap* maps[1] = {&h->m};
  return batch_upload(h, maps, 1, table);
}

// Node-parallel FP32 level operator / residual of every problem: ceil(N / threads) CTAs each.
cudaError_t flat_batch_table(const FlatArgs* a, const int* prob, int n, const int* active, int threads, void** table,
                             int* nctas) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  FlatBatch* h = new (std::nothrow) FlatBatch();
  if (!h) return cudaErrorMemoryAllocation;
  h->m.nrange = n;
  h->m.active = active;
  h->m.start[0] = 0;
  for (int i = 0; i < n; ++i) {
    if (a[i].Kx || a[i].s.pz() != a[i].s.P || a[i].s.P != a[0].s.P) { delete h; return cudaErrorInvalidValue; }
    FlatParams<float>& p = h->prm[i];
    p.s = a[i].s;
    p.x = (const float*)a[i].x;
    p.b = (const float*)a[i].b;
    p.y = (float*)a[i].y;
    p.cx = (float)a[i].cx;
    p.cz = (float)a[i].cz;
    p.mX = (const float*)a[i].mX;
    p.mZ = (const float*)a[i].mZ;
    p.residual = a[i].residual;
    p.Kx = nullptr;
    h->m.prob[i] = prob[i];
    const size_t N = (size_t)a[i].s.NX * a[i].s.NZ;
    h->m.start[i + 1] = h->m.start[i] + (int)((N + threads - 1) / threads);
  }
  *nctas = h->m.start[n];
  cudaError_t e = upload_table(h, table);
  delete h;
  return e;
}
cudaError_t flat_batch_launch(const void* table, int P, int nctas, int threads, cudaStream_t st) {
  const FlatBatch* t = static_cast<const FlatBatch*>(table);
  int grid = 0;
  cudaError_t e = cudaSuccess;
  switch (P) {
#define PMG_CASE(PP)                                                         \
  case PP:                                                                   \
    e = batch_grid(k_flat_np_batch<PP>, threads, 0, nctas, &grid);      \
    if (e != cudaSuccess) return e;                                          \
    k_flat_np_batch<PP><<<grid, threads, 0, st>>>(t);                        \
    break;
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5) PMG_CASE(6) PMG_CASE(7) PMG_CASE(8)
    PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// FP32 restriction (restrict_ = 1) or prolongation of every problem: one CTA per element column.
cudaError_t transfer_batch_table(const TransferArgs* a, const int* prob, int n, const int* active, int restrict_,
                                 void** table, int* nctas, size_t* smem) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  XferBatch* h = new (std::nothrow) XferBatch();
  if (!h) return cudaErrorMemoryAllocation;
  h->m.nrange = n;
  h->m.active = active;
  h->m.start[0] = 0;
  size_t sm = 0;
  for (int i = 0; i < n; ++i) {
    if (a[i].xf) { delete h; return cudaErrorInvalidValue; }
    h->prm[i] = transfer_params<float>(a[i]);
    h->m.prob[i] = prob[i];
    h->m.start[i + 1] = h->m.start[i] + a[i].f.Nx;
    sm = std::max(sm, transfer_smem(a[i], restrict_, sizeof(float)));
  }
  *nctas = h->m.start[n];
  *smem = sm;
  cudaError_t e = upload_table(h, table);
  delete h;
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> s_mask_r{0}, s_mask_p{0};
  return restrict_ ? ensure_max_smem(k_transfer_batch<1>, s_mask_r) : ensure_max_smem(k_transfer_batch<0>, s_mask_p);
}
template <int PF, int PC>
static cudaError_t launch_transfer_batch(const XferBatch* t, int restrict_, int nctas, int threads, size_t smem,
                                         cudaStream_t st) {
  int grid = 0;
  cudaError_t e;
  if (restrict_) {
    auto k = k_transfer_batch<1, PF, PC>;
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k, s_mask);
    if (e == cudaSuccess) e = batch_grid(k, threads, smem, nctas, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, st>>>(t);
  } else {
    auto k = k_transfer_batch<0, PF, PC>;
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k, s_mask);
    if (e == cudaSuccess) e = batch_grid(k, threads, smem, nctas, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, st>>>(t);
  }
  return cudaGetLastError();
}
cudaError_t transfer_batch_launch_pair(const void* table, int restrict_, int Pf, int Pc, int nctas, int threads,
                                       size_t smem, cudaStream_t st) {
  const XferBatch* t = static_cast<const XferBatch*>(table);
  switch (Pf * 16 + Pc) {
#define PMG_PAIR(PF, PC) case PF * 16 + PC: return launch_transfer_batch<PF, PC>(t, restrict_, nctas, threads, smem, st);
    PMG_PAIR(2, 1) PMG_PAIR(3, 2) PMG_PAIR(4, 3) PMG_PAIR(5, 3) PMG_PAIR(6, 4)
    PMG_PAIR(7, 4) PMG_PAIR(8, 5) PMG_PAIR(9, 5) PMG_PAIR(10, 6)
#undef PMG_PAIR
    default: return launch_transfer_batch<0, 0>(t, restrict_, nctas, threads, smem, st);
  }
}
cudaError_t transfer_batch_launch(const void* table, int restrict_, int nctas, int threads, size_t smem,
                                  cudaStream_t st) {
  const XferBatch* t = static_cast<const XferBatch*>(table);
  int grid = 0;
  cudaError_t e = restrict_ ? batch_grid(k_transfer_batch<1>, threads, smem, nctas, &grid)
                            : batch_grid(k_transfer_batch<0>, threads, smem, nctas, &grid);
  if (e != cudaSuccess) return e;
  if (restrict_) k_transfer_batch<1><<<grid, threads, smem, st>>>(t);
  else k_transfer_batch<0><<<grid, threads, smem, st>>>(t);
  return cudaGetLastError();
}

}  // namespace pmg
