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
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : (a.threads <= -32 && a.threads >= -256) ? a.threads
            : flat_tile_code_ok(a.threads) ? a.threads : 256;
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

// x_f += P x_c
template <typename T>
__device__ __forceinline__ void prolong_body(const TransferParams<T>& p, const int ex) {
  const Shape f = p.f, c = p.c;
  const int Pf = f.P, Pc = c.P, nf = Pf + 1, nc = Pc + 1;            // along x
  const int Pfz = f.pz(), Pcz = c.pz(), nfz = Pfz + 1, ncz = Pcz + 1;  // along sigma
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
    for (int l = 0; l < ncz; ++l) acc += Jzs[j * ncz + l] * Xc[k * NZcp + ez * Pcz + l];
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
template <typename T>
__global__ void __launch_bounds__(512) k_prolong(TransferParams<T> p) {
  prolong_body<T>(p, blockIdx.x);
}

// r_c = P^T r_f
template <typename T>
__device__ __forceinline__ void restrict_body(const TransferParams<T>& p, const int ex) {
  const Shape f = p.f, c = p.c;
  const int Pf = f.P, Pc = c.P, nf = Pf + 1, nc = Pc + 1;            // along x
  const int Pfz = f.pz(), Pcz = c.pz(), nfz = Pfz + 1, ncz = Pcz + 1;  // along sigma
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
      for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, li, m) * Xs[(e * Pf + m) * NZfp + iz];
      if (li == 0 && e == 1 && left)
        for (int m = 0; m < nf; ++m) kx += CT<T>::K(cT, Pf, Pf, m) * Xs[m * NZfp + iz];
      const int ez = min(iz / Pfz, f.Nz - 1), lj = iz - ez * Pfz;
      const T* col = Xs + q * NZfp;
      T kz = T(0);
      for (int m = 0; m < nfz; ++m) kz += CT<T>::K(cT, Pfz, lj, m) * col[ez * Pfz + m];
      if (lj == 0 && ez > 0)
        for (int m = 0; m < nfz; ++m) kz += CT<T>::K(cT, Pfz, Pfz, m) * col[(ez - 1) * Pfz + m];
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
        for (int j = 1; j < Pfz; ++j) acc += Jzs[j * ncz + 0] * col[ez * Pfz + j];
        if (ez > 0)
          for (int j = 1; j < Pfz; ++j) acc += Jzs[j * ncz + Pcz] * col[(ez - 1) * Pfz + j];
      } else {
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
__global__ void __launch_bounds__(512) k_restrict(TransferParams<T> p) {
  restrict_body<T>(p, blockIdx.x);
}

template <typename T>
static TransferParams<T> transfer_params(const TransferArgs& a) {
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
static size_t transfer_smem(const TransferArgs& a, int restrict_, size_t word) {
  int nf = a.f.P + 1, nc = a.c.P + 1, nfz = a.f.pz() + 1, ncz = a.c.pz() + 1;
  int NZfp = slab_pitch(a.f.NZ), NZcp = slab_pitch(a.c.NZ);
  if (restrict_) {
    size_t sm = ((size_t)(2 * a.f.P + 1) * (NZfp + NZcp) + nf * nc + nfz * ncz) * word + 16;
    if (a.xf) sm += ((size_t)(2 * a.f.P + 1) * (NZfp + 1) + a.f.NZ) * word;
    return sm;
  }
  return ((size_t)nc * (NZcp + NZfp) + nf * nc + nfz * ncz + (size_t)nf * NZfp) * word + 16;
}

template <typename T>
cudaError_t transfer(const TransferArgs& a, int restrict_, cudaStream_t st) {
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
  int nf = a.f.P + 1, nc = a.c.P + 1, nfz = a.f.pz() + 1, ncz = a.c.pz() + 1;
  int NZfp = slab_pitch(a.f.NZ), NZcp = slab_pitch(a.c.NZ);
  cudaError_t e;
  if (restrict_) {
    size_t sm = ((size_t)(2 * a.f.P + 1) * (NZfp + NZcp) + nf * nc + nfz * ncz) * sizeof(T) + 16;
    if (a.xf) sm += ((size_t)(2 * a.f.P + 1) * (NZfp + 1) + a.f.NZ) * sizeof(T);
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_restrict<T>, s_mask);
    if (e != cudaSuccess) return e;
    k_restrict<T><<<a.f.Nx, (a.threads >= 32 && a.threads <= 512) ? a.threads : 256, sm, st>>>(p);
  } else {
    size_t sm = ((size_t)nc * (NZcp + NZfp) + nf * nc + nfz * ncz + (size_t)nf * NZfp) * sizeof(T) + 16;
    static std::atomic<unsigned long long> s_mask{0};
    e = ensure_max_smem(k_prolong<T>, s_mask);
    if (e != cudaSuccess) return e;
    k_prolong<T><<<a.f.Nx, (a.threads >= 32 && a.threads <= 512) ? a.threads : 256, sm, st>>>(p);
  }
  return cudaGetLastError();
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
template <int RESTRICT>
__global__ void __launch_bounds__(512) k_transfer_batch(const XferBatch* tab) {
  batch_items(tab->m, [&](int r, int ex) {
    if (RESTRICT) restrict_body<float>(tab->prm[r], ex);
    else prolong_body<float>(tab->prm[r], ex);
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
