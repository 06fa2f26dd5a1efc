// Fused coarse part of the FP32 V-cycle (Sec. 5): every level from a given one down to the
// order-1 coarse solve and back up, as ONE cooperative persistent launch.  On the coarse
// levels each step of the V-cycle is a small kernel (a few hundred thousand nodes or
// fewer) whose run time is dominated by its launch and its ramp; here the same steps --
// Schwarz sweeps, level residuals, restrictions, prolongations, the coarse solve's
// forward transform, cyclic reduction and backward transform -- run back to back inside
// one kernel, separated by grid-wide barriers with bounded waits.
//
// The step list is recorded from the launch-per-step V-cycle itself (same arguments, same
// order), so the fused kernel computes what that path computes with the same device
// bodies: one CTA body per element column for sweeps and transfers (CTAs stride over the
// columns), one thread per node for residuals and the coarse transforms, one CTA per
// vertical mode for the cyclic reduction.
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_vtail)

namespace pmg {

// the eigenvector table's leading part: the orders up to kVtMaxP (the layout puts the
// lower orders first, so the offsets are those of the full table)
static __constant__ float cV32[fdm32_offset(kVtMaxP + 1, 0)];
static __constant__ float cK32[MAXP + 1][MAXP + 1][MAXP + 1];

cudaError_t init_consts_vtail32(const float* table, size_t n, const float* K, size_t nk) {
  if (n != (size_t)fdm32_table_size() || nk != (size_t)(MAXP + 1) * (MAXP + 1) * (MAXP + 1))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyToSymbol(cV32, table, sizeof(cV32));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(cK32, K, nk * sizeof(float));
}

}  // namespace pmg

#include "k_coarse.cuh"
#include "k_fdm32.cuh"
#include "k_levels.cuh"

namespace pmg {

struct VtOpDev {
  int kind;  // VT_SWEEP, VT_RESID, VT_RESTRICT, VT_PROLONG, VT_CFWD, VT_CPCR, VT_CBWD
  int P, O;  // order and overlap of the level (sweeps, residuals)
  int idx;   // parameter slot of its kind
};
enum { VT_CFWD = 4, VT_CPCR = 5, VT_CBWD = 6 };

struct VtCoarseDev {
  int NX1, NZ1, nsteps, periodic;
  const float* b;
  float* x;
  const double* V;
  const double* coef;
  const double* inv;
  double* work;
  double* gbuf;  // PCR ping-pong in global memory (nullptr: shared memory)
};

struct VtailTab {
  int nops;
  VtOpDev op[kVtMaxOps];
  Fdm32Params sw[kVtMaxSteps];
  FlatParams<float> rs[kVtMaxSteps];
  TransferParams<float> tr[kVtMaxSteps];
  VtCoarseDev co;
  unsigned* bar;       // [2] grid barrier words: arrivals, abort
  int* timeout_flag;
};

template <int P, int O>
__device__ __forceinline__ void vt_sweep_po(const Fdm32Params& p, unsigned char* smem, int ex) {
  switch (xclass32(p.s, ex)) {
    case 0: fdm32_body<P, O, 0, false>(p, smem, ex); break;
    case 1: fdm32_body<P, O, 1, false>(p, smem, ex); break;
    case 2: fdm32_body<P, O, 2, false>(p, smem, ex); break;
    default: fdm32_body<P, O, 3, false>(p, smem, ex); break;
  }
}
__device__ __forceinline__ void vt_sweep(int P, int O, const Fdm32Params& p, unsigned char* smem, int ex) {
  if (O == 0) {
    switch (P) {
      case 2: vt_sweep_po<2, 0>(p, smem, ex); break;
      case 3: vt_sweep_po<3, 0>(p, smem, ex); break;
      default: vt_sweep_po<4, 0>(p, smem, ex); break;
    }
  } else {
    switch (P) {
      case 3: vt_sweep_po<3, 1>(p, smem, ex); break;
      default: vt_sweep_po<4, 1>(p, smem, ex); break;
    }
  }
}
__device__ __forceinline__ void vt_resid(int P, const FlatParams<float>& p, size_t g) {
  switch (P) {
    case 2: flat_np_body<2, float, false>(p, g); break;
    case 3: flat_np_body<3, float, false>(p, g); break;
    default: flat_np_body<4, float, false>(p, g); break;
  }
}

__global__ void __launch_bounds__(kVtMaxThreads) k_vtail(const VtailTab* __restrict__ t, long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nops = t->nops;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (int k = 0; k < nops; ++k) {
    const VtOpDev op = t->op[k];
    switch (op.kind) {
      case VT_SWEEP: {
        const Fdm32Params& p = t->sw[op.idx];
        for (int ex = blockIdx.x; ex < p.s.Nx; ex += gridDim.x) {
          vt_sweep(op.P, op.O, p, smem_raw, ex);
          __syncthreads();
        }
        break;
      }
      case VT_RESID: {
        const FlatParams<float>& p = t->rs[op.idx];
        const size_t N = (size_t)p.s.NX * p.s.NZ;
        for (size_t g = tid; g < N; g += stride) vt_resid(op.P, p, g);
        break;
      }
      case VT_RESTRICT:
      case VT_PROLONG: {
        const TransferParams<float>& p = t->tr[op.idx];
        for (int ex = blockIdx.x; ex < p.f.Nx; ex += gridDim.x) {
          if (op.kind == VT_RESTRICT) restrict_body<float>(p, ex);
          else prolong_body<float>(p, ex);
          __syncthreads();
        }
        break;
      }
      case VT_CFWD: {
        const VtCoarseDev& c = t->co;
        const size_t n = (size_t)c.NX1 * (c.NZ1 - 1);
        for (size_t i = tid; i < n; i += stride) coarse_fwd_body<float>(c.NX1, c.NZ1, c.b, c.V, c.work, (int)i);
        break;
      }
      case VT_CPCR: {
        const VtCoarseDev& c = t->co;
        double* sbuf = reinterpret_cast<double*>(smem_raw);
        for (int m = blockIdx.x; m < c.NZ1 - 1; m += gridDim.x) {
          coarse_pcr_body(c.NX1, c.nsteps, c.periodic, c.coef, c.inv, c.work, c.gbuf, m, sbuf);
          __syncthreads();
        }
        break;
      }
      default: {  // VT_CBWD
        const VtCoarseDev& c = t->co;
        const size_t n = (size_t)c.NX1 * c.NZ1;
        for (size_t i = tid; i < n; i += stride) coarse_bwd_body<float>(c.NX1, c.NZ1, c.V, c.work, c.x, i);
        break;
      }
    }
    if (k + 1 < nops && !grid_sync_bounded(t->bar, wait_cycles, t->timeout_flag)) return;
  }
}

static bool vt_sweep_ok(const FdmArgs& a) {
  return a.s.pz() == a.s.P && !a.b && (!a.xout || a.xout == a.x) && a.zc == 0 &&
         ((a.overlap == 0 && a.s.P >= 2 && a.s.P <= kVtMaxP) || (a.overlap == 1 && a.s.P >= 3 && a.s.P <= kVtMaxP));
}

cudaError_t vtail_table(const VtStep* steps, int n, const CoarseArgs& co, const void* cb, void* cx, unsigned* bar,
                        int* timeout_flag, void** table, size_t* smem) {
  VtailTab* h = new (std::nothrow) VtailTab();
  if (!h) return cudaErrorMemoryAllocation;
  auto bad = [&]() { delete h; return cudaErrorInvalidValue; };
  int nsw = 0, nrs = 0, ntr = 0, nops = 0;
  size_t sm = 0;
  bool coarse = false;
  for (int i = 0; i < n; ++i) {
    const VtStep& s = steps[i];
    if (s.kind == VT_COARSE) {
      if (nops + 3 > kVtMaxOps || coarse) return bad();
      coarse = true;
      h->op[nops++] = VtOpDev{VT_CFWD, 1, 0, 0};
      h->op[nops++] = VtOpDev{VT_CPCR, 1, 0, 0};
      h->op[nops++] = VtOpDev{VT_CBWD, 1, 0, 0};
      continue;
    }
    if (nops + 1 > kVtMaxOps) return bad();
    if (s.kind == VT_SWEEP) {
      if (nsw >= kVtMaxSteps || !vt_sweep_ok(s.fdm)) return bad();
      h->sw[nsw] = fdm32_params(s.fdm);
      h->op[nops++] = VtOpDev{VT_SWEEP, s.fdm.s.P, s.fdm.overlap, nsw++};
      sm = std::max(sm, fdm32_smem(s.fdm.s.P, s.fdm.overlap, false, s.fdm.s));
    } else if (s.kind == VT_RESID) {
      const FlatArgs& a = s.flat;
      if (nrs >= kVtMaxSteps || a.Kx || a.s.pz() != a.s.P || a.s.P < 2 || a.s.P > kVtMaxP || !a.residual) return bad();
      FlatParams<float> p;
      p.s = a.s;
      p.x = (const float*)a.x;
      p.b = (const float*)a.b;
      p.y = (float*)a.y;
      p.cx = (float)a.cx;
      p.cz = (float)a.cz;
      p.mX = (const float*)a.mX;
      p.mZ = (const float*)a.mZ;
      p.residual = 1;
      p.Kx = nullptr;
      h->rs[nrs] = p;
      h->op[nops++] = VtOpDev{VT_RESID, a.s.P, 0, nrs++};
    } else if (s.kind == VT_RESTRICT || s.kind == VT_PROLONG) {
      if (ntr >= kVtMaxSteps || s.xfer.f.pz() != s.xfer.f.P || s.xfer.c.pz() != s.xfer.c.P) return bad();
      const int r = s.kind == VT_RESTRICT;
      h->tr[ntr] = transfer_params<float>(s.xfer);
      h->op[nops++] = VtOpDev{s.kind, s.xfer.f.P, 0, ntr++};
      sm = std::max(sm, transfer_smem(s.xfer, r, sizeof(float)));
    } else {
      return bad();
    }
  }
  if (!coarse || nops < 1) return bad();
  VtCoarseDev& c = h->co;
  c.NX1 = co.NX1;
  c.NZ1 = co.NZ1;
  c.nsteps = co.nsteps;
  c.periodic = co.periodic;
  c.b = (const float*)cb;
  c.x = (float*)cx;
  c.V = co.V;
  c.coef = co.coef;
  c.inv = co.inv;
  c.work = co.work;
  const size_t pcr_sm = 2 * (size_t)co.NX1 * sizeof(double);
  c.gbuf = pcr_sm > kVtPcrSmem ? co.pcr_buf : nullptr;
  if (!c.gbuf) sm = std::max(sm, pcr_sm);
  h->nops = nops;
  h->bar = bar;
  h->timeout_flag = timeout_flag;
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(VtailTab));
  if (e == cudaSuccess) e = cudaMemcpy(d, h, sizeof(VtailTab), cudaMemcpyHostToDevice);
  delete h;
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return e;
  }
  *table = d;
  *smem = sm;
  return cudaSuccess;
}

// CTAs of k_vtail that fit on one SM at once (0: none); the cooperative grid is at most
// this times the SM count.
cudaError_t vtail_occupancy(int threads, size_t smem, int* per_sm) {
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k_vtail, s_mask);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_vtail, threads, smem);
}

cudaError_t vtail_launch(const void* table, int grid, int threads, size_t smem, long long wait_cycles, cudaStream_t st) {
  if (threads < 32 || threads > kVtMaxThreads || threads % 32 || grid < 1) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k_vtail, s_mask);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_vtail, static_cast<const VtailTab*>(table), wait_cycles);
}

}  // namespace pmg
