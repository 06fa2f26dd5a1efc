// z-split FP32 Schwarz sweep (Sec. 5.3): the slab sweep of k_fdm32.cu with each element
// column split over CTAs of zc element rows, slabs staged by TMA bulk copies.  Its own
// translation unit (and copy of the constant tables) keeps the build parallel.
#include <algorithm>
#include <new>

#include "pmg_common.cuh"
#include "pmg_kernels.h"

namespace pmg {

static __constant__ float cV32[fdm32_table_size()];
static __constant__ float cK32[MAXP + 1][MAXP + 1][MAXP + 1];  // 1D LGL stiffness per order

cudaError_t init_consts_fdm32z(const float* table, size_t n, const float* K, size_t nk) {
  if (n != (size_t)fdm32_table_size() || nk != (size_t)(MAXP + 1) * (MAXP + 1) * (MAXP + 1))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyToSymbol(cV32, table, n * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(cK32, K, nk * sizeof(float));
}

}  // namespace pmg

#include "k_fdm32.cuh"

namespace pmg {

// ------------------------------------------------------------------------------------
// z-split sweep: one CTA per (element column, chunk of zc element rows).  The chunk's
// owned node rows are [ez0 P, ez1 P) (the surface row is never updated).  Their Schwarz
// corrections come from the subdomains of the chunk's elements and of the element just
// below and above it (whose blocks reach one or two owned rows), so the CTA transforms
// those halo elements too -- recomputation instead of an exchange along z; along x the
// slab-edge zones are exchanged as in k_fdm32.  The residual rows the transforms need and
// the iterate rows the update needs are staged by TMA (one 1D bulk copy per node column,
// 16-byte aligned: the copied run is widened to 16-byte boundaries, the column's shift
// recorded, a clipped tail fetched with plain loads), completed on one mbarrier whose
// wait is bounded: on a timeout the CTA raises the handle's timeout flag, waits for its
// copies, and leaves x unchanged.
// ------------------------------------------------------------------------------------
struct Fdm32zParams {
  Shape s;
  const float* r;
  float* x;     // iterate in
  float* xout;  // iterate out (may be x)
  int xzero;
  int post;
  float omega;
  const float* Vz;      // [4][NB][NB]
  const float* invden;  // [4][4][NB][NB]
  const float* wx;
  const float* wz;
  Scratch sc;
  int zc;                // element rows per CTA
  long long n;           // vector length NX NZ
  long long wait_cycles; // bound of the mbarrier wait (SM clock cycles)
  int* timeout_flag;     // set to 1 when a wait gives up
};

// Thread 0 of a z-split sweep CTA: stage the residual rows [rlo, rhi) and the iterate rows
// [olo, ohi) of the NB subdomain columns starting at global column c0.  Each column's run
// is widened to 16-byte boundaries [a0, a1) (clipped below the vector end; the clipped
// tail is fetched with plain loads) and copied by one TMA bulk copy to a 16-byte-aligned
// shared column; the column's shift (first row - a0) goes to RSH / XSH.  The byte total is
// announced on the mbarrier before the copies are issued.
template <int NB>
__device__ __noinline__ void fdm32z_issue(const Fdm32zParams& p, int c0, int rlo, int rhi, int olo, int ohi, float* R,
                                          float* XS, int RP, int XP, int* RSH, int* XSH, unsigned long long* bar) {
  const Shape& s = p.s;
  const long long nal = p.n & ~3ll;
  const bool with_x = !p.xzero && ohi > olo;
  unsigned total = 0;
  for (int a = 0; a < NB; ++a) {
    RSH[a] = 0;
    XSH[a] = 0;
    if (!col_valid(s, c0 + a)) continue;
    const long long base = (long long)wrap_col(s, c0 + a) * s.NZ;
    long long a0 = (base + rlo) & ~3ll, a1 = min((base + rhi + 3) & ~3ll, nal);
    RSH[a] = (int)(base + rlo - a0);
    if (a1 > a0) total += (unsigned)(a1 - a0) * 4u;
    if (with_x) {
      a0 = (base + olo) & ~3ll;
      a1 = min((base + ohi + 3) & ~3ll, nal);
      XSH[a] = (int)(base + olo - a0);
      if (a1 > a0) total += (unsigned)(a1 - a0) * 4u;
    }
  }
  mbar_arrive_expect_tx(bar, total);
  for (int a = 0; a < NB; ++a) {
    if (!col_valid(s, c0 + a)) continue;
    const long long base = (long long)wrap_col(s, c0 + a) * s.NZ;
    long long a0 = (base + rlo) & ~3ll, a1 = min((base + rhi + 3) & ~3ll, nal);
    if (a1 > a0) bulk_load_1d(R + a * RP, p.r + a0, (unsigned)(a1 - a0) * 4u, bar);
    for (long long g = max(a1, base + rlo); g < base + rhi; ++g) R[a * RP + (g - a0)] = p.r[g];
    if (with_x) {
      a0 = (base + olo) & ~3ll;
      a1 = min((base + ohi + 3) & ~3ll, nal);
      if (a1 > a0) bulk_load_1d(XS + a * XP, p.x + a0, (unsigned)(a1 - a0) * 4u, bar);
      for (long long g = max(a1, base + olo); g < base + ohi; ++g) XS[a * XP + (g - a0)] = p.x[g];
    }
  }
}

template <int P, int O, int XC>
__device__ __forceinline__ void fdm32z_body(const Fdm32zParams& p, unsigned char* smem_raw) {
  constexpr int NB = P + 1 + 2 * O;
  constexpr int ZW = 2 * O + 1;
  constexpr int OFF = fdm32_offset(P, O);
  constexpr int VX = OFF + XC * NB * NB;
  constexpr int VZI = OFF + 4 * NB * NB;
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz;
  const int ex = blockIdx.x, col0 = ex * P;
  const int ez0 = blockIdx.y * p.zc, ez1 = min(ez0 + p.zc, Nz);
  const int e_lo = max(ez0 - 1, 0), e_hi = min(ez1 + 1, Nz), ne = e_hi - e_lo;
  const int rfirst = e_lo * P - O;                       // node row of local row 0
  const int TR = ne * P + 2 * O + 1;                     // local rows of the transforms
  const int rlo = max(rfirst, 0), rhi = min(e_hi * P + O + 1, NZ - 1);  // residual rows read
  const int olo = ez0 * P, ohi = min(ez1 * P, NZ - 1), nown = ohi - olo;  // owned rows
  const Fdm32zLayout L = fdm32z_layout(P, O, p.zc);
  float* R = reinterpret_cast<float*>(smem_raw);  // [NB][RP] residual rows, later U [NB][UP]
  float* XS = R + NB * L.RP;                      // [NB][XP] iterate rows [olo, ohi)
  float* T1 = XS + NB * L.XP;                     // [NB][TP] local rows
  float* T3 = T1 + NB * L.TP;                     // [ne][NB][NB]
  float* VZ = T3 + L.T3n;                         // [4][NB][NB]
  float* ID = VZ + 4 * NB * NB;                   // [4][NB][NB]
  float* WZ = ID + 4 * NB * NB;                   // [TRmax] inverse cover counts of the local rows
  float* WX = WZ + L.TRmax;                       // [NB]
  int* RSH = reinterpret_cast<int*>(WX + NB);     // [NB] shift of each staged residual column
  int* XSH = RSH + NB;                            // [NB] shift of each staged iterate column
  int* s_ok = XSH + NB;                           // the copies arrived in time
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + L.bar_off);
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) fdm32z_issue<NB>(p, col0 - O, rlo, rhi, olo, ohi, R, XS, L.RP, L.XP, RSH, XSH, bar);
  // tables and weights while the copies fly; columns off the mesh read as zero
  for (int t = tid; t < 4 * NB * NB; t += nthr) {
    VZ[t] = p.Vz[t];
    ID[t] = p.invden[XC * 4 * NB * NB + t];
  }
  for (int t = tid; t < TR; t += nthr) {
    const int iz = rfirst + t;
    WZ[t] = (iz >= 0 && iz < NZ - 1) ? p.wz[iz] : 0.f;
  }
  if (tid < NB) {
    const int gc = col0 - O + tid;
    WX[tid] = col_valid(s, gc) ? p.wx[wrap_col(s, gc)] : 0.f;
  }
  for (int a = 0; a < NB; ++a) {
    if (col_valid(s, col0 - O + a)) continue;
    for (int t = tid; t < L.RP; t += nthr) R[a * L.RP + t] = 0.f;
  }
  // one thread waits (bounded) and the CTA follows its verdict, so that no thread skips a
  // barrier the others reach
  if (tid == 0) {
    const bool ok = mbar_wait_bounded(bar, 0, p.wait_cycles);
    if (!ok) {
      atomicExch(p.timeout_flag, 1);
      mbar_wait_bounded(bar, 0, kWaitCyclesDefault);  // the copies in flight land before exit
    }
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (*s_ok == 0) return;
  (void)mbar_try_wait(bar, 0);  // the phase is complete: each thread acquires the copied data
  // phase 1: T1 = Vx^T (W) R per local row (rows off [rlo, rhi) are zero)
  for (int lr = tid; lr < TR; lr += nthr) {
    const int iz = rfirst + lr;
    float rv[NB];
    const bool in = iz >= rlo && iz < rhi;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      float v = in ? R[a * L.RP + RSH[a] + (iz - rlo)] : 0.f;
      if (p.post) v *= WX[a] * WZ[lr];
      rv[a] = v;
    }
#pragma unroll
    for (int al = 0; al < NB; ++al) {
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < NB; ++a) acc = fmaf(cV32[VX + a * NB + al], rv[a], acc);
      T1[al * L.TP + lr] = acc;
    }
  }
  __syncthreads();
  // phase 2: T3 = Vz (D^-1 o (Vz^T T1_window)) per (element, x-mode)
  for (int t = tid; t < ne * NB; t += nthr) {
    const int ezl = t / NB, al = t - ezl * NB, ez = e_lo + ezl;
    const int zc = (ez == 0 ? 1 : 0) | (ez == Nz - 1 ? 2 : 0);
    const float* idn = ID + (zc * NB + al) * NB;
    const float* t1 = T1 + al * L.TP + ezl * P;
    float tz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) tz[b] = t1[b];
    float t2[NB];
    float* out = T3 + (ezl * NB) * NB + al;
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
  // phase 3: U = Vx (sum of the covering elements' T3) on the owned rows
  float* U = R;  // [NB][UP], owned row iz at iz - olo
  for (int lo = tid; lo < nown; lo += nthr) {
    const int iz = olo + lo;
    float sv[NB];
#pragma unroll
    for (int al = 0; al < NB; ++al) sv[al] = 0.f;
    const int e0 = (iz + O) / P;
#pragma unroll
    for (int d = -2; d <= 0; ++d) {
      const int ez = e0 + d;
      const int b = iz - ez * P + O;
      if (ez < e_lo || ez >= e_hi || b < 0 || b >= NB) continue;
      const float* src = T3 + ((ez - e_lo) * NB + b) * NB;
#pragma unroll
      for (int al = 0; al < NB; ++al) sv[al] += src[al];
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      float acc = 0.f;
#pragma unroll
      for (int al = 0; al < NB; ++al) acc = fmaf(cV32[VX + a * NB + al], sv[al], acc);
      U[a * L.UP + lo] = acc;
    }
  }
  __syncthreads();
  // phase 4: update the owned rows; the 2 ZW slab-edge columns by the two-party exchange
  const int e_left = ex, e_right = s.periodic ? (ex + 1) % s.Nx : ex + 1;
  const bool sh_left = s.periodic || ex != 0, sh_right = s.periodic || ex + 1 != s.Nx;
  unsigned long long* xb = reinterpret_cast<unsigned long long*>(p.sc.xbuf);
  for (int lo = tid; lo < nown; lo += nthr) {
    const int iz = olo + lo;
    const float wz = p.post ? 1.f : WZ[iz - rfirst];
    auto xold = [&](int a) { return p.xzero ? 0.f : XS[a * L.XP + XSH[a] + lo]; };
    auto store = [&](int a, float u) {
      const int c = wrap_col(s, col0 - O + a);
      const float w = p.post ? 1.f : WX[a] * wz;
      p.xout[(size_t)c * NZ + iz] = xold(a) + p.omega * w * u;
    };
#pragma unroll
    for (int a = 2 * O + 1; a < P; ++a) store(a, U[a * L.UP + lo]);
    unsigned long long old[2 * ZW];
    unsigned long long* slot[2 * ZW];
    float u[2 * ZW];
#pragma unroll
    for (int k = 0; k < 2 * ZW; ++k) {
      const int side = k / ZW, c = k - side * ZW, a = (side ? P : 0) + c;
      u[k] = U[a * L.UP + lo];
      old[k] = kEmpty64;
      slot[k] = nullptr;
      if (side ? sh_right : sh_left) {
        slot[k] = xb + ((size_t)(side ? e_right : e_left) * ZW + c) * NZ + iz;
        old[k] = atomicExch(slot[k], (unsigned long long)__float_as_uint(u[k]));
      } else if (col_valid(s, col0 - O + a)) {
        store(a, u[k]);  // wall: this CTA is the only contributor
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * ZW; ++k) {
      if (slot[k] && old[k] != kEmpty64) {  // second to arrive: the sum is complete
        atomicExch(slot[k], kEmpty64);
        const int side = k / ZW, c = k - side * ZW;
        store((side ? P : 0) + c, u[k] + __uint_as_float((unsigned)old[k]));
      }
    }
  }
}

template <int P, int O>
__global__ void __launch_bounds__(256) k_fdm32z(Fdm32zParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  switch (xclass32(p.s, blockIdx.x)) {
    case 0: fdm32z_body<P, O, 0>(p, smem_raw); break;
    case 1: fdm32z_body<P, O, 1>(p, smem_raw); break;
    case 2: fdm32z_body<P, O, 2>(p, smem_raw); break;
    default: fdm32z_body<P, O, 3>(p, smem_raw); break;
  }
}

template <int P, int O>
static cudaError_t launch_fdm32z(const Fdm32zParams& prm, int threads, cudaStream_t st) {
  const Fdm32zLayout L = fdm32z_layout(P, O, prm.zc);
  auto k = k_fdm32z<P, O>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)prm.s.Nx, (unsigned)((prm.s.Nz + prm.zc - 1) / prm.zc));
  k<<<grid, threads, L.bytes, st>>>(prm);
  return cudaGetLastError();
}

cudaError_t fdm_smooth32z(const FdmArgs& a, cudaStream_t st) {
  Fdm32zParams p;
  p.s = a.s;
  p.r = (const float*)a.r;
  p.x = (float*)a.x;
  p.xout = a.xout ? (float*)a.xout : (float*)a.x;
  p.xzero = a.xzero;
  p.post = a.post;
  p.omega = (float)a.omega;
  p.Vz = (const float*)a.Vz;
  p.invden = (const float*)a.invden;
  p.wx = (const float*)a.wx;
  p.wz = (const float*)a.wz;
  p.sc = a.sc;
  p.zc = a.zc;
  p.n = (long long)a.s.NX * a.s.NZ;
  p.wait_cycles = a.wait_cycles;
  p.timeout_flag = a.timeout_flag;
  const int thr = a.threads;
  if (a.overlap == 0) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm32z<PP, 0>(p, thr, st);
      PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  } else if (a.overlap == 1) {
    switch (a.s.P) {
#define PMG_CASE(PP) case PP: return launch_fdm32z<PP, 1>(p, thr, st);
      PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
      PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    }
  }
  return cudaErrorInvalidValue;
}

bool fdm32z_usable(const FdmArgs& a) {
  return a.zc >= 1 && !a.b && a.timeout_flag &&
         ((uintptr_t)a.r & 15u) == 0 && ((uintptr_t)a.x & 15u) == 0 && a.threads >= 32 && a.threads <= 256 &&
         a.threads % 32 == 0 && ((a.overlap == 0 && a.s.P >= 2) || (a.overlap == 1 && a.s.P >= 3)) &&
         a.s.P <= MAXP && fdm32z_layout(a.s.P, a.overlap, a.zc).bytes <= 227 * 1024;
}

}  // namespace pmg
