// FP32 fast-diagonalisation Schwarz sweep over one element column (Sec. 5.3): the CTA
// body shared by the one-launch-per-sweep kernel (k_fdm32.cu), the batched kernel
// (k_fdm32_batch.cu) and the fused coarse V-cycle (k_vtail.cu).  The including
// translation unit defines the constant tables cV32 (per-class eigenvectors,
// fdm32_offset layout) and cK32 (1D LGL stiffness) first.
#pragma once

namespace pmg {

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
__device__ __forceinline__ void fdm32_body(const Fdm32Params& p, unsigned char* smem_raw, const int ex) {
  constexpr int NB = P + 1 + 2 * O;
  constexpr int OFF = fdm32_offset(P, O);
  constexpr int VX = OFF + XC * NB * NB;  // x eigenvectors of this CTA's class
  constexpr int VZI = OFF + 4 * NB * NB;  // z eigenvectors of interior elements
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int col0 = ex * P;
  // T1 holds node rows -O .. NZ - 1 + O (row iz at iz + O); the rows beyond the mesh and
  // the surface row are zero, so the per-element windows need no bounds checks
  const int T1P = slab_pitch(NZ + 2 * O);
  float* R = reinterpret_cast<float*>(smem_raw);  // [NB][NZp]  input, later U
  float* T1 = R + NB * NZp;                        // [NB][T1P]
  float* T3 = T1 + NB * T1P;                       // [Nz][NB][NB] (ez, b, alpha)
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
    // one node row per thread over the NB subdomain columns of r and x (the surface row and
    // columns off the mesh read as zero); column offsets computed once per thread
    unsigned cb[NB];
    bool cv[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      cv[a] = col_valid(s, col0 - O + a);
      cb[a] = cv[a] ? (unsigned)wrap_col(s, col0 - O + a) * (unsigned)NZ : 0u;
    }
    for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
      const bool row = iz != NZ - 1;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        const bool ok = cv[a] && row;
        const size_t g = ok ? (size_t)(cb[a] + (unsigned)iz) : 0;
        cp_async_elem(&R[a * NZp + iz], p.r + g, ok);
        cp_async_elem(&XS[a * NZp + iz], p.x + g, ok && !p.xzero);
      }
    }
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
  if constexpr (O > 0) {
    for (int t = threadIdx.x; t < NB * 2 * O; t += blockDim.x) {
      const int al = t / (2 * O), k = t - al * (2 * O);
      T1[al * T1P + (k < O ? k : NZ + k)] = 0.f;  // rows -O..-1 and NZ..NZ-1+O
    }
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
      T1[al * T1P + iz + O] = acc;
    }
  }
  __syncthreads();
  // phase 2
  for (int t = threadIdx.x; t < NB * Nz; t += blockDim.x) {
    int ez = t / NB, al = t - ez * NB;
    int zc = (ez == 0 ? 1 : 0) | (ez == Nz - 1 ? 2 : 0);
    const float* idn = ID + (zc * NB + al) * NB;
    const float* t1 = T1 + al * T1P + ez * P;  // rows ez P - O .. ez P + P + O
    float tz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) tz[b] = t1[b];
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
  // interior columns (this CTA's subdomain alone covers them): one node row per thread
  for (int iz = threadIdx.x; iz < NZ - 1; iz += blockDim.x) {
#pragma unroll
    for (int a = 2 * O + 1; a < P; ++a) upd(a, iz, U[a * NZp + iz]);
  }
  // Edge zones of both sides (2 ZW node columns): one node row per thread, whose 2 ZW
  // partials (both edges) are swapped into their slots back to back (independent atomics
  // in flight together, one round trip to L2 per row) and then finalised where the partner
  // had already arrived.  The surface row is never updated and its slots are not used.
  {
    const int e_left = ex, e_right = s.periodic ? (ex + 1) % s.Nx : ex + 1;
    const bool sh_left = s.periodic || ex != 0, sh_right = s.periodic || ex + 1 != s.Nx;
    unsigned long long* const slot0 = xb + (size_t)e_left * ZW * NZ;   // [ZW][NZ] slots of the left edge
    unsigned long long* const slot1 = xb + (size_t)e_right * ZW * NZ;  // of the right edge
    for (int iz = threadIdx.x; iz < NZ - 1; iz += blockDim.x) {
      unsigned long long old[2][ZW];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const bool shared = side ? sh_right : sh_left;
        unsigned long long* const sl = side ? slot1 : slot0;
#pragma unroll
        for (int c = 0; c < ZW; ++c) {
          const int a = (side ? P : 0) + c;
          old[side][c] = kEmpty64;
          if (shared) old[side][c] = atomicExch(sl + (size_t)c * NZ + iz, (unsigned long long)__float_as_uint(U[a * NZp + iz]));
          else if (col_valid(s, col0 - O + a)) upd(a, iz, U[a * NZp + iz]);  // wall: the only contributor
        }
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        unsigned long long* const sl = side ? slot1 : slot0;
#pragma unroll
        for (int c = 0; c < ZW; ++c) {
          if (old[side][c] == kEmpty64) continue;  // first to arrive, or a wall edge
          atomicExch(sl + (size_t)c * NZ + iz, kEmpty64);  // second to arrive: the sum is complete
          const int a = (side ? P : 0) + c;
          upd(a, iz, U[a * NZp + iz] + __uint_as_float((unsigned)old[side][c]));
        }
      }
    }
  }
}

// host side: dynamic shared memory of one CTA, and the kernel parameters of a sweep
static inline size_t fdm32_smem(int P, int O, bool res, const Shape& s) {
  const int NB = P + 1 + 2 * O, XCOLS = res ? 3 * P + 1 : NB;
  const int NZp = slab_pitch(s.NZ), T1P = slab_pitch(s.NZ + 2 * O);
  size_t elems = (size_t)(NB + XCOLS) * NZp + (size_t)NB * T1P + (size_t)s.Nz * NB * NB + 8 * NB * NB + s.NZ + NB +
                 (res ? s.NZ + NB : 0);
  return ((elems * sizeof(float) + 15) & ~(size_t)15) + 16;
}

static inline Fdm32Params fdm32_params(const FdmArgs& a) {
  Fdm32Params p;
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
  p.b = (const float*)a.b;
  p.cx = (float)a.cx;
  p.cz = (float)a.cz;
  p.mX = (const float*)a.mX;
  p.mZ = (const float*)a.mZ;
  return p;
}

}  // namespace pmg
