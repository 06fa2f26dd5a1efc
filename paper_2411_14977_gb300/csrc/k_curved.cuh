// Actual-geometry operator kernel template, shared by the CUDA-core build (k_apply.cu,
// TC = 0) and the BF16 tensor-core build (k_apply_tc.cu, TC = 1 or 3).  The including
// translation unit defines the constant tables cT first (PMG_DEFINE_CONST_TABLES).
//
// TC != 0 (FP32 vectors): the four sum-factorised contractions U_r = D U, U_s = U D^T,
// D^T W_r, W_s D run on the tensor cores as mma.sync m16n8k16 tiles with BF16 operands
// and FP32 accumulation: the (P+1) x (P+1) matrix D (or D^T) padded to 16 x 16 is the A
// operand, eight node rows (or element columns) of the slab form the 16 x 8 B operand.
// TC = 1 rounds both operands to BF16 once; TC = 3 splits each into hi + lo BF16 parts
// and adds the three products hi*hi + hi*lo + lo*hi, which keeps about 16 significant
// bits of every product instead of 8.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

namespace pmg {


// Dot-product accumulator of the operator's contractions: a plain multiply-add for FP32
// and FP64 data.  For double-float data a running FP32 sum whose rounding errors (TwoSum)
// and the products' errors (the FMA TwoProd error plus the hi*lo cross terms) are
// collected in a second FP32 word and folded in once at the end: about 12 FP32
// operations per term instead of 18 for a normalised double-float multiply-add.  The
// dropped lo*lo products and the FP32 error word leave the result within a few units of
// 2^-48 of the terms' magnitudes, the accuracy of the double-float operator.
template <typename T>
struct DotAcc {
  T v;
  __device__ __forceinline__ DotAcc() : v(T(0)) {}
  __device__ __forceinline__ explicit DotAcc(T init) : v(init) {}
  __device__ __forceinline__ void fma(T a, T b) { v += a * b; }
  __device__ __forceinline__ T get() const { return v; }
};
template <>
struct DotAcc<df64> {
  float s, c;
  __device__ __forceinline__ DotAcc() : s(0.f), c(0.f) {}
  __device__ __forceinline__ explicit DotAcc(df64 init) : s(init.hi), c(init.lo) {}
  __device__ __forceinline__ void fma(df64 a, df64 b) {
    const float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    const float t = s + p, bb = t - s;
    c += ((s - (t - bb)) + (p - bb)) + pe;
    s = t;
  }
  __device__ __forceinline__ df64 get() const {  // TwoSum of the two words
    const float t = s + c, bb = t - s;
    return df64(t, (s - (t - bb)) + (c - bb));
  }
};

template <typename T>
struct CurvedParams {
  using IO = typename IOT<T>::type;  // global-memory type (FP64 for double-float compute)
  Shape s;
  const IO* x;       // input (MODE_DIV: u)
  const IO* x2;      // MODE_DIV: w
  const IO* b;       // MODE_RESIDUAL: load vector
  IO* y;             // output
  const IO* geo;     // [Nx][P+1][NG]: the column factors (4 constant depth, 5 mixed-stage, 6 varying depth)
  const IO* sigma;   // [NZ]
  T scale;           // MODE_DIV: scale
  int mask_input;    // 1: surface-row input read as zero
  double* result;    // MODE_RESIDUAL: ||r||^2, MODE_DOT: <x, y>
  Scratch sc;
};

// ---- BF16 tensor-core helpers (mma.sync.m16n8k16, fragment layouts of the PTX ISA)
__device__ __forceinline__ unsigned bf16_pack(float first, float second) {
  __nv_bfloat162 v = __floats2bfloat162_rn(first, second);  // first -> low 16 bits
  return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ void mma_bf16_16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

enum class TcKind { D, DT };  // A operand: D[r][k] or its transpose D[k][r]

// out(r, c) = sum_k A(r, k) B(k, c) for r, k < P+1 and the tile columns c of `ntiles` tiles
// of 8; the warps of the CTA take the tiles round robin.  getb(k, c) returns B (zero
// beyond the valid columns), put(r, c, v) is called for r < P+1 (c may exceed the valid
// range: put checks).
template <int P, int TC, class GetB, class Put>
__device__ __forceinline__ void tc_contract(TcKind kind, int ntiles, GetB getb, Put put) {
  constexpr int n = P + 1;
  static_assert(n <= 16, "one 16 x 16 A tile");
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // A fragment registers: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
  unsigned ah[4], al[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int r = g + ((q & 1) ? 8 : 0), k = 2 * t + ((q & 2) ? 8 : 0);
    float v0 = 0.f, v1 = 0.f;
    if (r < n && k < n) v0 = kind == TcKind::D ? cT.Df[P][r][k] : cT.Df[P][k][r];
    if (r < n && k + 1 < n) v1 = kind == TcKind::D ? cT.Df[P][r][k + 1] : cT.Df[P][k + 1][r];
    float h0 = bf16_round(v0), h1 = bf16_round(v1);
    ah[q] = bf16_pack(h0, h1);
    al[q] = bf16_pack(v0 - h0, v1 - h1);
  }
  for (int tt = warp; tt < ntiles; tt += nwarps) {
    const int c0 = tt * 8;
    // B fragment registers: (k = 2t..2t+1, col g), (k = 2t+8.., col g)
    float bv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int k = 2 * t + (q & 1) + ((q & 2) ? 8 : 0);
      bv[q] = k < n ? getb(k, c0 + g) : 0.f;
    }
    float bh[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bh[q] = bf16_round(bv[q]);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16_16816(c, ah, bf16_pack(bh[0], bh[1]), bf16_pack(bh[2], bh[3]));
    if (TC == 3) {
      mma_bf16_16816(c, ah, bf16_pack(bv[0] - bh[0], bv[1] - bh[1]), bf16_pack(bv[2] - bh[2], bv[3] - bh[3]));
      mma_bf16_16816(c, al, bf16_pack(bh[0], bh[1]), bf16_pack(bh[2], bh[3]));
    }
    // C fragment: (g, c0 + 2t..2t+1), (g + 8, c0 + 2t..)
    if (g < n) {
      put(g, c0 + 2 * t, c[0]);
      put(g, c0 + 2 * t + 1, c[1]);
    }
    if (g + 8 < n) {
      put(g + 8, c0 + 2 * t, c[2]);
      put(g + 8, c0 + 2 * t + 1, c[3]);
    }
  }
}

// MIX: the mixed-stage operator a(v, p) = int_{Omega^k} grad^k v . grad^(k-1) p (Sec. 3) with
// five column factors per node column (k_geometry_mixed): A = w d_k dsig/dx,
// B1 = w d_x(k-1) d_k / d_(k-1), B2 = w d_x(k), C = w (dx/dsig) / d_(k-1), E = d_x(k) d_x(k-1):
//   W_r = w_j (A U_r - sigma B1 U_s),  W_s = w_j (-sigma B2 U_r + C (1 + sigma^2 E) U_s).
// BATHY: the same-stage operator over a varying still-water depth h(x) (Sec. 2.2) with six
// column factors (k_geometry_bathy) [A, B, C, d_x, H = w h_x, h_x]; with s = h_x - sigma d_x:
//   W_r = w_j (A U_r + (H - sigma B) U_s),  W_s = w_j ((H - sigma B) U_r + C (1 + s^2) U_s).
// PZ: polynomial order along sigma when it differs from the order P along x (Sec. 5.1);
// the x-contractions use P + 1 nodes, the sigma-contractions PZ + 1.
// Block sum of an accumulator: double-float ones on the FP32 pipe, the others in FP64.
template <typename T>
__device__ __forceinline__ double block_acc_sum(const Acc<T>& a, double* red) { return block_sum(a.value(), red); }
template <>
__device__ __forceinline__ double block_acc_sum<df64>(const Acc<df64>& a, double* red) { return block_sum_df(a.s, red); }

template <int P, typename T, int MODE, int TC, bool MIX = false, bool BATHY = false, int PZ = P>
__device__ __forceinline__ void curved_body(const CurvedParams<T>& p, const int ex, const int nblocks) {
  static_assert(TC == 0 || PZ == P, "tensor-core path: equal orders");
  static_assert(TC == 0 || (std::is_same<T, float>::value && MODE != MODE_DIV), "tensor-core path: FP32 operator");
  static_assert(!MIX || (TC == 0 && (MODE == MODE_APPLY || MODE == MODE_RESIDUAL)), "mixed-stage: apply/residual");
  static_assert(!BATHY || (TC == 0 && !MIX && MODE != MODE_DIV), "varying depth: CUDA-core same-stage operator");
  constexpr int NG = MIX ? 5 : (BATHY ? 6 : 4);  // column factors per node column
  constexpr int n = P + 1;    // element nodes along x
  constexpr int nz = PZ + 1;  // along sigma
  const Shape s = p.s;
  const int NZ = s.NZ, Nz = s.Nz, NZp = slab_pitch(NZ);
  const int L = Nz * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NB = MODE == MODE_RESIDUAL ? 1 : 0;  // slabs of b staged beside x
  T* X = reinterpret_cast<T*>(smem_raw);   // [n][NZp]   input slab (kept to the epilogue)
  T* Ur = X + n * NZp;                      // [n][NZp]   U_r per node row, later Y
  T* Ws = Ur + n * NZp;                     // [Nz][nz][n] (ez, j, i): U_s then W_s
  T* Wr = Ws + L * nz;                      // [Nz][nz][n] (ez, j, i): W_r
  T* G = Wr + L * nz;                       // [n][NG]
  T* SG = G + NG * n;                       // [NZ] sigma
  T* BB = SG + NZ;                          // [n][NZp] b of the slab (MODE_RESIDUAL only)
  T* RW = BB + NB * n * NZp;                // [NZ] per row: w_j, w_j sigma, w_j sigma^2
  T* RWS = RW + NZ;
  T* RWS2 = RWS + NZ;
  T* GX = RWS2 + NZ;                        // [n] per column: factor 2 x factor 3
  size_t red_off = (((size_t)((2 + NB) * n * NZp + 2 * L * nz + NG * n + 4 * NZ + n) * sizeof(T)) + 15) &
                   ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem_raw + red_off);  // 34 doubles
  int* s_flag = reinterpret_cast<int*>(red + 34);
  T* Y = Ur;  // U_r is dead once the metric (phase 3) has read it

  const int col0 = ex * P;
  // ---- load the slab, the column factors and sigma
  for_slab(n, NZ, [&](int i, int iz) {
    size_t g = (size_t)wrap_col(s, col0 + i) * NZ + iz;
    bool ok = !(MODE != MODE_DIV && p.mask_input && iz == NZ - 1);
    cp_async_elem(&X[i * NZp + iz], p.x + g, ok);
    if (MODE == MODE_DIV) cp_async_elem(&Ur[i * NZp + iz], p.x2 + g, true);
    if (MODE == MODE_RESIDUAL) cp_async_elem(&BB[i * NZp + iz], p.b + g, true);
  });
  cp_async_wait_all();
  for (int t = threadIdx.x; t < NG * n; t += blockDim.x) G[t] = from_io<T>(p.geo[(size_t)ex * NG * n + t]);
  for (int t = threadIdx.x; t < NZ; t += blockDim.x) {
    const T sg = from_io<T>(p.sigma[t]);
    SG[t] = sg;
    if constexpr (!MIX && !BATHY && MODE != MODE_DIV) {
      // the row factors of the metric (phase 3): w_j, w_j sigma, w_j sigma^2
      const int ez = min(t / PZ, Nz - 1);
      const T w = CT<T>::w(cT, PZ, t - ez * PZ);
      const T ws = w * sg;
      RW[t] = w;
      RWS[t] = ws;
      RWS2[t] = ws * sg;
    }
  }
  if constexpr (!MIX && !BATHY && MODE != MODE_DIV) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) GX[t] = from_io<T>(p.geo[((size_t)ex * n + t) * NG + 2]) *
                                                           from_io<T>(p.geo[((size_t)ex * n + t) * NG + 3]);
  }
  __syncthreads();

  if constexpr (MODE != MODE_DIV) {
    if constexpr (TC != 0) {
      tc_contract<P, TC>(TcKind::D, (NZ + 7) / 8,
          [&](int k, int c) { return c < NZ ? (float)X[k * NZp + c] : 0.f; },
          [&](int i, int c, float v) { if (c < NZ) Ur[i * NZp + c] = v; });
      tc_contract<P, TC>(TcKind::D, (L + 7) / 8,
          [&](int k, int q) {
            if (q >= L) return 0.f;
            int ez = q / n, i = q - ez * n;
            return (float)X[i * NZp + ez * P + k];
          },
          [&](int j, int q, float v) {
            if (q < L) { int ez = q / n, i = q - ez * n; Ws[(ez * n + j) * n + i] = v; }
          });
    } else {
    // ---- phase 1: U_r along x, one node row per thread
    for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
      T xv[n];
#pragma unroll
      for (int m = 0; m < n; ++m) xv[m] = X[m * NZp + iz];
#pragma unroll
      for (int i = 0; i < n; ++i) {
        DotAcc<T> acc;
#pragma unroll
        for (int m = 0; m < n; ++m) acc.fma(CT<T>::D(cT, P, i, m), xv[m]);
        Ur[i * NZp + iz] = acc.get();
      }
    }
    // ---- phase 2: U_s along sigma, one (column i, element ez) per thread
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      int i = t % n, ez = t / n;
      T xv[nz];
#pragma unroll
      for (int m = 0; m < nz; ++m) xv[m] = X[i * NZp + ez * PZ + m];
#pragma unroll
      for (int j = 0; j < nz; ++j) {
        DotAcc<T> acc;
#pragma unroll
        for (int m = 0; m < nz; ++m) acc.fma(CT<T>::D(cT, PZ, j, m), xv[m]);
        Ws[(ez * nz + j) * n + i] = acc.get();
      }
    }
    }  // CUDA-core contractions
    __syncthreads();
    // ---- phase 3: pointwise metric
    for (int t = threadIdx.x; t < L * nz; t += blockDim.x) {
      int i = t % n, r = t / n, j = r % nz, ez = r / nz;
      int iz = ez * PZ + j;
      T wj = CT<T>::w(cT, PZ, j);
      T sg = SG[iz];
      T ur = Ur[i * NZp + iz];
      T us = Ws[t];
      if constexpr (BATHY) {
        const T* g = G + i * 6;
        T grr = wj * g[0];
        T grs = wj * (g[4] - sg * g[1]);
        T sl = g[5] - sg * g[3];
        T gss = wj * g[2] * (T(1) + sl * sl);
        Wr[t] = grr * ur + grs * us;
        Ws[t] = grs * ur + gss * us;
      } else if constexpr (MIX) {
        T grr = wj * G[i * 5 + 0];
        T grs = -wj * sg * G[i * 5 + 1];
        T gsr = -wj * sg * G[i * 5 + 2];
        T gss = wj * G[i * 5 + 3] * (T(1) + sg * sg * G[i * 5 + 4]);
        Wr[t] = grr * ur + grs * us;
        Ws[t] = gsr * ur + gss * us;
      } else {
        // grr = w_j g0, grs = -w_j sigma g1, gss = w_j g2 (1 + sigma^2 g3) from the row and
        // column factors staged above
        const T rw = RW[iz];
        T grr = rw * G[i * 4 + 0];
        T grs = -(RWS[iz] * G[i * 4 + 1]);
        T gss = rw * G[i * 4 + 2] + RWS2[iz] * GX[i];
        Wr[t] = grr * ur + grs * us;
        Ws[t] = grs * ur + gss * us;
      }
    }
  } else {
    // ---- divergence load vector: W_r = w_i w_j (d dsig/2) u,
    // W_s = w_i w_j (dx/2)(w + (h_x - sigma d_x) u).  Column factors in this mode:
    // A = w_i d dsig/2, B = w_i d_x, C = w_i dx/2, H = w_i h_x (zero over a constant depth).
    for (int t = threadIdx.x; t < L * nz; t += blockDim.x) {
      int i = t % n, r = t / n, j = r % nz, ez = r / nz;
      int iz = ez * PZ + j;
      T wj = CT<T>::w(cT, PZ, j);
      T u = X[i * NZp + iz], w = Ur[i * NZp + iz];
      Wr[t] = p.scale * wj * G[i * 4 + 0] * u;
      Ws[t] = p.scale * wj * (G[i * 4 + 2] * w + (G[i * 4 + 3] - SG[iz] * G[i * 4 + 1]) * (G[i * 4 + 2] / CT<T>::w(cT, P, i)) * u);
    }
  }
  __syncthreads();
  if constexpr (TC != 0) {
    // ---- phase 4a: Y[i][iz] = sum_k D[k][i] (W_r of the element(s) owning row iz)[k]
    tc_contract<P, TC>(TcKind::DT, (NZ + 7) / 8,
        [&](int k, int c) {
          if (c >= NZ) return 0.f;
          int ez = min(c / P, Nz - 1), j = c - ez * P;
          float v = Wr[(ez * n + j) * n + k];
          if (j == 0 && ez > 0) v += Wr[((ez - 1) * n + P) * n + k];
          return v;
        },
        [&](int i, int c, float v) { if (c < NZ) Y[i * NZp + c] = v; });
    __syncthreads();
    // ---- phase 4b: T[ez][j][i] = sum_k D[k][j] W_s[ez][k][i] into the W_r buffer
    tc_contract<P, TC>(TcKind::DT, (L + 7) / 8,
        [&](int k, int q) {
          if (q >= L) return 0.f;
          int ez = q / n, i = q - ez * n;
          return (float)Ws[(ez * n + k) * n + i];
        },
        [&](int j, int q, float v) {
          if (q < L) { int ez = q / n, i = q - ez * n; Wr[(ez * n + j) * n + i] = v; }
        });
    __syncthreads();
    // ---- phase 4c: rows shared by two elements take both elements' sums
    for_slab(n, NZ, [&](int i, int iz) {
      int ez = min(iz / P, Nz - 1), j = iz - ez * P;
      float v = Wr[(ez * n + j) * n + i];
      if (j == 0 && ez > 0) v += Wr[((ez - 1) * n + P) * n + i];
      Y[i * NZp + iz] += v;
    });
    __syncthreads();
  } else {
  // ---- phase 4a: x-contraction Y[i][iz] = sum_k D[k][i] sum_{ez owning iz} W_r
  for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
    int ez = min(iz / PZ, Nz - 1), j = iz - ez * PZ;
    T wv[n];
#pragma unroll
    for (int k = 0; k < n; ++k) wv[k] = Wr[(ez * nz + j) * n + k];
    if (j == 0 && ez > 0) {
#pragma unroll
      for (int k = 0; k < n; ++k) wv[k] += Wr[((ez - 1) * nz + PZ) * n + k];
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
      DotAcc<T> acc;
#pragma unroll
      for (int k = 0; k < n; ++k) acc.fma(CT<T>::D(cT, P, k, i), wv[k]);
      Y[i * NZp + iz] = acc.get();
    }
  }
  __syncthreads();
  // ---- phase 4b: sigma-contraction of the rows [ez PZ, ez PZ + PZ) owned by (i, ez)
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    int i = t % n, ez = t / n;
    T wv[nz];
#pragma unroll
    for (int k = 0; k < nz; ++k) wv[k] = Ws[(ez * nz + k) * n + i];
    DotAcc<T> below;
    if (ez > 0) {
#pragma unroll
      for (int k = 0; k < nz; ++k) below.fma(CT<T>::D(cT, PZ, k, PZ), Ws[((ez - 1) * nz + k) * n + i]);
    }
#pragma unroll
    for (int j = 0; j < PZ; ++j) {
      DotAcc<T> acc = (j == 0) ? below : DotAcc<T>();
#pragma unroll
      for (int k = 0; k < nz; ++k) acc.fma(CT<T>::D(cT, PZ, k, j), wv[k]);
      Y[i * NZp + ez * PZ + j] += acc.get();
    }
    if (ez == Nz - 1) {  // surface row: used by MODE_DIV only (masked otherwise)
      DotAcc<T> acc;
#pragma unroll
      for (int k = 0; k < nz; ++k) acc.fma(CT<T>::D(cT, PZ, k, PZ), wv[k]);
      Y[i * NZp + NZ - 1] += acc.get();
    }
  }
  __syncthreads();

  }  // CUDA-core contractions
  // ---- epilogue
  auto finish = [&](int ix, int i, int iz, T val, Acc<T>& ac) {  // i: local column of ix
    size_t g = (size_t)ix * NZ + iz;
    bool top = iz == NZ - 1;
    if (MODE == MODE_APPLY) {
      p.y[g] = top ? p.x[g] : to_io(val);
    } else if (MODE == MODE_RESIDUAL) {
      T r = top ? T(0) : BB[i * NZp + iz] - val;
      p.y[g] = to_io(r);
      ac.fma(r, r);
    } else if (MODE == MODE_DOT) {
      T v = top ? T(0) : val;
      p.y[g] = to_io(v);
      ac.fma(X[i * NZp + iz], v);
    } else {
      p.y[g] = to_io(top ? T(0) : val);
    }
  };
  Acc<T> acc;
  for_slab(P - 1, NZ, [&](int c, int iz) { finish(col0 + 1 + c, c + 1, iz, Y[(c + 1) * NZp + iz], acc); });
  const int nedges = s.periodic ? s.Nx : s.Nx + 1;
  T* eb = reinterpret_cast<T*>(p.sc.edgebuf);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    int i = side == 0 ? 0 : P;
    int e = side == 0 ? ex : (s.periodic ? (ex + 1) % s.Nx : ex + 1);
    bool single = !s.periodic && (e == 0 || e == s.Nx);
    int ix = e * P;
    Acc<T> eacc;
    if (single) {
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) finish(ix, i, iz, Y[i * NZp + iz], eacc);
    } else {
      T* buf = eb + (size_t)e * NZ;
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) atomic_add_t(buf + iz, Y[i * NZp + iz]);
      if (!edge_arrive(p.sc.edgecnt + e, 2, s_flag)) continue;
      for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) finish(ix, i, iz, take_t(buf + iz), eacc);
    }
    if (MODE == MODE_RESIDUAL || MODE == MODE_DOT) {
      double v = block_acc_sum(eacc, red);
      if (threadIdx.x == 0) p.sc.edgepart[e] = v;
    }
  }
  if (MODE == MODE_RESIDUAL || MODE == MODE_DOT) {
    double v = block_acc_sum(acc, red);
    grid_reduce(p.sc, v, nedges, p.result, red, s_flag, ex, nblocks);
  }
}

template <int P, typename T, int MODE, int TC, bool MIX = false, bool BATHY = false, int PZ = P>
__global__ void __launch_bounds__(512) k_curved(CurvedParams<T> p) {
  curved_body<P, T, MODE, TC, MIX, BATHY, PZ>(p, blockIdx.x, gridDim.x);
}

// Batched: one CTA per element column of every problem in the table (same-stage operator,
// constant depth, CUDA cores, equal orders); one instantiation per order, shared by every
// range of a table.
template <typename T, int MODE>
struct CurvedBatch {
  BatchMap m;
  CurvedParams<T> prm[kMaxBatch];
};
template <typename T, int MODE, int P>
__global__ void __launch_bounds__(256) k_curved_batch(const CurvedBatch<T, MODE>* tab) {
  batch_items(tab->m, [&](int r, int ex) {
    const CurvedParams<T>& p = tab->prm[r];
    curved_body<P, T, MODE, 0>(p, ex, p.s.Nx);
    __syncthreads();
  });
}

template <typename T>
static size_t curved_smem(int P, int NZ, int Nz, bool stage_b, int ng = 4, int PZ = -1) {
  int n = P + 1, nz = (PZ < 0 ? P : PZ) + 1, NZp = slab_pitch(NZ), L = Nz * n;
  size_t e = (size_t)(stage_b ? 3 : 2) * n * NZp + (size_t)2 * L * nz + (size_t)ng * n + 4 * (size_t)NZ + n;
  return ((e * sizeof(T) + 15) & ~(size_t)15) + 34 * sizeof(double) + 16;
}

template <int P, typename T, int MODE, int TC, bool MIX = false, bool BATHY = false, int PZ = P>
static cudaError_t launch_curved_p(const CurvedParams<T>& prm, int threads, cudaStream_t st) {
  size_t sm = curved_smem<T>(P, prm.s.NZ, prm.s.Nz, MODE == MODE_RESIDUAL, MIX ? 5 : (BATHY ? 6 : 4), PZ);
  auto k = k_curved<P, T, MODE, TC, MIX, BATHY, PZ>;
  static std::atomic<unsigned long long> s_mask{0};
  cudaError_t e = ensure_max_smem(k, s_mask);
  if (e != cudaSuccess) return e;
  k<<<prm.s.Nx, threads, sm, st>>>(prm);
  return cudaGetLastError();
}

template <typename T, int MODE, int TC, bool MIX = false, bool BATHY = false>
static cudaError_t launch_curved(const CurvedParams<T>& prm, int threads, cudaStream_t st) {
  switch (prm.s.P) {
#define PMG_CASE(PP) case PP: return launch_curved_p<PP, T, MODE, TC, MIX, BATHY>(prm, threads, st);
    PMG_CASE(1) PMG_CASE(2) PMG_CASE(3) PMG_CASE(4) PMG_CASE(5)
    PMG_CASE(6) PMG_CASE(7) PMG_CASE(8) PMG_CASE(9) PMG_CASE(10)
#undef PMG_CASE
    default: return cudaErrorInvalidValue;
  }
}


}  // namespace pmg
