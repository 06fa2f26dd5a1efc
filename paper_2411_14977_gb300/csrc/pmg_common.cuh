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
#include <cstring>
#include <new>

namespace pmg {

constexpr int MAXP = 10;
constexpr int MAXO = 1;
constexpr int MAXNB = MAXP + 1 + 2 * MAXO;

// Double-float number: value = hi + lo with |lo| <= ulp(hi)/2, two FP32 words (a 48-bit
// significand, FP32 exponent range).  Arithmetic from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA product error (TwoProd): the products
// and sums of the operator run on the FP32 pipe, which the GB300 issues 58x faster than
// its FP64 pipe.  Addition is the one-correction ("sloppy") variant: its error is within
// a few units of 2^-48 of the larger addend, i.e. relative to the summands, which is
// the accuracy the operator needs (its output is compared with |A||x|).
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ __forceinline__ explicit df64(float h) : hi(h), lo(0.f) {}
  __host__ __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
};
__host__ __device__ __forceinline__ df64 df64_from_double(double v) {
#ifdef __CUDA_ARCH__
  // Integer split of the FP64 bits (no FP64-pipe work): hi = the value truncated to 24
  // significant bits, lo = the remaining 29 mantissa bits, exact as an integer and rounded
  // once to 24 bits by the integer-to-float conversion.  Zero, denormals and magnitudes
  // below 2^-126 map to 0; magnitudes above the FP32 range to +-inf.
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;
  if (fe <= 0) return df64(0.f, 0.f);
  if (fe >= 255) return df64(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | (unsigned)(m >> 29)));
  const unsigned low = (unsigned)(m & 0x1FFFFFFFull);  // 29 bits, weight 2^(e - 1075)
  const int le = e - 1075 + 127;                       // biased exponent of 2^(e - 1075)
  float lo = 0.f;
  if (low != 0u) {
    const float l = __uint2float_rn(low);
    // 2^(e-1075): one normal factor, or 2^(le+64-127) * 2^-64 when le <= 0 (fe > 0 keeps
    // le + 64 > 0)
    lo = le > 0 ? l * __int_as_float(le << 23) : l * __int_as_float((le + 64) << 23) * __int_as_float(63 << 23);
  }
  return df64(hi, sign ? -lo : lo);
#else
  float h = (float)v;
  return df64(h, (float)(v - (double)h));
#endif
}
#ifdef __CUDA_ARCH__
// Exact FP32 -> FP64 by integer manipulation of the bits (no FP64-pipe work): normal values
// rebias the exponent; zero keeps its sign; a denormal m 2^-149 is normalised (its leading
// bit at 31 - clz(m)); infinities and NaNs take the all-ones exponent.
__device__ __forceinline__ double df64_f2d(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long de = e - 127u + 1023u, dm = (unsigned long long)m << 29;
  if (e == 255u) de = 2047u;
  if (e == 0u) {
    const int lead = 31 - __clz((int)m);               // 0..22 (unused when m == 0)
    de = m ? (unsigned long long)(lead - 149 + 1023) : 0ull;
    dm = m ? ((unsigned long long)(m << (23 - lead)) & 0x7FFFFFull) << 29 : 0ull;
  }
  return __longlong_as_double((long long)(sign | (de << 52) | dm));
}
#endif
__host__ __device__ __forceinline__ double df64_to_double(df64 a) {
#ifdef __CUDA_ARCH__
  return df64_f2d(a.hi) + df64_f2d(a.lo);
#else
  return (double)a.hi + (double)a.lo;
#endif
}
__device__ __forceinline__ df64 df64_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  float s = a + b;
  return df64(s, b - (s - a));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);  // TwoSum error of the high parts
  e += a.lo + b.lo;
  return df64_fast_two_sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // TwoProd error of the high parts
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df64_fast_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }

// Global-memory type of a compute type: double-float kernels read and write FP64.
template <typename T> struct IOT { using type = T; };
template <> struct IOT<df64> { using type = double; };
template <typename T> __host__ __device__ __forceinline__ T from_io(typename IOT<T>::type v) { return v; }
template <> __host__ __device__ __forceinline__ df64 from_io<df64>(double v) { return df64_from_double(v); }
__host__ __device__ __forceinline__ float to_io(float v) { return v; }
__host__ __device__ __forceinline__ double to_io(double v) { return v; }
__host__ __device__ __forceinline__ double to_io(df64 v) { return df64_to_double(v); }

struct ConstTables {
  double D[MAXP + 1][MAXP + 1][MAXP + 1];  // D[P][i][m] = d h_m/dr at r_i
  double K[MAXP + 1][MAXP + 1][MAXP + 1];  // 1D stiffness D^T diag(w) D
  double w[MAXP + 1][MAXP + 1];            // LGL weights
  float Df[MAXP + 1][MAXP + 1][MAXP + 1];
  float Kf[MAXP + 1][MAXP + 1][MAXP + 1];
  float wf[MAXP + 1][MAXP + 1];
  df64 Dd[MAXP + 1][MAXP + 1][MAXP + 1];  // D and w as double-float pairs
  df64 wd[MAXP + 1][MAXP + 1];
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
template <> struct CT<df64> {
  static __device__ __forceinline__ df64 D(const ConstTables& c, int P, int i, int m) { return c.Dd[P][i][m]; }
  static __device__ __forceinline__ df64 w(const ConstTables& c, int P, int i) { return c.wd[P][i]; }
};

// Scratch shared by all kernels of a handle (kernels on one stream run one at a time).
struct Scratch {
  void* xbuf;          // [max edges][2*MAXO+1][NZ] 8-byte slots holding the empty marker
  void* edgebuf;       // [max edges][2*MAXO+1][NZ] doubles, zero between launches
  unsigned* edgecnt;   // [max edges], zero between launches
  double* partials;    // [max CTAs]
  double* edgepart;    // [max edges]
  unsigned* redcnt;    // [1], zero between launches
};

// Mesh shape of one level.
struct Shape {
  int NX, NZ, Nx, Nz, P, periodic;
  int PZ;  // order along sigma when it differs from P (0: equal orders)
  __host__ __device__ int pz() const { return PZ > 0 ? PZ : P; }
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

// Asynchronous global -> shared copy of one element (cp.async, Ampere and later): the
// copies of a whole slab are in flight together instead of one load latency per element.
// valid == false writes zero and reads nothing (src must still be a valid address).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc, bool valid) {
  unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  int nbytes = valid ? (int)sizeof(T) : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(gsrc), "n"(sizeof(T)),
               "r"(nbytes)
               : "memory");
}
// Double-float slab element from an FP64 vector: converted in registers (no async copy).
__device__ __forceinline__ void cp_async_elem(df64* smem_dst, const double* gsrc, bool valid) {
  *smem_dst = valid ? df64_from_double(*gsrc) : df64(0.f);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- bulk copies (TMA) into shared memory, completed on an mbarrier -----------------
// A 1D cp.async.bulk copies a contiguous run of global memory into shared memory without
// per-element instructions; both addresses must be 16-byte aligned and the size a multiple
// of 16 bytes.  The copies of a CTA signal one mbarrier (transaction count = bytes); the
// waits are bounded in SM clock cycles so that a wait that cannot complete (a wrong byte
// count) ends with an error flag instead of a hang.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of bar for at most `cycles` SM clock cycles (0: give up at once).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long cycles) {
  if (cycles <= 0) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > cycles) return false;
  return true;
}
constexpr long long kWaitCyclesDefault = 1ll << 31;  // about one second at 2 GHz

// Grid-wide barrier of a cooperative launch (every CTA resident), on the arrival word
// bar[0] and the abort word bar[1].  Thread 0 of each CTA adds to the arrival word with
// release semantics (the CTA barrier before it orders the block's writes): CTA 0 adds
// 2^31 - (G - 1), every other CTA 1, so the G additions of one barrier sum to 2^31 and the
// word's top bit flips exactly when the last CTA arrives (its low bits return to their
// value at the start, zero).  Each CTA then polls with acquire loads until the bit differs
// from the value its own addition returned, for at most `cycles` SM clock cycles; a poll
// that gives up raises *flag and the abort word, and every poll that sees the abort word
// gives up at once.  Returns false (in every thread of the CTA) when the barrier was not
// completed: the caller leaves the kernel, and the owner clears bar[] before the next
// launch.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, long long cycles, int* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(add) : "memory");
    int ok = 1;
    const long long t0 = clock64();
    while (((ld_acquire_gpu(bar) ^ old) & 0x80000000u) == 0) {
      if (((volatile unsigned*)bar)[1]) { ok = 0; break; }
      if (clock64() - t0 > cycles) {
        atomicExch(flag, 1);
        atomicExch(bar + 1, 1u);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Calls f(c, iz) for every (c, iz) in [0, ncols) x [0, NZ), spread over the block with
// consecutive threads on consecutive iz (coalesced on a z-fastest slab); the flattened
// index advances by blockDim.x per step without an integer division per element.
template <class F>
__device__ __forceinline__ void for_slab(int ncols, int NZ, F&& f) {
  const int step = blockDim.x;
  const int dc = step / NZ, dz = step - dc * NZ;
  int c = threadIdx.x / NZ, iz = threadIdx.x - c * NZ;
  while (c < ncols) {
    f(c, iz);
    c += dc;
    iz += dz;
    if (iz >= NZ) { iz -= NZ; ++c; }
  }
}

// Accumulator for inner products and norms.  FP64 data: plain FP64.  FP32 data: a
// double-float (hi, lo) sum with error-free products (fmaf) and Knuth's TwoSum, which is
// FP64-accurate but runs on the FP32 pipe (the GB300 FP64 rate is 1/58 of its FP32
// rate; converting every FP32 element to FP64 made these kernels FP64-bound).
template <typename T>
struct Acc {
  double s = 0.0;
  __device__ __forceinline__ void fma(T a, T b) { s += (double)a * (double)b; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = hi + x;
    float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
  }
  __device__ __forceinline__ void fma(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    add(p);
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct Acc<df64> {  // inner products of double-float data, accumulated in double-float
  df64 s{0.f, 0.f};
  __device__ __forceinline__ void fma(df64 a, df64 b) { s = s + a * b; }
  __device__ __forceinline__ double value() const { return df64_to_double(s); }
};

// Sum of a double-float over the block on the FP32 pipe (one conversion to FP64 at the end);
// every thread gets the result.  red: >= 33 doubles of shared memory.
__device__ __forceinline__ double block_sum_df(df64 v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df64 w(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = v + w;
  }
  df64* rd = reinterpret_cast<df64*>(red);  // 33 pairs fit in 33 doubles
  __syncthreads();
  if (lane == 0) rd[wid] = v;
  __syncthreads();
  if (wid == 0) {
    df64 t = lane < nw ? rd[lane] : df64(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df64 w(__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o));
      t = t + w;
    }
    if (lane == 0) red[32] = df64_to_double(t);
  }
  __syncthreads();
  return red[32];
}

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
// double-float partials travel through the FP64 edge buffer (two addends into zero)
__device__ __forceinline__ void atomic_add_t(df64* p, df64 v) { atomicAdd(reinterpret_cast<double*>(p), df64_to_double(v)); }
__device__ __forceinline__ df64 take_t(df64* p) { return df64_from_double(take_t(reinterpret_cast<double*>(p))); }

// Fence-free two-party exchange of one value.  A slot holds a signalling-NaN marker
// between launches (arithmetic never produces a signalling NaN).  Each of the two
// contributors swaps its partial in; the one that gets a non-marker value back is second:
// it returns true with the sum in `total` (a + b == b + a, so the result does not depend
// on which party came first) and re-arms the slot.  The partial travels inside the atomic,
// so no memory fence or barrier is needed.
// Slots are 8 bytes for both element types (an FP32 partial sits in the low half).
constexpr unsigned long long kEmpty64 = 0x7FF4D00DD00DD00Dull;
__device__ __forceinline__ bool swap_exchange(unsigned long long* slot, float v, float& total) {
  unsigned long long old = atomicExch(slot, (unsigned long long)__float_as_uint(v));
  if (old == kEmpty64) return false;
  total = v + __uint_as_float((unsigned)old);
  atomicExch(slot, kEmpty64);
  return true;
}
__device__ __forceinline__ bool swap_exchange(unsigned long long* slot, double v, double& total) {
  unsigned long long old = atomicExch(slot, (unsigned long long)__double_as_longlong(v));
  if (old == kEmpty64) return false;
  total = v + __longlong_as_double((long long)old);
  atomicExch(slot, kEmpty64);
  return true;
}

// Edge exchange: after every thread has added its values into the zeroed buffer, the
// block learns whether it arrived last among `contributors` (true in every thread of the
// last block).  Release/acquire by thread 0 around the ticket: the barrier orders the
// block's adds before thread 0's fence, and fences are cumulative.
__device__ __forceinline__ bool edge_arrive(unsigned* cnt, int contributors, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(cnt, 1u);
    bool last = (int)t == contributors - 1;
    if (last) {
      *cnt = 0u;  // reset for the next launch
      __threadfence();
    }
    *s_flag = last ? 1 : 0;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Two-edge variant: after the block's adds for the edges it shares (need[k] != 0), one
// fence and both tickets back to back; last[k] is set in every thread.  Halves the
// serial latency of exchanging both element-edge zones of a slab.
__device__ __forceinline__ void edge_arrive2(unsigned* cnt0, unsigned* cnt1, const bool need[2], bool last[2],
                                             int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t0 = need[0] ? atomicAdd(cnt0, 1u) : 0u;
    unsigned t1 = need[1] ? atomicAdd(cnt1, 1u) : 0u;
    int f = 0;
    if (need[0] && t0 == 1u) { *cnt0 = 0u; f |= 1; }
    if (need[1] && t1 == 1u) { *cnt1 = 0u; f |= 2; }
    if (f) __threadfence();
    *s_flag = f;
  }
  __syncthreads();
  last[0] = (*s_flag & 1) != 0;
  last[1] = (*s_flag & 2) != 0;
}

// Deterministic grid reduction: block b stores partials[b]; the last block sums
// partials[0..nblocks) then edgepart[0..nedges) in index order into *out.  bx / nblocks:
// the block's index and the block count (a batched launch passes the problem's own).
__device__ __forceinline__ void grid_reduce(const Scratch& sc, double block_value, int nedges,
                                            double* out, double* red, int* s_flag, int bx, int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    sc.partials[bx] = block_value;
    __threadfence();
    unsigned t = atomicAdd(sc.redcnt, 1u);
    *s_flag = (t == (unsigned)nblocks - 1u) ? 1 : 0;
    if (*s_flag) __threadfence();
  }
  __syncthreads();
  if (*s_flag == 0) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += ((volatile double*)sc.partials)[i];
  for (int i = threadIdx.x; i < nedges; i += blockDim.x) v += ((volatile double*)sc.edgepart)[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    *out = v;
    *sc.redcnt = 0u;
  }
}

// ---- batches: one launch over the work items of many independent problems -----------
// A batched launch's work items are split into consecutive ranges, one per problem of the
// batch (range r belongs to problem prob[r] and covers items [start[r], start[r+1])); the
// ranges of problems whose solve has finished (active[prob] == 0) are skipped.
constexpr int kMaxBatch = 256;
struct BatchMap {
  int nrange;
  int start[kMaxBatch + 1];
  int prob[kMaxBatch];
  const int* active;  // per problem of the batch (device)
  const int2* item;   // [start[nrange]]: (range, item) of every CTA of a one-CTA-per-item launch
};
// A range works unless its problem is flagged inactive (active == NULL: every range works).
__device__ __forceinline__ bool range_active(const BatchMap& m, int r) {
  return !m.active || m.active[m.prob[r]];
}
// The item of a CTA of a batched launch (one CTA per item): its (range, item) pair from the
// table's map, one load; the CTA works on it unless the range's problem has finished.
template <class F>
__device__ __forceinline__ void batch_items(const BatchMap& m, F&& f) {
  const int2 ri = m.item[blockIdx.x];
  if (range_active(m, ri.x)) f(ri.x, ri.y);
}

// Deterministic reduction over the `nblocks` CTAs (local index bx) that one problem of a
// batched launch gives a vector kernel: as grid_reduce, with the problem's own partials
// and ticket.
__device__ __forceinline__ bool local_reduce_last(const Scratch& sc, int bx, int nblocks, double v0, double v1,
                                                  int* s_flag) {
  if (threadIdx.x == 0) {
    sc.partials[2 * bx] = v0;
    sc.partials[2 * bx + 1] = v1;
    __threadfence();
    *s_flag = (atomicAdd(sc.redcnt, 1u) == (unsigned)nblocks - 1u) ? 1 : 0;
    if (*s_flag) __threadfence();
  }
  __syncthreads();
  return *s_flag != 0;
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
  // the opt-in bound (227 KB) covers static and dynamic shared memory together
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024 - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) mask.fetch_or(bit);
  return e;
}

// Uploads a batched-launch table and the (range, item) map of each of its nmaps maps in
// one device allocation (owned by the caller, freed with one cudaFree): the table, then the
// maps, each map's item pointer set to its place in the block.
template <class Tab>
inline cudaError_t batch_upload(Tab* h, BatchMap* const* maps, int nmaps, void** table) {
  size_t off = (sizeof(Tab) + 15) & ~(size_t)15, total = off;
  for (int k = 0; k < nmaps; ++k) total += sizeof(int2) * (size_t)(maps[k]->start[maps[k]->nrange] + 1);
  char* hb = new (std::nothrow) char[total];
  if (!hb) return cudaErrorMemoryAllocation;
  char* d = nullptr;
  cudaError_t e = cudaMalloc(&d, total);
  if (e != cudaSuccess) {
    delete[] hb;
    return e;
  }
  size_t pos = off;
  for (int k = 0; k < nmaps; ++k) {
    BatchMap& m = *maps[k];
    int2* hm = reinterpret_cast<int2*>(hb + pos);
    for (int r = 0; r < m.nrange; ++r)
      for (int i = m.start[r]; i < m.start[r + 1]; ++i) hm[i] = make_int2(r, i - m.start[r]);
    m.item = reinterpret_cast<const int2*>(d + pos);
    pos += sizeof(int2) * (size_t)(m.start[m.nrange] + 1);
  }
  std::memcpy(hb, h, sizeof(Tab));
  e = cudaMemcpy(d, hb, total, cudaMemcpyHostToDevice);
  delete[] hb;
  if (e != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  *table = d;
  return cudaSuccess;
}

// Grid of a batched launch: one CTA per work item (the hardware block scheduler hands the
// items to the SMs as they free up: a measured 1.2x faster on the uneven 64-problem batch
// than a persistent grid of the SMs' resident CTAs taking the items round robin).
template <typename K>
inline cudaError_t batch_grid(K, int, size_t, int items, int* grid) {
  *grid = items > 0 ? items : 1;
  return cudaSuccess;
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
