// Kernels of the learned warm start: a periodic 1D convolutional network over the node
// columns of the tank (channels = features of a column, positions = columns x), its
// backward pass and the Adam update.  FP32 storage and arithmetic.
//
// A periodic convolution with K taps (K odd, centred) is a matrix product:
//   forward        Y[o][n]    = b[o] + sum_{q=(c,k)} W[o][c][k] X[c][x + k - K/2]      n = (s, x)
//   input grad     dX[c][n]   = sum_{(o,k)} W[o][c][k] dY[o][x - k + K/2]
//   weight grad    dW[o][q]   = sum_n dY[o][n] X[c][x + k - K/2],  db[o] = sum_n dY[o][n]
// (s = sample, indices mod X).  One tiled GEMM kernel serves all three through operand
// fetch functors that gather the shifted columns on the fly.  Activations are stored
// [sample][channel][x].
#include <cuda_runtime.h>
#include <stdint.h>

#include "pmg_kernels.h"

namespace pmg {

__device__ __forceinline__ int wrapx(int x, int X) {
  x %= X;
  return x < 0 ? x + X : x;
}

// ---- operand fetchers: A(i, k) of an M x Kd matrix, B(k, j) of a Kd x N matrix
struct FwdA {  // W[o][q]
  const float* W;
  int Kd;
  __device__ float operator()(int i, int k) const { return W[(size_t)i * Kd + k]; }
};
struct FwdB {  // X[c][x + k - K/2] of sample s, q = c*K + k, n = s*X + x
  const float* Xin;
  ConvDims d;
  __device__ float operator()(int q, int n) const {
    int c = q / d.K, k = q - c * d.K, s = n / d.X, x = n - s * d.X;
    return Xin[((size_t)s * d.C + c) * d.X + wrapx(x + k - d.K / 2, d.X)];
  }
};
struct BinA {  // W[o][c][k] as A[c][(o,k)]
  const float* W;
  ConvDims d;
  __device__ float operator()(int c, int q) const {
    int o = q / d.K, k = q - o * d.K;
    return W[((size_t)o * d.C + c) * d.K + k];
  }
};
struct BinB {  // dY[o][x - k + K/2] of sample s, q = (o,k)
  const float* dY;
  ConvDims d;
  __device__ float operator()(int q, int n) const {
    int o = q / d.K, k = q - o * d.K, s = n / d.X, x = n - s * d.X;
    return dY[((size_t)s * d.O + o) * d.X + wrapx(x - k + d.K / 2, d.X)];
  }
};
struct BwA {  // dY[o][n]
  const float* dY;
  ConvDims d;
  __device__ float operator()(int o, int n) const {
    int s = n / d.X, x = n - s * d.X;
    return dY[((size_t)s * d.O + o) * d.X + x];
  }
};
struct BwB {  // X[c][x + k - K/2] as B[n][q]
  const float* Xin;
  ConvDims d;
  __device__ float operator()(int n, int q) const {
    int c = q / d.K, k = q - c * d.K, s = n / d.X, x = n - s * d.X;
    return Xin[((size_t)s * d.C + c) * d.X + wrapx(x + k - d.K / 2, d.X)];
  }
};

// ---- output writers
struct OutAct {  // Y[s][o][x] = acc + bias[o]
  float* Y;
  const float* bias;
  ConvDims d;
  __device__ void operator()(int o, int n, float v) const {
    int s = n / d.X, x = n - s * d.X;
    Y[((size_t)s * d.O + o) * d.X + x] = v + (bias ? bias[o] : 0.f);
  }
};
struct OutIn {  // dX[s][c][x] = acc
  float* dX;
  ConvDims d;
  __device__ void operator()(int c, int n, float v) const {
    int s = n / d.X, x = n - s * d.X;
    dX[((size_t)s * d.C + c) * d.X + x] = v;
  }
};
struct OutW {  // dW[o][q] = acc
  float* dW;
  int Kd;
  __device__ void operator()(int o, int q, float v) const { dW[(size_t)o * Kd + q] = v; }
};

// C (M x N) = A (M x Kd) B (Kd x N); 64 x 64 tiles, 16-deep k steps, 256 threads with a
// 4 x 4 register block each.
template <class FA, class FB, class FO>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int Kd, FA fa, FB fb, FO fo) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk = t / 64, ii = t % 64;
      int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < Kd) ? fa(i, k) : 0.f;
      int j = j0 + ii;
      Bs[kk][ii] = (j < N && k < Kd) ? fb(k, j) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < M && j < N) fo(i, j, acc[r][c]);
    }
}

template <class FA, class FB, class FO>
static cudaError_t gemm(int M, int N, int Kd, FA fa, FB fb, FO fo, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm<<<grid, 256, 0, st>>>(M, N, Kd, fa, fb, fo);
  return cudaGetLastError();
}

cudaError_t nn_conv_forward(const ConvDims& d, const float* X, const float* W, const float* b, float* Y,
                            cudaStream_t st) {
  return gemm(d.O, d.S * d.X, d.C * d.K, FwdA{W, d.C * d.K}, FwdB{X, d}, OutAct{Y, b, d}, st);
}
cudaError_t nn_conv_backward_input(const ConvDims& d, const float* dY, const float* W, float* dX, cudaStream_t st) {
  return gemm(d.C, d.S * d.X, d.O * d.K, BinA{W, d}, BinB{dY, d}, OutIn{dX, d}, st);
}
cudaError_t nn_conv_backward_weight(const ConvDims& d, const float* X, const float* dY, float* dW, cudaStream_t st) {
  return gemm(d.O, d.C * d.K, d.S * d.X, BwA{dY, d}, BwB{X, d}, OutW{dW, d.C * d.K}, st);
}

// db[o] = sum over samples and positions of dY[s][o][x]
__global__ void k_bias_grad(ConvDims d, const float* dY, float* db) {
  int o = blockIdx.x;
  float acc = 0.f;
  for (int t = threadIdx.x; t < d.S * d.X; t += blockDim.x) {
    int s = t / d.X, x = t - s * d.X;
    acc += dY[((size_t)s * d.O + o) * d.X + x];
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[o] = red[0];
}
cudaError_t nn_bias_grad(const ConvDims& d, const float* dY, float* db, cudaStream_t st) {
  k_bias_grad<<<d.O, 256, 0, st>>>(d, dY, db);
  return cudaGetLastError();
}

// y = tanh(x) in place; dx = dy * (1 - y^2)
__global__ void k_tanh(size_t n, float* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = tanhf(y[i]);
}
__global__ void k_tanh_back(size_t n, const float* y, float* dy) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dy[i] *= 1.f - y[i] * y[i];
}
static unsigned egrid(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b ? b : 1) : 4096);
}
cudaError_t nn_tanh(size_t n, float* y, cudaStream_t st) {
  k_tanh<<<egrid(n), 256, 0, st>>>(n, y);
  return cudaGetLastError();
}
cudaError_t nn_tanh_back(size_t n, const float* y, float* dy, cudaStream_t st) {
  k_tanh_back<<<egrid(n), 256, 0, st>>>(n, y, dy);
  return cudaGetLastError();
}

// Loss of S output samples e = y - t, laid out [s][iz][x] (NZ rows of X periodic columns),
// with the surface row iz = NZ-1 masked (the guess keeps p_prev there):
//   L = (1/n) sum_i [ e_i^2 + lam ( (e_{iz+1} - e_i)^2 + (e_{x+1} - e_i)^2 ) ],  n = S NZ X
// (z pairs within a column, x pairs periodic).  The difference terms weight rough errors
// more, which is what the solve that follows pays for.  dy_i = dL/dy_i.
__global__ void k_loss(int S, int NZ, int X, const float* y, const float* t, float* dy, double lam, double* loss) {
  const size_t n = (size_t)S * NZ * X;
  auto err = [&](int s, int iz, int x) -> double {
    if (iz == NZ - 1) return 0.0;
    size_t k = ((size_t)s * NZ + iz) * X + x;
    return (double)y[k] - (double)t[k];
  };
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int x = (int)(i % X);
    int iz = (int)((i / X) % NZ);
    int s = (int)(i / ((size_t)X * NZ));
    double e = err(s, iz, x);
    double xp = err(s, iz, x + 1 == X ? 0 : x + 1), xm = err(s, iz, x == 0 ? X - 1 : x - 1);
    double g = e + lam * ((e - xp) + (e - xm));
    double l = e * e + lam * (xp - e) * (xp - e);
    if (iz + 1 < NZ) {
      double zp = err(s, iz + 1, x);
      g += lam * (e - zp);
      l += lam * (zp - e) * (zp - e);
    }
    if (iz > 0) g += lam * (e - err(s, iz - 1, x));
    dy[i] = iz == NZ - 1 ? 0.f : (float)(2.0 * g / (double)n);
    acc += l;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)n);
}
cudaError_t nn_loss(int S, int NZ, int X, const float* y, const float* t, float* dy, double lam, double* loss,
                    cudaStream_t st) {
  k_loss<<<egrid((size_t)S * NZ * X), 256, 0, st>>>(S, NZ, X, y, t, dy, lam, loss);
  return cudaGetLastError();
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void k_adam(size_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}
cudaError_t nn_adam(size_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                    int t, cudaStream_t st) {
  float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<egrid(n), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

// Network input of one sample, layout [channel][x]: channels
//   0: eta / s_eta,  1: (eta - eta_prev) / s_deta,  2: eta_x,
//   3 .. 3+Q-1: one-hot of the column's position x mod Q inside its element (Q = order),
//   3+Q+iz: p_prev[iz] / s_p
// (p_prev z-fastest: x * NZ + iz).  eta_prev is the surface of the solve that produced
// p_prev, so channel 1 carries the change of geometry the correction has to follow; the
// position channels let the translation-invariant convolution tell element-boundary
// columns from interior ones.
__global__ void k_pack(int X, int NZ, int Q, const double* eta, const double* eta_prev, const double* etax,
                       const double* p, NnScales sc, float* in) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int C = NZ + 3 + Q;
  if (t >= C * X) return;
  int c = t / X, x = t - c * X;
  double v;
  if (c == 0) v = eta[x] / sc.eta;
  else if (c == 1) v = (eta[x] - eta_prev[x]) / sc.deta;
  else if (c == 2) v = etax[x];
  else if (c < 3 + Q) v = (x % Q == c - 3) ? 1.0 : 0.0;
  else v = p[(size_t)x * NZ + (c - 3 - Q)] / sc.p;
  in[t] = (float)v;
}
cudaError_t nn_pack(int X, int NZ, int Q, const double* eta, const double* eta_prev, const double* etax,
                    const double* p, NnScales sc, float* in, cudaStream_t st) {
  int tot = (NZ + 3 + Q) * X;
  k_pack<<<(tot + 255) / 256, 256, 0, st>>>(X, NZ, Q, eta, eta_prev, etax, p, sc, in);
  return cudaGetLastError();
}
// x0 = p_prev + s_dp * out[iz][x] (the surface row keeps p_prev, which equals p_D there)
__global__ void k_unpack(int X, int NZ, const double* p, const float* out, double s_dp, double* x0) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)X * NZ) return;
  int x = (int)(t / NZ), iz = (int)(t - (size_t)x * NZ);
  double d = iz == NZ - 1 ? 0.0 : s_dp * (double)out[(size_t)iz * X + x];
  x0[t] = p[t] + d;
}
cudaError_t nn_unpack(int X, int NZ, const double* p, const float* out, double s_dp, double* x0, cudaStream_t st) {
  size_t tot = (size_t)X * NZ;
  k_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, NZ, p, out, s_dp, x0);
  return cudaGetLastError();
}
// training target of one sample: (p - p_prev) / s_dp in the output layout [iz][x]
__global__ void k_target(int X, int NZ, const double* p, const double* pprev, double s_dp, float* tgt) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)X * NZ) return;
  int iz = (int)(t / X), x = (int)(t - (size_t)iz * X);
  size_t g = (size_t)x * NZ + iz;
  tgt[t] = (float)((p[g] - pprev[g]) / s_dp);
}
cudaError_t nn_target(int X, int NZ, const double* p, const double* pprev, double s_dp, float* tgt, cudaStream_t st) {
  size_t tot = (size_t)X * NZ;
  k_target<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, NZ, p, pprev, s_dp, tgt);
  return cudaGetLastError();
}

}  // namespace pmg
