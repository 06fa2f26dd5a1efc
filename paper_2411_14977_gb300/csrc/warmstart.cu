// C ABI of the learned warm start (network state, forward/backward orchestration, Adam).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pmg.h"
#include "pmg_kernels.h"

namespace pmg {
void set_last_error(const char* msg);
}
using namespace pmg;

struct pmg_ws {
  int X = 0, NZ = 0, Q = 1, C = 0, H = 0, K = 0, maxS = 0;
  NnScales sc{1.0, 1.0, 1.0, 1.0};
  double lam = 0.0;  // weight of the first-difference terms of the loss
  size_t n1 = 0, n2 = 0, n3 = 0, np = 0;  // parameter counts per layer (W + b)
  float *par = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *a1 = nullptr, *a2 = nullptr, *out = nullptr, *d1 = nullptr, *d2 = nullptr, *dout = nullptr;
  float* in1 = nullptr;  // one packed sample for predict
  double* loss = nullptr;
  int step = 0;
  int device = 0;
  std::vector<void*> allocs;
  ~pmg_ws() {
    for (void* a : allocs) cudaFree(a);
  }
  float* W1() { return par; }
  float* b1() { return par + (size_t)H * C * K; }
  float* W2() { return par + n1; }
  float* b2() { return par + n1 + (size_t)H * H * K; }
  float* W3() { return par + n1 + n2; }
  float* b3() { return par + n1 + n2 + (size_t)NZ * H; }
};

namespace {

pmg_status ws_fail(pmg_status s, const char* msg) {
  set_last_error(msg);
  return s;
}
#define WCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return ws_fail(PMG_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

pmg_status forward(pmg_ws* w, const float* in, int S, float* out, cudaStream_t st) {
  ConvDims d1{S, w->C, w->H, w->X, w->K}, d2{S, w->H, w->H, w->X, w->K}, d3{S, w->H, w->NZ, w->X, 1};
  WCK(nn_conv_forward(d1, in, w->W1(), w->b1(), w->a1, st));
  WCK(nn_tanh((size_t)S * w->H * w->X, w->a1, st));
  WCK(nn_conv_forward(d2, w->a1, w->W2(), w->b2(), w->a2, st));
  WCK(nn_tanh((size_t)S * w->H * w->X, w->a2, st));
  WCK(nn_conv_forward(d3, w->a2, w->W3(), w->b3(), out, st));
  return PMG_OK;
}

pmg_status backward(pmg_ws* w, const float* in, const float* tgt, int S, cudaStream_t st) {
  ConvDims d1{S, w->C, w->H, w->X, w->K}, d2{S, w->H, w->H, w->X, w->K}, d3{S, w->H, w->NZ, w->X, 1};
  size_t nh = (size_t)S * w->H * w->X;
  WCK(cudaMemsetAsync(w->loss, 0, sizeof(double), st));
  WCK(nn_loss(S, w->NZ, w->X, w->out, tgt, w->dout, w->lam, w->loss, st));
  float* g = w->grad;
  WCK(nn_conv_backward_weight(d3, w->a2, w->dout, g + w->n1 + w->n2, st));
  WCK(nn_bias_grad(d3, w->dout, g + w->n1 + w->n2 + (size_t)w->NZ * w->H, st));
  WCK(nn_conv_backward_input(d3, w->dout, w->W3(), w->d2, st));
  WCK(nn_tanh_back(nh, w->a2, w->d2, st));
  WCK(nn_conv_backward_weight(d2, w->a1, w->d2, g + w->n1, st));
  WCK(nn_bias_grad(d2, w->d2, g + w->n1 + (size_t)w->H * w->H * w->K, st));
  WCK(nn_conv_backward_input(d2, w->d2, w->W2(), w->d1, st));
  WCK(nn_tanh_back(nh, w->a1, w->d1, st));
  WCK(nn_conv_backward_weight(d1, in, w->d1, g, st));
  WCK(nn_bias_grad(d1, w->d1, g + (size_t)w->H * w->C * w->K, st));
  return PMG_OK;
}

}  // namespace

extern "C" {

pmg_status pmg_ws_create(int n_cols, int col_len, int period, int hidden, int taps, int max_batch, uint64_t seed,
                         double s_eta, double s_deta, double s_p, double s_dp, pmg_ws** out) {
  if (!out) return ws_fail(PMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_cols < 1 || col_len < 2 || period < 1 || hidden < 1 || taps < 1 || !(taps & 1) || max_batch < 1 || !(s_eta > 0) ||
      !(s_deta > 0) || !(s_p > 0) || !(s_dp > 0))
    return ws_fail(PMG_ERR_INVALID, "bad network shape (taps must be odd) or non-positive scale");
  auto* w = new (std::nothrow) pmg_ws();
  if (!w) return ws_fail(PMG_ERR_OOM, "host allocation failed");
  cudaGetDevice(&w->device);
  w->X = n_cols;
  w->NZ = col_len;
  w->Q = period;
  w->C = col_len + 3 + period;
  w->H = hidden;
  w->K = taps;
  w->maxS = max_batch;
  w->sc = NnScales{s_eta, s_deta, s_p, s_dp};
  w->n1 = (size_t)w->H * w->C * w->K + w->H;
  w->n2 = (size_t)w->H * w->H * w->K + w->H;
  w->n3 = (size_t)w->NZ * w->H + w->NZ;
  w->np = w->n1 + w->n2 + w->n3;
  size_t nh = (size_t)max_batch * w->H * w->X, no = (size_t)max_batch * w->NZ * w->X;
  auto alloc = [&](float** p, size_t n) {
    if (cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(float)) != cudaSuccess) return false;
    w->allocs.push_back(*p);
    return cudaMemset(*p, 0, n * sizeof(float)) == cudaSuccess;
  };
  bool ok = alloc(&w->par, w->np) && alloc(&w->grad, w->np) && alloc(&w->m, w->np) && alloc(&w->v, w->np) &&
            alloc(&w->a1, nh) && alloc(&w->a2, nh) && alloc(&w->d1, nh) && alloc(&w->d2, nh) &&
            alloc(&w->out, no) && alloc(&w->dout, no) && alloc(&w->in1, (size_t)w->C * w->X);
  if (ok) {
    if (cudaMalloc(&w->loss, sizeof(double)) != cudaSuccess) ok = false;
    else w->allocs.push_back(w->loss);
  }
  if (!ok) {
    delete w;
    return ws_fail(PMG_ERR_OOM, "device allocation failed");
  }
  // Glorot-uniform weights from SplitMix64, zero biases, zero last layer
  std::vector<float> h(w->np, 0.f);
  uint64_t s = seed;
  auto uni = [&](float a) { return a * (2.f * (float)((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.f); };
  float a1 = std::sqrt(6.f / (float)(w->C * w->K + w->H * w->K));
  for (size_t i = 0; i < (size_t)w->H * w->C * w->K; ++i) h[i] = uni(a1);
  float a2 = std::sqrt(6.f / (float)(2 * w->H * w->K));
  for (size_t i = 0; i < (size_t)w->H * w->H * w->K; ++i) h[w->n1 + i] = uni(a2);
  if (cudaMemcpy(w->par, h.data(), w->np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    delete w;
    return ws_fail(PMG_ERR_CUDA, "upload failed");
  }
  *out = w;
  return PMG_OK;
}

pmg_status pmg_ws_destroy(pmg_ws* w) {
  if (w) {
    cudaDeviceSynchronize();
    delete w;
  }
  return PMG_OK;
}

pmg_status pmg_ws_set_roughness(pmg_ws* w, double lam) {
  if (!w || !(lam >= 0.0) || !std::isfinite(lam)) return ws_fail(PMG_ERR_INVALID, "bad roughness weight");
  w->lam = lam;
  return PMG_OK;
}

pmg_status pmg_ws_num_params(const pmg_ws* w, int64_t* n) {
  if (!w || !n) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  *n = (int64_t)w->np;
  return PMG_OK;
}

pmg_status pmg_ws_get_params(pmg_ws* w, float* host) {
  if (!w || !host) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  WCK(cudaMemcpy(host, w->par, w->np * sizeof(float), cudaMemcpyDeviceToHost));
  return PMG_OK;
}

pmg_status pmg_ws_set_params(pmg_ws* w, const float* host) {
  if (!w || !host) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  WCK(cudaMemcpy(w->par, host, w->np * sizeof(float), cudaMemcpyHostToDevice));
  WCK(cudaMemset(w->m, 0, w->np * sizeof(float)));
  WCK(cudaMemset(w->v, 0, w->np * sizeof(float)));
  w->step = 0;
  return PMG_OK;
}

pmg_status pmg_ws_pack(pmg_ws* w, const double* eta, const double* eta_prev, const double* etax,
                       const double* pprev, float* in, void* stream) {
  if (!w || !eta || !eta_prev || !etax || !pprev || !in) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  WCK(nn_pack(w->X, w->NZ, w->Q, eta, eta_prev, etax, pprev, w->sc, in, (cudaStream_t)stream));
  return PMG_OK;
}

pmg_status pmg_ws_target(pmg_ws* w, const double* p, const double* pprev, float* tgt, void* stream) {
  if (!w || !p || !pprev || !tgt) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  WCK(nn_target(w->X, w->NZ, p, pprev, w->sc.dp, tgt, (cudaStream_t)stream));
  return PMG_OK;
}

pmg_status pmg_ws_forward(pmg_ws* w, const float* in, int S, float* out, void* stream) {
  if (!w || !in || !out || S < 1 || S > w->maxS) return ws_fail(PMG_ERR_INVALID, "bad forward arguments");
  return forward(w, in, S, out, (cudaStream_t)stream);
}

pmg_status pmg_ws_predict(pmg_ws* w, const double* eta, const double* eta_prev, const double* etax,
                          const double* pprev, double* x0, void* stream) {
  if (!w || !eta || !eta_prev || !etax || !pprev || !x0) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  WCK(nn_pack(w->X, w->NZ, w->Q, eta, eta_prev, etax, pprev, w->sc, w->in1, st));
  pmg_status s = forward(w, w->in1, 1, w->out, st);
  if (s != PMG_OK) return s;
  WCK(nn_unpack(w->X, w->NZ, pprev, w->out, w->sc.dp, x0, st));
  return PMG_OK;
}

pmg_status pmg_ws_gradients(pmg_ws* w, const float* in, const float* tgt, int S, float* grad, double* loss,
                            void* stream) {
  if (!w || !in || !tgt || !grad || S < 1 || S > w->maxS) return ws_fail(PMG_ERR_INVALID, "bad gradient arguments");
  cudaStream_t st = (cudaStream_t)stream;
  pmg_status s = forward(w, in, S, w->out, st);
  if (s == PMG_OK) s = backward(w, in, tgt, S, st);
  if (s != PMG_OK) return s;
  WCK(cudaMemcpyAsync(grad, w->grad, w->np * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (loss) {
    WCK(cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    WCK(cudaStreamSynchronize(st));
  }
  return PMG_OK;
}

pmg_status pmg_ws_train_step(pmg_ws* w, const float* in, const float* tgt, int S, float lr, double* loss,
                             void* stream) {
  if (!w || !in || !tgt || S < 1 || S > w->maxS || !(lr > 0)) return ws_fail(PMG_ERR_INVALID, "bad training arguments");
  cudaStream_t st = (cudaStream_t)stream;
  pmg_status s = forward(w, in, S, w->out, st);
  if (s == PMG_OK) s = backward(w, in, tgt, S, st);
  if (s != PMG_OK) return s;
  w->step += 1;
  WCK(nn_adam(w->np, w->par, w->grad, w->m, w->v, lr, 0.9f, 0.999f, 1e-8f, w->step, st));
  if (loss) {
    WCK(cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    WCK(cudaStreamSynchronize(st));
  }
  return PMG_OK;
}

pmg_status pmg_ws_save(pmg_ws* w, const char* path) {
  if (!w || !path) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  std::vector<float> h(w->np);
  WCK(cudaMemcpy(h.data(), w->par, w->np * sizeof(float), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return ws_fail(PMG_ERR_INVALID, "cannot open file");
  int hdr[7] = {0x504D4757, 3, w->X, w->NZ, w->Q, w->H, w->K};  // magic, version, shape
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  std::fclose(f);
  return ok ? PMG_OK : ws_fail(PMG_ERR_INVALID, "write failed");
}

pmg_status pmg_ws_load(pmg_ws* w, const char* path) {
  if (!w || !path) return ws_fail(PMG_ERR_INVALID, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return ws_fail(PMG_ERR_INVALID, "cannot open file");
  int hdr[7];
  std::vector<float> h(w->np);
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 0x504D4757 && hdr[1] == 3 && hdr[2] == w->X &&
            hdr[3] == w->NZ && hdr[4] == w->Q && hdr[5] == w->H && hdr[6] == w->K && std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) return ws_fail(PMG_ERR_INVALID, "file does not match this network");
  return pmg_ws_set_params(w, h.data());
}

}  // extern "C"
