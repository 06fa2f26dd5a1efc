// Actual-geometry operator for different polynomial orders along x and sigma (Sec. 5.1):
// the k_curved template of k_curved.cuh with a separate sigma order, instantiated for the
// finest levels of the paper's scaling study (P_z = 8, P_x = 2..10, Sec. 6.3): apply,
// residual and inner-product modes in FP64, double-float and FP32, and the divergence load.
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_apply_aniso)

#include "k_curved.cuh"

namespace pmg {

template <typename T>
cudaError_t curved_op_aniso(const CurvedArgs& a, cudaStream_t st) {
  using IO = typename IOT<T>::type;
  if (a.tc || a.mix || a.bathy) return cudaErrorInvalidValue;
  CurvedParams<T> p;
  p.s = a.s;
  p.x = (const IO*)a.x;
  p.x2 = (const IO*)a.x2;
  p.b = (const IO*)a.b;
  p.y = (IO*)a.y;
  p.geo = (const IO*)a.geo;
  p.sigma = (const IO*)a.sigma;
  p.scale = from_io<T>((IO)a.scale);
  p.mask_input = a.mask_input;
  p.result = a.result;
  p.sc = a.sc;
  const int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  switch (a.s.P * 100 + a.s.pz()) {
#define PMG_PAIR(A, B)                                                                               \
    case A * 100 + B:                                                                                \
      switch (a.mode) {                                                                              \
        case MODE_APPLY: return launch_curved_p<A, T, MODE_APPLY, 0, false, false, B>(p, thr, st);   \
        case MODE_RESIDUAL: return launch_curved_p<A, T, MODE_RESIDUAL, 0, false, false, B>(p, thr, st); \
        case MODE_DOT: return launch_curved_p<A, T, MODE_DOT, 0, false, false, B>(p, thr, st);       \
        case MODE_DIV:                                                                               \
          if constexpr (std::is_same<T, double>::value)                                              \
            return launch_curved_p<A, T, MODE_DIV, 0, false, false, B>(p, thr, st);                  \
          return cudaErrorInvalidValue;                                                              \
      }                                                                                              \
      return cudaErrorInvalidValue;
    PMG_ANISO_FINE(PMG_PAIR)
#undef PMG_PAIR
  }
  return cudaErrorInvalidValue;
}
template cudaError_t curved_op_aniso<double>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op_aniso<float>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op_aniso<df64>(const CurvedArgs&, cudaStream_t);

}  // namespace pmg
