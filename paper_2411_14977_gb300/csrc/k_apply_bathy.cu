// Actual-geometry operator over a varying still-water depth h(x) (Sec. 2.2: sigma = (z + h)/d,
// d = eta + h): the k_curved template of k_curved.cuh with BATHY set, whose metric carries
// the bottom-slope cross term h_x - sigma d_x (six column factors, k_geometry_bathy).  Its
// own translation unit so that the constant-depth builds compile in parallel with it.
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_apply_bathy)

#include "k_curved.cuh"

namespace pmg {

template <typename T>
cudaError_t curved_op_bathy(const CurvedArgs& a, cudaStream_t st) {
  using IO = typename IOT<T>::type;
  if (a.tc || a.mix || !a.geo6) return cudaErrorInvalidValue;
  CurvedParams<T> p;
  p.s = a.s;
  p.x = (const IO*)a.x;
  p.x2 = nullptr;
  p.b = (const IO*)a.b;
  p.y = (IO*)a.y;
  p.geo = (const IO*)a.geo6;
  p.sigma = (const IO*)a.sigma;
  p.scale = from_io<T>((IO)a.scale);
  p.mask_input = a.mask_input;
  p.result = a.result;
  p.sc = a.sc;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : 256;
  switch (a.mode) {
    case MODE_APPLY: return launch_curved<T, MODE_APPLY, 0, false, true>(p, thr, st);
    case MODE_RESIDUAL: return launch_curved<T, MODE_RESIDUAL, 0, false, true>(p, thr, st);
    case MODE_DOT: return launch_curved<T, MODE_DOT, 0, false, true>(p, thr, st);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t curved_op_bathy<double>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op_bathy<float>(const CurvedArgs&, cudaStream_t);
template cudaError_t curved_op_bathy<df64>(const CurvedArgs&, cudaStream_t);

}  // namespace pmg
