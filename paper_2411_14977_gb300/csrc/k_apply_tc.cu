// BF16 tensor-core build of the actual-geometry operator (FP32 vectors in and out): the
// k_curved template of k_curved.cuh with its four sum-factorised contractions on
// mma.sync m16n8k16 (BF16 operands, FP32 accumulation), plain (TC = 1) or hi/lo split
// (TC = 3).  Used by the PMG_MIXED_BF16 inner solve and pmg_apply_bf16.
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_apply_tc)

#include "k_curved.cuh"

namespace pmg {

cudaError_t curved_op_tc(const CurvedArgs& a, cudaStream_t st) {
  CurvedParams<float> p;
  p.s = a.s;
  p.x = (const float*)a.x;
  p.x2 = nullptr;
  p.b = (const float*)a.b;
  p.y = (float*)a.y;
  p.geo = (const float*)a.geo;
  p.sigma = (const float*)a.sigma;
  p.scale = (float)a.scale;
  p.mask_input = a.mask_input;
  p.result = a.result;
  p.sc = a.sc;
  int thr = (a.threads >= 32 && a.threads <= 512) ? (a.threads / 32) * 32 : 256;
  const bool split = a.tc == 3;
  if (a.tc != 1 && a.tc != 3) return cudaErrorInvalidValue;
  switch (a.mode) {
    case MODE_APPLY:
      return split ? launch_curved<float, MODE_APPLY, 3>(p, thr, st) : launch_curved<float, MODE_APPLY, 1>(p, thr, st);
    case MODE_DOT:
      return split ? launch_curved<float, MODE_DOT, 3>(p, thr, st) : launch_curved<float, MODE_DOT, 1>(p, thr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pmg
