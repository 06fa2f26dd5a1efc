// Level kernels for different polynomial orders along x and sigma (Sec. 5.1: the higher
// order is semi-coarsened until the two match).  The templates of k_levels.cuh with a
// separate sigma order (and Schwarz overlap) instantiated for the order pairs of the
// paper's scaling study (N_z = 2, P_z = 8, P_x = 2..10, Sec. 6.3) and the levels that its
// semi-coarsening visits.  The sweep is the generic one (tables in shared memory).
#include "pmg_common.cuh"
#include "pmg_kernels.h"

PMG_DEFINE_CONST_TABLES(init_consts_levels_aniso)

#include "k_levels.cuh"

namespace pmg {

bool aniso_pair_supported(int P, int PZ, bool fine) {
#define PMG_PAIR(A, B) \
  if (P == A && PZ == B) return true;
  PMG_ANISO_FINE(PMG_PAIR)
  if (!fine) {
    PMG_ANISO_COARSE(PMG_PAIR)
  }
#undef PMG_PAIR
  return false;
}

template <typename T>
cudaError_t flat_op_aniso(const FlatArgs& a, cudaStream_t st) {
  if (a.Kx) return cudaErrorInvalidValue;  // varying depth takes equal orders
  FlatParams<T> p;
  p.s = a.s;
  p.x = (const T*)a.x;
  p.b = (const T*)a.b;
  p.y = (T*)a.y;
  p.cx = (T)a.cx;
  p.cz = (T)a.cz;
  p.mX = (const T*)a.mX;
  p.mZ = (const T*)a.mZ;
  p.residual = a.residual;
  p.Kx = nullptr;
  int thr = (a.threads >= 32 && a.threads <= 512) ? a.threads : (a.threads <= -32 && a.threads >= -256) ? a.threads : 256;
  switch (a.s.P * 100 + a.s.pz()) {
#define PMG_PAIR(A, B) \
    case A * 100 + B: return launch_flat_p<A, T, false, B>(p, thr, st);
    PMG_ANISO_FINE(PMG_PAIR)
    PMG_ANISO_COARSE(PMG_PAIR)
#undef PMG_PAIR
  }
  return cudaErrorInvalidValue;
}
template cudaError_t flat_op_aniso<double>(const FlatArgs&, cudaStream_t);
template cudaError_t flat_op_aniso<float>(const FlatArgs&, cudaStream_t);

constexpr int ov(int p) { return p >= 3 ? 1 : 0; }  // overlap 1 where the order allows it

template <typename T>
cudaError_t fdm_smooth_aniso(const FdmArgs& a, cudaStream_t st) {
  FdmParams<T> p;
  p.s = a.s;
  p.r = (const T*)a.r;
  p.x = (T*)a.x;
  p.post = a.post;
  p.omega = (T)a.omega;
  p.Vx = (const T*)a.Vx;
  p.Vz = (const T*)a.Vz;
  p.invden = (const T*)a.invden;
  p.wx = (const T*)a.wx;
  p.wz = (const T*)a.wz;
  p.sc = a.sc;
  p.xpercol = a.xpercol;
  const int thr = (a.threads >= 32 && a.threads <= 256) ? a.threads : 256;
  const int ox = a.overlap, oz = a.overlap_z < 0 ? a.overlap : a.overlap_z;
  switch (a.s.P * 100 + a.s.pz()) {
#define PMG_PAIR(A, B)                                                                                 \
    case A * 100 + B:                                                                                  \
      if (ox == 0 && oz == 0) return launch_fdm_p<A, 0, T, B, 0>(p, thr, st);                          \
      if (ox == ov(A) && oz == ov(B)) return launch_fdm_p<A, ov(A), T, B, ov(B)>(p, thr, st);          \
      return cudaErrorInvalidValue;
    PMG_ANISO_FINE(PMG_PAIR)
    PMG_ANISO_COARSE(PMG_PAIR)
#undef PMG_PAIR
  }
  return cudaErrorInvalidValue;
}
template cudaError_t fdm_smooth_aniso<double>(const FdmArgs&, cudaStream_t);
template cudaError_t fdm_smooth_aniso<float>(const FdmArgs&, cudaStream_t);

}  // namespace pmg
