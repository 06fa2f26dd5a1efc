#include "host_basis.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace pmg {

void legendre_orthonormal(int n, double x, double* out, double* dout) {
  // a_k P~_k = x P~_{k-1} - a_{k-1} P~_{k-2},  a_k = sqrt(k^2 / ((2k+1)(2k-1)))   (Sec. 4.3)
  // differentiated: a_k P~'_k = P~_{k-1} + x P~'_{k-1} - a_{k-1} P~'_{k-2}
  auto a = [](int k) { return std::sqrt((double)k * k / ((2.0 * k + 1.0) * (2.0 * k - 1.0))); };
  out[0] = 1.0 / std::sqrt(2.0);
  dout[0] = 0.0;
  if (n >= 1) {
    out[1] = std::sqrt(1.5) * x;
    dout[1] = std::sqrt(1.5);
  }
  for (int k = 2; k <= n; ++k) {
    out[k] = (x * out[k - 1] - a(k - 1) * out[k - 2]) / a(k);
    dout[k] = (out[k - 1] + x * dout[k - 1] - a(k - 1) * dout[k - 2]) / a(k);
  }
}

// Standard Legendre L_p (L_p(1) = 1) and derivative by Bonnet's recurrence
// k L_k = (2k-1) x L_{k-1} - (k-1) L_{k-2};  L_k' = k L_{k-1} + x L_{k-1}'.
static void legendre_std(int p, double x, double& L, double& dL) {
  double l0 = 1.0, l1 = x, d0 = 0.0, d1 = 1.0;
  if (p == 0) { L = 1.0; dL = 0.0; return; }
  for (int k = 2; k <= p; ++k) {
    double l2 = ((2.0 * k - 1.0) * x * l1 - (k - 1.0) * l0) / k;
    double d2 = k * l1 + x * d1;
    l0 = l1; l1 = l2; d0 = d1; d1 = d2;
  }
  L = l1;
  dL = d1;
}

void lgl(int p, std::vector<double>& x, std::vector<double>& w) {
  // interior nodes: roots of L_p'.  Newton on f = L_p' with f' = L_p'' from Legendre's
  // equation (1 - x^2) L'' = 2x L' - p(p+1) L; Chebyshev-Lobatto starting points.
  if (p < 1) throw std::invalid_argument("order < 1");
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre_std(p, t, L, dL);
      double ddL = (2.0 * t * dL - p * (p + 1.0) * L) / (1.0 - t * t);
      double step = dL / ddL;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[i] = t;
  }
  std::sort(x.begin(), x.end());
  for (int i = 0; i <= p; ++i) {
    double L, dL;
    legendre_std(p, x[i], L, dL);
    w[i] = 2.0 / (p * (p + 1.0) * L * L);
  }
}

bool invert(int n, std::vector<double>& a) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (std::fabs(a[piv * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    double s = 1.0 / a[c * n + c];
    for (int k = 0; k < n; ++k) { a[c * n + k] *= s; inv[c * n + k] *= s; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[c * n + k]; inv[r * n + k] -= f * inv[c * n + k]; }
    }
  }
  a = inv;
  return true;
}

std::vector<double> diff_matrix(int p) {
  int n = p + 1;
  std::vector<double> x, w;
  lgl(p, x, w);
  std::vector<double> V(n * n), Vr(n * n), P(n), dP(n);
  for (int i = 0; i < n; ++i) {
    legendre_orthonormal(p, x[i], P.data(), dP.data());
    for (int k = 0; k < n; ++k) { V[i * n + k] = P[k]; Vr[i * n + k] = dP[k]; }
  }
  std::vector<double> Vi = V;
  if (!invert(n, Vi)) throw std::runtime_error("singular Vandermonde");
  std::vector<double> D(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Vr[i * n + k] * Vi[k * n + j];
      D[i * n + j] = s;
    }
  return D;
}

std::vector<double> transfer_matrix(int pc, int pf) {
  // I = Phi V_c^-1, Phi_ik = P~_k(x^f_i), k <= pc   (Sec. 5.2)
  int nc = pc + 1, nf = pf + 1;
  std::vector<double> xc, wc, xf, wf;
  lgl(pc, xc, wc);
  lgl(pf, xf, wf);
  std::vector<double> V(nc * nc), P(nc), dP(nc);
  for (int i = 0; i < nc; ++i) {
    legendre_orthonormal(pc, xc[i], P.data(), dP.data());
    for (int k = 0; k < nc; ++k) V[i * nc + k] = P[k];
  }
  if (!invert(nc, V)) throw std::runtime_error("singular Vandermonde");
  std::vector<double> J(nf * nc, 0.0);
  for (int i = 0; i < nf; ++i) {
    legendre_orthonormal(pc, xf[i], P.data(), dP.data());
    for (int j = 0; j < nc; ++j) {
      double s = 0.0;
      for (int k = 0; k < nc; ++k) s += P[k] * V[k * nc + j];
      J[i * nc + j] = s;
    }
  }
  return J;
}

std::vector<int> coarsening_sequence(int P) {
  std::vector<int> s{P};
  while (s.back() > 2) s.push_back((s.back() + 2) / 2);  // ceil((p+1)/2)
  if (s.back() != 1) s.push_back(1);
  return s;
}

std::vector<std::pair<int, int>> semi_coarsening_sequence(int P, int Pz) {
  std::vector<std::pair<int, int>> s{{P, Pz}};
  int px = P, pz = Pz;
  while (px != pz) {
    if (px > pz) px = std::max(pz, (px + 2) / 2);
    else pz = std::max(px, (pz + 2) / 2);
    s.push_back({px, pz});
  }
  std::vector<int> iso = coarsening_sequence(px);
  for (size_t i = 1; i < iso.size(); ++i) s.push_back({iso[i], iso[i]});
  return s;
}

void sym_eig(int n, std::vector<double> a, std::vector<double>& Q, std::vector<double>& lam) {
  Q.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = a[p * n + p], aqq = a[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // Q <- Q J
          double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  lam.assign(n, 0.0);
  for (int i = 0; i < n; ++i) lam[i] = a[i * n + i];
}

void gen_eig_diag(int n, const std::vector<double>& K, const std::vector<double>& Mdiag,
                  std::vector<double>& V, std::vector<double>& lam) {
  // M^{-1/2} K M^{-1/2} = Q diag(lam) Q^T  =>  V = M^{-1/2} Q
  std::vector<double> A(n * n), Q;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = K[i * n + j] / std::sqrt(Mdiag[i] * Mdiag[j]);
  sym_eig(n, A, Q, lam);
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) V[i * n + k] = Q[i * n + k] / std::sqrt(Mdiag[i]);
}

}  // namespace pmg
