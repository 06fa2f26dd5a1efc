// Host-side reference-element basis and small dense linear algebra for the solver setup.
//
// Sec. 4.3: orthonormal Legendre polynomials (three-term recurrence), LGL nodes and
// weights, Vandermonde V, V_r, nodal derivative D_r = V_r V^-1.
// Sec. 5.2: p-transfer I = Phi V^-1 (coarse modal expansion evaluated at fine nodes).
// Sec. 5.1: level orders P_{n-1} = ceil((P_n + 1)/2), iterated to 2, then 1 appended.
// The generalized symmetric eigenproblems of the fast-diagonalisation Schwarz blocks are
// solved with the cyclic Jacobi method.
#pragma once
#include <utility>
#include <vector>

namespace pmg {

// LGL nodes (ascending) and weights of order p >= 1.
void lgl(int p, std::vector<double>& x, std::vector<double>& w);
// Orthonormal Legendre P~_0..P~_n at x (out[k]) and their derivatives (dout[k]).
void legendre_orthonormal(int n, double x, double* out, double* dout);
// Row-major (p+1)x(p+1) derivative matrix D[i*(p+1)+m] = d h_m / dr (r_i).
std::vector<double> diff_matrix(int p);
// Row-major (pf+1)x(pc+1) interpolation of order-pc nodal data at the order-pf nodes.
std::vector<double> transfer_matrix(int pc, int pf);
// Level orders from the coarsening rule.
std::vector<int> coarsening_sequence(int P);
// Level order pairs (p_x, p_z) for different orders (Sec. 5.1 semi-coarsening): while they
// differ, the higher one takes a step of the rule, not below the other; then both follow
// coarsening_sequence.
std::vector<std::pair<int, int>> semi_coarsening_sequence(int P, int Pz);

// In-place Gauss-Jordan inverse of a row-major n x n matrix; false if singular.
bool invert(int n, std::vector<double>& a);
// Symmetric eigendecomposition of a row-major n x n matrix by cyclic Jacobi rotations:
// a = Q diag(lam) Q^T, Q column k = eigenvector k (row-major storage Q[i*n+k]).
void sym_eig(int n, std::vector<double> a, std::vector<double>& Q, std::vector<double>& lam);
// Generalized problem K v = lam M v with M diagonal positive: V^T M V = I, V^T K V = diag.
void gen_eig_diag(int n, const std::vector<double>& K, const std::vector<double>& Mdiag,
                  std::vector<double>& V, std::vector<double>& lam);

}  // namespace pmg
