// 1D tables of the Q_p reference element, passed to every kernel by value
// (kernel parameters live in the constant bank, so a fully unrolled
// contraction reads its coefficients as constant-bank operands).
//
// Notation (Sec. 3.1): n = p + 1 Gauss-Lobatto nodes, q Gauss points.
//   B  (q x n)  B[a][j]  = phi_j(xi_a)                       Eq. (B1D)
//   D  (q x n)  D[a][j]  = phi_j'(xi_a)                      Eq. (D1D)
//   Dh (q x q)  Dh[a][b] = psi_b'(xi_a), psi_b the Lagrange polynomials of
//               the Gauss points; D = Dh B holds exactly for q >= n, so the
//               gradient tensor of Eq. (tensorGradient) can be applied as
//               "interpolate with B, then differentiate at the points".
// Even-odd folded forms (the symmetry noted in Sec. 6): for a 1D operator S
// (M x L) with S[M-1-a][L-1-b] = sigma S[a][b]:
//   Se[a][b] = (S[a][b] + S[a][L-1-b]) / 2   (b < L/2),  Se[a][L/2] = S[a][L/2] for odd L
//   So[a][b] = (S[a][b] - S[a][L-1-b]) / 2   (b < L/2)
// for a < ceil(M/2); row stride ceil(L/2) for Se and floor(L/2) for So.
#pragma once

#define HX_PMAX 8
#define HX_QMAX 10
#define HX_NMAX (HX_PMAX + 1)
#define HX_HALF_UP(x) (((x) + 1) / 2)

template <typename T>
struct HxTablesT {
  int p, q;
  // folded B (sigma = +1): M = q, L = n
  T Be[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_NMAX)];
  T Bo[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_NMAX)];
  // folded B^T (sigma = +1): M = n, L = q
  T Bte[HX_HALF_UP(HX_NMAX) * HX_HALF_UP(HX_QMAX)];
  T Bto[HX_HALF_UP(HX_NMAX) * HX_HALF_UP(HX_QMAX)];
  // folded Dh (sigma = -1): M = L = q
  T De[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  T Do[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  // folded Dh^T (sigma = -1)
  T Dte[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  T Dto[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  // Dh applied to an input given by the folded parts (E, O) of a centro-symmetric
  // interpolation along the same direction: the input's even/odd parts are 2E and 2O
  // (E alone for the middle entry of odd q), so the columns b < q/2 are doubled.
  T De2[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  T Do2[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  // Dh^T with the rows a < q/2 doubled: its folded outputs (2E, 2O) are then exactly the
  // even/odd parts of the result, ready to feed the next contraction along the same direction.
  T Dte2[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  T Dto2[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX)];
  // folded D (sigma = -1): M = q, L = n (derivative of the nodal basis at the Gauss points)
  T Dne[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_NMAX)];
  T Dno[HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_NMAX)];
  // folded D^T (sigma = -1): M = n, L = q
  T Dnte[HX_HALF_UP(HX_NMAX) * HX_HALF_UP(HX_QMAX)];
  T Dnto[HX_HALF_UP(HX_NMAX) * HX_HALF_UP(HX_QMAX)];
  // unfolded tables, row-major
  T B[HX_QMAX * HX_NMAX];
  T D[HX_QMAX * HX_NMAX];
  T xq[HX_QMAX];    // Gauss points on [-1, 1]
  T wq[HX_QMAX];    // Gauss weights
  T xn[HX_NMAX];    // Gauss-Lobatto nodes
  T wn[HX_NMAX];    // Gauss-Lobatto weights 2 / (p (p+1) P_p(x_j)^2) (the collocated mass, Sec. 5.1)
};

// FP64 tables (the operator path) and their FP32 rounding (the inner solver of
// the mixed-precision refinement)
typedef HxTablesT<double> HxTables;
typedef HxTablesT<float> HxTablesF;

#ifdef __cplusplus
// Host construction (basis.cpp). Returns 0 on success.
int hx_build_tables(int p, int q, HxTables* t);
// Round every table entry to FP32.
void hx_tables_to_float(const HxTables& d, HxTablesF* f);
#endif
