// Host construction of the 1D reference-element tables (Sec. 3.1).
//
// Gauss-Lobatto nodes: the endpoints and the interior roots of
// f(x) = x P_p(x) - P_{p-1}(x), which vanishes exactly where P_p' does because
// (1 - x^2) P_p' = p (P_{p-1} - x P_p); Newton uses f'(x) = (p + 1) P_p(x)
// at those roots.  Gauss points: roots of P_q, weights 2 / ((1 - x^2) P_q'^2).
// Lagrange tables by the barycentric formulas (Berrut & Trefethen, SIAM
// Review 46 (2004)).
#include <cmath>
#include <cstring>
#include <vector>

#include "hx_tables.h"

namespace {

void legendre_pair(int n, double x, double* pn, double* pn1) {
  // P_n(x) and P_{n-1}(x) by Bonnet's recurrence
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pn1 = a;
}

void symmetrize(std::vector<double>& x) {
  const int n = (int)x.size();
  for (int i = 0; i < n / 2; ++i) {
    double s = 0.5 * (x[n - 1 - i] - x[i]);
    x[i] = -s;
    x[n - 1 - i] = s;
  }
  if (n & 1) x[n / 2] = 0.0;
}

std::vector<double> gll(int p) {
  std::vector<double> x(p + 1);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);  // Chebyshev-Gauss-Lobatto start
    for (int it = 0; it < 100; ++it) {
      double P, Pm;
      legendre_pair(p, t, &P, &Pm);
      double dt = (t * P - Pm) / ((p + 1.0) * P);
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  symmetrize(x);
  return x;
}

void gauss(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q);
  w.resize(q);
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, Pm;
      legendre_pair(q, t, &P, &Pm);
      double dP = q * (t * P - Pm) / (t * t - 1.0);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  symmetrize(x);
  for (int i = 0; i < q; ++i) {
    double P, Pm;
    legendre_pair(q, x[i], &P, &Pm);
    double dP = q * (x[i] * P - Pm) / (x[i] * x[i] - 1.0);
    w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dP * dP);
  }
  for (int i = 0; i < q / 2; ++i) {
    double s = 0.5 * (w[i] + w[q - 1 - i]);
    w[i] = w[q - 1 - i] = s;
  }
}

std::vector<double> bary_weights(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (x[j] - x[m]);
  return lam;
}

// out (M x L) row-major: Lagrange basis of `nodes` evaluated at `pts`
void interp_matrix(const std::vector<double>& nodes, const std::vector<double>& pts, double* out) {
  const int L = (int)nodes.size(), M = (int)pts.size();
  std::vector<double> lam = bary_weights(nodes);
  for (int a = 0; a < M; ++a) {
    int hit = -1;
    for (int j = 0; j < L; ++j)
      if (pts[a] == nodes[j]) hit = j;
    if (hit >= 0) {
      for (int j = 0; j < L; ++j) out[a * L + j] = (j == hit) ? 1.0 : 0.0;
      continue;
    }
    double ell = 1.0;
    for (int m = 0; m < L; ++m) ell *= (pts[a] - nodes[m]);
    for (int j = 0; j < L; ++j) out[a * L + j] = ell * lam[j] / (pts[a] - nodes[j]);
  }
}

// out (q x q): derivative of the Lagrange basis of `x` at the points x themselves
void collocation_derivative(const std::vector<double>& x, double* out) {
  const int q = (int)x.size();
  std::vector<double> lam = bary_weights(x);
  for (int a = 0; a < q; ++a) {
    double diag = 0.0;
    for (int b = 0; b < q; ++b) {
      if (b == a) continue;
      double v = (lam[b] / lam[a]) / (x[a] - x[b]);
      out[a * q + b] = v;
      diag -= v;
    }
    out[a * q + a] = diag;
  }
}

// Fold S (M x L) with S[M-1-a][L-1-b] = sigma S[a][b] into even / odd parts.
void fold(const double* S, int M, int L, double* Se, double* So) {
  const int HL = L / 2, CL = (L + 1) / 2, CM = (M + 1) / 2;
  for (int a = 0; a < CM; ++a) {
    for (int b = 0; b < HL; ++b) {
      Se[a * CL + b] = 0.5 * (S[a * L + b] + S[a * L + (L - 1 - b)]);
      So[a * HL + b] = 0.5 * (S[a * L + b] - S[a * L + (L - 1 - b)]);
    }
    if (L & 1) Se[a * CL + HL] = S[a * L + HL];
  }
}

}  // namespace

int hx_build_tables(int p, int q, HxTables* t) {
  if (p < 1 || p > HX_PMAX || q < p + 1 || q > HX_QMAX) return -1;
  std::memset(t, 0, sizeof(*t));
  t->p = p;
  t->q = q;
  const int n = p + 1;
  std::vector<double> xn = gll(p), xq, wq;
  gauss(q, xq, wq);
  std::vector<double> B(q * n), Bt(n * q), Dh(q * q), Dht(q * q), D(q * n, 0.0);
  interp_matrix(xn, xq, B.data());
  collocation_derivative(xq, Dh.data());
  for (int a = 0; a < q; ++a)
    for (int j = 0; j < n; ++j) {
      Bt[j * q + a] = B[a * n + j];
      double s = 0.0;
      for (int b = 0; b < q; ++b) s += Dh[a * q + b] * B[b * n + j];
      D[a * n + j] = s;
    }
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) Dht[b * q + a] = Dh[a * q + b];
  fold(B.data(), q, n, t->Be, t->Bo);
  fold(Bt.data(), n, q, t->Bte, t->Bto);
  fold(Dh.data(), q, q, t->De, t->Do);
  fold(Dht.data(), q, q, t->Dte, t->Dto);
  {
    std::vector<double> Dt(n * q);
    for (int a = 0; a < q; ++a)
      for (int j = 0; j < n; ++j) Dt[j * q + a] = D[a * n + j];
    fold(D.data(), q, n, t->Dne, t->Dno);
    fold(Dt.data(), n, q, t->Dnte, t->Dnto);
  }
  {
    const int HQ = q / 2, CQ = (q + 1) / 2;
    for (int a = 0; a < CQ; ++a) {
      for (int b = 0; b < CQ; ++b) t->De2[a * CQ + b] = (b < HQ ? 2.0 : 1.0) * t->De[a * CQ + b];
      for (int b = 0; b < HQ; ++b) t->Do2[a * HQ + b] = 2.0 * t->Do[a * HQ + b];
      const double r = (a < HQ) ? 2.0 : 1.0;
      for (int b = 0; b < CQ; ++b) t->Dte2[a * CQ + b] = r * t->Dte[a * CQ + b];
      for (int b = 0; b < HQ; ++b) t->Dto2[a * HQ + b] = r * t->Dto[a * HQ + b];
    }
  }
  std::memcpy(t->B, B.data(), sizeof(double) * q * n);
  std::memcpy(t->D, D.data(), sizeof(double) * q * n);
  for (int i = 0; i < q; ++i) { t->xq[i] = xq[i]; t->wq[i] = wq[i]; }
  for (int i = 0; i < n; ++i) {
    double P, Pm;
    legendre_pair(p, xn[i], &P, &Pm);
    t->xn[i] = xn[i];
    t->wn[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  return 0;
}

void hx_tables_to_float(const HxTables& d, HxTablesF* f) {
  std::memset(f, 0, sizeof(*f));
  f->p = d.p;
  f->q = d.q;
  auto cp = [](const double* a, float* b, int n) {
    for (int i = 0; i < n; ++i) b[i] = (float)a[i];
  };
  const int H = HX_HALF_UP(HX_QMAX) * HX_HALF_UP(HX_QMAX);
  cp(d.Be, f->Be, H);
  cp(d.Bo, f->Bo, H);
  cp(d.Bte, f->Bte, H);
  cp(d.Bto, f->Bto, H);
  cp(d.De, f->De, H);
  cp(d.Do, f->Do, H);
  cp(d.Dte, f->Dte, H);
  cp(d.Dto, f->Dto, H);
  cp(d.De2, f->De2, H);
  cp(d.Do2, f->Do2, H);
  cp(d.Dte2, f->Dte2, H);
  cp(d.Dto2, f->Dto2, H);
  cp(d.Dne, f->Dne, H);
  cp(d.Dno, f->Dno, H);
  cp(d.Dnte, f->Dnte, H);
  cp(d.Dnto, f->Dnto, H);
  cp(d.B, f->B, HX_QMAX * HX_NMAX);
  cp(d.D, f->D, HX_QMAX * HX_NMAX);
  cp(d.xq, f->xq, HX_QMAX);
  cp(d.wq, f->wq, HX_QMAX);
  cp(d.xn, f->xn, HX_NMAX);
  cp(d.wn, f->wn, HX_NMAX);
}
