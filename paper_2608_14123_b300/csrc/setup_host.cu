// Host-side setup of one level: GLL basis, element geometry, face factors and
// penalties (Sec. 2.2), the nine 1D fast-diagonalization variants, weights and
// geometric surrogate (Sec. 4.3.1), and transfer matrices (Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dgfas_internal.h"
#include "setup_host.h"

namespace host {

// ---------------------------------------------------------------- GLL basis
static void legendre(int p, double x, double& P, double& Pm1) {
  double a = 1.0, b = x;
  if (p == 0) { P = 1.0; Pm1 = 0.0; return; }
  for (int n = 2; n <= p; ++n) {
    double c = ((2 * n - 1) * x * b - (n - 1) * a) / n;
    a = b;
    b = c;
  }
  P = b;
  Pm1 = a;
}

// GLL nodes (interior = roots of P_p') by Newton on (1-x^2) P_p'(x) = p (P_{p-1} - x P_p),
// whose derivative is -p (p+1) P_p; weights 2 / (p (p+1) P_p^2).
void gll(int p, std::vector<double>& x, std::vector<double>& w) {
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  for (int i = 0; i <= p; ++i) x[i] = -std::cos(M_PI * i / p);
  for (int i = 1; i < p; ++i) {
    double xi = x[i];
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre(p, xi, P, Pm1);
      double q = p * (Pm1 - xi * P);
      double dq = -p * (p + 1) * P;
      double dx = q / dq;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 0; i <= p / 2; ++i) {   // exact symmetry
    double s = 0.5 * (x[p - i] - x[i]);
    x[p - i] = s;
    x[i] = -s;
  }
  for (int i = 0; i <= p; ++i) {
    double P, Pm1;
    legendre(p, x[i], P, Pm1);
    w[i] = 2.0 / (p * (p + 1) * P * P);
  }
}

// Barycentric weights of the node set.
static std::vector<double> bary(const std::vector<double>& x) {
  int n = (int)x.size();
  std::vector<double> b(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) b[j] /= (x[j] - x[k]);
  return b;
}

// D[i][j] = l_j'(x_i): off-diagonal (b_j/b_i)/(x_i - x_j), diagonal = -sum of the row.
std::vector<double> diff_matrix(const std::vector<double>& x) {
  int n = (int)x.size();
  std::vector<double> b = bary(x), D(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) {
        D[i * n + j] = (b[j] / b[i]) / (x[i] - x[j]);
        s += D[i * n + j];
      }
    D[i * n + i] = -s;
  }
  return D;
}

// L[q][j] = l_j(y_q) on nodes x (barycentric formula of the second kind).
std::vector<double> interp(const std::vector<double>& x, const std::vector<double>& y) {
  int n = (int)x.size(), m = (int)y.size();
  std::vector<double> b = bary(x), L(m * n, 0.0);
  for (int q = 0; q < m; ++q) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (y[q] == x[j]) hit = j;
    if (hit >= 0) { L[q * n + hit] = 1.0; continue; }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += b[j] / (y[q] - x[j]);
    for (int j = 0; j < n; ++j) L[q * n + j] = (b[j] / (y[q] - x[j])) / den;
  }
  return L;
}

// ---------------------------------------------------------------- geometry
// Trilinear map x(xi) = sum_c N_c(xi) x_c and Jacobian J[a][b] = dx_a/dxi_b.
void trilinear(const double* cr, double x1, double x2, double x3, double X[3], double J[9]) {
  const double xi[3] = {x1, x2, x3};
  for (int a = 0; a < 3; ++a) X[a] = 0.0;
  for (int a = 0; a < 9; ++a) J[a] = 0.0;
  for (int c = 0; c < 8; ++c) {
    double s[3], f[3];
    for (int d = 0; d < 3; ++d) {
      s[d] = ((c >> d) & 1) ? 1.0 : -1.0;
      f[d] = 0.5 * (1.0 + s[d] * xi[d]);
    }
    double Nc = f[0] * f[1] * f[2];
    double dN[3] = {0.5 * s[0] * f[1] * f[2], 0.5 * s[1] * f[0] * f[2], 0.5 * s[2] * f[0] * f[1]};
    for (int a = 0; a < 3; ++a) {
      X[a] += Nc * cr[c * 3 + a];
      for (int b = 0; b < 3; ++b) J[a * 3 + b] += dN[b] * cr[c * 3 + a];
    }
  }
}

static double det3(const double* J) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

bool is_box(const double* cr, double h[3]) {
  for (int d = 0; d < 3; ++d) {
    double lo = cr[0 * 3 + d], hi = cr[(1 << d) * 3 + d];
    h[d] = hi - lo;
    if (!(h[d] > 0)) return false;
    for (int c = 0; c < 8; ++c) {
      double want = ((c >> d) & 1) ? hi : lo;
      if (std::fabs(cr[c * 3 + d] - want) > 1e-14 * (std::fabs(lo) + std::fabs(hi) + 1.0))
        return false;
    }
  }
  return true;
}

// Exact volume of a trilinear element: det J has degree <= 2 per direction,
// so the 2-point Gauss rule per direction is exact.
double exact_volume(const double* cr) {
  const double g = 1.0 / std::sqrt(3.0);
  double vol = 0.0;
  for (int a = -1; a <= 1; a += 2)
    for (int b = -1; b <= 1; b += 2)
      for (int c = -1; c <= 1; c += 2) {
        double X[3], J[9];
        trilinear(cr, a * g, b * g, c * g, X, J);
        vol += det3(J);
      }
  return vol;
}

// Geometric surrogate (Sec. 4.3.1): P1 Legendre coefficients of the map give
// the parallelepiped edges a_i; cuboid widths 2|a_i| scaled to the exact volume.
void surrogate_widths(const double* cr, double dx[3]) {
  double ell[3];
  for (int i = 0; i < 3; ++i) {
    double a[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
      double s = ((c >> i) & 1) ? 1.0 : -1.0;
      for (int k = 0; k < 3; ++k) a[k] += s * cr[c * 3 + k] / 8.0;
    }
    ell[i] = 2.0 * std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  }
  double vol = exact_volume(cr);
  double s = std::cbrt(vol / (ell[0] * ell[1] * ell[2]));
  for (int i = 0; i < 3; ++i) dx[i] = ell[i] * s;
}

// ---------------------------------------------------------------- FD tables
// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major).
// On return A's diagonal holds eigenvalues, V columns the eigenvectors.
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // A <- A J  (columns p, q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

int overlap_layers(int p, double delta) {
  std::vector<double> x, w;
  gll(p, x, w);
  int m = 0;
  for (int j = 0; j <= p; ++j)
    if (0.5 * (1.0 + x[j]) <= delta + 1e-14) ++m;
  return m;
}

static double quintic(double x) { return x * x * x * (10.0 - 15.0 * x + 6.0 * x * x); }

// One side variant (left, right in {'i','d','n'}): 1D SIP on the three standard
// cells with the centre's side conditions, restricted to the subdomain nodes;
// generalized eigenpairs L s = lam M s (S^T M S = I) and the weights.
void fd_variant(int p, int m, double mu_star, double delta, char left, char right,
                std::vector<double>& S, std::vector<double>& lam, std::vector<double>& W) {
  const int N = p + 1, n3 = 3 * N;
  std::vector<double> x, w;
  gll(p, x, w);
  std::vector<double> D = diff_matrix(x);
  const double mu = mu_star * p * (p + 1) / 4.0;
  std::vector<double> L(n3 * n3, 0.0), mass(n3, 0.0);
  bool cell[3] = {left == 'i' || left == 'f', true, right == 'i' || right == 'f'};
  for (int c = 0; c < 3; ++c) {
    if (!cell[c]) continue;
    for (int i = 0; i < N; ++i) {
      mass[c * N + i] = w[i];
      for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int q = 0; q < N; ++q) s += D[q * N + i] * w[q] * D[q * N + j];
        L[(c * N + i) * n3 + c * N + j] += s;
      }
    }
  }
  // face term with jump vector T and normal-derivative average Q: pen T T^T - Q T^T - T Q^T
  auto face = [&](const std::vector<double>& T, const std::vector<double>& Q, double pen) {
    for (int i = 0; i < n3; ++i)
      for (int j = 0; j < n3; ++j)
        L[i * n3 + j] += pen * T[i] * T[j] - Q[i] * T[j] - T[i] * Q[j];
  };
  for (int a = 0; a < 2; ++a) {
    int b = a + 1;
    if (!cell[a] || !cell[b]) continue;
    std::vector<double> T(n3, 0.0), Q(n3, 0.0);
    T[a * N + N - 1] = 1.0;
    T[b * N + 0] = -1.0;
    for (int j = 0; j < N; ++j) {
      Q[a * N + j] += 0.5 * D[(N - 1) * N + j];
      Q[b * N + j] += 0.5 * D[0 * N + j];
    }
    face(T, Q, mu);
  }
  if (left == 'd') {
    std::vector<double> T(n3, 0.0), Q(n3, 0.0);
    T[N] = 1.0;
    for (int j = 0; j < N; ++j) Q[N + j] = -D[0 * N + j];
    face(T, Q, 2.0 * mu);
  }
  if (right == 'd') {
    std::vector<double> T(n3, 0.0), Q(n3, 0.0);
    T[N + N - 1] = 1.0;
    for (int j = 0; j < N; ++j) Q[N + j] = D[(N - 1) * N + j];
    face(T, Q, 2.0 * mu);
  }
  std::vector<int> sel;
  if (left == 'i')
    for (int i = N - m; i < N; ++i) sel.push_back(i);
  for (int i = 0; i < N; ++i) sel.push_back(N + i);
  if (right == 'i')
    for (int i = 0; i < m; ++i) sel.push_back(2 * N + i);
  const int n = (int)sel.size();
  std::vector<double> C(n * n), V;
  std::vector<double> sq(n);
  for (int i = 0; i < n; ++i) sq[i] = std::sqrt(mass[sel[i]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      C[i * n + j] = 0.5 * (L[sel[i] * n3 + sel[j]] + L[sel[j] * n3 + sel[i]]) / (sq[i] * sq[j]);
  jacobi_eig(n, C, V);
  S.assign(n * n, 0.0);
  lam.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    lam[k] = C[k * n + k];
    for (int i = 0; i < n; ++i) S[i * n + k] = V[i * n + k] / sq[i];
  }
  // weights: product of the side factors phi(t), t = signed distance beyond the side
  auto phi = [&](double t) {
    double z = (delta - t) / (2.0 * delta);
    z = std::min(1.0, std::max(0.0, z));
    return quintic(z);
  };
  W.assign(n, 1.0);
  for (int s = 0; s < n; ++s) {
    int gidx = sel[s], c = gidx / N, i = gidx % N;
    double tl, tr;   // distance beyond the centre's left / right face
    if (c == 0) { tl = 0.5 * (1.0 - x[i]); tr = -1.0 - tl; }
    else if (c == 1) { tl = -0.5 * (1.0 + x[i]); tr = -0.5 * (1.0 - x[i]); }
    else { tr = 0.5 * (1.0 + x[i]); tl = -1.0 - tr; }
    double f = 1.0;
    if (left == 'i') f *= phi(tl);
    if (right == 'i') f *= phi(tr);
    W[s] = f;
  }
}

}  // namespace host
