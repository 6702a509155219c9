// sg_basis.cpp -- host-side 1D basis and extrapolation-coefficient math.
//
// GLL nodes/weights (Sec. 5.1): nodes are -1, +1 and the roots of P_p'; found by
// Newton's method from Chebyshev-Gauss-Lobatto starting points with P_p'' taken
// from Legendre's equation.  Weights w_i = 2 / (p (p+1) P_p(x_i)^2).
// Derivative matrix by barycentric interpolation: D_ij = (l_j / l_i) / (x_i - x_j),
// D_ii = -sum_{j != i} D_ij, with barycentric weights l_j = 1 / prod_{k!=j}(x_j - x_k).
//
// Extrapolation coefficients (Sec. 3.2, Eq. LSQRCoeffs): beta = V (V^T V)^{-1} v
// with V_ij = P_j(t_i); computed from a thin QR of V by twice-applied modified
// Gram-Schmidt: beta = Q R^{-T} v.  Sparse coefficients (Sec. 3.3, Eq.
// CPQRCoeffs): Householder QR of V^T with Businger-Golub column pivoting.
#include <cmath>
#include <cstring>
#include <vector>

namespace sgb {

static void legendre_all(int p, double x, double* P, double* dP) {
  // P_p(x) and P_p'(x) by the three-term recurrence (derivative recurrence too).
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (p == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < p; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double d2 = d0 + (2 * k + 1) * p1;   // P'_{k+1} = P'_{k-1} + (2k+1) P_k
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

double legendre_value(int j, double x) {
  double P, dP;
  legendre_all(j, x, &P, &dP);
  return P;
}

void gll(int p, double* x, double* w) {
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double xi = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_all(p, xi, &P, &dP);
      double d2P = (2.0 * xi * dP - p * (p + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre_all(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

void derivative(int p, const double* x, double* D) {
  const int n = p + 1;
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (x[j] - x[k]);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * n + j];
    }
    D[i * n + i] = -s;
  }
}

// Reference 1D stiffness Khat = D^T W D on [-1, 1].
void stiffness(int p, const double* D, const double* w, double* K) {
  const int n = p + 1;
  for (int a = 0; a < n; ++a)
    for (int l = 0; l < n; ++l) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += D[q * n + a] * w[q] * D[q * n + l];
      K[a * n + l] = s;
    }
}

static void vander(int M, int m, std::vector<double>& V, std::vector<double>& v) {
  const double h = 2.0 / (M - 1);
  V.assign((size_t)M * (m + 1), 0.0);
  v.assign(m + 1, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j <= m; ++j) V[i * (m + 1) + j] = legendre_value(j, -1.0 + i * h);
  for (int j = 0; j <= m; ++j) v[j] = legendre_value(j, 1.0 + h);
}

// EXTRAP(m, M) coefficients, oldest first.  Returns 0 on success.
int lsq_beta(int M, int m, double* beta) {
  if (M < 1 || m < 0 || m > M - 1) return -1;
  if (M == 1) { beta[0] = 1.0; return 0; }
  std::vector<double> V, v;
  vander(M, m, V, v);
  const int k = m + 1;
  // thin QR by modified Gram-Schmidt, applied twice per column
  std::vector<double> Q(V), R((size_t)k * k, 0.0);
  for (int j = 0; j < k; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        double c = 0.0;
        for (int r = 0; r < M; ++r) c += Q[r * k + i] * Q[r * k + j];
        for (int r = 0; r < M; ++r) Q[r * k + j] -= c * Q[r * k + i];
        R[i * k + j] += c;
      }
    double nrm = 0.0;
    for (int r = 0; r < M; ++r) nrm += Q[r * k + j] * Q[r * k + j];
    nrm = std::sqrt(nrm);
    R[j * k + j] = nrm;
    for (int r = 0; r < M; ++r) Q[r * k + j] /= nrm;
  }
  // y = R^{-T} v (forward substitution), beta = Q y
  std::vector<double> y(k);
  for (int i = 0; i < k; ++i) {
    double s = v[i];
    for (int j = 0; j < i; ++j) s -= R[j * k + i] * y[j];
    y[i] = s / R[i * k + i];
  }
  for (int r = 0; r < M; ++r) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += Q[r * k + j] * y[j];
    beta[r] = s;
  }
  return 0;
}

// SPEXTRAP(m, M) coefficients (m+1 non-zeros), oldest first.
int sparse_beta(int M, int m, double* beta) {
  if (M < 1 || m < 0 || m > M - 1) return -1;
  if (M == 1) { beta[0] = 1.0; return 0; }
  std::vector<double> V, v;
  vander(M, m, V, v);
  const int k = m + 1;
  // A = V^T (k x M), row-major A[r*M + c]
  std::vector<double> A((size_t)k * M);
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < M; ++c) A[r * M + c] = V[c * k + r];
  std::vector<int> perm(M);
  for (int c = 0; c < M; ++c) perm[c] = c;
  std::vector<double> qtv(v);   // Q^T v accumulated by the reflectors
  for (int j = 0; j < k; ++j) {
    double best = -1.0;
    std::vector<double> nr(M, 0.0);
    for (int c = j; c < M; ++c) {
      double s = 0.0;
      for (int r = j; r < k; ++r) s += A[r * M + c] * A[r * M + c];
      nr[c] = std::sqrt(s);
      if (nr[c] > best) best = nr[c];
    }
    const double tol = 64.0 * 2.220446049250313e-16 * best;
    int piv = -1;
    for (int c = j; c < M; ++c)   // ties: most recent time point (largest index)
      if (nr[c] >= best - tol && (piv < 0 || perm[c] > perm[piv])) piv = c;
    if (piv != j) {
      for (int r = 0; r < k; ++r) std::swap(A[r * M + j], A[r * M + piv]);
      std::swap(perm[j], perm[piv]);
    }
    // Householder reflector on rows j..k-1 of column j
    double nx = 0.0;
    for (int r = j; r < k; ++r) nx += A[r * M + j] * A[r * M + j];
    nx = std::sqrt(nx);
    double x0 = A[j * M + j];
    double alpha = (x0 >= 0.0) ? -nx : nx;
    std::vector<double> u(k, 0.0);
    for (int r = j; r < k; ++r) u[r] = A[r * M + j];
    u[j] -= alpha;
    double un = 0.0;
    for (int r = j; r < k; ++r) un += u[r] * u[r];
    un = std::sqrt(un);
    if (un > 0.0) {
      for (int r = j; r < k; ++r) u[r] /= un;
      for (int c = 0; c < M; ++c) {
        double s = 0.0;
        for (int r = j; r < k; ++r) s += u[r] * A[r * M + c];
        for (int r = j; r < k; ++r) A[r * M + c] -= 2.0 * u[r] * s;
      }
      double s = 0.0;
      for (int r = j; r < k; ++r) s += u[r] * qtv[r];
      for (int r = j; r < k; ++r) qtv[r] -= 2.0 * u[r] * s;
    }
  }
  // back substitution R_hat bhat = Q^T v
  std::vector<double> bh(k);
  for (int i = k - 1; i >= 0; --i) {
    double s = qtv[i];
    for (int j = i + 1; j < k; ++j) s -= A[i * M + j] * bh[j];
    bh[i] = s / A[i * M + i];
  }
  for (int c = 0; c < M; ++c) beta[c] = 0.0;
  for (int j = 0; j < k; ++j) beta[perm[j]] = bh[j];
  return 0;
}

}  // namespace sgb
