// Plain FP64 CPU oracle for the frozen Gaussian approximation (FGA) of
// Yang, Lu and Fomel, "Seismic modeling using the frozen Gaussian approximation".
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may load or call this
// file: only the tests, the smoke check and the benchmark's CPU-baseline leg do.
// It shares no code, header, table or helper with the CUDA implementation.
//
// What is here (the FBI step itself lives in fga_oracle.py, where the paper's
// "FFT on the small box" is a library call):
//   * the velocity medium: tensor-product cubic B-spline with analytic
//     derivatives up to third order (the paper does not say how c is
//     interpolated; the cubic B-spline is the reading chosen because the
//     dynamic ray equations need second derivatives of c);
//   * the Hamiltonian H = sigma c(Q)|P| (Eq. hamiltonian) and its first and
//     second derivatives, written out from their definitions;
//   * the ray equations (Eq. characline), the dynamic ray equations (Eqs. dzQ,
//     dzP), the amplitude equation (Eq. a_formu with Z from Eq. op_zZ) and the
//     action S, integrated with classical fourth-order Runge-Kutta (Numerical
//     test section);
//   * the divided-difference alternative for d_z Q and d_z P (the passage after
//     Eq. op_zZ): auxiliary rays from (q +- dq_j e_j, p) and (q, p +- dp_j e_j)
//     integrated with the ray, Z and dZ/dt from central differences across them;
//   * the reconstruction sum (Eq. recons), evaluated term by term with
//     std::exp of the full complex exponent;
//   * a brute-force FBI direct sum (Eq. psi) used only to pin the FFT route.
//
// Every routine is FP64, per Gaussian or per output point, with OpenMP only
// over independent Gaussians / output points (each result is summed in the
// same order whatever the thread count).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;
static const double kPi = 3.14159265358979323846;

namespace {

struct Grid {
  int dim;
  int64_t n[3];
  double h[3], o[3];
  int periodic[3];
};

Grid make_grid(int dim, const int64_t* n, const double* h, const double* o, const int* periodic) {
  Grid g;
  g.dim = dim;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = k < dim ? n[k] : 1;
    g.h[k] = k < dim ? h[k] : 1.0;
    g.o[k] = k < dim ? o[k] : 0.0;
    g.periodic[k] = k < dim ? periodic[k] : 0;
  }
  return g;
}

// ---------------------------------------------------------------------------
// Scalars. The ray system below is written once for a real scalar type R and its
// complex partner: R = double is the oracle itself; R = Dual carries, next to every
// value, its derivative along one direction V of the velocity coefficients (forward
// mode: a dual number x + x' e with e^2 = 0, so every operation applies the chain
// rule to the derivative part and leaves the value part exactly as in plain FP64).
// Branch decisions (the spline cell, the window cut, pivoting) follow the value, so
// the derivative is that of the piece the value lies on.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};

inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(const Dual& a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, const Dual& b) { return Dual(a + b.v, b.d); }
inline Dual operator-(const Dual& a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, const Dual& b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
inline bool operator<(const Dual& a, double b) { return a.v < b; }
inline Dual sqrt(const Dual& a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual fabs(const Dual& a) { return a.v < 0 ? -a : a; }

// Complex partner of Dual: complex value and complex derivative.
struct DualC {
  cplx v, d;
  DualC() : v(0.0), d(0.0) {}
  DualC(double re, double im) : v(re, im), d(0.0) {}
  DualC(const cplx& x) : v(x), d(0.0) {}
  DualC(const cplx& x, const cplx& dx) : v(x), d(dx) {}
  DualC(const Dual& re) : v(re.v), d(re.d) {}
};

inline DualC operator+(const DualC& a, const DualC& b) { return DualC(a.v + b.v, a.d + b.d); }
inline DualC operator-(const DualC& a, const DualC& b) { return DualC(a.v - b.v, a.d - b.d); }
inline DualC operator-(const DualC& a) { return DualC(-a.v, -a.d); }
inline DualC operator*(const DualC& a, const DualC& b) { return DualC(a.v * b.v, a.d * b.v + a.v * b.d); }
inline DualC operator/(const DualC& a, const DualC& b) {
  return DualC(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline DualC operator*(const DualC& a, const Dual& b) { return DualC(a.v * b.v, a.d * b.v + a.v * b.d); }
inline DualC operator*(const Dual& a, const DualC& b) { return b * a; }
inline DualC operator*(const DualC& a, double b) { return DualC(a.v * b, a.d * b); }
inline DualC operator*(double a, const DualC& b) { return DualC(a * b.v, a * b.d); }
inline DualC operator/(const DualC& a, double b) { return DualC(a.v / b, a.d / b); }
inline DualC operator-(const DualC& a, const Dual& b) { return DualC(a.v - b.v, a.d - b.d); }
inline DualC& operator+=(DualC& a, const DualC& b) { a = a + b; return a; }
inline DualC& operator-=(DualC& a, const DualC& b) { a = a - b; return a; }
inline DualC exp(const DualC& a) {
  cplx e = std::exp(a.v);
  return DualC(e, a.d * e);
}

template <class R> struct Num;
template <> struct Num<double> { typedef cplx C; };
template <> struct Num<Dual> { typedef DualC C; };

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double mag(const cplx& z) { return std::abs(z); }
inline double mag(const DualC& z) { return std::abs(z.v); }
inline double fmod_val(double x, double L) { return std::fmod(x, L); }
inline Dual fmod_val(const Dual& x, double L) { return Dual(std::fmod(x.v, L), x.d); }

// The spline coefficients C and, for the derivative, the direction V (a grid-shaped
// change of the coefficients; NULL = 0).
struct Coefs {
  const double* C;
  const double* V;
};
inline void coef_at(const Coefs& cf, int64_t i, double& out) { out = cf.C[i]; }
inline void coef_at(const Coefs& cf, int64_t i, Dual& out) { out = Dual(cf.C[i], cf.V ? cf.V[i] : 0.0); }

// ---------------------------------------------------------------------------
// Cubic B-spline beta_3 and its derivatives (order 0..3), piecewise by |t|.
// ---------------------------------------------------------------------------
template <class R>
R beta3(const R& t, int order) {
  using std::fabs;
  R at = fabs(t);
  double sg = val(t) < 0 ? -1.0 : 1.0;
  if (val(at) >= 2.0) return R(0.0);
  if (val(at) < 1.0) {
    switch (order) {
      case 0: return 2.0 / 3.0 - t * t + 0.5 * at * at * at;
      case 1: return -2.0 * t + 1.5 * t * at;
      case 2: return -2.0 + 3.0 * at;
      default: return R(3.0 * sg);
    }
  }
  R u = 2.0 - at;
  switch (order) {
    case 0: return u * u * u / 6.0;
    case 1: return -sg * u * u / 2.0;
    case 2: return u;
    default: return R(-sg);
  }
}

// Coefficient index along one axis: clamped on open axes, wrapped on periodic ones.
int64_t coef_index(const Grid& g, int k, int64_t i) {
  int64_t n = g.n[k];
  if (g.periodic[k]) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  if (i < 0) return 0;
  if (i > n - 1) return n - 1;
  return i;
}

// c(x) = sum_i C_i prod_k beta3((x_k - o_k)/h_k - i_k), and its derivatives.
// deriv[k] is the derivative order taken along axis k.
template <class R>
R spline_value(const Grid& g, const Coefs& cf, const R* x, const int* deriv) {
  int64_t base[3];
  R u[3];
  for (int k = 0; k < g.dim; ++k) {
    u[k] = (x[k] - g.o[k]) / g.h[k];
    base[k] = (int64_t)std::floor(val(u[k])) - 1;
  }
  R total(0.0);
  int ntaps = 1;
  for (int k = 0; k < g.dim; ++k) ntaps *= 4;
  for (int t = 0; t < ntaps; ++t) {
    int rem = t;
    int64_t flat = 0;
    R w(1.0);
    for (int k = 0; k < g.dim; ++k) {
      int tk = rem % 4;
      rem /= 4;
      int64_t i = base[k] + tk;
      w = w * (beta3(u[k] - (double)i, deriv[k]) / std::pow(g.h[k], deriv[k]));
      flat = flat * g.n[k] + coef_index(g, k, i);
    }
    R ci;
    coef_at(cf, flat, ci);
    total += ci * w;
  }
  return total;
}

template <class R>
struct Medium {
  R c;
  R grad[3];
  R hess[3][3];
};

template <class R>
Medium<R> medium_at(const Grid& g, const Coefs& cf, const R* x) {
  Medium<R> m;
  int d0[3] = {0, 0, 0};
  m.c = spline_value(g, cf, x, d0);
  for (int k = 0; k < g.dim; ++k) {
    int d1[3] = {0, 0, 0};
    d1[k] = 1;
    m.grad[k] = spline_value(g, cf, x, d1);
    for (int l = 0; l < g.dim; ++l) {
      int d2[3] = {0, 0, 0};
      d2[k] += 1;
      d2[l] += 1;
      m.hess[k][l] = spline_value(g, cf, x, d2);
    }
  }
  return m;
}

// ---------------------------------------------------------------------------
// Hamiltonian H = sigma c(Q) |P| (Eq. hamiltonian) and its derivatives.
// ---------------------------------------------------------------------------
template <class R>
struct HamDerivs {
  R H;
  R dHdQ[3], dHdP[3];
  R HQQ[3][3], HQP[3][3], HPP[3][3], HPQ[3][3];  // HQP[l][k] = d2H/dQ_l dP_k
};

template <class R>
HamDerivs<R> hamiltonian(const Grid& g, const Coefs& cf, int sigma, const R* Q, const R* P) {
  using std::sqrt;
  HamDerivs<R> r;
  int d = g.dim;
  Medium<R> m = medium_at(g, cf, Q);
  R pn(0.0);
  for (int k = 0; k < d; ++k) pn += P[k] * P[k];
  pn = sqrt(pn);
  R nh[3];
  for (int k = 0; k < d; ++k) nh[k] = P[k] / pn;
  double s = (double)sigma;
  r.H = s * m.c * pn;
  for (int k = 0; k < d; ++k) {
    r.dHdQ[k] = s * pn * m.grad[k];
    r.dHdP[k] = s * m.c * nh[k];
  }
  for (int l = 0; l < d; ++l)
    for (int k = 0; k < d; ++k) {
      r.HQQ[l][k] = s * pn * m.hess[l][k];
      r.HQP[l][k] = s * m.grad[l] * nh[k];
      r.HPQ[l][k] = s * nh[l] * m.grad[k];
      r.HPP[l][k] = s * m.c * ((l == k ? 1.0 : 0.0) - nh[l] * nh[k]) / pn;
    }
  return r;
}

// ---------------------------------------------------------------------------
// Per-Gaussian state and the right-hand side of the FGA ODE system.
// A = d_z Q and B = d_z P with (j,k) entry d_{z_j} Q_k (resp. P_k).
// ---------------------------------------------------------------------------
template <class R>
struct State {
  typedef typename Num<R>::C C;
  R Q[3], P[3];
  C A[3][3], B[3][3];
  C a;
  R S;
};

template <class R>
void state_zero(State<R>& s) {
  for (int i = 0; i < 3; ++i) {
    s.Q[i] = R(0.0);
    s.P[i] = R(0.0);
    for (int j = 0; j < 3; ++j) {
      s.A[i][j] = typename Num<R>::C(0.0, 0.0);
      s.B[i][j] = typename Num<R>::C(0.0, 0.0);
    }
  }
  s.a = typename Num<R>::C(0.0, 0.0);
  s.S = R(0.0);
}

// out = y + h * k
template <class R>
void state_axpy(int d, const State<R>& y, double h, const State<R>& k, State<R>& out) {
  for (int i = 0; i < d; ++i) {
    out.Q[i] = y.Q[i] + h * k.Q[i];
    out.P[i] = y.P[i] + h * k.P[i];
    for (int j = 0; j < d; ++j) {
      out.A[i][j] = y.A[i][j] + h * k.A[i][j];
      out.B[i][j] = y.B[i][j] + h * k.B[i][j];
    }
  }
  out.a = y.a + h * k.a;
  out.S = y.S + h * k.S;
}

// tr(Z^{-1} W) by solving Z X = W with Gaussian elimination (partial pivoting).
template <class C>
C trace_solve(int d, const C Zin[3][3], const C Win[3][3]) {
  C Z[3][3], W[3][3];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      Z[i][j] = Zin[i][j];
      W[i][j] = Win[i][j];
    }
  for (int col = 0; col < d; ++col) {
    int piv = col;
    for (int r = col + 1; r < d; ++r)
      if (mag(Z[r][col]) > mag(Z[piv][col])) piv = r;
    if (piv != col)
      for (int j = 0; j < d; ++j) {
        std::swap(Z[col][j], Z[piv][j]);
        std::swap(W[col][j], W[piv][j]);
      }
    for (int r = col + 1; r < d; ++r) {
      C f = Z[r][col] / Z[col][col];
      for (int j = 0; j < d; ++j) {
        Z[r][j] -= f * Z[col][j];
        W[r][j] -= f * W[col][j];
      }
    }
  }
  C X[3][3];
  for (int j = 0; j < d; ++j)
    for (int r = d - 1; r >= 0; --r) {
      C acc = W[r][j];
      for (int c = r + 1; c < d; ++c) acc -= Z[r][c] * X[c][j];
      X[r][j] = acc / Z[r][r];
    }
  C tr(0.0, 0.0);
  for (int i = 0; i < d; ++i) tr += X[i][i];
  return tr;
}

template <class R>
void rhs(const Grid& g, const Coefs& cf, int sigma, const State<R>& y, State<R>& dy) {
  typedef typename Num<R>::C C;
  int d = g.dim;
  state_zero(dy);
  HamDerivs<R> hd = hamiltonian(g, cf, sigma, y.Q, y.P);
  // Eq. characline
  for (int k = 0; k < d; ++k) {
    dy.Q[k] = hd.dHdP[k];
    dy.P[k] = -hd.dHdQ[k];
  }
  // Eqs. dzQ, dzP (componentwise form, summation over l)
  for (int j = 0; j < d; ++j)
    for (int k = 0; k < d; ++k) {
      C dA(0.0, 0.0), dB(0.0, 0.0);
      for (int l = 0; l < d; ++l) {
        dA += y.A[j][l] * hd.HQP[l][k] + y.B[j][l] * hd.HPP[l][k];
        dB += -y.A[j][l] * hd.HQQ[l][k] - y.B[j][l] * hd.HPQ[l][k];
      }
      dy.A[j][k] = dA;
      dy.B[j][k] = dB;
    }
  // Eq. a_formu with Z = d_z(Q + iP) = A + iB (Eq. op_zZ)
  const C I(0.0, 1.0);
  C Z[3][3], dZ[3][3];
  for (int j = 0; j < d; ++j)
    for (int k = 0; k < d; ++k) {
      Z[j][k] = y.A[j][k] + I * y.B[j][k];
      dZ[j][k] = dy.A[j][k] + I * dy.B[j][k];
    }
  R dot(0.0);
  for (int k = 0; k < d; ++k) dot += hd.dHdP[k] * hd.dHdQ[k];
  dy.a = y.a * (dot / hd.H) + 0.5 * y.a * trace_solve(d, Z, dZ);
  // action: dS/dt = P . dQ/dt - H
  R pq(0.0);
  for (int k = 0; k < d; ++k) pq += y.P[k] * dy.Q[k];
  dy.S = pq - hd.H;
}

template <class R>
void wrap_periodic(const Grid& g, State<R>& y) {
  for (int k = 0; k < g.dim; ++k) {
    if (!g.periodic[k]) continue;
    double L = g.n[k] * g.h[k];
    R r = fmod_val(y.Q[k] - g.o[k], L);
    if (val(r) < 0) r = r + L;
    y.Q[k] = g.o[k] + r;
  }
}

template <class R>
void rk4_step(const Grid& g, const Coefs& cf, int sigma, State<R>& y, double dt) {
  int d = g.dim;
  State<R> k1, k2, k3, k4, tmp;
  state_zero(tmp);
  rhs(g, cf, sigma, y, k1);
  state_axpy(d, y, 0.5 * dt, k1, tmp);
  rhs(g, cf, sigma, tmp, k2);
  state_axpy(d, y, 0.5 * dt, k2, tmp);
  rhs(g, cf, sigma, tmp, k3);
  state_axpy(d, y, dt, k3, tmp);
  rhs(g, cf, sigma, tmp, k4);
  State<R> out = y;
  for (int i = 0; i < d; ++i) {
    out.Q[i] = y.Q[i] + dt / 6.0 * (k1.Q[i] + 2.0 * k2.Q[i] + 2.0 * k3.Q[i] + k4.Q[i]);
    out.P[i] = y.P[i] + dt / 6.0 * (k1.P[i] + 2.0 * k2.P[i] + 2.0 * k3.P[i] + k4.P[i]);
    for (int j = 0; j < d; ++j) {
      out.A[i][j] = y.A[i][j] + dt / 6.0 * (k1.A[i][j] + 2.0 * k2.A[i][j] + 2.0 * k3.A[i][j] + k4.A[i][j]);
      out.B[i][j] = y.B[i][j] + dt / 6.0 * (k1.B[i][j] + 2.0 * k2.B[i][j] + 2.0 * k3.B[i][j] + k4.B[i][j]);
    }
  }
  out.a = y.a + dt / 6.0 * (k1.a + 2.0 * k2.a + 2.0 * k3.a + k4.a);
  out.S = y.S + dt / 6.0 * (k1.S + 2.0 * k2.S + 2.0 * k3.S + k4.S);
  wrap_periodic(g, out);
  y = out;
}

// Initial values Q = q, P = p, A = I, B = -iI, a = 2^{d/2}, S = 0.
template <class R>
void state_init(int d, const double* q, const double* p, State<R>& y) {
  typedef typename Num<R>::C C;
  state_zero(y);
  for (int k = 0; k < d; ++k) {
    y.Q[k] = R(q[k]);
    y.P[k] = R(p[k]);
    y.A[k][k] = C(1.0, 0.0);
    y.B[k][k] = C(0.0, -1.0);
  }
  y.a = C(std::pow(2.0, 0.5 * d), 0.0);
  y.S = R(0.0);
}

// ---------------------------------------------------------------------------
// Divided-difference form of Z (the alternative to Eqs. dzQ, dzP named after Eq.
// op_zZ). Besides its own ray the Gaussian carries 4d auxiliary rays, r = 4j + m:
// m = 0, 1 start at q +- dq_j e_j (p unchanged), m = 2, 3 at p +- dp_j e_j (q
// unchanged); all follow Eq. characline. With d_z = d_q - i d_p (Eq. op_zZ) and
// central differences,
//   Z_jk = d_{z_j}(Q_k + i P_k) = (Dq_j Q_k + Dp_j P_k) + i (Dq_j P_k - Dp_j Q_k),
//   Dq_j X = (X[4j] - X[4j+1])/(2 dq_j),  Dp_j X = (X[4j+2] - X[4j+3])/(2 dp_j),
// and dZ/dt the same differences of the auxiliary rays' right-hand sides; the
// amplitude and the action then follow Eq. a_formu and dS/dt = P.dQ/dt - H.
// ---------------------------------------------------------------------------
struct DDState {
  double Q[3], P[3];          // the Gaussian's own ray
  double Qa[12][3], Pa[12][3];  // the auxiliary rays
  cplx a;
  double S;
};

void dd_axpy(int d, const DDState& y, double h, const DDState& k, DDState& out) {
  for (int i = 0; i < d; ++i) {
    out.Q[i] = y.Q[i] + h * k.Q[i];
    out.P[i] = y.P[i] + h * k.P[i];
  }
  for (int r = 0; r < 4 * d; ++r)
    for (int i = 0; i < d; ++i) {
      out.Qa[r][i] = y.Qa[r][i] + h * k.Qa[r][i];
      out.Pa[r][i] = y.Pa[r][i] + h * k.Pa[r][i];
    }
  out.a = y.a + h * k.a;
  out.S = y.S + h * k.S;
}

// Z (or dZ/dt, from the auxiliary rays' rates) by central differences.
void dd_matrix(int d, const double Qa[12][3], const double Pa[12][3], const double* dq,
               const double* dp, cplx Z[3][3]) {
  const cplx I(0.0, 1.0);
  for (int j = 0; j < d; ++j)
    for (int k = 0; k < d; ++k) {
      double DqQ = (Qa[4 * j][k] - Qa[4 * j + 1][k]) / (2.0 * dq[j]);
      double DqP = (Pa[4 * j][k] - Pa[4 * j + 1][k]) / (2.0 * dq[j]);
      double DpQ = (Qa[4 * j + 2][k] - Qa[4 * j + 3][k]) / (2.0 * dp[j]);
      double DpP = (Pa[4 * j + 2][k] - Pa[4 * j + 3][k]) / (2.0 * dp[j]);
      Z[j][k] = (DqQ + DpP) + I * (DqP - DpQ);
    }
}

void dd_rhs(const Grid& g, const double* C, int sigma, const double* dq, const double* dp,
            const DDState& y, DDState& dy) {
  int d = g.dim;
  std::memset(&dy, 0, sizeof(DDState));
  const Coefs cf = {C, nullptr};
  HamDerivs<double> hd = hamiltonian<double>(g, cf, sigma, y.Q, y.P);
  for (int k = 0; k < d; ++k) {
    dy.Q[k] = hd.dHdP[k];
    dy.P[k] = -hd.dHdQ[k];
  }
  for (int r = 0; r < 4 * d; ++r) {
    HamDerivs<double> ha = hamiltonian<double>(g, cf, sigma, y.Qa[r], y.Pa[r]);
    for (int k = 0; k < d; ++k) {
      dy.Qa[r][k] = ha.dHdP[k];
      dy.Pa[r][k] = -ha.dHdQ[k];
    }
  }
  cplx Z[3][3], dZ[3][3];
  dd_matrix(d, y.Qa, y.Pa, dq, dp, Z);
  dd_matrix(d, dy.Qa, dy.Pa, dq, dp, dZ);
  double dot = 0.0;
  for (int k = 0; k < d; ++k) dot += hd.dHdP[k] * hd.dHdQ[k];
  dy.a = y.a * (dot / hd.H) + 0.5 * y.a * trace_solve(d, Z, dZ);
  double pq = 0.0;
  for (int k = 0; k < d; ++k) pq += y.P[k] * dy.Q[k];
  dy.S = pq - hd.H;
}

// The auxiliary rays are not wrapped on periodic axes (the medium is periodic, and
// their differences must not jump by a period); the Gaussian's own ray is.
void dd_rk4_step(const Grid& g, const double* C, int sigma, const double* dq, const double* dp,
                 DDState& y, double dt) {
  int d = g.dim;
  DDState k1, k2, k3, k4, tmp;
  std::memset(&tmp, 0, sizeof(DDState));
  dd_rhs(g, C, sigma, dq, dp, y, k1);
  dd_axpy(d, y, 0.5 * dt, k1, tmp);
  dd_rhs(g, C, sigma, dq, dp, tmp, k2);
  dd_axpy(d, y, 0.5 * dt, k2, tmp);
  dd_rhs(g, C, sigma, dq, dp, tmp, k3);
  dd_axpy(d, y, dt, k3, tmp);
  dd_rhs(g, C, sigma, dq, dp, tmp, k4);
  DDState out = y;
  for (int i = 0; i < d; ++i) {
    out.Q[i] = y.Q[i] + dt / 6.0 * (k1.Q[i] + 2.0 * k2.Q[i] + 2.0 * k3.Q[i] + k4.Q[i]);
    out.P[i] = y.P[i] + dt / 6.0 * (k1.P[i] + 2.0 * k2.P[i] + 2.0 * k3.P[i] + k4.P[i]);
  }
  for (int r = 0; r < 4 * d; ++r)
    for (int i = 0; i < d; ++i) {
      out.Qa[r][i] = y.Qa[r][i] + dt / 6.0 * (k1.Qa[r][i] + 2.0 * k2.Qa[r][i] + 2.0 * k3.Qa[r][i] + k4.Qa[r][i]);
      out.Pa[r][i] = y.Pa[r][i] + dt / 6.0 * (k1.Pa[r][i] + 2.0 * k2.Pa[r][i] + 2.0 * k3.Pa[r][i] + k4.Pa[r][i]);
    }
  out.a = y.a + dt / 6.0 * (k1.a + 2.0 * k2.a + 2.0 * k3.a + k4.a);
  out.S = y.S + dt / 6.0 * (k1.S + 2.0 * k2.S + 2.0 * k3.S + k4.S);
  for (int k = 0; k < d; ++k) {
    if (!g.periodic[k]) continue;
    double L = g.n[k] * g.h[k];
    double r = std::fmod(out.Q[k] - g.o[k], L);
    if (r < 0) r += L;
    out.Q[k] = g.o[k] + r;
  }
  y = out;
}

void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

// Output of a propagation: the values and, for R = Dual, their derivatives.
struct StateOut {
  double *Q, *P, *A, *B, *a, *S;
};

inline void put(double x, int64_t i, double* v, double*) { v[i] = x; }
inline void put(const Dual& x, int64_t i, double* v, double* dv) {
  v[i] = x.v;
  if (dv) dv[i] = x.d;
}
inline void put_c(const cplx& z, int64_t i, double* v, double*) {
  v[2 * i] = z.real();
  v[2 * i + 1] = z.imag();
}
inline void put_c(const DualC& z, int64_t i, double* v, double* dv) {
  v[2 * i] = z.v.real();
  v[2 * i + 1] = z.v.imag();
  if (dv) {
    dv[2 * i] = z.d.real();
    dv[2 * i + 1] = z.d.imag();
  }
}

template <class R>
int propagate_impl(const Grid& g, const Coefs& cf, int64_t nsteps, double dt, int64_t nG,
                   const int* sigma, const double* q, const double* p, const StateOut& out,
                   const StateOut& dout, int nthreads) {
  int d = g.dim;
  for (int64_t i = 0; i < nG; ++i) {
    double pn = 0.0;
    for (int k = 0; k < d; ++k) pn += p[i * d + k] * p[i * d + k];
    if (!(pn > 0.0)) return 2;
  }
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nG; ++i) {
    State<R> y;
    state_init(d, q + i * d, p + i * d, y);
    for (int64_t s = 0; s < nsteps; ++s) rk4_step(g, cf, sigma[i], y, dt);
    for (int k = 0; k < d; ++k) {
      put(y.Q[k], i * d + k, out.Q, dout.Q);
      put(y.P[k], i * d + k, out.P, dout.P);
      for (int l = 0; l < d; ++l) {
        put_c(y.A[k][l], (i * d + k) * d + l, out.A, dout.A);
        put_c(y.B[k][l], (i * d + k) * d + l, out.B, dout.B);
      }
    }
    put_c(y.a, i, out.a, dout.a);
    put(y.S, i, out.S, dout.S);
  }
  return 0;
}

// One term of Eq. recons at the point xp (without the factor W a psi (2 pi eps)^{-3d/2}
// e^{iS/eps}): the sum over the images inside the square window |x_k - Q_k| <= cut of
// exp(i P.(x - Q)/eps - |x - Q|^2/(2 eps)); periodic axes have L[k] > 0.
template <class R>
typename Num<R>::C window_term(int d, const double* L, double eps, double cut, const R* Qg,
                               const R* Pg, const double* xp) {
  typedef typename Num<R>::C C;
  const C I(0.0, 1.0);
  R img[3][5];
  int nimg[3];
  for (int k = 0; k < d; ++k) {
    nimg[k] = 0;
    R d0 = xp[k] - Qg[k];
    if (L[k] > 0.0) {
      for (int l = -2; l <= 2; ++l) {
        R dk = d0 + l * L[k];
        if (std::fabs(val(dk)) <= cut) img[k][nimg[k]++] = dk;
      }
    } else if (std::fabs(val(d0)) <= cut) {
      img[k][nimg[k]++] = d0;
    }
    if (nimg[k] == 0) return C(0.0, 0.0);
  }
  C sum(0.0, 0.0);
  int combos = 1;
  for (int k = 0; k < d; ++k) combos *= nimg[k];
  for (int cidx = 0; cidx < combos; ++cidx) {
    int rem = cidx;
    R phase(0.0), r2(0.0);
    for (int k = 0; k < d; ++k) {
      R dk = img[k][rem % nimg[k]];
      rem /= nimg[k];
      phase += Pg[k] * dk;
      r2 += dk * dk;
    }
    sum += exp(I * phase / eps - r2 / (2.0 * eps));
  }
  return sum;
}

inline void make_psi(const double* psi, const double*, int64_t i, cplx& out) {
  out = cplx(psi[2 * i], psi[2 * i + 1]);
}
inline void make_psi(const double* psi, const double* dpsi, int64_t i, DualC& out) {
  out = DualC(cplx(psi[2 * i], psi[2 * i + 1]),
              dpsi ? cplx(dpsi[2 * i], dpsi[2 * i + 1]) : cplx(0.0, 0.0));
}

template <class R>
int traces_impl(const Grid& g, const Coefs& cf, int64_t nsteps, double dt, int64_t record_every,
                int64_t nG, const int* sigma, const double* q, const double* p, const double* psi,
                const double* dpsi, double eps, double kappa, double W, int64_t nrx,
                const double* xr, double* out, double* dout, int nthreads) {
  typedef typename Num<R>::C C;
  int d = g.dim;
  double L[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) L[k] = g.periodic[k] ? g.n[k] * g.h[k] : 0.0;
  const int64_t nrec = nsteps / record_every + 1;
  const double cut = kappa * std::sqrt(eps);
  const double norm = std::pow(2.0 * kPi * eps, -1.5 * d);
  const C I(0.0, 1.0);
  int nt = nthreads > 0 ? nthreads : 1;
  std::vector<C> part((size_t)nt * nrec * nrx, C(0.0, 0.0));
  for (int64_t i = 0; i < nG; ++i) {
    double pn = 0.0;
    for (int k = 0; k < d; ++k) pn += p[i * d + k] * p[i * d + k];
    if (!(pn > 0.0)) return 2;
  }
  set_threads(nt);
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int64_t lo = nG * tid / nt, hi = nG * (tid + 1) / nt;
    C* acc = part.data() + (size_t)tid * nrec * nrx;
    for (int64_t i = lo; i < hi; ++i) {
      State<R> y;
      state_init(d, q + i * d, p + i * d, y);
      C ps;
      make_psi(psi, dpsi, i, ps);
      for (int64_t s = 0; s <= nsteps; ++s) {
        if (s % record_every == 0) {
          C pref = W * y.a * ps * norm * exp(I * y.S / eps);
          int64_t m = s / record_every;
          for (int64_t r = 0; r < nrx; ++r)
            acc[m * nrx + r] += pref * window_term(d, L, eps, cut, y.Q, y.P, xr + r * d);
        }
        if (s < nsteps) rk4_step(g, cf, sigma[i], y, dt);
      }
    }
  }
  for (int64_t e = 0; e < nrec * nrx; ++e) {
    C v(0.0, 0.0);
    for (int t = 0; t < nt; ++t) v += part[(size_t)t * nrec * nrx + e];
    put_c(v, e, out, dout);
  }
  return 0;
}

}  // namespace

extern "C" {

int orc_num_threads_available(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// c, grad c, Hessian of c and third derivatives at npts points x[npts][dim].
// Any of grad/hess/d3 may be NULL.
int orc_medium_eval(int dim, const int64_t* n, const double* h, const double* o, const int* periodic,
                    const double* C, int64_t npts, const double* x, double* c, double* grad,
                    double* hess, double* d3) {
  if (dim < 1 || dim > 3) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, nullptr};
  for (int64_t ip = 0; ip < npts; ++ip) {
    const double* xp = x + ip * dim;
    int d0[3] = {0, 0, 0};
    c[ip] = spline_value<double>(g, cf, xp, d0);
    for (int k = 0; k < dim; ++k) {
      if (grad) {
        int d1[3] = {0, 0, 0};
        d1[k] = 1;
        grad[ip * dim + k] = spline_value<double>(g, cf, xp, d1);
      }
      for (int l = 0; l < dim; ++l) {
        if (hess) {
          int d2[3] = {0, 0, 0};
          d2[k] += 1;
          d2[l] += 1;
          hess[(ip * dim + k) * dim + l] = spline_value<double>(g, cf, xp, d2);
        }
        if (d3)
          for (int m = 0; m < dim; ++m) {
            int dd[3] = {0, 0, 0};
            dd[k] += 1;
            dd[l] += 1;
            dd[m] += 1;
            d3[((ip * dim + k) * dim + l) * dim + m] = spline_value<double>(g, cf, xp, dd);
          }
      }
    }
  }
  return 0;
}

// H and its derivatives at one phase-space point (used by the tests to check
// the written-out derivatives against finite differences of H itself).
// out layout: H, dHdQ[d], dHdP[d], HQQ[d*d], HQP[d*d], HPP[d*d], HPQ[d*d].
int orc_hamiltonian(int dim, const int64_t* n, const double* h, const double* o, const int* periodic,
                    const double* C, int sigma, const double* Q, const double* P, double* out) {
  if (dim < 1 || dim > 3) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, nullptr};
  HamDerivs<double> r = hamiltonian<double>(g, cf, sigma, Q, P);
  int d = dim, at = 0;
  out[at++] = r.H;
  for (int k = 0; k < d; ++k) out[at++] = r.dHdQ[k];
  for (int k = 0; k < d; ++k) out[at++] = r.dHdP[k];
  for (int l = 0; l < d; ++l)
    for (int k = 0; k < d; ++k) out[at++] = r.HQQ[l][k];
  for (int l = 0; l < d; ++l)
    for (int k = 0; k < d; ++k) out[at++] = r.HQP[l][k];
  for (int l = 0; l < d; ++l)
    for (int k = 0; k < d; ++k) out[at++] = r.HPP[l][k];
  for (int l = 0; l < d; ++l)
    for (int k = 0; k < d; ++k) out[at++] = r.HPQ[l][k];
  return 0;
}

// Integrate nG Gaussians from t = 0 to t = nsteps*dt with RK4.
// Initial values: Q = q, P = p, A = I, B = -iI, a = 2^{d/2}, S = 0.
// Outputs (all [nG]-major): Q,P [nG][d]; A,B [nG][d][d][2] (re,im);
// a [nG][2]; S [nG]. |P| = 0 is rejected (returns 2).
int orc_propagate(int dim, const int64_t* n, const double* h, const double* o, const int* periodic,
                  const double* C, int64_t nsteps, double dt, int64_t nG, const int* sigma,
                  const double* q, const double* p, double* Qout, double* Pout, double* Aout,
                  double* Bout, double* aout, double* Sout, int nthreads) {
  if (dim < 1 || dim > 3) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, nullptr};
  const StateOut out = {Qout, Pout, Aout, Bout, aout, Sout};
  const StateOut none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  return propagate_impl<double>(g, cf, nsteps, dt, nG, sigma, q, p, out, none, nthreads);
}

// Tangent-linear propagation: orc_propagate of the coefficients C + e V to first order in
// e. The values (Qout .. Sout) equal orc_propagate's; dQ .. dS (same layouts) are their
// derivatives along V, d/de at e = 0, from the dual-number evaluation of the same RK4.
int orc_propagate_tangent(int dim, const int64_t* n, const double* h, const double* o,
                          const int* periodic, const double* C, const double* V, int64_t nsteps,
                          double dt, int64_t nG, const int* sigma, const double* q,
                          const double* p, double* Qout, double* Pout, double* Aout,
                          double* Bout, double* aout, double* Sout, double* dQ, double* dP,
                          double* dA, double* dB, double* da, double* dS, int nthreads) {
  if (dim < 1 || dim > 3) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, V};
  const StateOut out = {Qout, Pout, Aout, Bout, aout, Sout};
  const StateOut dout = {dQ, dP, dA, dB, da, dS};
  return propagate_impl<Dual>(g, cf, nsteps, dt, nG, sigma, q, p, out, dout, nthreads);
}

// orc_propagate with d_z Q, d_z P from divided differences (offsets dq[d], dp[d] > 0)
// instead of the dynamic ray equations; same outputs, A = d_z Q and B = d_z P being the
// central differences at the final time.
int orc_propagate_dd(int dim, const int64_t* n, const double* h, const double* o,
                     const int* periodic, const double* C, int64_t nsteps, double dt, int64_t nG,
                     const int* sigma, const double* q, const double* p, const double* dq,
                     const double* dp, double* Qout, double* Pout, double* Aout, double* Bout,
                     double* aout, double* Sout, int nthreads) {
  if (dim < 1 || dim > 3) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  int d = dim;
  for (int k = 0; k < d; ++k)
    if (!(dq[k] > 0.0) || !(dp[k] > 0.0)) return 3;
  for (int64_t i = 0; i < nG; ++i) {
    double pn = 0.0;
    for (int k = 0; k < d; ++k) pn += p[i * d + k] * p[i * d + k];
    if (!(pn > 0.0)) return 2;
  }
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nG; ++i) {
    DDState y;
    std::memset(&y, 0, sizeof(DDState));
    for (int k = 0; k < d; ++k) {
      y.Q[k] = q[i * d + k];
      y.P[k] = p[i * d + k];
    }
    for (int j = 0; j < d; ++j)
      for (int m = 0; m < 4; ++m) {
        int r = 4 * j + m;
        for (int k = 0; k < d; ++k) {
          y.Qa[r][k] = y.Q[k];
          y.Pa[r][k] = y.P[k];
        }
        if (m == 0) y.Qa[r][j] += dq[j];
        if (m == 1) y.Qa[r][j] -= dq[j];
        if (m == 2) y.Pa[r][j] += dp[j];
        if (m == 3) y.Pa[r][j] -= dp[j];
      }
    y.a = cplx(std::pow(2.0, 0.5 * d), 0.0);
    y.S = 0.0;
    for (int64_t s = 0; s < nsteps; ++s) dd_rk4_step(g, C, sigma[i], dq, dp, y, dt);
    for (int k = 0; k < d; ++k) {
      Qout[i * d + k] = y.Q[k];
      Pout[i * d + k] = y.P[k];
    }
    // A = d_z Q = Dq Q - i Dp Q, B = d_z P = Dq P - i Dp P
    for (int j = 0; j < d; ++j)
      for (int k = 0; k < d; ++k) {
        double DqQ = (y.Qa[4 * j][k] - y.Qa[4 * j + 1][k]) / (2.0 * dq[j]);
        double DqP = (y.Pa[4 * j][k] - y.Pa[4 * j + 1][k]) / (2.0 * dq[j]);
        double DpQ = (y.Qa[4 * j + 2][k] - y.Qa[4 * j + 3][k]) / (2.0 * dp[j]);
        double DpP = (y.Pa[4 * j + 2][k] - y.Pa[4 * j + 3][k]) / (2.0 * dp[j]);
        Aout[((i * d + j) * d + k) * 2 + 0] = DqQ;
        Aout[((i * d + j) * d + k) * 2 + 1] = -DpQ;
        Bout[((i * d + j) * d + k) * 2 + 0] = DqP;
        Bout[((i * d + j) * d + k) * 2 + 1] = -DpP;
      }
    aout[2 * i + 0] = y.a.real();
    aout[2 * i + 1] = y.a.imag();
    Sout[i] = y.S;
  }
  return 0;
}

// Reconstruction sum (Eq. recons) at npts points x[npts][dim]:
//   u(x) = sum_g W a_g psi_g (2 pi eps)^{-3d/2} e^{i S_g/eps}
//            e^{ i P_g.(x-Q_g)/eps - |x-Q_g|^2/(2 eps) }
// restricted to the square window |x_k - Q_k| <= kappa sqrt(eps) on every
// axis; on periodic axes (period L[k] > 0) every image x - Q + l L with
// |l| <= 2 inside the window contributes. Gaussians of both branches are
// passed together (the branch only mattered for the rays).
// a, psi: [nG][2] (re,im). Output ure, uim: [npts].
int orc_reconstruct(int dim, const double* L, double eps, double kappa, double W, int64_t nG,
                    const double* Q, const double* P, const double* a, const double* psi,
                    const double* S, int64_t npts, const double* x, double* ure, double* uim,
                    int nthreads) {
  if (dim < 1 || dim > 3) return 1;
  int d = dim;
  double cut = kappa * std::sqrt(eps);
  double norm = std::pow(2.0 * kPi * eps, -1.5 * d);
  const cplx I(0.0, 1.0);
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t ip = 0; ip < npts; ++ip) {
    const double* xp = x + ip * d;
    cplx u = 0.0;
    for (int64_t gi = 0; gi < nG; ++gi) {
      // images inside the window, per axis
      double img[3][5];
      int nimg[3];
      bool any = true;
      for (int k = 0; k < d; ++k) {
        nimg[k] = 0;
        double d0 = xp[k] - Q[gi * d + k];
        if (L[k] > 0.0) {
          for (int l = -2; l <= 2; ++l) {
            double dk = d0 + l * L[k];
            if (std::fabs(dk) <= cut) img[k][nimg[k]++] = dk;
          }
        } else if (std::fabs(d0) <= cut) {
          img[k][nimg[k]++] = d0;
        }
        if (nimg[k] == 0) any = false;
      }
      if (!any) continue;
      cplx sum = 0.0;
      int combos = 1;
      for (int k = 0; k < d; ++k) combos *= nimg[k];
      for (int cidx = 0; cidx < combos; ++cidx) {
        int rem = cidx;
        double phase = 0.0, r2 = 0.0;
        for (int k = 0; k < d; ++k) {
          double dk = img[k][rem % nimg[k]];
          rem /= nimg[k];
          phase += P[gi * d + k] * dk;
          r2 += dk * dk;
        }
        sum += std::exp(I * phase / eps - r2 / (2.0 * eps));
      }
      cplx ag(a[2 * gi], a[2 * gi + 1]);
      cplx pg(psi[2 * gi], psi[2 * gi + 1]);
      u += W * ag * pg * norm * std::exp(I * S[gi] / eps) * sum;
    }
    ure[ip] = u.real();
    uim[ip] = u.imag();
  }
  return 0;
}

// Brute-force FBI (Eq. psi discretised on the box): for each requested
// (q, p) pair,
//   psi(q,p) = prod_k h_k * sum_{j in box} f(q + r_j) w(r_j) e^{-i p.r_j/eps},
// r_{j,k} = (j_k - nb_k/2) h_k, w = prod_k w_k, w_k(r) = e^{-r^2/(2 eps)} on open
// axes and sum_{|l|<=2} e^{-(r + l L_k)^2/(2 eps)} on periodic ones; samples
// outside an open axis are zero, periodic ones wrap. q is given by its
// grid index qi[npairs][dim], p by its value pv[npairs][dim].
int orc_fbi_direct(int dim, const int64_t* n, const double* h, const int* periodic,
                   const double* f, double eps, const int64_t* nb, int64_t npairs,
                   const int64_t* qi, const double* pv, double* out /*[npairs][2]*/) {
  if (dim < 1 || dim > 3) return 1;
  int d = dim;
  const cplx I(0.0, 1.0);
  for (int64_t ip = 0; ip < npairs; ++ip) {
    int64_t total = 1;
    for (int k = 0; k < d; ++k) total *= nb[k];
    cplx acc = 0.0;
    for (int64_t t = 0; t < total; ++t) {
      int64_t rem = t;
      int64_t jj[3];
      for (int k = d - 1; k >= 0; --k) {
        jj[k] = rem % nb[k];
        rem /= nb[k];
      }
      bool inside = true;
      int64_t flat = 0;
      double w = 1.0, phase = 0.0;
      for (int k = 0; k < d; ++k) {
        double r = (double)(jj[k] - nb[k] / 2) * h[k];
        int64_t i = qi[ip * d + k] + jj[k] - nb[k] / 2;
        if (periodic[k]) {
          i %= n[k];
          if (i < 0) i += n[k];
          double Lk = n[k] * h[k], wk = 0.0;
          for (int l = -2; l <= 2; ++l) wk += std::exp(-(r + l * Lk) * (r + l * Lk) / (2.0 * eps));
          w *= wk;
        } else {
          if (i < 0 || i >= n[k]) inside = false;
          w *= std::exp(-r * r / (2.0 * eps));
        }
        flat = flat * n[k] + (inside ? i : 0);
        phase += pv[ip * d + k] * r;
      }
      if (!inside) continue;
      acc += f[flat] * w * std::exp(-I * phase / eps);
    }
    double hv = 1.0;
    for (int k = 0; k < d; ++k) hv *= h[k];
    out[2 * ip] = (hv * acc).real();
    out[2 * ip + 1] = (hv * acc).imag();
  }
  return 0;
}

// Traces: the field of Eq. recons at nrx receiver points x[nrx][dim] at the record
// times t_m = m * record_every * dt, m = 0 .. nsteps/record_every, with every Gaussian
// propagated by RK4 as in orc_propagate. out: [nrec][nrx][2] (re, im). The sum over
// Gaussians is split over nthreads fixed blocks and added up in block order.
int orc_traces(int dim, const int64_t* n, const double* h, const double* o, const int* periodic,
               const double* C, int64_t nsteps, double dt, int64_t record_every, int64_t nG,
               const int* sigma, const double* q, const double* p, const double* psi,
               double eps, double kappa, double W, int64_t nrx, const double* xr, double* out,
               int nthreads) {
  if (dim < 1 || dim > 3 || record_every < 1 || nsteps % record_every != 0) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, nullptr};
  return traces_impl<double>(g, cf, nsteps, dt, record_every, nG, sigma, q, p, psi, nullptr,
                             eps, kappa, W, nrx, xr, out, nullptr, nthreads);
}

// Tangent-linear traces: orc_traces for the coefficients C + e V and the weights
// psi + e dpsi, to first order in e (the set of Gaussians and their (q, p) held fixed).
// out equals orc_traces; dout ([nrec][nrx][2]) is d/de at e = 0 through the rays, the
// amplitude and the action (dual-number RK4) and through psi. The window cut
// |x_k - Q_k| <= kappa sqrt(eps) is decided on the value of Q.
int orc_traces_tangent(int dim, const int64_t* n, const double* h, const double* o,
                       const int* periodic, const double* C, const double* V, int64_t nsteps,
                       double dt, int64_t record_every, int64_t nG, const int* sigma,
                       const double* q, const double* p, const double* psi, const double* dpsi,
                       double eps, double kappa, double W, int64_t nrx, const double* xr,
                       double* out, double* dout, int nthreads) {
  if (dim < 1 || dim > 3 || record_every < 1 || nsteps % record_every != 0) return 1;
  Grid g = make_grid(dim, n, h, o, periodic);
  const Coefs cf = {C, V};
  return traces_impl<Dual>(g, cf, nsteps, dt, record_every, nG, sigma, q, p, psi, dpsi, eps,
                           kappa, W, nrx, xr, out, dout, nthreads);
}

}  // extern "C"
