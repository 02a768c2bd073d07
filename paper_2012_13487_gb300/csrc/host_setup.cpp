// Host-side set-up in FP64: velocity sets, reference operators, mesh.
//
// Velocity sets (Sec. II.A.3, Table 1): Gauss-Hermite rules are found as the
// roots of the orthonormal probabilists' Hermite polynomial h_n (bracketed by a
// sign scan, refined by bisection and Newton), with Christoffel weights
// 1/(n h_{n-1}(x)^2).  Newton-Cotes rules (Sec. III.B) use composite trapezoid
// weights times the Maxwellian density, corrected by a quadratic-in-xi^2 factor
// so that the moments of order 0, 2, 4 are exact.
//
// Reference operators (Sec. II.B.1): warp & blend nodes (alpha = 0) and the
// orthonormal Proriol-Koornwinder-Dubiner basis give V, Vr, Vs; Dr = Vr V^-1,
// Ds = Vs V^-1, M = (V V^T)^-1, LIFT = V (V^T E) with E built from the 1-D face
// mass matrices.
//
// Mesh (Sec. III): Cartesian cells split along the lower-left/upper-right
// diagonal, where neighbours and face orientation follow from the cell
// structure, or a general conforming triangulation of a rectangle given by its
// vertices and triangles, where neighbours are matched by shared edges.
#include "host_setup.h"

#include <algorithm>
#include <cmath>

namespace fedbm {
namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- linear algebra
using Mat = std::vector<double>;  // row-major square or rectangular

bool invert(int n, const Mat& a, Mat& inv) {
  Mat m = a;
  inv.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[size_t(r) * n + c]) > std::fabs(m[size_t(piv) * n + c])) piv = r;
    if (std::fabs(m[size_t(piv) * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(m[size_t(c) * n + j], m[size_t(piv) * n + j]);
        std::swap(inv[size_t(c) * n + j], inv[size_t(piv) * n + j]);
      }
    const double d = 1.0 / m[size_t(c) * n + c];
    for (int j = 0; j < n; ++j) {
      m[size_t(c) * n + j] *= d;
      inv[size_t(c) * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = m[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        m[size_t(r) * n + j] -= f * m[size_t(c) * n + j];
        inv[size_t(r) * n + j] -= f * inv[size_t(c) * n + j];
      }
    }
  }
  return true;
}

// C[n x m] = A[n x k] * B[k x m]
Mat matmul(int n, int k, int m, const Mat& A, const Mat& B) {
  Mat C(size_t(n) * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[size_t(i) * k + l];
      for (int j = 0; j < m; ++j) C[size_t(i) * m + j] += a * B[size_t(l) * m + j];
    }
  return C;
}

Mat transpose(int n, int m, const Mat& A) {
  Mat T(size_t(m) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[size_t(j) * n + i] = A[size_t(i) * m + j];
  return T;
}

// ---------------------------------------------------------------- Gauss-Hermite
// Orthonormal probabilists' Hermite recurrence:
// h_{k+1}(x) = (x h_k(x) - sqrt(k) h_{k-1}(x)) / sqrt(k+1), h_0 = 1.
void hermite_pair(int n, double x, double& hn, double& hnm1) {
  double prev = 0.0, cur = 1.0;
  for (int k = 0; k < n; ++k) {
    const double next = (x * cur - std::sqrt(double(k)) * prev) / std::sqrt(double(k + 1));
    prev = cur;
    cur = next;
  }
  hn = cur;
  hnm1 = prev;
}

bool gauss_hermite(int n, std::vector<double>& x, std::vector<double>& w) {
  x.clear();
  w.clear();
  if (n == 1) {
    x.push_back(0.0);
    w.push_back(1.0);
    return true;
  }
  const double B = std::sqrt(4.0 * n + 2.0) + 1.0;
  const int nscan = 40001;  // odd: the symmetric root x = 0 falls inside a cell
  double hn, hm, xa = -B;
  hermite_pair(n, xa, hn, hm);
  double fa = hn;
  for (int j = 1; j <= nscan; ++j) {
    const double xb = -B + 2.0 * B * j / nscan;
    hermite_pair(n, xb, hn, hm);
    const double fb = hn;
    if (fa != 0.0 && (fb == 0.0 || (fa < 0) != (fb < 0))) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
        const double mid = 0.5 * (lo + hi);
        double hmid, hx;
        hermite_pair(n, mid, hmid, hx);
        if ((hmid < 0) == (flo < 0)) {
          lo = mid;
          flo = hmid;
        } else {
          hi = mid;
        }
      }
      double r = 0.5 * (lo + hi);
      for (int it = 0; it < 3; ++it) {
        double h, h1;
        hermite_pair(n, r, h, h1);
        r -= h / (std::sqrt(double(n)) * h1);  // h_n' = sqrt(n) h_{n-1}
      }
      x.push_back(r);
    }
    xa = xb;
    fa = fb;
  }
  if (int(x.size()) != n) return false;
  std::sort(x.begin(), x.end());
  for (int j = 0; j < n / 2; ++j) {  // exact mirror symmetry
    const double a = 0.5 * (x[n - 1 - j] - x[j]);
    x[j] = -a;
    x[n - 1 - j] = a;
  }
  if (n % 2) x[n / 2] = 0.0;
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    double h, h1;
    hermite_pair(n, x[j], h, h1);
    w[j] = 1.0 / (n * h1 * h1);
  }
  for (int j = 0; j < n / 2; ++j) {
    const double a = 0.5 * (w[j] + w[n - 1 - j]);
    w[j] = w[n - 1 - j] = a;
  }
  return true;
}

bool newton_cotes(int n, double extent, double unit, std::vector<double>& x, std::vector<double>& w) {
  if (n < 2) return false;
  x.resize(n);
  w.resize(n);
  const double h = unit * 2.0 * extent / (n - 1);
  for (int j = 0; j < n; ++j) {
    x[j] = unit * (-extent + 2.0 * extent * j / (n - 1));
    const double trap = (j == 0 || j == n - 1) ? 0.5 * h : h;
    w[j] = trap * std::exp(-0.5 * x[j] * x[j]) / std::sqrt(2.0 * kPi);
  }
  for (int j = 0; j < n / 2; ++j) x[n - 1 - j] = -x[j];
  if (n % 2) x[n / 2] = 0.0;
  // weights times (a + b xi^2 + c xi^4) reproduce the moments 1, 1, 3
  double A[3][4];
  const double target[3] = {1.0, 1.0, 3.0};
  for (int m = 0; m < 3; ++m) {
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int j = 0; j < n; ++j) s += w[j] * std::pow(x[j], 2 * m + 2 * c);
      A[m][c] = s;
    }
    A[m][3] = target[m];
  }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    for (int j = 0; j < 4; ++j) std::swap(A[c][j], A[piv][j]);
    if (std::fabs(A[c][c]) < 1e-300) return false;
    for (int r = 0; r < 3; ++r) {
      if (r == c) continue;
      const double f = A[r][c] / A[c][c];
      for (int j = 0; j < 4; ++j) A[r][j] -= f * A[c][j];
    }
  }
  const double a = A[0][3] / A[0][0], b = A[1][3] / A[1][1], c = A[2][3] / A[2][2];
  for (int j = 0; j < n; ++j) {
    const double x2 = x[j] * x[j];
    w[j] *= a + b * x2 + c * x2 * x2;
  }
  return true;
}

// ---------------------------------------------------------------- 1-D polynomials
// Legendre P_n and its first two derivatives at x (|x| < 1 for derivatives).
void legendre(int n, double x, double& P, double& dP, double& d2P) {
  double pm = 1.0, pc = x;
  if (n == 0) {
    P = 1.0;
    dP = d2P = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
    pm = pc;
    pc = pn;
  }
  P = pc;
  dP = n * (x * pc - pm) / (x * x - 1.0);
  d2P = (2.0 * x * dP - n * (n + 1.0) * P) / (1.0 - x * x);
}

std::vector<double> gll_points(int p) {
  std::vector<double> g(p + 1);
  if (p == 0) {
    g[0] = 0.0;
    return g;
  }
  g[0] = -1.0;
  g[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double x = -std::cos(kPi * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(p, x, P, dP, d2P);
      const double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    g[j] = x;
  }
  for (int j = 0; j <= p / 2; ++j) {
    const double a = 0.5 * (g[p - j] - g[j]);
    g[j] = -a;
    g[p - j] = a;
  }
  if (p % 2 == 0) g[p / 2] = 0.0;
  return g;
}

// Normalised Jacobi polynomial P_n^(al,be)(x) (orthonormal on [-1,1] with
// weight (1-x)^al (1+x)^be).
double jacobi_normalised(int n, double al, double be, double x) {
  const double g0 = std::pow(2.0, -al - be - 1.0) * std::tgamma(al + be + 2.0) /
                    (std::tgamma(al + 1.0) * std::tgamma(be + 1.0));
  double p0 = std::sqrt(g0);
  if (n == 0) return p0;
  double p1 = 0.5 * ((al + be + 2.0) * x + (al - be)) * p0 * std::sqrt((al + be + 3.0) / ((al + 1.0) * (be + 1.0)));
  if (n == 1) return p1;
  double aold = 2.0 / (2.0 + al + be) * std::sqrt((al + 1.0) * (be + 1.0) / (al + be + 3.0));
  for (int i = 1; i < n; ++i) {
    const double h1 = 2.0 * i + al + be;
    const double anew = 2.0 / (h1 + 2.0) *
                        std::sqrt((i + 1.0) * (i + 1.0 + al + be) * (i + 1.0 + al) * (i + 1.0 + be) /
                                  ((h1 + 1.0) * (h1 + 3.0)));
    const double bnew = -(al * al - be * be) / (h1 * (h1 + 2.0));
    const double p2 = (-aold * p0 + (x - bnew) * p1) / anew;
    aold = anew;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double jacobi_normalised_deriv(int n, double al, double be, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + al + be + 1.0)) * jacobi_normalised(n - 1, al + 1.0, be + 1.0, x);
}

// ---------------------------------------------------------------- nodes
double warp_factor(int p, const std::vector<double>& gll, double r) {
  double warp = 0.0;
  for (int j = 0; j <= p; ++j) {
    const double rj = -1.0 + 2.0 * j / p;
    double l = 1.0;
    for (int m = 0; m <= p; ++m) {
      if (m == j) continue;
      const double rm = -1.0 + 2.0 * m / p;
      l *= (r - rm) / (rj - rm);
    }
    warp += (gll[j] - rj) * l;
  }
  if (std::fabs(r) < 1.0 - 1e-10) return warp / (1.0 - r * r);
  return 0.0;
}

void warp_blend_nodes(int p, std::vector<double>& r, std::vector<double>& s) {
  const int Np = num_nodes(p);
  r.assign(Np, 0.0);
  s.assign(Np, 0.0);
  if (p == 0) {
    r[0] = s[0] = -1.0 / 3.0;
    return;
  }
  const std::vector<double> gll = gll_points(p);
  const double sq3 = std::sqrt(3.0);
  int idx = 0;
  for (int i = 0; i <= p; ++i) {
    for (int j = 0; j <= p - i; ++j, ++idx) {
      const double L1 = double(i) / p, L3 = double(j) / p, L2 = 1.0 - L1 - L3;
      double X = -L2 + L3;
      double Y = (-L2 - L3 + 2.0 * L1) / sq3;
      const double w1 = 4.0 * L2 * L3 * warp_factor(p, gll, L3 - L2);
      const double w2 = 4.0 * L1 * L3 * warp_factor(p, gll, L1 - L3);
      const double w3 = 4.0 * L1 * L2 * warp_factor(p, gll, L2 - L1);
      X += w1 + std::cos(2.0 * kPi / 3.0) * w2 + std::cos(4.0 * kPi / 3.0) * w3;
      Y += std::sin(2.0 * kPi / 3.0) * w2 + std::sin(4.0 * kPi / 3.0) * w3;
      const double b1 = (sq3 * Y + 1.0) / 3.0;
      const double b2 = (-3.0 * X - sq3 * Y + 2.0) / 6.0;
      const double b3 = (3.0 * X - sq3 * Y + 2.0) / 6.0;
      r[idx] = -b2 + b3 - b1;
      s[idx] = -b2 - b3 + b1;
    }
  }
}

// Orthonormal simplex polynomial (i, j) and its gradient at (r, s).
void simplex_mode(int i, int j, double r, double s, double& val, double& dr, double& ds) {
  const double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  const double b = s;
  const double fa = jacobi_normalised(i, 0, 0, a), dfa = jacobi_normalised_deriv(i, 0, 0, a);
  const double gb = jacobi_normalised(j, 2.0 * i + 1.0, 0, b);
  const double dgb = jacobi_normalised_deriv(j, 2.0 * i + 1.0, 0, b);
  const double hb = 0.5 * (1.0 - b);
  val = std::sqrt(2.0) * fa * gb * std::pow(1.0 - b, i);
  double dmr = dfa * gb, dms = dfa * gb * 0.5 * (1.0 + a);
  if (i > 0) {
    dmr *= std::pow(hb, i - 1);
    dms *= std::pow(hb, i - 1);
  }
  double t = dgb * std::pow(hb, i);
  if (i > 0) t -= 0.5 * i * gb * std::pow(hb, i - 1);
  dms += fa * t;
  const double sc = std::pow(2.0, i + 0.5);
  dr = dmr * sc;
  ds = dms * sc;
}

}  // namespace

// ---------------------------------------------------------------- public API
double equilibrium(double w, double ex, double ey, double rho, double ux, double uy, int eq_order) {
  const double eu = ex * ux + ey * uy, uu = ux * ux + uy * uy;
  double poly = 1.0 + eu + 0.5 * (eu * eu - uu);
  if (eq_order == 3) poly += eu * (eu * eu / 6.0 - 0.5 * uu);
  return w * rho * poly;
}

bool build_velocity_set(const fedbm_velset_desc& d, VelocitySet& out, std::string& err) {
  std::vector<double> x, w;
  if (d.eq_order != 2 && d.eq_order != 3) {
    err = "eq_order must be 2 or 3";
    return false;
  }
  if (d.kind == FEDBM_VELSET_GH) {
    if (d.n < 1 || d.n > 40) {
      err = "GH velocity set: n must be in 1..40";
      return false;
    }
    if (!gauss_hermite(d.n, x, w)) {
      err = "GH root finding failed";
      return false;
    }
  } else if (d.kind == FEDBM_VELSET_NC) {
    if (d.n < 2 || d.n > 64) {
      err = "NC velocity set: n must be in 2..64";
      return false;
    }
    const double ext = d.nc_extent > 0 ? d.nc_extent : 4.0;
    const double unit = d.nc_sqrt2 ? std::sqrt(2.0) : 1.0;
    if (!newton_cotes(d.n, ext, unit, x, w)) {
      err = "NC weight correction failed";
      return false;
    }
  } else {
    err = "unknown velocity set kind";
    return false;
  }
  const int n = d.n;
  out.n = n;
  out.Q = n * n;
  out.ex.resize(out.Q);
  out.ey.resize(out.Q);
  out.w.resize(out.Q);
  for (int ix = 0; ix < n; ++ix)
    for (int iy = 0; iy < n; ++iy) {
      const int i = ix * n + iy;
      out.ex[i] = x[ix];
      out.ey[i] = x[iy];
      out.w[i] = w[ix] * w[iy];
    }
  return true;
}

bool build_ref_ops(int p, RefOps& o, std::string& err) {
  if (p < 0 || p > kMaxOrder) {
    err = "order must be in 0..6";
    return false;
  }
  const int Np = num_nodes(p), Nfp = p + 1;
  o.p = p;
  o.Np = Np;
  o.Nfp = Nfp;
  warp_blend_nodes(p, o.r, o.s);
  // face masks: row starts rs(i) = i(p+1) - i(i-1)/2
  o.fmask.assign(3 * Nfp, 0);
  for (int a = 0; a < Nfp; ++a) {
    const int rs = a * (p + 1) - a * (a - 1) / 2;
    o.fmask[0 * Nfp + a] = a;
    o.fmask[1 * Nfp + a] = rs + (p - a);
    o.fmask[2 * Nfp + a] = rs;
  }
  Mat V(size_t(Np) * Np), Vr(V.size()), Vs(V.size());
  for (int n = 0; n < Np; ++n) {
    int col = 0;
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p - i; ++j, ++col) {
        double v, dr, ds;
        simplex_mode(i, j, o.r[n], o.s[n], v, dr, ds);
        V[size_t(n) * Np + col] = v;
        Vr[size_t(n) * Np + col] = dr;
        Vs[size_t(n) * Np + col] = ds;
      }
  }
  Mat Vinv;
  if (!invert(Np, V, Vinv)) {
    err = "singular Vandermonde matrix";
    return false;
  }
  o.Dr = matmul(Np, Np, Np, Vr, Vinv);
  o.Ds = matmul(Np, Np, Np, Vs, Vinv);
  const Mat VT = transpose(Np, Np, V);
  Mat MM;
  if (!invert(Np, matmul(Np, Np, Np, V, VT), MM)) {
    err = "singular V V^T";
    return false;
  }
  o.M = MM;
  // E: face mass matrices of the face nodes in their 1-D coordinate
  Mat E(size_t(Np) * 3 * Nfp, 0.0);
  for (int f = 0; f < 3; ++f) {
    Mat V1(size_t(Nfp) * Nfp);
    for (int a = 0; a < Nfp; ++a) {
      const int node = o.fmask[f * Nfp + a];
      const double t = (f == 0) ? o.r[node] : o.s[node];
      for (int m = 0; m < Nfp; ++m) V1[size_t(a) * Nfp + m] = jacobi_normalised(m, 0, 0, t);
    }
    Mat M1;
    if (!invert(Nfp, matmul(Nfp, Nfp, Nfp, V1, transpose(Nfp, Nfp, V1)), M1)) {
      err = "singular face Vandermonde";
      return false;
    }
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b)
        E[size_t(o.fmask[f * Nfp + a]) * 3 * Nfp + f * Nfp + b] = M1[size_t(a) * Nfp + b];
  }
  o.LIFT = matmul(Np, Np, 3 * Nfp, V, matmul(Np, Np, 3 * Nfp, VT, E));
  return true;
}

namespace {

// Affine geometric factors, outward unit normals and Fscale = |face| / (2 J)
// of element k from its counter-clockwise vertices (Sec. II.B.1; J is the
// Jacobian of the map from the reference triangle of area 2).
void element_geometry(Mesh& m, int64_t k, double& rin_min) {
  const double* X = &m.vx[k * 3];
  const double* Y = &m.vy[k * 3];
  const double xr = 0.5 * (X[1] - X[0]), xs = 0.5 * (X[2] - X[0]);
  const double yr = 0.5 * (Y[1] - Y[0]), ys = 0.5 * (Y[2] - Y[0]);
  const double J = xr * ys - xs * yr;
  double* g = &m.geo[k * kGeoStride];
  g[0] = ys / J;   // rx
  g[1] = -yr / J;  // sx
  g[2] = -xs / J;  // ry
  g[3] = xr / J;   // sy
  double perim = 0.0;
  for (int f = 0; f < 3; ++f) {
    const int a = f, b = (f + 1) % 3;
    const double dx = X[b] - X[a], dy = Y[b] - Y[a];
    const double len = std::sqrt(dx * dx + dy * dy);
    perim += len;
    g[4 + 3 * f + 0] = dy / len;
    g[4 + 3 * f + 1] = -dx / len;
    g[4 + 3 * f + 2] = 0.5 * len / J;
  }
  g[13] = J;
  rin_min = std::min(rin_min, 2.0 * (2.0 * J) / perim);  // area = 2J
}

// Face node order runs with the counter-clockwise direction on faces 0 and 1
// and against it on face 2; two counter-clockwise elements sharing an edge
// traverse it in opposite directions, so their face nodes are listed in
// opposite order exactly when both or neither of the two faces is face 2.
int face_rev(int f, int g) { return int((f == 2) == (g == 2)); }

bool check_sides(const fedbm_mesh_desc& d, std::string& err) {
  for (int sd = 0; sd < 4; ++sd) {
    if (d.bc[sd] < FEDBM_BC_PERIODIC || d.bc[sd] > FEDBM_BC_WALL_EQ) {
      err = "mesh: unknown boundary kind";
      return false;
    }
  }
  const bool perx = d.bc[1] == FEDBM_BC_PERIODIC, pery = d.bc[0] == FEDBM_BC_PERIODIC;
  if (perx != (d.bc[3] == FEDBM_BC_PERIODIC) || pery != (d.bc[2] == FEDBM_BC_PERIODIC)) {
    err = "mesh: periodic sides must come in opposite pairs";
    return false;
  }
  for (int sd = 0; sd < 4; ++sd) {
    if (d.bc[sd] == FEDBM_BC_PERIODIC) continue;
    const double un = (sd == 0 || sd == 2) ? d.wall_uy[sd] : d.wall_ux[sd];
    if (un != 0.0) {
      err = "mesh: wall velocities must be tangential to the wall";
      return false;
    }
  }
  return true;
}

// General conforming triangulation of the rectangle [0, lx] x [0, ly]
// (Sec. III.B runs the cavity on unstructured meshes).  Neighbours are found
// by matching the vertex pairs of the element edges; boundary edges are given
// the side of the rectangle they lie on, and periodic sides are paired by the
// coordinates of their end points.
bool build_unstructured(const fedbm_mesh_desc& d, Mesh& m, std::string& err) {
  if (!d.vert_xy || !d.tri || d.nvert < 3 || d.ntri < 1 || d.ntri > (int64_t(1) << 27)) {
    err = "mesh: an unstructured mesh needs nvert >= 3, 1 <= ntri < 2^27 and both arrays";
    return false;
  }
  const int64_t K = d.ntri;
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int v = 0; v < d.nvert; ++v) {
    const double x = d.vert_xy[2 * v], y = d.vert_xy[2 * v + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) {
      err = "mesh: vertex coordinates must be finite";
      return false;
    }
    xmin = std::min(xmin, x);
    xmax = std::max(xmax, x);
    ymin = std::min(ymin, y);
    ymax = std::max(ymax, y);
  }
  const double ext = std::max(xmax - xmin, ymax - ymin);
  const double tol = 1e-10 * ext;
  if (!(ext > 0) || std::fabs(xmin) > tol || std::fabs(ymin) > tol) {
    err = "mesh: the vertices must span a rectangle [0, lx] x [0, ly]";
    return false;
  }
  m.nx = m.ny = 0;
  m.K = K;
  m.lx = xmax;
  m.ly = ymax;
  m.vx.assign(size_t(K) * 3, 0.0);
  m.vy.assign(size_t(K) * 3, 0.0);
  m.nbr.assign(size_t(K) * 3, 0);
  m.geo.assign(size_t(K) * kGeoStride, 0.0);
  double rin_min = 1e300;
  struct Edge {
    int64_t lo, hi, k;
    int f;
  };
  std::vector<Edge> edges;
  edges.reserve(size_t(K) * 3);
  for (int64_t k = 0; k < K; ++k) {
    int32_t v[3];
    for (int j = 0; j < 3; ++j) {
      v[j] = d.tri[k * 3 + j];
      if (v[j] < 0 || v[j] >= d.nvert) {
        err = "mesh: triangle " + std::to_string(k) + " has a vertex index out of range";
        return false;
      }
      m.vx[k * 3 + j] = d.vert_xy[2 * v[j]];
      m.vy[k * 3 + j] = d.vert_xy[2 * v[j] + 1];
    }
    const double* X = &m.vx[k * 3];
    const double* Y = &m.vy[k * 3];
    const double area2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
    if (!(area2 > 1e-14 * ext * ext)) {
      err = "mesh: triangle " + std::to_string(k) + " is degenerate or not counter-clockwise";
      return false;
    }
    element_geometry(m, k, rin_min);
    for (int f = 0; f < 3; ++f) {
      const int64_t a = v[f], b = v[(f + 1) % 3];
      edges.push_back({std::min(a, b), std::max(a, b), k, f});
    }
  }
  std::sort(edges.begin(), edges.end(), [](const Edge& x, const Edge& y) {
    return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : (x.k != y.k ? x.k < y.k : x.f < y.f));
  });
  // boundary edges per side, keyed by the coordinate along the side of their
  // end points (sorted) for periodic pairing
  struct Bnd {
    double t0, t1;
    int64_t k;
    int f;
  };
  std::vector<Bnd> bnd[4];
  for (size_t e = 0; e < edges.size();) {
    size_t n = 1;
    while (e + n < edges.size() && edges[e + n].lo == edges[e].lo && edges[e + n].hi == edges[e].hi) ++n;
    if (n > 2) {
      err = "mesh: an edge is shared by more than two triangles";
      return false;
    }
    if (n == 2) {
      const Edge& A = edges[e];
      const Edge& B = edges[e + 1];
      if (d.tri[A.k * 3 + A.f] == d.tri[B.k * 3 + B.f]) {
        err = "mesh: two triangles traverse a shared edge in the same direction";
        return false;
      }
      m.nbr[A.k * 3 + A.f] = encode_face(B.k, B.f, face_rev(A.f, B.f));
      m.nbr[B.k * 3 + B.f] = encode_face(A.k, A.f, face_rev(B.f, A.f));
    } else {
      const Edge& A = edges[e];
      const double x0 = d.vert_xy[2 * A.lo], y0 = d.vert_xy[2 * A.lo + 1];
      const double x1 = d.vert_xy[2 * A.hi], y1 = d.vert_xy[2 * A.hi + 1];
      int side = -1;
      if (std::fabs(y0) <= tol && std::fabs(y1) <= tol) side = 0;
      else if (std::fabs(x0 - xmax) <= tol && std::fabs(x1 - xmax) <= tol) side = 1;
      else if (std::fabs(y0 - ymax) <= tol && std::fabs(y1 - ymax) <= tol) side = 2;
      else if (std::fabs(x0) <= tol && std::fabs(x1) <= tol) side = 3;
      if (side < 0) {
        err = "mesh: a boundary edge of triangle " + std::to_string(A.k) + " is not on a side of the rectangle";
        return false;
      }
      const double t0 = (side == 0 || side == 2) ? std::min(x0, x1) : std::min(y0, y1);
      const double t1 = (side == 0 || side == 2) ? std::max(x0, x1) : std::max(y0, y1);
      bnd[side].push_back({t0, t1, A.k, A.f});
      m.nbr[A.k * 3 + A.f] = -(side + 1);
    }
    e += n;
  }
  for (int sd = 0; sd < 2; ++sd) {  // pairs (0, 2) and (1, 3)
    const int op = sd + 2;
    if (d.bc[sd] != FEDBM_BC_PERIODIC) continue;
    auto by_t = [](const Bnd& x, const Bnd& y) { return x.t0 < y.t0; };
    std::sort(bnd[sd].begin(), bnd[sd].end(), by_t);
    std::sort(bnd[op].begin(), bnd[op].end(), by_t);
    if (bnd[sd].size() != bnd[op].size()) {
      err = "mesh: periodic sides do not have matching edges";
      return false;
    }
    for (size_t j = 0; j < bnd[sd].size(); ++j) {
      const Bnd& A = bnd[sd][j];
      const Bnd& B = bnd[op][j];
      if (std::fabs(A.t0 - B.t0) > tol || std::fabs(A.t1 - B.t1) > tol) {
        err = "mesh: periodic sides do not have matching edges";
        return false;
      }
      m.nbr[A.k * 3 + A.f] = encode_face(B.k, B.f, face_rev(A.f, B.f));
      m.nbr[B.k * 3 + B.f] = encode_face(A.k, A.f, face_rev(B.f, A.f));
    }
  }
  m.rin_min = rin_min;
  return true;
}

}  // namespace

bool build_mesh(const fedbm_mesh_desc& d, Mesh& m, std::string& err) {
  if (!check_sides(d, err)) return false;
  if (d.ntri > 0 || d.nvert > 0 || d.tri || d.vert_xy) return build_unstructured(d, m, err);
  if (d.nx < 1 || d.ny < 1 || int64_t(d.nx) * d.ny > (int64_t(1) << 26)) {
    err = "mesh: nx, ny must be >= 1 and 2*nx*ny < 2^27";
    return false;
  }
  const bool perx = d.bc[1] == FEDBM_BC_PERIODIC, pery = d.bc[0] == FEDBM_BC_PERIODIC;
  m.nx = d.nx;
  m.ny = d.ny;
  m.lx = d.lx > 0 ? d.lx : 1.0;
  m.ly = d.ly > 0 ? d.ly : 1.0;
  const int nx = d.nx, ny = d.ny;
  m.K = 2 * nx * ny;
  m.vx.assign(size_t(m.K) * 3, 0.0);
  m.vy.assign(size_t(m.K) * 3, 0.0);
  m.nbr.assign(size_t(m.K) * 3, 0);
  m.geo.assign(size_t(m.K) * kGeoStride, 0.0);
  const double hx = m.lx / nx, hy = m.ly / ny;
  auto rev = face_rev;
  auto elem = [nx](int ix, int iy, int t) { return int64_t(2) * (int64_t(iy) * nx + ix) + t; };
  double rin_min = 1e300;
  for (int iy = 0; iy < ny; ++iy) {
    for (int ix = 0; ix < nx; ++ix) {
      const double x0 = ix * hx, x1 = (ix + 1) * hx, y0 = iy * hy, y1 = (iy + 1) * hy;
      const double tri[2][3][2] = {{{x0, y0}, {x1, y0}, {x1, y1}}, {{x0, y0}, {x1, y1}, {x0, y1}}};
      for (int t = 0; t < 2; ++t) {
        const int64_t k = elem(ix, iy, t);
        for (int v = 0; v < 3; ++v) {
          m.vx[k * 3 + v] = tri[t][v][0];
          m.vy[k * 3 + v] = tri[t][v][1];
        }
        int32_t* nb = &m.nbr[k * 3];
        if (t == 0) {
          // face 0: bottom edge -> cell below, triangle 1, face 1
          if (iy > 0) nb[0] = encode_face(elem(ix, iy - 1, 1), 1, rev(0, 1));
          else nb[0] = pery ? encode_face(elem(ix, ny - 1, 1), 1, rev(0, 1)) : -(0 + 1);
          // face 1: right edge -> cell to the right, triangle 1, face 2
          if (ix < nx - 1) nb[1] = encode_face(elem(ix + 1, iy, 1), 2, rev(1, 2));
          else nb[1] = perx ? encode_face(elem(0, iy, 1), 2, rev(1, 2)) : -(1 + 1);
          // face 2: diagonal -> same cell, triangle 1, face 0
          nb[2] = encode_face(elem(ix, iy, 1), 0, rev(2, 0));
        } else {
          nb[0] = encode_face(elem(ix, iy, 0), 2, rev(0, 2));
          // face 1: top edge -> cell above, triangle 0, face 0
          if (iy < ny - 1) nb[1] = encode_face(elem(ix, iy + 1, 0), 0, rev(1, 0));
          else nb[1] = pery ? encode_face(elem(ix, 0, 0), 0, rev(1, 0)) : -(2 + 1);
          // face 2: left edge -> cell to the left, triangle 0, face 1
          if (ix > 0) nb[2] = encode_face(elem(ix - 1, iy, 0), 1, rev(2, 1));
          else nb[2] = perx ? encode_face(elem(nx - 1, iy, 0), 1, rev(2, 1)) : -(3 + 1);
        }
        element_geometry(m, k, rin_min);
      }
    }
  }
  m.rin_min = rin_min;
  return true;
}

void node_coordinates(const Mesh& m, const RefOps& o, std::vector<double>& x, std::vector<double>& y) {
  x.resize(size_t(m.K) * o.Np);
  y.resize(x.size());
  for (int64_t k = 0; k < m.K; ++k)
    for (int n = 0; n < o.Np; ++n) {
      const double r = o.r[n], s = o.s[n];
      const double l0 = -0.5 * (r + s), l1 = 0.5 * (1.0 + r), l2 = 0.5 * (1.0 + s);
      x[k * o.Np + n] = l0 * m.vx[k * 3] + l1 * m.vx[k * 3 + 1] + l2 * m.vx[k * 3 + 2];
      y[k * o.Np + n] = l0 * m.vy[k * 3] + l1 * m.vy[k * 3 + 1] + l2 * m.vy[k * 3 + 2];
    }
}

double time_step(const Mesh& m, const VelocitySet& v, int p, double cfl) {
  double emax = 0.0;
  for (int i = 0; i < v.Q; ++i) emax = std::max(emax, std::sqrt(v.ex[i] * v.ex[i] + v.ey[i] * v.ey[i]));
  return cfl * m.rin_min / (emax * (p + 1) * (p + 1));
}

}  // namespace fedbm
