// Host-side set-up: KL expansion, PC basis, coupling tables and Galerkin coarse stencils.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "sg_internal.h"

// ---------------------------------------------------------------------------
// Truncated KL expansion (Sec. 2.1, Eqs. truncated-KLE, exponential-covariance)
// of the separable covariance exp(-|x1-y1|/L - |x2-y2|/L) on the unit square.
// 1-D problem on (-a, a), a = 1/2, c = 1/L: even eigenfunctions cos(w y) with
// c = w tan(w a), odd ones sin(w y) with w = -c tan(w a); lambda = 2c/(w^2+c^2).
// Roots are bracketed between the poles of tan and found by bisection to
// machine precision.
// ---------------------------------------------------------------------------
namespace {
double bisect(double lo, double hi, int parity, double a, double c) {
  auto f = [&](double w) { return parity == 0 ? c * std::cos(w * a) - w * std::sin(w * a)
                                              : w * std::cos(w * a) + c * std::sin(w * a); };
  double flo = f(lo);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double fm = f(mid);
    if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
  }
  return 0.5 * (lo + hi);
}

struct Mode1D { double lam, w; int parity; };

std::vector<Mode1D> kl_1d(int count, double corr_len) {
  const double a = 0.5, c = 1.0 / corr_len, pi = 3.14159265358979323846;
  std::vector<Mode1D> out;
  for (int k = 0; (int)out.size() < count; ++k) {
    // even: w a in (k pi, k pi + pi/2); the multiplied-out form c cos - w sin has no poles
    double w = bisect(k * pi / a, (k * pi + 0.5 * pi) / a, 0, a, c);
    out.push_back({2 * c / (w * w + c * c), w, 0});
    if ((int)out.size() >= count) break;
    w = bisect((k * pi + 0.5 * pi) / a, (k * pi + pi) / a, 1, a, c);
    out.push_back({2 * c / (w * w + c * c), w, 1});
  }
  return out;
}

double eval_1d(const Mode1D& md, double y) {
  const double a = 0.5;
  if (md.parity == 0) return std::cos(md.w * y) / std::sqrt(a + std::sin(2 * md.w * a) / (2 * md.w));
  return std::sin(md.w * y) / std::sqrt(a - std::sin(2 * md.w * a) / (2 * md.w));
}
}  // namespace

// The same modes at the centroids of the two right triangles of every cell (the paper's P1
// discretisation): entry 2e at (cx + 2/3, cy + 1/3) h, entry 2e + 1 at (cx + 1/3, cy + 2/3) h.
int kl_coef_p1_host(int n, int M, double sigma, double corr_len, double* coef, double* lam) {
  if (n < 3 || M < 0 || M > 64 || !coef || !(corr_len > 0)) return SG_E_ARG;
  const int nc1 = n - 1;
  const size_t Nt = 2 * (size_t)nc1 * nc1;
  std::vector<Mode1D> m1 = kl_1d(M + 1, corr_len);
  struct P2 { double lam; int i, j; };
  std::vector<P2> pairs;
  for (int i = 0; i <= M; ++i)
    for (int j = 0; j <= M; ++j) pairs.push_back({m1[i].lam * m1[j].lam, i, j});
  std::stable_sort(pairs.begin(), pairs.end(), [](const P2& x, const P2& y) {
    if (x.lam != y.lam) return x.lam > y.lam;
    return x.i < y.i;
  });
  for (size_t e = 0; e < Nt; ++e) coef[e] = 1.0;
  const double h = 1.0 / nc1;
  const double off[2][2] = {{2.0 / 3.0, 1.0 / 3.0}, {1.0 / 3.0, 2.0 / 3.0}};   // (x, y) in the cell, per triangle
  for (int k = 1; k <= M; ++k) {
    const P2& pr = pairs[k - 1];
    if (lam) lam[k - 1] = pr.lam;
    const double s = sigma * std::sqrt(pr.lam);
    double* row = coef + (size_t)k * Nt;
    for (int tri = 0; tri < 2; ++tri)
      for (int cy = 0; cy < nc1; ++cy) {
        const double by = eval_1d(m1[pr.j], cy * h - 0.5 + off[tri][1] * h);
        for (int cx = 0; cx < nc1; ++cx) {
          const double bx = eval_1d(m1[pr.i], cx * h - 0.5 + off[tri][0] * h);
          row[2 * ((size_t)cy * nc1 + cx) + tri] = s * bx * by;
        }
      }
  }
  return SG_OK;
}

int kl_coef_host(int n, int M, double sigma, double corr_len, const double* abar, double* coef, double* lam) {
  if (n < 3 || M < 0 || M > 64 || !coef || !(corr_len > 0)) return SG_E_ARG;
  const int nc1 = n - 1;
  const size_t Nc = (size_t)nc1 * nc1;
  std::vector<Mode1D> m1 = kl_1d(M + 1, corr_len);
  struct P2 { double lam; int i, j; };
  std::vector<P2> pairs;
  for (int i = 0; i <= M; ++i)
    for (int j = 0; j <= M; ++j) pairs.push_back({m1[i].lam * m1[j].lam, i, j});
  std::stable_sort(pairs.begin(), pairs.end(), [](const P2& x, const P2& y) {
    if (x.lam != y.lam) return x.lam > y.lam;
    return x.i < y.i;
  });
  for (size_t e = 0; e < Nc; ++e) coef[e] = abar ? abar[e] : 1.0;
  const double h = 1.0 / nc1;
  std::vector<double> bx(nc1), by(nc1);
  for (int k = 1; k <= M; ++k) {
    const P2& pr = pairs[k - 1];
    if (lam) lam[k - 1] = pr.lam;
    for (int t = 0; t < nc1; ++t) {
      double y = (t + 0.5) * h - 0.5;
      bx[t] = eval_1d(m1[pr.i], y);
      by[t] = eval_1d(m1[pr.j], y);
    }
    const double s = sigma * std::sqrt(pr.lam);
    double* row = coef + (size_t)k * Nc;
    for (int cy = 0; cy < nc1; ++cy)
      for (int cx = 0; cx < nc1; ++cx) row[(size_t)cy * nc1 + cx] = s * bx[cx] * by[cy];
  }
  return SG_OK;
}

// ---------------------------------------------------------------------------
// PC basis (Sec. 2.2, 3.3): multi-indices of total degree <= p, grouped by
// degree, descending lexicographic order inside a degree.
// ---------------------------------------------------------------------------
namespace {
void gen_level(int M, int q, int pos, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  if (pos == M - 1) {
    cur[pos] = q;
    out.push_back(cur);
    return;
  }
  for (int v = q; v >= 0; --v) {   // descending in the leading component first
    cur[pos] = v;
    gen_level(M, q - v, pos + 1, cur, out);
  }
}
}  // namespace

void build_basis(int M, int p, std::vector<int>& alpha, std::vector<int>& lvl_off) {
  alpha.clear();
  lvl_off.assign(1, 0);
  if (M == 0) {
    lvl_off.push_back(1);
    for (int q = 1; q <= p; ++q) lvl_off.push_back(1);
    return;
  }
  for (int q = 0; q <= p; ++q) {
    std::vector<std::vector<int>> lev;
    std::vector<int> cur(M, 0);
    gen_level(M, q, 0, cur, lev);
    for (auto& a : lev) alpha.insert(alpha.end(), a.begin(), a.end());
    lvl_off.push_back(lvl_off.back() + (int)lev.size());
  }
}

// Jacobi-matrix entries of the orthonormal 1-D families: xi q_n = gamma(n) q_{n+1} + gamma(n-1) q_{n-1}
// Legendre on U(-sqrt3, sqrt3): sqrt3 (n+1)/sqrt((2n+1)(2n+3)); Hermite on N(0,1): sqrt(n+1).
double gamma_1d(int family, int nn) {
  if (family == SG_LEGENDRE) return std::sqrt(3.0) * (nn + 1) / std::sqrt((2.0 * nn + 1) * (2.0 * nn + 3));
  return std::sqrt(nn + 1.0);
}

// Coupling tables of A = sum_k G_k (x) K_k (Eqs. def-stochastic, tensor-product):
// G_k(i,j) = gamma(min(alpha_k, beta_k)) when alpha, beta differ by one in component k.
void build_terms(const sg_ctx* h, int which, std::vector<int>& row_ptr, std::vector<int>& tj,
                 std::vector<int>& tk, std::vector<double>& tg) {
  const int P = h->P, M = h->M;
  std::map<std::vector<int>, int> index;
  for (int i = 0; i < P; ++i) index[std::vector<int>(h->alpha.begin() + (size_t)i * M, h->alpha.begin() + (size_t)(i + 1) * M)] = i;
  row_ptr.assign(1, 0);
  tj.clear(), tk.clear(), tg.clear();
  for (int i = 0; i < P; ++i) {
    std::vector<int> a(h->alpha.begin() + (size_t)i * M, h->alpha.begin() + (size_t)(i + 1) * M);
    // which: 0 all, 1 lower, 2 upper, 3 off-diagonal, 4 the mean (diagonal) term only
    if (which == 0 || which == 4) { tj.push_back(i); tk.push_back(0); tg.push_back(1.0); }
    for (int k = 0; k < M && which != 4; ++k) {
      if (which != 2 && a[k] > 0) {   // lower neighbour i - e_k
        std::vector<int> b = a;
        b[k] -= 1;
        tj.push_back(index.at(b)); tk.push_back(k + 1); tg.push_back(gamma_1d(h->family, a[k] - 1));
      }
      if (which != 1) {               // upper neighbour i + e_k
        std::vector<int> b = a;
        b[k] += 1;
        auto it = index.find(b);
        if (it != index.end()) { tj.push_back(it->second); tk.push_back(k + 1); tg.push_back(gamma_1d(h->family, a[k])); }
      }
    }
    row_ptr.push_back((int)tj.size());
  }
}

// ---------------------------------------------------------------------------
// Galerkin coarse operators for a variable mean coefficient: level-0 9-point
// stencil assembled from the Q1 element matrix times abar per cell, then
// A_{l+1} = P^T A_l P with bilinear P.  Stencil layout st[9 s + (dy+1)*3 + (dx+1)].
// ---------------------------------------------------------------------------
void galerkin_stencils(int n0, int nlev, const double* abar, std::vector<std::vector<double>>& st) {
  static const double Kref[4][4] = {{4, -1, -2, -1}, {-1, 4, -1, -2}, {-2, -1, 4, -1}, {-1, -2, -1, 4}};
  static const int cdx[4] = {0, 1, 1, 0}, cdy[4] = {0, 0, 1, 1};   // SW, SE, NE, NW
  st.assign(nlev, {});
  int n = n0, m = n - 2;
  st[0].assign((size_t)9 * m * m, 0.0);
  for (int cy = 0; cy < n - 1; ++cy)
    for (int cx = 0; cx < n - 1; ++cx) {
      double c = abar[(size_t)cy * (n - 1) + cx] / 6.0;
      for (int a = 0; a < 4; ++a) {
        int vx = cx + cdx[a], vy = cy + cdy[a];
        if (vx < 1 || vx > n - 2 || vy < 1 || vy > n - 2) continue;
        size_t s = (size_t)(vx - 1) + (size_t)(vy - 1) * m;
        for (int b = 0; b < 4; ++b) {
          int dx = cdx[b] - cdx[a], dy = cdy[b] - cdy[a];
          st[0][9 * s + (dy + 1) * 3 + (dx + 1)] += c * Kref[a][b];
        }
      }
    }
  // zero couplings to boundary vertices (they are not unknowns)
  for (int l = 0; l + 1 < nlev; ++l) {
    int nf = n, mf = nf - 2, nc = (nf + 1) / 2, mc = nc - 2;
    std::vector<double>& A = st[l];
    std::vector<double>& C = st[l + 1];
    C.assign((size_t)9 * mc * mc, 0.0);
    auto w1 = [](int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); };
    for (int VY = 1; VY <= nc - 2; ++VY)
      for (int VX = 1; VX <= nc - 2; ++VX) {
        size_t I = (size_t)(VX - 1) + (size_t)(VY - 1) * mc;
        for (int fy = 2 * VY - 1; fy <= 2 * VY + 1; ++fy)
          for (int fx = 2 * VX - 1; fx <= 2 * VX + 1; ++fx) {
            if (fx < 1 || fx > nf - 2 || fy < 1 || fy > nf - 2) continue;
            double pi = w1(fx - 2 * VX) * w1(fy - 2 * VY);
            size_t i = (size_t)(fx - 1) + (size_t)(fy - 1) * mf;
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                int gx = fx + dx, gy = fy + dy;
                if (gx < 1 || gx > nf - 2 || gy < 1 || gy > nf - 2) continue;
                double aij = A[9 * i + (dy + 1) * 3 + (dx + 1)];
                if (aij == 0.0) continue;
                // coarse parents of fine vertex (gx, gy)
                int x0 = gx / 2, x1 = (gx + 1) / 2, y0 = gy / 2, y1 = (gy + 1) / 2;
                for (int JY = y0; JY <= y1; ++JY)
                  for (int JX = x0; JX <= x1; ++JX) {
                    if (JX < 1 || JX > nc - 2 || JY < 1 || JY > nc - 2) continue;
                    double pj = w1(gx - 2 * JX) * w1(gy - 2 * JY);
                    if (pj == 0.0) continue;
                    int ox = JX - VX, oy = JY - VY;
                    C[9 * I + (oy + 1) * 3 + (ox + 1)] += pi * aij * pj;
                  }
              }
          }
      }
    n = nc;
  }
}
