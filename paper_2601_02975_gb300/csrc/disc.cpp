// One level of the discretisation (Sec. 4): classification of cut cells into
// SFV and PLG cells (Def. 4.1), the SFV stencil with ghost cells at the box
// walls (Sec. 4.1, Eq. 4.7a,b), the PLG fits (Sec. 4.2, Eq. 4.11-4.19), and
// the rows of A and N in A u = f - N g (Eq. 4.20).
//
// Ghost cells.  For a wall with condition alpha1 u + alpha2 du/dn = g (alpha1
// = 1, alpha2 = 0 for Dirichlet data; 0, 1 for Neumann data) and
// beta2 = alpha2 / h, the two ghost averages beyond an extendable face are
//   G1 = [ alpha1 (-77, 43, -17, 3) + beta2 (25, 45, -25, 5) ] . U + 60 g
//   G2 = [ alpha1 (-505, 335, -145, 27) + beta2 (-375, 725, -375, 75) ] . U + 300 g
// both divided by 2 (6 alpha1 + 25 beta2), with U = (U0..U3) the averages of
// the four cells inward from the wall (U0 touching it): the averages of the
// quartic with those four averages and the boundary datum.  These reduce to
// the paper's Dirichlet and Neumann formulas (Sec. 4.1) with the depth-2
// Dirichlet datum coefficient 300/12.
//
// Corner ghosts.  With a cross term (b != 0) the 5 x 5 stencil of the cells
// nearest a box corner reads cells beyond two walls, which Sec. 4.1 does not
// define.  Such a ghost is the ghost column of one wall at its depth,
// extrapolated beyond the other wall by the quartic through the five cells
// nearest the corner (weights (5,-10,10,-5,1) and (15,-40,45,-24,5)), averaged
// with the same construction in the other order.
//
// PLG lattice.  The paper cites its poised-lattice search without stating it.
// The lattice here is made of five grid lines (rows, or else columns) holding
// 5, 4, 3, 2 and 1 present cells of the 9 x 9 box around the cell (11 x 11,
// then 13 x 13, where that box holds none, as in the thin wedges at the kinks
// of a union of holes).  A cell at
// offset (u, v) costs u^2 + v^2, plus 2 if it is a cut cell other than the
// cell itself (its centroid lies off the grid line); each line takes its
// cheapest cells and the lines and counts minimise the total cost (ties:
// larger counts on lower lines first, rows before columns).  A set of points on five parallel lines with
// 5, 4, 3, 2, 1 points each is poised for quartics, and so are the averages
// of cells at those points.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <numeric>
#include <string>
#include <thread>

#include "setup.h"

namespace ccmg {

namespace {

const double kLap[5] = {-1, 16, -30, 16, -1};
const double kGrad[5] = {1, -8, 0, 8, -1};
const double kExt[2][5] = {{5, -10, 10, -5, 1}, {15, -40, 45, -24, 5}};
const int kRadius = 6;       // largest search box (13 x 13)
const int kRadiusFirst = 4;  // first search box (9 x 9)
const int kCutPenalty = 2;

void ghost_coefs(const Bc& bc, double h, double out[2][5]) {
  double a1 = 1.0, a2 = 0.0;
  if (bc.type == BC_N) { a1 = 0.0; a2 = 1.0; }
  else if (bc.type == BC_R) { a1 = bc.a1; a2 = bc.a2; }
  double b2 = a2 / h, den = 2.0 * (6.0 * a1 + 25.0 * b2);
  if (den == 0.0) throw SetupError(1, "degenerate Robin condition");
  const double g1a[4] = {-77, 43, -17, 3}, g1b[4] = {25, 45, -25, 5};
  const double g2a[4] = {-505, 335, -145, 27}, g2b[4] = {-375, 725, -375, 75};
  for (int q = 0; q < 4; ++q) {
    out[0][q] = (a1 * g1a[q] + b2 * g1b[q]) / den;
    out[1][q] = (a1 * g2a[q] + b2 * g2b[q]) / den;
  }
  out[0][4] = 60.0 / den;
  out[1][4] = 300.0 / den;
}

// cell index of the q-th cell inward from wall w at position t
inline int inward(int n, int w, int t, int q) {
  switch (w) {
    case 0: return q * n + t;               // south
    case 1: return t * n + (n - 1 - q);     // east
    case 2: return (n - 1 - q) * n + t;     // north
    default: return t * n + q;              // west
  }
}

// --- small dense linear algebra ---------------------------------------------
// Solve A x = b (n x n, row-major) by Gaussian elimination with partial pivoting.
bool lu_solve(std::vector<double> A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[p * n + k], A[c * n + k]);
      std::swap(b[p], b[c]);
    }
    for (int r = c + 1; r < n; ++r) {
      double l = A[r * n + c] / A[c * n + c];
      if (l == 0.0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= l * A[c * n + k];
      b[r] -= l * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return true;
}

// Minimum 2-norm solution of B x = rhs, B (m x n) with m < n of full row
// rank, by Householder QR of B^T: B^T = Q R, x = Q (R^-T rhs).
bool min_norm(const std::vector<double>& B, const std::vector<double>& rhs, int m, int n,
              std::vector<double>& x) {
  // T = B^T, n x m, column-major copy for the reflections
  std::vector<double> T((size_t)n * m);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < n; ++c) T[(size_t)r * n + c] = B[(size_t)r * n + c];  // column r of T
  std::vector<std::vector<double>> V(m);
  std::vector<double> Rdiag(m);
  for (int k = 0; k < m; ++k) {
    double* col = &T[(size_t)k * n];
    double nrm = 0;
    for (int i = k; i < n; ++i) nrm += col[i] * col[i];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    double alpha = col[k] > 0 ? -nrm : nrm;
    std::vector<double> v(n, 0.0);
    for (int i = k; i < n; ++i) v[i] = col[i];
    v[k] -= alpha;
    double vn = 0;
    for (int i = k; i < n; ++i) vn += v[i] * v[i];
    for (int j = k; j < m; ++j) {
      double* cj = &T[(size_t)j * n];
      double s = 0;
      for (int i = k; i < n; ++i) s += v[i] * cj[i];
      s = 2.0 * s / vn;
      for (int i = k; i < n; ++i) cj[i] -= s * v[i];
    }
    V[k] = v;
    Rdiag[k] = T[(size_t)k * n + k];
  }
  // R^T y = rhs (forward), R(i, j) = T[j*n + i] for i <= j
  std::vector<double> y(m);
  for (int i = 0; i < m; ++i) {
    double s = rhs[i];
    for (int j = 0; j < i; ++j) s -= T[(size_t)i * n + j] * y[j];
    if (T[(size_t)i * n + i] == 0.0) return false;
    y[i] = s / T[(size_t)i * n + i];
  }
  // x = Q [y; 0] = H_0 H_1 ... H_{m-1} [y; 0]
  x.assign(n, 0.0);
  for (int i = 0; i < m; ++i) x[i] = y[i];
  for (int k = m - 1; k >= 0; --k) {
    const std::vector<double>& v = V[k];
    double vn = 0, s = 0;
    for (int i = k; i < n; ++i) { vn += v[i] * v[i]; s += v[i] * x[i]; }
    s = 2.0 * s / vn;
    for (int i = k; i < n; ++i) x[i] -= s * v[i];
  }
  return true;
}

// basis monomials of total degree <= 4
struct Mono { int p, q; };
const std::vector<Mono>& basis() {
  static std::vector<Mono> b = [] {
    std::vector<Mono> v;
    for (int d = 0; d <= 4; ++d)
      for (int p = d; p >= 0; --p) v.push_back({p, d - p});
    return v;
  }();
  return b;
}

}  // namespace

// ---------------------------------------------------------------------------
void LevelDisc::row(int k, std::map<int, double>& arow, std::map<int, double>* nrow) const {
  arow.clear();
  if (nrow) nrow->clear();
  if (kind[k] == K_EMPTY) {
    arow[k] = 1.0;
    return;
  }
  if (kind[k] == K_PLG) {
    int r = (int)(std::lower_bound(plg.begin(), plg.end(), k) - plg.begin());
    for (int q = 0; q < 15; ++q) arow[lattice[r][q]] += beta[r][q];
    if (nrow && bd_of_plg[r] >= 0) (*nrow)[4 * n + bd_of_plg[r]] += beta[r][15];
    return;
  }
  const int i = k % n, j = k / n;
  const double h2 = h * h;
  auto ghost = [&](int w, int t, int m, double wt) {   // m = depth 1 or 2
    for (int q = 0; q < 4; ++q) arow[inward(n, w, t, q)] += wt * gc[w][m - 1][q];
    if (nrow) (*nrow)[w * n + t] += wt * gc[w][m - 1][4];
  };
  auto add = [&](int ii, int jj, double wt) {
    bool ox = ii < 0 || ii >= n, oy = jj < 0 || jj >= n;
    if (!ox && !oy) { arow[jj * n + ii] += wt; return; }
    if (ox && oy) {
      int wx = ii < 0 ? 3 : 1, mx = ii < 0 ? -ii : ii - n + 1;
      int wy = jj < 0 ? 0 : 2, my = jj < 0 ? -jj : jj - n + 1;
      for (int q = 0; q < 5; ++q) {
        ghost(wx, jj < 0 ? q : n - 1 - q, mx, 0.5 * wt * kExt[my - 1][q]);
        ghost(wy, ii < 0 ? q : n - 1 - q, my, 0.5 * wt * kExt[mx - 1][q]);
      }
      return;
    }
    if (ii >= n) ghost(1, jj, ii - n + 1, wt);
    else if (ii < 0) ghost(3, jj, -ii, wt);
    else if (jj >= n) ghost(2, ii, jj - n + 1, wt);
    else ghost(0, ii, -jj, wt);
  };
  for (int m = -2; m <= 2; ++m) {
    add(i + m, j, a * kLap[m + 2] / (12.0 * h2));
    add(i, j + m, c * kLap[m + 2] / (12.0 * h2));
  }
  if (b != 0.0)
    for (int m1 = -2; m1 <= 2; ++m1)
      for (int m2 = -2; m2 <= 2; ++m2)
        if (m1 && m2) add(i + m1, j + m2, b * kGrad[m1 + 2] * kGrad[m2 + 2] / (144.0 * h2));
}

LevelDisc discretize(const Problem& P, int n) {
  LevelDisc D;
  D.P = &P;
  D.n = n;
  D.a = P.a;
  D.b = P.b;
  D.c = P.c;
  D.geom = build_geometry(P, n);
  const LevelGeom& G = D.geom;
  D.h = G.h;
  const double h = G.h;
  D.diag = -30.0 * (P.a + P.c) / (12.0 * h * h);
  for (int w = 0; w < 4; ++w) ghost_coefs(P.bc[w], h, D.gc[w]);
  for (int w = 0; w < 4; ++w) {
    D.ext[w].assign(n, 0);
    if (n < 4) continue;
    for (int t = 0; t < n; ++t) {
      bool ok = true;
      for (int q = 0; q < 4; ++q) ok = ok && G.type[inward(n, w, t, q)] == CT_FULL;
      D.ext[w][t] = ok;
    }
  }
  auto ghost_ok = [&](int ii, int jj) {
    bool ox = ii < 0 || ii >= n, oy = jj < 0 || jj >= n;
    if (ox && oy) {
      if (n < 5) return false;
      int wx = ii < 0 ? 3 : 1, wy = jj < 0 ? 0 : 2;
      for (int q = 0; q < 5; ++q) {
        if (!D.ext[wx][jj < 0 ? q : n - 1 - q]) return false;
        if (!D.ext[wy][ii < 0 ? q : n - 1 - q]) return false;
      }
      return true;
    }
    if (ii >= n) return (bool)D.ext[1][jj];
    if (ii < 0) return (bool)D.ext[3][jj];
    if (jj >= n) return (bool)D.ext[2][ii];
    return (bool)D.ext[0][ii];
  };
  // --- Def. 4.1 ------------------------------------------------------------
  D.kind.assign((size_t)n * n, K_EMPTY);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      int k = j * n + i;
      if (G.type[k] == CT_EMPTY) continue;
      bool sfv = G.type[k] == CT_FULL;
      for (int dj = -2; dj <= 2 && sfv; ++dj)
        for (int di = -2; di <= 2 && sfv; ++di) {
          if (P.b == 0.0 && di && dj) continue;
          int ii = i + di, jj = j + dj;
          if (ii >= 0 && jj >= 0 && ii < n && jj < n) sfv = G.type[jj * n + ii] == CT_FULL;
          else sfv = ghost_ok(ii, jj);
        }
      D.kind[k] = sfv ? K_SFV : K_PLG;
    }
  // --- PLG cells: lattice and fit --------------------------------------------
  for (int k = 0; k < n * n; ++k)
    if (D.kind[k] == K_PLG) D.plg.push_back(k);
  const auto& B = basis();
  // the fits are independent: computed on all host cores into per-cell slots,
  // then appended in PLG order (the result does not depend on the threads)
  struct PlgOut {
    std::array<int, 15> lat{};
    std::array<double, 16> bt{};
    bool withb = false;
    int err = 0;
    const char* msg = "";
  };
  std::vector<PlgOut> outs(D.plg.size());
  auto fit_one = [&](size_t pr) {
    const int k = D.plg[pr];
    PlgOut& O = outs[pr];
    const int i0 = k % n, j0 = k / n;
    // lattice: dynamic programme over lines
    struct Cand { int cost; int orient; std::vector<int> key; std::vector<int> cells; bool ok = false; };
    Cand best;
    for (int R = kRadiusFirst; R <= kRadius && !best.ok; ++R)
    for (int orient = 0; orient < 2; ++orient) {
      std::vector<std::vector<int>> avail(2 * kRadius + 1);
      // cost of the cell at offset (u, v): u^2 + v^2, plus kCutPenalty for a
      // cut cell other than the cell itself (its centroid is off the line)
      int cost[2 * kRadius + 1][2 * kRadius + 1];
      for (int v = -R; v <= R; ++v) {
        auto& us = avail[v + kRadius];
        for (int u = -R; u <= R; ++u) {
          int di = orient == 0 ? u : v, dj = orient == 0 ? v : u;
          int ii = i0 + di, jj = j0 + dj;
          if (ii >= 0 && jj >= 0 && ii < n && jj < n && G.type[jj * n + ii] != CT_EMPTY) {
            us.push_back(u);
            bool cut = G.type[jj * n + ii] == CT_CUT && (di != 0 || dj != 0);
            cost[v + kRadius][u + kRadius] = u * u + v * v + (cut ? kCutPenalty : 0);
          }
        }
        const int* cv = cost[v + kRadius];
        std::sort(us.begin(), us.end(), [&](int x, int y) {
          int cx = cv[x + kRadius], cy = cv[y + kRadius];
          return cx != cy ? cx < cy : x < y;
        });
      }
      const int counts[5] = {5, 4, 3, 2, 1};
      struct St { bool have = false; int cost = 0; std::vector<int> key; std::vector<int> asg; };
      std::vector<St> nxt(32), cur(32);
      nxt[31].have = true;
      nxt[31].asg.assign(2 * kRadius + 1, 0);
      for (int v = R; v >= -R; --v) {
        const auto& us = avail[v + kRadius];
        for (int mask = 0; mask < 32; ++mask) {
          St bestS;
          auto consider = [&](int cost, std::vector<int> key, std::vector<int> asg) {
            if (!bestS.have || cost < bestS.cost || (cost == bestS.cost && key < bestS.key)) {
              bestS.have = true;
              bestS.cost = cost;
              bestS.key = std::move(key);
              bestS.asg = std::move(asg);
            }
          };
          if (nxt[mask].have) {
            std::vector<int> key{0};
            key.insert(key.end(), nxt[mask].key.begin(), nxt[mask].key.end());
            consider(nxt[mask].cost, key, nxt[mask].asg);
          }
          for (int bit = 0; bit < 5; ++bit) {
            int cnt = counts[bit];
            if ((mask >> bit) & 1 || (int)us.size() < cnt) continue;
            int m2 = mask | (1 << bit);
            if (!nxt[m2].have) continue;
            int rc = 0;
            for (int q = 0; q < cnt; ++q) rc += cost[v + kRadius][us[q] + kRadius];
            std::vector<int> key{-cnt};
            key.insert(key.end(), nxt[m2].key.begin(), nxt[m2].key.end());
            std::vector<int> asg = nxt[m2].asg;
            asg[v + kRadius] = cnt;
            consider(nxt[m2].cost + rc, key, asg);
          }
          cur[mask] = bestS;
        }
        std::swap(nxt, cur);
      }
      if (!nxt[0].have) continue;
      if (!best.ok || nxt[0].cost < best.cost) {
        best.ok = true;
        best.cost = nxt[0].cost;
        best.orient = orient;
        best.cells.clear();
        for (int v = -R; v <= R; ++v) {
          int cnt = nxt[0].asg[v + kRadius];
          for (int q = 0; q < cnt; ++q) {
            int u = avail[v + kRadius][q];
            int di = orient == 0 ? u : v, dj = orient == 0 ? v : u;
            best.cells.push_back((j0 + dj) * n + (i0 + di));
          }
        }
      }
    }
    if (!best.ok || best.cells.size() != 15) {
      O.err = 3;
      O.msg = "no poised lattice for a PLG cell";
      return;
    }
    std::sort(best.cells.begin(), best.cells.end());
    std::array<int, 15> lat;
    std::copy(best.cells.begin(), best.cells.end(), lat.begin());
    O.lat = lat;
    // --- fit: rows basis functions, columns lattice cells (+ boundary) -------
    bool withb = false;
    std::vector<BNode> bn;
    if (G.type[k] == CT_CUT) {
      bn = boundary_nodes(P, G, k);
      withb = !bn.empty();
    }
    const int nc = withb ? 16 : 15;
    std::vector<double> M((size_t)15 * nc, 0.0), rhs(15, 0.0);
    for (int c = 0; c < 15; ++c) {
      int kj = lat[c];
      double m0[kMoments], ms[kMoments];
      G.moments(kj, m0);
      shift_moments(m0, (kj % n) - i0, (kj / n) - j0, ms);
      for (int r = 0; r < 15; ++r) M[(size_t)r * nc + c] = ms[midx(B[r].p, B[r].q)] / ms[0];
    }
    {
      double mi[kMoments];
      G.moments(k, mi);
      auto avg = [&](int p, int q) { return mi[midx(p, q)] / mi[0]; };
      for (int r = 0; r < 15; ++r) {
        int p = B[r].p, q = B[r].q;
        double v = 0;
        if (p >= 2) v += P.a * p * (p - 1) * avg(p - 2, q);
        if (p >= 1 && q >= 1) v += P.b * p * q * avg(p - 1, q - 1);
        if (q >= 2) v += P.c * q * (q - 1) * avg(p, q - 2);
        rhs[r] = v / (h * h);
      }
    }
    std::array<double, 16> bt{};
    if (withb) {
      double px = G.x0 + (i0 + 0.5) * h, py = G.y0 + (j0 + 0.5) * h, ws = 0;
      std::vector<double> col(15, 0.0);
      for (const BNode& nd : bn) {
        const Bc& bc = P.bc[nd.bc];
        double a1 = bc.type == BC_D ? 1.0 : bc.type == BC_N ? 0.0 : bc.a1;
        double a2 = bc.type == BC_D ? 0.0 : bc.type == BC_N ? 1.0 : bc.a2;
        double X = (nd.x - px) / h, Y = (nd.y - py) / h;
        for (int r = 0; r < 15; ++r) {
          int p = B[r].p, q = B[r].q;
          double phi = std::pow(X, p) * std::pow(Y, q);
          double gx = p ? p * std::pow(X, p - 1) * std::pow(Y, q) / h : 0.0;
          double gy = q ? q * std::pow(X, p) * std::pow(Y, q - 1) / h : 0.0;
          col[r] += nd.w * (a1 * phi + a2 * (gx * nd.nx + gy * nd.ny));
        }
        ws += nd.w;
      }
      for (int r = 0; r < 15; ++r) M[(size_t)r * nc + 15] = col[r] / ws;
      // weighted minimum norm (Eq. 4.17-4.18): beta = W^1/2 pinv(M W^1/2) rhs
      double sw[16];
      for (int c = 0; c < 15; ++c) {
        int kj = lat[c];
        double d = std::hypot((double)(kj % n - i0), (double)(kj / n - j0));
        sw[c] = 1.0 / std::sqrt(std::max(d, 0.5));
      }
      sw[15] = 1.0 / std::sqrt(0.5);
      std::vector<double> Ms(M);
      for (int r = 0; r < 15; ++r)
        for (int c = 0; c < 16; ++c) Ms[(size_t)r * 16 + c] *= sw[c];
      std::vector<double> g;
      if (!min_norm(Ms, rhs, 15, 16, g)) {
        O.err = 3;
        O.msg = "singular PLG fit";
        return;
      }
      for (int c = 0; c < 16; ++c) bt[c] = sw[c] * g[c];
      O.withb = true;
    } else {
      std::vector<double> x(rhs);
      if (!lu_solve(M, x, 15)) {
        O.err = 3;
        O.msg = "singular PLG fit";
        return;
      }
      for (int c = 0; c < 15; ++c) bt[c] = x[c];
      bt[15] = 0.0;
    }
    O.bt = bt;
  };
  {
    const size_t np = D.plg.size();
    unsigned T = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    if (np < 256) T = 1;
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < T; ++t)
      pool.emplace_back([&, t] {
        for (size_t r = t; r < np; r += T) fit_one(r);
      });
    for (size_t r = 0; r < np; r += T) fit_one(r);
    for (auto& th : pool) th.join();
    for (size_t r = 0; r < np; ++r) {
      if (outs[r].err) throw SetupError(outs[r].err, outs[r].msg);
      D.lattice.push_back(outs[r].lat);
      if (outs[r].withb) {
        D.bd_of_plg.push_back((int)D.bd_cells.size());
        D.bd_cells.push_back(D.plg[r]);
      } else {
        D.bd_of_plg.push_back(-1);
      }
      D.beta.push_back(outs[r].bt);
    }
  }
  // --- block of the smoother: PLG cells + corner blocks when b != 0 --------
  std::vector<int> blk(D.plg);
  if (P.b != 0.0) {
    int R = std::min(4, n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int k = j * n + i;
        if (D.kind[k] == K_SFV && std::min(i, n - 1 - i) < R && std::min(j, n - 1 - j) < R)
          blk.push_back(k);
      }
  }
  // order: by the nearest boundary curve, then along it (Def. 5.1)
  {
    const int nh = (int)P.holes.size();
    std::vector<int> grp(nh);
    std::iota(grp.begin(), grp.end(), 0);
    std::function<int(int)> root = [&](int x) { while (grp[x] != x) x = grp[x]; return x; };
    const int ns = 720;
    for (int e = 0; e < nh; ++e)
      for (int f = e + 1; f < nh; ++f) {
        bool ov = false;
        for (int s = 0; s < ns && !ov; ++s) {
          double x, y;
          P.holes[e].at(6.283185307179586 * s / ns, x, y);
          ov = P.holes[f].level(x, y) < 0;
        }
        if (ov) grp[root(e)] = root(f);
      }
    std::vector<double> gx(nh, 0), gy(nh, 0), gn(nh, 0);
    for (int e = 0; e < nh; ++e) {
      int r = root(e);
      gx[r] += P.holes[e].cx; gy[r] += P.holes[e].cy; gn[r] += 1;
    }
    const double L = P.x1 - P.x0;
    std::vector<std::tuple<int, double, int>> keys;
    for (int k : blk) {
      double x = G.x0 + (k % n + 0.5) * h, y = G.y0 + (k / n + 0.5) * h;
      double d[4] = {y - P.y0, P.x1 - x, P.y1 - y, x - P.x0};
      int side = (int)(std::min_element(d, d + 4) - d);
      double s_box[4] = {x - P.x0, L + y - P.y0, 2 * L + P.x1 - x, 3 * L + P.y1 - y};
      double bestd = d[side], bests = s_box[side];
      int bestg = 0;
      for (int e = 0; e < nh; ++e) {
        const int nsm = 1024;
        for (int s = 0; s < nsm; ++s) {
          double hx, hy;
          P.holes[e].at(6.283185307179586 * s / nsm, hx, hy);
          double dd = std::hypot(hx - x, hy - y);
          if (dd < bestd) {
            int r = root(e);
            bestd = dd;
            bestg = 1 + r;
            double ang = std::atan2(hy - gy[r] / gn[r], hx - gx[r] / gn[r]);
            bests = ang < 0 ? ang + 6.283185307179586 : ang;
          }
        }
      }
      keys.emplace_back(bestg, bests, k);
    }
    std::sort(keys.begin(), keys.end());
    for (auto& t : keys) D.block.push_back(std::get<2>(t));
  }
  std::map<int, double> ar, nr;
  for (int k : D.block) {
    D.row(k, ar, nullptr);
    D.block_rows.push(ar);
  }
  for (int k = 0; k < n * n; ++k) {
    if (D.kind[k] == K_EMPTY) continue;
    // only PLG rows (boundary datum) and the rows of cells within two cells
    // of a box wall (ghost data) have terms in N
    const int i = k % n, j = k / n;
    if (D.kind[k] != K_PLG && i >= 2 && j >= 2 && i < n - 2 && j < n - 2) continue;
    D.row(k, ar, &nr);
    if (!nr.empty()) {
      D.nrows.push(nr);
      D.nrow_cell.push_back(k);
    }
  }
  return D;
}

}  // namespace ccmg
