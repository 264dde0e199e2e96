// Per-cell steps of the setup, written once for the host and the device.
//
// Each function here computes the table entries of ONE cell from read-only
// inputs: the classification of a control volume (Sec. 3.1), the moments of
// a cut cell from its boundary pieces (Sec. 4.2), its kind (Def. 4.1), the
// poised lattice of a PLG cell (Def. 4.3, the reading of the lattice rule
// stated in disc.cpp), its fit (Eq. 4.14, or the weighted minimum norm of
// Eq. 4.17-4.18), and the nearest sample of a boundary curve that orders the
// exactly solved block (Def. 5.1).  disc.cpp runs them on
// host threads; setup_dev.cu runs them as CUDA kernels, one thread per cell.
//
// Both builds evaluate the same expressions in the same order with IEEE
// double operations only (+ - * / and sqrt, all correctly rounded, and rint,
// floor, ceil, fmod, exact; no contraction into fused multiply-adds: the
// host compiler gets -ffp-contract=off and the device translation unit
// --fmad=false), and the curves' sines and cosines come from sin_cos below,
// so the two give the same bits.  The one exception is the level function
// of the flower and rectangle holes (hypot, atan2, cos), used only to
// classify cells that no curve crosses: their centres lie at least h/2 from
// the curve, so the sign cannot differ.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define CC_HD __host__ __device__
#else
#define CC_HD
#endif
// keep the device code of the long fixed-count loops rolled (compile time)
#ifdef __CUDA_ARCH__
#define CC_ROLLED _Pragma("unroll 1")
#else
#define CC_ROLLED
#endif

namespace ccmg {

constexpr double kTwoPi = 6.283185307179586476925286766559;

namespace cell {

// sin t and cos t, the same bits on the host and the device.  Additive range
// reduction (Cody and Waite): k = the integer nearest t 2/pi, r = t - k pi/2
// with pi/2 split into P1 + P2 + P3, P1 and P2 of 30 significant bits so that
// k P1 and k P2 are exact for |k| < 2^23; then the Taylor series of sin and
// cos about 0 on |r| <= pi/4 (to r^17 and r^18: the first omitted terms are
// below 1e-19), and the quadrant k mod 4.
CC_HD inline void sin_cos(double t, double* s, double* c) {
  const double P1 = 1.5707963276654482, P2 = -8.705515692000731e-10, P3 = -3.50343439808993e-19;
  const double k = rint(t * 0.6366197723675814);
  const double r = ((t - k * P1) - k * P2) - k * P3;
  const double r2 = r * r;
  const double sr = r + r * r2 * (-0.16666666666666666 + r2 * (0.008333333333333333 +
                    r2 * (-0.0001984126984126984 + r2 * (2.7557319223985893e-06 +
                    r2 * (-2.505210838544172e-08 + r2 * (1.6059043836821613e-10 +
                    r2 * (-7.647163731819816e-13 + r2 * 2.8114572543455206e-15)))))));
  const double cr = 1.0 + r2 * (-0.5 + r2 * (0.041666666666666664 + r2 * (-0.001388888888888889 +
                    r2 * (2.48015873015873e-05 + r2 * (-2.755731922398589e-07 +
                    r2 * (2.08767569878681e-09 + r2 * (-1.1470745597729725e-11 +
                    r2 * 4.779477332387385e-14)))))));
  const long long q = ((long long)k % 4 + 4) % 4;
  if (q == 0) { *s = sr; *c = cr; }
  else if (q == 1) { *s = cr; *c = -sr; }
  else if (q == 2) { *s = -sr; *c = -cr; }
  else { *s = -cr; *c = sr; }
}

// side k of a kind-2 hole at parameter t: the corner index and the fraction
CC_HD inline void rect_side(double t, int& k, double& tau) {
  const double q = kTwoPi / 4;
  double tm = fmod(t, kTwoPi);
  if (tm < 0) tm += kTwoPi;
  k = (int)floor(tm / q);
  if (k > 3) k = 3;
  tau = (tm - k * q) / q;
}

}  // namespace cell

// A hole: kind 0 the ellipse c + R(th) (r1 cos t, r2 sin t); kind 1 the
// flower c + (r1 + r2 cos(petals t)) (cos t, sin t) (Sec. 6.2); kind 2
// everything outside the rectangle with corner c and sides r1 (direction th)
// and r2 (direction th + pi/2), whose sides are the curve, followed
// clockwise around the rectangle as t grows (a quarter of [0, 2pi) each), so
// that the domain is on the left from high to low t as for the other holes.
struct Hole {
  double cx, cy, r1, r2, th, co, si;
  int kind = 0;
  int petals = 0;
  // point and derivative at parameter t
  CC_HD void at(double t, double& x, double& y) const {
    if (kind == 2) {
      double vx[4], vy[4], tau;
      int k;
      corners_cw(vx, vy);
      cell::rect_side(t, k, tau);
      const int k1 = (k + 1) % 4;
      x = vx[k] + tau * (vx[k1] - vx[k]);
      y = vy[k] + tau * (vy[k1] - vy[k]);
      return;
    }
    double st, ct;
    cell::sin_cos(t, &st, &ct);
    if (kind == 1) {
      double sp, cp;
      cell::sin_cos(petals * t, &sp, &cp);
      const double r = r1 + r2 * cp;
      x = cx + r * ct;
      y = cy + r * st;
      return;
    }
    x = cx + co * r1 * ct - si * r2 * st;
    y = cy + si * r1 * ct + co * r2 * st;
  }
  CC_HD void dat(double t, double& dx, double& dy) const {
    if (kind == 2) {
      double vx[4], vy[4], tau;
      int k;
      corners_cw(vx, vy);
      cell::rect_side(t, k, tau);
      const int k1 = (k + 1) % 4;
      dx = (vx[k1] - vx[k]) / (kTwoPi / 4);
      dy = (vy[k1] - vy[k]) / (kTwoPi / 4);
      return;
    }
    double st, ct;
    cell::sin_cos(t, &st, &ct);
    if (kind == 1) {
      double sp, cp;
      cell::sin_cos(petals * t, &sp, &cp);
      const double r = r1 + r2 * cp, dr = -r2 * petals * sp;
      dx = dr * ct - r * st;
      dy = dr * st + r * ct;
      return;
    }
    dx = -co * r1 * st - si * r2 * ct;
    dy = -si * r1 * st + co * r2 * ct;
  }
  CC_HD double halfwidth() const {
    return kind == 2 ? 1e300 : kind == 1 ? r1 - r2 : (r1 < r2 ? r1 : r2);
  }
  // kind 2, in the order of t
  CC_HD void corners_cw(double vx[4], double vy[4]) const {
    // counter-clockwise: c, c + r1 e, c + r1 e + r2 e', c + r2 e'; clockwise
    // from c: c, c + r2 e', c + r1 e + r2 e', c + r1 e
    vx[0] = cx;                       vy[0] = cy;
    vx[1] = cx - r2 * si;             vy[1] = cy + r2 * co;
    vx[2] = cx + r1 * co - r2 * si;   vy[2] = cy + r1 * si + r2 * co;
    vx[3] = cx + r1 * co;             vy[3] = cy + r1 * si;
  }
  // < 0 inside the hole
  CC_HD double level(double x, double y) const {
    if (kind == 2) {
      // the smallest inward-normal distance to the rectangle's side lines:
      // positive inside the rectangle, negative in the hole
      double vx[4], vy[4];
      corners_cw(vx, vy);
      double out = 0;
      for (int i = 0; i < 4; ++i) {
        // counter-clockwise side from corner a to corner b
        const int a = (4 - i) % 4, b = (3 - i + 4) % 4;
        const double ex = vx[b] - vx[a], ey = vy[b] - vy[a], L = hypot(ex, ey);
        const double d = (-ey * (x - vx[a]) + ex * (y - vy[a])) / L;
        out = (i == 0 || d < out) ? d : out;
      }
      return out;
    }
    double dx = x - cx, dy = y - cy;
    if (kind == 1) return hypot(dx, dy) - (r1 + r2 * cos(petals * atan2(dy, dx)));
    double u = co * dx + si * dy, v = -si * dx + co * dy;
    return (u / r1) * (u / r1) + (v / r2) * (v / r2) - 1.0;
  }
};

// A quadrature node on the boundary of a cut cell: position, outward unit
// normal, weight |ds|, boundary condition index.
struct BNode { double x, y, nx, ny, w; int bc; };

// An oriented boundary piece of a cut cell: a straight piece of a face, or an
// arc of a hole from parameter ta down to tb.
struct Piece {
  bool arc;
  double xa, ya, xb, yb;  // end points (start, end)
  int hole;               // arcs
  double ta, tb;          // arcs: parameter from ta to tb (tb < ta)
  int bc;                 // index into Problem::bc, -1 for interior faces
  int face;               // face pieces: 0 bottom, 1 right, 2 top, 3 left; arcs -1
};

// Gauss-Legendre rules on [-1, 1]: 5 points for straight pieces, 10 for each
// sub-arc of at most 0.25 rad
struct Rules510 { double sx[5], sw[5], ax[10], aw[10]; };

namespace cell {

enum : uint8_t { T_EMPTY = 0, T_FULL = 1, T_CUT = 2 };   // LevelGeom::type
enum : uint8_t { K_EMPTY_ = 0, K_SFV_ = 1, K_PLG_ = 2 };  // LevelDisc::kind

constexpr int kNM = 28;            // moments x^p y^q, p + q <= 6
constexpr int kLatR = 6;           // largest box of the first search: 13 x 13
constexpr int kLatR0 = 4;          // first search box: 9 x 9
constexpr int kLatRFar = 12;       // the far search, where 13 x 13 holds no lattice: up to 25 x 25
constexpr int kCutPenalty = 2;     // extra cost of a cut cell in a lattice
constexpr int kCurveSamples = 1024;

CC_HD inline int mi(int p, int q) { int d = p + q; return d * (d + 1) / 2 + q; }

CC_HD inline double ipow(double x, int p) {
  double r = 1.0;
  for (int k = 0; k < p; ++k) r *= x;
  return r;
}

// --- classification of a control volume no curve crosses (Sec. 3.1) --------
CC_HD inline bool outside_all(const Hole* holes, int nh, double x, double y) {
  for (int e = 0; e < nh; ++e)
    if (holes[e].level(x, y) <= 0.0) return false;
  return true;
}

// --- Def. 4.1: SFV if the cell is full and every cell of its stencil (5
// points per direction; the 5 x 5 box when b != 0) is full or a usable
// ghost; ext[w * n + t] flags the extendable wall positions of wall w.
CC_HD inline bool ghost_ok(const uint8_t* ext, int n, int ii, int jj) {
  const bool ox = ii < 0 || ii >= n, oy = jj < 0 || jj >= n;
  if (ox && oy) {
    if (n < 5) return false;
    const int wx = ii < 0 ? 3 : 1, wy = jj < 0 ? 0 : 2;
    for (int q = 0; q < 5; ++q) {
      if (!ext[wx * n + (jj < 0 ? q : n - 1 - q)]) return false;
      if (!ext[wy * n + (ii < 0 ? q : n - 1 - q)]) return false;
    }
    return true;
  }
  if (ii >= n) return ext[1 * n + jj] != 0;
  if (ii < 0) return ext[3 * n + jj] != 0;
  if (jj >= n) return ext[2 * n + ii] != 0;
  return ext[0 * n + ii] != 0;
}

CC_HD inline uint8_t kind_of(const uint8_t* type, const uint8_t* ext, int n, bool cross, int k) {
  if (type[k] == T_EMPTY) return K_EMPTY_;
  const int i = k % n, j = k / n;
  bool sfv = type[k] == T_FULL;
  for (int dj = -2; dj <= 2 && sfv; ++dj)
    for (int di = -2; di <= 2 && sfv; ++di) {
      if (!cross && di && dj) continue;
      const int ii = i + di, jj = j + dj;
      if (ii >= 0 && jj >= 0 && ii < n && jj < n) sfv = type[jj * n + ii] == T_FULL;
      else sfv = ghost_ok(ext, n, ii, jj);
    }
  return sfv ? K_SFV_ : K_PLG_;
}

// --- the poised lattice of PLG cell k -----------------------------------------
// Five grid lines (rows, or else columns) of the search box carry 5, 4, 3, 2
// and 1 present cells; a cell at offset (u, v) costs u^2 + v^2, plus
// kCutPenalty for a cut cell other than k; each line takes its cheapest
// cells (ties: smaller u); the lines and counts minimise the total cost,
// ties to the lexicographically larger count vector from the lowest line up;
// rows before columns on equal cost; the 9 x 9 box first, then 11 x 11 and
// 13 x 13 where a smaller one holds no such set, and then the far search
// (plg_lattice_far).  out: the 15 cells, sorted.
// The cheapest lattice of the box of half-width R on lines of one orientation
// (0: rows, 1: columns), sorted; its cost in *cost_out; false if none.  RM
// is the largest half-width the arrays hold (R <= RM); the result does not
// depend on it.
template <int RM = kLatR>
CC_HD inline bool plg_lattice_box(const uint8_t* type, int n, int k, int R, int orient, int out[15],
                                   int* cost_out) {
  constexpr int kLatW = 2 * RM + 1;
  const int i0 = k % n, j0 = k / n;
  struct St { int cost; int8_t have; int8_t asg[kLatW]; };
  int8_t avail[kLatW][kLatW];
  int8_t navail[kLatW];
  int16_t cost[kLatW][kLatW];
  for (int v = -R; v <= R; ++v) {
    const int vi = v + RM;
    int na = 0;
    for (int u = -R; u <= R; ++u) {
      const int di = orient == 0 ? u : v, dj = orient == 0 ? v : u;
      const int ii = i0 + di, jj = j0 + dj;
      if (ii >= 0 && jj >= 0 && ii < n && jj < n && type[jj * n + ii] != T_EMPTY) {
        const bool cut = type[jj * n + ii] == T_CUT && (di != 0 || dj != 0);
        cost[vi][u + RM] = (int16_t)(u * u + v * v + (cut ? kCutPenalty : 0));
        // insertion by (cost, u); u grows, so equal costs keep their order
        int p = na++;
        while (p > 0 && cost[vi][avail[vi][p - 1] + RM] > cost[vi][u + RM]) {
          avail[vi][p] = avail[vi][p - 1];
          --p;
        }
        avail[vi][p] = (int8_t)u;
      }
    }
    navail[vi] = (int8_t)na;
  }
  St nxt[32], cur[32];
  for (int m = 0; m < 32; ++m) {
    nxt[m].have = 0;
    nxt[m].cost = 0;
    for (int q = 0; q < kLatW; ++q) nxt[m].asg[q] = 0;
  }
  nxt[31].have = 1;
  CC_ROLLED
  for (int v = R; v >= -R; --v) {
    const int vi = v + RM;
    CC_ROLLED
    for (int mask = 0; mask < 32; ++mask) {
      St& b = cur[mask];
      b.have = 0;
      // candidate (cost c, count cn on line v, the rest from state s)
      auto consider = [&](int c, int cn, const St& s) {
        bool better = !b.have || c < b.cost;
        if (b.have && c == b.cost) {
          // keys: (-count of line v, -count of line v+1, ...), smaller wins
          int cmp = 0;
          for (int w = vi; w < kLatW && cmp == 0; ++w) {
            const int ka = -(w == vi ? cn : s.asg[w]), kb = -b.asg[w];
            cmp = ka < kb ? -1 : ka > kb ? 1 : 0;
          }
          better = cmp < 0;
        }
        if (better) {
          b.have = 1;
          b.cost = c;
          for (int w = 0; w < kLatW; ++w) b.asg[w] = s.asg[w];
          b.asg[vi] = (int8_t)cn;
        }
      };
      if (nxt[mask].have) consider(nxt[mask].cost, 0, nxt[mask]);
      for (int bit = 0; bit < 5; ++bit) {
        const int cnt = 5 - bit;
        if (((mask >> bit) & 1) || navail[vi] < cnt) continue;
        const int m2 = mask | (1 << bit);
        if (!nxt[m2].have) continue;
        int rc = 0;
        for (int q = 0; q < cnt; ++q) rc += cost[vi][avail[vi][q] + RM];
        consider(nxt[m2].cost + rc, cnt, nxt[m2]);
      }
    }
    for (int m = 0; m < 32; ++m) nxt[m] = cur[m];
  }
  if (!nxt[0].have) return false;
  *cost_out = nxt[0].cost;
  int c = 0;
  for (int v = -R; v <= R; ++v) {
    const int vi = v + RM, cnt = nxt[0].asg[vi];
    for (int q = 0; q < cnt; ++q) {
      const int u = avail[vi][q];
      const int di = orient == 0 ? u : v, dj = orient == 0 ? v : u;
      out[c++] = (j0 + dj) * n + (i0 + di);
    }
  }
  for (int a = 1; a < 15; ++a) {
    const int x = out[a];
    int p = a;
    while (p > 0 && out[p - 1] > x) { out[p] = out[p - 1]; --p; }
    out[p] = x;
  }
  return true;
}

// The rule's lattice: the 9 x 9 box first, then 11 x 11 and 13 x 13 where a
// smaller one holds no such set; rows before columns on equal cost.
CC_HD inline bool plg_lattice(const uint8_t* type, int n, int k, int out[15]) {
  bool found = false;
  int best_cost = 0;
  CC_ROLLED
  for (int R = kLatR0; R <= kLatR && !found; ++R)
    for (int orient = 0; orient < 2; ++orient) {
      int tmp[15], c = 0;
      if (!plg_lattice_box(type, n, k, R, orient, tmp, &c)) continue;
      if (!found || c < best_cost) {
        found = true;
        best_cost = c;
        for (int q = 0; q < 15; ++q) out[q] = tmp[q];
      }
    }
  return found;
}

// The far search of the rule, where the 13 x 13 box holds no lattice (a
// cell near the tip of a thin wedge between two holes): the boxes 15 x 15 to
// 25 x 25 in turn, rows before columns on equal cost, as above.  Host only
// (its arrays are four times those of the first search).
inline bool plg_lattice_far(const uint8_t* type, int n, int k, int out[15]) {
  for (int R = kLatR + 1; R <= kLatRFar; ++R) {
    bool found = false;
    int best_cost = 0;
    for (int orient = 0; orient < 2; ++orient) {
      int tmp[15], c = 0;
      if (!plg_lattice_box<kLatRFar>(type, n, k, R, orient, tmp, &c)) continue;
      if (!found || c < best_cost) {
        found = true;
        best_cost = c;
        for (int q = 0; q < 15; ++q) out[q] = tmp[q];
      }
    }
    if (found) return true;
  }
  return false;
}

// --- moments ---------------------------------------------------------------
// moments of the full unit cell about its centre: (1/2)^p / (p + 1) for even
// p (0 for odd), times the same in q
CC_HD inline void full_moments(double out[kNM]) {
  for (int d = 0; d <= 6; ++d)
    for (int q = 0; q <= d; ++q) {
      const int p = d - q;
      const double mp = (p % 2) ? 0.0 : ipow(0.5, p) / (p + 1);
      const double mq = (q % 2) ? 0.0 : ipow(0.5, q) / (q + 1);
      out[mi(p, q)] = mp * mq;
    }
}

// scaled moments about the centre p moved to p - (dx, dy) h
CC_HD inline void shift_moments(const double in[kNM], double dx, double dy, double out[kNM]) {
  double C[7][7];
  for (int a = 0; a < 7; ++a) {
    for (int b = 0; b < 7; ++b) C[a][b] = 0.0;
    C[a][0] = C[a][a] = 1.0;
    for (int b = 1; b < a; ++b) C[a][b] = C[a - 1][b - 1] + C[a - 1][b];
  }
  double px[7], py[7];
  px[0] = py[0] = 1;
  for (int k = 1; k < 7; ++k) { px[k] = px[k - 1] * dx; py[k] = py[k - 1] * dy; }
  CC_ROLLED
  for (int d = 0; d <= 6; ++d)
    for (int q = 0; q <= d; ++q) {
      const int p = d - q;
      double s = 0;
      for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= q; ++b) s += C[p][a] * C[q][b] * px[p - a] * py[q - b] * in[mi(a, b)];
      out[mi(p, q)] = s;
    }
}

// --- small dense solves ----------------------------------------------------
// A x = b, A 15 x 15 row-major (overwritten), Gaussian elimination with
// partial pivoting; b becomes x.  false if a pivot is zero.
CC_HD inline bool lu_solve15(double* A, double* b) {
  const int n = 15;
  CC_ROLLED
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) { double t = A[p * n + k]; A[p * n + k] = A[c * n + k]; A[c * n + k] = t; }
      double t = b[p]; b[p] = b[c]; b[c] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      const double l = A[r * n + c] / A[c * n + c];
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

// Minimum 2-norm solution x[16] of B x = rhs, B 15 x 16 row-major of full
// row rank: Householder QR of B^T = Q R, then x = Q (R^-T rhs).
CC_HD inline bool min_norm15x16(const double* B, const double* rhs, double* x) {
  const int m = 15, n = 16;
  double T[15][16];     // T[r] = column r of B^T = row r of B
  double V[15][16];
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < n; ++c) T[r][c] = B[r * n + c];
  CC_ROLLED
  for (int k = 0; k < m; ++k) {
    double nrm = 0;
    for (int i = k; i < n; ++i) nrm += T[k][i] * T[k][i];
    nrm = sqrt(nrm);
    if (nrm == 0.0) return false;
    const double alpha = T[k][k] > 0 ? -nrm : nrm;
    for (int i = 0; i < n; ++i) V[k][i] = i >= k ? T[k][i] : 0.0;
    V[k][k] -= alpha;
    double vn = 0;
    for (int i = k; i < n; ++i) vn += V[k][i] * V[k][i];
    for (int j = k; j < m; ++j) {
      double s = 0;
      for (int i = k; i < n; ++i) s += V[k][i] * T[j][i];
      s = 2.0 * s / vn;
      for (int i = k; i < n; ++i) T[j][i] -= s * V[k][i];
    }
  }
  // R^T y = rhs (forward), R(i, j) = T[j][i] for i <= j
  double y[15];
  for (int i = 0; i < m; ++i) {
    double s = rhs[i];
    for (int j = 0; j < i; ++j) s -= T[i][j] * y[j];
    if (T[i][i] == 0.0) return false;
    y[i] = s / T[i][i];
  }
  // x = Q [y; 0] = H_0 H_1 ... H_14 [y; 0]
  for (int i = 0; i < n; ++i) x[i] = i < m ? y[i] : 0.0;
  CC_ROLLED
  for (int k = m - 1; k >= 0; --k) {
    double vn = 0, s = 0;
    for (int i = k; i < n; ++i) { vn += V[k][i] * V[k][i]; s += V[k][i] * x[i]; }
    s = 2.0 * s / vn;
    for (int i = k; i < n; ++i) x[i] -= s * V[k][i];
  }
  return true;
}

// --- the fit of PLG cell k (Sec. 4.2) -----------------------------------------
// Columns: the 15 lattice cells (their scaled moments about k's centre give
// the cell averages of the 15 monomials of degree <= 4), plus, for a cut cell
// with boundary data, the averaged boundary functional alpha1 phi + alpha2
// dphi/dn over its boundary nodes.  Rows: the monomials, degree by degree,
// x^d first.  rhs: <L phi>_k.  Square system: Eq. 4.14; with the boundary
// column: the weighted minimum norm of Eq. 4.17-4.18 with weights
// w = max(|offset|, 1/2) (1/2 for the boundary column), computed as
// beta = W^1/2 pinv(M W^1/2) rhs.  mom(kj, out) gives the scaled moments of
// cell kj about its own centre; a12[2 bc + 0/1] = (alpha1, alpha2) of
// condition bc.  beta[15] is 0 without boundary data.  false if singular.
template <class Mom>
CC_HD inline bool plg_fit(int k, int n, double h, double a, double b, double c, const int lat[15],
                          const Mom& mom, const BNode* bn, int nb, const double* a12,
                          double x0, double y0, double beta[16]) {
  const int i0 = k % n, j0 = k / n;
  const bool withb = nb > 0;
  const int nc = withb ? 16 : 15;
  double M[15 * 16], rhs[15];
  CC_ROLLED
  for (int col = 0; col < 15; ++col) {
    const int kj = lat[col];
    double m0[kNM], ms[kNM];
    mom(kj, m0);
    shift_moments(m0, (double)((kj % n) - i0), (double)((kj / n) - j0), ms);
    int r = 0;
    for (int d = 0; d <= 4; ++d)
      for (int p = d; p >= 0; --p, ++r) M[r * nc + col] = ms[mi(p, d - p)] / ms[0];
  }
  {
    double m[kNM];
    mom(k, m);
    int r = 0;
    for (int d = 0; d <= 4; ++d)
      for (int p = d; p >= 0; --p, ++r) {
        const int q = d - p;
        double v = 0;
        if (p >= 2) v += a * p * (p - 1) * (m[mi(p - 2, q)] / m[0]);
        if (p >= 1 && q >= 1) v += b * p * q * (m[mi(p - 1, q - 1)] / m[0]);
        if (q >= 2) v += c * q * (q - 1) * (m[mi(p, q - 2)] / m[0]);
        rhs[r] = v / (h * h);
      }
  }
  if (!withb) {
    if (!lu_solve15(M, rhs)) return false;
    for (int col = 0; col < 15; ++col) beta[col] = rhs[col];
    beta[15] = 0.0;
    return true;
  }
  const double px = x0 + (i0 + 0.5) * h, py = y0 + (j0 + 0.5) * h;
  double colb[15], ws = 0;
  for (int r = 0; r < 15; ++r) colb[r] = 0.0;
  CC_ROLLED
  for (int s = 0; s < nb; ++s) {
    const BNode& nd = bn[s];
    const double a1 = a12[2 * nd.bc], a2 = a12[2 * nd.bc + 1];
    const double X = (nd.x - px) / h, Y = (nd.y - py) / h;
    int r = 0;
    for (int d = 0; d <= 4; ++d)
      for (int p = d; p >= 0; --p, ++r) {
        const int q = d - p;
        const double phi = ipow(X, p) * ipow(Y, q);
        const double gx = p ? p * ipow(X, p - 1) * ipow(Y, q) / h : 0.0;
        const double gy = q ? q * ipow(X, p) * ipow(Y, q - 1) / h : 0.0;
        colb[r] += nd.w * (a1 * phi + a2 * (gx * nd.nx + gy * nd.ny));
      }
    ws += nd.w;
  }
  for (int r = 0; r < 15; ++r) M[r * 16 + 15] = colb[r] / ws;
  double sw[16];
  for (int col = 0; col < 15; ++col) {
    const int kj = lat[col];
    const int di = kj % n - i0, dj = kj / n - j0;
    const double d = sqrt((double)(di * di + dj * dj));
    sw[col] = 1.0 / sqrt(d > 0.5 ? d : 0.5);
  }
  sw[15] = 1.0 / sqrt(0.5);
  for (int r = 0; r < 15; ++r)
    for (int col = 0; col < 16; ++col) M[r * 16 + col] *= sw[col];
  double g[16];
  if (!min_norm15x16(M, rhs, g)) return false;
  for (int col = 0; col < 16; ++col) beta[col] = sw[col] * g[col];
  return true;
}

// --- moments of a cut cell (Sec. 4.2) -----------------------------------------
// Quadrature points along a piece: fn(x, y, dx w, dy w) for each node.
template <class F>
CC_HD inline void walk_piece(const Hole* holes, const Piece& pc, const Rules510& R, F&& fn) {
  if (!pc.arc) {
    for (int q = 0; q < 5; ++q) {
      const double tau = 0.5 * (R.sx[q] + 1.0), wt = 0.5 * R.sw[q];
      fn(pc.xa + tau * (pc.xb - pc.xa), pc.ya + tau * (pc.yb - pc.ya), (pc.xb - pc.xa) * wt,
         (pc.yb - pc.ya) * wt);
    }
    return;
  }
  const Hole& H = holes[pc.hole];
  int nsub = (int)ceil(fabs(pc.tb - pc.ta) / 0.25);
  if (nsub < 1) nsub = 1;
  CC_ROLLED
  for (int s = 0; s < nsub; ++s) {
    const double s0 = pc.ta + (pc.tb - pc.ta) * s / nsub, s1 = pc.ta + (pc.tb - pc.ta) * (s + 1) / nsub;
    for (int q = 0; q < 10; ++q) {
      const double t = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * R.ax[q];
      const double wt = 0.5 * (s1 - s0) * R.aw[q];
      double x, y, dx, dy;
      H.at(t, x, y);
      H.dat(t, dx, dy);
      fn(x, y, dx * wt, dy * wt);
    }
  }
}

// adds the scaled moments integral X^p Y^q dX dY (X = (x - px)/h, Y the
// same) of the piece's contribution by Green's theorem: the contour
// integral of X^(p+1) Y^q / (p+1) dY
CC_HD inline void piece_moments(const Hole* holes, const Piece& pc, double px, double py, double h,
                                const Rules510& R, double m[kNM]) {
  walk_piece(holes, pc, R, [&](double x, double y, double, double dy) {
    const double X = (x - px) / h, Y = (y - py) / h, dY = dy / h;
    double xp[8], yq[7];
    xp[0] = 1;
    yq[0] = 1;
    for (int k = 1; k < 8; ++k) xp[k] = xp[k - 1] * X;
    for (int k = 1; k < 7; ++k) yq[k] = yq[k - 1] * Y;
    for (int d = 0; d <= 6; ++d)
      for (int q = 0; q <= d; ++q) {
        const int p = d - q;
        m[mi(p, q)] += xp[p + 1] * yq[q] * dY / (p + 1);
      }
  });
}

// --- Def. 5.1 ordering: the nearest of ns samples (sx, sy) of one curve to
// (x, y), by squared distance (ties: the first); returns its index and
// writes the squared distance
CC_HD inline int nearest_sample(const double* sx, const double* sy, int ns, double x, double y,
                                double* d2out) {
  int best = 0;
  double bd = 0;
  for (int s = 0; s < ns; ++s) {
    const double dx = sx[s] - x, dy = sy[s] - y;
    const double d2 = dx * dx + dy * dy;
    if (s == 0 || d2 < bd) { bd = d2; best = s; }
  }
  *d2out = bd;
  return best;
}

}  // namespace cell
}  // namespace ccmg
