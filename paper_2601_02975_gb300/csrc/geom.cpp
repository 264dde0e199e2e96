// Cut cells of a box minus a union of ellipses (Sec. 3.1) and the merging of
// small cells (the merging step of Alg. 1), in FP64 on the host.
//
// A cut cell is described by its oriented boundary pieces: the parts of its
// four faces that lie in the domain (counter-clockwise) and the arcs of hole
// boundaries inside it (clockwise around the hole), so the cell is on the
// left of every piece.  Area integrals then follow from Green's theorem,
//   integral_C X^p Y^q dA = contour integral X^(p+1) Y^q / (p+1) dY,
// in the scaled coordinates X = (x - px)/h, Y = (y - py)/h about the centre
// of the control volume (Sec. 4.2, quadrature paragraph).  Faces are
// integrated by 5-point Gauss-Legendre (exact for these polynomials), arcs by
// 10-point Gauss-Legendre on sub-arcs of at most 0.25 rad.
//
// The merging step of Alg. 1 is applied once in row-major order (y index outer) with
// the current volumes; the merge target is a present neighbour reached
// through a shared face piece of positive length (following the chain of
// earlier merges), minimising |vol + vol' - h^2|, ties (scores within
// 1e-9 h^2 of the smallest) to the first of the neighbours in the order
// -x, +x, -y, +y.  A level whose cut cells have more
// than one connected component violates the precondition of Alg. 1 and is
// marked unresolved.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <set>

#include "setup.h"

namespace ccmg {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

namespace {


struct Rules {
  std::vector<double> sx, sw, ax, aw, ix, iw;
  Rules510 r510;
  Rules() {
    gauss_legendre(5, sx, sw);
    gauss_legendre(10, ax, aw);
    gauss_legendre(6, ix, iw);
    std::copy(sx.begin(), sx.end(), r510.sx);
    std::copy(sw.begin(), sw.end(), r510.sw);
    std::copy(ax.begin(), ax.end(), r510.ax);
    std::copy(aw.begin(), aw.end(), r510.aw);
  }
};
const Rules& rules() {
  static Rules r;
  return r;
}


// Quadrature points along a piece: position and the vector weight (dx, dy).
template <class F>
void walk(const Problem& P, const Piece& pc, F&& fn) {
  cell::walk_piece(P.holes.data(), pc, rules().r510, fn);
}

void piece_moments(const Problem& P, const Piece& pc, double px, double py, double h,
                   double m[kMoments]) {
  cell::piece_moments(P.holes.data(), pc, px, py, h, rules().r510, m);
}

// parameters t in [0, 2pi) with A cos t + B sin t = C
void trig_roots(double A, double B, double C, std::vector<double>& out) {
  double R = std::hypot(A, B);
  if (std::fabs(C) >= R) return;
  double phi = std::atan2(B, A), d = std::acos(C / R);
  for (double t : {phi + d, phi - d}) {
    t = std::fmod(t, kTwoPi);
    if (t < 0) t += kTwoPi;
    out.push_back(t);
  }
}

// Crossings of a flower with the grid line x = c (axis 0) or y = c (axis 1).
// Between consecutive extrema of the coordinate (cyclically) the coordinate
// is monotone, so each such arc crosses the line at most once; the crossing
// is refined by bisection.  A line met only at an extremum is touched, not
// crossed (tips and valleys of the flower lie on grid lines), and gives none.
double bisect_root(const std::function<double(double)>& f, double a, double b) {
  double fa = f(a);
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b), fm = f(m);
    if (fm == 0.0 || b - a < 1e-15) return m;
    if ((fm < 0) == (fa < 0)) { a = m; fa = fm; } else { b = m; }
  }
  return 0.5 * (a + b);
}

// parameters in [0, 2pi) where coordinate `axis` of the flower is extremal
std::vector<double> flower_extrema(const Hole& H, int axis) {
  const int ns = 4096;
  std::function<double(double)> d = [&](double t) {
    double dx, dy;
    H.dat(t, dx, dy);
    return axis == 0 ? dx : dy;
  };
  std::vector<double> out;
  double d0 = d(0.0);
  for (int k = 0; k < ns; ++k) {
    const double ta = kTwoPi * k / ns, tb = kTwoPi * (k + 1) / ns, d1 = d(tb);
    if (d0 == 0.0) out.push_back(ta);
    else if (d0 * d1 < 0.0) out.push_back(bisect_root(d, ta, tb));
    d0 = d1;
  }
  return out;
}

void flower_line_roots(const Hole& H, int axis, double c, std::vector<double>& out) {
  const double tol = 1e-13;
  const std::vector<double> ext = flower_extrema(H, axis);
  std::function<double(double)> f = [&](double t) {
    double x, y;
    H.at(t, x, y);
    return (axis == 0 ? x : y) - c;
  };
  std::vector<double> r;
  const size_t m = ext.size();
  for (size_t q = 0; q < m; ++q) {
    const double a = ext[q], b = q + 1 < m ? ext[q + 1] : ext[0] + kTwoPi;
    const double fa = f(a), fb = f(b);
    if (std::fabs(fa) <= tol || std::fabs(fb) <= tol || fa * fb > 0.0) continue;
    double t = std::fmod(bisect_root(f, a, b), kTwoPi);
    if (t < 0.0 || t >= kTwoPi) t = 0.0;
    r.push_back(t);
  }
  std::sort(r.begin(), r.end());
  r.erase(std::unique(r.begin(), r.end()), r.end());
  out.insert(out.end(), r.begin(), r.end());
}

// Crossings of a kind-2 hole's sides with the grid line x = c (axis 0) or
// y = c (axis 1): one per side whose ends lie strictly on the two sides of
// the line; a corner on the line (within 1e-13) is a crossing when its two
// sides leave to the two sides of the line, and is only touched otherwise.
void rect_line_roots(const Hole& H, int axis, double c, std::vector<double>& out) {
  const double tol = 1e-13, q = kTwoPi / 4;
  double vx[4], vy[4];
  H.corners_cw(vx, vy);
  const double* v = axis == 0 ? vx : vy;
  for (int k = 0; k < 4; ++k) {
    const double f0 = v[k] - c, fp = v[(k + 3) % 4] - c, f1 = v[(k + 1) % 4] - c;
    if (std::fabs(f0) <= tol) {
      if (fp * f1 < 0.0 && std::fabs(fp) > tol && std::fabs(f1) > tol) out.push_back(k * q);
      continue;
    }
    if (std::fabs(f1) <= tol || f0 * f1 > 0.0) continue;
    out.push_back(k * q + q * f0 / (f0 - f1));
  }
}

// crossings of hole i with hole j: bracket sign changes of j's level function
// along i, then refine with the Illinois variant of regula falsi
void hole_crossings(const Hole& hi, const Hole& hj, std::vector<double>& out) {
  const int ns = 3000;
  auto f = [&](double t) {
    double x, y;
    hi.at(t, x, y);
    return hj.level(x, y);
  };
  double ta = 0, fa = f(0);
  for (int s = 1; s <= ns; ++s) {
    double tb = kTwoPi * s / ns, fb = f(tb);
    if (fa == 0.0) {
      out.push_back(ta);
    } else if ((fa < 0) != (fb < 0) && fb != 0.0) {
      double a = ta, b = tb, ya = fa, yb = fb;
      int side = 0;
      for (int it = 0; it < 200 && b - a > 1e-16; ++it) {
        double m = (a * yb - b * ya) / (yb - ya);
        if (!(m > a && m < b)) m = 0.5 * (a + b);
        double ym = f(m);
        if (ym == 0.0) { a = b = m; break; }
        if ((ym < 0) == (ya < 0)) {
          a = m; ya = ym;
          if (side == -1) yb *= 0.5;
          side = -1;
        } else {
          b = m; yb = ym;
          if (side == 1) ya *= 0.5;
          side = 1;
        }
      }
      out.push_back(0.5 * (a + b));
    }
    ta = tb;
    fa = fb;
  }
}

bool outside_all(const Problem& P, double x, double y, int skip = -1) {
  for (size_t k = 0; k < P.holes.size(); ++k)
    if ((int)k != skip && P.holes[k].level(x, y) <= 0.0) return false;
  return true;
}

// The closed loops the pieces form (the connected components of a cut cell):
// each as its pieces in chaining order and its scaled area, in the order of
// their first pieces.
struct Loop { std::vector<int> idx; double area; };

std::vector<Loop> chain_loops(const Problem& P, const std::vector<Piece>& pcs, double px, double py,
                              double h) {
  std::vector<Loop> out;
  std::vector<char> used(pcs.size(), 0);
  const double tol = 1e-10 * h;
  for (size_t s = 0; s < pcs.size(); ++s) {
    if (used[s]) continue;
    used[s] = 1;
    Loop L;
    L.idx.push_back((int)s);
    double m[kMoments];
    std::fill(m, m + kMoments, 0.0);
    piece_moments(P, pcs[s], px, py, h, m);
    double ex = pcs[s].xb, ey = pcs[s].yb;
    int guard = 0;
    while (std::hypot(ex - pcs[s].xa, ey - pcs[s].ya) > tol) {
      int nxt = -1;
      for (size_t q = 0; q < pcs.size(); ++q)
        if (!used[q] && std::hypot(pcs[q].xa - ex, pcs[q].ya - ey) <= tol) {
          nxt = (int)q;
          break;
        }
      if (nxt < 0 || ++guard > 100000)
        throw SetupError(2, "cut-cell boundary pieces do not close");
      used[nxt] = 1;
      L.idx.push_back(nxt);
      piece_moments(P, pcs[nxt], px, py, h, m);
      ex = pcs[nxt].xb;
      ey = pcs[nxt].yb;
    }
    L.area = m[0];
    out.push_back(std::move(L));
  }
  return out;
}

}  // namespace

void shift_moments(const double in[kMoments], double dx, double dy, double out[kMoments]) {
  cell::shift_moments(in, dx, dy, out);
}

void LevelGeom::moments(int k, double out[kMoments]) const {
  auto it = cut.find(k);
  if (it != cut.end()) {
    std::copy(it->second.mom, it->second.mom + kMoments, out);
    return;
  }
  cell::full_moments(out);
}

static std::vector<Piece> full_faces(const LevelGeom& G, int i, int j) {
  int n = G.n;
  double xl = G.x0 + i * G.h, xr = xl + G.h, yb = G.y0 + j * G.h, yt = yb + G.h;
  std::vector<Piece> v;
  v.push_back({false, xl, yb, xr, yb, -1, 0, 0, j == 0 ? 0 : -1, 0});
  v.push_back({false, xr, yb, xr, yt, -1, 0, 0, i == n - 1 ? 1 : -1, 1});
  v.push_back({false, xr, yt, xl, yt, -1, 0, 0, j == n - 1 ? 2 : -1, 2});
  v.push_back({false, xl, yt, xl, yb, -1, 0, 0, i == 0 ? 3 : -1, 3});
  return v;
}

// Alg. 1's choice of a neighbour: the candidate whose volume with vol_add
// comes closest to h^2.  Scores within 1e-9 h^2 of the smallest are ties
// (they differ by rounding only, e.g. the mirror cells on a diagonal of a
// disk): the first such candidate wins, so the choice does not depend on
// rounding.
static int closest_to_h2(const LevelGeom& G, const std::vector<int>& cand, double vol_add) {
  const double h2 = G.h * G.h;
  std::vector<double> score(cand.size());
  double smin = 0;
  for (size_t q = 0; q < cand.size(); ++q) {
    score[q] = std::fabs(G.vol[cand[q]] + vol_add - h2);
    smin = q == 0 ? score[q] : std::min(smin, score[q]);
  }
  for (size_t q = 0; q < cand.size(); ++q)
    if (score[q] <= smin + 1e-9 * h2) return cand[q];
  return cand[0];
}

LevelGeom build_geometry(const Problem& P, int n, SetupDevice* dev) {
  LevelGeom G;
  G.n = n;
  G.x0 = P.x0;
  G.y0 = P.y0;
  G.h = (P.x1 - P.x0) / n;
  const double h = G.h;
  if (std::fabs((P.y1 - P.y0) - h * n) > 1e-12 * std::max(1.0, P.y1 - P.y0))
    throw SetupError(1, "the box must be square");
  const int nh = (int)P.holes.size();
  std::map<int, std::vector<Piece>> arcs;      // cell -> arcs
  std::map<int, std::vector<double>> vline;    // vertical line i -> y of crossings
  std::map<int, std::vector<double>> hline;    // horizontal line j -> x of crossings
  for (int e = 0; e < nh; ++e) {
    const Hole& H = P.holes[e];
    double hx = std::hypot(H.r1 * H.co, H.r2 * H.si), hy = std::hypot(H.r1 * H.si, H.r2 * H.co);
    double bx0 = H.cx - hx, bx1 = H.cx + hx, by0 = H.cy - hy, by1 = H.cy + hy;   // bounding box
    if (H.kind == 1) {
      bx0 = H.cx - H.r1 - H.r2; bx1 = H.cx + H.r1 + H.r2;
      by0 = H.cy - H.r1 - H.r2; by1 = H.cy + H.r1 + H.r2;
    } else if (H.kind == 2) {
      double vx[4], vy[4];
      H.corners_cw(vx, vy);
      bx0 = *std::min_element(vx, vx + 4); bx1 = *std::max_element(vx, vx + 4);
      by0 = *std::min_element(vy, vy + 4); by1 = *std::max_element(vy, vy + 4);
    }
    std::vector<double> ts;
    if (H.kind == 2)   // the corners are kinks: arcs end there
      for (int k = 0; k < 4; ++k) ts.push_back(k * kTwoPi / 4);
    int i0 = std::max(0, (int)std::floor((bx0 - P.x0) / h));
    int i1 = std::min(n, (int)std::ceil((bx1 - P.x0) / h));
    for (int i = i0; i <= i1; ++i) {
      std::vector<double> r;
      if (H.kind == 2) rect_line_roots(H, 0, P.x0 + i * h, r);
      else if (H.kind == 1) flower_line_roots(H, 0, P.x0 + i * h, r);
      else trig_roots(H.co * H.r1, -H.si * H.r2, P.x0 + i * h - H.cx, r);
      for (double t : r) {
        double x, y;
        H.at(t, x, y);
        ts.push_back(t);
        vline[i].push_back(y);
      }
    }
    int j0 = std::max(0, (int)std::floor((by0 - P.y0) / h));
    int j1 = std::min(n, (int)std::ceil((by1 - P.y0) / h));
    for (int j = j0; j <= j1; ++j) {
      std::vector<double> r;
      if (H.kind == 2) rect_line_roots(H, 1, P.y0 + j * h, r);
      else if (H.kind == 1) flower_line_roots(H, 1, P.y0 + j * h, r);
      else trig_roots(H.si * H.r1, H.co * H.r2, P.y0 + j * h - H.cy, r);
      for (double t : r) {
        double x, y;
        H.at(t, x, y);
        ts.push_back(t);
        hline[j].push_back(x);
      }
    }
    for (int f = 0; f < nh; ++f)
      if (f != e) hole_crossings(H, P.holes[f], ts);
    std::sort(ts.begin(), ts.end());
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    std::vector<std::pair<double, double>> segs;   // (from, to), from > to
    if (ts.empty()) {
      segs.push_back({kTwoPi, 0.0});
    } else {
      for (size_t k = 0; k < ts.size(); ++k) {
        double lo = ts[k], hi = (k + 1 < ts.size()) ? ts[k + 1] : ts[0] + kTwoPi;
        segs.push_back({hi, lo});
      }
    }
    for (auto& sg : segs) {
      double tm = 0.5 * (sg.first + sg.second), xm, ym;
      H.at(tm, xm, ym);
      if (!outside_all(P, xm, ym, e)) continue;
      int ii = (int)std::floor((xm - P.x0) / h), jj = (int)std::floor((ym - P.y0) / h);
      if (ii < 0 || jj < 0 || ii >= n || jj >= n) throw SetupError(2, "a hole leaves the box");
      Piece pc;
      pc.arc = true;
      pc.hole = e;
      pc.ta = sg.first;
      pc.tb = sg.second;
      H.at(pc.ta, pc.xa, pc.ya);
      H.at(pc.tb, pc.xb, pc.yb);
      pc.bc = 4 + e;
      pc.face = -1;
      arcs[jj * n + ii].push_back(pc);
    }
  }

  // the cells no curve crosses: full or empty by their centre
  G.type.assign((size_t)n * n, CT_EMPTY);
  G.vol.assign((size_t)n * n, 0.0);
  {
    std::vector<uint8_t> crossed((size_t)n * n, 0);
    for (auto& kv : arcs) crossed[kv.first] = 1;
    if (dev) {
      dev->classify(P, n, h, crossed.data(), G.type.data());
    } else {
      parallel_rows(n, [&](int j) {
        for (int i = 0; i < n; ++i) {
          const int k = j * n + i;
          if (crossed[k]) continue;
          const double xc = P.x0 + (i + 0.5) * h, yc = P.y0 + (j + 0.5) * h;
          if (cell::outside_all(P.holes.data(), (int)P.holes.size(), xc, yc)) G.type[k] = CT_FULL;
        }
      });
    }
    parallel_rows(n, [&](int j) {
      for (int k = j * n; k < (j + 1) * n; ++k)
        if (G.type[k] == CT_FULL) G.vol[k] = h * h;
    });
  }
  // the cut cells: boundary pieces and components here, moments below
  std::vector<int> ccell;
  std::vector<Cut> ccut;
  std::vector<double> cpx, cpy;
  struct Orphan { int k; std::vector<Piece> pcs; };
  std::vector<Orphan> orphans;   // the components a cell does not keep
  for (auto& kv : arcs) {
    int k = kv.first, j = k / n, i = k % n;
    double xl = P.x0 + i * h, xr = xl + h, yb = P.y0 + j * h, yt = yb + h;
    double px = xl + 0.5 * h, py = yb + 0.5 * h;
    Cut C;
    C.pieces = kv.second;
    for (int f = 0; f < 4; ++f) C.face[f] = false;
    // faces counter-clockwise: bottom, right, top, left
    struct E { double ax, ay, bx, by; bool horiz; const std::vector<double>* cr; int bc; };
    static const std::vector<double> none;
    auto crs = [&](std::map<int, std::vector<double>>& m, int key) -> const std::vector<double>* {
      auto it = m.find(key);
      return it == m.end() ? &none : &it->second;
    };
    E edges[4] = {{xl, yb, xr, yb, true, crs(hline, j), j == 0 ? 0 : -1},
                  {xr, yb, xr, yt, false, crs(vline, i + 1), i == n - 1 ? 1 : -1},
                  {xr, yt, xl, yt, true, crs(hline, j + 1), j == n - 1 ? 2 : -1},
                  {xl, yt, xl, yb, false, crs(vline, i), i == 0 ? 3 : -1}};
    for (int f = 0; f < 4; ++f) {
      const E& ed = edges[f];
      double ca = ed.horiz ? ed.ax : ed.ay, cb = ed.horiz ? ed.bx : ed.by;
      double lo = std::min(ca, cb), hi = std::max(ca, cb);
      std::vector<double> pts{lo};
      for (double v : *ed.cr)
        if (v > lo && v < hi) pts.push_back(v);
      pts.push_back(hi);
      std::sort(pts.begin(), pts.end());
      if (ca > cb) std::reverse(pts.begin(), pts.end());
      for (size_t s = 0; s + 1 < pts.size(); ++s) {
        Piece pc;
        pc.arc = false;
        pc.hole = -1;
        pc.ta = pc.tb = 0;
        if (ed.horiz) { pc.xa = pts[s]; pc.xb = pts[s + 1]; pc.ya = pc.yb = ed.ay; }
        else { pc.ya = pts[s]; pc.yb = pts[s + 1]; pc.xa = pc.xb = ed.ax; }
        if (!outside_all(P, 0.5 * (pc.xa + pc.xb), 0.5 * (pc.ya + pc.yb))) continue;
        pc.bc = ed.bc;
        pc.face = f;
        C.pieces.push_back(pc);
        C.face[f] = true;
      }
    }
    std::vector<Loop> loops = chain_loops(P, C.pieces, px, py, h);
    int n_out = 0;
    for (const Loop& L : loops) n_out += L.area > 0;
    const int n_in = (int)loops.size() - n_out;
    if (n_out >= 2 && n_in == 0) {
      // Alg. 1, cells of several components: the largest stays (its pieces
      // in chaining order), the others join a face neighbour below
      size_t big = 0;
      for (size_t q = 1; q < loops.size(); ++q)
        if (loops[q].area > loops[big].area) big = q;
      for (size_t q = 0; q < loops.size(); ++q) {
        if (q == big) continue;
        Orphan O{k, {}};
        for (int t : loops[q].idx) O.pcs.push_back(C.pieces[t]);
        orphans.push_back(std::move(O));
      }
      std::vector<Piece> keep;
      for (int t : loops[big].idx) keep.push_back(C.pieces[t]);
      C.pieces.swap(keep);
      for (int f = 0; f < 4; ++f) C.face[f] = false;
      for (const Piece& pc : C.pieces)
        if (!pc.arc) C.face[pc.face] = true;
    } else if (n_out != 1) {
      G.resolved = false;
      G.reason = "cell (" + std::to_string(i) + "," + std::to_string(j) + ") has " +
                 std::to_string(n_out) + " components";
    }
    ccell.push_back(k);
    ccut.push_back(std::move(C));
    cpx.push_back(px);
    cpy.push_back(py);
  }
  {
    const int nc = (int)ccell.size();
    std::vector<double> mom((size_t)nc * kMoments, 0.0);
    if (dev && nc) {
      std::vector<Piece> pcs;
      std::vector<int> ptr(1, 0);
      for (const Cut& C : ccut) {
        pcs.insert(pcs.end(), C.pieces.begin(), C.pieces.end());
        ptr.push_back((int)pcs.size());
      }
      dev->moments(P, h, ccell, pcs, ptr, cpx, cpy, quad_rules(), mom.data());
    } else {
      parallel_rows(nc, [&](int r) {
        for (const Piece& pc : ccut[r].pieces)
          cell::piece_moments(P.holes.data(), pc, cpx[r], cpy[r], h, quad_rules(), &mom[(size_t)r * kMoments]);
      }, 16);
    }
    for (int r = 0; r < nc; ++r) {
      Cut& C = ccut[r];
      std::copy(&mom[(size_t)r * kMoments], &mom[(size_t)r * kMoments] + kMoments, C.mom);
      if (C.mom[0] <= 0) continue;   // empty
      const int k = ccell[r];
      G.type[k] = CT_CUT;
      G.vol[k] = C.mom[0] * h * h;
      G.cut[k] = std::move(C);
    }
  }
  // Alg. 1, the other components of a cell: each joins the face neighbour
  // across one of its own face pieces (order -x, +x, -y, +y) whose volume
  // with it comes closest to h^2, near-ties to the first
  for (const Orphan& O : orphans) {
    const int k = O.k, i = k % n, j = k / n;
    const double px = P.x0 + (i + 0.5) * h, py = P.y0 + (j + 0.5) * h;
    double mk[kMoments];
    std::fill(mk, mk + kMoments, 0.0);
    for (const Piece& pc : O.pcs) piece_moments(P, pc, px, py, h, mk);
    const double vk = mk[0] * h * h;
    bool on[4] = {false, false, false, false};
    for (const Piece& pc : O.pcs)
      if (!pc.arc) on[pc.face] = true;
    static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1}, fidx[4] = {3, 1, 0, 2};
    std::vector<int> cand;
    for (int q = 0; q < 4; ++q) {
      const int ii = i + di[q], jj = j + dj[q];
      if (!on[fidx[q]] || ii < 0 || jj < 0 || ii >= n || jj >= n) continue;
      if (G.type[jj * n + ii] != CT_EMPTY) cand.push_back(jj * n + ii);
    }
    if (cand.empty()) {
      G.resolved = false;
      G.reason = "a component of cell (" + std::to_string(i) + "," + std::to_string(j) +
                 ") has no neighbour";
      continue;
    }
    const int best = closest_to_h2(G, cand, vk);
    const int bi = best % n, bj = best / n;
    if (!G.cut.count(best)) {
      Cut T;
      T.pieces = full_faces(G, bi, bj);
      for (int f = 0; f < 4; ++f) T.face[f] = true;
      cell::full_moments(T.mom);
      G.cut[best] = T;
    }
    Cut& T = G.cut[best];
    double sh[kMoments];
    shift_moments(mk, i - bi, j - bj, sh);
    for (int q = 0; q < kMoments; ++q) T.mom[q] += sh[q];
    T.pieces.insert(T.pieces.end(), O.pcs.begin(), O.pcs.end());
    G.vol[best] += vk;
    G.type[best] = CT_CUT;
  }

  // ---- Alg. 1, merging of small cells -----------------------------------------
  G.owner.assign((size_t)n * n, -1);
  parallel_rows(n, [&](int j) {
    for (int k = j * n; k < (j + 1) * n; ++k)
      if (G.type[k] != CT_EMPTY) G.owner[k] = k;
  });
  std::function<int(int)> root = [&](int k) {
    while (G.owner[k] != k) k = G.owner[k];
    return k;
  };
  const double h2 = h * h;
  // only cut cells can be small (a full cell has volume h^2), and merging
  // only grows cells: visiting the cut cells in index order is the row-major
  // pass over all cells
  std::vector<int> small_cand;
  for (const auto& kv : G.cut) small_cand.push_back(kv.first);
  for (int k : small_cand) {
    if (G.type[k] == CT_EMPTY || G.vol[k] >= P.eps * h2) continue;
    int i = k % n, j = k / n;
    const bool* face = G.cut.count(k) ? G.cut[k].face : nullptr;
    static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1}, fidx[4] = {3, 1, 0, 2};
    std::vector<int> cand;
    for (int q = 0; q < 4; ++q) {
      if (face && !face[fidx[q]]) continue;
      int ii = i + di[q], jj = j + dj[q];
      if (ii < 0 || jj < 0 || ii >= n || jj >= n) continue;
      int kk = jj * n + ii;
      if (G.owner[kk] < 0) continue;
      int t = root(kk);
      if (t != k && std::find(cand.begin(), cand.end(), t) == cand.end()) cand.push_back(t);
    }
    if (cand.empty()) throw SetupError(2, "a small cut cell has no neighbour to merge into");
    const int best = closest_to_h2(G, cand, G.vol[k]);
    int bi = best % n, bj = best / n;
    double mk[kMoments], mt[kMoments], sh[kMoments];
    G.moments(k, mk);
    G.moments(best, mt);
    shift_moments(mk, i - bi, j - bj, sh);
    if (!G.cut.count(best)) {
      Cut T;
      T.pieces = full_faces(G, bi, bj);
      for (int f = 0; f < 4; ++f) T.face[f] = true;
      std::copy(mt, mt + kMoments, T.mom);
      G.cut[best] = T;
    }
    Cut& T = G.cut[best];
    for (int q = 0; q < kMoments; ++q) T.mom[q] = mt[q] + sh[q];
    auto it = G.cut.find(k);
    if (it != G.cut.end()) {
      T.pieces.insert(T.pieces.end(), it->second.pieces.begin(), it->second.pieces.end());
      G.cut.erase(it);
    }
    G.vol[best] += G.vol[k];
    G.vol[k] = 0;
    G.type[k] = CT_EMPTY;
    G.type[best] = CT_CUT;
    G.owner[k] = best;
  }
  {
    std::vector<int> own(G.owner.size());
    parallel_rows(n, [&](int j) {
      for (int k = j * n; k < (j + 1) * n; ++k) own[k] = G.owner[k] >= 0 ? root(k) : -1;
    });
    G.owner.swap(own);
  }
  return G;
}

std::vector<BNode> boundary_nodes(const Problem& P, const LevelGeom& G, int k) {
  std::vector<BNode> out;
  auto it = G.cut.find(k);
  if (it == G.cut.end()) return out;
  for (const Piece& pc : it->second.pieces) {
    if (pc.bc < 0) continue;
    walk(P, pc, [&](double x, double y, double dx, double dy) {
      double ds = std::hypot(dx, dy);
      // the cell is on the left: the outward normal is the right-hand normal
      out.push_back({x, y, dy / ds, -dx / ds, ds, pc.bc});
    });
  }
  return out;
}

std::vector<std::array<double, 3>> volume_nodes(const Problem& P, const LevelGeom& G, int k) {
  std::vector<std::array<double, 3>> out;
  auto it = G.cut.find(k);
  if (it == G.cut.end()) return out;
  int i = k % G.n;
  double px = G.x0 + (i + 0.5) * G.h;
  const Rules& R = rules();
  double vol = G.vol[k];
  for (const Piece& pc : it->second.pieces) {
    walk(P, pc, [&](double x, double y, double, double dy) {
      if (dy == 0.0) return;
      double half = 0.5 * (x - px);
      for (size_t q = 0; q < R.ix.size(); ++q)
        out.push_back({px + half * (1.0 + R.ix[q]), y, dy * half * R.iw[q] / vol});
    });
  }
  return out;
}

const Rules510& quad_rules() { return rules().r510; }

}  // namespace ccmg
