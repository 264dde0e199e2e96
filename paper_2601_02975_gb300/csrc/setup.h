// Host-side (FP64) construction of the per-level tables: cut cells (Sec. 3),
// classification and fits (Sec. 4), block-smoother and bottom factorisations
// (Sec. 5).  Everything here runs once per domain in cc_setup.
#pragma once
#include <algorithm>
#include <array>
#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

namespace ccmg {

enum CellType : uint8_t { CT_EMPTY = 0, CT_FULL = 1, CT_CUT = 2 };
enum CellKind : uint8_t { K_EMPTY = 0, K_SFV = 1, K_PLG = 2 };
enum BcType { BC_D = 0, BC_N = 1, BC_R = 2 };

struct SetupError : std::runtime_error {
  int code;
  SetupError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

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
  void at(double t, double& x, double& y) const;
  void dat(double t, double& dx, double& dy) const;
  double level(double x, double y) const;   // < 0 inside the hole
  double halfwidth() const {
    return kind == 2 ? 1e300 : kind == 1 ? r1 - r2 : std::min(r1, r2);
  }
  void corners_cw(double vx[4], double vy[4]) const;   // kind 2, in the order of t
};

struct Bc { int type; double a1, a2; };

struct Problem {
  double x0, y0, x1, y1;
  std::vector<Hole> holes;
  std::vector<Bc> bc;   // 4 box sides (S, E, N, W), then one per hole
  double a, b, c;
  double eps;
};

// moment index of x^p y^q, p + q <= 6
constexpr int kMoments = 28;
inline int midx(int p, int q) { int d = p + q; return d * (d + 1) / 2 + q; }

struct Piece {           // oriented boundary piece of a cut cell
  bool arc;
  double xa, ya, xb, yb;  // end points (start, end)
  int hole;               // arcs
  double ta, tb;          // arcs: parameter from ta to tb (tb < ta)
  int bc;                 // index into Problem::bc, -1 for interior faces
};

struct BNode { double x, y, nx, ny, w; int bc; };

struct Cut {
  std::vector<Piece> pieces;
  double mom[kMoments];   // integral of X^p Y^q dX dY, X = (x - px)/h, about the own centre
  bool face[4];           // a face piece in the domain on bottom, right, top, left
};

struct LevelGeom {
  int n = 0;
  double h = 0, x0 = 0, y0 = 0;
  std::vector<uint8_t> type;   // CellType
  std::vector<double> vol;
  std::vector<int> owner;      // control volume -> cell holding it, -1 none
  std::map<int, Cut> cut;      // non-full present cells (ordered by index)
  bool resolved = true;
  std::string reason;
  void moments(int k, double out[kMoments]) const;
};

LevelGeom build_geometry(const Problem& P, int n);

// boundary quadrature of cut cell k (nodes on pieces with bc >= 0)
std::vector<BNode> boundary_nodes(const Problem& P, const LevelGeom& G, int k);
// volume quadrature of cut cell k: (x, y, w), sum w = 1
std::vector<std::array<double, 3>> volume_nodes(const Problem& P, const LevelGeom& G, int k);

// shift scaled moments from centre p to centre p - (dx, dy) h
void shift_moments(const double in[kMoments], double dx, double dy, double out[kMoments]);

// Gauss-Legendre rule on [-1, 1]
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// ---------------------------------------------------------------------------
struct SparseRows {            // CSR
  std::vector<int64_t> ptr{0};
  std::vector<int> col;
  std::vector<double> val;
  void push(const std::map<int, double>& row) {
    for (auto& kv : row) { col.push_back(kv.first); val.push_back(kv.second); }
    ptr.push_back((int64_t)col.size());
  }
  int rows() const { return (int)ptr.size() - 1; }
};

struct LevelDisc {
  int n = 0;
  double h = 0;
  LevelGeom geom;
  std::vector<uint8_t> kind;          // CellKind
  std::vector<int> plg;               // PLG cells, row-major
  std::vector<std::array<int, 15>> lattice;
  std::vector<std::array<double, 16>> beta;   // beta_1..15, beta_b
  std::vector<int> bd_cells;          // cut PLG cells with a boundary datum, row-major
  std::vector<int> bd_of_plg;         // per PLG cell: index into bd_cells or -1
  std::vector<int> block;             // exactly solved cells in solve order
  SparseRows block_rows;              // full row of A for each block cell (all columns)
  SparseRows nrows;                   // N: row r belongs to cell nrow_cell[r]
  std::vector<int> nrow_cell;
  double gc[4][2][5];                 // ghost coefficients per wall, depth, (U0..U3, datum)
  std::vector<uint8_t> ext[4];        // wall cell extendable, per wall and position
  double diag;                        // SFV centre weight
  // full row of A for one cell (SFV via stencil + ghosts, PLG via beta,
  // empty: identity); datum terms of N into nrow
  void row(int k, std::map<int, double>& arow, std::map<int, double>* nrow) const;
  double a = 0, b = 0, c = 0;
  const Problem* P = nullptr;
};

LevelDisc discretize(const Problem& P, int n);

}  // namespace ccmg
