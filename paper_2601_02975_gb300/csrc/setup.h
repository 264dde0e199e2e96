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
#include <thread>
#include <unordered_map>
#include <vector>

#include "setup_cell.h"

namespace ccmg {

enum CellType : uint8_t { CT_EMPTY = 0, CT_FULL = 1, CT_CUT = 2 };
enum CellKind : uint8_t { K_EMPTY = 0, K_SFV = 1, K_PLG = 2 };
enum BcType { BC_D = 0, BC_N = 1, BC_R = 2 };

struct SetupError : std::runtime_error {
  int code;
  SetupError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// a failed CUDA call of the device setup steps (err: the cudaError_t value)
struct DeviceError : std::runtime_error {
  int err;
  DeviceError(int e, const std::string& m) : std::runtime_error(m), err(e) {}
};

struct Bc { int type; double a1, a2; };

// f(j) for every j in [0, n), on up to 32 host threads in interleaved
// order; f must write only its own outputs
template <class F>
void parallel_rows(int n, F&& f, int min_per_thread = 64) {
  unsigned T = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
  if (n < (int)T * min_per_thread) T = std::max(1, n / min_per_thread);
  if (T <= 1) {
    for (int j = 0; j < n; ++j) f(j);
    return;
  }
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < T; ++t)
    pool.emplace_back([&, t] {
      for (int j = (int)t; j < n; j += (int)T) f(j);
    });
  for (int j = 0; j < n; j += (int)T) f(j);
  for (auto& th : pool) th.join();
}

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

// The per-cell steps of the setup (classification of the cells no curve
// crosses, Def. 4.1 kinds, lattices, fits, curve-order samples) run on the
// device when a SetupDevice is given (setup_dev.cu), else on host threads;
// both run the functions of setup_cell.h and give the same tables.
class SetupDevice;

LevelGeom build_geometry(const Problem& P, int n, SetupDevice* dev = nullptr);

// boundary quadrature of cut cell k (nodes on pieces with bc >= 0)
std::vector<BNode> boundary_nodes(const Problem& P, const LevelGeom& G, int k);
// volume quadrature of cut cell k: (x, y, w), sum w = 1
std::vector<std::array<double, 3>> volume_nodes(const Problem& P, const LevelGeom& G, int k);

// shift scaled moments from centre p to centre p - (dx, dy) h
void shift_moments(const double in[kMoments], double dx, double dy, double out[kMoments]);

// Gauss-Legendre rule on [-1, 1]
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// the rules of the cut-cell quadrature (straight pieces, sub-arcs)
const Rules510& quad_rules();

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

LevelDisc discretize(const Problem& P, int n, SetupDevice* dev = nullptr);

// Device execution of the per-cell setup steps (setup_dev.cu): FP64 CUDA
// kernels, one thread per cell, on the given stream; every call is
// synchronous (its results are in host memory on return).  A failed CUDA
// call throws DeviceError with its error text.
class SetupDevice {
 public:
  explicit SetupDevice(void* stream);
  ~SetupDevice();
  SetupDevice(const SetupDevice&) = delete;
  SetupDevice& operator=(const SetupDevice&) = delete;
  // type[k] = CT_FULL if crossed[k] == 0 and the cell's centre lies
  // outside every hole, else CT_EMPTY
  void classify(const Problem& P, int n, double h, const uint8_t* crossed, uint8_t* type);
  // scaled moments (28 each) of cut cells cells[r] about (px[r], py[r])
  // from their boundary pieces pieces[ptr[r], ptr[r+1]) (Green's theorem)
  void moments(const Problem& P, double h, const std::vector<int>& cells,
               const std::vector<Piece>& pieces, const std::vector<int>& ptr,
               const std::vector<double>& px, const std::vector<double>& py, const Rules510& R,
               double* mom);
  // Def. 4.1 kind of every cell; keeps the type map on the device for the
  // calls below
  void kinds(int n, bool cross, const uint8_t* type, const uint8_t* ext, uint8_t* kind);
  // lattice of each cell of plg (15 ints each); ok[r] = 0 where none exists
  void lattices(int n, const std::vector<int>& plg, int* lat, uint8_t* ok);
  // fits of the cells of plg with the lattices lat: cut cells (sorted) and
  // their moments, boundary nodes of plg cell r in bnode[bptr[r], bptr[r+1])
  void fits(int n, double h, double x0, double y0, double a, double b, double c,
            const std::vector<int>& plg, const int* lat, const std::vector<int>& cut_cells,
            const std::vector<double>& cut_mom, const std::vector<BNode>& bnode,
            const std::vector<int>& bptr, const std::vector<double>& a12, double* beta,
            uint8_t* ok);
  // for each of m points and each of nh curves (ns samples each, sx/sy
  // nh * ns): the nearest sample and its squared distance (m * nh each)
  void nearest(const double* sx, const double* sy, int nh, int ns, const double* px,
               const double* py, int m, int* idx, double* d2);
  // the inverse of the n x n row-major A in place by Gauss-Jordan with
  // partial pivoting, bitwise the host's dense inversion (the same
  // operations in the same order per element); false if singular
  bool invert(std::vector<double>& A, int n);
  double kernel_ms = 0;   // device time of the kernels so far

 private:
  struct Impl;
  Impl* p_;
};

}  // namespace ccmg
