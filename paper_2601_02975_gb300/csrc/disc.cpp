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

LevelDisc discretize(const Problem& P, int n, SetupDevice* dev) {
  LevelDisc D;
  D.P = &P;
  D.n = n;
  D.a = P.a;
  D.b = P.b;
  D.c = P.c;
  D.geom = build_geometry(P, n, dev);
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
  // --- Def. 4.1 ------------------------------------------------------------
  std::vector<uint8_t> extf((size_t)4 * n, 0);
  for (int w = 0; w < 4; ++w)
    for (int t = 0; t < n; ++t) extf[(size_t)w * n + t] = D.ext[w][t];
  const bool cross = P.b != 0.0;
  D.kind.assign((size_t)n * n, K_EMPTY);
  if (dev) {
    dev->kinds(n, cross, G.type.data(), extf.data(), D.kind.data());
  } else {
    parallel_rows(n, [&](int j) {
      for (int k = j * n; k < (j + 1) * n; ++k)
        D.kind[k] = cell::kind_of(G.type.data(), extf.data(), n, cross, k);
    });
  }
  // --- PLG cells: lattice and fit --------------------------------------------
  for (int k = 0; k < n * n; ++k)
    if (D.kind[k] == K_PLG) D.plg.push_back(k);
  const size_t np = D.plg.size();
  const int npi = (int)np;
  std::vector<int> lat(np * 15);
  std::vector<uint8_t> ok(np, 0);
  if (dev) {
    if (np) dev->lattices(n, D.plg, lat.data(), ok.data());
  } else {
    parallel_rows(npi, [&](int r) {
      ok[r] = cell::plg_lattice(G.type.data(), n, D.plg[r], &lat[(size_t)15 * r]);
    }, 16);
  }
  // the far search for the cells whose 13 x 13 box holds no lattice (rare:
  // the tips of thin wedges), on host threads for both paths
  std::vector<int> far;
  for (size_t r = 0; r < np; ++r)
    if (!ok[r]) far.push_back((int)r);
  parallel_rows((int)far.size(), [&](int q) {
    const int r = far[q];
    ok[r] = cell::plg_lattice_far(G.type.data(), n, D.plg[r], &lat[(size_t)15 * r]);
  }, 1);
  for (size_t r = 0; r < np; ++r)
    if (!ok[r]) throw SetupError(3, "no poised lattice for a PLG cell");
  // boundary nodes of the cut PLG cells, the moments of the cut cells, and
  // (alpha1, alpha2) of each condition
  std::vector<BNode> bnode;
  std::vector<int> bptr(np + 1, 0);
  for (size_t r = 0; r < np; ++r) {
    if (G.type[D.plg[r]] == CT_CUT) {
      std::vector<BNode> bn = boundary_nodes(P, G, D.plg[r]);
      bnode.insert(bnode.end(), bn.begin(), bn.end());
    }
    bptr[r + 1] = (int)bnode.size();
  }
  std::vector<double> a12;
  for (const Bc& bc : P.bc) {
    a12.push_back(bc.type == BC_D ? 1.0 : bc.type == BC_N ? 0.0 : bc.a1);
    a12.push_back(bc.type == BC_D ? 0.0 : bc.type == BC_N ? 1.0 : bc.a2);
  }
  std::vector<double> beta(np * 16);
  if (dev) {
    std::vector<int> cut_cells;
    std::vector<double> cut_mom;
    for (const auto& kv : G.cut) {
      cut_cells.push_back(kv.first);
      cut_mom.insert(cut_mom.end(), kv.second.mom, kv.second.mom + kMoments);
    }
    if (np)
      dev->fits(n, h, G.x0, G.y0, P.a, P.b, P.c, D.plg, lat.data(), cut_cells, cut_mom, bnode,
                bptr, a12, beta.data(), ok.data());
  } else {
    auto mom = [&](int kj, double* o) { G.moments(kj, o); };
    parallel_rows(npi, [&](int r) {
      const int nb = bptr[r + 1] - bptr[r];
      ok[r] = cell::plg_fit(D.plg[r], n, h, P.a, P.b, P.c, &lat[(size_t)15 * r], mom,
                            nb ? &bnode[bptr[r]] : nullptr, nb, a12.data(), G.x0, G.y0,
                            &beta[(size_t)16 * r]);
    }, 16);
  }
  // a row whose own coefficient is not negative takes the first alternative
  // lattice (the cheapest of each box, 9 x 9 to 13 x 13, rows then columns)
  // whose fit gives a negative one, if any; on host threads for both paths
  {
    auto mom = [&](int kj, double* o) { G.moments(kj, o); };
    parallel_rows(npi, [&](int r) {
      if (!ok[r]) return;
      const int k = D.plg[r];
      auto diag = [k](const int* la, const double* be) {
        for (int q = 0; q < 15; ++q)
          if (la[q] == k) return be[q];
        return 0.0;
      };
      int* la = &lat[(size_t)15 * r];
      double* be = &beta[(size_t)16 * r];
      if (diag(la, be) < 0.0) return;
      const int nb = bptr[r + 1] - bptr[r];
      for (int R = cell::kLatR0; R <= cell::kLatR; ++R)
        for (int orient = 0; orient < 2; ++orient) {
          int alt[15], cost = 0;
          if (!cell::plg_lattice_box(G.type.data(), n, k, R, orient, alt, &cost)) continue;
          if (std::equal(alt, alt + 15, la)) continue;
          double b2[16];
          if (!cell::plg_fit(k, n, h, P.a, P.b, P.c, alt, mom, nb ? &bnode[bptr[r]] : nullptr, nb,
                             a12.data(), G.x0, G.y0, b2))
            continue;
          if (diag(alt, b2) < 0.0) {
            std::copy(alt, alt + 15, la);
            std::copy(b2, b2 + 16, be);
            return;
          }
        }
    }, 16);
  }
  for (size_t r = 0; r < np; ++r) {
    if (!ok[r]) throw SetupError(3, "singular PLG fit");
    std::array<int, 15> la;
    std::copy(&lat[15 * r], &lat[15 * r] + 15, la.begin());
    D.lattice.push_back(la);
    if (bptr[r + 1] > bptr[r]) {
      D.bd_of_plg.push_back((int)D.bd_cells.size());
      D.bd_cells.push_back(D.plg[r]);
    } else {
      D.bd_of_plg.push_back(-1);
    }
    std::array<double, 16> bt;
    std::copy(&beta[16 * r], &beta[16 * r] + 16, bt.begin());
    D.beta.push_back(bt);
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
    // the nearest of 1024 samples of each curve to each block cell's centre
    const int nsm = cell::kCurveSamples;
    const int m = (int)blk.size();
    std::vector<double> sx((size_t)nh * nsm), sy((size_t)nh * nsm), cx(m), cy(m);
    for (int e = 0; e < nh; ++e)
      for (int s = 0; s < nsm; ++s)
        P.holes[e].at(6.283185307179586 * s / nsm, sx[(size_t)e * nsm + s], sy[(size_t)e * nsm + s]);
    for (int r = 0; r < m; ++r) {
      cx[r] = G.x0 + (blk[r] % n + 0.5) * h;
      cy[r] = G.y0 + (blk[r] / n + 0.5) * h;
    }
    std::vector<int> near((size_t)m * nh);
    std::vector<double> near_d2((size_t)m * nh);
    if (nh && m) {
      if (dev) {
        dev->nearest(sx.data(), sy.data(), nh, nsm, cx.data(), cy.data(), m, near.data(),
                     near_d2.data());
      } else {
        parallel_rows(m, [&](int r) {
          for (int e = 0; e < nh; ++e)
            near[(size_t)r * nh + e] = cell::nearest_sample(&sx[(size_t)e * nsm], &sy[(size_t)e * nsm],
                                                            nsm, cx[r], cy[r], &near_d2[(size_t)r * nh + e]);
        }, 16);
      }
    }
    const double L = P.x1 - P.x0;
    std::vector<std::tuple<int, double, int>> keys;
    for (int r = 0; r < m; ++r) {
      const int k = blk[r];
      const double x = cx[r], y = cy[r];
      double d[4] = {y - P.y0, P.x1 - x, P.y1 - y, x - P.x0};
      int side = (int)(std::min_element(d, d + 4) - d);
      double s_box[4] = {x - P.x0, L + y - P.y0, 2 * L + P.x1 - x, 3 * L + P.y1 - y};
      double bestd = d[side], bests = s_box[side];
      int bestg = 0;
      for (int e = 0; e < nh; ++e) {
        const double dd = std::sqrt(near_d2[(size_t)r * nh + e]);
        if (dd < bestd) {
          const int s = near[(size_t)r * nh + e];
          const double hx = sx[(size_t)e * nsm + s], hy = sy[(size_t)e * nsm + s];
          int rt = root(e);
          bestd = dd;
          bestg = 1 + rt;
          double ang = std::atan2(hy - gy[rt] / gn[rt], hx - gx[rt] / gn[rt]);
          bests = ang < 0 ? ang + 6.283185307179586 : ang;
        }
      }
      keys.emplace_back(bestg, bests, k);
    }
    std::sort(keys.begin(), keys.end());
    for (auto& t : keys) D.block.push_back(std::get<2>(t));
  }
  // rows of A for the block cells and of N: built on host threads, stored
  // in cell order
  {
    const int mb = (int)D.block.size();
    std::vector<std::map<int, double>> br(mb);
    parallel_rows(mb, [&](int r) { D.row(D.block[r], br[r], nullptr); }, 16);
    for (const auto& row : br) D.block_rows.push(row);
  }
  {
    // only PLG rows (boundary datum) and the rows of cells within two cells
    // of a box wall (ghost data) have terms in N
    std::vector<int> cells;
    for (int k = 0; k < n * n; ++k) {
      if (D.kind[k] == K_EMPTY) continue;
      const int i = k % n, j = k / n;
      if (D.kind[k] != K_PLG && i >= 2 && j >= 2 && i < n - 2 && j < n - 2) continue;
      cells.push_back(k);
    }
    const int nc = (int)cells.size();
    std::vector<std::map<int, double>> nr(nc);
    parallel_rows(nc, [&](int r) {
      std::map<int, double> ar;
      D.row(cells[r], ar, &nr[r]);
    }, 16);
    for (int r = 0; r < nc; ++r)
      if (!nr[r].empty()) {
        D.nrows.push(nr[r]);
        D.nrow_cell.push_back(cells[r]);
      }
  }
  return D;
}

}  // namespace ccmg
