// Device kernels of the cut-cell multigrid cycle (Sec. 5), templated on the
// cycle precision T (float or double).  Level vectors are N x N row-major.
//
// Cell classes on the device: 0 empty, 1 stencil cell (an SFV cell relaxed
// by weighted Jacobi, Eq. 5.7), 2 block cell (solved exactly by the block
// smoother, Eq. 5.8: the PLG cells, plus the 4 x 4 box corners when b != 0).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace ccmg {

constexpr int TX = 32;   // tile width (cells) of the stencil kernels
constexpr int TY = 8;    // thread rows of a CTA (256 threads = TX x TY)
constexpr int HALO = 2;  // stencil radius
constexpr int SX = TX + 2 * HALO;
constexpr int SY = TY + 2 * HALO;
// A CTA covers TX x (TY * RPT) cells; each thread computes RPT rows, ly =
// ty + TY * r, so that a warp always touches one shared-memory row.
template <int RPT>
struct Tile {
  static constexpr int H = TY * RPT;
  static constexpr int SH = H + 2 * HALO;
};

enum : uint8_t { C_EMPTY = 0, C_STENCIL = 1, C_BLOCK = 2 };

// Programmatic dependent launch: every kernel lets the next kernel of the
// stream begin launching at once, then waits until the previous kernel has
// completed and its writes are visible before it reads anything.  The launch
// latency of a kernel then overlaps the execution of the one before it.
// g_pdl_trigger: 1 lets dependents launch at kernel entry, 2 at exit, 0 never
// (they then launch when the kernel completes).
__device__ int g_pdl_trigger = 0;

__device__ __forceinline__ void pdl_enter() {
  if (g_pdl_trigger == 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_exit() {
  if (g_pdl_trigger == 2) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Constant per-level stencil data: weights of the 5 x 5 SFV stencil (Eq.
// 4.7a,b) and the homogeneous ghost coefficients of each wall, in the
// arithmetic type of the kernel (FP32 kernels must not touch the FP64 pipe).
template <class T>
struct StencilP {
  int n;
  int cross;               // b != 0
  T w[25];                 // (dj + 2) * 5 + (di + 2)
  T gh[4][2][4];           // wall (S, E, N, W), depth - 1, inward cell q
  T omega_over_diag;       // omega / D (D the centre weight)
  T sx, sy, sxy;           // a / (12 h^2), c / (12 h^2), b / (144 h^2)
};
using StencilParams = StencilP<double>;

template <class T>
StencilP<T> stencil_as(const StencilParams& d) {
  StencilP<T> o;
  o.n = d.n;
  o.cross = d.cross;
  for (int k = 0; k < 25; ++k) o.w[k] = (T)d.w[k];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 4; ++c) o.gh[a][b][c] = (T)d.gh[a][b][c];
  o.omega_over_diag = (T)d.omega_over_diag;
  o.sx = (T)d.sx;
  o.sy = (T)d.sy;
  o.sxy = (T)d.sxy;
  return o;
}

// ---- tile loader: u (+ prolonged e) with ghosts beyond the box walls --------
template <class T>
__device__ __forceinline__ T cell_value(const T* __restrict__ u, const T* __restrict__ ec,
                                        int n, int gx, int gy, bool zero) {
  T v = zero ? T(0) : u[(size_t)gy * n + gx];
  if (ec) v += ec[(size_t)(gy >> 1) * (n >> 1) + (gx >> 1)];
  return v;
}

// Value at (gx, gy) of the extended grid: a cell of u (+ I(ec)), or, beyond
// one box wall, the homogeneous part of that wall's ghost formula; 0 beyond
// two walls (no stencil cell reaches there: b != 0 puts the box-corner cells
// in the exactly solved block).
template <class T>
__device__ __forceinline__ T halo_value(const T* __restrict__ u, const T* __restrict__ ec,
                                        const StencilP<T>& P, int gx, int gy, bool zero) {
  const int n = P.n;
  const bool ox = gx < 0 || gx >= n, oy = gy < 0 || gy >= n;
  if (!ox && !oy) return cell_value(u, ec, n, gx, gy, zero);
  T acc = T(0);
  if (ox != oy && n >= 4) {
    int w, t, m;
    if (gx >= n) { w = 1; t = gy; m = gx - n; }
    else if (gx < 0) { w = 3; t = gy; m = -gx - 1; }
    else if (gy >= n) { w = 2; t = gx; m = gy - n; }
    else { w = 0; t = gx; m = -gy - 1; }
    if (m > 1) return T(0);   // beyond the two ghost layers (tile padding only)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int cx, cy;
      switch (w) {
        case 0: cx = t; cy = q; break;
        case 1: cx = n - 1 - q; cy = t; break;
        case 2: cx = t; cy = n - 1 - q; break;
        default: cx = q; cy = t; break;
      }
      acc += P.gh[w][m][q] * cell_value(u, ec, n, cx, cy, zero);
    }
  }
  return acc;
}

template <class T, int SHT = SY>
__device__ __forceinline__ void load_tile(T (*s)[SX], const T* __restrict__ u,
                                          const T* __restrict__ ec, const StencilP<T>& P,
                                          int x0, int y0, bool zero) {
#pragma unroll 4
  for (int idx = threadIdx.x; idx < SX * SHT; idx += blockDim.x) {
    int ly = idx / SX, lx = idx % SX;
    s[ly][lx] = halo_value(u, ec, P, x0 + lx - HALO, y0 + ly - HALO, zero);
  }
}

// (A u) at one cell from the values v(di, dj) of its 5 x 5 neighbourhood, in
// one fixed order of the terms, so that the tile kernels and the point
// evaluation below give the same bits.
template <class T, bool CROSS, class V>
__device__ __forceinline__ T apply_A_by(const T* w, V v) {
  T acc = w[2 * 5 + 0] * v(-2, 0) + w[2 * 5 + 1] * v(-1, 0) + w[2 * 5 + 2] * v(0, 0) +
          w[2 * 5 + 3] * v(1, 0) + w[2 * 5 + 4] * v(2, 0);
  acc += w[0 * 5 + 2] * v(0, -2) + w[1 * 5 + 2] * v(0, -1) + w[3 * 5 + 2] * v(0, 1) +
         w[4 * 5 + 2] * v(0, 2);
  if (CROSS) {
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      if (dj == 0) continue;
#pragma unroll
      for (int di = -2; di <= 2; ++di) {
        if (di == 0) continue;
        acc += w[(dj + 2) * 5 + (di + 2)] * v(di, dj);
      }
    }
  }
  return acc;
}

template <class T, bool CROSS>
__device__ __forceinline__ T apply_A(const T (*s)[SX], const T* w, int lx, int ly) {
  // lx, ly: tile-interior coordinates (0-based)
  const int cx = lx + HALO, cy = ly + HALO;
  return apply_A_by<T, CROSS>(w, [&](int di, int dj) { return s[cy + dj][cx + di]; });
}

// One Jacobi update (Eq. 5.7) of the stencil cell (gx, gy) evaluated straight
// from global memory: what the tile sweep writes there.
template <class T, bool CROSS>
__device__ __forceinline__ T sweep_point(const T* __restrict__ u, const T* __restrict__ ec,
                                         const T* __restrict__ b, const StencilP<T>& P, int gx,
                                         int gy, bool zero) {
  T Au = apply_A_by<T, CROSS>(P.w, [&](int di, int dj) {
    return halo_value(u, ec, P, gx + di, gy + dj, zero);
  });
  T uc = cell_value(u, ec, P.n, gx, gy, zero);
  return uc + P.omega_over_diag * (b[(size_t)gy * P.n + gx] - Au);
}

// ---- a1: weighted Jacobi sweep on stencil cells (Eq. 5.7) --------------------
// u_out = u + omega/D (b - A u) on stencil cells; other cells are left as
// they are in u_out (block cells are written by the block solve).  With ec,
// the sweep reads u + I(ec) (Eq. 5.11) instead of u (the first post-sweep,
// fused with the prolongation); with zero it reads 0 (a coarse level's first
// sweep, whose initial guess is 0, Alg. 2).
template <class T, bool CROSS, int RPT = 1>
__global__ void __launch_bounds__(TX * TY)
k_sweep(const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ b,
        const uint8_t* __restrict__ cls, const T* __restrict__ ec, StencilP<T> P, int zero) {
  pdl_enter();
  constexpr int TH = Tile<RPT>::H;
  __shared__ T s[Tile<RPT>::SH][SX];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TH;
  const int n = P.n;
  const int lx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gx = x0 + lx;
  // issue the loads of b and of the class map before the tile barrier
  T bv[RPT];
  uint8_t cv[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int gy = y0 + ty + TY * r;
    const bool in = gx < n && gy < n;
    const size_t k = (size_t)gy * n + gx;
    cv[r] = in ? cls[k] : (uint8_t)C_EMPTY;
    bv[r] = in ? b[k] : T(0);
  }
  load_tile<T, Tile<RPT>::SH>(s, u_in, ec, P, x0, y0, zero != 0);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int ly = ty + TY * r, gy = y0 + ly;
    if (cv[r] != C_STENCIL) continue;
    T Au = apply_A<T, CROSS>(s, P.w, lx, ly);
    T uc = s[ly + HALO][lx + HALO];
    u_out[(size_t)gy * n + gx] = uc + P.omega_over_diag * (bv[r] - Au);
  }
  pdl_exit();
}

// ---- a1, multicolour variant (outside the paper): one colour class in place ---
// The SFV cells are relaxed class by class, each class with the latest values
// of the others: u_i += omega / D (b - A u)_i for the cells of class `color`.
// The classes, (i + j) mod 4 for b = 0 and (i + 4 j) mod 15 for b != 0, hold no
// two cells that one row couples (wall ghosts included), so a class is
// updated in place: no cell of the class reads another.
__device__ __forceinline__ int mc_color(int gx, int gy, bool cross) {
  return cross ? (gx + 4 * gy) % 15 : (gx + gy) % 4;
}
__host__ __device__ inline int mc_colors(bool cross) { return cross ? 15 : 4; }

template <class T, bool CROSS>
__global__ void __launch_bounds__(TX * TY)
k_sweep_color(T* __restrict__ u, const T* __restrict__ b, const uint8_t* __restrict__ cls,
              StencilP<T> P, int color) {
  pdl_enter();
  __shared__ T s[SY][SX];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int n = P.n;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool in = gx < n && gy < n;
  const size_t k = (size_t)gy * n + gx;
  const bool mine = in && mc_color(gx, gy, CROSS) == color && cls[k] == C_STENCIL;
  const T bv = mine ? b[k] : T(0);
  // the window holds cells of other classes only where this class reads
  load_tile<T>(s, u, nullptr, P, x0, y0, false);
  __syncthreads();
  if (mine) {
    const T Au = apply_A<T, CROSS>(s, P.w, lx, ly);
    u[k] = s[ly + HALO][lx + HALO] + P.omega_over_diag * (bv - Au);
  }
  pdl_exit();
}

// ---- a1 on large grids: 32 x 32 tiles, 4 consecutive rows per thread ---------
// The stencil is a dxx + c dyy + b dx(dy) with the one-dimensional formulas of
// Eq. 4.7a,b.  Each thread reads the 5 values of each row of its 8-row window
// once, forms the row's second difference and gradient in x, and combines
// them along y for its 4 outputs; the loader walks the halo tile in 2-D.
constexpr int WY = 32;          // tile height of the windowed sweep
constexpr int WSH = WY + 2 * HALO;

template <class T>
__device__ __forceinline__ void load_tile_2d(T (*s)[SX], const T* __restrict__ u,
                                             const T* __restrict__ ec, const StencilP<T>& P,
                                             int x0, int y0, bool zero) {
  const int n = P.n;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const bool interior = x0 >= HALO && y0 >= HALO && x0 + SX - HALO <= n && y0 + WSH - HALO <= n;
  if (interior) {
#pragma unroll
    for (int ly = ty; ly < WSH; ly += TY) {
      const size_t row = (size_t)(y0 + ly - HALO) * n + (x0 - HALO);
      s[ly][tx] = zero ? T(0) : u[row + tx];
      if (tx < SX - TX) s[ly][tx + TX] = zero ? T(0) : u[row + tx + TX];
      if (ec) {
        const int gy = y0 + ly - HALO;
        const size_t crow = (size_t)(gy >> 1) * (n >> 1);
        s[ly][tx] += ec[crow + ((x0 - HALO + tx) >> 1)];
        if (tx < SX - TX) s[ly][tx + TX] += ec[crow + ((x0 - HALO + tx + TX) >> 1)];
      }
    }
  } else {
    load_tile<T, WSH>(s, u, ec, P, x0, y0, zero);
  }
}

template <class T, bool CROSS>
__global__ void __launch_bounds__(TX * TY)
k_sweep_w(const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ b,
          const uint8_t* __restrict__ cls, const T* __restrict__ ec, StencilP<T> P, int zero) {
  pdl_enter();
  __shared__ T s[WSH][SX];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * WY;
  const int n = P.n;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gx = x0 + tx, gy0 = y0 + 4 * ty;
  T bv[4];
  uint8_t cv[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gy = gy0 + r;
    const bool in = gx < n && gy < n;
    const size_t k = (size_t)gy * n + gx;
    cv[r] = in ? cls[k] : (uint8_t)C_EMPTY;
    bv[r] = in ? b[k] : T(0);
  }
  load_tile_2d<T>(s, u_in, ec, P, x0, y0, zero != 0);
  __syncthreads();
  // rows 4 ty - 2 .. 4 ty + 5 of the window (tile rows 4 ty .. 4 ty + 7)
  T lx[8], gxr[8], cc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const T* row = &s[4 * ty + k][tx];
    const T v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3], v4 = row[4];
    lx[k] = T(16) * (v1 + v3) - T(30) * v2 - (v0 + v4);
    gxr[k] = T(8) * (v3 - v1) + (v0 - v4);
    cc[k] = v2;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (cv[r] != C_STENCIL) continue;
    const int j = r + 2;
    const T ly = T(16) * (cc[j - 1] + cc[j + 1]) - T(30) * cc[j] - (cc[j - 2] + cc[j + 2]);
    T Au = P.sx * lx[j] + P.sy * ly;
    if (CROSS) Au += P.sxy * (T(8) * (gxr[j + 1] - gxr[j - 1]) + (gxr[j - 2] - gxr[j + 2]));
    u_out[(size_t)(gy0 + r) * n + gx] = cc[j] + P.omega_over_diag * (bv[r] - Au);
  }
  pdl_exit();
}

// ---- a1 streamed: persistent, multi-buffered windowed sweep (FP32) -----------
// The arithmetic of k_sweep_w on the same 32 x 32 tiles, but each CTA walks a
// sequence of tiles and copies the next tile's u window, b, class bytes and
// (on the fused post-sweep) coarse correction global -> shared with cp.async
// while it computes the current one, so loads stay in flight for the whole
// lifetime of the CTA.  Every copy is a 16-byte chunk that lies wholly inside
// or wholly outside the grid (N a multiple of 16); outside chunks are
// zero-filled and no byte is read for them.  Wall ghosts are formed in shared
// memory from the loaded inward cells.
constexpr int PW = 40;          // u window row: x0 - 4 .. x0 + 35 (16-byte aligned start)
constexpr int CWC = 24;         // coarse row: x0/2 - 4 .. x0/2 + 19
constexpr int CHC = 18;         // coarse rows: y0/2 - 1 .. y0/2 + 16

struct __align__(16) SweepStage {
  float u[WSH][PW];
  float b[WY][TX];
  uint8_t c[WY][TX];
  float e[CHC][CWC];
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-thread copy assignments of the streamed sweep, fixed for every tile:
// thread t copies u-window chunks t and t + 256 (36 rows x 10 chunks), b chunk
// t (32 x 8), class chunk t < 64 (32 x 2) and coarse chunk t < 108 (18 x 6).
struct SweepLanes {
  int ur0, uc0, ur1, uc1;     // u window: row, column of the chunk (ur1 < 0: none)
  int br, bc, cr, cc, er, ec; // b, class, coarse (cr / er < 0: none)
  __device__ __forceinline__ SweepLanes(int t) {
    ur0 = t / (PW / 4); uc0 = 4 * (t % (PW / 4));
    const int t1 = t + TX * TY;
    ur1 = t1 < WSH * (PW / 4) ? t1 / (PW / 4) : -1;
    uc1 = 4 * (t1 % (PW / 4));
    br = t / (TX / 4); bc = 4 * (t % (TX / 4));
    cr = t < WY * (TX / 16) ? t / (TX / 16) : -1;
    cc = 16 * (t % (TX / 16));
    er = t < CHC * (CWC / 4) ? t / (CWC / 4) : -1;
    ec = 4 * (t % (CWC / 4));
  }
};

__device__ __forceinline__ void sweep_issue(SweepStage& st, const SweepLanes& ln,
                                            const float* __restrict__ u, const float* __restrict__ b,
                                            const uint8_t* __restrict__ cls,
                                            const float* __restrict__ ec, int n, int x0, int y0,
                                            bool zero) {
  {
    const int gy = y0 - HALO + ln.ur0, gx = x0 - 4 + ln.uc0;
    const bool ok = !zero && gy >= 0 && gy < n && gx >= 0 && gx < n;
    cp_async16(&st.u[ln.ur0][ln.uc0], ok ? u + (size_t)gy * n + gx : u, ok);
  }
  if (ln.ur1 >= 0) {
    const int gy = y0 - HALO + ln.ur1, gx = x0 - 4 + ln.uc1;
    const bool ok = !zero && gy >= 0 && gy < n && gx >= 0 && gx < n;
    cp_async16(&st.u[ln.ur1][ln.uc1], ok ? u + (size_t)gy * n + gx : u, ok);
  }
  {
    const int gy = y0 + ln.br, gx = x0 + ln.bc;
    const bool ok = gy < n && gx < n;
    cp_async16(&st.b[ln.br][ln.bc], ok ? b + (size_t)gy * n + gx : b, ok);
  }
  if (ln.cr >= 0) {
    const int gy = y0 + ln.cr, gx = x0 + ln.cc;
    const bool ok = gy < n && gx < n;
    cp_async16(&st.c[ln.cr][ln.cc], ok ? cls + (size_t)gy * n + gx : cls, ok);
  }
  if (ec && ln.er >= 0) {
    const int nc = n >> 1;
    const int cy = (y0 >> 1) - 1 + ln.er, cx = (x0 >> 1) - 4 + ln.ec;
    const bool ok = cy >= 0 && cy < nc && cx >= 0 && cx < nc;
    cp_async16(&st.e[ln.er][ln.ec], ok ? ec + (size_t)cy * nc + cx : ec, ok);
  }
}

// u + I(ec) on the in-grid cells of the window (one 4-cell chunk per step:
// the chunk's cells pair up on 2 coarse cells), then the wall ghosts (the
// homogeneous part of each wall's formula, as halo_value)
__device__ __forceinline__ void sweep_fixup(SweepStage& st, const SweepLanes& ln, const float* ec,
                                            const StencilP<float>& P, int x0, int y0) {
  const int n = P.n;
  if (ec) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int r = k ? ln.ur1 : ln.ur0, c = k ? ln.uc1 : ln.uc0;
      if (r < 0) continue;
      const int gy = y0 - HALO + r, gx = x0 - 4 + c;
      if (gy < 0 || gy >= n || gx < 0 || gx >= n) continue;
      const float* e = &st.e[(gy >> 1) - ((y0 >> 1) - 1)][(gx >> 1) - ((x0 >> 1) - 4)];
      float4 v = *reinterpret_cast<float4*>(&st.u[r][c]);
      v.x += e[0];
      v.y += e[0];
      v.z += e[1];
      v.w += e[1];
      *reinterpret_cast<float4*>(&st.u[r][c]) = v;
    }
    __syncthreads();
  }
  const bool wl = x0 == 0, wr = x0 + TX >= n, wb = y0 == 0, wt = y0 + WY >= n;
  if (!(wl || wr || wb || wt)) return;
  // 2 ghost layers x WSH rows on the side walls, 2 x PW columns on the others
  for (int i = threadIdx.x; i < 2 * WSH; i += blockDim.x) {
    const int m = i / WSH, r = i % WSH;
    const int gy = y0 - HALO + r;
    if (gy < 0 || gy >= n) continue;
    if (wl) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += P.gh[3][m][q] * st.u[r][4 + q];
      st.u[r][3 - m] = acc;
    }
    if (wr) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += P.gh[1][m][q] * st.u[r][(n - 1 - q) - (x0 - 4)];
      st.u[r][(n + m) - (x0 - 4)] = acc;
    }
  }
  for (int i = threadIdx.x; i < 2 * PW; i += blockDim.x) {
    const int m = i / PW, c = i % PW;
    const int gx = x0 - 4 + c;
    if (gx < 0 || gx >= n) continue;
    if (wb) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += P.gh[0][m][q] * st.u[HALO + q][c];
      st.u[HALO - 1 - m][c] = acc;
    }
    if (wt) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += P.gh[2][m][q] * st.u[(n - 1 - q) - (y0 - HALO)][c];
      st.u[(n + m) - (y0 - HALO)][c] = acc;
    }
  }
}

// window columns 4 q4 .. 4 q4 + 11 of window row r (three 16-byte vectors):
// the x-stencil of tile columns 4 q4 .. 4 q4 + 3 at w[2 + k .. 6 + k]
__device__ __forceinline__ void load12(const SweepStage& S, int r, int q4, float* w) {
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const float4 a = *reinterpret_cast<const float4*>(&S.u[r][4 * q4 + 4 * v]);
    w[4 * v] = a.x; w[4 * v + 1] = a.y; w[4 * v + 2] = a.z; w[4 * v + 3] = a.w;
  }
}

// tile cursor: tile (bx, by) of a tpr-wide grid of tiles, advanced by the
// grid size with an add and a carry (no division per tile)
struct TileCursor {
  int bx, by;
  __device__ __forceinline__ void advance(int dx, int dy, int tpr) {
    bx += dx;
    by += dy;
    if (bx >= tpr) {
      bx -= tpr;
      ++by;
    }
  }
};

template <bool CROSS>
__global__ void __launch_bounds__(TX * TY)
k_sweep_p(const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ b,
          const uint8_t* __restrict__ cls, const float* __restrict__ ec, StencilP<float> P,
          int zero) {
  constexpr int NS = 2;            // stages: one tile in flight while one is computed
  pdl_enter();
  __shared__ SweepStage st[NS];
  const int n = P.n;
  const int tpr = (n + TX - 1) / TX, rows = (n + WY - 1) / WY;
  const int q4 = threadIdx.x & 7, row = threadIdx.x >> 3;
  const SweepLanes ln(threadIdx.x);
  const int dx = (int)gridDim.x % tpr, dy = (int)gridDim.x / tpr;
  TileCursor ct{(int)blockIdx.x % tpr, (int)blockIdx.x / tpr};   // tile being computed
  TileCursor it = ct;                                              // next tile to copy
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    if (it.by < rows) sweep_issue(st[k], ln, u_in, b, cls, ec, n, it.bx * TX, it.by * WY, zero != 0);
    cp_async_commit();
    it.advance(dx, dy, tpr);
  }
  for (int i = 0; ct.by < rows; ++i) {
    if (it.by < rows)
      sweep_issue(st[(i + NS - 1) % NS], ln, u_in, b, cls, ec, n, it.bx * TX, it.by * WY, zero != 0);
    cp_async_commit();
    it.advance(dx, dy, tpr);
    cp_async_wait<NS - 1>();      // the group of the tile being computed is complete
    __syncthreads();
    SweepStage& S = st[i % NS];
    const int x0 = ct.bx * TX, y0 = ct.by * WY;
    sweep_fixup(S, ln, ec, P, x0, y0);
    __syncthreads();
    // thread (q4, row): tile row `row`, tile columns 4 q4 .. 4 q4 + 3 (window
    // columns 4 q4 + 4 .. + 7), read as 16-byte vectors; per cell the
    // arithmetic and its order are k_sweep_w's
    const int rr = row + HALO;
    float w[12];
    load12(S, rr, q4, w);
    float c[5][4];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      if (d == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[2][k] = w[4 + k];
      } else {
        const float4 v = *reinterpret_cast<const float4*>(&S.u[rr - 2 + d][4 * q4 + 4]);
        c[d][0] = v.x; c[d][1] = v.y; c[d][2] = v.z; c[d][3] = v.w;
      }
    }
    float g[5][4];
    if (CROSS) {
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        if (d == 2) continue;
        float wd[12];
        load12(S, rr - 2 + d, q4, wd);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          g[d][k] = 8.f * (wd[5 + k] - wd[3 + k]) + (wd[2 + k] - wd[6 + k]);
      }
    }
    const float4 bv = *reinterpret_cast<const float4*>(&S.b[row][4 * q4]);
    const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
    const uint32_t cl = *reinterpret_cast<const uint32_t*>(&S.c[row][4 * q4]);
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float lx = 16.f * (w[3 + k] + w[5 + k]) - 30.f * w[4 + k] - (w[2 + k] + w[6 + k]);
      const float ly = 16.f * (c[1][k] + c[3][k]) - 30.f * c[2][k] - (c[0][k] + c[4][k]);
      float Au = P.sx * lx + P.sy * ly;
      if (CROSS) Au += P.sxy * (8.f * (g[3][k] - g[1][k]) + (g[0][k] - g[4][k]));
      o[k] = c[2][k] + P.omega_over_diag * (bb[k] - Au);
    }
    float* out = u_out + (size_t)(y0 + row) * n + x0 + 4 * q4;
    const uint32_t all = C_STENCIL * 0x01010101u;
    if (cl == all) {
      *reinterpret_cast<float4*>(out) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (((cl >> (8 * k)) & 0xffu) == C_STENCIL) out[k] = o[k];
    }
    __syncthreads();
    ct.advance(dx, dy, tpr);
  }
  cp_async_wait<0>();
  pdl_exit();
}

// ---- a4: residual and restriction (Eq. 5.10) ---------------------------------
// r = b - A u on stencil cells, 0 on block and empty cells (the block residual
// is zero after a block-smoother sweep); rc = average of the 4 children,
// 0 on empty coarse cells.  With uc, also the stencil-cell part of the coarse
// level's first sweep (wd_c = omega / D of the coarse level).
template <class T, bool CROSS>
__global__ void __launch_bounds__(TX * TY)
k_resid_restrict(const T* __restrict__ u, const T* __restrict__ b, const uint8_t* __restrict__ cls,
                 const uint8_t* __restrict__ cls_c, T* __restrict__ rc, StencilP<T> P,
                 T* __restrict__ uc, T wd_c) {
  pdl_enter();
  __shared__ T s[SY][SX];
  __shared__ T r[TY][TX];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  load_tile<T>(s, u, nullptr, P, x0, y0, false);
  __syncthreads();
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int gx = x0 + lx, gy = y0 + ly, n = P.n;
  T rv = T(0);
  if (gx < n && gy < n) {
    const size_t k = (size_t)gy * n + gx;
    if (cls[k] == C_STENCIL) rv = b[k] - apply_A<T, CROSS>(s, P.w, lx, ly);
  }
  r[ly][lx] = rv;
  __syncthreads();
  if (threadIdx.x < (TX / 2) * (TY / 2)) {
    const int cx = threadIdx.x % (TX / 2), cy = threadIdx.x / (TX / 2);
    const int nc = n >> 1;
    const int gcx = (x0 >> 1) + cx, gcy = (y0 >> 1) + cy;
    if (gcx < nc && gcy < nc) {
      const size_t kc = (size_t)gcy * nc + gcx;
      T v = T(0.25) * (r[2 * cy][2 * cx] + r[2 * cy][2 * cx + 1] + r[2 * cy + 1][2 * cx] +
                       r[2 * cy + 1][2 * cx + 1]);
      const uint8_t cc = cls_c[kc];
      rc[kc] = cc == C_EMPTY ? T(0) : v;
      // the coarse level's first sweep from a zero initial guess is pointwise,
      // u_c = omega / D_c * b_c (Eq. 5.7 with u = 0): written here with it
      if (uc && cc == C_STENCIL) uc[kc] = wd_c * v;
    }
  }
  pdl_exit();
}

// ---- Alg. 3 descent: restriction of a right-hand side (Eq. 5.10) -------------
// rc = average of the 4 children (empty children count 0), 0 on empty coarse
// cells.  Unlike the cycle's restriction, block cells keep their value: the
// FMG cycle restricts the residual of the iterate as it is.
template <class Tin, class Tout>
__global__ void k_restrict_rhs(const Tin* __restrict__ r, const uint8_t* __restrict__ cls,
                               const uint8_t* __restrict__ cls_c, Tout* __restrict__ rc, int n) {
  pdl_enter();
  const int nc = n >> 1;
  const int64_t kc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kc >= (int64_t)nc * nc) return;
  const int cx = (int)(kc % nc), cy = (int)(kc / nc);
  const size_t k00 = (size_t)(2 * cy) * n + 2 * cx, k10 = k00 + n;
  auto v = [&](size_t k) { return cls[k] == C_EMPTY ? Tin(0) : r[k]; };
  const Tin s = Tin(0.25) * (v(k00) + v(k10) + v(k00 + 1) + v(k10 + 1));
  rc[kc] = cls_c[kc] == C_EMPTY ? Tout(0) : (Tout)s;
}

// ---- a8 / Eq. 4.23: residual on stencil cells, max-norm ----------------------
// |r| is folded into *rmax as ordered bits (non-negative doubles order like
// their bit patterns).
__device__ __forceinline__ void atomic_max_abs(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(fabs(v)));
}

// ---- a8 off the FP64 pipe: residual with the stencil differences in fixed point
// The SFV stencil (Eq. 4.7a,b) is a u_xx + c u_yy + b u_xy with integer
// difference weights: A u = sx Lx + sy Ly + sxy Gxy, Lx = 16 (u_{i-1} +
// u_{i+1}) - 30 u_i - (u_{i-2} + u_{i+2}) (Ly the same in y) and Gxy the
// product of the 5-point gradients (1, -8, 0, 8, -1) in x and y.  The tile's
// values (ghosts included) are scaled by a power of two so that the largest
// is below 2^52 and rounded to 64-bit integers (a fixed-point accumulator
// restricted to one 64-bit word, in the manner of Kulisch's long
// accumulator); Lx, Ly and Gxy are then exact integer sums (|Gxy| < 324 *
// 2^52 < 2^61), and only their conversion, the three products with the
// FP64 constants and the subtraction from b round.  That is 7 FP64
// operations per cell instead of the 25 products of the direct evaluation,
// on a GPU whose FP64 rate is a small fraction of its FP32 rate, with no
// accuracy lost: each integer sum is exact, where the direct evaluation
// rounds every one of its 25 terms.
__device__ __forceinline__ int fx_exponent(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// v * 2^(1075 - E) rounded to the nearest integer (ties away from zero),
// E >= the biased exponent of v; integer operations only
__device__ __forceinline__ long long fx_from(double v, int E) {
  const long long bits = __double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0) return 0;                              // zero (and subnormals, far below 2^-53 max)
  const long long m = (bits & 0xfffffffffffffLL) | 0x10000000000000LL;
  const int sh = E - e;                               // value = m * 2^(e - E) in units of 2^(1075 - E)
  long long r;
  if (sh == 0) r = m;
  else if (sh < 63) r = ((m >> (sh - 1)) + 1) >> 1;
  else r = 0;
  return bits < 0 ? -r : r;
}

template <class Tout, bool CROSS>
__global__ void __launch_bounds__(TX * TY)
k_resid_fx(const double* __restrict__ u, const double* __restrict__ b, const uint8_t* __restrict__ cls,
           Tout* __restrict__ r, StencilP<double> P, unsigned long long* rmax, Tout* __restrict__ e0,
           Tout wd) {
  pdl_enter();
  __shared__ double s[SY][SX];
  __shared__ long long q[SY][SX];
  __shared__ int emax[TX * TY / 32];
  __shared__ double red[TX * TY / 32];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int gx = x0 + lx, gy = y0 + ly, n = P.n;
  const bool in = gx < n && gy < n;
  const size_t k = (size_t)gy * n + gx;
  const uint8_t c = in ? cls[k] : (uint8_t)C_EMPTY;
  const double bk = in && c == C_STENCIL ? b[k] : 0.0;
  load_tile<double>(s, u, nullptr, P, x0, y0, false);
  __syncthreads();
  // the window's largest biased exponent
  int e = 0;
  for (int idx = threadIdx.x; idx < SX * SY; idx += blockDim.x) e = max(e, fx_exponent((&s[0][0])[idx]));
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) emax[threadIdx.x >> 5] = e;
  __syncthreads();
  int E = 0;
#pragma unroll
  for (int w = 0; w < TX * TY / 32; ++w) E = max(E, emax[w]);
  // every |value| < 2^(E - 1023) is scaled below 2^52; E >= 53 keeps one
  // unit, 2^(E - 1075), a normal number (smaller values round to 0)
  E = max(E + 1, 53);
  for (int idx = threadIdx.x; idx < SX * SY; idx += blockDim.x)
    (&q[0][0])[idx] = fx_from((&s[0][0])[idx], E);
  __syncthreads();
  double av = 0.0;
  if (c == C_STENCIL) {
    const int cx = lx + HALO, cy = ly + HALO;
    const long long* row = q[cy];
    const long long Lx = 16 * (row[cx - 1] + row[cx + 1]) - 30 * row[cx] - (row[cx - 2] + row[cx + 2]);
    const long long Ly = 16 * (q[cy - 1][cx] + q[cy + 1][cx]) - 30 * q[cy][cx] - (q[cy - 2][cx] + q[cy + 2][cx]);
    // one unit of the fixed point is 2^(E - 1075)
    const double unit = __longlong_as_double((long long)(E - 52) << 52);
    double Au = (P.sx * unit) * __ll2double_rn(Lx) + (P.sy * unit) * __ll2double_rn(Ly);
    if (CROSS) {
      long long g[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        const long long* rr = q[cy - 2 + d];
        g[d] = 8 * (rr[cx + 1] - rr[cx - 1]) - (rr[cx + 2] - rr[cx - 2]);
      }
      const long long Gxy = 8 * (g[3] - g[1]) - (g[4] - g[0]);
      Au += (P.sxy * unit) * __ll2double_rn(Gxy);
    }
    const double rv = bk - Au;
    r[k] = (Tout)rv;
    if (e0) e0[k] = wd * (Tout)rv;
    av = fabs(rv);
  } else if (in && c == C_EMPTY) {
    r[k] = Tout(0);
  }
  if (rmax) {
    for (int o = 16; o > 0; o >>= 1) av = fmax(av, __shfl_xor_sync(0xffffffffu, av, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = av;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < TX * TY / 32; ++w) m = fmax(m, red[w]);
      atomic_max_abs(rmax, m);
    }
  }
  pdl_exit();
}

// residual of block rows from their full sparse rows (FP64)
template <class Tout>
__global__ void k_block_resid(int m, const int* __restrict__ cell, const int64_t* __restrict__ ptr,
                              const int* __restrict__ col, const double* __restrict__ val,
                              const double* __restrict__ u, const double* __restrict__ b,
                              Tout* __restrict__ r, unsigned long long* rmax) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double av = 0.0;
  if (i < m) {
    double acc = 0.0;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) acc += val[q] * u[col[q]];
    double rv = b[cell[i]] - acc;
    r[cell[i]] = (Tout)rv;
    av = fabs(rv);
  }
  if (rmax) {
    for (int o = 16; o > 0; o >>= 1) av = fmax(av, __shfl_xor_sync(0xffffffffu, av, o));
    if ((threadIdx.x & 31) == 0) atomic_max_abs(rmax, av);
  }
}

// ---- a2 + a3: exact solve on the block (Eq. 5.8) ------------------------------
// The block rows are ordered along the boundary curves (Def. 5.1), where the
// block matrix is banded up to its periodic corner (Lemma 5.2, Def. 5.3).
// Small blocks are solved with their dense inverse in one launch.  Larger
// ones are cut into chunks of consecutive rows; a row of a chunk that couples
// to a later chunk (or, across the periodic corner, to the last one) is an
// interface row, all other rows are interior rows.  Interior rows couple only
// to their own chunk and to interface rows, so with t the gathered right-hand
// side the exact solution is
//   x_I(c) = inv(A_cc) t_I(c) - W_c x_S,       W_c = inv(A_cc) A_{c,S},
//   S x_S = t_S - sum_c V_c t_I(c),            V_c = A_{S,c} inv(A_cc),
// S = A_SS - sum_c A_{S,c} inv(A_cc) A_{c,S} the interface Schur complement.
// Setup (FP64, host) stores per chunk the stacked [inv(A_cc); V_c] (launch 1)
// and the rows of inv(S) that the chunk needs with W_c (launch 2), each
// contiguous, so one bulk (TMA) copy stages them in shared memory before the
// kernel waits on its predecessor.  Launch 1 gathers t, forms z = inv(A_cc)
// t_I and the chunk's contributions V_c t_I to the interface right-hand
// side; launch 2 sums those contributions in a fixed order, applies its rows
// of inv(S) and finishes x_I = z - W_c x_S.  Both launch one CTA per chunk.
struct ChunkDev {
  int p0, p1;        // block positions [p0, p1) of the chunk's rows
  int ni, nv;        // interior rows; interface rows that read the interior (V_c rows)
  int nr, nw, nown;  // rows of inv(S) held; W_c columns; interface rows of the chunk
  int ipos_off;      // interior block positions: ipos[ipos_off .. + ni)
  int v_off;         // q slot of each V_c row: vslot[v_off .. + nv)
  int w_off;         // row of inv(S) (index into the held rows) of each W_c column
  int o_off;         // own interface rows: orow[o_off ..] (held-row index), opos (position)
  int b1n, b2n;      // elements of the two stages (multiples of 4)
  long long b1, b2;  // element offsets of the two stages in the blob
};

struct BlockDev {
  int m;
  const int* cell;          // [m] grid cell of block position
  int gk;                   // gather width: terms per row (padded)
  const int* gcol;          // [gk * m] term-major: entry q of row p at q * m + p
  const void* gval;         // T, padded terms have value 0
  const int* tptr;          // [m+1] terms beyond gk (rows longer than the width)
  const int* tcol;
  const void* tval;         // T
  const int* alias_ptr;     // [m+1] merged-away control volumes owned by each block cell
  const int* alias_cell;    //       (they carry the owner's value for Eq. 5.11)
  // dense form: the inverse of the whole block, row-major, row stride ld
  int dense, ld;
  const void* ainv;         // T
  // chunked form
  int nch, ns, nslots;
  const ChunkDev* ch;       // [nch]
  const int* slot;          // [m] row of a position within its chunk: interior rows first
  const int* sidx;          // [m] interface index of a position, -1 for interior rows
  const int* ipos;          // interior positions of every chunk
  const int* vslot;         // q slot of every V_c row
  const int* wrow;          // held-row index of every W_c column
  const int* orow;          // held-row index of every own interface row
  const int* opos;          //   and its block position
  const int* qptr;          // [ns+1] slots of each interface's contributions (chunk order)
  const void* blob;         // T, the per-chunk stages
  int stage1, stage2;       // 1: the stage is copied to shared memory (it fits)
  int rows1, rows2;         // largest ni + nv; largest nr (partial-sum buffer sizes)
  // work vectors (per handle)
  void* tS;                 // T [ns]    gathered t of the interface rows
  void* z;                  // T [m]     inv(A_cc) t_I at interior positions
  void* q;                  // T [slots] contributions V_c t_I
  unsigned int* fault;      // set when a bounded wait expires
};

template <class T>
__device__ __forceinline__ void block_write(const BlockDev& B, T* u, int p, T v) {
  u[B.cell[p]] = v;
  for (int q = B.alias_ptr[p]; q < B.alias_ptr[p + 1]; ++q) u[B.alias_cell[q]] = v;
}

// The destinations of block row p (its cell and up to two merged-away
// cells), loaded ahead of the product so the final writes wait on nothing.
struct BlockDst {
  int cell = -1, a0 = 0, a1 = 0, al[2] = {-1, -1};
  __device__ __forceinline__ void load(const BlockDev& B, int p) {
    if (p >= B.m) return;
    cell = B.cell[p];
    a0 = B.alias_ptr[p];
    a1 = B.alias_ptr[p + 1];
    if (a1 > a0) al[0] = B.alias_cell[a0];
    if (a1 > a0 + 1) al[1] = B.alias_cell[a0 + 1];
  }
  template <class T>
  __device__ __forceinline__ void write(const BlockDev& B, T* u, T v) const {
    u[cell] = v;
    if (a1 > a0) u[al[0]] = v;
    if (a1 > a0 + 1) u[al[1]] = v;
    for (int q = a0 + 2; q < a1; ++q) u[B.alias_cell[q]] = v;
  }
};

// t = b - A(block, rest) u for block row p: the padded terms are laid out
// term-major, so the loads of consecutive rows are coalesced and the loads of
// one row are independent of one another.
template <class T>
__device__ __forceinline__ T block_rhs(const BlockDev& B, const T* __restrict__ b,
                                       const T* __restrict__ u, int p) {
  const T* gval = static_cast<const T*>(B.gval);
  T acc = b[B.cell[p]];
#pragma unroll 8
  for (int q = 0; q < B.gk; ++q) {
    size_t e = (size_t)q * B.m + p;
    acc -= gval[e] * u[B.gcol[e]];
  }
  const T* tval = static_cast<const T*>(B.tval);
  for (int q = B.tptr[p]; q < B.tptr[p + 1]; ++q) acc -= tval[q] * u[B.tcol[q]];
  return acc;
}

// ---- bulk (TMA) copies global -> shared, completed on an mbarrier ---------------
// A device-wide flag that kernels set when a bounded wait expires; the solve
// loop reads it with every norm and reports CC_ERR_TIMEOUT.
constexpr unsigned kWaitLimit = 1u << 20;     // polls of a bounded wait (about 0.1 s)
constexpr unsigned kBulkPiece = 32768;        // bytes per bulk copy instruction

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// One thread: initialise the barrier for one arrival, announce `bytes`, and
// copy them (16-byte aligned on both sides, a multiple of 16) into shared memory.
__device__ __forceinline__ void bulk_stage(void* sdst, const void* gsrc, unsigned bytes,
                                           uint64_t* bar) {
  const unsigned b = smem_u32(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  const unsigned d = smem_u32(sdst);
  for (unsigned off = 0; off < bytes; off += kBulkPiece) {
    const unsigned n = bytes - off < kBulkPiece ? bytes - off : kBulkPiece;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d + off),
        "l"(static_cast<const char*>(gsrc) + off), "r"(n), "r"(b)
        : "memory");
  }
}

// Wait for phase 0 of the barrier, at most kWaitLimit polls; false if it expired.
__device__ __forceinline__ bool bulk_wait(uint64_t* bar) {
  const unsigned b = smem_u32(bar);
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b)
        : "memory");
    if (done) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

// All threads wait for the staged copy (after a CTA barrier, so that the
// barrier's initialisation by thread 0 is visible); if the wait expired
// anywhere the CTA flags the fault, waits once more (bounded) for its copy in
// flight, and the caller returns without using the data.  Ends with a CTA
// barrier.
__device__ __forceinline__ bool stage_ready(bool staged, uint64_t* bar, unsigned int* fault) {
  __syncthreads();
  const int bad = staged && !bulk_wait(bar);
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0 && fault) atomicOr(fault, 1u);
    if (staged) bulk_wait(bar);
    return false;
  }
  return true;
}

// ---- chunked exact block solve (the two launches) -------------------------------
constexpr int kChunkThreads = 256;   // threads of both launches; a chunk has at most this many rows
constexpr int kRB = 9;               // rows per lane of cta_gemv_cm: products of up to 288 rows
constexpr int kGatherMax = 16;       // the ELL width of the gather (gk) never exceeds it

// y[0..rows) = M x, M column-major (rows x cols, column stride ld), x in
// shared memory: lane l of warp w accumulates rows l, l + 32, ... over the
// columns w, w + nwarps, ...; the partial sums of the warps go through part
// (nwarps x rows) and are added in warp order.  Ends with a CTA barrier.
template <class T>
__device__ void cta_gemv_cm(const T* M, int rows, int ld, int cols, const T* x, T* part, T* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T acc[kRB];
#pragma unroll
  for (int i = 0; i < kRB; ++i) acc[i] = T(0);
  for (int c = warp; c < cols; c += nw) {
    const T xc = x[c];
    const T* col = M + (size_t)c * ld;
#pragma unroll
    for (int i = 0; i < kRB; ++i) {
      const int r = lane + 32 * i;
      if (r < rows) acc[i] += col[r] * xc;
    }
  }
#pragma unroll
  for (int i = 0; i < kRB; ++i) {
    const int r = lane + 32 * i;
    if (r < rows) part[warp * rows + r] = acc[i];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += part[w * rows + r];
    y[r] = s;
  }
  __syncthreads();
}

// y[0..rows) = M x, M row-major (rows x cols, row stride ld), x in shared
// memory: warp w takes rows w, w + nwarps, ... (four at a time), its lanes
// split the columns and each row's sum is reduced across the warp in a fixed
// order.  Ends with a CTA barrier.
template <class T>
__device__ void cta_gemv_rm(const T* M, int rows, int ld, int cols, const T* x, T* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = warp; r0 < rows; r0 += 4 * nw) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int c = lane; c < cols; c += 32) {
      const T xc = x[c];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + i * nw;
        if (r < rows) acc[i] += M[(size_t)r * ld + c] * xc;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T v = acc[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int r = r0 + i * nw;
      if (lane == 0 && r < rows) y[r] = v;
    }
  }
  __syncthreads();
}

// Shared-memory layout of the two launches (elements of T); st1 / st2 are
// the staged regions (0 when the stage is read from global memory).  Launch
// 2 ends with the interface pointers qptr as ints.
struct ChunkSmem {
  int st1, st2;       // staged regions
  int ns4, sl4;       // interface count and contribution-slot count, rounded up to 4
  int rows1, rows2;   // largest ni + nv; largest nr
  int nwmax, nimax;   // largest nw; largest ni
  __host__ __device__ int p1_tl() const { return st1; }
  __host__ __device__ int p1_part() const { return st1 + kChunkThreads; }
  __host__ __device__ int p1_y() const { return p1_part() + (kChunkThreads / 32) * rows1; }
  __host__ __device__ int p1_total() const { return p1_y() + rows1; }
  __host__ __device__ int p2_ys() const { return st2; }
  __host__ __device__ int p2_q() const { return st2 + ns4; }
  __host__ __device__ int p2_xr() const { return p2_q() + sl4; }
  __host__ __device__ int p2_xw() const { return p2_xr() + rows2; }
  __host__ __device__ int p2_part() const { return p2_xw() + nwmax; }
  __host__ __device__ int p2_y() const {
    return p2_part() + (kChunkThreads / 32) * (rows2 > nimax ? rows2 : nimax);
  }
  __host__ __device__ int p2_total() const { return p2_y() + nimax; }
  // bytes of launch 2 at element size w: the elements, then ns4 + 4 ints
  __host__ __device__ size_t p2_bytes(int w) const { return (size_t)p2_total() * w + (size_t)(ns4 + 4) * 4; }
};

// Phase 1 of the chunked solve, one CTA per chunk: gather t of the chunk's
// rows, then z = inv(A_cc) t_I and the contributions q = V_c t_I, with
// [inv(A_cc); V_c] staged in shared memory.  Everything that comes from
// setup (the row's gather terms, its slot, the output index of each product
// row) is read by p1_load, before the wait on the previous kernel; after it,
// one batch of independent loads of b and u.
template <class T>
struct P1Pre {
  bool on;
  int cell, sl, si, t0, t1;
  int col[kGatherMax];
  T val[kGatherMax];
  int oi[2];
};

template <class T>
__device__ __forceinline__ void p1_load(const BlockDev& B, const ChunkDev& C, P1Pre<T>& r) {
  const int tid = threadIdx.x;
  r.on = tid < C.p1 - C.p0;
  const int p = C.p0 + tid;
  r.cell = 0; r.sl = 0; r.si = -1; r.t0 = 0; r.t1 = 0;
  const T* gval = static_cast<const T*>(B.gval);
  if (r.on) {
    r.cell = B.cell[p];
    r.sl = B.slot[p];
    r.si = B.sidx[p];
    r.t0 = B.tptr[p];
    r.t1 = B.tptr[p + 1];
  }
#pragma unroll
  for (int k = 0; k < kGatherMax; ++k) {
    const bool use = r.on && k < B.gk;
    const size_t e = (size_t)k * B.m + p;
    r.col[k] = use ? B.gcol[e] : 0;
    r.val[k] = use ? gval[e] : T(0);
  }
  // output index of product rows tid and tid + kChunkThreads: interior rows
  // go to z at their block position, V_c rows to their contribution slot
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int q = tid + k * kChunkThreads;
    r.oi[k] = q < C.ni ? B.ipos[C.ipos_off + q] : q < C.ni + C.nv ? B.vslot[C.v_off + q - C.ni] : -1;
  }
}

// after the wait: false (nothing written but the gathered t) if the staged
// copy did not arrive
template <class T>
__device__ __forceinline__ bool p1_run(const BlockDev& B, const ChunkSmem& L, const ChunkDev& C,
                                       const P1Pre<T>& r, const T* __restrict__ b,
                                       const T* __restrict__ u, T* sm, uint64_t* bar) {
  const int tid = threadIdx.x;
  T* tl = sm + L.p1_tl();
  if (r.on) {
    T acc = b[r.cell];
#pragma unroll
    for (int k = 0; k < kGatherMax; ++k)
      if (k < B.gk) acc -= r.val[k] * u[r.col[k]];
    const T* tval = static_cast<const T*>(B.tval);
    for (int k = r.t0; k < r.t1; ++k) acc -= tval[k] * u[B.tcol[k]];
    tl[r.sl] = acc;
    if (r.si >= 0) static_cast<T*>(B.tS)[r.si] = acc;
  }
  if (!stage_ready(B.stage1 != 0, bar, B.fault)) return false;
  const T* M = B.stage1 ? sm : static_cast<const T*>(B.blob) + C.b1;
  T* y = sm + L.p1_y();
  cta_gemv_cm<T>(M, C.ni + C.nv, C.ni + C.nv, C.ni, tl, sm + L.p1_part(), y);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int q = tid + k * kChunkThreads;
    if (r.oi[k] < 0) continue;
    if (q < C.ni) static_cast<T*>(B.z)[r.oi[k]] = y[q];
    else static_cast<T*>(B.q)[r.oi[k]] = y[q];
  }
  return true;
}

// Phase 2, one CTA per chunk: with the held rows of inv(S) (row-major) and
// W_c (column-major) staged, form the interface right-hand side t_S - the
// sum of contributions (each interface's in chunk order), x = inv(S) rows
// times it, then x_I = z - W_c x_S, and write the interior and own
// interface rows (with their merged-away cells).  p2_load reads the setup
// data (the interface pointers into shared memory, this thread's rows and
// their destinations); after the wait, t_S, the contributions and z come in
// one batch of independent loads.
struct P2Pre {
  bool hi, ho;
  int pi, ro, wr;
  BlockDst di, dob;
};

__device__ __forceinline__ void p2_load(const BlockDev& B, const ChunkDev& C, int* qp, P2Pre& r) {
  const int tid = threadIdx.x;
  for (int k = tid; k <= B.ns; k += blockDim.x) qp[k] = B.qptr[k];
  r.hi = tid < C.ni;
  r.ho = tid < C.nown;
  r.pi = r.hi ? B.ipos[C.ipos_off + tid] : 0;
  r.ro = r.ho ? B.orow[C.o_off + tid] : 0;
  r.wr = tid < C.nw ? B.wrow[C.w_off + tid] : 0;
  if (r.hi) r.di.load(B, r.pi);
  if (r.ho) r.dob.load(B, B.opos[C.o_off + tid]);
}

template <class T>
__device__ __forceinline__ void p2_run(const BlockDev& B, const ChunkSmem& L, const ChunkDev& C,
                                       const P2Pre& r, const int* qp, T* __restrict__ u, T* sm,
                                       uint64_t* bar) {
  const int tid = threadIdx.x;
  T* ys = sm + L.p2_ys();
  T* qs = sm + L.p2_q();
  const T* tS = static_cast<const T*>(B.tS);
  const T* q = static_cast<const T*>(B.q);
  for (int k = tid; k < B.ns; k += blockDim.x) ys[k] = tS[k];
  for (int j = tid; j < B.nslots; j += blockDim.x) qs[j] = q[j];
  const T zi = r.hi ? static_cast<const T*>(B.z)[r.pi] : T(0);
  __syncthreads();
  for (int k = tid; k < B.ns; k += blockDim.x) {
    T acc = ys[k];
    for (int j = qp[k]; j < qp[k + 1]; ++j) acc -= qs[j];
    ys[k] = acc;
  }
  if (!stage_ready(B.stage2 != 0, bar, B.fault)) return;
  const T* S = B.stage2 ? sm : static_cast<const T*>(B.blob) + C.b2;
  const T* W = S + (size_t)C.nr * B.ns;
  T* xr = sm + L.p2_xr();
  T* xw = sm + L.p2_xw();
  T* part = sm + L.p2_part();
  T* y = sm + L.p2_y();
  cta_gemv_rm<T>(S, C.nr, B.ns, B.ns, ys, xr);
  if (tid < C.nw) xw[tid] = xr[r.wr];
  __syncthreads();
  cta_gemv_cm<T>(W, C.ni, C.ni, C.nw, xw, part, y);
  if (r.hi) r.di.write(B, u, zi - y[tid]);
  if (r.ho) r.dob.write(B, u, xr[r.ro]);
}

// Launch 1: phase 1.
template <class T>
__global__ void __launch_bounds__(kChunkThreads) k_block_p1(BlockDev B, ChunkSmem L,
                                                          const T* __restrict__ b,
                                                          const T* __restrict__ u) {
  extern __shared__ float4 smem_f4[];
  __shared__ __align__(8) uint64_t bar;
  T* sm = reinterpret_cast<T*>(smem_f4);
  const ChunkDev C = B.ch[blockIdx.x];
  if (B.stage1 && threadIdx.x == 0)
    bulk_stage(sm, static_cast<const T*>(B.blob) + C.b1, (unsigned)(C.b1n * sizeof(T)), &bar);
  P1Pre<T> r;
  p1_load<T>(B, C, r);
  pdl_enter();
  p1_run<T>(B, L, C, r, b, u, sm, &bar);
  pdl_exit();
}

// Launch 2: phase 2.
template <class T>
__global__ void __launch_bounds__(kChunkThreads) k_block_p2(BlockDev B, ChunkSmem L,
                                                          T* __restrict__ u) {
  extern __shared__ float4 smem_f4[];
  __shared__ __align__(8) uint64_t bar;
  T* sm = reinterpret_cast<T*>(smem_f4);
  int* qp = reinterpret_cast<int*>(sm + L.p2_total());
  const ChunkDev C = B.ch[blockIdx.x];
  if (B.stage2 && threadIdx.x == 0)
    bulk_stage(sm, static_cast<const T*>(B.blob) + C.b2, (unsigned)(C.b2n * sizeof(T)), &bar);
  P2Pre r;
  p2_load(B, C, qp, r);
  pdl_enter();
  p2_run<T>(B, L, C, r, qp, u, sm, &bar);
  pdl_exit();
}

// 16-byte vectors for the rows of a dense inverse
template <class T>
using vec16_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
__device__ __forceinline__ float dot16(const float4& a, const float* t) {
  const float4 b = *reinterpret_cast<const float4*>(t);
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double dot16(const double2& a, const double* t) {
  const double2 b = *reinterpret_cast<const double2*>(t);
  return a.x * b.x + a.y * b.y;
}

// Dense block solve in one launch: every CTA gathers the whole right-hand
// side t = b - A(block, rest) u into its shared memory (the gather reads no
// block cell, so rows written meanwhile by other CTAs do not disturb it), then
// applies its share of the rows of inv(A_block), one warp per row.  Each warp
// loads the first PFV 16-byte vectors per lane of its row of the inverse into
// registers before waiting on the previous kernel (the inverse is setup data),
// so those loads overlap the wait and the gather.
template <class T>
__global__ void __launch_bounds__(1024, 1) k_block_dense(BlockDev B, const T* __restrict__ b,
                                                      T* __restrict__ u) {
  using V = vec16_t<T>;
  constexpr int W = 16 / sizeof(T);
  constexpr int PFV = sizeof(T) == 4 ? 4 : 3;
  extern __shared__ float4 smem_f4[];
  T* t = reinterpret_cast<T*>(smem_f4);
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int r0 = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nv = B.ld / W;
  const V* A0 = reinterpret_cast<const V*>(static_cast<const T*>(B.ainv) +
                                           (size_t)min(r0, B.m - 1) * B.ld);
  V a[PFV];
#pragma unroll
  for (int j = 0; j < PFV; ++j) {
    const int c = lane + 32 * j;
    if (c < nv) a[j] = A0[c];
    else a[j] = V{};
  }
  BlockDst dst;
  if (lane == 0) dst.load(B, r0);
  // everything above reads setup data only; b and u come from earlier kernels
  pdl_enter();
  for (int p = threadIdx.x; p < B.ld; p += blockDim.x) t[p] = p < B.m ? block_rhs(B, b, u, p) : T(0);
  __syncthreads();
  for (int r = r0; r < B.m; r += gridDim.x * wpb) {
    const V* A = reinterpret_cast<const V*>(static_cast<const T*>(B.ainv) + (size_t)r * B.ld);
    T acc = T(0);
    int c0 = lane;
    if (r == r0) {
#pragma unroll
      for (int j = 0; j < PFV; ++j) {
        const int c = lane + 32 * j;
        if (c < nv) acc += dot16(a[j], t + c * W);
      }
      c0 = lane + 32 * PFV;
    }
#pragma unroll 4
    for (int c = c0; c < nv; c += 32) acc += dot16(A[c], t + c * W);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (r == r0) dst.write(B, u, acc);
      else block_write(B, u, r, acc);
    }
  }
  pdl_exit();
}

// ---- a7: bottom solve, u = inv(A_c) b (FP64 matrix, row-major) --------------
// One warp per row; the FP64 products keep the coarsest-level solve exact to
// rounding whatever the cycle precision.
template <class T>
__global__ void k_bottom(const double* __restrict__ Ainv, int nc, const T* __restrict__ b,
                         T* __restrict__ u) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nc) { pdl_exit(); return; }
  const double* A = Ainv + (size_t)r * nc;
  double acc = 0.0;
#pragma unroll 4
  for (int c = lane; c < nc; c += 32) acc += A[c] * (double)b[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) u[r] = (T)acc;
  pdl_exit();
}

// ---- a0: b = f - N g -----------------------------------------------------------
__global__ void k_rhs_copy(const double* __restrict__ f, const uint8_t* __restrict__ cls,
                           double* __restrict__ b, int64_t nn) {
  pdl_enter();
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn) b[k] = cls[k] == C_EMPTY ? 0.0 : f[k];
}
__global__ void k_rhs_n(int rows, const int* __restrict__ cell, const int64_t* __restrict__ ptr,
                        const int* __restrict__ col, const double* __restrict__ val,
                        const double* __restrict__ g, double* __restrict__ b) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  double acc = 0.0;
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) acc += val[q] * g[col[q]];
  b[cell[i]] -= acc;
}

// ---- small helpers ---------------------------------------------------------------
template <class T>
__global__ void k_owner_fix(int cnt, const int* __restrict__ dst, const int* __restrict__ src,
                            T* __restrict__ e) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) e[dst[i]] = e[src[i]];
}

template <class T>
__global__ void k_prolong_add(T* __restrict__ u, const T* __restrict__ ec,
                              const uint8_t* __restrict__ cls, int n) {
  pdl_enter();
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)n * n) return;
  if (cls[k] == C_EMPTY) return;
  int gx = (int)(k % n), gy = (int)(k / n);
  u[k] += ec[(size_t)(gy >> 1) * (n >> 1) + (gx >> 1)];
}

// u64 += e (non-empty cells)
template <class T>
__global__ void k_update(double* __restrict__ u, const T* __restrict__ e,
                         const uint8_t* __restrict__ cls, int64_t nn) {
  pdl_enter();
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn && cls[k] != C_EMPTY) u[k] += (double)e[k];
}

template <class A, class B>
__global__ void k_convert(const A* __restrict__ x, B* __restrict__ y, int64_t nn) {
  pdl_enter();
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn) y[k] = (B)x[k];
}

// ---- Krylov outer iteration (cc_options.krylov): FGMRES building blocks ------
// Not part of the paper's solver, which iterates the cycle alone: a restarted
// flexible GMRES in FP64 whose preconditioner is one FP32 cycle.  Every sum
// below runs in a fixed order, so a solve gives the same bits every time.
constexpr int KR_MAXV = 33;     // vectors of one multi-dot: restart length <= 32, plus one
constexpr int KR_BLOCKS = 152;  // CTAs of a multi-dot (one wave: one per SM at 156 registers)

// part[blk * nv + i] = this CTA's share of sum_k w[k] x_i[k] for i < nx, with
// x_i = x + i nn; when self, part[blk * nv + nx] is its share of sum_k w[k]^2
// (nv = nx + self).
__global__ void __launch_bounds__(256) k_mdot(const double* __restrict__ x, int nx,
                                              const double* __restrict__ w, int self, int64_t nn,
                                              double* __restrict__ part) {
  pdl_enter();
  __shared__ double red[8][KR_MAXV + 1];
  double acc[KR_MAXV];
#pragma unroll
  for (int i = 0; i < KR_MAXV; ++i) acc[i] = 0.0;
  double ws = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double wk = w[k];
#pragma unroll
    for (int i = 0; i < KR_MAXV; ++i)
      if (i < nx) acc[i] += wk * x[(size_t)i * nn + k];
    ws += wk * wk;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KR_MAXV; ++i) {
    if (i >= nx) break;
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if (lane == 0) red[warp][KR_MAXV] = ws;
  __syncthreads();
  const int nv = nx + self;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const int src = i < nx ? i : KR_MAXV;
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q][src];
    part[(size_t)blockIdx.x * nv + i] = v;
  }
  pdl_exit();
}

// out[i] = sum over the nb CTAs of part[b * nv + i]; one warp per vector
__global__ void k_mdot_sum(const double* __restrict__ part, int nv, int nb, double* __restrict__ out) {
  pdl_enter();
  const int i = blockIdx.x, lane = threadIdx.x;
  double v = 0.0;
  for (int b = lane; b < nb; b += 32) v += part[(size_t)b * nv + i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[i] = v;
  pdl_exit();
}

// y = (y - sum_{i < nx} c[i] x_i) * scale, x_i = x + i nn (c in device memory)
__global__ void k_maxpy(const double* __restrict__ x, int nx, const double* __restrict__ c,
                        double* __restrict__ y, double scale, int64_t nn) {
  pdl_enter();
  __shared__ double cs[KR_MAXV];
  for (int i = threadIdx.x; i < nx; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x) {
    double v = y[k];
    for (int i = 0; i < nx; ++i) v -= cs[i] * x[(size_t)i * nn + k];
    y[k] = v * scale;
  }
  pdl_exit();
}

// z = e on present control volumes, 0 on empty ones (to FP64)
template <class T>
__global__ void k_widen_masked(const T* __restrict__ e, const uint8_t* __restrict__ cls,
                               double* __restrict__ z, int64_t nn) {
  pdl_enter();
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn) z[k] = cls[k] == C_EMPTY ? 0.0 : (double)e[k];
}

// The convergence test of a solve on the device (Alg. 3's outer iteration,
// stopping on the relative max-norm residual): the state the host keeps in
// its own loop otherwise, updated by one thread from the max-norm word the
// residual kernels leave in norm[0] (and the bounded-wait fault word in
// norm[1]).
struct LoopState {
  double bn, first, rel, tol;
  int it, max_cycles, status, pad;
};

__global__ void k_loop_init(LoopState* st, double tol, int max_cycles) {
  st->bn = 1.0;
  st->first = -1.0;
  st->rel = 0.0;
  st->tol = tol;
  st->it = 0;
  st->max_cycles = max_cycles;
  st->status = CC_ERR_NOT_CONVERGED;
  st->pad = 0;
}

// mode 0: norm[0] holds |b|_inf; mode 1: the residual of the initial guess;
// mode 2: the residual after one more iteration.  Modes 1 and 2 set the
// loop's condition: 1 to run another iteration.
__global__ void k_loop_step(LoopState* st, const unsigned long long* __restrict__ norm, int mode,
                            cudaGraphConditionalHandle cond) {
  pdl_enter();
  const double v = __longlong_as_double((long long)norm[0]);
  if (mode == 0) {
    st->bn = v == 0.0 ? 1.0 : v;
    pdl_exit();
    return;
  }
  unsigned int more = 0;
  const double rel = v / st->bn;
  if (mode == 2) ++st->it;
  st->rel = rel;
  if (mode == 1) st->first = rel;
  if (norm[1] != 0) {
    st->status = CC_ERR_TIMEOUT;
  } else if (rel < st->tol) {
    st->status = CC_OK;
  } else if (mode == 2 && (!isfinite(rel) || (st->first > 0 && rel > 1e3 * st->first))) {
    st->status = CC_ERR_DIVERGED;
  } else if (st->it >= st->max_cycles) {
    st->status = CC_ERR_NOT_CONVERGED;
  } else {
    more = 1;
  }
  cudaGraphSetConditional(cond, more);
  pdl_exit();
}

__global__ void k_absmax(const double* __restrict__ x, int64_t nn, unsigned long long* out) {
  pdl_enter();
  double av = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x)
    av = fmax(av, fabs(x[k]));
  for (int o = 16; o > 0; o >>= 1) av = fmax(av, __shfl_xor_sync(0xffffffffu, av, o));
  if ((threadIdx.x & 31) == 0) atomic_max_abs(out, av);
}

}  // namespace ccmg
