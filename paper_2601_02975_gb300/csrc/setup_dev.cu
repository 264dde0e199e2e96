// The per-cell steps of the setup as FP64 CUDA kernels (Sec. 3.1, the
// moments of Sec. 4.2, Def. 4.1, Def. 4.3, Eq. 4.14 and 4.17-4.18, Def.
// 5.1), one thread per cell, running the functions of setup_cell.h.  This translation unit is compiled with
// --fmad=false so that its products and sums round exactly as the host's
// (-ffp-contract=off): the tables it builds are the host's, bit for bit.
//
// The host keeps the steps that search curves or depend on earlier cells:
// the crossings of the grid lines and the cut cells' boundary pieces, the
// merging of Alg. 1 (sequential by definition), the boundary quadrature
// nodes, the rows of A and N, and the factorisations of the block smoother.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "setup.h"

namespace ccmg {

namespace {

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    throw DeviceError((int)e, buf);
  }
}
#define SCK(x) check((x), #x)

__global__ void k_classify(const Hole* __restrict__ holes, int nh, int n, double x0, double y0,
                           double h, const uint8_t* __restrict__ crossed, uint8_t* __restrict__ type) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(k % n), j = (int)(k / n);
    uint8_t t = cell::T_EMPTY;
    if (!crossed[k]) {
      const double xc = x0 + (i + 0.5) * h, yc = y0 + (j + 0.5) * h;
      if (cell::outside_all(holes, nh, xc, yc)) t = cell::T_FULL;
    }
    type[k] = t;
  }
}

__global__ void k_cut_moments(const Hole* __restrict__ holes, int nc, double h,
                              const Piece* __restrict__ pieces, const int* __restrict__ ptr,
                              const double* __restrict__ px, const double* __restrict__ py,
                              Rules510 R, double* __restrict__ mom) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc) return;
  double m[cell::kNM];
  for (int q = 0; q < cell::kNM; ++q) m[q] = 0.0;
  for (int s = ptr[r]; s < ptr[r + 1]; ++s) cell::piece_moments(holes, pieces[s], px[r], py[r], h, R, m);
  for (int q = 0; q < cell::kNM; ++q) mom[(int64_t)cell::kNM * r + q] = m[q];
}

__global__ void k_kinds(const uint8_t* __restrict__ type, const uint8_t* __restrict__ ext, int n,
                        int cross, uint8_t* __restrict__ kind) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x)
    kind[k] = cell::kind_of(type, ext, n, cross != 0, (int)k);
}

__global__ void k_lattice(const uint8_t* __restrict__ type, int n, const int* __restrict__ plg,
                          int np, int* __restrict__ lat, uint8_t* __restrict__ ok) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= np) return;
  int out[15];
  const bool f = cell::plg_lattice(type, n, plg[r], out);
  for (int q = 0; q < 15; ++q) lat[(int64_t)15 * r + q] = f ? out[q] : -1;
  ok[r] = f;
}

// scaled moments of cell kj about its own centre: the cut cells' from the
// table (cut_cells sorted), the full cell's otherwise
struct DevMoments {
  const int* cells;
  const double* mom;
  int ncut;
  __device__ void operator()(int kj, double* out) const {
    int lo = 0, hi = ncut;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cells[mid] < kj) lo = mid + 1;
      else hi = mid;
    }
    if (lo < ncut && cells[lo] == kj) {
      for (int q = 0; q < cell::kNM; ++q) out[q] = mom[(int64_t)cell::kNM * lo + q];
    } else {
      cell::full_moments(out);
    }
  }
};

struct FitArgs {
  int n, np;
  double h, x0, y0, a, b, c;
  const int* plg;
  const int* lat;
  DevMoments mom;
  const BNode* bnode;
  const int* bptr;
  const double* a12;
  double* beta;
  uint8_t* ok;
};

__global__ void __launch_bounds__(64) k_fit(FitArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.np) return;
  int lat[15];
  for (int q = 0; q < 15; ++q) lat[q] = A.lat[(int64_t)15 * r + q];
  const int b0 = A.bptr[r], nb = A.bptr[r + 1] - b0;
  double beta[16];
  const bool f = cell::plg_fit(A.plg[r], A.n, A.h, A.a, A.b, A.c, lat, A.mom,
                               nb ? A.bnode + b0 : nullptr, nb, A.a12, A.x0, A.y0, beta);
  for (int q = 0; q < 16; ++q) A.beta[(int64_t)16 * r + q] = f ? beta[q] : 0.0;
  A.ok[r] = f;
}

__global__ void k_nearest(const double* __restrict__ sx, const double* __restrict__ sy, int nh,
                          int ns, const double* __restrict__ px, const double* __restrict__ py,
                          int m, int* __restrict__ idx, double* __restrict__ d2) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * nh) return;
  const int r = (int)(t / nh), e = (int)(t % nh);
  double d;
  idx[t] = cell::nearest_sample(sx + (int64_t)e * ns, sy + (int64_t)e * ns, ns, px[r], py[r], &d);
  d2[t] = d;
}

// Gauss-Jordan step c of [A | J] (the identity half J kept in the order of
// the pivot steps, as the host's dense inversion keeps it): pivot search
// (the first row of largest magnitude in column c), row swap, scaling of
// the pivot row, and the multipliers of column c.  One CTA.
__global__ void __launch_bounds__(1024) k_gj_pivot(double* __restrict__ A, double* __restrict__ J, int n,
                                                  int c, double tol, int* __restrict__ orig,
                                                  int* __restrict__ cols, double* __restrict__ lcol,
                                                  int* __restrict__ flag) {
  __shared__ double sv[32];
  __shared__ int sr[32];
  __shared__ int piv;
  __shared__ double dinv;
  if (*flag) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double bv = -1.0;
  int br = n;
  for (int r = c + tid; r < n; r += blockDim.x) {
    const double v = fabs(A[(int64_t)r * n + c]);
    if (v > bv) { bv = v; br = r; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, bv, o);
    const int orr = __shfl_down_sync(0xffffffffu, br, o);
    if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
  }
  if (lane == 0) { sv[warp] = bv; sr[warp] = br; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > sv[0] || (sv[w] == sv[0] && sr[w] < sr[0])) { sv[0] = sv[w]; sr[0] = sr[w]; }
    piv = sr[0];
    if (!(piv < n && fabs(A[(int64_t)piv * n + c]) > tol)) *flag = 1;
  }
  __syncthreads();
  if (*flag) return;
  const int p = piv;
  if (p != c) {
    for (int k = c + tid; k < n; k += blockDim.x) {
      const double t = A[(int64_t)p * n + k];
      A[(int64_t)p * n + k] = A[(int64_t)c * n + k];
      A[(int64_t)c * n + k] = t;
    }
    for (int k = tid; k < c; k += blockDim.x) {
      const double t = J[(int64_t)p * n + k];
      J[(int64_t)p * n + k] = J[(int64_t)c * n + k];
      J[(int64_t)c * n + k] = t;
    }
    if (tid == 0) { const int t = orig[p]; orig[p] = orig[c]; orig[c] = t; }
  }
  __syncthreads();
  if (tid == 0) {
    cols[c] = orig[c];
    J[(int64_t)c * n + c] = 1.0;
    dinv = 1.0 / A[(int64_t)c * n + c];
  }
  __syncthreads();
  const double d = dinv;
  for (int k = c + tid; k < n; k += blockDim.x) A[(int64_t)c * n + k] *= d;
  for (int k = tid; k <= c; k += blockDim.x) J[(int64_t)c * n + k] *= d;
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) lcol[r] = r == c ? 0.0 : A[(int64_t)r * n + c];
}

// Gauss-Jordan step c: every row r != c with a nonzero multiplier l loses l
// times the pivot row, in columns c.. of A and 0..c of J.
__global__ void k_gj_elim(double* __restrict__ A, double* __restrict__ J, int n, int c,
                          const double* __restrict__ lcol, const int* __restrict__ flag) {
  if (*flag) return;
  const int64_t w = (int64_t)n + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / w), t = (int)(e % w);
    const double l = lcol[r];
    if (r == c || l == 0.0) continue;
    if (t <= c) J[(int64_t)r * n + t] -= l * J[(int64_t)c * n + t];
    else A[(int64_t)r * n + (t - 1)] -= l * A[(int64_t)c * n + (t - 1)];
  }
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// the stream, timing events and the type map of the level being built
struct SetupDevice::Impl {
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  uint8_t* type = nullptr;      // the type map of the current level
  size_t type_cap = 0;
  int type_n = 0;
  // a scratch allocation for the duration of one call
  struct Scratch {
    Impl* I;
    std::vector<void*> ps;
    template <class T> T* get(size_t count) {
      void* p = nullptr;
      SCK(cudaMalloc(&p, count * sizeof(T) + 16));
      ps.push_back(p);
      return static_cast<T*>(p);
    }
    template <class T> T* put(const T* h, size_t count) {
      T* d = get<T>(count);
      if (count) SCK(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, I->s));
      return d;
    }
    ~Scratch() {
      cudaStreamSynchronize(I->s);
      for (void* p : ps) cudaFree(p);
    }
  };
  void ensure_type(size_t nn) {
    if (type_cap >= nn) return;
    if (type) cudaFree(type);
    type = nullptr;
    SCK(cudaMalloc(&type, nn));
    type_cap = nn;
  }
  void begin() { SCK(cudaEventRecord(e0, s)); }
  void end(double& ms) {
    SCK(cudaEventRecord(e1, s));
    SCK(cudaGetLastError());
    SCK(cudaEventSynchronize(e1));
    float t = 0;
    SCK(cudaEventElapsedTime(&t, e0, e1));
    ms += t;
  }
};

SetupDevice::SetupDevice(void* stream) : p_(new Impl) {
  p_->s = (cudaStream_t)stream;
  try {
    SCK(cudaEventCreate(&p_->e0));
    SCK(cudaEventCreate(&p_->e1));
  } catch (...) {
    if (p_->e0) cudaEventDestroy(p_->e0);
    delete p_;
    throw;
  }
}

SetupDevice::~SetupDevice() {
  cudaStreamSynchronize(p_->s);
  if (p_->type) cudaFree(p_->type);
  cudaEventDestroy(p_->e0);
  cudaEventDestroy(p_->e1);
  delete p_;
}

void SetupDevice::classify(const Problem& P, int n, double h, const uint8_t* crossed, uint8_t* type) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const size_t nn = (size_t)n * n;
  const int nh = (int)P.holes.size();
  const Hole* dh = S.put(P.holes.data(), (size_t)nh);
  const uint8_t* dc = S.put(crossed, nn);
  uint8_t* dt = S.get<uint8_t>(nn);
  I.begin();
  k_classify<<<grid_for((int64_t)nn, 256), 256, 0, I.s>>>(dh, nh, n, P.x0, P.y0, h, dc, dt);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(type, dt, nn, cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

void SetupDevice::moments(const Problem& P, double h, const std::vector<int>& cells,
                          const std::vector<Piece>& pieces, const std::vector<int>& ptr,
                          const std::vector<double>& px, const std::vector<double>& py,
                          const Rules510& R, double* mom) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const int nc = (int)cells.size();
  const Hole* dh = S.put(P.holes.data(), P.holes.size());
  const Piece* dp = S.put(pieces.data(), pieces.size());
  const int* dptr = S.put(ptr.data(), ptr.size());
  const double* dx = S.put(px.data(), px.size());
  const double* dy = S.put(py.data(), py.size());
  double* dm = S.get<double>((size_t)cell::kNM * nc);
  I.begin();
  k_cut_moments<<<(nc + 63) / 64, 64, 0, I.s>>>(dh, nc, h, dp, dptr, dx, dy, R, dm);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(mom, dm, (size_t)cell::kNM * nc * sizeof(double), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

void SetupDevice::kinds(int n, bool cross, const uint8_t* type, const uint8_t* ext, uint8_t* kind) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const size_t nn = (size_t)n * n;
  I.ensure_type(nn);
  I.type_n = n;
  SCK(cudaMemcpyAsync(I.type, type, nn, cudaMemcpyHostToDevice, I.s));
  const uint8_t* de = S.put(ext, (size_t)4 * n);
  uint8_t* dk = S.get<uint8_t>(nn);
  I.begin();
  k_kinds<<<grid_for((int64_t)nn, 256), 256, 0, I.s>>>(I.type, de, n, cross ? 1 : 0, dk);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(kind, dk, nn, cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

void SetupDevice::lattices(int n, const std::vector<int>& plg, int* lat, uint8_t* ok) {
  Impl& I = *p_;
  if (I.type_n != n) throw DeviceError(1, "lattices: no type map of this level on the device");
  Impl::Scratch S{&I, {}};
  const int np = (int)plg.size();
  const int* dp = S.put(plg.data(), (size_t)np);
  int* dl = S.get<int>((size_t)15 * np);
  uint8_t* dok = S.get<uint8_t>((size_t)np);
  I.begin();
  k_lattice<<<(np + 127) / 128, 128, 0, I.s>>>(I.type, n, dp, np, dl, dok);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(lat, dl, (size_t)15 * np * sizeof(int), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaMemcpyAsync(ok, dok, (size_t)np, cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

void SetupDevice::fits(int n, double h, double x0, double y0, double a, double b, double c,
                       const std::vector<int>& plg, const int* lat, const std::vector<int>& cut_cells,
                       const std::vector<double>& cut_mom, const std::vector<BNode>& bnode,
                       const std::vector<int>& bptr, const std::vector<double>& a12, double* beta,
                       uint8_t* ok) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const int np = (int)plg.size();
  FitArgs A;
  A.n = n;
  A.np = np;
  A.h = h;
  A.x0 = x0;
  A.y0 = y0;
  A.a = a;
  A.b = b;
  A.c = c;
  A.plg = S.put(plg.data(), (size_t)np);
  A.lat = S.put(lat, (size_t)15 * np);
  A.mom.cells = S.put(cut_cells.data(), cut_cells.size());
  A.mom.mom = S.put(cut_mom.data(), cut_mom.size());
  A.mom.ncut = (int)cut_cells.size();
  A.bnode = S.put(bnode.data(), bnode.size());
  A.bptr = S.put(bptr.data(), bptr.size());
  A.a12 = S.put(a12.data(), a12.size());
  A.beta = S.get<double>((size_t)16 * np);
  A.ok = S.get<uint8_t>((size_t)np);
  I.begin();
  k_fit<<<(np + 63) / 64, 64, 0, I.s>>>(A);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(beta, A.beta, (size_t)16 * np * sizeof(double), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaMemcpyAsync(ok, A.ok, (size_t)np, cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

bool SetupDevice::invert(std::vector<double>& A, int n) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const size_t nn = (size_t)n * n;
  double amax = 0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  std::vector<int> orig(n);
  for (int i = 0; i < n; ++i) orig[i] = i;
  double* dA = S.put(A.data(), nn);
  double* dJ = S.get<double>(nn);
  SCK(cudaMemsetAsync(dJ, 0, nn * sizeof(double), I.s));
  int* dorig = S.put(orig.data(), (size_t)n);
  int* dcols = S.get<int>((size_t)n);
  double* dl = S.get<double>((size_t)n);
  int* dflag = S.get<int>(1);
  SCK(cudaMemsetAsync(dflag, 0, sizeof(int), I.s));
  const int g = grid_for((int64_t)n * (n + 1), 256);
  I.begin();
  for (int c = 0; c < n; ++c) {
    k_gj_pivot<<<1, 1024, 0, I.s>>>(dA, dJ, n, c, 1e-14 * amax, dorig, dcols, dl, dflag);
    k_gj_elim<<<g, 256, 0, I.s>>>(dA, dJ, n, c, dl, dflag);
  }
  I.end(kernel_ms);
  int flag = 0;
  std::vector<double> Jh(nn);
  std::vector<int> cols(n);
  SCK(cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaMemcpyAsync(Jh.data(), dJ, nn * sizeof(double), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaMemcpyAsync(cols.data(), dcols, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
  if (flag) return false;
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < n; ++j) A[(size_t)r * n + cols[j]] = Jh[(size_t)r * n + j];
  return true;
}

void SetupDevice::nearest(const double* sx, const double* sy, int nh, int ns, const double* px,
                          const double* py, int m, int* idx, double* d2) {
  Impl& I = *p_;
  Impl::Scratch S{&I, {}};
  const size_t nt = (size_t)m * nh;
  const double* dsx = S.put(sx, (size_t)nh * ns);
  const double* dsy = S.put(sy, (size_t)nh * ns);
  const double* dpx = S.put(px, (size_t)m);
  const double* dpy = S.put(py, (size_t)m);
  int* di = S.get<int>(nt);
  double* dd = S.get<double>(nt);
  I.begin();
  k_nearest<<<(int)((nt + 127) / 128), 128, 0, I.s>>>(dsx, dsy, nh, ns, dpx, dpy, m, di, dd);
  I.end(kernel_ms);
  SCK(cudaMemcpyAsync(idx, di, nt * sizeof(int), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaMemcpyAsync(d2, dd, nt * sizeof(double), cudaMemcpyDeviceToHost, I.s));
  SCK(cudaStreamSynchronize(I.s));
}

}  // namespace ccmg
