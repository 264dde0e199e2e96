// C ABI of the cut-cell multigrid library: hierarchy construction (host,
// FP64), device tables, the multigrid cycle (Alg. 2) and the solve loops.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/ccmg.h"
#include "kernels.cuh"
#include "setup.h"

using namespace ccmg;

namespace {

// kernels launched by the current host thread (read around each solve)
thread_local int64_t t_launches = 0;

struct CudaError {
  cudaError_t e;
};
// text of the last CUDA error seen by a call from this host thread
thread_local char t_last_error[256] = "";
inline void note_error(cudaError_t e, const char* what) {
  snprintf(t_last_error, sizeof(t_last_error), "%s: %s (%s)", what, cudaGetErrorString(e),
           cudaGetErrorName(e));
}
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      note_error(e_, #x);                       \
      throw CudaError{e_};                      \
    }                                           \
  } while (0)

// Launch with the programmatic-stream-serialisation attribute (PDL); the
// kernels call pdl_enter() first, which waits for the previous kernel's
// completion and memory flush, so only the launch latency overlaps.
// CCMG_PDL in the environment: 0 off, 1 on with dependents released at kernel
// entry, 2 (default) on with release at exit, 3 on without explicit release.
int pdl_mode() {
  static const int mode = [] {
    const char* e = getenv("CCMG_PDL");
    return e ? atoi(e) : 2;
  }();
  return mode;
}
bool pdl_enabled() { return pdl_mode() != 0; }

// publish the trigger placement to the device (once per device)
void pdl_setup_device() {
  int trig = pdl_mode() == 1 ? 1 : pdl_mode() == 2 ? 2 : 0;
  CK(cudaMemcpyToSymbol(g_pdl_trigger, &trig, sizeof(int)));
}

template <typename... KArgs, typename... Args>
void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args... args) {
  ++t_launches;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

// ---------------------------------------------------------------------------
// dense helpers (host, FP64)
// A reusable barrier for the threads of one host computation.
struct HostBarrier {
  std::mutex m;
  std::condition_variable cv;
  unsigned n, count = 0;
  uint64_t gen = 0;
  explicit HostBarrier(unsigned n_) : n(n_) {}
  void wait() {
    std::unique_lock<std::mutex> lk(m);
    const uint64_t g = gen;
    if (++count == n) {
      count = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return gen != g; });
    }
  }
};

// in-place inverse by Gauss-Jordan with partial pivoting; false if singular.
// From n = 512 on, the row eliminations of each pivot step are split over
// host threads; every element sees the same operations in the same order as
// with one thread, so the result does not depend on the thread count.
bool invert(std::vector<double>& A, int n) {
  // [A | I] Gauss-Jordan with the identity half stored by pivot step: column
  // j of J holds column cols[j] of I, the identity column of the row chosen as
  // pivot j.  Before its step a row's own identity entry is implicit, and
  // every other entry outside the first c + 1 columns is an exact zero, so
  // step c updates columns c.. of A and 0..c of J only.
  std::vector<double> J((size_t)n * n, 0.0);
  std::vector<int> orig(n), cols(n);
  for (int i = 0; i < n; ++i) orig[i] = i;
  double amax = 0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  auto pivot = [&](int c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (!(std::fabs(A[(size_t)p * n + c]) > 1e-14 * amax)) return false;
    if (p != c) {
      for (int k = c; k < n; ++k) std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
      for (int k = 0; k < c; ++k) std::swap(J[(size_t)p * n + k], J[(size_t)c * n + k]);
      std::swap(orig[p], orig[c]);
    }
    cols[c] = orig[c];
    J[(size_t)c * n + c] = 1.0;
    double d = 1.0 / A[(size_t)c * n + c];
    for (int k = c; k < n; ++k) A[(size_t)c * n + k] *= d;
    for (int k = 0; k <= c; ++k) J[(size_t)c * n + k] *= d;
    return true;
  };
  auto eliminate = [&](int c, int r0, int r1) {
    const double* ac = &A[(size_t)c * n];
    const double* jc = &J[(size_t)c * n];
    for (int r = r0; r < r1; ++r) {
      if (r == c) continue;
      double* ar = &A[(size_t)r * n];
      double* jr = &J[(size_t)r * n];
      const double l = ar[c];
      if (l == 0.0) continue;
      for (int k = c; k < n; ++k) ar[k] -= l * ac[k];
      for (int k = 0; k <= c; ++k) jr[k] -= l * jc[k];
    }
  };
  unsigned T = 1;
  if (n >= 512) T = std::max(1u, std::min({std::thread::hardware_concurrency(), 16u, (unsigned)(n / 128)}));
  if (T == 1) {
    for (int c = 0; c < n; ++c) {
      if (!pivot(c)) return false;
      eliminate(c, 0, n);
    }
  } else {
    HostBarrier bar(T);
    bool singular = false;
    auto work = [&](unsigned t) {
      const int r0 = (int)((int64_t)n * t / T), r1 = (int)((int64_t)n * (t + 1) / T);
      for (int c = 0; c < n; ++c) {
        if (t == 0) singular = !pivot(c);
        bar.wait();                      // pivot row ready (or the matrix is singular)
        if (singular) return;
        eliminate(c, r0, r1);
        bar.wait();                      // column c eliminated everywhere
      }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < T; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    if (singular) return false;
  }
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < n; ++j) A[(size_t)r * n + cols[j]] = J[(size_t)r * n + j];
  return true;
}


// row-major n x m -> column-major
std::vector<double> to_cm(const std::vector<double>& A, int rows, int cols) {
  std::vector<double> B((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) B[(size_t)c * rows + r] = A[(size_t)r * cols + c];
  return B;
}

// ---------------------------------------------------------------------------
// exact block solve plan (host)
struct BlockPlan {
  int m = 0;
  std::vector<int> cell;
  std::vector<int64_t> gptr{0};
  std::vector<int> gcol;
  std::vector<double> gval;
  int gk = 0;                          // ELL width of the gather
  std::vector<int> ell_col;            // [gk * m] term-major
  std::vector<double> ell_val;
  std::vector<int> tail_ptr{0}, tail_col;   // terms beyond the width
  std::vector<double> tail_val;
  std::vector<int> alias_ptr{0}, alias_cell;
  double error = 0;    // backward error of the solve on a fixed vector (FP64, host)
  int band = 0;        // bandwidth of the block in curve order (couplings <= 64 apart)
  // dense form (m <= kDenseMax): the inverse, row-major
  bool dense = false;
  std::vector<double> ainv;
  // chunked form
  int nch = 0, ns = 0, s = 0, nslots = 0;
  std::vector<ChunkDev> ch;
  std::vector<int> slot, sidx, ipos, vslot, wrow, orow, opos, qptr, spos;
  std::vector<double> blob;
  ChunkSmem sm{};      // shared-memory layout at w = 1 element (st1, st2 filled per precision)
  int b1max = 0, b2max = 0;
};

const int kDenseMax = 1024;     // blocks up to this size: dense inverse, one launch
// dynamic shared memory of one CTA that the chunked launches may use (the
// opt-in limit is 227 KiB per CTA, static shared memory included)
const int kSmemBudget = 226 * 1024;

// The chunked solve applied to t in FP64, as the device does it.
void apply_chunked(const BlockPlan& B, const std::vector<double>& t, std::vector<double>& x) {
  const int m = B.m;
  std::vector<double> z(m, 0.0), q(std::max(1, B.nslots), 0.0), ys(B.ns, 0.0);
  x.assign(m, 0.0);
  for (const ChunkDev& C : B.ch) {
    std::vector<double> tl(C.p1 - C.p0);
    for (int p = C.p0; p < C.p1; ++p) tl[B.slot[p]] = t[p];
    const double* M = &B.blob[C.b1];
    const int ld = C.ni + C.nv;
    for (int r = 0; r < ld; ++r) {
      double acc = 0;
      for (int k = 0; k < C.ni; ++k) acc += M[(size_t)k * ld + r] * tl[k];
      if (r < C.ni) z[B.ipos[C.ipos_off + r]] = acc;
      else q[B.vslot[C.v_off + r - C.ni]] = acc;
    }
  }
  for (int k = 0; k < B.ns; ++k) {
    double acc = t[B.spos[k]];
    for (int j = B.qptr[k]; j < B.qptr[k + 1]; ++j) acc -= q[j];
    ys[k] = acc;
  }
  for (const ChunkDev& C : B.ch) {
    const double* S = &B.blob[C.b2];
    const double* W = S + (size_t)C.nr * B.ns;
    std::vector<double> xr(C.nr, 0.0), xw(C.nw);
    for (int r = 0; r < C.nr; ++r)
      for (int k = 0; k < B.ns; ++k) xr[r] += S[(size_t)r * B.ns + k] * ys[k];
    for (int k = 0; k < C.nw; ++k) xw[k] = xr[B.wrow[C.w_off + k]];
    for (int r = 0; r < C.ni; ++r) {
      double acc = 0;
      for (int k = 0; k < C.nw; ++k) acc += W[(size_t)k * C.ni + r] * xw[k];
      const int pos = B.ipos[C.ipos_off + r];
      x[pos] = z[pos] - acc;
    }
    for (int k = 0; k < C.nown; ++k) x[B.opos[C.o_off + k]] = xr[B.orow[C.o_off + k]];
  }
}

void apply_dense(const BlockPlan& B, const std::vector<double>& t, std::vector<double>& x) {
  x.assign(B.m, 0.0);
  for (int r = 0; r < B.m; ++r) {
    double acc = 0;
    for (int k = 0; k < B.m; ++k) acc += B.ainv[(size_t)r * B.m + k] * t[k];
    x[r] = acc;
  }
}

// Apply the solve to a fixed vector and return the normwise backward error
// |A x - t|_inf / (|A|_inf |x|_inf).
double block_plan_error(const BlockPlan& B, const std::vector<std::map<int, double>>& Abb) {
  const int m = B.m;
  std::vector<double> t(m), x;
  for (int p = 0; p < m; ++p) t[p] = std::sin(1.0 + 0.7 * p) + 0.25 * std::cos(3.1 * p);
  if (B.dense) apply_dense(B, t, x);
  else apply_chunked(B, t, x);
  double rmax = 0, amax = 0, xmax = 0;
  for (int p = 0; p < m; ++p) {
    double acc = -t[p], arow = 0;
    for (auto& kv : Abb[p]) { acc += kv.second * x[kv.first]; arow += std::fabs(kv.second); }
    rmax = std::max(rmax, std::fabs(acc));
    amax = std::max(amax, arow);
    xmax = std::max(xmax, std::fabs(x[p]));
  }
  return rmax / (amax * xmax);
}

// padded term-major (ELL) copy of the gather rows
void make_ell(BlockPlan& B) {
  const int m = B.m;
  // width: the longest PLG row (at most 15 terms); the few longer rows
  // (box-corner rows with ghost expansions) spill into a tail.  The chunked
  // launch holds a row's terms in registers, kGatherMax of them.
  B.gk = 0;
  for (int p = 0; p < m; ++p) B.gk = std::max<int>(B.gk, (int)(B.gptr[p + 1] - B.gptr[p]));
  B.gk = std::min(B.gk, kGatherMax);
  B.ell_col.assign((size_t)B.gk * m, 0);
  B.ell_val.assign((size_t)B.gk * m, 0.0);
  B.tail_ptr.assign(1, 0);
  B.tail_col.clear();
  B.tail_val.clear();
  for (int p = 0; p < m; ++p) {
    int q = 0;
    for (int64_t e = B.gptr[p]; e < B.gptr[p + 1]; ++e, ++q) {
      if (q < B.gk) {
        B.ell_col[(size_t)q * m + p] = B.gcol[e];
        B.ell_val[(size_t)q * m + p] = B.gval[e];
      } else {
        B.tail_col.push_back(B.gcol[e]);
        B.tail_val.push_back(B.gval[e]);
      }
    }
    for (; q < B.gk; ++q) B.ell_col[(size_t)q * m + p] = B.cell[p];   // value 0
    B.tail_ptr.push_back((int)B.tail_col.size());
  }
}

inline int round4(int v) { return (v + 3) & ~3; }

// Structure of the chunked solve for chunks of s rows (no numbers): interface
// rows, interior lists, the interface rows each chunk reads and is read by.
struct ChunkShape {
  int s = 0, nch = 0, ns = 0;
  std::vector<int> sidx, spos;
  std::vector<std::vector<int>> I, own, sout, sin, held;   // per chunk
  double cost = 0;   // largest per-CTA stage bytes (FP32), doubled beyond one wave
  bool ok = true;
};

ChunkShape chunk_shape(const std::vector<std::map<int, double>>& Abb, int s) {
  ChunkShape S;
  const int m = (int)Abb.size();
  S.s = s;
  S.nch = (m + s - 1) / s;
  std::vector<char> iface(m, 0);
  for (int r = 0; r < m; ++r)
    for (auto& kv : Abb[r]) {
      const int c = kv.first, cr = r / s, cc = c / s;
      if (cr != cc) iface[cr < cc ? r : c] = 1;
    }
  S.sidx.assign(m, -1);
  for (int p = 0; p < m; ++p)
    if (iface[p]) { S.sidx[p] = (int)S.spos.size(); S.spos.push_back(p); }
  S.ns = (int)S.spos.size();
  S.I.resize(S.nch);
  S.own.resize(S.nch);
  S.sout.resize(S.nch);
  S.sin.resize(S.nch);
  S.held.resize(S.nch);
  std::vector<std::vector<int>> readers(S.ns);   // interior chunks an interface row reads
  for (int p = 0; p < m; ++p) {
    if (iface[p]) {
      S.own[p / s].push_back(S.sidx[p]);
      for (auto& kv : Abb[p])
        if (!iface[kv.first]) readers[S.sidx[p]].push_back(kv.first / s);
    } else {
      S.I[p / s].push_back(p);
    }
  }
  for (int i = 0; i < S.ns; ++i) {
    auto& v = readers[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    for (int c : v) S.sin[c].push_back(i);
  }
  double worst = 0;
  for (int c = 0; c < S.nch; ++c) {
    std::vector<int> so;
    for (int p : S.I[c])
      for (auto& kv : Abb[p])
        if (iface[kv.first]) so.push_back(S.sidx[kv.first]);
    std::sort(so.begin(), so.end());
    so.erase(std::unique(so.begin(), so.end()), so.end());
    S.sout[c] = so;
    std::vector<int> hd = so;
    hd.insert(hd.end(), S.own[c].begin(), S.own[c].end());
    std::sort(hd.begin(), hd.end());
    hd.erase(std::unique(hd.begin(), hd.end()), hd.end());
    S.held[c] = hd;
    const double ni = (double)S.I[c].size(), nv = (double)S.sin[c].size();
    // launch 1 forms up to 2 product rows per thread, launch 2 takes one
    // interior row, one own interface row and one W_c column per thread
    if (ni + nv > 32 * kRB || so.size() > (size_t)kChunkThreads) S.ok = false;
    const double b1 = (ni + nv) * ni, b2 = (double)hd.size() * S.ns + ni * (double)so.size();
    worst = std::max(worst, 4.0 * (b1 + b2));
  }
  S.cost = worst * (S.nch > 148 ? 2.0 : 1.0);
  return S;
}

// Numbers of the chunked solve for shape S (FP64): chunk inverses, V_c, W_c,
// the interface Schur complement and its inverse, laid out per chunk.
// a dense inversion: the host's, or the device's (bitwise the same)
using Inverter = std::function<bool(std::vector<double>&, int)>;

void build_chunked(BlockPlan& B, const std::vector<std::map<int, double>>& Abb, const ChunkShape& S,
                   const Inverter* inv = nullptr) {
  const int m = B.m, ns = S.ns, nch = S.nch;
  B.s = S.s;
  B.nch = nch;
  B.ns = ns;
  B.spos = S.spos;
  B.sidx = S.sidx;
  B.slot.assign(m, 0);
  B.ch.assign(nch, ChunkDev{});
  B.ipos.clear();
  B.vslot.clear();
  B.wrow.clear();
  B.orow.clear();
  B.opos.clear();
  B.blob.clear();
  // q slots: the contributions to interface i, in chunk order
  B.qptr.assign(ns + 1, 0);
  for (int c = 0; c < nch; ++c)
    for (int i : S.sin[c]) ++B.qptr[i + 1];
  for (int i = 0; i < ns; ++i) B.qptr[i + 1] += B.qptr[i];
  B.nslots = B.qptr[ns];
  std::vector<int> qnext(B.qptr.begin(), B.qptr.end() - 1);
  std::vector<double> Sm((size_t)ns * ns, 0.0);
  for (int i = 0; i < ns; ++i)
    for (auto& kv : Abb[S.spos[i]])
      if (S.sidx[kv.first] >= 0) Sm[(size_t)i * ns + S.sidx[kv.first]] += kv.second;
  // per chunk: inverse of the interior block, V_c and W_c (parallel over chunks)
  std::vector<std::vector<double>> Ainv(nch), V(nch), W(nch);
  std::atomic<int> next{0};
  std::atomic<bool> singular{false};
  auto work = [&]() {
    for (int c = next++; c < nch; c = next++) {
      const auto& Ic = S.I[c];
      const int ni = (int)Ic.size(), nv = (int)S.sin[c].size(), nw = (int)S.sout[c].size();
      std::unordered_map<int, int> lp;
      for (int k = 0; k < ni; ++k) lp[Ic[k]] = k;
      std::vector<double> A((size_t)ni * ni, 0.0);
      for (int k = 0; k < ni; ++k)
        for (auto& kv : Abb[Ic[k]]) {
          auto it = lp.find(kv.first);
          if (it != lp.end()) A[(size_t)k * ni + it->second] += kv.second;
        }
      if (ni && !invert(A, ni)) { singular = true; continue; }
      // W_c = inv(A_cc) A_{c,S} on the columns sout[c]
      std::unordered_map<int, int> wc;
      for (int k = 0; k < nw; ++k) wc[S.sout[c][k]] = k;
      std::vector<double> AcS((size_t)ni * nw, 0.0);
      for (int k = 0; k < ni; ++k)
        for (auto& kv : Abb[Ic[k]])
          if (S.sidx[kv.first] >= 0) AcS[(size_t)k * nw + wc[S.sidx[kv.first]]] += kv.second;
      std::vector<double> Wc((size_t)ni * nw, 0.0);
      for (int r = 0; r < ni; ++r)
        for (int k = 0; k < ni; ++k) {
          const double a = A[(size_t)r * ni + k];
          if (a == 0.0) continue;
          for (int j = 0; j < nw; ++j) Wc[(size_t)r * nw + j] += a * AcS[(size_t)k * nw + j];
        }
      // V_c = A_{S,c} inv(A_cc) on the rows sin[c]
      std::vector<double> Vc((size_t)nv * ni, 0.0);
      for (int a = 0; a < nv; ++a)
        for (auto& kv : Abb[S.spos[S.sin[c][a]]]) {
          auto it = lp.find(kv.first);
          if (it == lp.end()) continue;
          const double v = kv.second;
          const double* ar = &A[(size_t)it->second * ni];
          for (int k = 0; k < ni; ++k) Vc[(size_t)a * ni + k] += v * ar[k];
        }
      Ainv[c].swap(A);
      W[c].swap(Wc);
      V[c].swap(Vc);
    }
  };
  {
    const unsigned T = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < T && (int)t < nch; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
  }
  if (singular) throw SetupError(3, "singular interior block of the smoother");
  // Schur complement: S -= A_{S,c} W_c, in chunk order
  for (int c = 0; c < nch; ++c) {
    const int ni = (int)S.I[c].size(), nw = (int)S.sout[c].size();
    std::unordered_map<int, int> lp;
    for (int k = 0; k < ni; ++k) lp[S.I[c][k]] = k;
    for (int i : S.sin[c])
      for (auto& kv : Abb[S.spos[i]]) {
        auto it = lp.find(kv.first);
        if (it == lp.end()) continue;
        const double a = kv.second;
        const double* wr = &W[c][(size_t)it->second * nw];
        for (int j = 0; j < nw; ++j) Sm[(size_t)i * ns + S.sout[c][j]] -= a * wr[j];
      }
  }
  if (ns && !(inv ? (*inv)(Sm, ns) : invert(Sm, ns)))
    throw SetupError(3, "singular interface Schur complement");
  // per-chunk tables and the two stages
  for (int c = 0; c < nch; ++c) {
    ChunkDev& C = B.ch[c];
    const auto& Ic = S.I[c];
    const int ni = (int)Ic.size(), nv = (int)S.sin[c].size(), nw = (int)S.sout[c].size();
    const int nr = (int)S.held[c].size(), nown = (int)S.own[c].size();
    C.p0 = c * S.s;
    C.p1 = std::min(m, (c + 1) * S.s);
    C.ni = ni; C.nv = nv; C.nr = nr; C.nw = nw; C.nown = nown;
    C.ipos_off = (int)B.ipos.size();
    C.v_off = (int)B.vslot.size();
    C.w_off = (int)B.wrow.size();
    C.o_off = (int)B.orow.size();
    for (int k = 0; k < ni; ++k) { B.slot[Ic[k]] = k; B.ipos.push_back(Ic[k]); }
    for (int k = 0; k < nown; ++k) B.slot[S.spos[S.own[c][k]]] = ni + k;
    for (int i : S.sin[c]) B.vslot.push_back(qnext[i]++);
    std::unordered_map<int, int> hidx;
    for (int k = 0; k < nr; ++k) hidx[S.held[c][k]] = k;
    for (int j : S.sout[c]) B.wrow.push_back(hidx[j]);
    for (int i : S.own[c]) { B.orow.push_back(hidx[i]); B.opos.push_back(S.spos[i]); }
    // stage 1: [inv(A_cc); V_c], column-major, ld = ni + nv
    const int ld = ni + nv;
    C.b1 = (long long)B.blob.size();
    C.b1n = round4(ld * ni);
    B.blob.resize(B.blob.size() + C.b1n, 0.0);
    double* s1 = &B.blob[C.b1];
    for (int k = 0; k < ni; ++k) {
      for (int r = 0; r < ni; ++r) s1[(size_t)k * ld + r] = Ainv[c][(size_t)r * ni + k];
      for (int a = 0; a < nv; ++a) s1[(size_t)k * ld + ni + a] = V[c][(size_t)a * ni + k];
    }
    // stage 2: the held rows of inv(S) (row-major, ld = ns), then W_c (column-major, ld = ni)
    C.b2 = (long long)B.blob.size();
    C.b2n = round4(nr * ns + ni * nw);
    B.blob.resize(B.blob.size() + C.b2n, 0.0);
    double* s2 = &B.blob[C.b2];
    for (int r = 0; r < nr; ++r)
      for (int k = 0; k < ns; ++k) s2[(size_t)r * ns + k] = Sm[(size_t)S.held[c][r] * ns + k];
    double* w2 = s2 + (size_t)nr * ns;
    for (int j = 0; j < nw; ++j)
      for (int r = 0; r < ni; ++r) w2[(size_t)j * ni + r] = W[c][(size_t)r * nw + j];
  }
  ChunkSmem L{};
  L.ns4 = round4(ns);
  L.sl4 = round4(B.nslots);
  B.b1max = B.b2max = 0;
  for (const ChunkDev& C : B.ch) {
    L.rows1 = std::max(L.rows1, C.ni + C.nv);
    L.rows2 = std::max(L.rows2, C.nr);
    L.nwmax = std::max(L.nwmax, C.nw);
    L.nimax = std::max(L.nimax, C.ni);
    B.b1max = std::max(B.b1max, C.b1n);
    B.b2max = std::max(B.b2max, C.b2n);
  }
  L.rows1 = round4(L.rows1);
  L.rows2 = round4(L.rows2);
  L.nwmax = round4(L.nwmax);
  L.nimax = round4(L.nimax);
  B.sm = L;
}

// Shared-memory layout of the chunked launches at element size w: the
// stages are staged when the launch's whole layout fits the budget.
ChunkSmem chunk_smem(const BlockPlan& B, int w, int& stage1, int& stage2) {
  ChunkSmem L = B.sm;
  L.st1 = B.b1max;
  stage1 = (size_t)L.p1_total() * w <= (size_t)kSmemBudget;
  if (!stage1) L.st1 = 0;
  L.st2 = B.b2max;
  stage2 = L.p2_bytes(w) <= (size_t)kSmemBudget;
  if (!stage2) L.st2 = 0;
  return L;
}

std::vector<BlockPlan> plan_block_candidates(const LevelDisc& D, int k, const Inverter* inv = nullptr);

BlockPlan plan_block(const LevelDisc& D, const Inverter* inv = nullptr) {
  return std::move(plan_block_candidates(D, 1, inv)[0]);
}

// The exact block of level D as dense or chunked plans: the dense inverse
// for small blocks; else the chunk shapes in the order of the cost model,
// keeping the first k that solve to rounding accuracy (backward error below
// 1e-13 on a fixed vector), or the most accurate one if none does.
std::vector<BlockPlan> plan_block_candidates(const LevelDisc& D, int k, const Inverter* inv) {
  BlockPlan B;
  const int m = (int)D.block.size();
  B.m = m;
  if (m == 0) return std::vector<BlockPlan>(1, B);
  B.cell = D.block;
  std::unordered_map<int, int> pos;
  for (int p = 0; p < m; ++p) pos[D.block[p]] = p;
  std::vector<std::map<int, double>> Abb(m);
  for (int p = 0; p < m; ++p) {
    for (int64_t q = D.block_rows.ptr[p]; q < D.block_rows.ptr[p + 1]; ++q) {
      int c = D.block_rows.col[q];
      double v = D.block_rows.val[q];
      auto it = pos.find(c);
      if (it != pos.end()) Abb[p][it->second] += v;
      else { B.gcol.push_back(c); B.gval.push_back(v); }
    }
    B.gptr.push_back((int64_t)B.gcol.size());
  }
  for (int p = 0; p < m; ++p)
    for (auto& kv : Abb[p])
      if (std::abs(kv.first - p) <= 64) B.band = std::max(B.band, std::abs(kv.first - p));
  make_ell(B);
  if (m <= kDenseMax) {
    // small blocks: the dense inverse of the whole block (Gauss-Jordan)
    std::vector<double> A((size_t)m * m, 0.0);
    for (int p = 0; p < m; ++p)
      for (auto& kv : Abb[p]) A[(size_t)p * m + kv.first] += kv.second;
    if (!(inv ? (*inv)(A, m) : invert(A, m))) throw SetupError(3, "singular block of the smoother");
    B.ainv.swap(A);
    B.dense = true;
    B.error = block_plan_error(B, Abb);
    std::vector<BlockPlan> one;
    one.push_back(std::move(B));
    return one;
  }
  // chunk sizes by the largest per-CTA stage; keep the cheapest whose
  // backward error on a fixed vector is at the level of rounding
  std::vector<ChunkShape> shapes;
  for (int s : {48, 64, 80, 96, 112, 128, 160, 192, 224, 256}) {
    if (s >= m) break;
    ChunkShape S = chunk_shape(Abb, s);
    if (S.ok) shapes.push_back(std::move(S));
  }
  std::sort(shapes.begin(), shapes.end(), [](const ChunkShape& a, const ChunkShape& b) { return a.cost < b.cost; });
  BlockPlan best;
  bool have = false;
  std::vector<BlockPlan> good;
  for (const ChunkShape& S : shapes) {
    BlockPlan P = B;
    try {
      build_chunked(P, Abb, S, inv);
    } catch (SetupError&) {
      continue;
    }
    P.error = block_plan_error(P, Abb);
    if (P.error < 1e-13) {
      good.push_back(std::move(P));
      if ((int)good.size() >= k) break;
      continue;
    }
    if (!have || P.error < best.error) { best = std::move(P); have = true; }
  }
  if (!good.empty()) return good;
  if (!have) throw SetupError(3, "singular block of the smoother");
  std::vector<BlockPlan> one;
  one.push_back(std::move(best));
  return one;
}
// ---------------------------------------------------------------------------
// device memory
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Pool {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  template <class T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) throw CudaError{e};
    ptrs.push_back(p);
    bytes += (int64_t)(n * sizeof(T));
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* d = alloc<T>(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
  ~Pool() { release(); }
};

template <class T>
std::vector<T> cast_vec(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

struct BlockDevSet {
  BlockDev d64, d32;
  ChunkSmem sm64{}, sm32{};   // shared-memory layouts of the chunked launches
};

struct Level {
  int n = 0;
  int64_t nn = 0;
  int sweep_grid = 0;        // CTAs of the streamed FP32 sweep (0: one wave at full occupancy)
  StencilParams sp;          // FP64 stencil data
  StencilP<float> spf;       // the same in FP32
  uint8_t* cls = nullptr;
  double* u64[2] = {nullptr, nullptr};
  double* b64 = nullptr;
  float* u32[2] = {nullptr, nullptr};
  float* b32 = nullptr;
  // host-side plan and discretisation, shared by the clones of a hierarchy
  std::shared_ptr<BlockPlan> planp = std::make_shared<BlockPlan>();
  BlockPlan& plan() { return *planp; }
  const BlockPlan& plan() const { return *planp; }
  BlockDevSet blk;
  // full block rows (FP64) for residuals
  int* brow_cell = nullptr;
  int64_t* brow_ptr = nullptr;
  int* brow_col = nullptr;
  double* brow_val = nullptr;
  // owner fix-up list: merged-away control volumes of this level
  int nfix = 0;
  int* fix_dst = nullptr;
  int* fix_src = nullptr;
  std::shared_ptr<LevelDisc> discp = std::make_shared<LevelDisc>();
  LevelDisc& disc() { return *discp; }
  const LevelDisc& disc() const { return *discp; }
};

}  // namespace

// Scratch of cc_smooth_noalloc: one file-scope device array per device.  Host
// code cannot use the symbol's host-side address; cc_setup looks up the
// device address with the handle's device current and keeps it in the handle
// (clones share it), so a handle made after a device reset holds the address
// in the new context, and the sweep itself makes no lookup.
static __device__ __align__(256) double g_noalloc_scratch[CC_NOALLOC_SCRATCH_DOUBLES];

namespace {
double* noalloc_scratch() {
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  return static_cast<double*>(p);
}
}  // namespace

struct cc_hierarchy {
  Problem P;
  cc_options opt;
  int device = 0;
  std::vector<std::unique_ptr<Level>> lv;
  std::shared_ptr<Pool> pool = std::make_shared<Pool>();   // this handle's device memory
  std::shared_ptr<Pool> tables;   // a clone: the source's memory, which holds the shared tables
  double* bottom_inv = nullptr;   // column-major FP64
  double bottom_error = 0;
  int nc_bottom = 0;
  double* noalloc = nullptr;      // the device's cc_smooth_noalloc scratch (looked up at setup)
  double setup_seconds = 0;       // wall time of the cc_setup that built the tables
  double setup_tables_seconds = 0;  // of which discretize (all levels)
  double setup_kernel_ms = 0;     // device time of its setup kernels
  // finest-level extras
  double* f_rhs = nullptr;        // b of the finest level (FP64)
  double* r64 = nullptr;          // FP64 residual
  double* h_u_dev = nullptr;      // staging for cc_solve_host
  double* h_f_dev = nullptr;
  double* h_g_dev = nullptr;
  int* nrow_cell = nullptr;
  int64_t* nrow_ptr = nullptr;
  int* nrow_col = nullptr;
  double* nrow_val = nullptr;
  int n_nrows = 0;
  unsigned long long* d_norm = nullptr;   // [2]
  unsigned long long* h_norm = nullptr;   // pinned
  cudaEvent_t step_ev = nullptr;          // recorded at the end of every solve step
  int n_g = 0, n_bd = 0;
  int64_t n_dof = 0;
  // kernel timing (cc_kernel_timing): which kernel, its event pairs and the
  // algorithmic bytes of the launch each pair brackets
  int timing = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<double> ev_bytes, ev_rbytes;   // algorithmic and actually moved bytes
  size_t ev_used = 0;
  int64_t timed_launches = 0;
  double timed_ms = 0;
  double timed_bytes = 0, timed_rbytes = 0;
  // level-0 FP64 buffer that holds u during a cycle
  int cur64 = 0;
  // submit/poll worker
  std::mutex qmu;
  std::condition_variable qcv;
  std::deque<uint64_t> queue;
  std::thread worker;
  bool stop = false;
  std::vector<cc_hierarchy*> slots;     // serving clones (slot 0 is the handle itself)
  int64_t slot_bytes = 0;               // device memory of the clones, counted in g_serve_used
  cudaStream_t wstream = nullptr;
  // cuda graphs of one solve iteration
  cudaGraphExec_t gexec[8] = {};             // [timed kernel][mixed]
  int64_t gexec_launches[8] = {};            // kernels in one replay of each graph
  size_t gexec_events[8] = {};               // timing event pairs in each graph
  cudaStream_t gstream = nullptr;
  // Krylov outer iteration (cc_options.krylov = k): basis V [(k + 1) nn],
  // preconditioned vectors Z [k nn], a zero right-hand side, multi-dot
  // partials and results, the least-squares coefficients, and their pinned
  // host copies; the preconditioner cycle's graph and the buffer it ends in
  int kr_k = 0;
  double* kr_u = nullptr;   // the solution and right-hand side of a Krylov solve (the
  double* kr_b = nullptr;   // level-0 u and b buffers are the preconditioner's scratch)
  double* kr_v = nullptr;
  double* kr_z = nullptr;
  double* kr_zero = nullptr;
  double* kr_part = nullptr;
  double* kr_dot = nullptr;
  double* kr_y = nullptr;
  double* kr_dot_host = nullptr;
  double* kr_y_host = nullptr;
  cudaGraphExec_t kr_graph = nullptr;
  int64_t kr_graph_launches = 0;
  int kr_cur = 0;
  // the device-resident solve loop (cc_options.device_loop): one graph whose
  // conditional WHILE node repeats the iteration while the convergence test
  // on the device asks for more; its state and a pinned copy
  cudaGraphExec_t loop_exec = nullptr;
  LoopState* d_loop = nullptr;
  LoopState* h_loop = nullptr;
  int64_t loop_pre_launches = 0;        // kernels before the loop (once per solve)
  int64_t loop_body_launches = 0;       // kernels per loop iteration
  bool loop_failed = false;             // the graph could not be built: host loop
};

namespace {

// ---------------------------------------------------------------------------
// request registry for cc_submit / cc_poll
struct Request {
  cc_hierarchy* h;
  const double* f;
  const double* g;
  double* u;
  double tol;
  cc_result res;
  bool done = false;
};

// the setup cache (cc_options.cache): key of the setup arguments -> a
// hierarchy owned by the cache, which hands out clones of it
std::mutex g_cache_mu;
std::map<std::string, cc_hierarchy*> g_cache;

std::string setup_key(const cc_domain* dom, double a, double b, double c, const cc_bc* bc,
                      int n_bc, int n, const cc_options& o, int device) {
  std::string k;
  auto put = [&](const void* p, size_t len) { k.append(static_cast<const char*>(p), len); };
  put(&device, sizeof(device));
  put(&dom->x0, sizeof(double));
  put(&dom->y0, sizeof(double));
  put(&dom->x1, sizeof(double));
  put(&dom->y1, sizeof(double));
  for (int i = 0; i < dom->n_holes; ++i) {
    const cc_hole& e = dom->holes[i];
    put(&e.kind, sizeof(int));
    put(&e.cx, sizeof(double));
    put(&e.cy, sizeof(double));
    put(&e.r1, sizeof(double));
    put(&e.r2, sizeof(double));
    put(&e.theta, sizeof(double));
  }
  put(&a, sizeof(a));
  put(&b, sizeof(b));
  put(&c, sizeof(c));
  for (int i = 0; i < n_bc; ++i) {
    put(&bc[i].type, sizeof(int));
    put(&bc[i].alpha1, sizeof(double));
    put(&bc[i].alpha2, sizeof(double));
  }
  put(&n, sizeof(n));
  put(&o.eps, sizeof(o.eps));
  put(&o.omega, sizeof(o.omega));
  put(&o.min_coarse_n, sizeof(o.min_coarse_n));
  put(&o.hole_cells, sizeof(o.hole_cells));
  return k;
}

// device memory held by the serving clones of all handles, and its cap
// (cc_serve_budget; 0: no cap)
std::atomic<int64_t> g_serve_used{0};
std::atomic<int64_t> g_serve_budget{0};
std::mutex g_reqmu;
std::unordered_map<uint64_t, Request> g_req;
std::atomic<uint64_t> g_next_id{1};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

cc_status from_setup(int code) {
  switch (code) {
    case 1: return CC_ERR_ARG;
    case 2: return CC_ERR_GEOMETRY;
    case 3: return CC_ERR_SINGULAR;
    default: return CC_ERR_ARG;
  }
}

StencilParams make_stencil(const LevelDisc& D, double omega) {
  StencilParams P;
  std::memset(&P, 0, sizeof(P));
  P.n = D.n;
  P.cross = D.b != 0.0;
  const double lap[5] = {-1, 16, -30, 16, -1}, grad[5] = {1, -8, 0, 8, -1};
  const double h2 = D.h * D.h;
  for (int m = -2; m <= 2; ++m) {
    P.w[2 * 5 + (m + 2)] += D.a * lap[m + 2] / (12.0 * h2);
    P.w[(m + 2) * 5 + 2] += D.c * lap[m + 2] / (12.0 * h2);
  }
  if (P.cross)
    for (int m1 = -2; m1 <= 2; ++m1)
      for (int m2 = -2; m2 <= 2; ++m2)
        if (m1 && m2) P.w[(m2 + 2) * 5 + (m1 + 2)] += D.b * grad[m1 + 2] * grad[m2 + 2] / (144.0 * h2);
  for (int w = 0; w < 4; ++w)
    for (int d = 0; d < 2; ++d)
      for (int q = 0; q < 4; ++q) P.gh[w][d][q] = D.gc[w][d][q];
  P.omega_over_diag = omega / D.diag;
  P.sx = D.a / (12.0 * h2);
  P.sy = D.c / (12.0 * h2);
  P.sxy = D.b / (144.0 * h2);
  return P;
}

// The block's read-only tables at precision T (shared by clones); the work
// vectors are the handle's own (alloc_block_work).
template <class T>
BlockDev upload_block(Pool& pool, const BlockPlan& B, cudaStream_t s) {
  BlockDev d;
  std::memset(&d, 0, sizeof(d));
  d.m = B.m;
  if (B.m == 0) return d;
  d.cell = pool.upload(B.cell, s);
  d.gk = B.gk;
  d.gcol = pool.upload(B.ell_col, s);
  d.gval = pool.upload(cast_vec<T>(B.ell_val), s);
  d.tptr = pool.upload(B.tail_ptr, s);
  d.tcol = pool.upload(B.tail_col, s);
  d.tval = pool.upload(cast_vec<T>(B.tail_val), s);
  d.alias_ptr = pool.upload(B.alias_ptr, s);
  d.alias_cell = pool.upload(B.alias_cell, s);
  d.dense = B.dense ? 1 : 0;
  if (B.dense) {
    // row-major with 16-byte rows, zero padded, for vector loads
    const int w = 16 / (int)sizeof(T);
    d.ld = (B.m + w - 1) / w * w;
    std::vector<T> a((size_t)d.ld * B.m, T(0));
    for (int r = 0; r < B.m; ++r)
      for (int c = 0; c < B.m; ++c) a[(size_t)r * d.ld + c] = (T)B.ainv[(size_t)r * B.m + c];
    d.ainv = pool.upload(a, s);
    return d;
  }
  d.nch = B.nch;
  d.ns = B.ns;
  d.nslots = B.nslots;
  d.ch = pool.upload(B.ch, s);
  d.slot = pool.upload(B.slot, s);
  d.sidx = pool.upload(B.sidx, s);
  d.ipos = pool.upload(B.ipos, s);
  d.vslot = pool.upload(B.vslot, s);
  d.wrow = pool.upload(B.wrow, s);
  d.orow = pool.upload(B.orow, s);
  d.opos = pool.upload(B.opos, s);
  d.qptr = pool.upload(B.qptr, s);
  d.blob = pool.upload(cast_vec<T>(B.blob), s);
  chunk_smem(B, (int)sizeof(T), d.stage1, d.stage2);
  d.rows1 = B.sm.rows1;
  d.rows2 = B.sm.rows2;
  return d;
}

// the handle's work vectors of a chunked block solve, and its fault word
template <class T>
void alloc_block_work(Pool& pool, const BlockPlan& B, BlockDev& d, unsigned int* fault) {
  d.fault = fault;
  if (B.m == 0 || B.dense) return;
  d.tS = pool.alloc<T>(std::max(1, B.ns));
  d.z = pool.alloc<T>(B.m);
  d.q = pool.alloc<T>(std::max(1, B.nslots));
}

inline dim3 tiles(int n) { return dim3((n + TX - 1) / TX, (n + TY - 1) / TY); }
inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// the cycle
template <class T> T* ubuf(Level& L, int i);
template <> double* ubuf<double>(Level& L, int i) { return L.u64[i]; }
template <> float* ubuf<float>(Level& L, int i) { return L.u32[i]; }
template <class T> T* bbuf(Level& L);
template <> double* bbuf<double>(Level& L) { return L.b64; }
template <> float* bbuf<float>(Level& L) { return L.b32; }
template <class T> const BlockDev& bdev(Level& L);
template <> const BlockDev& bdev<double>(Level& L) { return L.blk.d64; }
template <> const BlockDev& bdev<float>(Level& L) { return L.blk.d32; }

template <class T> const StencilP<T>& sparams(Level& L);
template <> const StencilP<double>& sparams<double>(Level& L) { return L.sp; }
template <> const StencilP<float>& sparams<float>(Level& L) { return L.spf; }

// Jacobi sweep on level L: 32 x 32 tiles (4 rows per thread) on large grids,
// 32 x 8 tiles on small ones, where more CTAs matter more than fewer loads.
// CTAs of the streamed sweep: one wave at its occupancy
template <bool CROSS>
int sweep_p_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_p<CROSS>, TX * TY, 0);
    return std::max(1, sms) * std::max(1, occ);
  }();
  return blocks;
}

template <class T>
void launch_sweep(Level& L, const T* in, T* out, const T* b, const T* ec, bool zero,
                  cudaStream_t s) {
  const auto& P = sparams<T>(L);
  if constexpr (std::is_same<T, float>::value) {
    if (L.n >= 256 && L.n % 32 == 0) {
      const int nt = (L.n / TX) * (L.n / WY);
      const int g = L.sweep_grid > 0 ? L.sweep_grid
                                     : std::min(nt, L.sp.cross ? sweep_p_blocks<true>() : sweep_p_blocks<false>());
      if (L.sp.cross)
        pdl_launch(k_sweep_p<true>, g, TX * TY, 0, s, in, out, b, L.cls, ec, P, (int)zero);
      else
        pdl_launch(k_sweep_p<false>, g, TX * TY, 0, s, in, out, b, L.cls, ec, P, (int)zero);
      return;
    }
  }
  if (L.n >= 256) {
    dim3 g((L.n + TX - 1) / TX, (L.n + WY - 1) / WY);
    if (L.sp.cross) pdl_launch(k_sweep_w<T, true>, g, TX * TY, 0, s, in, out, b, L.cls, ec, P, zero);
    else pdl_launch(k_sweep_w<T, false>, g, TX * TY, 0, s, in, out, b, L.cls, ec, P, zero);
  } else {
    if (L.sp.cross) pdl_launch(k_sweep<T, true, 1>, tiles(L.n), TX * TY, 0, s, in, out, b, L.cls, ec, P, zero);
    else pdl_launch(k_sweep<T, false, 1>, tiles(L.n), TX * TY, 0, s, in, out, b, L.cls, ec, P, zero);
  }
}

// event pair around one timed launch (the pairs are created up front by
// cc_kernel_timing, so none is created while a graph is being captured)
bool time_begin(cc_hierarchy* H, cudaStream_t s) {
  if (H->ev_used >= H->ev.size()) return false;
  CK(cudaEventRecordWithFlags(H->ev[H->ev_used].first, s, cudaEventRecordExternal));
  return true;
}
void time_end(cc_hierarchy* H, cudaStream_t s, double bytes, double rbytes) {
  CK(cudaEventRecordWithFlags(H->ev[H->ev_used].second, s, cudaEventRecordExternal));
  H->ev_bytes[H->ev_used] = bytes;
  H->ev_rbytes[H->ev_used] = rbytes;
  ++H->ev_used;
}

// Algorithmic bytes of one exact block solve as the method prices it
// (Eq. 5.8 with the factors of Def. 5.3): the gather terms (column,
// coefficient, gathered value), b and the cell of every row, the banded LU
// factors (2 band + 1 per row) and the write of every row.
double block_method_bytes(const BlockPlan& P, int w) {
  const double m = P.m, nnz = (double)P.gptr[P.m];
  return nnz * (4 + 2 * w) + m * (4 + w) + m * (2.0 * P.band + 1) * w + m * w;
}

// Bytes the library's form of the solve reads and writes: the gather as
// above, the dense inverse or the two stages of every chunk, the interface
// vectors (written once, read by every chunk) and the writes.
double block_read_bytes(const BlockPlan& P, int w) {
  const double m = P.m, nnz = (double)P.gptr[P.m], na = (double)P.alias_cell.size();
  double b = nnz * (4 + 2 * w) + m * (4 + w) + (m + na) * w;
  if (P.dense) return b + m * m * w;
  b += (double)P.blob.size() * w;
  b += (double)P.nch * (P.ns + P.nslots) * w + 2.0 * (P.ns + m + P.nslots) * w;
  return b;
}

// The chunked launches may use up to kSmemBudget bytes of dynamic shared
// memory (the attribute is per function; set once per device)
void chunk_smem_attributes() {
  CK(cudaFuncSetAttribute(k_block_p1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
  CK(cudaFuncSetAttribute(k_block_p2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
  CK(cudaFuncSetAttribute(k_block_p1<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
  CK(cudaFuncSetAttribute(k_block_p2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
}

template <class T> const ChunkSmem& csmem(Level& L);
template <> const ChunkSmem& csmem<double>(Level& L) { return L.blk.sm64; }
template <> const ChunkSmem& csmem<float>(Level& L) { return L.blk.sm32; }

// one exact block solve (Eq. 5.8) of level L on the stencil-swept u, with the
// block's tables B (the handle's, or the same with other work vectors)
template <class T>
void launch_block(const BlockPlan& P, const BlockDev& B, const ChunkSmem& sm, T* u, const T* b,
                  cudaStream_t s) {
  if (P.dense) {
    // 1024-thread CTAs: every thread gathers at most one row, every warp
    // applies one row of the inverse
    pdl_launch(k_block_dense<T>, (unsigned)((P.m + 31) / 32), 1024, (size_t)B.ld * sizeof(T), s, B, b, u);
    return;
  }
  pdl_launch(k_block_p1<T>, P.nch, kChunkThreads, (size_t)sm.p1_total() * sizeof(T), s, B, sm, b,
             (const T*)u);
  pdl_launch(k_block_p2<T>, P.nch, kChunkThreads, sm.p2_bytes((int)sizeof(T)), s, B, sm, u);
}

template <class T>
void block_solve(cc_hierarchy* H, Level& L, T* u, const T* b, cudaStream_t s) {
  const BlockPlan& P = L.plan();
  if (P.m == 0) return;
  const bool timed = (H->timing == CC_TIME_BLOCK || (H->timing == CC_TIME_FINE_BLOCK && &L == H->lv[0].get())) &&
                     time_begin(H, s);
  launch_block<T>(P, bdev<T>(L), csmem<T>(L), u, b, s);
  if (timed) time_end(H, s, block_method_bytes(P, (int)sizeof(T)), block_read_bytes(P, (int)sizeof(T)));
}

// the multicolour variant's sweep, in place on u: the initial guess (0, or u
// plus the interpolated coarse correction), the colour classes in order, then
// the exact block solve
template <class T>
void color_passes(Level& L, T* u, const T* b, cudaStream_t s) {
  const bool cross = L.sp.cross != 0;
  for (int c = 0; c < mc_colors(cross); ++c) {
    if (cross) pdl_launch(k_sweep_color<T, true>, tiles(L.n), TX * TY, 0, s, u, b, (const uint8_t*)L.cls, sparams<T>(L), c);
    else pdl_launch(k_sweep_color<T, false>, tiles(L.n), TX * TY, 0, s, u, b, (const uint8_t*)L.cls, sparams<T>(L), c);
  }
}

template <class T>
void sweep_mc(cc_hierarchy* H, Level& L, T* u, bool zero, const T* ec, cudaStream_t s) {
  if (zero) CK(cudaMemsetAsync(u, 0, L.nn * sizeof(T), s));
  if (ec) pdl_launch(k_prolong_add<T>, nblk(L.nn), 256, 0, s, u, ec, L.cls, L.n);
  color_passes<T>(L, u, (const T*)bbuf<T>(L), s);
  block_solve<T>(H, L, u, bbuf<T>(L), s);
}

template <class T>
void sweep(cc_hierarchy* H, int l, int& cur, bool zero, const T* ec, cudaStream_t s) {
  Level& L = *H->lv[l];
  if (H->opt.smoother == CC_SMOOTHER_MCGS) {
    sweep_mc<T>(H, L, ubuf<T>(L, cur), zero, ec, s);
    return;
  }
  T* in = ubuf<T>(L, cur);
  T* out = ubuf<T>(L, 1 - cur);
  const bool timed = H->timing == CC_TIME_FINE_SWEEP && l == 0 && time_begin(H, s);
  launch_sweep<T>(L, in, out, bbuf<T>(L), ec, zero, s);
  if (timed) time_end(H, s, 3.0 * sizeof(T) * (double)L.nn, 3.0 * sizeof(T) * (double)L.nn);
  block_solve<T>(H, L, out, bbuf<T>(L), s);
  cur = 1 - cur;
}

template <class T>
void bottom(cc_hierarchy* H, int l, int cur, cudaStream_t s) {
  Level& L = *H->lv[l];
  int nc = H->nc_bottom;
  pdl_launch(k_bottom<T>, (nc + 7) / 8, 256, 0, s, H->bottom_inv, nc, bbuf<T>(L), ubuf<T>(L, cur));
}

// Alg. 2 (gamma = 1) or its W form (gamma = 2) on level l; cur[l] tracks the
// buffer that holds u.
// With pre, the stencil cells of the first pre-sweep from the zero initial
// guess were written by the kernel that made this level's right-hand side
// (the restriction, or the FP64 residual of the refinement loop); only its
// block solve is left.
// Visits of level l + 1 from level l: gamma = 1 (V) or 2 (W) of Alg. 2, W
// only on the w_depth finest levels when w_depth > 0; Alg. 3 runs the cycle
// that fmg_cycle names.  A second visit of the bottom level would repeat the
// same exact solve on the same right-hand side, so it is left out.
int cycle_gamma(const cc_hierarchy* H, int l) {
  const cc_options& o = H->opt;
  const int c = o.cycle == CC_CYCLE_FMG ? o.fmg_cycle : o.cycle;
  if (c != CC_CYCLE_W) return 1;
  if (o.w_depth > 0 && l >= o.w_depth) return 1;
  if (l + 2 == (int)H->lv.size()) return 1;
  return 2;
}

// With ec0, the initial guess is u + I(ec0) (0 + I(ec0) with zero), the
// interpolated coarse solution of Alg. 3; the interpolation is fused into the
// first pre-sweep.
template <class T>
void cycle_level(cc_hierarchy* H, int l, std::vector<int>& cur, bool zero, cudaStream_t s,
                 bool pre = false, const T* ec0 = nullptr) {
  const int nl = (int)H->lv.size();
  Level& L = *H->lv[l];
  if (l == nl - 1) {
    bottom<T>(H, l, cur[l], s);
    return;
  }
  const int nu1 = H->opt.nu1, nu2 = H->opt.nu2;
  const int gamma = cycle_gamma(H, l);
  bool z = zero;
  for (int k = 0; k < nu1; ++k) {
    if (k == 0 && pre) {
      block_solve<T>(H, L, ubuf<T>(L, 1 - cur[l]), bbuf<T>(L), s);
      cur[l] = 1 - cur[l];
    } else {
      sweep<T>(H, l, cur[l], z, k == 0 ? ec0 : (const T*)nullptr, s);
    }
    z = false;
  }
  if (z) {   // nu1 == 0 on a zero initial guess: materialise u = 0
    CK(cudaMemsetAsync(ubuf<T>(L, cur[l]), 0, L.nn * sizeof(T), s));
  }
  if (nu1 == 0 && ec0)
    pdl_launch(k_prolong_add<T>, nblk(L.nn), 256, 0, s, ubuf<T>(L, cur[l]), ec0, L.cls, L.n);
  Level& C = *H->lv[l + 1];
  // the coarse level's first visit starts from zero: its first sweep is
  // written by the restriction kernel (not on the bottom level, which has none)
  const bool fuse_c = l + 1 < nl - 1 && nu1 > 0 && H->opt.smoother == CC_SMOOTHER_JACOBI;
  T* uc = fuse_c ? ubuf<T>(C, 1 - cur[l + 1]) : nullptr;
  const T wd_c = sparams<T>(C).omega_over_diag;
  if (L.sp.cross)
    pdl_launch(k_resid_restrict<T, true>, tiles(L.n), TX * TY, 0, s, ubuf<T>(L, cur[l]), bbuf<T>(L), L.cls,
               C.cls, bbuf<T>(C), sparams<T>(L), uc, wd_c);
  else
    pdl_launch(k_resid_restrict<T, false>, tiles(L.n), TX * TY, 0, s, ubuf<T>(L, cur[l]), bbuf<T>(L), L.cls,
               C.cls, bbuf<T>(C), sparams<T>(L), uc, wd_c);
  for (int g = 0; g < gamma; ++g) cycle_level<T>(H, l + 1, cur, g == 0, s, g == 0 && fuse_c);
  // merged-away coarse cells already hold their owner's value (written by
  // the block solve, or by the alias rows of the bottom matrix)
  T* ec = ubuf<T>(C, cur[l + 1]);
  if (nu2 == 0) {
    pdl_launch(k_prolong_add<T>, nblk(L.nn), 256, 0, s, ubuf<T>(L, cur[l]), ec, L.cls, L.n);
    return;
  }
  for (int k = 0; k < nu2; ++k) sweep<T>(H, l, cur[l], false, k == 0 ? ec : (const T*)nullptr, s);
}

// b of level l + 1 = restriction of r (a right-hand side of level l, Alg. 3)
template <class Tin, class Tout>
void restrict_rhs(cc_hierarchy* H, int l, const Tin* r, cudaStream_t s) {
  Level& L = *H->lv[l];
  Level& C = *H->lv[l + 1];
  pdl_launch(k_restrict_rhs<Tin, Tout>, nblk(C.nn), 256, 0, s, r, L.cls, C.cls, bbuf<Tout>(C), L.n);
}

// the solution buffer of level 1
template <class T>
T* L1u(cc_hierarchy* H, const std::vector<int>& cur) { return ubuf<T>(*H->lv[1], cur[1]); }

// FP64 residual r = b - A u on the finest level, max |r| into d_norm[0]; with
// e0, also the stencil-cell part of the first sweep of the next cycle on
// A e = r from e = 0 (wd = omega / D in Tout)
template <class Tout>
void residual64(cc_hierarchy* H, const double* u, const double* b, Tout* r, cudaStream_t s,
                Tout* e0 = nullptr, Tout wd = Tout(0)) {
  Level& L = *H->lv[0];
  if (L.sp.cross)
    pdl_launch(k_resid_fx<Tout, true>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, r, L.sp, H->d_norm, e0, wd);
  else
    pdl_launch(k_resid_fx<Tout, false>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, r, L.sp, H->d_norm, e0, wd);
  if (L.plan().m)
    pdl_launch(k_block_resid<Tout>, nblk(L.plan().m), 256, 0, s, L.plan().m, L.brow_cell, L.brow_ptr, L.brow_col,
                                                       L.brow_val, u, b, r, H->d_norm);
}

void assemble_rhs(cc_hierarchy* H, const double* f, const double* g, double* b, cudaStream_t s) {
  Level& L = *H->lv[0];
  pdl_launch(k_rhs_copy, nblk(L.nn), 256, 0, s, f, L.cls, b, L.nn);
  if (H->n_nrows)
    pdl_launch(k_rhs_n, nblk(H->n_nrows), 256, 0, s, H->n_nrows, H->nrow_cell, H->nrow_ptr, H->nrow_col,
                                             H->nrow_val, g, b);
}

double read_norm(cc_hierarchy* H, cudaStream_t s) {
  CK(cudaMemcpyAsync(H->h_norm, H->d_norm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  unsigned long long v = H->h_norm[0];
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

// Alg. 3 below level l0, whose right-hand side is in place: restrict it down
// to the coarsest level, solve there, and climb back with one cycle per level
// from the interpolated coarse solution.  The solution of level l0 + 1 is
// left in its buffer cur[l0 + 1].
template <class T>
void fmg_below(cc_hierarchy* H, int l0, std::vector<int>& cur, cudaStream_t s) {
  const int nl = (int)H->lv.size();
  for (int l = l0 + 1; l + 1 < nl; ++l) restrict_rhs<T, T>(H, l, bbuf<T>(*H->lv[l]), s);
  bottom<T>(H, nl - 1, cur[nl - 1], s);
  for (int l = nl - 2; l > l0; --l)
    cycle_level<T>(H, l, cur, true, s, false, (const T*)ubuf<T>(*H->lv[l + 1], cur[l + 1]));
}

// Mixed mode: the FP64 residual kernel also writes the stencil cells of the
// next FP32 cycle's first sweep (into u32[1], its output buffer; the cycle
// starts in buffer 0) when that cycle has a pre-sweep on the finest level
// from a zero initial guess (not in Alg. 3, which starts it from I(e)).
bool mixed_pre(cc_hierarchy* H) {
  return H->opt.nu1 > 0 && H->lv.size() > 1 && H->opt.cycle != CC_CYCLE_FMG &&
         H->opt.smoother == CC_SMOOTHER_JACOBI;
}
float* mixed_e0(cc_hierarchy* H) { return mixed_pre(H) ? H->lv[0]->u32[1] : nullptr; }

// one iteration of the solve loop, recorded for graph capture or launched
// directly: FP64 mode: cycle on (u, b) then r = b - A u; mixed mode:
// r = b - A u (FP64, written as the FP32 cycle right-hand side), FP32 cycle
// from 0, u += e.
void iteration(cc_hierarchy* H, bool mixed, cudaStream_t s) {
  Level& L = *H->lv[0];
  std::vector<int> cur(H->lv.size(), 0);
  CK(cudaMemsetAsync(H->d_norm, 0, sizeof(unsigned long long), s));
  const bool fmg = H->opt.cycle == CC_CYCLE_FMG && H->lv.size() > 1;
  if (!mixed) {
    cur[0] = H->cur64;
    if (fmg) {
      // u + FMG(r): the finest-level cycle of Alg. 3 on the residual
      // equation from I(e_1) equals the same cycle on A u = b from
      // u + I(e_1) (the cycle is affine with error propagator I - N A)
      restrict_rhs<double, double>(H, 0, H->r64, s);
      fmg_below<double>(H, 0, cur, s);
      cycle_level<double>(H, 0, cur, false, s, false, (const double*)L1u<double>(H, cur));
    } else {
      cycle_level<double>(H, 0, cur, false, s);
    }
    if (cur[0] != H->cur64)
      CK(cudaMemcpyAsync(L.u64[H->cur64], L.u64[cur[0]], L.nn * sizeof(double),
                         cudaMemcpyDeviceToDevice, s));
    residual64<double>(H, L.u64[H->cur64], L.b64, H->r64, s);
  } else {
    if (fmg) {
      restrict_rhs<float, float>(H, 0, L.b32, s);
      fmg_below<float>(H, 0, cur, s);
      cycle_level<float>(H, 0, cur, true, s, false, (const float*)L1u<float>(H, cur));
    } else {
      cycle_level<float>(H, 0, cur, true, s, mixed_pre(H));
    }
    pdl_launch(k_update<float>, nblk(L.nn), 256, 0, s, L.u64[H->cur64], L.u32[cur[0]], L.cls, L.nn);
    residual64<float>(H, L.u64[H->cur64], L.b64, L.b32, s, mixed_e0(H), L.spf.omega_over_diag);
  }
}

// ---- Krylov outer iteration (cc_options.krylov) -------------------------------
// Restarted flexible GMRES (right preconditioning) on A u = b in FP64; the
// preconditioner is one FP32 cycle from zero on the vector as right-hand
// side.  The Arnoldi vectors are orthogonalised by classical Gram-Schmidt run
// twice; the small least-squares problem is solved on the host with Givens
// rotations.  Not part of the paper's solver: an option for domains where the
// cycle alone diverges.

// buffers of the handle's Krylov iteration (restart length opt.krylov)
void ensure_krylov(cc_hierarchy* H, cudaStream_t s) {
  const int k = H->opt.krylov;
  if (k <= H->kr_k || H->opt.host_only) return;
  const int64_t nn = H->lv[0]->nn;
  if (!H->kr_u) {
    H->kr_u = H->pool->alloc<double>(nn);
    H->kr_b = H->pool->alloc<double>(nn);
  }
  H->kr_v = H->pool->alloc<double>((size_t)(k + 1) * nn);
  H->kr_z = H->pool->alloc<double>((size_t)k * nn);
  H->kr_zero = H->pool->alloc<double>(nn);
  CK(cudaMemsetAsync(H->kr_zero, 0, nn * sizeof(double), s));
  H->kr_part = H->pool->alloc<double>((size_t)KR_BLOCKS * KR_MAXV);
  H->kr_dot = H->pool->alloc<double>(KR_MAXV);
  H->kr_y = H->pool->alloc<double>(KR_MAXV);
  if (H->kr_dot_host) cudaFreeHost(H->kr_dot_host);
  if (H->kr_y_host) cudaFreeHost(H->kr_y_host);
  H->kr_dot_host = nullptr;
  H->kr_y_host = nullptr;
  CK(cudaMallocHost(&H->kr_dot_host, KR_MAXV * sizeof(double)));
  CK(cudaMallocHost(&H->kr_y_host, KR_MAXV * sizeof(double)));
  H->kr_k = k;
}

double* kr_vec(cc_hierarchy* H, int i) { return H->kr_v + (size_t)i * H->lv[0]->nn; }
double* kr_zvec(cc_hierarchy* H, int i) { return H->kr_z + (size_t)i * H->lv[0]->nn; }

// out[0..nx) = <w, V_i> (and out[nx] = <w, w> when self) into kr_dot, then
// its pinned host copy; the caller records the step event after it
void kr_dots(cc_hierarchy* H, int nx, const double* w, int self, cudaStream_t s) {
  const int64_t nn = H->lv[0]->nn;
  const int nv = nx + self;
  pdl_launch(k_mdot, KR_BLOCKS, 256, 0, s, (const double*)H->kr_v, nx, w, self, nn, H->kr_part);
  pdl_launch(k_mdot_sum, nv, 32, 0, s, (const double*)H->kr_part, nv, KR_BLOCKS, H->kr_dot);
  CK(cudaMemcpyAsync(H->kr_dot_host, H->kr_dot, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
}

// the preconditioner's cycle from zero, in the handle's precision, on the
// level-0 right-hand side buffer (b32 or b64); leaves e in u32 / u64[kr_cur]
void kr_cycle(cc_hierarchy* H, cudaStream_t s) {
  std::vector<int> cur(H->lv.size(), 0);
  if (H->opt.precision == CC_PREC_MIXED) cycle_level<float>(H, 0, cur, true, s, false);
  else cycle_level<double>(H, 0, cur, true, s, false);
  H->kr_cur = cur[0];
}

// z = M^-1 v: v into the cycle's right-hand side (narrowed to FP32 in the
// mixed mode), one cycle, e widened and zeroed on empty control volumes
void kr_precond(cc_hierarchy* H, const double* v, double* z, cudaStream_t s) {
  Level& L = *H->lv[0];
  const bool mixed = H->opt.precision == CC_PREC_MIXED;
  if (mixed) pdl_launch(k_convert<double, float>, nblk(L.nn), 256, 0, s, v, L.b32, L.nn);
  else CK(cudaMemcpyAsync(L.b64, v, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (H->opt.use_graphs) {
    if (!H->kr_graph) {
      cudaGraph_t gr;
      int64_t before = t_launches;
      CK(cudaStreamBeginCapture(H->gstream, cudaStreamCaptureModeThreadLocal));
      kr_cycle(H, H->gstream);
      CK(cudaStreamEndCapture(H->gstream, &gr));
      CK(cudaGraphInstantiate(&H->kr_graph, gr, 0));
      CK(cudaGraphDestroy(gr));
      H->kr_graph_launches = t_launches - before;
      t_launches = before;
    }
    CK(cudaGraphLaunch(H->kr_graph, s));
    t_launches += H->kr_graph_launches;
  } else {
    kr_cycle(H, s);
  }
  if (mixed)
    pdl_launch(k_widen_masked<float>, nblk(L.nn), 256, 0, s, (const float*)L.u32[H->kr_cur],
               (const uint8_t*)L.cls, z, L.nn);
  else
    pdl_launch(k_widen_masked<double>, nblk(L.nn), 256, 0, s, (const double*)L.u64[H->kr_cur],
               (const uint8_t*)L.cls, z, L.nn);
}

// One solve as a sequence of steps that never wait on the GPU: every step
// enqueues its work and the copy of one norm to pinned memory, then records
// the handle's step event; the next step runs once that event has completed.
// A host thread can so drive several solves (on distinct handles) at once.
struct SolveTask {
  cc_hierarchy* H = nullptr;
  const double* f = nullptr;
  const double* g = nullptr;
  double* u = nullptr;
  double tol = 0;
  cudaStream_t s = nullptr;
  bool device_loop = false;   // may run its iterations in the handle's loop graph
  int phase = 0;   // 0 start, 1 |b| pending, 2 first residual pending, 3 cycle pending,
                   // 4 result copy pending, 5 done
  double bn = 1, rel = 0, first = -1;
  int it = 0;
  int64_t launches = 0;
  cc_result res{};
  // Krylov state: column j of the Hessenberg matrix being built, the
  // restart's initial residual norm, the rotated least-squares system
  int kj = 0;
  double kbeta = 0;
  std::vector<double> kH, kcs, ksn, kg, kh1;
};

void enqueue_norm(cc_hierarchy* H, cudaStream_t s) {
  CK(cudaMemcpyAsync(H->h_norm, H->d_norm, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(H->step_ev, s));
}

double host_norm(const cc_hierarchy* H) {
  unsigned long long v = H->h_norm[0];
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

// one solve iteration (a cycle, the FP64 residual and its norm), replayed
// from the handle's graph when graphs are on
void launch_iteration(cc_hierarchy* H, bool mixed, cudaStream_t s) {
  const int gi = (mixed ? 1 : 0) + 2 * H->timing;
  if (H->opt.use_graphs) {
    if (!H->gexec[gi]) {
      cudaGraph_t gr;
      int64_t before = t_launches;
      H->ev_used = 0;
      CK(cudaStreamBeginCapture(H->gstream, cudaStreamCaptureModeThreadLocal));
      iteration(H, mixed, H->gstream);
      CK(cudaStreamEndCapture(H->gstream, &gr));
      CK(cudaGraphInstantiate(&H->gexec[gi], gr, 0));
      CK(cudaGraphDestroy(gr));
      H->gexec_launches[gi] = t_launches - before;
      H->gexec_events[gi] = H->ev_used;
      t_launches = before;
    }
    CK(cudaGraphLaunch(H->gexec[gi], s));
    t_launches += H->gexec_launches[gi];
  } else {
    H->ev_used = 0;
    iteration(H, mixed, s);
  }
  enqueue_norm(H, s);
}

// durations of the timed launches of the iteration just completed
void collect_timing(cc_hierarchy* H, bool mixed) {
  if (!H->timing) return;
  const int gi = (mixed ? 1 : 0) + 2 * H->timing;
  size_t ne = H->opt.use_graphs ? H->gexec_events[gi] : H->ev_used;
  for (size_t i = 0; i < ne; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, H->ev[i].first, H->ev[i].second));
    H->timed_ms += ms;
    H->timed_bytes += H->ev_bytes[i];
    H->timed_rbytes += H->ev_rbytes[i];
    ++H->timed_launches;
  }
  if (!H->opt.use_graphs) H->ev_used = 0;
}

// Build the handle's solve-loop graph: the |b| read-out, the residual of the
// initial guess and its test, then a WHILE node whose body is one iteration
// (the same captured launches as the host loop's graph) and its test.  False
// (and the host loop from then on) where the graph cannot be built.
bool ensure_loop(cc_hierarchy* H, bool mixed) {
  if (H->loop_exec) return true;
  if (H->loop_failed) return false;
  Level& L = *H->lv[0];
  if (!H->d_loop) H->d_loop = H->pool->alloc<LoopState>(1);
  if (!H->h_loop) CK(cudaMallocHost(&H->h_loop, sizeof(LoopState)));
  const cudaStream_t gs = H->gstream;
  const int64_t before = t_launches;
  cudaGraph_t G = nullptr;
  try {
    CK(cudaGraphCreate(&G, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, G, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(gs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    pdl_launch(k_loop_step, 1, 1, 0, gs, H->d_loop, (const unsigned long long*)H->d_norm, 0, cond);
    CK(cudaMemsetAsync(H->d_norm, 0, sizeof(unsigned long long), gs));
    if (mixed) residual64<float>(H, L.u64[0], L.b64, L.b32, gs, mixed_e0(H), L.spf.omega_over_diag);
    else residual64<double>(H, L.u64[0], L.b64, H->r64, gs);
    pdl_launch(k_loop_step, 1, 1, 0, gs, H->d_loop, (const unsigned long long*)H->d_norm, 1, cond);
    H->loop_pre_launches = t_launches - before;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(gs, &cs, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(gs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamEndCapture(gs, &G));
    const int64_t b0 = t_launches;
    CK(cudaStreamBeginCaptureToGraph(gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    H->ev_used = 0;
    iteration(H, mixed, gs);
    pdl_launch(k_loop_step, 1, 1, 0, gs, H->d_loop, (const unsigned long long*)H->d_norm, 2, cond);
    CK(cudaStreamEndCapture(gs, &body));
    H->loop_body_launches = t_launches - b0;
    CK(cudaGraphInstantiate(&H->loop_exec, G, 0));
    CK(cudaGraphDestroy(G));
  } catch (CudaError&) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(gs, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(gs, &junk);
      if (junk && junk != G) cudaGraphDestroy(junk);
    }
    if (G) cudaGraphDestroy(G);
    cudaGetLastError();
    H->loop_exec = nullptr;
    H->loop_failed = true;
  }
  t_launches = before;
  return H->loop_exec != nullptr;
}

bool use_device_loop(const cc_hierarchy* H) {
  return H->opt.device_loop && H->opt.use_graphs && !H->opt.krylov && !H->timing &&
         H->opt.max_cycles > 0;
}

void finish_task(SolveTask& T) {
  Level& L = *T.H->lv[0];
  const double* sol = T.H->opt.krylov ? T.H->kr_u : L.u64[T.H->cur64];
  CK(cudaMemcpyAsync(T.u, sol, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, T.s));
  CK(cudaEventRecord(T.H->step_ev, T.s));
  T.phase = 4;
}

// Krylov: start a restart; the residual is in V_0, its squared 2-norm goes
// to the host
void kr_restart(SolveTask& T) {
  kr_dots(T.H, 0, kr_vec(T.H, 0), 1, T.s);
  CK(cudaEventRecord(T.H->step_ev, T.s));
  T.phase = 10;
}

// Krylov: first half of Arnoldi step j: Z_j = M^-1 V_j, V_{j+1} = -A Z_j (the
// FP64 residual of Z_j against a zero right-hand side), and the projections
// of V_{j+1} on V_0..V_j to the host
void kr_arnoldi(SolveTask& T) {
  cc_hierarchy* H = T.H;
  const int j = T.kj;
  kr_precond(H, kr_vec(H, j), kr_zvec(H, j), T.s);
  residual64<double>(H, kr_zvec(H, j), H->kr_zero, kr_vec(H, j + 1), T.s);
  kr_dots(H, j + 1, kr_vec(H, j + 1), 0, T.s);
  CK(cudaEventRecord(H->step_ev, T.s));
  T.phase = 11;
}

// Krylov: end of a restart after m Arnoldi steps.  The Hessenberg matrix is
// that of the operator -A M^-1, so with y solving the rotated triangular
// system the update is u -= Z y; then the true FP64 residual goes to V_0 and
// its max-norm to the host.
void kr_end_restart(SolveTask& T, int m) {
  cc_hierarchy* H = T.H;
  Level& L = *H->lv[0];
  const int k = H->opt.krylov;
  std::vector<double> y(m, 0.0);
  for (int i = m - 1; i >= 0; --i) {
    double v = T.kg[i];
    for (int q = i + 1; q < m; ++q) v -= T.kH[(size_t)q * (k + 1) + i] * y[q];
    const double d = T.kH[(size_t)i * (k + 1) + i];
    y[i] = d != 0.0 ? v / d : 0.0;
  }
  for (int i = 0; i < m; ++i) H->kr_y_host[i] = y[i];
  CK(cudaMemcpyAsync(H->kr_y, H->kr_y_host, m * sizeof(double), cudaMemcpyHostToDevice, T.s));
  pdl_launch(k_maxpy, KR_BLOCKS, 256, 0, T.s, (const double*)H->kr_z, m, (const double*)H->kr_y, H->kr_u,
             1.0, L.nn);
  CK(cudaMemsetAsync(H->d_norm, 0, sizeof(unsigned long long), T.s));
  residual64<double>(H, H->kr_u, H->kr_b, kr_vec(H, 0), T.s);
  enqueue_norm(H, T.s);
  T.phase = 13;
}

// Advance T by one step (its previous step has completed on the GPU); true
// once the solve is done and its result copied out.
bool solve_step(SolveTask& T) {
  cc_hierarchy* H = T.H;
  Level& L = *H->lv[0];
  const bool mixed = H->opt.precision == CC_PREC_MIXED;
  const cudaStream_t s = T.s;
  const int64_t l0 = t_launches;
  // a bounded wait that expired in a kernel ends the solve
  if ((T.phase == 1 || T.phase == 2 || T.phase == 3 || T.phase == 13) && H->h_norm[1] != 0) {
    T.res.status = CC_ERR_TIMEOUT;
    finish_task(T);
    T.launches += t_launches - l0;
    T.res.kernels = T.launches;
    return false;
  }
  switch (T.phase) {
    case 0: {
      H->cur64 = 0;
      T.res.status = CC_ERR_NOT_CONVERGED;
      H->h_norm[1] = 0;
      const bool dloop = T.device_loop && use_device_loop(H) && ensure_loop(H, mixed);
      CK(cudaMemsetAsync(H->d_norm + 1, 0, sizeof(unsigned long long), s));
      if (H->opt.krylov) ensure_krylov(H, s);
      {
        double* b0 = H->opt.krylov ? H->kr_b : L.b64;
        double* u0 = H->opt.krylov ? H->kr_u : L.u64[0];
        assemble_rhs(H, T.f, T.g, b0, s);
        CK(cudaMemcpyAsync(u0, T.u, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(H->d_norm, 0, sizeof(unsigned long long), s));
        pdl_launch(k_absmax, 152 * 4, 256, 0, s, (const double*)b0, L.nn, H->d_norm);
      }
      if (dloop) {
        // the whole iteration on the device: one graph launch, then the
        // solution and the loop's state come back once
        pdl_launch(k_loop_init, 1, 1, 0, s, H->d_loop, T.tol, H->opt.max_cycles);
        CK(cudaGraphLaunch(H->loop_exec, s));
        t_launches += H->loop_pre_launches;
        CK(cudaMemcpyAsync(T.u, L.u64[H->cur64], L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(H->h_loop, H->d_loop, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(H->step_ev, s));
        T.phase = 20;
        break;
      }
      enqueue_norm(H, s);
      T.phase = 1;
      break;
    }
    case 20:   // the device loop has finished
      T.it = H->h_loop->it;
      T.rel = H->h_loop->rel;
      T.res.status = (cc_status)H->h_loop->status;
      T.res.cycles = T.it;
      T.res.rel_res = T.rel;
      t_launches += T.it * H->loop_body_launches;
      T.phase = 5;
      break;
    case 1:
      // residual of the initial guess (in the mixed mode it is also the first
      // FP32 right-hand side)
      T.bn = host_norm(H);
      if (T.bn == 0.0) T.bn = 1.0;
      CK(cudaMemsetAsync(H->d_norm, 0, sizeof(unsigned long long), s));
      if (H->opt.krylov) residual64<double>(H, H->kr_u, H->kr_b, kr_vec(H, 0), s);
      else if (mixed) residual64<float>(H, L.u64[0], L.b64, L.b32, s, mixed_e0(H), L.spf.omega_over_diag);
      else residual64<double>(H, L.u64[0], L.b64, H->r64, s);
      enqueue_norm(H, s);
      T.phase = 2;
      break;
    case 2:
      T.rel = T.first = host_norm(H) / T.bn;
      if (T.rel < T.tol) {
        T.res.status = CC_OK;
        finish_task(T);
      } else if (H->opt.max_cycles <= 0) {
        finish_task(T);
      } else if (H->opt.krylov) {
        kr_restart(T);
      } else {
        launch_iteration(H, mixed, s);
        T.phase = 3;
      }
      break;
    case 3:
      T.rel = host_norm(H) / T.bn;
      collect_timing(H, mixed);
      ++T.it;
      if (T.rel < T.tol) {
        T.res.status = CC_OK;
        finish_task(T);
      } else if (!std::isfinite(T.rel) || (T.first > 0 && T.rel > 1e3 * T.first)) {
        T.res.status = CC_ERR_DIVERGED;
        finish_task(T);
      } else if (T.it >= H->opt.max_cycles) {
        finish_task(T);
      } else {
        launch_iteration(H, mixed, s);
      }
      break;
    case 10: {   // Krylov: squared 2-norm of the restart's residual
      const int k = H->opt.krylov;
      T.kbeta = std::sqrt(std::max(H->kr_dot_host[0], 0.0));
      if (!std::isfinite(T.kbeta)) {
        T.res.status = CC_ERR_DIVERGED;
        finish_task(T);
        break;
      }
      if (T.kbeta == 0.0) {
        T.res.status = CC_OK;
        finish_task(T);
        break;
      }
      T.kH.assign((size_t)k * (k + 1), 0.0);   // column j at j (k + 1)
      T.kcs.assign(k, 0.0);
      T.ksn.assign(k, 0.0);
      T.kg.assign(k + 1, 0.0);
      T.kg[0] = T.kbeta;
      pdl_launch(k_maxpy, KR_BLOCKS, 256, 0, s, (const double*)nullptr, 0, (const double*)nullptr,
                 kr_vec(H, 0), 1.0 / T.kbeta, L.nn);
      T.kj = 0;
      kr_arnoldi(T);
      break;
    }
    case 11: {   // Krylov: first projections of V_{j+1}; subtract them, project again
      const int j = T.kj;
      T.kh1.assign(H->kr_dot_host, H->kr_dot_host + j + 1);
      pdl_launch(k_maxpy, KR_BLOCKS, 256, 0, s, (const double*)H->kr_v, j + 1, (const double*)H->kr_dot,
                 kr_vec(H, j + 1), 1.0, L.nn);
      kr_dots(H, j + 1, kr_vec(H, j + 1), 1, s);
      CK(cudaEventRecord(H->step_ev, s));
      T.phase = 12;
      break;
    }
    case 12: {   // Krylov: second projections and |w|^2 give column j of the Hessenberg matrix
      const int k = H->opt.krylov, j = T.kj;
      double* col = &T.kH[(size_t)j * (k + 1)];
      double h2n = 0.0;
      for (int i = 0; i <= j; ++i) {
        const double h2 = H->kr_dot_host[i];
        col[i] = T.kh1[i] + h2;
        h2n += h2 * h2;
      }
      const double hn = std::sqrt(std::max(H->kr_dot_host[j + 1] - h2n, 0.0));
      col[j + 1] = hn;
      pdl_launch(k_maxpy, KR_BLOCKS, 256, 0, s, (const double*)H->kr_v, j + 1, (const double*)H->kr_dot,
                 kr_vec(H, j + 1), hn > 0.0 ? 1.0 / hn : 1.0, L.nn);
      for (int i = 0; i < j; ++i) {
        const double t = T.kcs[i] * col[i] + T.ksn[i] * col[i + 1];
        col[i + 1] = -T.ksn[i] * col[i] + T.kcs[i] * col[i + 1];
        col[i] = t;
      }
      const double d = std::hypot(col[j], col[j + 1]);
      T.kcs[j] = d > 0.0 ? col[j] / d : 1.0;
      T.ksn[j] = d > 0.0 ? col[j + 1] / d : 0.0;
      col[j] = d;
      col[j + 1] = 0.0;
      T.kg[j + 1] = -T.ksn[j] * T.kg[j];
      T.kg[j] = T.kcs[j] * T.kg[j];
      ++T.it;
      const double est = std::fabs(T.kg[j + 1]);
      const int m = j + 1;
      if (!std::isfinite(est) || !std::isfinite(d)) {
        T.res.status = CC_ERR_DIVERGED;
        finish_task(T);
      } else if (est < T.tol * T.bn || m == k || hn == 0.0 || T.it >= H->opt.max_cycles) {
        kr_end_restart(T, m);
      } else {
        T.kj = m;
        kr_arnoldi(T);
      }
      break;
    }
    case 13:   // Krylov: max-norm of the true residual after a restart
      T.rel = host_norm(H) / T.bn;
      if (T.rel < T.tol) {
        T.res.status = CC_OK;
        finish_task(T);
      } else if (!std::isfinite(T.rel) || (T.first > 0 && T.rel > 1e3 * T.first)) {
        T.res.status = CC_ERR_DIVERGED;
        finish_task(T);
      } else if (T.it >= H->opt.max_cycles) {
        finish_task(T);
      } else {
        kr_restart(T);
      }
      break;
    case 4:
      T.res.cycles = T.it;
      T.res.rel_res = T.rel;
      T.phase = 5;
      break;
  }
  T.launches += t_launches - l0;
  T.res.kernels = T.launches;
  return T.phase == 5;
}

// Drive every task to completion, advancing each as soon as its last step
// has completed on the GPU.  The handles must be distinct.
void run_solves(std::vector<SolveTask>& T) {
  size_t left = T.size();
  for (auto& t : T)
    if (solve_step(t)) --left;
  while (left) {
    bool moved = false;
    for (auto& t : T) {
      if (t.phase == 5) continue;
      cudaError_t q = cudaEventQuery(t.H->step_ev);
      if (q == cudaErrorNotReady) continue;
      CK(q);
      if (solve_step(t)) --left;
      moved = true;
    }
    if (!moved) std::this_thread::yield();
  }
}

cc_status solve_impl(cc_hierarchy* H, const double* f, const double* g, double* u, double tol,
                     cudaStream_t s, cc_result* out) {
  std::vector<SolveTask> T(1);
  T[0].H = H;
  T[0].f = f;
  T[0].g = g;
  T[0].u = u;
  T[0].tol = tol;
  T[0].s = s;
  // one solve alone: its iterations run in the loop graph.  Batches and
  // served requests keep the host loop, under which concurrent solves on
  // several streams overlapped better (8 concurrent 1024^2 solves: 35 ms
  // against 52 ms with loop graphs)
  T[0].device_loop = true;
  run_solves(T);
  if (out) *out = T[0].res;
  return T[0].res.status;
}

// The serving scheduler of a handle (continuous batching).  Requests wait in
// the handle's queue; whenever a slot is free (the handle itself, or a clone
// created on demand up to serve_slots and within the serving memory budget)
// the oldest request is admitted and started, and every request in flight is
// advanced as soon as its previous step has completed on the GPU, so
// requests that arrive while others run overlap with them on the device.
void worker_loop(cc_hierarchy* H) {
  if (cudaSetDevice(H->device) != cudaSuccess) return;
  struct Active {
    uint64_t id;
    double t_start;
    SolveTask task;
  };
  std::vector<int> busy;                       // per slot: index into act, or -1
  std::vector<Active> act;
  if (H->slots.empty()) H->slots.push_back(H);
  busy.assign(H->slots.size(), -1);
  for (;;) {
    // admit
    for (;;) {
      int free_slot = -1;
      for (size_t k = 0; k < busy.size(); ++k)
        if (busy[k] < 0) { free_slot = (int)k; break; }
      uint64_t id = 0;
      {
        std::unique_lock<std::mutex> lk(H->qmu);
        if (act.empty())
          H->qcv.wait(lk, [&] { return H->stop || !H->queue.empty(); });
        if (H->queue.empty()) {
          if (H->stop && act.empty()) return;
          break;
        }
        if (free_slot < 0 && (int)H->slots.size() >= std::max(1, H->opt.serve_slots)) break;
        if (free_slot < 0) {
          // a new clone, if the serving budget allows it
          cc_hierarchy* c = nullptr;
          const int64_t est = H->slots.size() > 1 ? H->slot_bytes / (int64_t)(H->slots.size() - 1)
                                                  : H->pool->bytes;
          const int64_t cap = g_serve_budget.load();
          if (cap > 0 && g_serve_used.load() + est > cap) break;
          if (cc_clone(H, (cc_stream)H->wstream, &c) != CC_OK) break;
          H->slots.push_back(c);
          H->slot_bytes += c->pool->bytes;
          g_serve_used += c->pool->bytes;
          busy.push_back(-1);
          free_slot = (int)busy.size() - 1;
        }
        id = H->queue.front();
        H->queue.pop_front();
      }
      Request rq;
      {
        std::lock_guard<std::mutex> lk(g_reqmu);
        rq = g_req[id];
      }
      Active a;
      a.id = id;
      a.t_start = now_s();
      cc_hierarchy* S = H->slots[free_slot];
      a.task.H = S;
      a.task.f = rq.f;
      a.task.g = rq.g;
      a.task.u = rq.u;
      a.task.tol = rq.tol;
      a.task.s = S == H ? H->wstream : S->gstream;
      busy[free_slot] = (int)act.size();
      act.push_back(a);
      try {
        solve_step(act.back().task);
      } catch (CudaError&) {
        act.back().task.res.status = CC_ERR_CUDA;
        act.back().task.phase = 5;
      }
    }
    // advance
    bool moved = false;
    for (size_t k = 0; k < busy.size(); ++k) {
      if (busy[k] < 0) continue;
      Active& a = act[busy[k]];
      cudaError_t q = cudaEventQuery(a.task.H->step_ev);
      if (q == cudaErrorNotReady) continue;
      bool done = true;
      if (q == cudaSuccess) {
        try {
          done = solve_step(a.task);
        } catch (CudaError&) {
          a.task.res.status = CC_ERR_CUDA;
        }
      } else {
        (void)cudaGetLastError();
        a.task.res.status = CC_ERR_CUDA;
      }
      moved = true;
      if (!done) continue;
      cc_result res = a.task.res;
      {
        std::lock_guard<std::mutex> lk(g_reqmu);
        auto it = g_req.find(a.id);
        if (it != g_req.end()) {
          res.t_submit = it->second.res.t_submit;
          res.t_start = a.t_start;
          res.t_done = now_s();
          it->second.res = res;
          it->second.done = true;
        }
      }
      // release the slot; keep act compact
      const int idx = busy[k];
      busy[k] = -1;
      if (idx != (int)act.size() - 1) {
        act[idx] = act.back();
        for (auto& b : busy)
          if (b == (int)act.size() - 1) b = idx;
      }
      act.pop_back();
    }
    if (!moved) std::this_thread::yield();
  }
}

void destroy_hierarchy(cc_hierarchy* H) {
  if (!H) return;
  if (H->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(H->qmu);
      H->stop = true;
    }
    H->qcv.notify_all();
    H->worker.join();
  }
  for (size_t k = 1; k < H->slots.size(); ++k) destroy_hierarchy(H->slots[k]);
  g_serve_used -= H->slot_bytes;
  H->slots.clear();
  if (!H->opt.host_only) cudaDeviceSynchronize();
  for (auto& g : H->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (H->kr_graph) cudaGraphExecDestroy(H->kr_graph);
  if (H->loop_exec) cudaGraphExecDestroy(H->loop_exec);
  if (H->h_loop) cudaFreeHost(H->h_loop);
  if (H->kr_dot_host) cudaFreeHost(H->kr_dot_host);
  if (H->kr_y_host) cudaFreeHost(H->kr_y_host);
  for (auto& e : H->ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (H->step_ev) cudaEventDestroy(H->step_ev);
  if (H->wstream) cudaStreamDestroy(H->wstream);
  if (H->gstream) cudaStreamDestroy(H->gstream);
  if (H->h_norm) cudaFreeHost(H->h_norm);
  H->pool.reset();
  H->tables.reset();
  delete H;
}

}  // namespace

// ============================================================================
// ---- launch shapes timed on the device (cc_options.autotune) ----------------
const int kTuneMaxM = 8192;     // largest exact block whose chunk size is timed
const int kTuneCandidates = 3;  // chunk shapes timed per block (the cheapest by the cost model)

// device milliseconds of `reps` runs of f() on s, after 3 untimed runs
template <class F>
float time_launches(cudaStream_t s, int reps, F&& f) {
  struct Ev {
    cudaEvent_t e = nullptr;
    ~Ev() { if (e) cudaEventDestroy(e); }
  } e0, e1;
  CK(cudaEventCreate(&e0.e));
  CK(cudaEventCreate(&e1.e));
  for (int i = 0; i < 3; ++i) f();
  CK(cudaEventRecord(e0.e, s));
  for (int i = 0; i < reps; ++i) f();
  CK(cudaEventRecord(e1.e, s));
  CK(cudaEventSynchronize(e1.e));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0.e, e1.e));
  return ms;
}

// the fastest of candidate plans of one exact block: each is uploaded to a
// temporary pool and timed over 20 FP32 solves on zero vectors
int tune_block_plan(std::vector<BlockPlan>& cand, int64_t nn, cudaStream_t s, unsigned int* fault) {
  if (cand.size() < 2) return 0;
  Pool tmp;
  float* u = tmp.alloc<float>(nn);
  float* b = tmp.alloc<float>(nn);
  CK(cudaMemsetAsync(u, 0, nn * sizeof(float), s));
  CK(cudaMemsetAsync(b, 0, nn * sizeof(float), s));
  int best = 0;
  float best_ms = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    BlockDev d = upload_block<float>(tmp, cand[i], s);
    alloc_block_work<float>(tmp, cand[i], d, fault);
    int s1, s2;
    const ChunkSmem sm = chunk_smem(cand[i], (int)sizeof(float), s1, s2);
    const float ms = time_launches(s, 20, [&] { launch_block<float>(cand[i], d, sm, u, (const float*)b, s); });
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best = (int)i;
    }
  }
  CK(cudaStreamSynchronize(s));
  return best;
}

// CTAs of the streamed FP32 sweep of level L: every multiple of the SM count
// up to the occupancy limit, and one CTA per tile, each timed over 20
// sweeps; remembered per (device, grid size, cross term) for the process
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_sweep_tune;

int tune_sweep(Level& L, int device, cudaStream_t s) {
  const bool cross = L.sp.cross != 0;
  const auto key = std::make_tuple(device, L.n, cross ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_sweep_tune.find(key);
    if (it != g_sweep_tune.end()) return it->second;
  }
  const int nt = (L.n / TX) * (L.n / WY);
  int sms = 0, occ = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  if (cross) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_p<true>, TX * TY, 0));
  else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep_p<false>, TX * TY, 0));
  std::vector<int> grids;
  for (int k = 1; k <= std::max(1, occ); ++k) grids.push_back(std::min(nt, sms * k));
  grids.push_back(nt);
  std::sort(grids.begin(), grids.end());
  grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
  int best = 0;
  float best_ms = 0;
  for (int g : grids) {
    L.sweep_grid = g;
    const float ms = time_launches(s, 20, [&] {
      launch_sweep<float>(L, (const float*)L.u32[0], L.u32[1], (const float*)L.b32, (const float*)nullptr,
                          false, s);
    });
    if (best == 0 || ms < best_ms) {
      best_ms = ms;
      best = g;
    }
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_sweep_tune[key] = best;
  return best;
}

extern "C" {

void cc_default_options(cc_options* o) {
  if (!o) return;
  o->eps = 0.1;
  o->nu1 = 3;
  o->nu2 = 3;
  o->omega = 0.5;
  o->cycle = CC_CYCLE_V;
  o->min_coarse_n = 4;
  o->precision = CC_PREC_FP64;
  o->max_cycles = 100;
  o->use_graphs = 1;
  o->host_only = 0;
  o->fmg_cycle = CC_CYCLE_V;
  o->w_depth = 0;
  o->serve_slots = 4;
  o->cache = 0;
  o->hole_cells = 2.0;
  o->krylov = 0;
  o->smoother = CC_SMOOTHER_JACOBI;
  o->device_setup = 1;
  o->device_loop = 1;
  o->autotune = 1;
}

const char* cc_last_error_string(void) { return t_last_error; }

const char* cc_status_string(cc_status s) {
  switch (s) {
    case CC_OK: return "ok";
    case CC_ERR_ARG: return "invalid argument";
    case CC_ERR_GEOMETRY: return "domain not resolved by the grid";
    case CC_ERR_SINGULAR: return "singular fit or factorisation";
    case CC_ERR_NO_MEMORY: return "out of memory";
    case CC_ERR_NOT_CONVERGED: return "not converged";
    case CC_ERR_DIVERGED: return "diverged";
    case CC_ERR_TIMEOUT: return "timeout";
    case CC_ERR_CUDA: return "CUDA error";
    case CC_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

cc_status cc_setup(const cc_domain* dom, double a, double b, double c, const cc_bc* bc, int n_bc,
                   int n, const cc_options* opt, cc_stream stream, cc_handle* out) {
  t_last_error[0] = '\0';
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  if (!dom || !bc || n < 4 || (dom->n_holes > 0 && !dom->holes)) return CC_ERR_ARG;
  if (!(b * b < 4 * a * c) || !(a > 0)) return CC_ERR_ARG;
  if (n_bc != 4 + dom->n_holes) return CC_ERR_ARG;
  cc_options o;
  cc_default_options(&o);
  if (opt) o = *opt;
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 == 0 || o.min_coarse_n < 4 || o.max_cycles < 1 ||
      !(o.eps > 0 && o.eps < 1) || (o.cycle < 1 || o.cycle > 3) ||
      (o.fmg_cycle != CC_CYCLE_V && o.fmg_cycle != CC_CYCLE_W) || o.w_depth < 0 ||
      o.serve_slots < 1 || !(o.hole_cells > 0) || o.krylov < 0 || o.krylov > KR_MAXV - 1 ||
      (o.krylov && o.cycle == CC_CYCLE_FMG) ||
      (o.smoother != CC_SMOOTHER_JACOBI && o.smoother != CC_SMOOTHER_MCGS))
    return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the setup cache: a clone of the hierarchy of an identical earlier call
  std::string key;
  if (o.cache && !o.host_only) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_CUDA;
    key = setup_key(dom, a, b, c, bc, n_bc, n, o, dev);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      cc_status st = cc_clone(it->second, stream, out);
      if (st == CC_OK) {
        (*out)->opt = o;
        try {
          ensure_krylov(*out, s);
          CK(cudaStreamSynchronize(s));
        } catch (CudaError& e) {
          destroy_hierarchy(*out);
          *out = nullptr;
          return e.e == cudaErrorMemoryAllocation ? CC_ERR_NO_MEMORY : CC_ERR_CUDA;
        }
      }
      return st;
    }
  }
  const double t_setup0 = now_s();
  cc_hierarchy* H = new cc_hierarchy();
  H->opt = o;
  Problem& P = H->P;
  P.x0 = dom->x0; P.y0 = dom->y0; P.x1 = dom->x1; P.y1 = dom->y1;
  P.a = a; P.b = b; P.c = c; P.eps = o.eps;
  for (int k = 0; k < dom->n_holes; ++k) {
    const cc_hole& hh = dom->holes[k];
    if (!(hh.r1 > 0 && hh.r2 > 0) ||
        (hh.kind != CC_HOLE_ELLIPSE && hh.kind != CC_HOLE_FLOWER && hh.kind != CC_HOLE_OUTSIDE_RECT)) {
      delete H;
      return CC_ERR_ARG;
    }
    if (hh.kind == CC_HOLE_FLOWER && !(hh.r2 < hh.r1 && hh.theta >= 1 && hh.theta == std::floor(hh.theta))) {
      delete H;
      return CC_ERR_ARG;
    }
    Hole e{hh.cx, hh.cy, hh.r1, hh.r2, hh.theta, std::cos(hh.theta), std::sin(hh.theta)};
    e.kind = hh.kind;
    e.petals = hh.kind == CC_HOLE_FLOWER ? (int)hh.theta : 0;
    P.holes.push_back(e);
  }
  for (int k = 0; k < n_bc; ++k) {
    if (bc[k].type < 0 || bc[k].type > 2) { delete H; return CC_ERR_ARG; }
    P.bc.push_back({bc[k].type, bc[k].alpha1, bc[k].alpha2});
  }
  const bool dev = !o.host_only;
  std::unique_ptr<SetupDevice> sdev;
  try {
    if (dev) {
      CK(cudaGetDevice(&H->device));
      H->noalloc = noalloc_scratch();
      if (o.device_setup) sdev = std::make_unique<SetupDevice>((void*)s);
      pdl_setup_device();
      chunk_smem_attributes();
      // norm words: [0] the max-norm of a residual, [1] the fault word of
      // bounded waits in the kernels
      H->d_norm = H->pool->alloc<unsigned long long>(2);
      CK(cudaMemsetAsync(H->d_norm, 0, 2 * sizeof(unsigned long long), s));
    }
    // levels: halve while the level is resolved and discretisable (Eq. 5.9)
    int nl = n;
    while (true) {
      // a coarse level must resolve every hole: hole_cells cells across its
      // smaller semi-axis (the precondition of Alg. 1, made concrete)
      if (!H->lv.empty()) {
        double hl = (P.x1 - P.x0) / nl;
        bool fine_enough = true;
        for (const Hole& e : P.holes) fine_enough = fine_enough && e.halfwidth() >= o.hole_cells * hl;
        if (!fine_enough) break;
      }
      LevelDisc D;
      try {
        const double t_d = now_s();
        D = discretize(P, nl, sdev.get());
        H->setup_tables_seconds += now_s() - t_d;
        if (!D.geom.resolved) throw SetupError(2, D.geom.reason);
      } catch (SetupError& e) {
        if (H->lv.empty()) throw;
        break;
      }
      auto L = std::make_unique<Level>();
      L->disc() = std::move(D);
      L->n = nl;
      L->nn = (int64_t)nl * nl;
      H->lv.push_back(std::move(L));
      if (nl % 2 || nl / 2 < o.min_coarse_n || H->lv.size() >= 30) break;
      nl /= 2;
    }
    // every level but the finest must keep the box walls extendable in the
    // same rows: nothing else is required for the cycle.
    for (size_t l = 0; l < H->lv.size(); ++l) {
      Level& L = *H->lv[l];
      const LevelDisc& D = L.disc();
      L.disc().P = &H->P;
      L.sp = make_stencil(D, o.omega);
      L.spf = stencil_as<float>(L.sp);
      // merged-away control volumes take their owner's value (Eq. 5.11)
      auto attach_aliases = [&](BlockPlan& B) {
        std::unordered_map<int, int> pos;
        for (int p = 0; p < B.m; ++p) pos[B.cell[p]] = p;
        std::vector<std::vector<int>> al(B.m);
        for (int64_t k = 0; l > 0 && k < L.nn; ++k)
          if (D.geom.type[k] == CT_EMPTY && D.geom.owner[k] >= 0 && D.geom.owner[k] != k) {
            auto it = pos.find(D.geom.owner[k]);
            if (it == pos.end()) throw SetupError(3, "a merged cell is not in the exact block");
            al[it->second].push_back((int)k);
          }
        B.alias_ptr.assign(1, 0);
        B.alias_cell.clear();
        for (auto& v : al) {
          B.alias_cell.insert(B.alias_cell.end(), v.begin(), v.end());
          B.alias_ptr.push_back((int)B.alias_cell.size());
        }
      };
      // dense inverses of 256 rows and more on the device with the setup steps
      const Inverter dev_inv = [&](std::vector<double>& A, int n) {
        return n >= 256 ? sdev->invert(A, n) : invert(A, n);
      };
      const Inverter* inv = sdev ? &dev_inv : nullptr;
      const int mblk = (int)D.block.size();
      if (dev && o.autotune && l + 1 < H->lv.size() && mblk > kDenseMax && mblk <= kTuneMaxM) {
        // chunk size: the fastest of the cost model's cheapest plans
        std::vector<BlockPlan> cand = plan_block_candidates(D, kTuneCandidates, inv);
        for (BlockPlan& B : cand) attach_aliases(B);
        const int pick = tune_block_plan(cand, L.nn, s, reinterpret_cast<unsigned int*>(H->d_norm + 1));
        L.plan() = std::move(cand[pick]);
      } else {
        L.plan() = plan_block(D, inv);
        attach_aliases(L.plan());
      }
      if (!dev) continue;
      std::vector<uint8_t> cls(L.nn, C_EMPTY);
      for (int64_t k = 0; k < L.nn; ++k)
        if (D.kind[k] != K_EMPTY) cls[k] = C_STENCIL;
      for (int k : D.block) cls[k] = C_BLOCK;
      L.cls = H->pool->upload(cls, s);
      for (int i = 0; i < 2; ++i) {
        L.u64[i] = H->pool->alloc<double>(L.nn);
        L.u32[i] = H->pool->alloc<float>(L.nn);
        CK(cudaMemsetAsync(L.u64[i], 0, L.nn * sizeof(double), s));
        CK(cudaMemsetAsync(L.u32[i], 0, L.nn * sizeof(float), s));
      }
      L.b64 = H->pool->alloc<double>(L.nn);
      L.b32 = H->pool->alloc<float>(L.nn);
      CK(cudaMemsetAsync(L.b64, 0, L.nn * sizeof(double), s));
      CK(cudaMemsetAsync(L.b32, 0, L.nn * sizeof(float), s));
      if (o.autotune && L.n >= 256 && L.n % 32 == 0) L.sweep_grid = tune_sweep(L, H->device, s);
      if (l + 1 < H->lv.size()) {
        unsigned int* fault = reinterpret_cast<unsigned int*>(H->d_norm + 1);
        L.blk.d64 = upload_block<double>(*H->pool, L.plan(), s);
        L.blk.d32 = upload_block<float>(*H->pool, L.plan(), s);
        alloc_block_work<double>(*H->pool, L.plan(), L.blk.d64, fault);
        alloc_block_work<float>(*H->pool, L.plan(), L.blk.d32, fault);
        if (!L.plan().dense && L.plan().m) {
          int s1, s2;
          L.blk.sm64 = chunk_smem(L.plan(), 8, s1, s2);
          L.blk.sm32 = chunk_smem(L.plan(), 4, s1, s2);
        }
      }
      if (!D.block.empty()) {
        L.brow_cell = H->pool->upload(D.block, s);
        L.brow_ptr = H->pool->upload(D.block_rows.ptr, s);
        L.brow_col = H->pool->upload(D.block_rows.col, s);
        L.brow_val = H->pool->upload(D.block_rows.val, s);
      }
      std::vector<int> fd, fs;
      for (int64_t k = 0; k < L.nn; ++k)
        if (D.geom.type[k] == CT_EMPTY && D.geom.owner[k] >= 0 && D.geom.owner[k] != k) {
          fd.push_back((int)k);
          fs.push_back(D.geom.owner[k]);
        }
      L.nfix = (int)fd.size();
      if (L.nfix) {
        L.fix_dst = H->pool->upload(fd, s);
        L.fix_src = H->pool->upload(fs, s);
      }
    }
    // bottom: dense inverse of the coarsest level's matrix
    if (dev) {
      Level& L = *H->lv.back();
      const int nc = (int)L.nn;
      if (nc > 4096) throw SetupError(1, "coarsest level too large for the dense bottom solve");
      std::vector<double> A((size_t)nc * nc, 0.0);
      std::map<int, double> ar;
      for (int k = 0; k < nc; ++k) {
        L.disc().row(k, ar, nullptr);
        for (auto& kv : ar) A[(size_t)k * nc + kv.first] += kv.second;
        // a merged-away control volume repeats its owner's value (Eq. 5.11)
        int own = L.disc().geom.owner[k];
        if (H->lv.size() > 1 && L.disc().kind[k] == K_EMPTY && own >= 0 && own != k)
          A[(size_t)k * nc + own] = -1.0;
      }
      std::vector<double> A0(A);
      const bool inv_ok = (sdev && nc >= 256) ? sdev->invert(A, nc) : invert(A, nc);
      if (!inv_ok) throw SetupError(3, "singular coarsest-level matrix");
      {
        std::vector<double> t(nc), x(nc, 0.0);
        for (int k = 0; k < nc; ++k) t[k] = std::sin(1.0 + 0.7 * k) + 0.25 * std::cos(3.1 * k);
        for (int r = 0; r < nc; ++r) {
          double acc = 0;
          for (int k = 0; k < nc; ++k) acc += A[(size_t)r * nc + k] * t[k];
          x[r] = acc;
        }
        double rmax = 0, amax = 0, xmax = 0;
        for (int r = 0; r < nc; ++r) {
          double acc = -t[r], arow = 0;
          for (int k = 0; k < nc; ++k) { acc += A0[(size_t)r * nc + k] * x[k]; arow += std::fabs(A0[(size_t)r * nc + k]); }
          rmax = std::max(rmax, std::fabs(acc));
          amax = std::max(amax, arow);
          xmax = std::max(xmax, std::fabs(x[r]));
        }
        H->bottom_error = rmax / (amax * xmax);
      }
      if (dev) H->bottom_inv = H->pool->upload(A, s);   // row-major
      H->nc_bottom = nc;
    }
    // finest level: N rows, residual buffers, norms
    {
      Level& L = *H->lv[0];
      const LevelDisc& D = L.disc();
      H->n_bd = (int)D.bd_cells.size();
      H->n_g = 4 * n + H->n_bd;
      H->n_nrows = D.nrows.rows();
      int64_t dof = 0;
      for (int64_t k = 0; k < L.nn; ++k) dof += D.kind[k] != K_EMPTY;
      H->n_dof = dof;
      if (!dev) goto done;
      if (H->n_nrows) {
        H->nrow_cell = H->pool->upload(D.nrow_cell, s);
        H->nrow_ptr = H->pool->upload(D.nrows.ptr, s);
        H->nrow_col = H->pool->upload(D.nrows.col, s);
        H->nrow_val = H->pool->upload(D.nrows.val, s);
      }
      H->r64 = H->pool->alloc<double>(L.nn);
      CK(cudaMemsetAsync(H->r64, 0, L.nn * sizeof(double), s));
      CK(cudaMallocHost(&H->h_norm, 2 * sizeof(unsigned long long)));
      H->h_norm[0] = H->h_norm[1] = 0;
      CK(cudaEventCreateWithFlags(&H->step_ev, cudaEventDisableTiming));
      ensure_krylov(H, s);
    }
    CK(cudaStreamCreateWithFlags(&H->gstream, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(s));
  done:;
    if (sdev) H->setup_kernel_ms = sdev->kernel_ms;
    sdev.reset();
  } catch (SetupError& e) {
    cc_status st = from_setup(e.code);
    snprintf(t_last_error, sizeof(t_last_error), "%s", e.what());
    sdev.reset();
    destroy_hierarchy(H);
    return st;
  } catch (DeviceError& e) {
    snprintf(t_last_error, sizeof(t_last_error), "%s", e.what());
    sdev.reset();
    destroy_hierarchy(H);
    return e.err == (int)cudaErrorMemoryAllocation ? CC_ERR_NO_MEMORY : CC_ERR_CUDA;
  } catch (CudaError& e) {
    destroy_hierarchy(H);
    return e.e == cudaErrorMemoryAllocation ? CC_ERR_NO_MEMORY : CC_ERR_CUDA;
  } catch (std::bad_alloc&) {
    destroy_hierarchy(H);
    return CC_ERR_NO_MEMORY;
  }
  H->setup_seconds = now_s() - t_setup0;
  if (!key.empty()) {
    // the cache keeps a clone of its own, so destroying H leaves it valid
    cc_hierarchy* T = nullptr;
    if (cc_clone(H, stream, &T) == CC_OK) {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      if (!g_cache.emplace(key, T).second) destroy_hierarchy(T);
    }
  }
  *out = H;
  return CC_OK;
}

cc_status cc_cache_clear(void) {
  std::map<std::string, cc_hierarchy*> old;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    old.swap(g_cache);
  }
  for (auto& kv : old) destroy_hierarchy(kv.second);
  return CC_OK;
}

cc_status cc_query(cc_handle H, cc_info* out) {
  if (!H || !out) return CC_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->n = H->lv[0]->n;
  out->n_levels = (int)H->lv.size();
  out->n_dof = H->n_dof;
  out->n_bd = H->n_bd;
  out->n_g = H->n_g;
  out->n_plg = (int)H->lv[0]->disc().plg.size();
  out->n_block = (int)H->lv[0]->disc().block.size();
  out->device_bytes = H->pool->bytes;
  for (size_t l = 0; l < H->lv.size() && l < 32; ++l) {
    out->level_n[l] = H->lv[l]->n;
    out->block_error = std::max(out->block_error, H->lv[l]->plan().error);
    out->block_m[l] = H->lv[l]->plan().m;
    out->block_chunks[l] = H->lv[l]->plan().dense ? 0 : H->lv[l]->plan().nch;
  }
  out->bottom_error = H->bottom_error;
  for (size_t l = 0; l < H->lv.size() && l < 32; ++l) {
    const Level& L = *H->lv[l];
    out->sweep_ctas[l] = L.sweep_grid;
    if (!H->opt.host_only && L.n >= 256 && L.n % 32 == 0 && L.sweep_grid == 0)
      out->sweep_ctas[l] = std::min((L.n / TX) * (L.n / WY),
                                    L.sp.cross ? sweep_p_blocks<true>() : sweep_p_blocks<false>());
    out->block_chunk_rows[l] = (L.plan().m && !L.plan().dense) ? L.plan().s : 0;
  }
  out->setup_seconds = H->setup_seconds;
  out->setup_tables_seconds = H->setup_tables_seconds;
  out->setup_kernel_ms = H->setup_kernel_ms;
  return CC_OK;
}

cc_status cc_level_block(cc_handle H, int level, int* h_cells, int* m) {
  if (!H || !m || level < 0 || level >= (int)H->lv.size()) return CC_ERR_ARG;
  const std::vector<int>& b = H->lv[level]->disc().block;
  *m = (int)b.size();
  if (h_cells) std::copy(b.begin(), b.end(), h_cells);
  return CC_OK;
}

cc_status cc_destroy(cc_handle H) {
  if (!H) return CC_ERR_ARG;
  destroy_hierarchy(H);
  return CC_OK;
}

cc_status cc_cell_types(cc_handle H, uint8_t* h_type, uint8_t* h_kind, double* h_vol) {
  if (!H || !h_type) return CC_ERR_ARG;
  const LevelDisc& D = H->lv[0]->disc();
  std::copy(D.geom.type.begin(), D.geom.type.end(), h_type);
  if (h_kind) std::copy(D.kind.begin(), D.kind.end(), h_kind);
  if (h_vol) std::copy(D.geom.vol.begin(), D.geom.vol.end(), h_vol);
  return CC_OK;
}

cc_status cc_quadrature_nodes(cc_handle H, int* n_cut, int64_t* nv, int64_t* nb, int* h_cell,
                              int64_t* h_vptr, double* h_vnode, int64_t* h_bptr, double* h_bnode,
                              int* h_bbc) {
  if (!H || !n_cut || !nv || !nb) return CC_ERR_ARG;
  const LevelDisc& D = H->lv[0]->disc();
  const LevelGeom& G = D.geom;
  int nc = 0;
  int64_t v = 0, bcount = 0;
  for (auto& kv : G.cut) {
    auto vn = volume_nodes(H->P, G, kv.first);
    if (h_cell) {
      h_cell[nc] = kv.first;
      h_vptr[nc] = v;
      for (size_t q = 0; q < vn.size(); ++q)
        for (int t = 0; t < 3; ++t) h_vnode[3 * (v + (int64_t)q) + t] = vn[q][t];
    }
    v += (int64_t)vn.size();
    ++nc;
  }
  if (h_cell && h_vptr) h_vptr[nc] = v;
  for (size_t r = 0; r < D.bd_cells.size(); ++r) {
    auto bn = boundary_nodes(H->P, G, D.bd_cells[r]);
    double ws = 0;
    for (auto& x : bn) ws += x.w;
    if (h_bptr) {
      h_bptr[r] = bcount;
      for (size_t q = 0; q < bn.size(); ++q) {
        double* o = h_bnode + 5 * (bcount + (int64_t)q);
        o[0] = bn[q].x; o[1] = bn[q].y; o[2] = bn[q].nx; o[3] = bn[q].ny; o[4] = bn[q].w / ws;
        h_bbc[bcount + (int64_t)q] = bn[q].bc;
      }
    }
    bcount += (int64_t)bn.size();
  }
  if (h_bptr) h_bptr[D.bd_cells.size()] = bcount;
  *n_cut = nc;
  *nv = v;
  *nb = bcount;
  return CC_OK;
}

cc_status cc_clone(cc_handle S, cc_stream stream, cc_handle* out) {
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  if (!S || S->opt.host_only) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cc_hierarchy* H = nullptr;
  try {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != S->device) return CC_ERR_ARG;
    H = new cc_hierarchy();
    H->P = S->P;
    H->opt = S->opt;
    H->device = S->device;
    H->noalloc = S->noalloc;
    H->tables = S->tables ? S->tables : S->pool;
    H->bottom_inv = S->bottom_inv;
    H->bottom_error = S->bottom_error;
    H->nc_bottom = S->nc_bottom;
    H->nrow_cell = S->nrow_cell;
    H->nrow_ptr = S->nrow_ptr;
    H->nrow_col = S->nrow_col;
    H->nrow_val = S->nrow_val;
    H->n_nrows = S->n_nrows;
    H->n_g = S->n_g;
    H->n_bd = S->n_bd;
    H->n_dof = S->n_dof;
    H->d_norm = H->pool->alloc<unsigned long long>(2);
    CK(cudaMemsetAsync(H->d_norm, 0, 2 * sizeof(unsigned long long), s));
    unsigned int* fault = reinterpret_cast<unsigned int*>(H->d_norm + 1);
    const size_t nl = S->lv.size();
    for (size_t l = 0; l < nl; ++l) {
      // shares the plan, the discretisation and every device table ...
      auto L = std::make_unique<Level>(*S->lv[l]);
      // ... and gets its own work arrays
      for (int i = 0; i < 2; ++i) {
        L->u64[i] = H->pool->alloc<double>(L->nn);
        L->u32[i] = H->pool->alloc<float>(L->nn);
        CK(cudaMemsetAsync(L->u64[i], 0, L->nn * sizeof(double), s));
        CK(cudaMemsetAsync(L->u32[i], 0, L->nn * sizeof(float), s));
      }
      L->b64 = H->pool->alloc<double>(L->nn);
      L->b32 = H->pool->alloc<float>(L->nn);
      CK(cudaMemsetAsync(L->b64, 0, L->nn * sizeof(double), s));
      CK(cudaMemsetAsync(L->b32, 0, L->nn * sizeof(float), s));
      const BlockPlan& B = L->plan();
      if (l + 1 < nl && B.m > 0) {
        alloc_block_work<double>(*H->pool, B, L->blk.d64, fault);
        alloc_block_work<float>(*H->pool, B, L->blk.d32, fault);
      }
      H->lv.push_back(std::move(L));
    }
    Level& L0 = *H->lv[0];
    H->r64 = H->pool->alloc<double>(L0.nn);
    CK(cudaMemsetAsync(H->r64, 0, L0.nn * sizeof(double), s));
    CK(cudaMallocHost(&H->h_norm, 2 * sizeof(unsigned long long)));
    H->h_norm[0] = H->h_norm[1] = 0;
    CK(cudaEventCreateWithFlags(&H->step_ev, cudaEventDisableTiming));
    ensure_krylov(H, s);
    CK(cudaStreamCreateWithFlags(&H->gstream, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(s));
  } catch (CudaError& e) {
    if (H) destroy_hierarchy(H);
    return e.e == cudaErrorMemoryAllocation ? CC_ERR_NO_MEMORY : CC_ERR_CUDA;
  }
  *out = H;
  return CC_OK;
}

cc_status cc_solve_batch(int n, const cc_handle* h, const double* const* f, const double* const* g,
                         double* const* u, const double* tol, const cc_stream* streams,
                         cc_result* out) {
  t_last_error[0] = '\0';
  if (n < 0 || (n > 0 && (!h || !f || !u || !tol))) return CC_ERR_ARG;
  std::vector<SolveTask> T(n);
  for (int i = 0; i < n; ++i) {
    cc_hierarchy* H = h[i];
    if (!H || H->opt.host_only || !f[i] || !u[i] || (H->n_g && (!g || !g[i])) || !(tol[i] > 0))
      return CC_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (h[j] == H) {
        snprintf(t_last_error, sizeof(t_last_error),
                 "cc_solve_batch: handle %d repeats handle %d (use cc_clone)", i, j);
        return CC_ERR_ARG;
      }
    T[i].H = H;
    T[i].f = f[i];
    T[i].g = g ? g[i] : nullptr;
    T[i].u = u[i];
    T[i].tol = tol[i];
    T[i].s = streams ? (cudaStream_t)streams[i] : H->gstream;
  }
  try {
    if (!streams) CK(cudaDeviceSynchronize());
    run_solves(T);
  } catch (CudaError&) {
    return CC_ERR_CUDA;
  }
  cc_status st = CC_OK;
  for (int i = 0; i < n; ++i) {
    if (out) out[i] = T[i].res;
    if (st == CC_OK && T[i].res.status != CC_OK) st = T[i].res.status;
  }
  return st;
}

cc_status cc_solve(cc_handle H, const double* f, const double* g, double* u, double tol,
                   cc_stream stream, cc_result* out) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || !f || !u || (H->n_g && !g) || !(tol > 0)) return CC_ERR_ARG;
  try {
    return solve_impl(H, f, g, u, tol, (cudaStream_t)stream, out);
  } catch (CudaError&) {
    return CC_ERR_CUDA;
  }
}

cc_status cc_solve_host(cc_handle H, const double* hf, const double* hg, double* hu, double tol,
                        cc_stream stream, cc_result* out) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || !hf || !hu || (H->n_g && !hg) || !(tol > 0)) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    Level& L = *H->lv[0];
    if (!H->h_u_dev) {
      H->h_u_dev = H->pool->alloc<double>(L.nn);
      H->h_f_dev = H->pool->alloc<double>(L.nn);
      H->h_g_dev = H->pool->alloc<double>(std::max(1, H->n_g));
    }
    CK(cudaMemcpyAsync(H->h_f_dev, hf, L.nn * sizeof(double), cudaMemcpyHostToDevice, s));
    if (H->n_g) CK(cudaMemcpyAsync(H->h_g_dev, hg, H->n_g * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(H->h_u_dev, hu, L.nn * sizeof(double), cudaMemcpyHostToDevice, s));
    cc_status st = solve_impl(H, H->h_f_dev, H->h_g_dev, H->h_u_dev, tol, s, out);
    CK(cudaMemcpyAsync(hu, H->h_u_dev, L.nn * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
  } catch (CudaError& e) {
    return e.e == cudaErrorMemoryAllocation ? CC_ERR_NO_MEMORY : CC_ERR_CUDA;
  }
}

cc_status cc_submit(cc_handle H, const double* f, const double* g, double* u, double tol,
                    uint64_t* req_id) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || !f || !u || !req_id || (H->n_g && !g) || !(tol > 0)) return CC_ERR_ARG;
  try {
    if (!H->worker.joinable()) {
      CK(cudaStreamCreateWithFlags(&H->wstream, cudaStreamNonBlocking));
      H->worker = std::thread(worker_loop, H);
    }
  } catch (CudaError&) {
    return CC_ERR_CUDA;
  }
  uint64_t id = g_next_id++;
  Request rq{H, f, g, u, tol, cc_result{}, false};
  rq.res.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(g_reqmu);
    g_req[id] = rq;
  }
  {
    std::lock_guard<std::mutex> lk(H->qmu);
    H->queue.push_back(id);
  }
  H->qcv.notify_one();
  *req_id = id;
  return CC_OK;
}

cc_status cc_serve_budget(int64_t bytes) {
  if (bytes < 0) return CC_ERR_ARG;
  g_serve_budget = bytes;
  return CC_OK;
}

cc_status cc_poll(uint64_t id, cc_result* out) {
  std::lock_guard<std::mutex> lk(g_reqmu);
  auto it = g_req.find(id);
  if (it == g_req.end()) return CC_ERR_ARG;
  if (!it->second.done) return CC_ERR_BUSY;
  if (out) *out = it->second.res;
  cc_status st = it->second.res.status;
  g_req.erase(it);
  return st;
}

// ---- operator-level entry points -------------------------------------------
cc_status cc_assemble_rhs(cc_handle H, const double* f, const double* g, double* b, cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || !f || !b || (H->n_g && !g)) return CC_ERR_ARG;
  try {
    assemble_rhs(H, f, g, b, (cudaStream_t)st);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_residual(cc_handle H, int l, const double* u, const double* b, double* r, cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || l < 0 || l >= (int)H->lv.size() || !u || !b || !r) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    Level& L = *H->lv[l];
    if (L.sp.cross)
      pdl_launch(k_resid_fx<double, true>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, r, L.sp, nullptr,
                 (double*)nullptr, 0.0);
    else
      pdl_launch(k_resid_fx<double, false>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, r, L.sp, nullptr,
                 (double*)nullptr, 0.0);
    if (!L.disc().block.empty())
      pdl_launch(k_block_resid<double>, nblk((int64_t)L.disc().block.size()), 256, 0, s, 
          (int)L.disc().block.size(), L.brow_cell, L.brow_ptr, L.brow_col, L.brow_val, u, b, r, nullptr);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_smooth(cc_handle H, int l, double* u, const double* b, cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || l < 0 || l + 1 >= (int)H->lv.size() || !u || !b) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    Level& L = *H->lv[l];
    CK(cudaMemcpyAsync(L.u64[0], u, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(L.u64[1], u, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(L.b64, b, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int cur = 0;
    sweep<double>(H, l, cur, false, (const double*)nullptr, s);
    pdl_launch(k_rhs_copy, nblk(L.nn), 256, 0, s, L.u64[cur], L.cls, u, L.nn);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_restrict_residual(cc_handle H, int l, const double* u, const double* b, double* rc,
                               cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || l < 0 || l + 1 >= (int)H->lv.size() || !u || !b || !rc) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    Level& L = *H->lv[l];
    Level& C = *H->lv[l + 1];
    if (L.sp.cross)
      pdl_launch(k_resid_restrict<double, true>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, C.cls, rc, L.sp,
                 (double*)nullptr, 0.0);
    else
      pdl_launch(k_resid_restrict<double, false>, tiles(L.n), TX * TY, 0, s, u, b, L.cls, C.cls, rc, L.sp,
                 (double*)nullptr, 0.0);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_prolong_add(cc_handle H, int l, const double* ec, double* u, cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || l < 0 || l + 1 >= (int)H->lv.size() || !ec || !u) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    Level& L = *H->lv[l];
    Level& C = *H->lv[l + 1];
    double* tmp = C.u64[1];
    CK(cudaMemcpyAsync(tmp, ec, C.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (C.nfix) pdl_launch(k_owner_fix<double>, nblk(C.nfix), 256, 0, s, C.nfix, C.fix_dst, C.fix_src, tmp);
    pdl_launch(k_prolong_add<double>, nblk(L.nn), 256, 0, s, u, tmp, L.cls, L.n);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_cycle(cc_handle H, double* u, const double* b, cc_stream st) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || !u || !b) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    Level& L = *H->lv[0];
    std::vector<int> cur(H->lv.size(), 0);
    if (H->opt.precision == CC_PREC_MIXED) {
      // the cycle of the mixed mode: FP32 on u and b rounded to FP32
      pdl_launch(k_convert<double, float>, nblk(L.nn), 256, 0, s, (const double*)u, L.u32[0], L.nn);
      pdl_launch(k_convert<double, float>, nblk(L.nn), 256, 0, s, b, L.b32, L.nn);
      cycle_level<float>(H, 0, cur, false, s);
      pdl_launch(k_convert<float, double>, nblk(L.nn), 256, 0, s, (const float*)L.u32[cur[0]], u, L.nn);
    } else {
      CK(cudaMemcpyAsync(L.u64[0], u, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(L.b64, b, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      cycle_level<double>(H, 0, cur, false, s);
      CK(cudaMemcpyAsync(u, L.u64[cur[0]], L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

}  // extern "C"

// ---- allocation-free sweep ---------------------------------------------------

extern "C" {

cc_status cc_smooth_noalloc(cc_handle H, int l, double* u, const double* b, cc_stream st) {
  t_last_error[0] = '\0';
  if (!H || H->opt.host_only || l < 0 || l + 1 >= (int)H->lv.size() || !u || !b) return CC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)st;
  try {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != H->device) {
      snprintf(t_last_error, sizeof(t_last_error),
               "cc_smooth_noalloc: current device %d is not the handle's device %d", dev, H->device);
      return CC_ERR_ARG;
    }
    Level& L = *H->lv[l];
    const BlockPlan& P = L.plan();
    const bool chunked = P.m > 0 && !P.dense;
    const int64_t need = L.nn + (chunked ? (int64_t)P.ns + P.m + P.nslots : 0);
    if (need > CC_NOALLOC_SCRATCH_DOUBLES) {
      snprintf(t_last_error, sizeof(t_last_error),
               "cc_smooth_noalloc: level %d needs %lld doubles of scratch, more than the %d "
               "available", l, (long long)need, CC_NOALLOC_SCRATCH_DOUBLES);
      return CC_ERR_ARG;
    }
    double* scr = H->noalloc;
    double* out = scr;                      // [0, nn): Jacobi output
    BlockDev B = L.blk.d64;                 // the handle's tables, temporaries in scratch
    B.fault = nullptr;                      // nothing of the handle is written
    if (chunked) {
      B.tS = scr + L.nn;                    // [nn, nn + ns): interface right-hand sides
      B.z = scr + L.nn + P.ns;              // [.., + m): chunk interior solutions
      B.q = scr + L.nn + P.ns + P.m;        // [.., + slots): interface contributions
    }
    if (H->opt.smoother == CC_SMOOTHER_MCGS) {
      // the multicolour variant works in place, on a copy of u
      CK(cudaMemcpyAsync(out, u, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      color_passes<double>(L, out, b, s);
    } else {
      launch_sweep<double>(L, u, out, b, (const double*)nullptr, false, s);
    }
    if (P.m) launch_block<double>(P, B, L.blk.sm64, out, b, s);
    // every non-empty cell of `out` was written above; empty cells go out as 0
    pdl_launch(k_rhs_copy, nblk(L.nn), 256, 0, s, out, L.cls, u, L.nn);
    CK(cudaGetLastError());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_level_tables(cc_handle H, int l, uint8_t* h_kind, int* h_lattice, double* h_beta,
                          int* n_plg) {
  if (!H || l < 0 || l >= (int)H->lv.size()) return CC_ERR_ARG;
  const LevelDisc& D = H->lv[l]->disc();
  if (h_kind) std::copy(D.kind.begin(), D.kind.end(), h_kind);
  for (size_t r = 0; r < D.plg.size(); ++r) {
    if (h_lattice) std::copy(D.lattice[r].begin(), D.lattice[r].end(), h_lattice + 15 * r);
    if (h_beta) std::copy(D.beta[r].begin(), D.beta[r].end(), h_beta + 16 * r);
  }
  if (n_plg) *n_plg = (int)D.plg.size();
  return CC_OK;
}

cc_status cc_kernel_timing(cc_handle H, int which) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H || which < CC_TIME_OFF || which > CC_TIME_FINE_BLOCK) return CC_ERR_ARG;
  H->timing = which;
  H->ev_used = 0;
  H->timed_launches = 0;
  H->timed_ms = 0;
  H->timed_bytes = 0;
  H->timed_rbytes = 0;
  try {
    // event pairs for every timed launch of one solve iteration, created up
    // front so that none is created during graph capture: a cycle visits
    // level l at most 2^l times (W; V and FMG fewer), each visit sweeps
    // nu1 + nu2 times
    const int nl = (int)H->lv.size();
    size_t per = (size_t)(H->opt.nu1 + H->opt.nu2) * ((size_t)1 << std::min(nl, 12)) * 2;
    if (which == CC_TIME_FINE_SWEEP || which == CC_TIME_FINE_BLOCK) per = (size_t)(H->opt.nu1 + H->opt.nu2);
    while (which != CC_TIME_OFF && H->ev.size() < per) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      H->ev.push_back({a, b});
    }
    H->ev_bytes.assign(H->ev.size(), 0.0);
    H->ev_rbytes.assign(H->ev.size(), 0.0);
  } catch (CudaError&) { return CC_ERR_CUDA; }
  return CC_OK;
}

cc_status cc_kernel_timing_read(cc_handle H, int64_t* launches, double* total_ms,
                                double* bytes_per_launch, double* moved_bytes_per_launch) {
  if (H && H->opt.host_only) return CC_ERR_ARG;
  if (!H) return CC_ERR_ARG;
  try {
    CK(cudaDeviceSynchronize());
  } catch (CudaError&) { return CC_ERR_CUDA; }
  if (launches) *launches = H->timed_launches;
  if (total_ms) *total_ms = H->timed_ms;
  if (bytes_per_launch)
    *bytes_per_launch = H->timed_launches ? H->timed_bytes / (double)H->timed_launches : 0.0;
  if (moved_bytes_per_launch)
    *moved_bytes_per_launch = H->timed_launches ? H->timed_rbytes / (double)H->timed_launches : 0.0;
  return CC_OK;
}

}  // extern "C"
